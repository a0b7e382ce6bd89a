"""The oracle pins catch plausible mistakes.

Each case plants one mistake in a copy of nair_oracle.c (a dropped term, a
wrong sign, a transposed operand, an off-by-one, a wrong comparison), builds
it, and runs the pins of tests/test_oracle_pins.py against it: at least one pin
must fail.  The shipped oracle is never modified.
"""
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "nair_oracle.c")

# (name, exact text in nair_oracle.c, planted replacement)
MUTATIONS = [
    ("inverse: pivot reciprocal dropped", "double rinv = 1.0 / d;", "double rinv = 1.0;"),
    ("C/F key: measure order reversed", "if (lam[i] != lam[j]) return lam[i] > lam[j];",
     "if (lam[i] != lam[j]) return lam[i] < lam[j];"),
    ("strength: threshold ignored", "L->snorm[p] > 0.0 && L->snorm[p] >= thr);", "L->snorm[p] > 0.0);"),
    ("Neumann: D^-1 term of the Horner step dropped",
     "memcpy(acc + (size_t)j * bb, init->v + (size_t)p * bb, sizeof(double) * bb);",
     "memset(acc + (size_t)j * bb, 0, sizeof(double) * bb);"),
    ("block product: right operand transposed",
     "for (int t = 0; t < b; ++t) s = fma(a[r * b + t], bv[t * b + cc], s);",
     "for (int t = 0; t < b; ++t) s = fma(a[r * b + t], bv[cc * b + t], s);"),
    ("restriction: sign of R_cf lost", "dst[e] = negate ? -src[e] : src[e];", "dst[e] = src[e];"),
    ("interpolation: weakest instead of strongest C neighbour",
     "if (best < 0 || L->snorm[p] > bs) { best = j; bs = L->snorm[p]; }",
     "if (best < 0 || L->snorm[p] < bs) { best = j; bs = L->snorm[p]; }"),
    ("A P merge: later blocks overwrite instead of add", "c[k] = c[k] + a[k];", "c[k] = a[k];"),
    ("L: sign of -D^-1 A lost", "o[r * b + c] = -s;", "o[r * b + c] = s;"),
    ("Jacobi: off-diagonal coupling added", "for (int c = 0; c < b; ++c) s -= a[c] * xj[c];",
     "for (int c = 0; c < b; ++c) s += a[c] * xj[c];"),
    ("Jacobi: old iterate kept", "x[(size_t)i * b + r] = s;", "x[(size_t)i * b + r] += s;"),
    ("F-relaxation: one sweep short",
     "for (int s = 0; s < H->f_sweeps; ++s) jacobi(b, L, 0, f, x, tmp);",
     "for (int s = 1; s < H->f_sweeps; ++s) jacobi(b, L, 0, f, x, tmp);"),
    ("transposed cycle: F sweeps before C sweeps",
     "  for (int s = 0; s < H->c_sweeps; ++s) jacobi_t(b, L, 1, f, x, tmp);\n"
     "  for (int s = 0; s < H->f_sweeps; ++s) jacobi_t(b, L, 0, f, x, tmp);",
     "  for (int s = 0; s < H->f_sweeps; ++s) jacobi_t(b, L, 0, f, x, tmp);\n"
     "  for (int s = 0; s < H->c_sweeps; ++s) jacobi_t(b, L, 1, f, x, tmp);"),
    ("transposed Jacobi: D^-1 not transposed", "s += d[c * b + r] * res[c];", "s += d[r * b + c] * res[c];"),
    ("transposed interpolation: R_cf block not transposed", "xf[r] += rv[t * b + r] * xcc[t];",
     "xf[r] += rv[r * b + t] * xcc[t];"),
    ("P^T restriction: F residuals dropped", "    if (J < 0) continue;\n    for (int r = 0; r < b; ++r) rc",
     "    if (J < 0 || !L->cf[i]) continue;\n    for (int r = 0; r < b; ++r) rc"),
    ("transposed coarse solve: K^-1 instead of K^-T", "dense_lu_solve_t(L->n, L->lu, L->piv, x);",
     "dense_lu_solve(L->n, L->lu, L->piv, x);"),
    ("F-cycle: V-cycle correction skipped", "if (type == 1) cycle(H, l + 1, 0, fc, xc, 0);", ";"),
    ("F-cycle: V-cycle correction from zero", "if (type == 1) cycle(H, l + 1, 0, fc, xc, 0);",
     "if (type == 1) cycle(H, l + 1, 0, fc, xc, 1);"),
    ("F-cycle: V-cycles below the first coarse level", "cycle(H, l + 1, type, fc, xc, 1);",
     "cycle(H, l + 1, 0, fc, xc, 1);"),
    ("nonzero guess: residual not formed", "for (size_t k = 0; k < n; ++k) r[k] = f[k] - r[k];",
     "for (size_t k = 0; k < n; ++k) r[k] = f[k];"),
    ("nonzero guess: interpolation replaces x",
     "x[(size_t)i * b + rr] = zero ? v : x[(size_t)i * b + rr] + v;", "x[(size_t)i * b + rr] = v;"),
    ("scalar: blocks not scaled by D^-1", "for (int t = 0; t < b; ++t) acc = fma(Di[r * b + t], a[t * b + c], acc);",
     "acc = a[r * b + c];"),
    ("scalar: explicit zeros stored", "if (blk[c] != 0.0) {", "if (1) {"),
    ("scalar: D^-1 not applied before the cycle", "block_diag_apply(E, H->bo, H->Do, v, t, 0);",
     "memcpy(t, v, sizeof(double) * n);"),
    ("filter: strict < instead of inclusive <=", "!(block_norm2(b, M->v + (size_t)p * bb) <= thr)",
     "!(block_norm2(b, M->v + (size_t)p * bb) < thr)"),
    ("filter: threshold from the row's largest block",
     "if (M->ci[p] == i) dn = block_norm2(b, M->v + (size_t)p * bb);",
     "dn = fmax(dn, block_norm2(b, M->v + (size_t)p * bb));"),
    ("filter: diagonal block not exempt", "int keep = (M->ci[p] == i) || !(", "int keep = !("),
    # R_cf has no diagonal block, so a filter of R_cf takes its row's largest block as the scale
    ("filter: R_cf filtered as well", "spgemm(b, nC, nF, &Acf, NULL, &L->Delta, NULL, NULL, 1, &L->Rcf);",
     "spgemm(b, nC, nF, &Acf, NULL, &L->Delta, NULL, NULL, 1, &L->Rcf);\n"
     "    for (int c = 0; c < nC; ++c) {\n"
     "      double mx = 0.0;\n"
     "      for (int p = L->Rcf.rp[c]; p < L->Rcf.rp[c + 1]; ++p) mx = fmax(mx, block_norm2(b, L->Rcf.v + (size_t)p * bb));\n"
     "      for (int p = L->Rcf.rp[c]; p < L->Rcf.rp[c + 1]; ++p)\n"
     "        if (block_norm2(b, L->Rcf.v + (size_t)p * bb) <= tol2 * mx) memset(L->Rcf.v + (size_t)p * bb, 0, sizeof(double) * bb);\n"
     "    }"),
    ("filter: only the last Neumann iterate filtered", "if (targets & 1) filter_bsr(b, &Tn, tol2);",
     "if ((targets & 1) && t == k - 1) filter_bsr(b, &Tn, tol2);"),
    ("filter: coarse operator left unfiltered", "if (targets & 2) filter_bsr(b, &Nx->A, tol2);", ";"),
    ("scalar adjoint: D^-1 not transposed", "block_diag_apply(E, H->bo, H->Do, t, z, 1);",
     "block_diag_apply(E, H->bo, H->Do, t, z, 0);"),
]

PINS = [
    lambda o: pins.test_block_inverse_matches_dense_inverse(o, 6),
    lambda o: pins.test_cf_star_by_hand(o),
    lambda o: pins.test_cf_measure_priority_by_hand(o),
    lambda o: pins.test_strength_rule_by_hand(o),
    lambda o: pins.test_cf_invariants(o, "C2", 8, 2),
    lambda o: pins.test_neumann_error_identity(o, "C3", 2, 1),
    lambda o: pins.test_exact_neumann_gives_ideal_restriction_and_schur(o, 1),
    lambda o: pins.test_galerkin_product_and_wap_identity(o, "C2", 2, 2),
    lambda o: pins.test_chain_closed_form(o),
    lambda o: pins.test_exact_settings_one_vcycle_solves(o, 1),
    lambda o: pins.test_minimal_f_sweeps_two_level(o),
    lambda o: pins.test_error_propagation_is_strictly_block_lower_triangular(o),
    lambda o: pins.test_fgmres_matches_dense_solve(o, "C2", 8, 2),
    lambda o: pins.test_transposed_cycle_is_adjoint_of_vcycle(o, "C2", 4, 2, 2, 2, 1),
    lambda o: pins.test_transposed_cycle_exact_under_ideal_interpolation(o, 1),
    lambda o: pins.test_cycles_match_composed_error_propagation(o, "V", "C2", 4, 2, 2, 3, 1),
    lambda o: pins.test_cycles_match_composed_error_propagation(o, "F", "C2", 4, 2, 2, 3, 1),
    lambda o: pins.test_scalar_scaled_matrix(o, "C2", 4, 2),
    lambda o: pins.test_scalar_exact_under_ideal_settings(o, 1),
    lambda o: pins.test_scalar_preconditioner_composition(o, "C2", 4, 2, 2),
    lambda o: pins.test_filter_rule_boundary_by_hand(o),
    lambda o: pins.test_filter_threshold_is_the_diagonal_block(o),
    lambda o: pins.test_filter_keeps_diagonal_block(o),
    lambda o: pins.test_filter_targets_in_the_hierarchy(o, 3),
    lambda o: pins.test_filter_targets_in_the_hierarchy(o, 1),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new):
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation target not unique: {old}"
    src = tmp_path / "mutant.c"
    src.write_text(text.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(lib), str(src), "-lm"])
    caught = []
    with oracle.use_library(str(lib)):
        for pin in PINS:
            try:
                pin(oracle)
            except Exception as e:  # a failed assertion or an oracle error status
                caught.append(type(e).__name__)
    assert caught, f"no pin caught the planted mistake: {name}"
