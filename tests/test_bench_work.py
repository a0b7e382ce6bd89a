"""The benchmark's algorithmic-work accounting of the block-Jacobi sweeps, on
CPU: `bench.sweep_work` reads a hierarchy's exported levels, so an oracle
hierarchy (same export layout as the GPU solver's) stands in for the GPU one.
The counts are checked against sums written out here from the level arrays,
and the shortened F-sweep row lists against full sweeps computed here."""
import numpy as np
import pytest

import bench
import dgtransport as D


@pytest.fixture(scope="module")
def hier(oracle_lib):
    P = D.make_problem("C2", N=12)
    return P, oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], neumann_degree=2, max_coarse=4)


def test_l0_width_is_face_node_count():
    """Level-0 coupling blocks of P1..P6 DG have p + 1 nonzero columns; blocks
    with more nonzero columns than the kernels provide are not compressed."""
    for name, p in (("C1", 1), ("C2", 2), ("C5", 3), ("C3", 6)):
        P = D.make_problem(name, N=6, p=p)
        rows = np.repeat(np.arange(P["E"]), np.diff(P["row_ptr"]))
        off = P["col"] != rows
        assert bench.l0_width(P["vals"][off], P["b"]) == p + 1
    full = np.ones((4, 6, 6))
    assert bench.l0_width(full, 6) == 0
    assert bench.l0_width(np.ones((3, 32, 32)), 32) == 0


def _level_arrays(lev):
    rows = np.repeat(np.arange(lev["E"]), np.diff(lev["row_ptr"]))
    return rows, lev["col"], lev["cf"], lev["col"] != rows


@pytest.mark.parametrize("split", [False, True])
def test_sweep_work_counts(hier, split):
    """With split, the F sweeps after the first on levels >= 1 count only their
    F-column couplings (x_C does not change while they run), and the first F
    sweep there also writes h = f - A_FC x_C."""
    P, H = hier
    b, SF = P["b"], 3
    work = bench.sweep_work(H, H.nlev, b, SF, 1, split=split)
    assert H.nlev >= 3
    for l in range(H.nlev):
        lev = H.level(l)
        if lev["coarsest"]:
            assert not any(key[0] == l for key in work)
            continue
        rows, ci, cf, off = _level_arrays(lev)
        masks = bench.f_sweep_rows(rows, ci, cf, off, SF)
        for k, upd in enumerate(masks + [cf == 1]):
            sel = upd[rows] & off
            if split and l >= 1 and 1 <= k < SF:
                sel = sel & (cf[ci] == 0)
            nrow = int(upd.sum())
            if (l, k) not in work:  # nothing to update or copy
                assert nrow == 0
                continue
            flops, byts = work[(l, k)]
            if l == 0:  # scaled, column-compressed couplings: b * W FMAs per block, no D^-1
                assert flops == 2.0 * int(sel.sum()) * b * (P["p"] + 1)
            else:       # classical form: exact off-diagonal nonzeros plus b^2 per row for D^-1
                nnz = int(np.count_nonzero(lev["vals"][sel].reshape(int(sel.sum()), -1)))
                assert flops == 2.0 * (nnz + nrow * b * b)
            assert byts >= 16.0 * nrow * b


def test_sweep_work_counts_scaled_f_sweeps(hier):
    """With ymode, the F sweeps on levels >= 1 apply no D^-1: the first sums
    the exact nonzeros of its couplings, the later ones b per nonzero row of
    the right-scaled F couplings A_ij D_jj^-1; the C sweep takes the scaled
    blocks for its F columns and converts every F row (b^2 FMAs each)."""
    P, H = hier
    b, SF = P["b"], 3
    work = bench.sweep_work(H, H.nlev, b, SF, 1, split=True, ymode=True)
    base = bench.sweep_work(H, H.nlev, b, SF, 1, split=True)
    for l in range(H.nlev):
        lev = H.level(l)
        if lev["coarsest"]:
            continue
        rows, ci, cf, off = _level_arrays(lev)
        masks = bench.f_sweep_rows(rows, ci, cf, off, SF)
        vals = lev["vals"]
        nzr = np.count_nonzero(np.any(vals != 0, axis=2), axis=1)
        nnzb = np.count_nonzero(vals.reshape(len(vals), -1), axis=1)
        for k, upd in enumerate(masks + [cf == 1]):
            if (l, k) not in work:
                continue
            if l == 0:
                assert work[(l, k)] == base[(l, k)]
                continue
            sel = upd[rows] & off
            if 1 <= k < SF:
                sel = sel & (cf[ci] == 0)
            fcol = sel & (cf[ci] == 0) if k >= 1 else np.zeros_like(sel)
            nnz = int(nnzb[sel & ~fcol].sum()) + b * int(nzr[fcol].sum())
            flops, byts = work[(l, k)]
            if k < SF:
                assert flops == 2.0 * nnz
            else:
                assert flops == 2.0 * (nnz + (int((cf == 1).sum()) + int((cf == 0).sum())) * b * b)
            assert byts >= 16.0 * int(upd.sum()) * b


def test_sweep_work_forms_select_the_accounting_per_level(hier):
    """forms (the library's per-level relaxation form) picks the accounting
    level by level: form 3 counts as split + ymode, form 2 as split only, and
    form 0 (block-row kernel) as neither."""
    P, H = hier
    b, SF = P["b"], 3
    n = H.nlev
    plain = bench.sweep_work(H, n, b, SF, 1)
    split = bench.sweep_work(H, n, b, SF, 1, split=True)
    yform = bench.sweep_work(H, n, b, SF, 1, split=True, ymode=True)
    forms = [1] + [3 if l % 3 == 1 else 2 if l % 3 == 2 else 0 for l in range(1, n)]
    mixed = bench.sweep_work(H, n, b, SF, 1, forms=forms)
    assert set(mixed) == set(plain)
    for (l, k), w in mixed.items():
        ref = plain if l == 0 or forms[l] == 0 else split if forms[l] == 2 else yform
        assert w == ref[(l, k)], (l, k)


def _transpose_level(lev, b):
    """Block transpose of a level matrix with its inverse diagonal blocks:
    (A^T)_ji = (A_ij)^T, rows sorted by column, (D_ii^{-1})^T."""
    E = lev["E"]
    rows = np.repeat(np.arange(E), np.diff(lev["row_ptr"]))
    order = np.lexsort((rows, lev["col"]))
    trows, tcols = lev["col"][order], rows[order]
    t = dict(lev)
    t["row_ptr"] = np.concatenate(([0], np.cumsum(np.bincount(trows, minlength=E)))).astype(np.int32)
    t["col"] = tcols.astype(np.int32)
    t["vals"] = np.ascontiguousarray(lev["vals"][order].transpose(0, 2, 1))
    t["dinv"] = np.ascontiguousarray(lev["dinv"].reshape(-1, b, b).transpose(0, 2, 1))
    return t


@pytest.mark.parametrize("transposed", [False, True])
def test_f_sweep_rows_cover_every_changing_row(hier, transposed):
    """Block-Jacobi F sweeps computed over all F rows: every F row outside the
    list of sweep k keeps its value of sweep k - 1 bit for bit, and the lists
    shrink (the premise of the shortened F sweeps), for A and for A^T (the
    transposed cycle's F sweeps, with A's C/F split)."""
    P, H = hier
    b, SF = P["b"], 4
    rng = np.random.default_rng(5)
    shrunk = 0
    for l in range(H.nlev):
        lev = H.level(l)
        if lev["coarsest"]:
            continue
        if transposed:
            lev = _transpose_level(lev, b)
        rows, ci, cf, off = _level_arrays(lev)
        masks = bench.f_sweep_rows(rows, ci, cf, off, SF)
        A = lev["vals"]
        dinv = lev["dinv"].reshape(-1, b, b)
        f = rng.standard_normal((lev["E"], b))
        x = rng.standard_normal((lev["E"], b))
        F = np.flatnonzero(cf == 0)
        for k in range(SF):
            prod = np.einsum("prc,pc->pr", A[off], x[ci[off]])
            acc = np.zeros_like(x)
            np.add.at(acc, rows[off], prod)
            new = x.copy()
            new[F] = np.einsum("irc,ic->ir", dinv[F], f[F] - acc[F])
            if k >= 1:
                keep = (cf == 0) & ~masks[k]
                assert np.array_equal(new[keep], x[keep]), (l, k)
                shrunk += int(keep.sum())
            x = new
    assert shrunk > 0


def test_hbm_peak_falls_back_without_measurement(monkeypatch, tmp_path):
    peak, src = bench.hbm_peak_gbs()
    assert peak > 1000.0 and src in ("measured", "fallback")
    monkeypatch.setattr(bench.os.path, "abspath", lambda p: str(tmp_path / "bench.py"))
    assert bench.hbm_peak_gbs() == (6800.0, "fallback")
