"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: dense
inverses and Schur complements (numpy), closed forms, exact-solver special
cases and the invariants the paper states.  No test here needs a GPU.
"""
import numpy as np
import pytest

import dgtransport as D
from conftest import bsr_dense


def tiny(name="C1", N=4, p=1, **kw):
    return D.make_problem(name, N=N, p=p, **kw)


def dof_sets(cf, b):
    F = np.nonzero(cf == 0)[0]
    C = np.nonzero(cf == 1)[0]
    fd = (F[:, None] * b + np.arange(b)[None, :]).ravel()
    cd = (C[:, None] * b + np.arange(b)[None, :]).ravel()
    return F, C, fd, cd


def block_forward_substitution(P):
    """x* for a block lower-triangular system (Sec. 2.1: forward solve)."""
    b = P["b"]
    E = P["E"]
    x = np.zeros(P["n"])
    rhs = P["rhs"]
    for i in range(E):
        s = rhs[i * b:(i + 1) * b].copy()
        dblk = None
        for k in range(P["row_ptr"][i], P["row_ptr"][i + 1]):
            j = P["col"][k]
            if j < i:
                s -= P["vals"][k] @ x[j * b:(j + 1) * b]
            elif j == i:
                dblk = P["vals"][k]
            else:
                raise AssertionError("not block lower triangular")
        x[i * b:(i + 1) * b] = np.linalg.solve(dblk, s)
    return x


def chain(n, c=0.5):
    """1D upwind chain, b = 1: x_i - c x_{i-1} = f_i."""
    rp = [0]
    col = []
    vals = []
    for i in range(n):
        if i > 0:
            col.append(i - 1)
            vals.append(-c)
        col.append(i)
        vals.append(1.0)
        rp.append(len(col))
    return (np.array(rp, dtype=np.int32), np.array(col, dtype=np.int32),
            np.array(vals, dtype=np.float64).reshape(-1, 1, 1))


# -----------------------------------------------------------------------------
# generator
# -----------------------------------------------------------------------------

@pytest.mark.parametrize("p", [1, 2, 3, 6])
def test_generator_reproduces_constant_solution(p):
    """u = 1 with sigma = q = 1 and inflow g = 1 lies in P_p: DG is exact."""
    P = tiny("C3", N=5, p=p, g=1.0)
    A = bsr_dense(P["row_ptr"], P["col"], P["vals"])
    u = np.linalg.solve(A, P["rhs"])
    assert np.max(np.abs(u - 1.0)) < 1e-10


def test_generator_structure():
    P = D.make_problem("C1")
    b, p = P["b"], P["p"]
    faces = 3 * 32 * 32 - 2 * 32
    # one upwind coupling per interior face, (p+1)^2 nonzeros each
    assert P["nnzb"] == P["E"] + faces
    assert np.count_nonzero(P["vals"]) == P["E"] * b * b + faces * (p + 1) ** 2
    rows = np.repeat(np.arange(P["E"]), np.diff(P["row_ptr"]))
    assert np.all(P["col"] <= rows)          # block lower triangular (topological order)
    assert abs(P["mass"].sum() - 1.0) < 1e-12  # sum of element areas


# -----------------------------------------------------------------------------
# a1: block inverse
# -----------------------------------------------------------------------------

@pytest.mark.parametrize("b", [1, 3, 6, 10, 28])
def test_block_inverse_matches_dense_inverse(oracle_lib, b):
    r = np.random.default_rng(b)
    for trial in range(5):
        A = r.standard_normal((b, b))
        if trial == 0:
            A = A + 3 * b * np.eye(b)
        X = oracle_lib.block_inverse(A)
        assert np.linalg.norm(X @ A - np.eye(b)) <= 1e-11 * np.linalg.cond(A)
        assert np.allclose(X, np.linalg.inv(A), rtol=1e-9, atol=1e-12 * np.abs(X).max())


def test_block_inverse_singular(oracle_lib):
    A = np.ones((3, 3))
    with pytest.raises(oracle_lib.OracleError):
        oracle_lib.block_inverse(A)


# -----------------------------------------------------------------------------
# a2 / a3: strength and C/F splitting
# -----------------------------------------------------------------------------

def test_cf_star_by_hand(oracle_lib):
    """Points 1..4 depend only on point 0: lambda_0 = 4, others 0 -> C F F F F."""
    n = 5
    rp = [0, 1]
    col = [0]
    vals = [2.0]
    for i in range(1, n):
        col += [0, i]
        vals += [-1.0, 2.0]
        rp.append(len(col))
    H = oracle_lib.Hierarchy(np.array(rp), np.array(col), np.array(vals).reshape(-1, 1, 1),
                             max_coarse=1, max_levels=2, filter_targets=0)
    lev = H.level(0)
    assert lev["cf"].tolist() == [1, 0, 0, 0, 0]
    assert lev["lam"].tolist() == [4, 0, 0, 0, 0]
    assert lev["ipc"].tolist() == [0, 0, 0, 0, 0]


def test_cf_measure_priority_by_hand(oracle_lib):
    """Classical measure (Sec. 5.1): of two competing undecided points the one more
    points depend on becomes C.  Point 1 depends on 0; point 2 on 0 and 1:
    lambda = (2, 1, 0) -> 2 is F at once, 0 beats 1 and becomes C, 1 becomes F."""
    rp = np.array([0, 1, 3, 6], dtype=np.int32)
    col = np.array([0, 0, 1, 0, 1, 2], dtype=np.int32)
    vals = np.array([2.0, -1.0, 2.0, -1.0, -1.0, 2.0]).reshape(-1, 1, 1)
    H = oracle_lib.Hierarchy(rp, col, vals, max_coarse=1, max_levels=2, filter_targets=0)
    lev = H.level(0)
    assert lev["lam"].tolist() == [2, 1, 0]
    assert lev["cf"].tolist() == [1, 0, 0]


def test_strength_rule_by_hand(oracle_lib):
    """Row 2 of a 3-point system: |a_20| = 1, |a_21| = 0.05; theta = 0.1 keeps only 0."""
    rp = np.array([0, 1, 3, 6], dtype=np.int32)
    col = np.array([0, 0, 1, 0, 1, 2], dtype=np.int32)
    vals = np.array([1.0, -0.5, 1.0, -1.0, -0.05, 1.0]).reshape(-1, 1, 1)
    H = oracle_lib.Hierarchy(rp, col, vals, theta=0.1, max_coarse=1, max_levels=2)
    s = H.level(0)["strong"].tolist()
    assert s == [0, 1, 0, 1, 0, 0]
    # theta = 0.3: |a_21|^2 = 0.0025 < 0.09 -> still weak; theta = 0.01 -> strong
    H2 = oracle_lib.Hierarchy(rp, col, vals, theta=0.01, max_coarse=1, max_levels=2)
    assert H2.level(0)["strong"].tolist() == [0, 1, 0, 1, 1, 0]


@pytest.mark.parametrize("name,N,p", [("C1", 8, 1), ("C2", 8, 2), ("C3", 6, 3)])
def test_cf_invariants(oracle_lib, name, N, p):
    P = tiny(name, N=N, p=p)
    H = oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], max_coarse=4)
    for l in range(H.nlev - 1):
        lev = H.level(l)
        cf, strong, rp, col = lev["cf"], lev["strong"].astype(bool), lev["row_ptr"], lev["col"]
        E = lev["E"]
        assert set(np.unique(cf)) <= {0, 1}
        lam = np.zeros(E, dtype=np.int64)
        for i in range(E):
            for k in range(rp[i], rp[i + 1]):
                if strong[k]:
                    lam[col[k]] += 1
        assert np.array_equal(lam, lev["lam"])
        for i in range(E):
            if cf[i] == 0:
                has_c = any(strong[k] and cf[col[k]] == 1 for k in range(rp[i], rp[i + 1]))
                assert has_c or lam[i] == 0
        # one-point interpolation: strongest strong C neighbour, smallest index on ties
        cidx = np.cumsum(cf) - 1
        for i in range(E):
            if cf[i] == 1:
                assert lev["ipc"][i] == cidx[i]
                continue
            cands = [(k, col[k]) for k in range(rp[i], rp[i + 1]) if strong[k] and cf[col[k]] == 1]
            if not cands:
                assert lev["ipc"][i] == -1
                continue
            nrm = [np.sum(lev["vals"][k] ** 2) for k, _ in cands]
            best = max(nrm)
            # norms equal up to summation rounding: accept any near-maximal candidate
            ok = [cidx[j] for (k, j), s in zip(cands, nrm) if s >= best * (1 - 1e-12)]
            assert lev["ipc"][i] in ok


# -----------------------------------------------------------------------------
# a4 / a5 / a7: Neumann series, ideal restriction, Schur complement
# -----------------------------------------------------------------------------

def two_level(oracle_lib, P, **kw):
    par = dict(max_levels=2, max_coarse=1, max_dense=100000)
    par.update(kw)
    return oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], **par)


def dense_L(A, cf, strong, rp, col, b):
    """L = I - D_ff^{-1} A_ff^S over strong F-F blocks, built directly (numpy)."""
    F = np.nonzero(cf == 0)[0]
    fpos = {int(e): k for k, e in enumerate(F)}
    nF = len(F)
    Lm = np.zeros((nF * b, nF * b))
    for a, i in enumerate(F):
        Dii = A[i * b:(i + 1) * b, i * b:(i + 1) * b]
        Di = np.linalg.inv(Dii)
        for k in range(rp[i], rp[i + 1]):
            j = col[k]
            if j != i and strong[k] and cf[j] == 0:
                c = fpos[int(j)]
                Lm[a * b:(a + 1) * b, c * b:(c + 1) * b] = -Di @ A[i * b:(i + 1) * b, j * b:(j + 1) * b]
    return Lm


@pytest.mark.parametrize("k", [0, 1, 2, 3])
@pytest.mark.parametrize("name,p", [("C1", 1), ("C3", 2), ("C2", 2)])
def test_neumann_error_identity(oracle_lib, name, p, k):
    """I - Delta A^S_ff = L^{k+1} for any degree k (Sec. 4.1), unfiltered."""
    P = tiny(name, N=4, p=p)
    H = two_level(oracle_lib, P, neumann_degree=k, filter_targets=0, theta=0.1)
    lev = H.level(0)
    b = P["b"]
    A = bsr_dense(P["row_ptr"], P["col"], P["vals"])
    Lm = dense_L(A, lev["cf"], lev["strong"], lev["row_ptr"], lev["col"], b)
    nF = lev["nF"]
    Dg = np.zeros_like(Lm)
    F = np.nonzero(lev["cf"] == 0)[0]
    for a, i in enumerate(F):
        Dg[a * b:(a + 1) * b, a * b:(a + 1) * b] = A[i * b:(i + 1) * b, i * b:(i + 1) * b]
    AS = Dg @ (np.eye(nF * b) - Lm)   # A_ff restricted to strong blocks
    Delta = bsr_dense(lev["D_rp"], lev["D_ci"], lev["D_v"], nF, nF)
    lhs = np.eye(nF * b) - Delta @ AS
    rhs = np.linalg.matrix_power(Lm, k + 1)
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * max(1.0, np.max(np.abs(rhs)))
    Ld = bsr_dense(lev["L_rp"], lev["L_ci"], lev["L_v"], nF, nF)
    assert np.max(np.abs(Ld - Lm)) <= 1e-13 * max(1.0, np.abs(Lm).max())


def longest_ff_path(lev):
    """d_f: longest path in the F-F graph of L (footnote to Eq. neumann)."""
    nF = lev["nF"]
    depth = np.zeros(nF, dtype=np.int64)
    for i in range(nF):
        for k in range(lev["L_rp"][i], lev["L_rp"][i + 1]):
            j = lev["L_ci"][k]
            assert j < i   # lower triangular in the F order
            depth[i] = max(depth[i], depth[j] + 1)
    return int(depth.max()) if nF else 0


@pytest.mark.parametrize("p", [1, 2])
def test_exact_neumann_gives_ideal_restriction_and_schur(oracle_lib, p):
    """theta = 0, no filtering, k >= d_f on triangular A: Delta = A_ff^{-1},
    R = R_ideal and K = R A P = K_A (Eq. neumann, Lemma ideal restriction)."""
    P = tiny("C1", N=4, p=p)
    b = P["b"]
    H = two_level(oracle_lib, P, neumann_degree=40, filter_targets=0, theta=0.0)
    lev = H.level(0)
    assert longest_ff_path(lev) <= 40
    A = bsr_dense(P["row_ptr"], P["col"], P["vals"])
    F, C, fd, cd = dof_sets(lev["cf"], b)
    Aff, Afc, Acf, Acc = A[np.ix_(fd, fd)], A[np.ix_(fd, cd)], A[np.ix_(cd, fd)], A[np.ix_(cd, cd)]
    Affi = np.linalg.inv(Aff)
    Delta = bsr_dense(lev["D_rp"], lev["D_ci"], lev["D_v"], len(F), len(F))
    assert np.max(np.abs(Delta - Affi)) <= 1e-12 * np.abs(Affi).max()
    Rcf = bsr_dense(lev["R_rp"], lev["R_ci"], lev["R_v"], len(C), len(F))
    Rid = -Acf @ Affi
    assert np.max(np.abs(Rcf - Rid)) <= 1e-12 * max(1.0, np.abs(Rid).max())
    KA = Acc - Acf @ Affi @ Afc
    K = bsr_dense(H.level(1)["row_ptr"], H.level(1)["col"], H.level(1)["vals"], len(C), len(C))
    assert np.max(np.abs(K - KA)) <= 1e-12 * np.abs(KA).max()


@pytest.mark.parametrize("name,p,k", [("C1", 1, 1), ("C2", 2, 2), ("C3", 3, 1)])
def test_galerkin_product_and_wap_identity(oracle_lib, name, p, k):
    """K equals R A P formed densely from the oracle's R and P (Eq. rap), and
    K - K_A = delta_R A_ff^{-1} delta_P (Sec. 3.3)."""
    P = tiny(name, N=4, p=p)
    b = P["b"]
    H = two_level(oracle_lib, P, neumann_degree=k, filter_targets=0, theta=0.1)
    lev = H.level(0)
    A = bsr_dense(P["row_ptr"], P["col"], P["vals"])
    F, C, fd, cd = dof_sets(lev["cf"], b)
    nC, nF = len(C), len(F)
    Rcf = bsr_dense(lev["R_rp"], lev["R_ci"], lev["R_v"], nC, nF)
    W = np.zeros((nF * b, nC * b))
    for a, i in enumerate(F):
        J = lev["ipc"][i]
        if J >= 0:
            W[a * b:(a + 1) * b, J * b:(J + 1) * b] = np.eye(b)
    Aff, Afc, Acf, Acc = A[np.ix_(fd, fd)], A[np.ix_(fd, cd)], A[np.ix_(cd, fd)], A[np.ix_(cd, cd)]
    K_dense = Rcf @ Aff @ W + Acf @ W + Rcf @ Afc + Acc
    K = bsr_dense(H.level(1)["row_ptr"], H.level(1)["col"], H.level(1)["vals"], nC, nC)
    scale = np.abs(K_dense).max()
    assert np.max(np.abs(K - K_dense)) <= 1e-12 * scale
    KA = Acc - Acf @ np.linalg.inv(Aff) @ Afc
    dR = Rcf @ Aff + Acf
    dP = Aff @ W + Afc
    assert np.max(np.abs((K_dense - KA) - dR @ np.linalg.inv(Aff) @ dP)) <= 1e-10 * scale


# -----------------------------------------------------------------------------
# a8: filtering (Sec. 5.2, block form: drop X_ij when ||X_ij||_F^2 <= tol^2 ||X_ii||_F^2)
# -----------------------------------------------------------------------------

def bsr_rows(rows):
    """Block-CSR arrays from a list of block rows [[(col, block), ...], ...]."""
    rp, col, vals = [0], [], []
    for r in rows:
        for j, blk in r:
            col.append(j)
            vals.append(np.asarray(blk, dtype=np.float64))
        rp.append(len(col))
    return np.array(rp, dtype=np.int32), np.array(col, dtype=np.int32), np.array(vals)


def test_filter_rule_boundary_by_hand(oracle_lib):
    """tol = 0.5 (tol^2 = 0.25 exactly) and identity diagonal blocks
    (||X_ii||^2 = 2) put the threshold at exactly 0.5.  Row 0's coupling
    [[.5, .5], [0, 0]] has ||X||^2 = 0.5, on the threshold: dropped, the rule is
    inclusive.  Row 1's [[.5, .5 + 2^-53], [0, 0]] has ||X||^2 = 0.5 + 2^-53
    (the rounded sum), one ulp above: kept.  Kept blocks are copied bit for bit."""
    I2 = np.eye(2)
    up = np.nextafter(0.5, 1.0)
    assert up == 0.5 + 2.0 ** -53
    X0 = np.array([[0.5, 0.5], [0.0, 0.0]])
    X1 = np.array([[0.5, up], [0.0, 0.0]])
    rp, col, vals = bsr_rows([[(0, I2), (1, X0)], [(0, X1), (1, I2)]])
    rp2, ci2, v2 = oracle_lib.filter_blocks(rp, col, vals, 0.5)
    assert rp2.tolist() == [0, 1, 3]
    assert ci2.tolist() == [0, 0, 1]
    assert np.array_equal(v2, np.array([I2, X1, I2]))


def test_filter_threshold_is_the_diagonal_block(oracle_lib):
    """The threshold scales with the row's own diagonal block, not with the
    row's largest block.  tol = 0.6 (tol^2 = 0.36), b = 1:
      row 0: diagonal 1, couplings 100, 2, 0.5 -> threshold 0.36: keeps 100 and 2
             (4 > 0.36), drops 0.5 (0.25 <= 0.36); a threshold from the largest
             block (0.36 * 1e4) would drop 2 as well;
      row 1: diagonal 10, coupling 5 -> threshold 36: drops 5 (25 <= 36); a
             threshold from the largest off-diagonal block (0.36 * 25) would keep it."""
    rp, col, vals = bsr_rows([
        [(0, [[1.0]]), (1, [[100.0]]), (2, [[2.0]]), (3, [[0.5]])],
        [(0, [[5.0]]), (1, [[10.0]])],
        [(2, [[1.0]])],
        [(3, [[1.0]])],
    ])
    rp2, ci2, v2 = oracle_lib.filter_blocks(rp, col, vals, 0.6)
    assert rp2.tolist() == [0, 3, 4, 5, 6]
    assert ci2.tolist() == [0, 1, 2, 1, 2, 3]
    assert v2.ravel().tolist() == [1.0, 100.0, 2.0, 10.0, 1.0, 1.0]


def test_filter_keeps_diagonal_block(oracle_lib):
    """The diagonal block is never dropped, however small.  tol = 2 (tol^2 = 4):
      row 0: diagonal 1e-3 I (||.||^2 = 2e-6, below its own threshold 8e-6),
             couplings 1e-3 I (dropped: 2e-6 <= 8e-6) and I (kept);
      row 1: a zero diagonal block (threshold 0) and a zero coupling (dropped:
             0 <= 0); the diagonal stays;
      row 2: the diagonal alone."""
    I2 = np.eye(2)
    Z2 = np.zeros((2, 2))
    rp, col, vals = bsr_rows([
        [(0, 1e-3 * I2), (1, 1e-3 * I2), (2, I2)],
        [(0, Z2), (1, Z2)],
        [(2, I2)],
    ])
    rp2, ci2, v2 = oracle_lib.filter_blocks(rp, col, vals, 2.0)
    assert rp2.tolist() == [0, 2, 3, 4]
    assert ci2.tolist() == [0, 2, 1, 2]
    assert np.array_equal(v2, np.array([1e-3 * I2, I2, Z2, I2]))


def block_norms2(M, b):
    """Squared Frobenius norm of every b x b block of a dense matrix."""
    nr, nc = M.shape[0] // b, M.shape[1] // b
    return (M.reshape(nr, b, nc, b) ** 2).sum(axis=(1, 3))


def filter_dense(M, pattern, b, tol):
    """The filtering rule on a dense square block matrix with its block pattern:
    returns the kept pattern and the matrix with the dropped blocks zeroed.
    Also returns the smallest relative distance of a stored off-diagonal
    block's squared norm to its threshold (the margin of the decisions)."""
    nrm = block_norms2(M, b)
    n = nrm.shape[0]
    thr = tol * tol * np.diag(nrm)[:, None]
    off = pattern & ~np.eye(n, dtype=bool)
    drop = off & (nrm <= thr)
    with np.errstate(divide="ignore", invalid="ignore"):
        rel = np.abs(nrm - thr) / np.where(thr > 0, thr, 1.0)
    margin = float(rel[off].min()) if off.any() else np.inf
    keep = pattern & ~drop
    mask = np.kron(keep, np.ones((b, b), dtype=bool))
    return keep, np.where(mask, M, 0.0), margin


def block_pattern(rp, col, nr, nc):
    S = np.zeros((nr, nc), dtype=bool)
    for i in range(nr):
        S[i, col[rp[i]:rp[i + 1]]] = True
    return S


@pytest.mark.parametrize("targets", [0, 1, 2, 3])
def test_filter_targets_in_the_hierarchy(oracle_lib, targets):
    """Which matrices are filtered (Sec. 5.2, block form; the filter_targets
    bits): each Neumann iterate T_{t+1} = D^{-1} + L T_t when bit 0 is set, the
    coarse operator A_{l+1} when bit 1 is set, and R_cf = -A_cf Delta never.
    Delta, R_cf and K are rebuilt here in numpy from A, the splitting, the
    strength flags and P: block patterns by boolean products of the structure,
    values by dense products, the rule applied to each filtered matrix.  tol =
    0.5 makes the filter drop blocks of both Delta and K on this problem, and
    every decision lies at least 1e-6 (relative) away from its threshold."""
    tol = 0.5
    k = 2
    P = tiny("C2", N=6, p=2)
    b = P["b"]
    H = two_level(oracle_lib, P, neumann_degree=k, filter_targets=targets, filter_tol=tol, theta=0.1)
    lev = H.level(0)
    A = bsr_dense(P["row_ptr"], P["col"], P["vals"])
    cf, strong, rp, col = lev["cf"], lev["strong"].astype(bool), lev["row_ptr"], lev["col"]
    F, C, fd, cd = dof_sets(cf, b)
    nF, nC = len(F), len(C)
    SA = block_pattern(rp, col, lev["E"], lev["E"])
    # Horner with the rule applied to every iterate when bit 0 is set
    Lm = dense_L(A, cf, strong, rp, col, b)
    SL = np.abs(block_norms2(Lm, b)) > 0
    SL |= block_pattern(lev["L_rp"], lev["L_ci"], nF, nF)  # structural zero blocks as well
    Dg = np.zeros((nF * b, nF * b))
    for a, i in enumerate(F):
        Dg[a * b:(a + 1) * b, a * b:(a + 1) * b] = np.linalg.inv(A[i * b:(i + 1) * b, i * b:(i + 1) * b])
    eyeF = np.eye(nF, dtype=bool)
    T, ST = Dg.copy(), eyeF.copy()
    dropped_delta = 0
    for _ in range(k):
        T = Dg + Lm @ T
        ST = eyeF | ((SL.astype(int) @ ST.astype(int)) > 0)
        if targets & 1:
            keep, T, margin = filter_dense(T, ST, b, tol)
            assert margin > 1e-6
            dropped_delta += int(ST.sum() - keep.sum())
            ST = keep
    SD = block_pattern(lev["D_rp"], lev["D_ci"], nF, nF)
    assert np.array_equal(SD, ST)
    Delta = bsr_dense(lev["D_rp"], lev["D_ci"], lev["D_v"], nF, nF)
    assert np.max(np.abs(Delta - T)) <= 1e-12 * np.abs(T).max()
    assert (dropped_delta > 0) == bool(targets & 1)
    # R_cf = -A_cf Delta over all its structural blocks: never filtered
    SAcf = SA[np.ix_(C, F)]
    SR = (SAcf.astype(int) @ SD.astype(int)) > 0
    assert np.array_equal(block_pattern(lev["R_rp"], lev["R_ci"], nC, nF), SR)
    Acf = A[np.ix_(cd, fd)]
    Rn = -Acf @ Delta
    Rcf = bsr_dense(lev["R_rp"], lev["R_ci"], lev["R_v"], nC, nF)
    assert np.max(np.abs(Rcf - Rn)) <= 1e-12 * np.abs(Rn).max()
    # K = (AP)_C + R_cf (AP)_F, filtered when bit 1 is set
    W = np.zeros((lev["E"] * b, nC * b))
    SP = np.zeros((lev["E"], nC), dtype=bool)
    for i in range(lev["E"]):
        J = lev["ipc"][i]
        if J >= 0:
            W[i * b:(i + 1) * b, J * b:(J + 1) * b] = np.eye(b)
            SP[i, J] = True
    AP = A @ W
    SAP = (SA.astype(int) @ SP.astype(int)) > 0
    Kd = AP[cd] + Rcf @ AP[fd]
    SK = SAP[C] | ((SR.astype(int) @ SAP[F].astype(int)) > 0)
    nK = int(SK.sum())
    if targets & 2:
        SK, Kd, margin = filter_dense(Kd, SK, b, tol)
        assert margin > 1e-6
    assert (int(SK.sum()) < nK) == bool(targets & 2)
    L1 = H.level(1)
    assert np.array_equal(block_pattern(L1["row_ptr"], L1["col"], nC, nC), SK)
    K = bsr_dense(L1["row_ptr"], L1["col"], L1["vals"], nC, nC)
    assert np.max(np.abs(K - Kd)) <= 1e-12 * np.abs(Kd).max()


def test_chain_closed_form(oracle_lib):
    """1D upwind chain: R_ideal and the Schur complement have closed forms
    R_{c,f} = c^{c-f} and K_{c,c'} = -c^{c-c'} (c' the previous C point)."""
    n = 40
    cval = 0.5
    rp, col, vals = chain(n, cval)
    H = oracle_lib.Hierarchy(rp, col, vals, theta=0.0, filter_targets=0, neumann_degree=n,
                             max_levels=2, max_coarse=1)
    lev = H.level(0)
    cf = lev["cf"]
    C = np.nonzero(cf == 1)[0]
    F = np.nonzero(cf == 0)[0]
    fpos = {int(f): a for a, f in enumerate(F)}
    K = bsr_dense(H.level(1)["row_ptr"], H.level(1)["col"], H.level(1)["vals"], len(C), len(C))
    R = bsr_dense(lev["R_rp"], lev["R_ci"], lev["R_v"], len(C), len(F))
    for a, c in enumerate(C):
        assert K[a, a] == 1.0
        prev = C[C < c]
        for a2 in range(len(C)):
            if a2 != a:
                want = -(cval ** (c - prev[-1])) if (len(prev) and C[a2] == prev[-1]) else 0.0
                assert abs(K[a, a2] - want) <= 1e-15
        lo = prev[-1] if len(prev) else -1
        for f in F:
            want = cval ** (c - f) if lo < f < c else 0.0
            assert abs(R[a, fpos[int(f)]] - want) <= 1e-15


# -----------------------------------------------------------------------------
# a9 - a14: cycle
# -----------------------------------------------------------------------------

@pytest.mark.parametrize("p", [1, 2])
def test_exact_settings_one_vcycle_solves(oracle_lib, p):
    """R_ideal at every level plus enough F-Jacobi sweeps to be exact on the
    nilpotent F block: one V-cycle from zero solves A x = f (Lemma ideal
    restriction, applied recursively)."""
    P = tiny("C1", N=6, p=p)
    H = oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], theta=0.0, filter_targets=0,
                             neumann_degree=80, max_coarse=2, f_sweeps=80, c_sweeps=1)
    assert H.nlev >= 3
    A = bsr_dense(P["row_ptr"], P["col"], P["vals"])
    x = H.vcycle(P["rhs"])
    xs = np.linalg.solve(A, P["rhs"])
    assert np.linalg.norm(x - xs) <= 1e-11 * np.linalg.norm(xs)


def dense_transfer(lev, b):
    """Dense A_l, R = [R_cf I], P (one-point) and the F / C block-Jacobi
    matrices of one exported oracle level."""
    A = bsr_dense(lev["row_ptr"], lev["col"], lev["vals"])
    E = lev["E"]
    n = E * b
    cf = lev["cf"]
    C = np.nonzero(cf == 1)[0]
    F = np.nonzero(cf == 0)[0]
    nC = len(C)
    I = np.eye(b)
    P = np.zeros((n, nC * b))
    for i in range(E):
        J = lev["ipc"][i]
        if J >= 0:
            P[i * b:(i + 1) * b, J * b:(J + 1) * b] = I
    R = np.zeros((nC * b, n))
    for c, i in enumerate(C):
        R[c * b:(c + 1) * b, i * b:(i + 1) * b] = I
        for q in range(lev["R_rp"][c], lev["R_rp"][c + 1]):
            j = F[lev["R_ci"][q]]
            R[c * b:(c + 1) * b, j * b:(j + 1) * b] = lev["R_v"][q]
    DF = np.zeros((n, n))
    DC = np.zeros((n, n))
    for i in range(E):
        (DC if cf[i] else DF)[i * b:(i + 1) * b, i * b:(i + 1) * b] = lev["dinv"][i]
    return A, R, P, DF, DC


def composed_cycle(H, l, kind, fs, cs, b):
    """The cycle as a matrix, composed from its error propagation (Eq. relax,
    Eq. cgc): I - M_l A_l = S_C^cs S_F^fs (I - P B R A_l), with B the coarse
    solver: B = M_{l+1}^V (V-cycle) or, for the F-cycle, the F-cycle followed by
    a V-cycle from its result: I - B A_c = (I - M^V A_c)(I - M^F A_c)."""
    lev = H.level(l)
    if lev["coarsest"]:
        A = bsr_dense(lev["row_ptr"], lev["col"], lev["vals"])
        return np.linalg.inv(A)
    A, R, P, DF, DC = dense_transfer(lev, b)
    Ac = R @ A @ P
    MV = composed_cycle(H, l + 1, "V", fs, cs, b)
    if kind == "V":
        B = MV
    else:
        MF = composed_cycle(H, l + 1, "F", fs, cs, b)
        B = MF + MV - MV @ Ac @ MF
    n = A.shape[0]
    Id = np.eye(n)
    E = Id - P @ B @ R @ A
    for _ in range(fs):
        E = (Id - DF @ A) @ E
    for _ in range(cs):
        E = (Id - DC @ A) @ E
    return (Id - E) @ np.linalg.inv(A)


@pytest.mark.parametrize("kind", ["V", "F"])
@pytest.mark.parametrize("name,N,p,k,fs,cs", [("C2", 4, 2, 2, 3, 1), ("C3", 4, 1, 1, 1, 1),
                                             ("C1", 5, 1, 2, 1, 2)])
def test_cycles_match_composed_error_propagation(oracle_lib, kind, name, N, p, k, fs, cs):
    """The oracle's V- and F-cycles against the same cycles composed in numpy
    from the exported level operators (R, P, D^-1, A_l and the coarse
    operators; the coarse operator used by the composition is R A P formed
    densely, which the Galerkin pin ties to the stored one)."""
    P = tiny(name, N=N, p=p)
    H = oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], neumann_degree=k, max_coarse=2,
                             filter_targets=0, f_sweeps=fs, c_sweeps=cs, cycle=kind)
    assert H.nlev >= 4
    n, b = P["n"], P["b"]
    M = np.stack([H.vcycle(e) for e in np.eye(n)], axis=1)
    Mc = composed_cycle(H, 0, kind, fs, cs, b)
    assert np.abs(M - Mc).max() <= 1e-11 * np.abs(Mc).max()
    if kind == "F":  # the F-cycle is a different operator from the V-cycle
        H.set_cycle("V")
        MV = np.stack([H.vcycle(e) for e in np.eye(n)], axis=1)
        assert np.abs(MV - M).max() >= 1e-6 * np.abs(M).max()


def test_fcycle_solve_matches_dense_and_converges_faster(oracle_lib):
    """FGMRES with the F-cycle (Sec. 6 scaling study) reaches the dense solution
    in no more iterations than with the V-cycle."""
    P = tiny("C3", N=8, p=3)
    A = bsr_dense(P["row_ptr"], P["col"], P["vals"])
    xs = np.linalg.solve(A, P["rhs"])
    its = {}
    for kind in ("V", "F"):
        H = oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], neumann_degree=1, max_coarse=2,
                                 cycle=kind)
        r = H.solve(P["rhs"])
        assert r["status"] == 0 and r["relres"] <= 1e-10
        assert np.linalg.norm(r["x"] - xs) <= 1e-8 * np.linalg.norm(xs)
        its[kind] = r["iterations"]
    assert its["F"] <= its["V"]


def test_minimal_f_sweeps_two_level(oracle_lib):
    """Two levels, R = R_ideal (theta = 0, no filtering, k >= d_f): after the exact
    coarse-grid correction the F error is propagated by L, nilpotent of degree
    d_f + 1, so exactly d_f + 1 Jacobi F sweeps make one cycle exact and d_f do not
    (Lemma ideal restriction; Sec. 4.1)."""
    P = tiny("C3", N=6, p=1)   # jittered mesh: the F-F graph has paths (d_f = 2)
    par = dict(theta=0.0, filter_targets=0, neumann_degree=60, max_levels=2, max_coarse=1,
               max_dense=100000, c_sweeps=0)
    H = oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], **par)
    df = longest_ff_path(H.level(0))
    assert df >= 2
    A = bsr_dense(P["row_ptr"], P["col"], P["vals"])
    xs = np.linalg.solve(A, P["rhs"])
    x_ok = H.vcycle(P["rhs"], f_sweeps=df + 1, c_sweeps=0)
    x_short = H.vcycle(P["rhs"], f_sweeps=df, c_sweeps=0)
    assert np.linalg.norm(x_ok - xs) <= 1e-12 * np.linalg.norm(xs)
    assert np.linalg.norm(x_short - xs) >= 1e-8 * np.linalg.norm(xs)


def test_error_propagation_is_strictly_block_lower_triangular(oracle_lib):
    """Remark (nilpotent error propagation): with truncated Neumann R and Jacobi
    F-relaxation on a triangular A, the multilevel error propagation
    E = I - M^{-1} A is strictly block lower triangular, hence nilpotent."""
    P = tiny("C1", N=4, p=1)
    b, n, E = P["b"], P["n"], P["E"]
    H = oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], neumann_degree=1, max_coarse=2)
    assert H.nlev >= 3
    A = bsr_dense(P["row_ptr"], P["col"], P["vals"])
    Minv = np.stack([H.vcycle(e) for e in np.eye(n)], axis=1)
    Em = np.eye(n) - Minv @ A
    scale = np.abs(Em).max()
    for i in range(E):
        blk = Em[i * b:(i + 1) * b, i * b:]
        assert np.abs(blk).max() <= 1e-13 * scale
    assert np.abs(np.linalg.matrix_power(Em, E)).max() <= 1e-10 * scale


# -----------------------------------------------------------------------------
# a15: FGMRES
# -----------------------------------------------------------------------------

def test_fgmres_triangular_matches_forward_substitution(oracle_lib):
    P = D.make_problem("C1")
    H = oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], neumann_degree=1)
    r = H.solve(P["rhs"])
    assert r["status"] == 0
    xs = block_forward_substitution(P)
    assert np.linalg.norm(r["x"] - xs) <= 1e-9 * np.linalg.norm(xs)
    assert r["relres"] <= 1e-10
    h = r["history"]
    assert np.all(np.diff(h) <= 1e-14)    # GMRES residuals never increase
    assert h[-1] <= 1e-10 and h[0] == 1.0


@pytest.mark.parametrize("name,N,p", [("C2", 8, 2), ("C3", 6, 3)])
def test_fgmres_matches_dense_solve(oracle_lib, name, N, p):
    P = tiny(name, N=N, p=p)
    H = oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], neumann_degree=2, max_coarse=4)
    r = H.solve(P["rhs"], restart=5)
    A = bsr_dense(P["row_ptr"], P["col"], P["vals"])
    xs = np.linalg.solve(A, P["rhs"])
    assert r["status"] == 0 and r["relres"] <= 1e-10
    assert np.linalg.norm(r["x"] - xs) <= 1e-8 * np.linalg.norm(xs)


# -----------------------------------------------------------------------------
# scalar nAIR (block-diagonal scaling, then coarsening by degree of freedom)
# -----------------------------------------------------------------------------

def scaled_dense(P):
    """D^{-1} A with D the block diagonal of A (numpy inverses)."""
    b, E = P["b"], P["E"]
    A = bsr_dense(P["row_ptr"], P["col"], P["vals"])
    Dinv = np.zeros_like(A)
    for i in range(E):
        sl = slice(i * b, (i + 1) * b)
        Dinv[sl, sl] = np.linalg.inv(A[sl, sl])
    return A, Dinv, Dinv @ A


@pytest.mark.parametrize("name,N,p", [("C1", 4, 1), ("C2", 4, 2), ("C3", 3, 3)])
def test_scalar_scaled_matrix(oracle_lib, name, N, p):
    """Level 0 of scalar nAIR is D^{-1} A stored by degree of freedom: unit
    diagonal, no coupling inside an element (D_ii^{-1} A_ii = I exactly), the
    structural zeros of the face couplings not stored, sorted columns."""
    P = tiny(name, N=N, p=p)
    b = P["b"]
    H = oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], scalar=True)
    lev = H.level(0)
    assert lev["E"] == P["n"] and lev["vals"].shape[1:] == (1, 1)
    S = bsr_dense(lev["row_ptr"], lev["col"], lev["vals"])
    A, Dinv, DA = scaled_dense(P)
    for i in range(P["E"]):
        sl = slice(i * b, (i + 1) * b)
        DA[sl, sl] = np.eye(b)
    assert np.array_equal(S != 0, DA != 0)
    assert np.abs(S - DA).max() <= 1e-13 * np.abs(DA).max()
    assert np.all(np.diag(S) == 1.0)
    assert np.all(lev["vals"] != 0.0)
    for i in range(lev["E"]):
        c = lev["col"][lev["row_ptr"][i]:lev["row_ptr"][i + 1]]
        assert np.all(np.diff(c) > 0)


@pytest.mark.parametrize("p", [1, 2])
def test_scalar_exact_under_ideal_settings(oracle_lib, p):
    """Scalar nAIR under ideal settings (theta = 0, no filtering, exact Neumann,
    enough F sweeps): the cycle solves (D^{-1} A) y = D^{-1} f exactly, so the
    preconditioner applied to f is A^{-1} f (Lemma ideal restriction)."""
    P = tiny("C1", N=5, p=p)
    H = oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], scalar=True, theta=0.0, filter_targets=0,
                             neumann_degree=80, max_coarse=2, f_sweeps=80, c_sweeps=1)
    assert H.nlev >= 3
    A = bsr_dense(P["row_ptr"], P["col"], P["vals"])
    xs = np.linalg.solve(A, P["rhs"])
    x = H.vcycle(P["rhs"])
    assert np.linalg.norm(x - xs) <= 1e-11 * np.linalg.norm(xs)


@pytest.mark.parametrize("name,N,p", [("C2", 8, 2), ("C3", 6, 3)])
def test_scalar_solve_matches_dense(oracle_lib, name, N, p):
    P = tiny(name, N=N, p=p)
    H = oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], scalar=True, neumann_degree=2)
    r = H.solve(P["rhs"], restart=10)
    A = bsr_dense(P["row_ptr"], P["col"], P["vals"])
    xs = np.linalg.solve(A, P["rhs"])
    assert r["status"] == 0 and r["relres"] <= 1e-10
    assert np.linalg.norm(r["x"] - xs) <= 1e-8 * np.linalg.norm(xs)
    w = D.functional_weights(P["n"])
    ra = H.solve(w, transposed=True, restart=10)
    assert ra["status"] == 0
    assert np.linalg.norm(ra["x"] - np.linalg.solve(A.T, w)) <= 1e-8 * np.linalg.norm(ra["x"])


@pytest.mark.parametrize("name,N,p,k", [("C2", 4, 2, 2), ("C3", 3, 2, 1)])
def test_scalar_preconditioner_composition(oracle_lib, name, N, p, k):
    """The scalar preconditioner is M_s D^{-1} (M_s the cycle of the scaled
    matrix, pinned by the composition test on its own hierarchy) and the
    transposed one is its transpose D^{-T} M_s^T."""
    P = tiny(name, N=N, p=p)
    n = P["n"]
    H = oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], scalar=True, neumann_degree=k,
                             max_coarse=4, filter_targets=0)
    assert H.nlev >= 3
    _, Dinv, _ = scaled_dense(P)
    M = np.stack([H.vcycle(e) for e in np.eye(n)], axis=1)
    Ms = composed_cycle(H, 0, "V", k + 1, 1, 1)
    assert np.abs(M - Ms @ Dinv).max() <= 1e-11 * np.abs(M).max()
    MT = np.stack([H.vcycle(e, transposed=True) for e in np.eye(n)], axis=1)
    assert np.abs(MT - M.T).max() <= 1e-12 * np.abs(M).max()


# -----------------------------------------------------------------------------
# a16: adjoint
# -----------------------------------------------------------------------------

def dense_cycle(H, n, **kw):
    """The cycle with zero initial guess as a dense matrix (columns = images of e_k)."""
    return np.stack([H.vcycle(e, **kw) for e in np.eye(n)], axis=1)


@pytest.mark.parametrize("name,N,p,k", [("C1", 4, 1, 1), ("C2", 4, 2, 2), ("C3", 4, 2, 1)])
@pytest.mark.parametrize("fs,cs", [(2, 1), (3, 0), (1, 2), (0, 0)])
def test_transposed_cycle_is_adjoint_of_vcycle(oracle_lib, name, N, p, k, fs, cs):
    """The transposed cycle (R^T interpolation, P^T restriction, C then F
    pre-sweeps with the transposed diagonal-block inverses, K^T coarse solve) is
    the transpose of the V-cycle as a linear map: M_T = M^T.  Compared on
    unit vectors against the dense forward cycle."""
    P = tiny(name, N=N, p=p)
    H = oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], neumann_degree=k, max_coarse=2)
    assert H.nlev >= 3
    n = P["n"]
    M = dense_cycle(H, n, f_sweeps=fs, c_sweeps=cs)
    MT = dense_cycle(H, n, f_sweeps=fs, c_sweeps=cs, transposed=True)
    scale = np.abs(M).max()
    assert np.abs(MT - M.T).max() <= 1e-13 * scale


@pytest.mark.parametrize("p", [1, 2])
def test_transposed_cycle_exact_under_ideal_interpolation(oracle_lib, p):
    """Corollary (ideal interpolation): for A^T, R^T with exact Neumann R is the
    ideal interpolation -(A^T)_ff^{-1} (A^T)_fc; an exact F solve before the
    coarse-grid correction (enough Jacobi F sweeps on the nilpotent F block)
    makes every level exact, so one transposed cycle solves A^T y = w."""
    P = tiny("C1", N=6, p=p)
    H = oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], theta=0.0, filter_targets=0,
                             neumann_degree=80, max_coarse=2, f_sweeps=80, c_sweeps=1)
    assert H.nlev >= 3
    A = bsr_dense(P["row_ptr"], P["col"], P["vals"])
    w = D.functional_weights(P["n"])
    y = H.vcycle(w, transposed=True)
    ys = np.linalg.solve(A.T, w)
    assert np.linalg.norm(y - ys) <= 1e-11 * np.linalg.norm(ys)
    # too few F sweeps: the pre-relaxation is no longer an exact F solve
    H2 = oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], theta=0.0, filter_targets=0,
                              neumann_degree=80, max_coarse=2, f_sweeps=1, c_sweeps=1)
    y2 = H2.vcycle(w, transposed=True)
    assert np.linalg.norm(y2 - ys) >= 1e-6 * np.linalg.norm(ys)


@pytest.mark.parametrize("name,N,p", [("C2", 8, 2), ("C3", 6, 3)])
def test_transposed_solve_matches_dense_solve(oracle_lib, name, N, p):
    """FGMRES on A^T with the transposed cycle of the forward hierarchy."""
    P = tiny(name, N=N, p=p)
    H = oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], neumann_degree=2, max_coarse=4)
    w = D.functional_weights(P["n"])
    r = H.solve(w, transposed=True, restart=5)
    A = bsr_dense(P["row_ptr"], P["col"], P["vals"])
    ys = np.linalg.solve(A.T, w)
    assert r["status"] == 0 and r["relres"] <= 1e-10
    assert np.linalg.norm(r["x"] - ys) <= 1e-8 * np.linalg.norm(ys)
    assert np.all(np.diff(r["history"]) <= 1e-14)


def test_transpose_and_adjoint_gradients(oracle_lib):
    """A^T lambda = w by nAIR on A^T; gradients of J = w . x against central
    finite differences of dense solves."""
    P = D.make_problem("C2", N=4, keep_parts=True)
    b, E, n = P["b"], P["E"], P["n"]
    trp, tci, tv = oracle_lib.transpose(P["row_ptr"], P["col"], P["vals"])
    A = bsr_dense(P["row_ptr"], P["col"], P["vals"])
    assert np.array_equal(bsr_dense(trp, tci, tv), A.T)
    w = D.functional_weights(n)
    Hf = oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], neumann_degree=2, max_coarse=4)
    Ht = oracle_lib.Hierarchy(trp, tci, tv, neumann_degree=2, max_coarse=4)
    x = Hf.solve(P["rhs"], tol=1e-13)["x"]
    lam = Ht.solve(w, tol=1e-13)["x"]
    lam_t = Hf.solve(w, tol=1e-13, transposed=True)["x"]
    assert np.linalg.norm(lam_t - lam) <= 1e-10 * np.linalg.norm(lam)
    gs, gq = oracle_lib.gradients(P["mass"], lam, x)

    def J(sig, q):
        vals = P["vals0"].copy()
        vals[P["diag_pos"]] += sig[:, None, None] * P["mass"]
        Ad = bsr_dense(P["row_ptr"], P["col"], vals)
        rhs = np.einsum("eij,ej->ei", P["mass"], q.reshape(E, b)).ravel()
        return w @ np.linalg.solve(Ad, rhs)

    sig0 = P["sigma"].copy()
    q0 = P["q"].copy()
    eps = 1e-6
    for e in [0, 5, E - 1]:
        sp, sm = sig0.copy(), sig0.copy()
        sp[e] += eps
        sm[e] -= eps
        fd = (J(sp, q0) - J(sm, q0)) / (2 * eps)
        assert abs(fd - gs[e]) <= 1e-6 * max(1.0, abs(fd))
    for i in [0, 7, n - 1]:
        qp, qm = q0.copy(), q0.copy()
        qp[i] += eps
        qm[i] -= eps
        fd = (J(sig0, qp) - J(sig0, qm)) / (2 * eps)
        assert abs(fd - gq[i]) <= 1e-6 * max(1.0, abs(fd))
