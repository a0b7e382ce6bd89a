"""The F relaxation in the scaled variable y_F = D_FF x_F computes the block-Jacobi
iterates of the paper's F relaxation (Sec. 5.1): on a coarse level of an oracle
hierarchy, k F sweeps and one C sweep written out in numpy in the x form and in
the y form (right-scaled couplings A_ij D_jj^{-1}, one D^{-1} at the end) agree
to rounding, forward and for the transposed level operator.  CPU only; the GPU
kernels of the y form are checked against the oracle in the GPU parity tests."""
import numpy as np
import pytest

import dgtransport as D


def _blocks(lev, b):
    E = lev["E"]
    rp, ci, v = lev["row_ptr"], lev["col"], lev["vals"]
    A = np.zeros((E * b, E * b))
    for i in range(E):
        for p in range(rp[i], rp[i + 1]):
            j = ci[p]
            A[i * b:(i + 1) * b, j * b:(j + 1) * b] = v[p]
    return A


def _relax_x(A, Dinv, cf, b, f, x0, nf):
    """k F sweeps (block Jacobi on the F rows, x_C fixed), then one C sweep."""
    E = len(cf)
    x = x0.copy()
    idx = lambda S: np.concatenate([np.arange(i * b, (i + 1) * b) for i in S]) if len(S) else np.zeros(0, int)
    F, C = idx(np.where(cf == 0)[0]), idx(np.where(cf == 1)[0])
    Ablk = A.copy()
    for i in range(E):  # off-diagonal part
        Ablk[i * b:(i + 1) * b, i * b:(i + 1) * b] = 0.0
    for _ in range(nf):
        r = f - Ablk @ x
        xn = x.copy()
        for i in np.where(cf == 0)[0]:
            xn[i * b:(i + 1) * b] = Dinv[i] @ r[i * b:(i + 1) * b]
        x = xn
    r = f - Ablk @ x
    for i in np.where(cf == 1)[0]:
        x[i * b:(i + 1) * b] = Dinv[i] @ r[i * b:(i + 1) * b]
    return x


def _relax_y(A, Dinv, cf, b, f, x0, nf):
    """The same sweeps on y_F = D_FF x_F: h = f_F - A_FC x_C once, y^1 = h -
    A_FF x_F^0, y^{k+1} = h - sum_j (A_ij D_jj^{-1}) y_j, then the C sweep reads
    y_F through the scaled blocks, and x_F = D_FF^{-1} y_F at the end."""
    E = len(cf)
    Fe, Ce = np.where(cf == 0)[0], np.where(cf == 1)[0]
    idx = lambda S: np.concatenate([np.arange(i * b, (i + 1) * b) for i in S]) if len(S) else np.zeros(0, int)
    F, C = idx(Fe), idx(Ce)
    off = A.copy()
    for i in range(E):
        off[i * b:(i + 1) * b, i * b:(i + 1) * b] = 0.0
    S = off.copy()  # right-scaled couplings in F columns: A_ij D_jj^{-1}
    for j in Fe:
        S[:, j * b:(j + 1) * b] = off[:, j * b:(j + 1) * b] @ Dinv[j]
    xC = x0[C]
    h = f[F] - off[np.ix_(F, C)] @ xC
    y = h - off[np.ix_(F, F)] @ x0[F]
    for _ in range(nf - 1):
        y = h - S[np.ix_(F, F)] @ y
    rC = f[C] - S[np.ix_(C, F)] @ y - off[np.ix_(C, C)] @ xC
    x = np.zeros_like(x0)
    for k, i in enumerate(Ce):
        x[i * b:(i + 1) * b] = Dinv[i] @ rC[k * b:(k + 1) * b]
    for k, i in enumerate(Fe):
        x[i * b:(i + 1) * b] = Dinv[i] @ y[k * b:(k + 1) * b]
    return x


@pytest.mark.parametrize("transposed", [False, True])
def test_y_form_f_relaxation_equals_block_jacobi(oracle_lib, transposed):
    P = D.make_problem("C2", N=6)
    H = oracle_lib.Hierarchy(P["row_ptr"], P["col"], P["vals"], neumann_degree=2, max_coarse=4)
    b = P["b"]
    lev = H.level(1)
    assert not lev["coarsest"]
    A = _blocks(lev, b)
    cf = lev["cf"]
    Dinv = np.array(lev["dinv"])
    if transposed:  # the transposed cycle's F sweeps: A^T with (D_ii^{-1})^T
        A = A.T.copy()
        Dinv = Dinv.transpose(0, 2, 1).copy()
    n = lev["E"] * b
    rng = np.random.default_rng(5)
    f = rng.uniform(-1, 1, n)
    x0 = rng.uniform(-1, 1, n)
    for nf in (1, 2, 3, 5):
        xa = _relax_x(A, Dinv, cf, b, f, x0, nf)
        xb = _relax_y(A, Dinv, cf, b, f, x0, nf)
        assert np.linalg.norm(xa - xb) <= 1e-13 * np.linalg.norm(xa), nf
