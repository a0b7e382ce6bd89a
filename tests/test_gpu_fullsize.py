"""Parity at the full workload sizes, in the configuration the benchmark times.

C2 (786,432 unknowns): the whole hierarchy (C/F splittings, patterns, values)
and the residual history against the FP64 oracle run to completion.
C3 (917,504 unknowns, b = 28): hierarchy against the oracle, mixed precision
against FP64.  C5 (5,242,880 unknowns): too large for the oracle in a test, so
it is checked by properties that hold at any size: the FP64 residual of the
returned forward and adjoint solutions recomputed independently on the host
(scipy BSR products), and the mixed-precision forward and adjoint solutions and
gradients against the all-FP64 GPU solve.  The adjoint solves use the
transposed cycle of the forward hierarchy (C2: against the oracle's).
"""
import numpy as np
import pytest

import dgtransport as D

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nair():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1704_05001_gb300 as nair
    return nair


@pytest.fixture(scope="module")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host_residual(P, x, w=None):
    """||rhs - A x|| / ||rhs||, or ||w - A^T x|| / ||w|| when w is given."""
    sp = pytest.importorskip("scipy.sparse")
    b = P["b"]
    A = sp.bsr_matrix((P["vals"], P["col"], P["row_ptr"]), shape=(P["n"], P["n"]), blocksize=(b, b))
    if w is not None:
        return np.linalg.norm(w - A.T @ x) / np.linalg.norm(w)
    r = P["rhs"] - A @ x
    return np.linalg.norm(r) / np.linalg.norm(P["rhs"])


def same_hierarchy(S, H):
    assert S.num_levels() == H.nlev
    for l in range(H.nlev):
        g, o = S.level(l), H.level(l)
        assert np.array_equal(g["row_ptr"], o["row_ptr"]) and np.array_equal(g["col"], o["col"]), l
        d = np.abs(g["vals"] - o["vals"]).reshape(len(o["vals"]), -1).max(axis=1)
        s = np.maximum(np.abs(o["vals"]).reshape(len(o["vals"]), -1).max(axis=1), 1e-300)
        assert np.max(d / s) <= 1e-12, l
        if not o["coarsest"]:
            assert np.array_equal(g["cf"], o["cf"]), l
            assert np.array_equal(g["ipc"], o["ipc"]), l
            assert np.array_equal(g["R_ci"], o["R_ci"]), l


def test_c2_full_hierarchy_and_history(nair, oracle_mod):
    P = D.make_problem("C2")
    k = P["neumann_degree"]
    S = nair.NairSolver(dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]), neumann_degree=k)
    x, rep = S.solve(dev(P["rhs"]))
    H = oracle_mod.Hierarchy(P["row_ptr"], P["col"], P["vals"], neumann_degree=k)
    same_hierarchy(S, H)
    ref = H.solve(P["rhs"])
    assert rep["iterations"] == ref["iterations"]
    assert np.max(np.abs(rep["history"] - ref["history"])) <= 1e-12
    xs = x.cpu().numpy()
    assert host_residual(P, xs) <= 1e-10
    assert np.linalg.norm(xs - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])
    # C4: the adjoint through the transposed cycle of the same hierarchy
    w = D.functional_weights(P["n"])
    lam, repa = S.adjoint_solve(dev(w))
    refa = H.solve(w, transposed=True)
    assert repa["iterations"] == refa["iterations"]
    assert np.max(np.abs(repa["history"] - refa["history"])) <= 1e-12
    assert host_residual(P, lam.cpu().numpy(), w) <= 1e-10


def test_c2_full_fcycle_k3(nair):
    """The F-cycle with Neumann degree 3 (Sec. 6 scaling study) on the full C2
    problem: FP64 residual recomputed on the host, in both precisions."""
    P = D.make_problem("C2")
    args = (dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]))
    for prec in ("fp64", "mixed"):
        S = nair.NairSolver(*args, neumann_degree=3, cycle_type="F", precision=prec)
        x, rep = S.solve(dev(P["rhs"]))
        assert rep["rel_res"] <= 1e-10
        assert host_residual(P, x.cpu().numpy()) <= 1e-10
        S.close()


def test_c2_full_scalar(nair):
    """Scalar nAIR on the full C2 problem: FP64 residual recomputed on the host,
    forward in both precisions and the adjoint."""
    P = D.make_problem("C2")
    args = (dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]))
    w = D.functional_weights(P["n"])
    for prec in ("fp64", "mixed"):
        S = nair.NairSolver(*args, neumann_degree=2, scalar=1, precision=prec)
        x, rep = S.solve(dev(P["rhs"]))
        assert rep["rel_res"] <= 1e-10
        assert host_residual(P, x.cpu().numpy()) <= 1e-10
        lam, repa = S.adjoint_solve(dev(w))
        assert host_residual(P, lam.cpu().numpy(), w) <= 1e-10
        S.close()


def test_c3_full_hierarchy_and_mixed(nair, oracle_mod):
    P = D.make_problem("C3")
    args = (dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]))
    S = nair.NairSolver(*args, neumann_degree=1)
    x64, r64 = S.solve(dev(P["rhs"]))
    H = oracle_mod.Hierarchy(P["row_ptr"], P["col"], P["vals"], neumann_degree=1)
    same_hierarchy(S, H)
    ref = H.solve(P["rhs"])
    assert r64["iterations"] == ref["iterations"]
    assert np.max(np.abs(r64["history"] - ref["history"])) <= 1e-12
    Sm = nair.NairSolver(*args, neumann_degree=1, precision="mixed")
    xm, rm = Sm.solve(dev(P["rhs"]))
    xs, xms = x64.cpu().numpy(), xm.cpu().numpy()
    assert host_residual(P, xs) <= 1e-10 and host_residual(P, xms) <= 1e-10
    assert np.linalg.norm(xms - xs) <= 1e-8 * np.linalg.norm(xs)


def test_c5_full_forward_adjoint_mixed_vs_fp64(nair):
    P = D.make_problem("C5")
    n, E = P["n"], P["E"]
    args = (dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]))
    w = dev(D.functional_weights(n))
    out = {}
    for prec in ("fp64", "mixed"):
        S = nair.NairSolver(*args, neumann_degree=P["neumann_degree"], precision=prec)
        x, rep = S.solve(dev(P["rhs"]))
        lam, repa = S.adjoint_solve(w)
        gs, gq = nair.gradients(dev(P["mass"]), lam, x)
        assert rep["rel_res"] <= 1e-10 and repa["rel_res"] <= 1e-10
        assert host_residual(P, lam.cpu().numpy(), w.cpu().numpy()) <= 1e-10
        out[prec] = (x.cpu().numpy(), gs.cpu().numpy(), gq.cpu().numpy())
        S.close()
    x64, gs64, gq64 = out["fp64"]
    xm, gsm, gqm = out["mixed"]
    assert host_residual(P, x64) <= 1e-10 and host_residual(P, xm) <= 1e-10
    assert np.linalg.norm(xm - x64) <= 1e-8 * np.linalg.norm(x64)
    assert np.linalg.norm(gsm - gs64) <= 1e-8 * np.linalg.norm(gs64)
    assert np.linalg.norm(gqm - gq64) <= 1e-8 * np.linalg.norm(gq64)
