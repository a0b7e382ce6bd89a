"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Bar (from the method's arithmetic): bit-exact C/F splittings, strength flags,
interpolation maps and sparsity patterns; hierarchy values identical (the GPU
setup uses the oracle's canonical fma order, so equality is expected, and the
test allows 1e-12 relative per row); residual histories within 1e-12 absolute
(they are already relative to ||b||) with identical iteration counts.
"""
import numpy as np
import pytest

import dgtransport as D

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nair():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1704_05001_gb300 as nair
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return nair


@pytest.fixture(scope="module")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_rows(a, b):
    """max over block rows of |a - b| / max |b| in that row (values as (nnzb, b, b))."""
    if a.size == 0:
        return 0.0
    d = np.abs(a - b).reshape(len(a), -1).max(axis=1)
    s = np.maximum(np.abs(b).reshape(len(b), -1).max(axis=1), 1e-300)
    return float(np.max(d / s))


CASES = [
    ("C1", 32, 1, 1),       # full C1: P1, constant flow, triangular
    ("C2", 16, 2, 2),       # P2 rotating flow, log-normal sigma
    ("C3", 6, 6, 1),        # P6 jittered, b = 28
    ("C5", 12, 3, 1),       # P3 jittered rotating
    ("C3", 10, 4, 2),       # b = 15, k = 2
]


def compare_hierarchies(S, H, b, check_setup_data=True):
    assert S.num_levels() == H.nlev
    for l in range(H.nlev):
        g = S.level(l)
        o = H.level(l)
        assert g["E"] == o["E"] and g["nnzb"] == o["nnzb"], f"level {l} sizes"
        assert np.array_equal(g["row_ptr"], o["row_ptr"]), f"level {l} row pointers"
        assert np.array_equal(g["col"], o["col"]), f"level {l} pattern"
        assert rel_rows(g["vals"], o["vals"]) <= 1e-12, f"level {l} values"
        assert np.array_equal(g["dinv"], o["dinv"]), f"level {l} diagonal inverses"
        if o["coarsest"]:
            continue
        assert np.array_equal(g["cf"], o["cf"]), f"level {l} C/F"
        assert np.array_equal(g["ipc"], o["ipc"]), f"level {l} interpolation"
        assert np.array_equal(g["R_rp"], o["R_rp"]) and np.array_equal(g["R_ci"], o["R_ci"]), f"level {l} R pattern"
        assert rel_rows(g["R_v"], o["R_v"]) <= 1e-12, f"level {l} R values"
        if check_setup_data:
            assert np.array_equal(g["strong"], o["strong"]), f"level {l} strength"
            assert np.array_equal(g["lam"], o["lam"]), f"level {l} lambda"
            assert np.array_equal(g["D_rp"], o["D_rp"]) and np.array_equal(g["D_ci"], o["D_ci"]), f"level {l} Delta pattern"
            assert rel_rows(g["D_v"], o["D_v"]) <= 1e-12, f"level {l} Delta values"
            assert np.array_equal(g["L_ci"], o["L_ci"]), f"level {l} L pattern"
            assert rel_rows(g["L_v"], o["L_v"]) <= 1e-12, f"level {l} L values"


@pytest.mark.parametrize("b", [1, 3, 6, 10, 15, 21, 28, 32])
def test_block_inverse_bitwise(nair, oracle_mod, b):
    r = np.random.default_rng(100 + b)
    nblk = 333
    A = r.standard_normal((nblk, b, b)) + np.eye(b) * (0.5 * b)
    X = nair.block_inverse(dev(A)).cpu().numpy()
    for k in range(nblk):
        assert np.array_equal(X[k], oracle_mod.block_inverse(A[k]))


@pytest.mark.parametrize("b", [3, 6, 10, 15, 21, 28])
def test_block_inverse_pivot_ties_bitwise(nair, oracle_mod, b):
    """Small-integer blocks: equal |entries| in a pivot column are common, zero
    diagonals force row exchanges, and -0.0 meets +0.0; the first row of largest
    magnitude must win exactly as in the oracle."""
    r = np.random.default_rng(200 + b)
    blocks = []
    while len(blocks) < 200:
        A = r.integers(-2, 3, size=(b, b)).astype(np.float64)
        A[r.random((b, b)) < 0.2] = -0.0
        try:
            X = oracle_mod.block_inverse(A)
        except oracle_mod.OracleError:
            continue
        blocks.append((A, X))
    A = np.stack([a for a, _ in blocks])
    X = nair.block_inverse(dev(A)).cpu().numpy()
    for k, (_, Xo) in enumerate(blocks):
        assert np.array_equal(X[k].view(np.uint64), Xo.view(np.uint64))


@pytest.mark.parametrize("b", [3, 6, 28, 32])
def test_block_inverse_singular(nair, b):
    A = np.ones((40, b, b))
    with pytest.raises(nair.NairError) as e:
        nair.block_inverse(dev(A))
    assert e.value.status == 2


@pytest.mark.parametrize("name,N,p,k", CASES)
def test_hierarchy_and_solve_parity(nair, oracle_mod, name, N, p, k):
    P = D.make_problem(name, N=N, p=p)
    b = P["b"]
    params = dict(neumann_degree=k, max_coarse=4)
    S = nair.NairSolver(dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]), keep_setup_data=1, **params)
    H = oracle_mod.Hierarchy(P["row_ptr"], P["col"], P["vals"], **params)
    compare_hierarchies(S, H, b)
    x, rep = S.solve(dev(P["rhs"]))
    ref = H.solve(P["rhs"])
    assert ref["status"] == 0
    assert rep["iterations"] == ref["iterations"]
    assert np.max(np.abs(rep["history"] - ref["history"])) <= 1e-12
    assert rep["rel_res"] <= 1e-10
    xs = x.cpu().numpy()
    assert np.linalg.norm(xs - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])
    # one V-cycle on a seeded vector
    f = D.rng.uniform(7, P["n"]) - 0.5
    z = S.vcycle(dev(f)).cpu().numpy()
    zr = H.vcycle(f)
    assert np.linalg.norm(z - zr) <= 1e-12 * np.linalg.norm(zr)
    S.close()


def test_exact_settings_one_cycle(nair):
    """theta = 0, no filtering, k and F sweeps beyond the F-graph depth: one
    V-cycle solves the triangular system (Lemma ideal restriction)."""
    P = D.make_problem("C1", N=6, p=1)
    S = nair.NairSolver(dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]), strength_theta=0.0,
                        filter_targets=0, neumann_degree=64, f_sweeps=64, max_coarse=2)
    x = S.vcycle(dev(P["rhs"])).cpu().numpy()
    from conftest import bsr_dense
    A = bsr_dense(P["row_ptr"], P["col"], P["vals"])
    xs = np.linalg.solve(A, P["rhs"])
    assert np.linalg.norm(x - xs) <= 1e-11 * np.linalg.norm(xs)


def test_edge_single_element(nair, oracle_mod):
    """E = 1: the fine level is the coarsest; the dense solve is the whole method."""
    r = np.random.default_rng(5)
    A = (r.standard_normal((1, 6, 6)) + 6 * np.eye(6))
    rp = np.array([0, 1], dtype=np.int32)
    ci = np.array([0], dtype=np.int32)
    rhs = r.standard_normal(6)
    S = nair.NairSolver(dev(rp), dev(ci), dev(A))
    x, rep = S.solve(dev(rhs))
    assert S.num_levels() == 1
    assert np.allclose(x.cpu().numpy(), np.linalg.solve(A[0], rhs), rtol=1e-12, atol=1e-14)
    assert rep["iterations"] == 1


def test_edge_chain_b1(nair, oracle_mod):
    """Scalar 1D upwind chain (b = 1), a ragged multi-level case."""
    n = 1000
    rp, col, vals = [0], [], []
    for i in range(n):
        if i > 0:
            col.append(i - 1)
            vals.append(-0.9)
        col.append(i)
        vals.append(1.0)
        rp.append(len(col))
    rp = np.array(rp, dtype=np.int32)
    col = np.array(col, dtype=np.int32)
    vals = np.array(vals).reshape(-1, 1, 1)
    rhs = np.ones(n)
    S = nair.NairSolver(dev(rp), dev(col), dev(vals), keep_setup_data=1, max_coarse=4)
    H = oracle_mod.Hierarchy(rp, col, vals, max_coarse=4)
    compare_hierarchies(S, H, 1)
    x, rep = S.solve(dev(rhs))
    ref = H.solve(rhs)
    assert rep["iterations"] == ref["iterations"]
    assert np.max(np.abs(rep["history"] - ref["history"])) <= 1e-12


def test_edge_block32_triangular(nair, oracle_mod):
    """Largest block size (b = 32) on a random block lower-triangular matrix."""
    r = np.random.default_rng(32)
    E, b = 40, 32
    rp, col, vals = [0], [], []
    for i in range(E):
        nb = sorted(set(int(j) for j in r.integers(0, i, size=min(i, 3)))) if i else []
        for j in nb:
            col.append(j)
            vals.append(r.standard_normal((b, b)) * 0.05)
        col.append(i)
        vals.append(r.standard_normal((b, b)) + b * np.eye(b))
        rp.append(len(col))
    rp = np.array(rp, dtype=np.int32)
    col = np.array(col, dtype=np.int32)
    vals = np.array(vals)
    rhs = r.standard_normal(E * b)
    S = nair.NairSolver(dev(rp), dev(col), dev(vals), keep_setup_data=1, max_coarse=4)
    H = oracle_mod.Hierarchy(rp, col, vals, max_coarse=4)
    compare_hierarchies(S, H, b)
    x, rep = S.solve(dev(rhs))
    ref = H.solve(rhs)
    assert rep["iterations"] == ref["iterations"]
    assert np.max(np.abs(rep["history"] - ref["history"])) <= 1e-12


def test_invalid_inputs_rejected(nair):
    P = D.make_problem("C1", N=4)
    col = P["col"].copy()
    col[[1, 2]] = col[[2, 1]]  # unsorted row
    with pytest.raises(nair.NairError) as e:
        nair.NairSolver(dev(P["row_ptr"]), dev(col), dev(P["vals"]))
    assert e.value.status == 1
    vals = P["vals"].copy()
    vals[P["diag_pos"][3]] = 0.0
    with pytest.raises(nair.NairError) as e:
        nair.NairSolver(dev(P["row_ptr"]), dev(P["col"]), dev(vals))
    assert e.value.status == 2


def test_zero_rhs_and_maxiter(nair):
    P = D.make_problem("C2", N=8)
    S = nair.NairSolver(dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]), maxiter=1, neumann_degree=2)
    x, rep = S.solve(dev(np.zeros(P["n"])))
    assert rep["iterations"] == 0 and float(x.abs().max()) == 0.0
    x, rep = S.solve(dev(P["rhs"]), check=False)
    assert rep["status"] == 3 and rep["iterations"] == 1


def test_adjoint_parity_and_gradients(nair, oracle_mod):
    """Adjoint by a second hierarchy built for A^T (adjoint_mode "rebuild")."""
    P = D.make_problem("C2", N=12, keep_parts=True)
    b, E, n = P["b"], P["E"], P["n"]
    params = dict(neumann_degree=2, max_coarse=4)
    S = nair.NairSolver(dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]), keep_setup_data=1,
                        adjoint_mode="rebuild", **params)
    w = D.functional_weights(n)
    lam, rep = S.adjoint_solve(dev(w))
    trp, tci, tv = oracle_mod.transpose(P["row_ptr"], P["col"], P["vals"])
    Ht = oracle_mod.Hierarchy(trp, tci, tv, **params)
    ref = Ht.solve(w)
    assert S.num_levels(adjoint=True) == Ht.nlev
    for l in range(Ht.nlev - 1):
        assert np.array_equal(S.level(l, adjoint=True)["cf"], Ht.level(l)["cf"])
    assert rep["iterations"] == ref["iterations"]
    assert np.max(np.abs(rep["history"] - ref["history"])) <= 1e-12
    x, _ = S.solve(dev(P["rhs"]))
    gs, gq = nair.gradients(dev(P["mass"]), lam, x)
    ogs, ogq = oracle_mod.gradients(P["mass"], lam.cpu().numpy(), x.cpu().numpy())
    assert np.allclose(gs.cpu().numpy(), ogs, rtol=1e-12, atol=1e-15 * np.abs(ogs).max())
    assert np.allclose(gq.cpu().numpy(), ogq, rtol=1e-12, atol=1e-15 * np.abs(ogq).max())


def test_scalar_row_sweeps_parity(nair, oracle_mod):
    """A C2 problem large enough that the F and C sweeps of level 1 run with one
    thread group per row, where FP64 sweeps take the scalar-row form (one thread
    per row and component over the blocks whose row is nonzero, threads sorted
    by entry count) and the F sweeps iterate on y = D x: V-cycles, the solve
    and the transposed cycle (its F sweeps on y = D^T x) against the oracle."""
    import torch
    P = D.make_problem("C2", N=224)
    params = dict(neumann_degree=2, max_coarse=4)
    H = oracle_mod.Hierarchy(P["row_ptr"], P["col"], P["vals"], **params)
    L1 = H.level(1)
    wave = torch.cuda.get_device_properties(0).multi_processor_count * 1536
    avg = len(L1["col"]) / L1["E"]
    assert avg <= 4.0 and min(L1["nF"], L1["nC"]) * P["b"] * 2 > wave  # one group per row
    S = nair.NairSolver(dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]), **params)
    forms = S.sweep_forms()
    assert forms[0] == 1 and forms[1] == 3, forms  # level 1: scalar rows, F sweeps in y
    f = D.rng.uniform(17, P["n"]) - 0.5
    for rep in range(2):
        z = S.vcycle(dev(f)).cpu().numpy()
        zr = H.vcycle(f)
        assert np.linalg.norm(z - zr) <= 1e-12 * np.linalg.norm(zr)
    x, rep = S.solve(dev(P["rhs"]))
    ref = H.solve(P["rhs"])
    assert rep["iterations"] == ref["iterations"]
    assert np.max(np.abs(rep["history"] - ref["history"])) <= 1e-12
    for rep in range(2):
        zt = S.adjoint_vcycle(dev(f)).cpu().numpy()
        zr = H.vcycle(f, transposed=True)
        assert np.linalg.norm(zt - zr) <= 1e-12 * np.linalg.norm(zr)
    assert S.sweep_forms(transposed=True)[1] == 3
    S.close()


@pytest.mark.parametrize("name,N,p,k", [("C2", 12, 2, 2), ("C3", 6, 3, 1)])
@pytest.mark.parametrize("fs,cs", [(2, 1), (4, 2), (5, 0), (8, 1), (9, 1)])
def test_vcycle_sweep_counts_parity(nair, oracle_mod, name, N, p, k, fs, cs):
    """Forward V-cycles with 2 to 9 F sweeps and 0 to 2 C sweeps against the
    oracle, which updates every F row in every F sweep: the GPU cycle updates
    only the rows whose inputs changed (up to 8 F sweeps; more use full sweeps).
    As an F-cycle too, whose second visit of a level starts from a nonzero
    iterate and sweeps every row."""
    P = D.make_problem(name, N=N, p=p)
    params = dict(neumann_degree=k, max_coarse=4, f_sweeps=fs, c_sweeps=cs)
    S = nair.NairSolver(dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]), **params)
    H = oracle_mod.Hierarchy(P["row_ptr"], P["col"], P["vals"], **params)
    f = D.rng.uniform(13, P["n"]) - 0.5
    for rep in range(2):
        z = S.vcycle(dev(f)).cpu().numpy()
        zr = H.vcycle(f)
        assert np.linalg.norm(z - zr) <= 1e-12 * np.linalg.norm(zr)
    S.close()
    S = nair.NairSolver(dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]), cycle_type="F", **params)
    H.set_cycle("F")
    z = S.vcycle(dev(f)).cpu().numpy()
    zr = H.vcycle(f)
    assert np.linalg.norm(z - zr) <= 1e-12 * np.linalg.norm(zr)
    S.close()


@pytest.mark.parametrize("name,N,p,k", CASES)
@pytest.mark.parametrize("fs,cs,graphs", [(0, 1, 1), (3, 0, 1), (1, 2, 0), (0, 1, 0), (4, 2, 1), (9, 1, 1)])
def test_transposed_cycle_parity(nair, oracle_mod, name, N, p, k, fs, cs, graphs):
    """The transposed cycle of the forward hierarchy (R^T interpolation, P^T
    restriction, C then F pre-sweeps on A^T) against the oracle's, on a seeded
    vector; fs = 0 means k + 1 F sweeps.  Graph replay and direct launches."""
    P = D.make_problem(name, N=N, p=p)
    params = dict(neumann_degree=k, max_coarse=4, c_sweeps=cs)
    if fs:
        params["f_sweeps"] = fs
    S = nair.NairSolver(dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]), use_graphs=graphs, **params)
    H = oracle_mod.Hierarchy(P["row_ptr"], P["col"], P["vals"], **params)
    f = D.rng.uniform(11, P["n"]) - 0.5
    for rep in range(2):  # the second call replays what the first built
        z = S.adjoint_vcycle(dev(f)).cpu().numpy()
        zr = H.vcycle(f, transposed=True)
        assert np.linalg.norm(z - zr) <= 1e-12 * np.linalg.norm(zr)
    # the forward cycle is unchanged by the transposed form living beside it
    zf = S.vcycle(dev(f)).cpu().numpy()
    assert np.linalg.norm(zf - H.vcycle(f)) <= 1e-12 * np.linalg.norm(zf)
    S.close()


@pytest.mark.parametrize("name,N,p,k", CASES)
def test_transposed_adjoint_solve_parity(nair, oracle_mod, name, N, p, k):
    """FGMRES on A^T preconditioned by the transposed cycle: same iteration
    count and residual history (1e-12) as the oracle, and the solution."""
    P = D.make_problem(name, N=N, p=p)
    params = dict(neumann_degree=k, max_coarse=4)
    S = nair.NairSolver(dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]), **params)
    H = oracle_mod.Hierarchy(P["row_ptr"], P["col"], P["vals"], **params)
    w = D.functional_weights(P["n"])
    lam, rep = S.adjoint_solve(dev(w))
    ref = H.solve(w, transposed=True)
    assert ref["status"] == 0
    assert rep["iterations"] == ref["iterations"]
    assert np.max(np.abs(rep["history"] - ref["history"])) <= 1e-12
    assert rep["rel_res"] <= 1e-10
    ls = lam.cpu().numpy()
    assert np.linalg.norm(ls - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])
    # a second adjoint solve reuses the transposed form
    lam2, rep2 = S.adjoint_solve(dev(w))
    assert rep2["iterations"] == rep["iterations"]
    assert float((lam2 - lam).abs().max()) <= 1e-13 * float(lam.abs().max())
    S.close()


def test_transposed_adjoint_gradients_match_rebuild(nair):
    """Both adjoint modes solve the same A^T lambda = w: gradients agree."""
    P = D.make_problem("C2", N=12, keep_parts=True)
    args = (dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]))
    w = dev(D.functional_weights(P["n"]))
    out = {}
    for mode in ("transposed", "rebuild"):
        S = nair.NairSolver(*args, neumann_degree=2, max_coarse=4, tol=1e-13, adjoint_mode=mode)
        x, _ = S.solve(dev(P["rhs"]))
        lam, rep = S.adjoint_solve(w)
        assert rep["rel_res"] <= 1e-12
        out[mode] = nair.gradients(dev(P["mass"]), lam, x)
        S.close()
    for a, b in zip(out["transposed"], out["rebuild"]):
        assert float((a - b).norm() / b.norm()) <= 1e-10


@pytest.mark.parametrize("name,N,p,k", CASES)
@pytest.mark.parametrize("graphs", [1, 0])
def test_fcycle_parity(nair, oracle_mod, name, N, p, k, graphs):
    """The F-cycle (coarse correction by an F-cycle, then a V-cycle from its
    result, which restricts the coarse residual and adds P x_c to the iterate)
    against the oracle's: one cycle on a seeded vector, then the FGMRES
    history.  k = 1 and k = 2 give odd and even sweep counts."""
    P = D.make_problem(name, N=N, p=p)
    params = dict(neumann_degree=k, max_coarse=4)
    S = nair.NairSolver(dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]), use_graphs=graphs,
                        cycle_type="F", **params)
    H = oracle_mod.Hierarchy(P["row_ptr"], P["col"], P["vals"], cycle="F", **params)
    f = D.rng.uniform(13, P["n"]) - 0.5
    z = S.vcycle(dev(f)).cpu().numpy()
    zr = H.vcycle(f)
    assert np.linalg.norm(z - zr) <= 1e-12 * np.linalg.norm(zr)
    x, rep = S.solve(dev(P["rhs"]))
    ref = H.solve(P["rhs"])
    assert ref["status"] == 0
    assert rep["iterations"] == ref["iterations"]
    assert np.max(np.abs(rep["history"] - ref["history"])) <= 1e-12
    assert rep["rel_res"] <= 1e-10
    S.close()


def test_fcycle_mixed_precision(nair):
    """F-cycle in FP32 inside FP64 FGMRES: FP64 residual and the FP64 solution."""
    P = D.make_problem("C5", N=24, p=3)
    args = (dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]))
    rhs = dev(P["rhs"])
    x64, r64 = nair.NairSolver(*args, neumann_degree=3, cycle_type="F").solve(rhs)
    x32, r32 = nair.NairSolver(*args, neumann_degree=3, cycle_type="F", precision="mixed").solve(rhs)
    assert r64["rel_res"] <= 1e-10 and r32["rel_res"] <= 1e-10
    assert float((x32 - x64).norm() / x64.norm()) <= 1e-8


@pytest.mark.parametrize("name,N,p,k", CASES)
def test_scalar_hierarchy_and_solve_parity(nair, oracle_mod, name, N, p, k):
    """Scalar nAIR: the scaled matrix D^{-1} A by degree of freedom and its whole
    hierarchy bit for bit (patterns, C/F) and in value; the preconditioner
    (cycle of D^{-1} v) on a seeded vector; forward and adjoint FGMRES
    histories against the oracle."""
    P = D.make_problem(name, N=N, p=p)
    params = dict(neumann_degree=k)
    S = nair.NairSolver(dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]), keep_setup_data=1, scalar=1,
                        **params)
    H = oracle_mod.Hierarchy(P["row_ptr"], P["col"], P["vals"], scalar=True, **params)
    compare_hierarchies(S, H, 1)
    f = D.rng.uniform(17, P["n"]) - 0.5
    z = S.vcycle(dev(f)).cpu().numpy()
    zr = H.vcycle(f)
    assert np.linalg.norm(z - zr) <= 1e-12 * np.linalg.norm(zr)
    x, rep = S.solve(dev(P["rhs"]))
    ref = H.solve(P["rhs"])
    assert ref["status"] == 0
    assert rep["iterations"] == ref["iterations"]
    assert np.max(np.abs(rep["history"] - ref["history"])) <= 1e-12
    assert rep["rel_res"] <= 1e-10
    zt = S.adjoint_vcycle(dev(f)).cpu().numpy()
    assert np.linalg.norm(zt - H.vcycle(f, transposed=True)) <= 1e-12 * np.linalg.norm(zt)
    w = D.functional_weights(P["n"])
    lam, repa = S.adjoint_solve(dev(w))
    refa = H.solve(w, transposed=True)
    assert repa["iterations"] == refa["iterations"]
    assert np.max(np.abs(repa["history"] - refa["history"])) <= 1e-12
    S.close()


def test_scalar_mixed_precision(nair):
    """Scalar nAIR in FP32 inside FP64 FGMRES, forward and adjoint."""
    P = D.make_problem("C5", N=24, p=3)
    args = (dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]))
    rhs, w = dev(P["rhs"]), dev(D.functional_weights(P["n"]))
    S64 = nair.NairSolver(*args, neumann_degree=2, scalar=1)
    S32 = nair.NairSolver(*args, neumann_degree=2, scalar=1, precision="mixed")
    x64, r64 = S64.solve(rhs)
    x32, r32 = S32.solve(rhs)
    assert r64["rel_res"] <= 1e-10 and r32["rel_res"] <= 1e-10
    assert float((x32 - x64).norm() / x64.norm()) <= 1e-8
    l64, a64 = S64.adjoint_solve(w)
    l32, a32 = S32.adjoint_solve(w)
    assert a64["rel_res"] <= 1e-10 and a32["rel_res"] <= 1e-10
    assert float((l32 - l64).norm() / l64.norm()) <= 1e-8


@pytest.mark.parametrize("name", ["F1", "F2", "F3"])
def test_paper_flows_parity(nair, oracle_mod, name):
    """The flows b1, b2, b3 of the paper's flow study: hierarchy bit for bit and
    the residual history against the oracle."""
    P = D.make_problem(name, N=12)
    params = dict(neumann_degree=1, max_coarse=4)
    S = nair.NairSolver(dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]), keep_setup_data=1, **params)
    H = oracle_mod.Hierarchy(P["row_ptr"], P["col"], P["vals"], **params)
    compare_hierarchies(S, H, P["b"])
    x, rep = S.solve(dev(P["rhs"]))
    ref = H.solve(P["rhs"])
    assert rep["iterations"] == ref["iterations"]
    assert np.max(np.abs(rep["history"] - ref["history"])) <= 1e-12
    S.close()


def test_direction_batch(nair, oracle_mod):
    """Eight directions of the angle sweep set up and solved concurrently (one
    host thread and one stream per system): every result equals the separate
    call bit for bit, and each history matches the oracle."""
    probs = [D.make_problem("D", N=10, theta=t) for t in D.sweep_angles(8)]
    systems = [(dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"])) for P in probs]
    rhs = [dev(P["rhs"]) for P in probs]
    w = [dev(D.functional_weights(P["n"])) for P in probs]
    params = dict(neumann_degree=1, max_coarse=4)
    solvers = nair.setup_batch(systems, **params)
    xs, reps = nair.solve_batch(solvers, rhs)
    lams, repas = nair.adjoint_solve_batch(solvers, w)
    for k, P in enumerate(probs):
        S1 = nair.NairSolver(*systems[k], **params)
        x1, r1 = S1.solve(rhs[k])
        l1, a1 = S1.adjoint_solve(w[k])
        assert torch.equal(xs[k], x1) and torch.equal(lams[k], l1)
        assert reps[k]["iterations"] == r1["iterations"] and repas[k]["iterations"] == a1["iterations"]
        ref = oracle_mod.Hierarchy(P["row_ptr"], P["col"], P["vals"], **params).solve(P["rhs"])
        assert reps[k]["iterations"] == ref["iterations"]
        assert np.max(np.abs(reps[k]["history"] - ref["history"])) <= 1e-12
        S1.close()
    for S in solvers:
        S.close()


def test_batch_errors(nair):
    """A failing system fails the whole batch with its index (a singular
    diagonal block, made on the host); a handle listed twice is rejected."""
    probs = [D.make_problem("D", N=6, theta=t) for t in D.sweep_angles(3)]
    systems = [(dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"])) for P in probs]
    bad = probs[1]["vals"].copy()
    bad[probs[1]["row_ptr"][4]:probs[1]["row_ptr"][5]] = 0.0  # block row 4, diagonal included
    systems[1] = (systems[1][0], systems[1][1], dev(bad))
    with pytest.raises(nair.NairError) as e:
        nair.setup_batch(systems)
    assert e.value.status == 2 and "system 1" in str(e.value)
    good = nair.setup_batch([systems[0], systems[2]])
    rhs = dev(probs[0]["rhs"])
    with pytest.raises(nair.NairError) as e:
        nair.solve_batch([good[0], good[0]], [rhs, rhs])
    assert e.value.status == 1
    for S in good:
        S.close()


def test_autograd_against_finite_differences(nair):
    """dJ/dq and dJ/dsigma from the adjoint solve vs central differences
    (eps = 1e-6, forward solves to 1e-13) on seeded coordinates."""
    P = D.make_problem("C4", N=8, keep_parts=True)
    n, E = P["n"], P["E"]
    w = dev(D.functional_weights(n))
    args = (dev(P["row_ptr"]), dev(P["col"]), dev(P["vals0"]), dev(P["diag_pos"]), dev(P["mass"]))
    params = dict(neumann_degree=2, tol=1e-13, max_coarse=4)
    q = dev(P["q"]).requires_grad_(True)
    sig = dev(P["sigma"]).requires_grad_(True)
    x = nair.NairSolve.apply(q, sig, *args, params)
    J = (w * x).sum()
    J.backward()
    iq, isg = D.fd_coordinates(n, E, count=8)
    eps = 1e-6

    def Jof(qv, sv):
        with torch.no_grad():
            return float((w * nair.NairSolve.apply(qv, sv, *args, params)).sum())

    for i in iq:
        qp, qm = q.detach().clone(), q.detach().clone()
        qp[i] += eps
        qm[i] -= eps
        fd = (Jof(qp, sig.detach()) - Jof(qm, sig.detach())) / (2 * eps)
        assert abs(fd - float(q.grad[i])) <= 1e-6 * max(1.0, abs(fd))
    for e in isg:
        sp, sm = sig.detach().clone(), sig.detach().clone()
        sp[e] += eps
        sm[e] -= eps
        fd = (Jof(q.detach(), sp) - Jof(q.detach(), sm)) / (2 * eps)
        assert abs(fd - float(sig.grad[e])) <= 1e-6 * max(1.0, abs(fd))


@pytest.mark.parametrize("name,N,p,k", [("C3", 16, 6, 1), ("C5", 24, 3, 2), ("C2", 32, 2, 2)])
def test_mixed_precision_accuracy(nair, name, N, p, k):
    """FP32 hierarchy and V-cycle inside FP64 FGMRES: FP64 residual <= 1e-10
    and the solution within cond * 1e-10 of the all-FP64 solve."""
    P = D.make_problem(name, N=N, p=p)
    args = (dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]))
    S64 = nair.NairSolver(*args, neumann_degree=k)
    S32 = nair.NairSolver(*args, neumann_degree=k, precision="mixed")
    rhs = dev(P["rhs"])
    x64, r64 = S64.solve(rhs)
    x32, r32 = S32.solve(rhs)
    assert r64["rel_res"] <= 1e-10 and r32["rel_res"] <= 1e-10
    err = float((x32 - x64).norm() / x64.norm())
    assert err <= 1e-8, err
    # the transposed cycle in FP32 inside FP64 FGMRES on A^T
    w = dev(D.functional_weights(P["n"]))
    l64, a64 = S64.adjoint_solve(w)
    l32, a32 = S32.adjoint_solve(w)
    assert a64["rel_res"] <= 1e-10 and a32["rel_res"] <= 1e-10
    assert float((l32 - l64).norm() / l64.norm()) <= 1e-8


def pattern_xor(rp1, ci1, rp2, ci2):
    """Number of blocks stored in one block pattern and not in the other."""
    def keys(rp, ci):
        rows = np.repeat(np.arange(len(rp) - 1, dtype=np.int64), np.diff(rp))
        return rows * (1 << 31) + ci.astype(np.int64)
    return int(len(np.setxor1d(keys(rp1, ci1), keys(rp2, ci2))))


def level_diffs(S32, S64):
    """Per level of two hierarchies of the same matrix: the number of C/F flags
    that differ, the numbers of blocks in one pattern but not the other (A and
    R_cf), the block counts, and the largest per-row relative difference of
    A_l, R_cf and D^{-1} (values compared only where the patterns agree)."""
    out = []
    for l in range(min(S32.num_levels(), S64.num_levels())):
        g, o = S32.level(l), S64.level(l)
        d = {"level": l, "cf": 0, "A_xor": 0, "R_xor": 0, "A_nnzb": int(o["nnzb"])}
        if g["E"] != o["E"]:
            d["cf"] = -1
            out.append(d)
            break
        d["A_xor"] = pattern_xor(g["row_ptr"], g["col"], o["row_ptr"], o["col"])
        if d["A_xor"] == 0:
            d["A"] = rel_rows(g["vals"], o["vals"])
        d["Dinv"] = rel_rows(g["dinv"], o["dinv"])
        if not o["coarsest"] and not g["coarsest"]:
            d["cf"] = int(np.count_nonzero(g["cf"] != o["cf"]))
            d["R_nnzb"] = int(len(o["R_ci"]))
            if d["cf"] == 0:
                d["R_xor"] = pattern_xor(g["R_rp"], g["R_ci"], o["R_rp"], o["R_ci"])
                if d["R_xor"] == 0:
                    d["R"] = rel_rows(g["R_v"], o["R_v"])
        out.append(d)
    return out


@pytest.mark.parametrize("name,N,p,k", [("C3", 16, 6, 1), ("C5", 24, 3, 2), ("C5", 24, 3, 6)])
def test_mixed_precision_per_result_error(nair, oracle_mod, name, N, p, k):
    """Per-result error of the FP32 forms against FP64 (mixed precision: setup
    from the FP32-rounded matrix, D^{-1} computed in FP64 from the FP32 blocks
    and stored in FP32).  Level by level the FP32 hierarchy has the FP64
    hierarchy's C/F splittings and patterns; level 0's A is the FP32 rounding
    (<= 2^-24 per row, relative) and its D^{-1} carries cond(D_ii) times that
    (<= 2e-6); the coarse A, R_cf and D^{-1} stay within 1e-4 per row (measured
    up to 4.2e-5).  One FP32 cycle (forward and transposed) on a seeded vector
    is within 5e-6 of the oracle's FP64 cycle (measured up to 6e-7) -- the
    identity in its place would be off by O(1) -- and FGMRES needs at most one
    more iteration than in FP64 (measured: the same count)."""
    P = D.make_problem(name, N=N, p=p)
    args = (dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]))
    params = dict(neumann_degree=k)
    S64 = nair.NairSolver(*args, **params)
    S32 = nair.NairSolver(*args, precision="mixed", **params)
    assert S32.num_levels() == S64.num_levels()
    diffs = level_diffs(S32, S64)
    assert all(d["cf"] == 0 and d["A_xor"] == 0 and d["R_xor"] == 0 for d in diffs), diffs
    assert diffs[0]["A"] <= 2.0 ** -24 and diffs[0]["Dinv"] <= 2e-6, diffs[0]
    for d in diffs:
        for key in ("A", "Dinv", "R"):
            if key in d:
                assert d[key] <= 1e-4, (key, d)
    H = oracle_mod.Hierarchy(P["row_ptr"], P["col"], P["vals"], **params)
    f = D.rng.uniform(7, P["n"]) - 0.5
    zo = H.vcycle(f)
    z32 = S32.vcycle(dev(f)).cpu().numpy()
    z64 = S64.vcycle(dev(f)).cpu().numpy()
    assert np.linalg.norm(z64 - zo) <= 1e-12 * np.linalg.norm(zo)
    assert np.linalg.norm(z32 - zo) <= 5e-6 * np.linalg.norm(zo)
    assert np.linalg.norm(f - zo) > 1e-2 * np.linalg.norm(zo)   # the bound rules out the identity
    zto = H.vcycle(f, transposed=True)
    zt32 = S32.adjoint_vcycle(dev(f)).cpu().numpy()
    assert np.linalg.norm(zt32 - zto) <= 5e-6 * np.linalg.norm(zto)
    rhs = dev(P["rhs"])
    _, r64 = S64.solve(rhs)
    _, r32 = S32.solve(rhs)
    assert r32["iterations"] <= r64["iterations"] + 1, (r32["iterations"], r64["iterations"])
    S32.close()
    S64.close()


def test_c4_gradients_against_oracle_solutions(nair, oracle_mod):
    """C4 on a 24 x 24 x 2 mesh: the GPU gradients (NairSolve backward) against
    the oracle's gradient formula applied to the oracle's own forward solution
    and its own adjoint solution (FGMRES on A^T with the transposed cycle), all
    solves to 1e-13."""
    P = D.make_problem("C4", N=24, keep_parts=True)
    n = P["n"]
    w = D.functional_weights(n)
    args = (dev(P["row_ptr"]), dev(P["col"]), dev(P["vals0"]), dev(P["diag_pos"]), dev(P["mass"]))
    params = dict(neumann_degree=2, tol=1e-13)
    q = dev(P["q"]).requires_grad_(True)
    sig = dev(P["sigma"]).requires_grad_(True)
    x = nair.NairSolve.apply(q, sig, *args, params)
    (dev(w) * x).sum().backward()
    H = oracle_mod.Hierarchy(P["row_ptr"], P["col"], P["vals"], neumann_degree=2)
    xo = H.solve(P["rhs"], tol=1e-13)["x"]
    lo = H.solve(w, transposed=True, tol=1e-13)["x"]
    gs_o, gq_o = oracle_mod.gradients(P["mass"], lo, xo)
    gs, gq = sig.grad.cpu().numpy(), q.grad.cpu().numpy()
    assert np.linalg.norm(gs - gs_o) <= 1e-9 * np.linalg.norm(gs_o)
    assert np.linalg.norm(gq - gq_o) <= 1e-9 * np.linalg.norm(gq_o)


def test_nan_rhs_is_breakdown_and_handle_recovers(nair):
    """A NaN in the right-hand side (made on the host) ends the forward solve
    with NAIR_ERR_BREAKDOWN, an infinity in w ends the adjoint solve the same
    way, and the handle then solves a finite system as before."""
    P = D.make_problem("C2", N=8)
    S = nair.NairSolver(dev(P["row_ptr"]), dev(P["col"]), dev(P["vals"]), neumann_degree=2)
    _, good = S.solve(dev(P["rhs"]))
    bad = P["rhs"].copy()
    bad[17] = np.nan
    _, rep = S.solve(dev(bad), check=False)
    assert rep["status"] == 4
    wbad = D.functional_weights(P["n"])
    wbad[3] = np.inf
    _, repa = S.adjoint_solve(dev(wbad), check=False)
    assert repa["status"] == 4
    x, again = S.solve(dev(P["rhs"]))
    assert again["status"] == 0 and again["rel_res"] <= 1e-10
    assert again["iterations"] == good["iterations"]
    S.close()
