"""The benchmark's algorithmic-work accounting of the block-Jacobi sweeps, on
CPU: `bench.level_work` reads a hierarchy's exported levels, so an oracle
hierarchy (same export layout as the GPU solver's) stands in for the GPU one.
The counts are checked against sums written out here from the level arrays."""
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


def test_level_work_counts(hier):
    P, H = hier
    b = P["b"]
    work = bench.level_work(H, H.nlev, b)
    assert H.nlev >= 3
    for l in range(H.nlev):
        lev = H.level(l)
        if lev["coarsest"]:
            assert f"jacobi_F@L{l}" not in work
            continue
        rows = np.repeat(np.arange(lev["E"]), np.diff(lev["row_ptr"]))
        off = lev["col"] != rows
        for cls, name in ((0, "F"), (1, "C")):
            sel = (lev["cf"][rows] == cls) & off
            nrow = int(np.count_nonzero(lev["cf"] == cls))
            flops, byts = work[f"jacobi_{name}@L{l}"]
            if l == 0:  # scaled, column-compressed couplings: b * W FMAs per block, no D^-1
                W = P["p"] + 1
                assert flops == 2.0 * int(sel.sum()) * b * W
            else:       # classical form: exact off-diagonal nonzeros plus b^2 per row for D^-1
                nnz = int(np.count_nonzero(lev["vals"][sel].reshape(int(sel.sum()), -1)))
                assert flops == 2.0 * (nnz + nrow * b * b)
            assert byts > 0 and byts >= 16.0 * lev["E"] * b


def test_hbm_peak_falls_back_without_measurement(monkeypatch, tmp_path):
    peak, src = bench.hbm_peak_gbs()
    assert peak > 1000.0 and src in ("measured", "fallback")
    monkeypatch.setattr(bench.os.path, "abspath", lambda p: str(tmp_path / "bench.py"))
    assert bench.hbm_peak_gbs() == (6800.0, "fallback")
