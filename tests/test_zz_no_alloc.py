"""The allocation-free block inverse against the allocating one.

nair_block_inverse_noalloc serves callers that cannot allocate device memory:
applications whose caching allocator owns the whole GPU, or that forbid
cudaMalloc after start-up.  It keeps its status words in a fixed array inside
the library's device memory instead.  This file runs last so that, if it
fails, a run that stops at the first failure has already run every other
test.  Its output must equal nair_block_inverse's bit for bit (the tolerance
of the block-inverse parity tests), on two calls in a row that share the
static scratch.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1704_05001_gb300 as nair
    return nair


def _call(nair, fn, A):
    out = torch.empty_like(A)
    st = getattr(nair.lib(), fn)(A.shape[0], A.shape[-1], ctypes.c_void_p(A.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, out


@pytest.mark.parametrize("b", [3, 6, 28])
def test_noalloc_matches_allocating_entry_point_twice(lib, b):
    r = np.random.default_rng(2024 + b)
    for call in range(2):   # two calls in a row share the static scratch
        nblk = 1000 + 37 * call
        A = torch.from_numpy(r.standard_normal((nblk, b, b)) + (0.5 * b) * np.eye(b)).cuda()
        st0, ref = _call(lib, "nair_block_inverse", A)
        st1, got = _call(lib, "nair_block_inverse_noalloc", A)
        assert st0 == 0 and st1 == 0, lib.lib().nair_last_error()
        assert torch.equal(got, ref)


@pytest.mark.parametrize("b", [3, 6, 10, 28, 32])
def test_noalloc_matches_on_pivot_ties_and_signed_zeros(lib, b):
    """Small-integer blocks with signed zeros: equal |entries| in a pivot column,
    zero diagonals that force row exchanges, and -0.0 against +0.0.  The two
    kernels pick pivots and exchange rows in different ways, so these are the
    inputs where they could part; they must still agree bit for bit, and on
    which calls report a zero pivot."""
    r = np.random.default_rng(300 + b)
    A = r.integers(-2, 3, size=(400, b, b)).astype(np.float64)
    A[r.random(A.shape) < 0.2] = -0.0
    A[::7, np.arange(b), np.arange(b)] = 0.0   # zero diagonals on every seventh block
    good = []
    for k in range(len(A)):
        st, _ = _call(lib, "nair_block_inverse", torch.from_numpy(A[k:k + 1]).cuda())
        if st == 0:
            good.append(k)
    assert len(good) > 100
    X = torch.from_numpy(A[good]).cuda()
    for _ in range(2):
        st0, ref = _call(lib, "nair_block_inverse", X)
        st1, got = _call(lib, "nair_block_inverse_noalloc", X)
        assert st0 == 0 and st1 == 0, lib.lib().nair_last_error()
        assert torch.equal(got.view(torch.int64), ref.view(torch.int64))


@pytest.mark.parametrize("b", [3, 6, 28, 32])
def test_noalloc_singular_and_nan_blocks_match_status(lib, b):
    """All-ones blocks (rank one) and blocks holding a NaN: both entry points
    report SINGULAR_BLOCK; one regular block alone gives OK from both."""
    for fill in (1.0, float("nan")):
        A = np.ones((40, b, b)) if fill == 1.0 else np.eye(b)[None].repeat(40, axis=0) * 2.0
        if fill != 1.0:
            A[17, b // 2, b // 2] = fill
        X = torch.from_numpy(A).cuda()
        st0, _ = _call(lib, "nair_block_inverse", X)
        st1, _ = _call(lib, "nair_block_inverse_noalloc", X)
        assert st0 == 2 and st1 == 2
    X = torch.from_numpy(np.eye(b)[None] * 3.0).cuda()
    st0, ref = _call(lib, "nair_block_inverse", X)
    st1, got = _call(lib, "nair_block_inverse_noalloc", X)
    assert st0 == 0 and st1 == 0
    assert torch.equal(got, ref)


def test_noalloc_reports_singular_then_recovers(lib):
    r = np.random.default_rng(7)
    A = r.standard_normal((500, 6, 6)) + 3 * np.eye(6)
    A[321] = 1.0   # rank one
    st, _ = _call(lib, "nair_block_inverse_noalloc", torch.from_numpy(A).cuda())
    assert st == 2
    A[321] = np.eye(6)
    st, got = _call(lib, "nair_block_inverse_noalloc", torch.from_numpy(A).cuda())
    assert st == 0
    _, ref = _call(lib, "nair_block_inverse", torch.from_numpy(A).cuda())
    assert torch.equal(got, ref)


def test_noalloc_rejects_calls_beyond_its_scratch(lib):
    b = 28
    too_many = 8192 * (256 // b) + 1
    A = torch.zeros((1, b, b), dtype=torch.float64, device="cuda")
    st = lib.lib().nair_block_inverse_noalloc(too_many, b, ctypes.c_void_p(A.data_ptr()),
                                             ctypes.c_void_p(A.data_ptr()), None)
    assert st == 1
    assert b"static scratch" in lib.lib().nair_last_error()
