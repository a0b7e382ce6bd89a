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
