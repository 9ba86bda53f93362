"""The allocation-free error pass, id_reconstruct_error_noalloc, against the
regular id_reconstruct_error.

The no-allocation entry point exists for callers that must not allocate device
memory: their own allocator already holds the GPU's memory, they run to a fixed
memory budget, or they cannot accept the device-wide synchronisation of
cudaMalloc/cudaFree.  It keeps its scratch in a fixed device array that all
calls share.  These tests call it twice in a row through the C ABI.  The
second call gets new inputs, so a stale value left by the first call would
show.  Each result must match the regular entry point within the tolerance of
the error-pass parity tests.  This file is collected last on purpose, so that
a run which stops at the first failure has already run every other test.
"""
import ctypes as C

import pytest
import torch

from synthetic import gaussian_matrix, low_rank_matrix

pytestmark = pytest.mark.gpu


def _noalloc(lib, A, J, P, k, dtype_code):
    fro, mx = C.c_double(-1.0), C.c_double(-1.0)
    st = lib.id_reconstruct_error_noalloc(
        C.c_void_p(A.data_ptr()), A.stride(1), A.shape[0], A.shape[1], dtype_code,
        C.c_void_p(J.data_ptr()), C.c_void_p(P.data_ptr()), k, C.byref(fro), C.byref(mx),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, fro.value, mx.value


@pytest.mark.parametrize("dtype,code,etol", [(torch.float32, 0, 1e-4), (torch.float64, 1, 1e-10)])
def test_noalloc_matches_regular_entry_on_two_calls(dtype, code, etol):
    from paper_1905_13257_gb300 import IdSketch, load
    lib = load()
    cases = []
    # m >= 128 takes the tensor-core error pass for FP32 data, m < 128 the
    # plain one; both run twice in a row
    for seed, (m, n, k) in enumerate([(5000, 300, 24), (3001, 120, 7), (100, 40, 5)]):
        A = gaussian_matrix(m, n, seed=seed + 10, dtype=dtype, device="cuda")
        A = A + 5 * low_rank_matrix(m, n, 3, seed=seed, dtype=dtype, device="cuda")
        g = torch.Generator().manual_seed(seed)
        J = torch.randperm(n, generator=g)[:k].to(torch.int32)
        P = torch.randn((k, n), generator=g, dtype=torch.float64) * 0.2
        cases.append((A, J, P, k))
    for A, J, P, k in cases:                       # two calls in a row
        m, n = A.shape
        st, fro, mx = _noalloc(lib, A, J.cuda(), P.cuda(), k, code)
        assert st == 0
        sk = IdSketch(m, n, k, max(k, 8), seed=0, dtype=dtype)
        fro_ref, mx_ref = sk.reconstruct_error(A, J, P)
        sk.close()
        assert abs(fro - fro_ref) <= etol * fro_ref
        assert abs(mx - mx_ref) <= etol * mx_ref


def test_noalloc_rejects_p_beyond_capacity():
    from paper_1905_13257_gb300 import _binding as B
    lib = B.load()
    n, k = B.ID_NOALLOC_MAX_KN // 8 + 1, 8         # k * n just above the capacity
    A = torch.zeros((n, 16), dtype=torch.float32, device="cuda").T
    J = torch.arange(k, dtype=torch.int32, device="cuda")
    P = torch.zeros((k, n), dtype=torch.float64, device="cuda")
    st, fro, mx = _noalloc(lib, A, J, P, k, 0)
    assert st == B.ID_ERR_INVALID_ARG


@pytest.mark.parametrize("dtype,code,etol", [(torch.float32, 0, 1e-4), (torch.float64, 1, 1e-10)])
def test_noalloc_at_the_capacity_limit(dtype, code, etol):
    """k * n exactly ID_NOALLOC_MAX_KN: accepted, and equal to the regular
    entry point's result."""
    from paper_1905_13257_gb300 import IdSketch
    from paper_1905_13257_gb300 import _binding as B
    lib = B.load()
    k = 8
    n = B.ID_NOALLOC_MAX_KN // k
    m = 300
    A = gaussian_matrix(m, n, seed=5, dtype=dtype, device="cuda")
    A = A + 3 * low_rank_matrix(m, n, 4, seed=6, dtype=dtype, device="cuda")
    g = torch.Generator().manual_seed(7)
    J = torch.randperm(n, generator=g)[:k].to(torch.int32)
    P = torch.randn((k, n), generator=g, dtype=torch.float64) * 0.2
    st, fro, mx = _noalloc(lib, A, J.cuda(), P.cuda(), k, code)
    assert st == 0
    sk = IdSketch(m, n, k, k, seed=0, dtype=dtype)
    fro_ref, mx_ref = sk.reconstruct_error(A, J, P)
    sk.close()
    assert abs(fro - fro_ref) <= etol * fro_ref
    assert abs(mx - mx_ref) <= etol * mx_ref
