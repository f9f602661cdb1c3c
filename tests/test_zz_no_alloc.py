"""lbm_field_sums_noalloc: the diagnostics sums for callers that cannot allocate device
memory (for instance a host that owns all device memory through its own arena or pool, or
a service whose device memory is fixed when it starts).  The entry point takes caller-owned device fields and a
caller-owned device result and keeps its block partial sums in a fixed-size array in the
library's device image, so it never calls an allocator.

The test calls it through the C ABI twice in a row, on two different states, and checks
each result against lbm_get_diagnostics of the same state (same sums, same block order,
so they agree to round-off; the bar is the 1e-10 of the parity tests).  This file is
collected last so that a failure here leaves every other test already run."""
import ctypes

import numpy as np
import pytest

from paper_2603_22902_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for the gpu tests")
    from paper_2603_22902_gb300 import build as B
    B.build()
    from paper_2603_22902_gb300 import lbm as L
    lib = L.library()
    lib.lbm_field_sums_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.lbm_field_sums_noalloc.restype = ctypes.c_int
    return L


def test_noalloc_sums_match_diagnostics_on_two_calls(lbm):
    import torch
    lib = lbm.library()
    case = W.sessile_drop(n=96, R=28.0, ny=80, theta=70.0)
    N = case.N
    s = lbm.Solver(case).set_fields()
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.full((2 * N + 2,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        s.step(150)
        F = s.fields()
        rc = lib.lbm_field_sums_noalloc(F["phi"].data_ptr(), F["fl"].data_ptr(), case.nx, case.ny, N,
                                        out.data_ptr(), stream)
        assert rc == lbm.LBM_OK, lib.lbm_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        d = s.diagnostics()
        for p in range(N):
            assert abs(got[p] - d["mass"][p]) <= 1e-10 * max(1.0, abs(d["mass"][p])), (call, p)
            assert abs(got[N + p] - d["solid"][p]) <= 1e-10 * max(1.0, abs(d["solid"][p])), (call, p)
        assert abs(got[2 * N] - d["max_sum_dev"]) <= 1e-10
        assert got[2 * N + 1] == 0.0 and d["nonfinite"] == 0
        assert d["solid"][0] > 0.0 or call == 0   # the state changes between the calls
    s.close()


def test_noalloc_rejects_sizes_beyond_its_limits(lbm):
    import torch
    lib = lbm.library()
    a = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = lib.lbm_field_sums_noalloc(a.data_ptr(), a.data_ptr(), 2, 2, 5, a.data_ptr(), None)
    assert rc == lbm.LBM_EINVAL
    assert b"LBM_MAXN" in lib.lbm_last_error(None)
    rc = lib.lbm_field_sums_noalloc(a.data_ptr(), a.data_ptr(), 1 << 16, 1 << 16, 2, a.data_ptr(), None)
    assert rc == lbm.LBM_EINVAL
    assert b"2^31" in lib.lbm_last_error(None)


def test_noalloc_sums_on_a_lattice_beyond_one_row_per_block(lbm):
    # 512 x 512 = 262 144 cells: more than 608 blocks x 256 threads, so the grid-stride
    # loop folds several cells into each of the fixed 608 scratch rows
    import torch
    lib = lbm.library()
    case = W.sessile_drop()
    N = case.N
    assert case.nx * case.ny > 608 * 256
    s = lbm.Solver(case).set_fields()
    s.step(40)
    F = s.fields()
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.full((2 * N + 2,), float("nan"), dtype=torch.float64, device="cuda")
    rc = lib.lbm_field_sums_noalloc(F["phi"].data_ptr(), F["fl"].data_ptr(), case.nx, case.ny, N,
                                    out.data_ptr(), stream)
    assert rc == lbm.LBM_OK, lib.lbm_last_error(None)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    d = s.diagnostics()
    for p in range(N):
        assert abs(got[p] - d["mass"][p]) <= 1e-10 * abs(d["mass"][p]), p
        assert abs(got[N + p] - d["solid"][p]) <= 1e-10 * max(1.0, abs(d["solid"][p])), p
    assert abs(got[2 * N] - d["max_sum_dev"]) <= 1e-10
    assert got[2 * N + 1] == 0.0
    s.close()


def test_noalloc_counts_a_nonfinite_cell_of_its_inputs(lbm):
    import torch
    lib = lbm.library()
    case = W.sessile_drop(n=96, R=28.0, ny=80, theta=70.0)
    N = case.N
    s = lbm.Solver(case).set_fields()
    s.step(20)
    F = s.fields()
    phi = F["phi"].clone()
    phi[1, 33, 47] = float("nan")
    out = torch.zeros(2 * N + 2, dtype=torch.float64, device="cuda")
    rc = lib.lbm_field_sums_noalloc(phi.data_ptr(), F["fl"].data_ptr(), case.nx, case.ny, N, out.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert rc == lbm.LBM_OK, lib.lbm_last_error(None)
    torch.cuda.synchronize()
    assert out[2 * N + 1].item() == 1.0
    s.close()
