"""msf_cfl_dt_noalloc: the CFL time step computed with no device allocation.

It is meant for callers that cannot call cudaMalloc (a caching allocator that
owns the device memory, real-time loops that must avoid the implicit device
synchronisation of an allocation, fixed memory budgets). Its answer must match
the time step msf_step takes from the same state, on two calls in a row: the
second call reuses the scratch array the first one left behind.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import paper_1704_00519_gb300.cases as cs

pytestmark = pytest.mark.gpu


def _smooth_single_material(nx=96, ny=64):
    x, y = cs.centres((nx, ny), (0.0, 0.0), (1.5, 1.0))
    rho = 1.0 + 0.3 * np.exp(-((x - 0.6) ** 2 + (y - 0.5) ** 2) / 0.02)
    prim = np.stack([rho.ravel(), np.full(nx * ny, 0.4), np.full(nx * ny, -0.2),
                     (1.0 + 0.1 * np.sin(3 * x) * np.cos(2 * y)).ravel()])[None]
    return cs.Case("smooth", 2, (nx, ny), (0.0, 0.0), (1.5, 1.0), [[0, 0], [1, 1]], [1.4], [0.3],
                   np.full((ny, nx), 10.0), np.zeros((ny, nx), np.int32), prim, 10.0)


def test_noalloc_cfl_matches_step_dt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00519_gb300 import build
    build.build()
    import paper_1704_00519_gb300.msf as msf
    case = _smooth_single_material()
    s = msf.Solver(case)
    cells = case.cells
    Q = torch.empty((1, case.nv, cells), dtype=torch.float64, device="cuda")
    dt_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    eos = msf.msf_eos(case.gamma[0], case.pinf[0])
    h = (C.c_double * 2)(1.5 / case.n[0], 1.0 / case.n[1])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        s.get_state_device(Q)
        dt_dev.zero_()
        st = msf.msf_cfl_dt_noalloc(C.c_void_p(Q.data_ptr()), cells, 2, C.byref(eos), h, 0.6,
                                    C.c_void_p(dt_dev.data_ptr()), stream)
        assert st == msf.MSF_OK, msf.msf_last_error(None)
        torch.cuda.synchronize()
        s.step(1)  # the library's own step takes its time step from the same state
        ref = s.last_dt()
        assert dt_dev.item() == pytest.approx(ref, rel=1e-12, abs=0.0)


def test_noalloc_cfl_rejects_oversized_state():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1704_00519_gb300.msf as msf
    eos = msf.msf_eos(1.4, 0.0)
    h = (C.c_double * 1)(0.01)
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = msf.msf_cfl_dt_noalloc(C.c_void_p(dummy.data_ptr()), 4194304 + 1, 1, C.byref(eos), h, 0.6,
                                C.c_void_p(dummy.data_ptr()), None)
    assert st == msf.MSF_EINVAL
    assert b"MSF_NOALLOC_MAX_CELLS" in msf.msf_last_error(None)
