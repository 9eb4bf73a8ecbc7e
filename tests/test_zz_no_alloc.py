"""msf_cfl_dt_noalloc: the CFL time step computed with no device allocation.

It is meant for callers that cannot call cudaMalloc (a caching allocator that
owns the device memory, real-time loops that must avoid the implicit device
synchronisation of an allocation, fixed memory budgets). Its answer must match
the time step msf_step takes from the same state, on two calls in a row: the
second call reuses the scratch array the first one left behind. A call after a
larger one must ignore the partial maxima the larger call left beyond its own
blocks, and a non-physical cell must give NaN, never a finite step.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import paper_1704_00519_gb300.cases as cs

pytestmark = pytest.mark.gpu

MAX_CELLS = 4194304


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00519_gb300 import build
    build.build()
    import paper_1704_00519_gb300.msf as msf
    return msf, torch


def _single_material(shape, seed, speed=0.4, peak_at_end=False):
    """One stiffened gas on a box with h = 1/64 along every axis, smooth random
    density and pressure, velocity of size `speed`; with peak_at_end the
    largest wave speed sits in the last cell, which the last partial maximum
    holds."""
    dim = len(shape)
    rng = np.random.default_rng(seed)
    cells = int(np.prod(shape))
    hi = tuple(n / 64.0 for n in shape)
    rho = 1.0 + 0.3 * rng.random(cells)
    p = 1.0 + 0.2 * rng.random(cells)
    vel = speed * (2.0 * rng.random((dim, cells)) - 1.0)
    if peak_at_end:
        vel[:, -1] = 3.0 * speed
    prim = np.concatenate([rho[None], vel, p[None]])[None]
    bc = [[0, 0]] * dim
    return cs.Case("single", dim, tuple(shape), (0.0,) * dim, hi, bc, [1.4], [0.3],
                   np.full(cells, 10.0), np.zeros(cells, np.int32), prim, 10.0)


def _noalloc_dt(msf, torch, case, Q):
    dt_dev = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    eos = msf.msf_eos(case.gamma[0], case.pinf[0])
    h = (C.c_double * case.dim)(*[(case.hi[d] - case.lo[d]) / case.n[d] for d in range(case.dim)])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = msf.msf_cfl_dt_noalloc(C.c_void_p(Q.data_ptr()), case.cells, case.dim, C.byref(eos), h, 0.6,
                                C.c_void_p(dt_dev.data_ptr()), stream)
    assert st == msf.MSF_OK, msf.msf_last_error(None)
    torch.cuda.synchronize()
    return dt_dev.item()


def _dt_pair(msf, torch, case):
    """(no-allocation dt, dt msf_step takes) from the same initial state."""
    s = msf.Solver(case)
    Q = torch.empty((1, case.nv, case.cells), dtype=torch.float64, device="cuda")
    s.get_state_device(Q)
    dt = _noalloc_dt(msf, torch, case, Q)
    s.step(1)
    ref = s.last_dt()
    s.close()
    return dt, ref


def _smooth_single_material(nx=96, ny=64):
    x, y = cs.centres((nx, ny), (0.0, 0.0), (1.5, 1.0))
    rho = 1.0 + 0.3 * np.exp(-((x - 0.6) ** 2 + (y - 0.5) ** 2) / 0.02)
    prim = np.stack([rho.ravel(), np.full(nx * ny, 0.4), np.full(nx * ny, -0.2),
                     (1.0 + 0.1 * np.sin(3 * x) * np.cos(2 * y)).ravel()])[None]
    return cs.Case("smooth", 2, (nx, ny), (0.0, 0.0), (1.5, 1.0), [[0, 0], [1, 1]], [1.4], [0.3],
                   np.full((ny, nx), 10.0), np.zeros((ny, nx), np.int32), prim, 10.0)


def test_noalloc_cfl_matches_step_dt(env):
    msf, torch = env
    case = _smooth_single_material()
    s = msf.Solver(case)
    Q = torch.empty((1, case.nv, case.cells), dtype=torch.float64, device="cuda")
    for _ in range(2):
        s.get_state_device(Q)
        dt = _noalloc_dt(msf, torch, case, Q)
        s.step(1)  # the library's own step takes its time step from the same state
        assert dt == pytest.approx(s.last_dt(), rel=1e-12, abs=0.0)


@pytest.mark.parametrize("shapes", [
    [(MAX_CELLS,), (MAX_CELLS - 1,), (257,)],
    [(2048, 2048), (257, 1)],
    [(256, 128, 128), (7, 6, 5)],
], ids=["1d", "2d", "3d"])
def test_noalloc_cfl_sizes_large_then_small(env, shapes):
    """Exactly MSF_NOALLOC_MAX_CELLS cells (16384 partial maxima, the final
    kernel's strided loop at full length), one cell fewer (a partial last
    block) and then a small state whose wave speeds are all below the large
    states': each dt equals msf_step's, so the small call read none of the
    larger calls' leftover partials."""
    msf, torch = env
    for k, shape in enumerate(shapes):
        large = int(np.prod(shape)) > 1000
        case = _single_material(shape, seed=k, speed=2.0 if large else 0.1, peak_at_end=large)
        dt, ref = _dt_pair(msf, torch, case)
        assert dt == pytest.approx(ref, rel=1e-12, abs=0.0), (shape, dt, ref)


@pytest.mark.parametrize("bad", ["negative_pressure", "zero_density"])
def test_noalloc_cfl_reports_a_non_physical_cell_as_nan(env, bad):
    """A cell with p + pinf < 0, or an empty cell (rho = 0), makes msf_step
    refuse the state with a device-detected error; the no-allocation bound
    must not drop that cell: dt is NaN."""
    msf, torch = env
    case = _single_material((40, 30), seed=5)
    s = msf.Solver(case)
    Q = torch.empty((1, case.nv, case.cells), dtype=torch.float64, device="cuda")
    s.get_state_device(Q)
    c = 617
    if bad == "negative_pressure":
        rho = Q[0, 0, c].item()
        ke = 0.5 * (Q[0, 1, c].item() ** 2 + Q[0, 2, c].item() ** 2) / rho
        Q[0, 3, c] = ke + (-1.0 + 1.4 * 0.3) / 0.4  # p = -1 < -pinf
    else:
        Q[0, :, c] = 0.0
    dt = _noalloc_dt(msf, torch, case, Q)
    assert np.isnan(dt)
    s.set_conserved(Q)
    with pytest.raises(msf.MsfError) as ei:
        s.step(1)
    assert ei.value.status in (msf.MSF_ENEGATIVE, msf.MSF_ENONFINITE, msf.MSF_EBAND)
    s.close()


def test_noalloc_cfl_rejects_oversized_state(env):
    msf, torch = env
    eos = msf.msf_eos(1.4, 0.0)
    h = (C.c_double * 1)(0.01)
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = msf.msf_cfl_dt_noalloc(C.c_void_p(dummy.data_ptr()), MAX_CELLS + 1, 1, C.byref(eos), h, 0.6,
                                C.c_void_p(dummy.data_ptr()), None)
    assert st == msf.MSF_EINVAL
    assert b"MSF_NOALLOC_MAX_CELLS" in msf.msf_last_error(None)
