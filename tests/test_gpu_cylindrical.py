"""GPU path of the axisymmetric grid and the free-surface ambient (Case II,
Sec. 3.2) against the oracle: the FP64 build matches it bit for bit, the
FP32-bulk form within the FP32 tolerance; r-weighted conservation on the
device; the entry points that do not take such grids refuse them."""
import numpy as np
import pytest

import paper_1704_00519_gb300.cases as cs
from oracle import oracle as orc
from test_gpu_parity import FP32_L1, FP64_L1, compare, run_pair
from test_oracle_cylindrical import _layers, _prim_1d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def msf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00519_gb300 import build
    build.build()
    import paper_1704_00519_gb300.msf as m
    return m


def _rest_case(held):
    n, p0 = 120, 0.7
    x, phi, chi = _layers(n, [0.3137, 0.6521, 0.8713])
    states = [(0.2, 0, p0), (1.0, 0, p0), (0.5, 0, p0), (1.0, 0, p0)]
    fs = (3, 1.0, p0, 0.1, 0.2, p0) if held else None
    return cs.Case("cyl_rest", 1, (n,), (0.0,), (1.0,), [[cs.REFLECTIVE, cs.TRANSMISSIVE]],
                   [1.4, 1.667, 3.0, 1.4], [0.0, 0.2, 0.5, 0.0], phi, chi, _prim_1d(states, n), 1.0,
                   geom=1, free_surface=fs)


def _tube_case(n=160):
    x, phi, chi = _layers(n, [0.35, 0.55])
    states = [(1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (0.8, 0.3, 0.6)]
    return cs.Case("cyl_tube", 1, (n,), (0.0,), (1.0,), [[cs.REFLECTIVE, cs.TRANSMISSIVE]],
                   [1.4, 1.667, 1.4], [0.0, 0.0, 0.0], phi, chi, _prim_1d(states, n), 0.25, geom=1)


@pytest.mark.parametrize("held", [False, True])
def test_cylindrical_rest_fp64(msf, held):
    o, s, eo = run_pair(msf, _rest_case(held), 40, t_end=1.0)
    assert eo == 0
    compare(o, s, FP64_L1, exact=True)


def test_cylindrical_tube_fp64(msf):
    o, s, eo = run_pair(msf, _tube_case(), 120)
    assert eo == 0
    compare(o, s, FP64_L1, exact=True)


def test_cylindrical_tube_conservation_on_device(msf):
    """Device totals (r-weighted) and ledger: per-material mass and the summed
    energy change only through the boundary."""
    case = _tube_case()
    s = msf.Solver(case)
    tot0, _ = s.totals()
    s.step(120, case.t_end)
    tot, led = s.totals()
    assert s.counters()["merge"] == 0
    scale = np.abs(tot0).sum()
    assert np.abs(tot[:, 0] - tot0[:, 0] - led[:, 0]).max() / scale < 1e-13
    assert abs((tot[:, 2] - tot0[:, 2] - led[:, 2]).sum()) / scale < 1e-13


@pytest.mark.parametrize("n,steps", [(160, 300), (320, 200)])
def test_icf_fp64(msf, n, steps):
    o, s, eo = run_pair(msf, cs.icf_implosion(n), steps)
    assert eo == 0
    compare(o, s, FP64_L1, exact=True)


def test_icf_full_run_fp64(msf):
    """Case II to t = 0.3 (past stagnation) at 640 cells: bit-identical to the
    oracle, core and shell masses conserved."""
    case = cs.icf_implosion(640)
    o, s, eo = run_pair(msf, case, 100000)
    assert eo == 0
    compare(o, s, FP64_L1, exact=True)
    assert s.state()["t"] == case.t_end
    tot, led = s.totals()
    o0 = orc.Oracle(case)
    tot0, _ = o0.totals()
    for m in (0, 1):
        assert abs(tot[m, 0] - tot0[m, 0]) / tot0[m, 0] < 1e-12


def test_icf_quarter_plane_fp64(msf):
    """The free surface on a two-dimensional Cartesian grid (a circle)."""
    o, s, eo = run_pair(msf, cs.icf_quarter_plane(64), 60)
    assert eo == 0
    compare(o, s, FP64_L1, exact=True)


def test_icf_fp32(msf):
    o, s, eo = run_pair(msf, cs.icf_implosion(320), 200, precision=1)
    assert eo == 0
    compare(o, s, FP32_L1)


@pytest.mark.parametrize("precision", [0, 1])
def test_icf_batched_matches_oracle(msf, precision):
    """The shell-thickness study as one batched launch (one CTA per instance):
    every instance bit-identical to the oracle in FP64, within the FP32
    tolerance in the FP32-bulk form."""
    steps = 150
    cases = cs.icf_shell_study(160, 5)
    batch = msf.Batch(cases, precision=precision)
    batch.step(steps, 1.0)
    assert batch.launches_per_step() == 1
    for i, c in enumerate(cases):
        o = orc.Oracle(c)
        assert o.step(steps, 1.0) == 0
        a, b = batch.state(i), o.state()
        if precision == 0:
            assert a["t"] == b["t"]
            assert np.array_equal(a["Q"], b["Q"]), (i, np.abs(a["Q"] - b["Q"]).max())
            assert np.array_equal(a["chi"], b["chi"])
        else:
            assert a["t"] == pytest.approx(b["t"], rel=1e-5)
            ra, rb = a["Q"][:, 0].sum(0), b["Q"][:, 0].sum(0)
            assert np.abs(ra - rb).sum() / np.abs(rb).sum() <= FP32_L1


def test_cylindrical_tape_refused(msf):
    """The tape and adjoint entry points take Cartesian grids without a free
    surface only."""
    s = msf.Solver(cs.icf_implosion(160))
    with pytest.raises(msf.MsfError) as ei:
        s.tape_bytes()
    assert ei.value.status == msf.MSF_EUNSUPPORTED
    s.close()
