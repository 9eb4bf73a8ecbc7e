"""GPU path (through the C ABI) against the CPU oracle on the same seeded
inputs, element by element.

FP64 mode: the strict build (-fmad=false on the device, -ffp-contract=off in
the oracle) evaluates every expression as the oracle states it (the WENO5
weights as Jiang and Shu define them included), so the states are expected
to agree to the last bit; the gate is L1 relative density error <= 1e-10,
plus max |dQ| <= 1e-12 * max|Q|.
FP32-bulk mode: L1 relative density error <= 2e-5.
"""
import numpy as np
import pytest

import paper_1704_00519_gb300.cases as cs
from oracle import oracle as orc

pytestmark = pytest.mark.gpu

FP64_L1 = 1e-10
orc_ENEGATIVE = 2
FP32_L1 = 2e-5


@pytest.fixture(scope="module")
def msf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00519_gb300 import build
    build.build()
    import paper_1704_00519_gb300.msf as m
    return m


def l1_rho(Qa, Qb):
    ra, rb = Qa[:, 0].sum(0), Qb[:, 0].sum(0)
    return float(np.abs(ra - rb).sum() / np.abs(rb).sum())


def run_pair(msf, case, steps, t_end=None, precision=0, openmp=False, **opts):
    t_end = case.t_end if t_end is None else t_end
    o = orc.Oracle(case, openmp=openmp, **opts)
    eo = o.step(steps, t_end)
    s = msf.Solver(case, precision=precision, **opts)
    s.step(steps, t_end)
    return o, s, eo


def compare(o, s, tol_l1, exact=False):
    a, b = s.state(), o.state()
    # FP32-bulk time steps come from an FP32 CFL bound
    assert a["t"] == pytest.approx(b["t"], rel=1e-14 if exact else 1e-5, abs=1e-15)
    l1 = l1_rho(a["Q"], b["Q"])
    scale = np.abs(b["Q"]).max()
    dmax = np.abs(a["Q"] - b["Q"]).max()
    assert np.all(np.isfinite(a["Q"]))
    assert l1 <= tol_l1, (l1, dmax)
    if exact:
        assert dmax <= 1e-12 * scale, dmax
        assert np.array_equal(a["chi"], b["chi"])
        assert np.abs(a["phi"] - b["phi"]).max() <= 1e-12
        assert np.abs(a["alpha"] - b["alpha"]).max() <= 1e-12
        ca, cb = s.counters(), o.counters()
        assert ca == cb, (ca, cb)
    return l1, dmax


def test_shock_tube_full_run_fp64(msf):
    case = cs.shock_tube_3(400)
    o, s, eo = run_pair(msf, case, 100000)
    assert eo == 0
    l1, dmax = compare(o, s, FP64_L1, exact=True)
    assert s.state()["t"] == 0.2


@pytest.mark.parametrize("seed", range(4))
def test_random_1d_fp64(msf, seed):
    rng = np.random.default_rng(seed)
    case = cs.riemann_1d(rng, ncell=int(rng.integers(150, 700)))
    o, s, eo = run_pair(msf, case, 40)
    assert eo == 0
    compare(o, s, FP64_L1, exact=True)


@pytest.mark.parametrize("n,nmat,seed", [((37, 29), 3, 1), ((75, 37), 4, 8), ((75, 37), 4, 14), ((33, 9), 2, 3),
                                         ((64, 16), 3, 4)])
def test_random_2d_fp64(msf, n, nmat, seed):
    case = cs.random_case(2, n, nmat, seed)
    o, s, eo = run_pair(msf, case, 15)
    assert eo == 0
    compare(o, s, FP64_L1, exact=True)


def test_device_errors_match_oracle(msf):
    """A violent random four-material start that drives a state non-physical:
    the GPU path reports the same error as the oracle (the oracle may also
    flag a non-finite state of the same step; a non-physical state takes
    precedence in the status)."""
    case = cs.random_case(2, (75, 37), 4, 2)
    o = orc.Oracle(case)
    assert o.step(15, case.t_end) & orc_ENEGATIVE
    s = msf.Solver(case)
    with pytest.raises(msf.MsfError) as ei:
        s.step(15, case.t_end)
    assert ei.value.status == msf.MSF_ENEGATIVE
    with pytest.raises(msf.MsfError) as ei:
        s.step(1, case.t_end)
    assert ei.value.status == msf.MSF_ESTATE


def test_triple_point_fp64(msf):
    case = cs.triple_point(112, 48)
    o, s, eo = run_pair(msf, case, 60)
    assert eo == 0
    compare(o, s, FP64_L1, exact=True)


def test_shock_bubbles_inflow_fp64(msf):
    case = cs.shock_bubbles(96, 32)
    o, s, eo = run_pair(msf, case, 30)
    assert eo == 0
    compare(o, s, FP64_L1, exact=True)


@pytest.mark.parametrize("seed", [4, 6, 9])
def test_random_3d_fp64(msf, seed):
    case = cs.random_case(3, (18, 13, 11), 2 + seed % 2, seed)
    o, s, eo = run_pair(msf, case, 4)
    assert eo == 0
    compare(o, s, FP64_L1, exact=True)


def test_tiny_and_ragged_grids_fp64(msf):
    for case in (cs.random_case(1, (7,), 2, 11), cs.random_case(2, (5, 3), 2, 12), cs.random_case(2, (3, 5), 2, 20),
                 cs.random_case(2, (1, 6), 2, 20)):
        o, s, eo = run_pair(msf, case, 5)
        compare(o, s, FP64_L1, exact=True)


def test_scale_separation_filament_fp64(msf):
    case = cs.scale_sep_demo("filament", n=10)
    o, s, eo = run_pair(msf, case, 2, t_end=10.0)
    compare(o, s, FP64_L1, exact=True)
    assert not np.any(s.state()["chi"] == 2)


@pytest.mark.parametrize("dim,n,nmat,seed", [(2, (23, 19), 3, 3), (2, (23, 19), 4, 5), (3, (10, 9, 8), 3, 3),
                                             (2, (23, 19), 3, 1), (2, (30, 26), 4, 3)])
def test_junction_equilibrium_fp64(msf, dim, n, nmat, seed):
    """Resting junctions (the conservation correction firing, and faces that
    no local field covers closed by the indicators of their two cells): the
    GPU keeps u = 0, p = 1 to round-off and equals the oracle."""
    from test_oracle_pins import _max_dev
    case = cs.random_case(dim, n, nmat, seed, at_rest=True, p_equal=True)
    o, s, eo = run_pair(msf, case, 10, t_end=10.0, scale_sep=0, reinit=0)
    assert eo == 0
    compare(o, s, FP64_L1, exact=True)
    du, dp = _max_dev(case, s.state())
    assert du < 1e-12 and dp < 1e-12


@pytest.mark.parametrize("lit,ln", [(1, 0), (0, 1), (1, 1)])
def test_literal_interaction_options_fp64(msf, lit, ln):
    """The printed forms of the reduced model (Sec. 2.3.2), kept for
    comparison: the GPU equals the oracle with each switch, on a resting
    triple point (which drifts under them) and on a random network."""
    from test_oracle_pins import _resting_triple_point
    for case, steps in ((_resting_triple_point(), 20), (cs.random_case(2, (37, 29), 3, 1), 10)):
        o, s, eo = run_pair(msf, case, steps, t_end=10.0, scale_sep=0, reinit=0, literal_reduced=lit,
                            literal_normal=ln)
        assert eo == 0
        compare(o, s, FP64_L1, exact=True)


@pytest.mark.parametrize("maker,steps", [
    (lambda: __import__("test_oracle_pins")._leblanc(400), 100000),
    (lambda: __import__("test_oracle_pins")._leblanc(400, two=True), 100000),
    (lambda: cs.triple_point(112, 48), 60),
    (lambda: cs.shock_bubbles(96, 32), 30),
    (lambda: cs.random_case(3, (18, 13, 11), 2, 4), 4),
], ids=["leblanc", "leblanc_interface", "triple_point", "bubbles_inflow", "random_3d"])
def test_positivity_limiter_fp64_and_fp32(msf, maker, steps):
    """The positivity-preserving flux limiter (option positivity = 1): FP64
    equals the oracle (LeBlanc's problem runs to t = 6 only with it); the
    FP32-bulk form is within the FP32 tolerance."""
    case = maker()
    o, s, eo = run_pair(msf, case, steps, positivity=1)
    assert eo == 0
    compare(o, s, FP64_L1, exact=True)
    s32 = msf.Solver(case, precision=msf.MSF_FP32_BULK, positivity=1)
    s32.step(steps, case.t_end)
    compare(o, s32, FP32_L1)


def test_correction_choice_at_start_up_fp64(msf):
    """The T-junction of the oracle pin: with each material made the lightest
    in turn, and with densities where the lightest by mass is neither the
    lightest by density nor the smallest fraction, the GPU's corrected volume
    fractions at start-up equal the oracle's."""
    from test_oracle_pins import _t_junction
    r = np.array([0.5588756756756762, 0.1844666212111825, 0.23894901960784248])
    configs = [[1e-3, 1.0, 1.0], [1.0, 1e-3, 1.0], [1.0, 1.0, 1e-3],
               [1.0, 5.45, 0.9 * r[0] / r[2]]]
    for rho in configs:
        case = _t_junction(rho)
        a, b = msf.Solver(case).state()["alpha"], orc.Oracle(case).state()["alpha"]
        assert np.abs(a - b).max() <= 1e-15, rho


@pytest.mark.parametrize("y0,y1,new_chi", [(0.42, 0.49, 0), (0.41, 0.48, 1)])
def test_scale_separation_by_hand_fp64(msf, y0, y1, new_chi):
    """The one-row filament of the oracle pin, one step at rest: the GPU equals
    the oracle, and the filament row took chi_1* with phi* = 0.04."""
    from test_oracle_pins import _one_row_filament
    case = _one_row_filament(y0, y1)
    o, s, eo = run_pair(msf, case, 1, t_end=10.0, reinit=0)
    assert eo == 0
    compare(o, s, FP64_L1, exact=True)
    st = s.state()
    assert np.all(st["chi"][40:50] == new_chi)
    assert np.abs(st["phi"][40:50] - 0.04).max() < 1e-12


def test_scale_separation_droplet_fp64(msf):
    """The droplet demo of Sec. 2.3.3, 10 steps: the GPU equals the oracle
    (the neck's two cells separated, their content following their volume,
    two new triple points) and the totals are kept."""
    case = cs.scale_sep_demo("droplet", n=10)
    s0 = msf.Solver(case)
    tot0, _ = s0.totals()
    o, s, eo = run_pair(msf, case, 10, t_end=10.0)
    assert eo == 0
    compare(o, s, FP64_L1, exact=True)
    assert s.counters()["merge"] == 2
    tot, led = s.totals()
    assert np.abs((tot - tot0 - led).sum(0)).max() <= 1e-13 * np.abs(tot0).sum()


@pytest.mark.parametrize("maker,steps", [(lambda: cs.triple_point(112, 48), 60), (lambda: cs.shock_bubbles(96, 32), 30),
                                         (lambda: cs.shock_tube_3(400), 200)])
def test_fp32_bulk_form(msf, maker, steps):
    case = maker()
    o, s, eo = run_pair(msf, case, steps, precision=msf.MSF_FP32_BULK)
    l1, dmax = compare(o, s, FP32_L1)


@pytest.mark.parametrize("precision", [0, 1])
def test_gpu_conservation(msf, precision):
    case = cs.triple_point(112, 48)
    s = msf.Solver(case, precision=precision)
    tot0, _ = s.totals()
    s.step(100, case.t_end)
    tot, led = s.totals()
    scale = max(np.abs(tot0).sum(), np.abs(tot).sum())
    d = tot - tot0 - led
    if s.counters()["merge"] == 0:
        assert np.abs(d[:, 0]).max() / scale < 1e-12
    assert np.abs(d.sum(0)).max() / scale < 1e-12


def test_full_size_triple_point(msf):
    """896 x 384 (the benchmark workload): three steps element by element
    against the oracle, then 200 steps that must stay finite and conservative."""
    case = cs.triple_point(896, 384)
    o, s, eo = run_pair(msf, case, 3)
    compare(o, s, FP64_L1, exact=True)
    s2 = msf.Solver(case, precision=msf.MSF_FP32_BULK)
    tot0, _ = s2.totals()
    s2.step(200, case.t_end)
    tot, led = s2.totals()
    st = s2.state()
    assert np.all(np.isfinite(st["Q"]))
    scale = max(np.abs(tot0).sum(), np.abs(tot).sum())
    assert np.abs((tot - tot0 - led).sum(0)).max() / scale < 1e-12


@pytest.mark.parametrize("maker,steps", [(lambda: cs.shock_bubbles(2048, 512), 200),
                                         (lambda: cs.shock_sphere((256, 128, 128)), 12)],
                         ids=["shock_bubbles_2048x512", "shock_sphere_256x128x128"])
def test_full_size_fp32_form_against_fp64(msf, maker, steps):
    """Full-size two-bubble (2D) and sphere (3D) shock interactions: the
    FP32-bulk form against the plain FP64 path after the same steps (L1 of the
    density), and per-material mass plus summed momentum and energy conserved
    through the FP64 boundary ledger in both."""
    case = maker()
    states = []
    for prec in (msf.MSF_FP64, msf.MSF_FP32_BULK):
        s = msf.Solver(case, precision=prec)
        tot0, _ = s.totals()
        s.step(steps, case.t_end)
        tot, led = s.totals()
        st = s.state()
        assert np.all(np.isfinite(st["Q"]))
        scale = max(np.abs(tot0).sum(), np.abs(tot).sum())
        d = tot - tot0 - led
        if s.counters()["merge"] == 0:
            assert np.abs(d[:, 0]).max() / scale < 1e-12
        assert np.abs(d.sum(0)).max() / scale < 1e-12
        states.append(st)
        s.close()
    assert l1_rho(states[1]["Q"], states[0]["Q"]) <= FP32_L1


@pytest.mark.parametrize("maker", [lambda: cs.shock_sphere((48, 32, 32)),
                                   lambda: cs.random_case(3, (48, 32, 32), 3, 8)], ids=["sphere", "random3"])
def test_3d_fp64_many_tiles(msf, maker):
    """3D at 48 x 32 x 32 (6 x 4 x 8 flux tiles of 8 x 8 x 4, persistent CTAs
    taking them from the counter, band and idle tiles among them) for 10
    steps (the random network: junctions where the correction fires): the
    FP64 path equals the oracle."""
    case = maker()
    o, s, eo = run_pair(msf, case, 10, openmp=True)
    assert eo == 0
    compare(o, s, FP64_L1, exact=True)


def test_two_bubbles_512x128_50_steps(msf):
    """The two-bubble shock (inflow, walls, two heavy and light bubbles) at
    512 x 128, 50 steps: 256 flux tiles of 32 x 8, persistent-CTA scheduling
    and idle tiles with many tiles in flight; FP64 equals the oracle, the
    FP32-bulk form is within the FP32 tolerance."""
    case = cs.shock_bubbles(512, 128)
    o, s, eo = run_pair(msf, case, 50, openmp=True)
    assert eo == 0
    compare(o, s, FP64_L1, exact=True)
    s32 = msf.Solver(case, precision=msf.MSF_FP32_BULK)
    s32.step(50, case.t_end)
    compare(o, s32, FP32_L1)


@pytest.mark.parametrize("gamma_right", [1.667, 1.249])
def test_paper_case_one_rk2_fp64(msf, gamma_right):
    """The paper's Case I (helium | air | helium between walls; the R22
    variant) with its two-stage TVD Runge-Kutta, full run to t = 0.1: FP64
    bit-identical to the oracle."""
    case = cs.he_air_tube(200, gamma_right)
    o, s, eo = run_pair(msf, case, 100000, rk_stages=2)
    assert eo == 0
    compare(o, s, FP64_L1, exact=True)


def test_rk2_triple_point_fp64_and_fp32(msf):
    case = cs.triple_point(112, 48)
    o, s, eo = run_pair(msf, case, 40, rk_stages=2)
    compare(o, s, FP64_L1, exact=True)
    s32 = msf.Solver(case, precision=msf.MSF_FP32_BULK, rk_stages=2)
    s32.step(40, case.t_end)
    compare(o, s32, FP32_L1)


def test_tait_water_pulse_fp64(msf):
    """Tait's equation (Sec. 2.1), 1D water acoustics, full run: the GPU and
    the oracle evaluate (rho/rho0)^gamma with two different math libraries
    (pow may differ in the last bit), so the gate is the FP64 tolerance."""
    case = cs.water_pulse(400)
    o, s, eo = run_pair(msf, case, 100000)
    assert eo == 0
    compare(o, s, FP64_L1)


def test_helium_water_case_fp64_fp32_and_conservation(msf):
    """Mach-6 air shock, helium bubble and a Tait water column (Sec. 3.6
    states) on a coarse grid: FP64 against the oracle within the FP64
    tolerance; the FP32-bulk form within the FP32 tolerance; per-material
    mass and summed momentum and energy through the ledger."""
    case = cs.shock_helium_water(128, 32)
    o, s, eo = run_pair(msf, case, 30)
    assert eo == 0
    compare(o, s, FP64_L1)
    s32 = msf.Solver(case, precision=msf.MSF_FP32_BULK)
    tot0, _ = s32.totals()
    s32.step(30, case.t_end)
    compare(o, s32, FP32_L1)
    tot, led = s32.totals()
    scale = max(np.abs(tot0).sum(), np.abs(tot).sum())
    d = tot - tot0 - led
    if s32.counters()["merge"] == 0:
        assert np.abs(d[:, 0]).max() / scale < 1e-12
    assert np.abs(d.sum(0)).max() / scale < 1e-12


def test_adjoint_refuses_tait_materials(msf):
    import torch
    case = cs.water_pulse(64)
    s = msf.Solver(case)
    tp = s.new_tape()
    s.step_taped(tp, case.t_end)
    lam = torch.zeros((1, 3, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(msf.MsfError) as e:
        s.adjoint_step(tp, lam)
    assert e.value.status == msf.MSF_EUNSUPPORTED


def test_host_validation_rejects_bad_levelset(msf):
    case = cs.shock_tube_3(50)
    s = msf.Solver(case)
    bad = case.phi.copy()
    bad[3] = -1.0
    with pytest.raises(msf.MsfError):
        s.set_levelset(bad, case.chi, case.prim)
    chi = case.chi.copy()
    chi[0] = 7
    with pytest.raises(msf.MsfError):
        s.set_levelset(case.phi, chi, case.prim)


def test_device_inputs_and_set_state_roundtrip(msf):
    import torch
    case = cs.triple_point(56, 24)
    s = msf.Solver(case)
    dev = torch.device("cuda")
    s.set_levelset(torch.tensor(case.phi.ravel(), device=dev), torch.tensor(case.chi.ravel(), device=dev),
                   torch.tensor(case.prim, device=dev))
    s.step(5)
    st = s.state()
    s2 = msf.Solver(case)
    s2.set_state(st["Q"], st["phi"], st["chi"], st["t"])
    s.step(5)
    s2.step(5)
    a, b = s.state(), s2.state()
    assert np.array_equal(a["Q"], b["Q"])
    assert a["t"] == b["t"]


@pytest.mark.parametrize("maker,prec,opts", [
    (lambda: cs.triple_point(56, 24), 0, {}),
    (lambda: cs.triple_point(56, 24), 1, {}),
    (lambda: cs.shock_tube_3(100), 0, dict(rk_stages=2)),
    (lambda: cs.random_case(3, (10, 9, 8), 2, 2), 1, dict(scale_sep=0, reinit=0)),
])
def test_launch_count_matches_graph(msf, maker, prec, opts):
    """The kernel count one step reports equals the kernel nodes of the step
    graph the first call captures (the call raises when they differ)."""
    case = maker()
    s = msf.Solver(case, precision=prec, **opts)
    s.step(2, case.t_end)
    assert s.launches_per_step() > 0
    s.close()
