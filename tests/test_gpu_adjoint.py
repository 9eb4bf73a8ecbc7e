"""Tapes, replay at frozen interface evolution and the adjoint step, through
the C ABI on the GPU.

* A taped step is the plain step (bitwise), and replaying its tapes from the
  same initial state reproduces the trajectory (bitwise, FP64).
* The GPU replay agrees with the oracle's replay of the same tapes from a
  perturbed state (the oracle implements the same frozen-interface step
  independently).
* The adjoint is checked by dot products: for random seeds lam_K and random
  relative perturbations dQ0 of the initial state, <lam_0, dQ0> from the
  adjoint chain equals the central difference of <lam_K, Q^K> along dQ0,
  computed by replaying the tapes (GPU and oracle); EOS and inflow partials
  against central differences of contexts with perturbed parameters.
* Pins independent of both implementations: with reflective walls total mass
  and total energy are invariants of the replay map, so their adjoint is
  exactly the seed (ones on the density / energy of every material).

The Lax-Friedrichs coefficient of a face is a maximum over its stencil; on
piecewise-constant data many stencils hold exact ties, where the step is not
differentiable (a central difference then averages one-sided slopes while
the adjoint returns one of them). The Q-direction checks therefore start from
the case's state with 1% relative noise (no exact ties), and take central
differences with steps far below the noise.
"""
import dataclasses

import numpy as np
import pytest

import paper_1704_00519_gb300.cases as cs
from oracle import oracle as orc

pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-5
EOS_RTOL = 1e-4
NOISE = 1e-2
EPS = 1e-7


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00519_gb300 import build
    build.build()
    import paper_1704_00519_gb300.msf as m
    return m, torch


def noisy_state(torch, case, Q0, seed=1):
    g = np.random.default_rng(seed)
    return Q0 * torch.tensor(1.0 + NOISE * g.uniform(-1, 1, Q0.shape), device=Q0.device)


def _opts(case):
    """Run options a case needs (the paper's Case I runs the two-stage scheme)."""
    return {"rk_stages": 2} if case.name == "he_air_tube" else {}


def record(msf, case, steps, precision=0, Q0=None):
    s = msf.Solver(case, precision=precision, **_opts(case))
    if Q0 is not None:
        s.set_conserved(Q0)
    tapes = []
    for _ in range(steps):
        tp = s.new_tape()
        s.step_taped(tp, case.t_end)
        tapes.append(tp)
    return s, tapes


def replay_state(msf, torch, case, tapes, Q0, precision=0):
    s = msf.Solver(case, precision=precision, **_opts(case))
    s.set_conserved(Q0)
    for tp in tapes:
        s.replay_step(tp)
    Q = torch.empty((case.nmat, case.nv, case.cells), dtype=torch.float64, device="cuda")
    s.get_state_device(Q)
    s.close()
    return Q


def adjoint_chain(s, tapes, lam):
    d_eos = np.zeros((s.N, 2))
    d_inf = np.zeros((3, 2, 5))
    for tp in reversed(tapes):
        lam, de, di = s.adjoint_step(tp, lam)
        d_eos += de
        d_inf += di
    return lam, d_eos, d_inf


CASES = {
    "shock_tube_3": (lambda: cs.shock_tube_3(120), 8),
    "he_air_tube_rk2": (lambda: cs.he_air_tube(120), 8),
    "riemann_1d": (lambda: cs.riemann_1d(np.random.default_rng(5), 160, 3), 8),
    "triple_point": (lambda: cs.triple_point(56, 24), 6),
    "shock_bubbles_inflow": (lambda: cs.shock_bubbles(96, 32), 6),
    "random_2d": (lambda: cs.random_case(2, (37, 29), 3, 1), 5),
    "shock_sphere_3d": (lambda: cs.shock_sphere((24, 12, 12)), 4),
}


@pytest.mark.parametrize("name,precision", [("triple_point", 0), ("shock_sphere_3d", 0), ("triple_point", 1)])
def test_taped_step_and_replay_are_the_forward_step(env, name, precision):
    """FP32-bulk form included: its two-dimensional forward step runs the
    ghost-state sweeps tiled (all sweeps in one launch), the replay one sweep
    per launch; the two give the same bits."""
    msf, torch = env
    case, steps = CASES[name][0](), CASES[name][1]
    s_plain = msf.Solver(case, precision=precision)
    Q0 = torch.empty((case.nmat, case.nv, case.cells), dtype=torch.float64, device="cuda")
    s_plain.get_state_device(Q0)
    s_plain.step(steps, case.t_end)
    s_tape, tapes = record(msf, case, steps, precision=precision)
    a, b = s_plain.state(), s_tape.state()
    assert np.array_equal(a["Q"], b["Q"])
    assert np.array_equal(a["phi"], b["phi"]) and np.array_equal(a["chi"], b["chi"])
    Qr = replay_state(msf, torch, case, tapes, Q0, precision=precision)
    assert np.array_equal(Qr.cpu().numpy(), a["Q"])


@pytest.mark.parametrize("name", ["shock_tube_3", "triple_point", "shock_bubbles_inflow"])
def test_replay_matches_oracle_replay(env, name):
    """Tapes recorded by the GPU are the oracle's tapes (bitwise forward);
    both replay them from the same perturbed initial state."""
    msf, torch = env
    case, steps = CASES[name][0](), CASES[name][1]
    s, tapes = record(msf, case, steps)
    o = orc.Oracle(case)
    otapes = [o.step_taped(case.t_end) for _ in range(steps)]
    L = orc.Oracle(case)
    Q0 = L.state()["Q"]
    rng = np.random.default_rng(3)
    Qp = Q0 * (1.0 + 1e-3 * rng.uniform(-1, 1, Q0.shape))
    L.set_conserved(Qp)
    for tp in otapes:
        L.replay_step(tp)
    Qg = replay_state(msf, torch, case, tapes, torch.tensor(Qp, device="cuda")).cpu().numpy()
    Qo = L.state()["Q"]
    scale = np.abs(Qo).max()
    assert np.abs(Qg - Qo).max() <= 1e-12 * scale


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_dot_product_against_central_differences(env, name):
    msf, torch = env
    case, steps = CASES[name][0](), CASES[name][1]
    ref = msf.Solver(case)
    Q0 = torch.empty((case.nmat, case.nv, case.cells), dtype=torch.float64, device="cuda")
    ref.get_state_device(Q0)
    Q0 = noisy_state(torch, case, Q0)
    s, tapes = record(msf, case, steps, Q0=Q0)
    rng = np.random.default_rng(11)
    lamK = torch.tensor(rng.uniform(-1, 1, Q0.shape), device="cuda")
    dQ = Q0 * torch.tensor(rng.uniform(-1, 1, Q0.shape), device="cuda")
    lam0, _, _ = adjoint_chain(s, tapes, lamK)
    adj = float((lam0 * dQ).sum())
    eps = EPS
    Jp = float((lamK * replay_state(msf, torch, case, tapes, Q0 + eps * dQ)).sum())
    Jm = float((lamK * replay_state(msf, torch, case, tapes, Q0 - eps * dQ)).sum())
    fd = (Jp - Jm) / (2 * eps)
    assert abs(adj - fd) <= GRAD_RTOL * max(abs(fd), abs(adj)), (adj, fd)


def _with(case, **kw):
    return dataclasses.replace(case, **kw)


@pytest.mark.parametrize("name", ["shock_tube_3", "riemann_1d", "triple_point", "shock_bubbles_inflow",
                                  "shock_sphere_3d"])
def test_adjoint_eos_and_inflow_partials(env, name):
    msf, torch = env
    case, steps = CASES[name][0](), CASES[name][1]
    ref = msf.Solver(case)
    Q0 = torch.empty((case.nmat, case.nv, case.cells), dtype=torch.float64, device="cuda")
    ref.get_state_device(Q0)
    Q0 = noisy_state(torch, case, Q0, seed=2)
    s, tapes = record(msf, case, steps, Q0=Q0)
    rng = np.random.default_rng(7)
    lamK = torch.tensor(rng.uniform(-1, 1, Q0.shape), device="cuda")
    _, d_eos, d_inf = adjoint_chain(s, tapes, lamK)

    def J(c):
        return float((lamK * replay_state(msf, torch, c, tapes, Q0)).sum())

    checks = []
    for m in range(case.nmat):
        g = list(case.gamma)
        h = 1e-7 * g[m]
        gp, gm = list(g), list(g)
        gp[m] += h
        gm[m] -= h
        checks.append(("gamma", m, d_eos[m, 0], (J(_with(case, gamma=gp)) - J(_with(case, gamma=gm))) / (2 * h)))
        pinf = list(case.pinf)
        h = 1e-7 * max(pinf[m], 1.0)
        pp, pm = list(pinf), list(pinf)
        pp[m] += h
        pm[m] = max(pm[m] - h, 0.0)
        if pinf[m] - h >= 0.0:
            checks.append(("pinf", m, d_eos[m, 1], (J(_with(case, pinf=pp)) - J(_with(case, pinf=pm))) / (2 * h)))
    if case.inflow_prim is not None and any(b == cs.INFLOW for bb in case.bc for b in bb):
        for v in range(case.nv):
            ip = np.array(case.inflow_prim)
            h = 1e-7 * max(abs(ip[0, 0, v]), 1.0)
            a, b = ip.copy(), ip.copy()
            a[0, 0, v] += h
            b[0, 0, v] -= h
            checks.append(("inflow", v, d_inf[0, 0, v],
                           (J(_with(case, inflow_prim=a)) - J(_with(case, inflow_prim=b))) / (2 * h)))
    for kind, k, adj, fd in checks:
        tol = EOS_RTOL * max(abs(fd), abs(adj)) + 1e-9 * float(lamK.abs().sum())
        assert abs(adj - fd) <= tol, (kind, k, adj, fd)


@pytest.mark.parametrize("name", ["triple_point", "random_2d"])
def test_adjoint_of_conserved_totals_is_the_seed(env, name):
    """Reflective box: total mass and total energy are invariants of the
    replay map, whatever the state and EOS: their adjoint is the seed."""
    msf, torch = env
    case, steps = CASES[name][0](), CASES[name][1]
    case = _with(case, bc=[[cs.REFLECTIVE, cs.REFLECTIVE]] * case.dim)
    s, tapes = record(msf, case, steps)
    for v in (0, case.nv - 1):
        seed = torch.zeros((case.nmat, case.nv, case.cells), dtype=torch.float64, device="cuda")
        seed[:, v] = 1.0
        lam0, d_eos, _ = adjoint_chain(s, tapes, seed)
        assert float((lam0 - seed).abs().max()) <= 1e-13
        assert np.abs(d_eos).max() <= 1e-9


def test_adjoint_against_oracle_differences(env):
    """The GPU adjoint against central differences of the oracle's replay."""
    msf, torch = env
    case, steps = cs.triple_point(56, 24), 4
    Q0 = orc.Oracle(case).state()["Q"]
    Q0 = noisy_state(torch, case, torch.tensor(Q0), seed=4).numpy()
    s, tapes = record(msf, case, steps, Q0=torch.tensor(Q0, device="cuda"))
    o = orc.Oracle(case)
    o.set_conserved(Q0)
    otapes = [o.step_taped(case.t_end) for _ in range(steps)]
    rng = np.random.default_rng(19)
    lamK = rng.uniform(-1, 1, Q0.shape)
    dQ = Q0 * rng.uniform(-1, 1, Q0.shape)
    lam0, _, _ = adjoint_chain(s, tapes, torch.tensor(lamK, device="cuda"))
    adj = float((lam0.cpu().numpy() * dQ).sum())

    def J(Qs):
        L = orc.Oracle(case)
        L.set_conserved(Qs)
        for tp in otapes:
            L.replay_step(tp)
        return float((lamK * L.state()["Q"]).sum())

    eps = EPS
    fd = (J(Q0 + eps * dQ) - J(Q0 - eps * dQ)) / (2 * eps)
    assert abs(adj - fd) <= GRAD_RTOL * max(abs(fd), abs(adj)), (adj, fd)


def _objectives(prob, adj, torch, Qs, dts, alphas, eos, x, wall, farea):
    """J1: bubble mass-centroid x displacement; J2: y = 0 wall pressure impulse."""
    J1 = adj.mass_centroid_x(Qs[-1], 1, x) - adj.mass_centroid_x(Qs[0], 1, x)
    J2 = sum(dt * adj.wall_pressure(Q, eos, a, wall, farea) for Q, dt, a in zip(Qs[1:], dts, alphas))
    return J1, J2


def test_shock_bubble_gradients_autograd_fd_and_oracle(env):
    """3D shock on a heavy sphere (32 x 16 x 16, the workload's small
    counterpart): d(J1, J2)/d(rho_bubble, gamma_bubble, Mach) through the
    torch.autograd.Function (adjoint steps) against central differences of
    the GPU replay and of the oracle's replay, within 1e-4 relative at
    h = 1e-6 (relative). The step is piecewise smooth (maxima and minima in
    the Lax-Friedrichs and HLLC wave speeds), so a difference with
    h = 1e-3 is a secant across kinks; it is computed too and must agree
    within 1e-2."""
    msf, torch = env
    from paper_1704_00519_gb300 import adjoint as adj
    K = 10
    prob = adj.ShockBubble((32, 16, 16))
    th0 = prob.theta0()
    case0 = prob.case(th0)
    solver = msf.Solver(case0)
    st0 = solver.state()
    alpha0 = torch.tensor(st0["alpha"], device="cuda")
    xs = torch.tensor(cs.centres(prob.n, case0.lo, case0.hi)[0].ravel(), device="cuda")
    wall = torch.tensor(np.nonzero(cs.centres(prob.n, case0.lo, case0.hi)[1].ravel() < 1.0 / prob.n[1])[0],
                        device="cuda")
    h = [(case0.hi[d] - case0.lo[d]) / prob.n[d] for d in range(3)]
    farea = h[0] * h[2]

    theta = th0.clone().cuda().requires_grad_(True)
    eos = prob.eos(theta)
    inflow = prob.inflow(theta)
    Q = prob.conserved(prob.prim(theta, "cuda"), eos, alpha0)
    tapes, Qs, dts, alphas = [], [Q], [], []
    for _ in range(K):
        Q = adj.MsfStep.apply(Q, eos, inflow, solver, case0.t_end, tapes)
        Qs.append(Q)
        dts.append(adj.tape_dt(tapes[-1]))
        alphas.append(torch.tensor(solver.state()["alpha"], device="cuda"))
    J1, J2 = _objectives(prob, adj, torch, Qs, dts, alphas, eos, xs, wall, farea)
    g1 = torch.autograd.grad(J1, theta, retain_graph=True)[0].cpu().numpy()
    g2 = torch.autograd.grad(J2, theta)[0].cpu().numpy()

    def replay_objectives(th, oracle=False):
        th = torch.tensor(th, dtype=torch.float64)
        c = prob.case(th)
        thd = th.cuda()
        e = prob.eos(thd)
        Q0 = prob.conserved(prob.prim(thd, "cuda"), e, alpha0)
        out = [Q0]
        if oracle:
            L = orc.Oracle(c)
            L.set_conserved(Q0.cpu().numpy())
            for tp in otapes:
                L.replay_step(tp)
                out.append(torch.tensor(L.state()["Q"], device="cuda"))
        else:
            s = msf.Solver(c)
            s.set_conserved(Q0)
            for tp in tapes:
                s.replay_step(tp)
                Qn = torch.empty_like(Q0)
                s.get_state_device(Qn)
                out.append(Qn)
        j1, j2 = _objectives(prob, adj, torch, out, dts, alphas, e, xs, wall, farea)
        return float(j1), float(j2)

    o = orc.Oracle(case0)
    otapes = [o.step_taped(case0.t_end) for _ in range(K)]
    for oracle, hrel, tol in ((False, 1e-6, 1e-4), (True, 1e-6, 1e-4), (False, 1e-3, 1e-2)):
        fd1, fd2 = np.zeros(3), np.zeros(3)
        for i in range(3):
            hh = hrel * float(th0[i])
            tp_, tm_ = th0.numpy().copy(), th0.numpy().copy()
            tp_[i] += hh
            tm_[i] -= hh
            a1, a2 = replay_objectives(tp_, oracle)
            b1, b2 = replay_objectives(tm_, oracle)
            fd1[i], fd2[i] = (a1 - b1) / (2 * hh), (a2 - b2) / (2 * hh)
        for g, fd in ((g1, fd1), (g2, fd2)):
            scale = np.abs(fd).max()
            print("shock-bubble gradient", "oracle" if oracle else "gpu", hrel, g, fd)
            assert np.abs(g - fd).max() <= tol * scale, (oracle, hrel, g, fd)


def test_fp32_form_adjoint_close_to_fp64(env):
    """The FP32-bulk context's adjoint (stencil states in float, adjoint
    accumulated in double) of the same tapes against the FP64 adjoint."""
    msf, torch = env
    case, steps = CASES["shock_bubbles_inflow"][0](), 4
    ref = msf.Solver(case)
    Q0 = torch.empty((case.nmat, case.nv, case.cells), dtype=torch.float64, device="cuda")
    ref.get_state_device(Q0)
    Q0 = noisy_state(torch, case, Q0, seed=5)
    s64, tapes = record(msf, case, steps, Q0=Q0)
    s32 = msf.Solver(case, precision=msf.MSF_FP32_BULK)
    rng = np.random.default_rng(23)
    lamK = torch.tensor(rng.uniform(-1, 1, Q0.shape), device="cuda")
    l64, e64, _ = adjoint_chain(s64, tapes, lamK)
    l32, e32, _ = adjoint_chain(s32, tapes, lamK)
    rel = float((l32 - l64).abs().sum() / l64.abs().sum())
    assert rel <= 1e-4, rel
    assert np.abs(e32 - e64).max() <= 1e-4 * np.abs(e64).max()
