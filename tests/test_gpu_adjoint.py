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
"""
import dataclasses

import numpy as np
import pytest

import paper_1704_00519_gb300.cases as cs
from oracle import oracle as orc

pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-5


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00519_gb300 import build
    build.build()
    import paper_1704_00519_gb300.msf as m
    return m, torch


def record(msf, case, steps, precision=0):
    s = msf.Solver(case, precision=precision)
    tapes = []
    for _ in range(steps):
        tp = s.new_tape()
        s.step_taped(tp, case.t_end)
        tapes.append(tp)
    return s, tapes


def replay_state(msf, torch, case, tapes, Q0, precision=0):
    s = msf.Solver(case, precision=precision)
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
    "riemann_1d": (lambda: cs.riemann_1d(np.random.default_rng(5), 160, 3), 8),
    "triple_point": (lambda: cs.triple_point(56, 24), 6),
    "shock_bubbles_inflow": (lambda: cs.shock_bubbles(96, 32), 6),
    "random_2d": (lambda: cs.random_case(2, (37, 29), 3, 1), 5),
    "shock_sphere_3d": (lambda: cs.shock_sphere((24, 12, 12)), 4),
}


@pytest.mark.parametrize("name", ["triple_point", "shock_sphere_3d"])
def test_taped_step_and_replay_are_the_forward_step(env, name):
    msf, torch = env
    case, steps = CASES[name][0](), CASES[name][1]
    s_plain = msf.Solver(case)
    Q0 = torch.empty((case.nmat, case.nv, case.cells), dtype=torch.float64, device="cuda")
    s_plain.get_state_device(Q0)
    s_plain.step(steps, case.t_end)
    s_tape, tapes = record(msf, case, steps)
    a, b = s_plain.state(), s_tape.state()
    assert np.array_equal(a["Q"], b["Q"])
    assert np.array_equal(a["phi"], b["phi"]) and np.array_equal(a["chi"], b["chi"])
    Qr = replay_state(msf, torch, case, tapes, Q0)
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
    s, tapes = record(msf, case, steps)
    ref = msf.Solver(case)
    Q0 = torch.empty((case.nmat, case.nv, case.cells), dtype=torch.float64, device="cuda")
    ref.get_state_device(Q0)
    rng = np.random.default_rng(11)
    lamK = torch.tensor(rng.uniform(-1, 1, Q0.shape), device="cuda")
    dQ = Q0 * torch.tensor(rng.uniform(-1, 1, Q0.shape), device="cuda")
    lam0, _, _ = adjoint_chain(s, tapes, lamK)
    adj = float((lam0 * dQ).sum())
    eps = 1e-6
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
    s, tapes = record(msf, case, steps)
    ref = msf.Solver(case)
    Q0 = torch.empty((case.nmat, case.nv, case.cells), dtype=torch.float64, device="cuda")
    ref.get_state_device(Q0)
    rng = np.random.default_rng(7)
    lamK = torch.tensor(rng.uniform(-1, 1, Q0.shape), device="cuda")
    _, d_eos, d_inf = adjoint_chain(s, tapes, lamK)

    def J(c):
        return float((lamK * replay_state(msf, torch, c, tapes, Q0)).sum())

    checks = []
    for m in range(case.nmat):
        g = list(case.gamma)
        h = 1e-6 * g[m]
        gp, gm = list(g), list(g)
        gp[m] += h
        gm[m] -= h
        checks.append(("gamma", m, d_eos[m, 0], (J(_with(case, gamma=gp)) - J(_with(case, gamma=gm))) / (2 * h)))
        pinf = list(case.pinf)
        h = 1e-6 * max(pinf[m], 1.0)
        pp, pm = list(pinf), list(pinf)
        pp[m] += h
        pm[m] = max(pm[m] - h, 0.0)
        if pinf[m] - h >= 0.0:
            checks.append(("pinf", m, d_eos[m, 1], (J(_with(case, pinf=pp)) - J(_with(case, pinf=pm))) / (2 * h)))
    if case.inflow_prim is not None and any(b == cs.INFLOW for bb in case.bc for b in bb):
        for v in range(case.nv):
            ip = np.array(case.inflow_prim)
            h = 1e-6 * max(abs(ip[0, 0, v]), 1.0)
            a, b = ip.copy(), ip.copy()
            a[0, 0, v] += h
            b[0, 0, v] -= h
            checks.append(("inflow", v, d_inf[0, 0, v],
                           (J(_with(case, inflow_prim=a)) - J(_with(case, inflow_prim=b))) / (2 * h)))
    for kind, k, adj, fd in checks:
        tol = GRAD_RTOL * max(abs(fd), abs(adj)) + 1e-9 * float(lamK.abs().sum())
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
    s, tapes = record(msf, case, steps)
    o = orc.Oracle(case)
    otapes = [o.step_taped(case.t_end) for _ in range(steps)]
    Q0 = orc.Oracle(case).state()["Q"]
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

    eps = 1e-6
    fd = (J(Q0 + eps * dQ) - J(Q0 - eps * dQ)) / (2 * eps)
    assert abs(adj - fd) <= GRAD_RTOL * max(abs(fd), abs(adj)), (adj, fd)
