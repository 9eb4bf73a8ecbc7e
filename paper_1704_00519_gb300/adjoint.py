"""Gradients through the GPU step at frozen interface evolution.

``MsfStep`` is a ``torch.autograd.Function`` around one TVD-RK3 step of a
``msf.Solver``: the forward pass takes the step with ``msf_step_taped`` (the
tape is the stage checkpoint: Q^n and the level set of every stage); the
backward pass calls ``msf_adjoint_step``, which recomputes the stages from the
tape and pulls the adjoint back through them. The derivative is that of the
step with the interface evolution and the time step held at the recorded
ones (fixed interface topology): the level set moves as recorded, while the
flow (Sec. 2.3 of the paper: fluxes, interface exchange, mixing) responds to
the state and the EOS parameters.

Objectives for the three-dimensional shock-bubble workload (a Mach-1.22 air
shock on a heavy sphere) and their parameters theta = (rho_bubble,
gamma_bubble, Mach) are built here from plain torch operations:
  * the initial state Q^0(theta) = alpha * cons(prim(theta)) with the
    post-shock state from the Rankine-Hugoniot relations;
  * J1, the x-displacement of the bubble material's centre of mass (at fixed
    interface topology its volume fractions are the recorded ones, so the
    centroid that responds to theta is the mass-weighted one);
  * J2, the pressure impulse on the y = 0 wall, sum_n dt_n sum_cells
    sum_m alpha^m p^m |face|.
"""
from __future__ import annotations

import numpy as np
import torch

from . import cases as cs


class MsfStep(torch.autograd.Function):
    """Q^{n+1} = step(Q^n; gamma, pinf, inflow) of a single-instance solver.

    Inputs: Q (float64 device [N, NV, cells]), eos (float64 [N, 2]: gamma,
    pinf, which must be the solver's), inflow (float64 [3, 2, 5], the solver's
    inflow primitive states), the solver, t_end. The solver's level set must
    be the one the state belongs to (the output of the previous step); the
    forward pass overwrites the solver's conserved state with Q. When
    tape_log is a list, the step's tape is appended to it (for replays)."""

    @staticmethod
    def forward(ctx, Q, eos, inflow, solver, t_end, tape_log=None):
        solver.set_conserved(Q.detach().contiguous())
        tape = solver.new_tape()
        solver.step_taped(tape, t_end)
        if tape_log is not None:
            tape_log.append(tape)
        out = torch.empty_like(Q)
        solver.get_state_device(out)
        ctx.solver = solver
        ctx.tape = tape
        ctx.eos_device = eos.device
        ctx.inflow_device = inflow.device
        return out

    @staticmethod
    def backward(ctx, g):
        lam_in, d_eos, d_inf = ctx.solver.adjoint_step(ctx.tape, g.detach().to(torch.float64).contiguous())
        return (lam_in, torch.as_tensor(d_eos, device=ctx.eos_device),
                torch.as_tensor(d_inf, device=ctx.inflow_device), None, None, None)


def tape_dt(tape):
    """Time step of a tape (header: t, dt)."""
    return float(tape[:16].view(torch.float64)[1])


# ---------------------------------------------------------- shock-bubble problem
def rankine_hugoniot(gamma, rho0, p0, mach):
    """Post-shock (rho, u, p) behind a normal shock of Mach number `mach`
    moving into gas at rest (ideal gas), differentiable in every argument."""
    c0 = torch.sqrt(gamma * p0 / rho0)
    s = mach * c0
    m2 = mach * mach
    p1 = p0 * (1.0 + 2.0 * gamma / (gamma + 1.0) * (m2 - 1.0))
    rho1 = rho0 * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    u1 = s * (1.0 - rho0 / rho1)
    return rho1, u1, p1


class ShockBubble:
    """Mach-M air shock on one heavy sphere (3D) or disc (2D); theta =
    (rho_bubble, gamma_bubble, Mach). Case geometry from cases.shock_sphere."""

    def __init__(self, n=(32, 16, 16), x_shock=0.25):
        self.n = tuple(n)
        self.x_shock = x_shock
        self.base = cs.shock_sphere(self.n, x_shock=x_shock)
        self.dim = self.base.dim

    def theta0(self):
        return torch.tensor([3.154, 1.249, 1.22], dtype=torch.float64)

    def case(self, theta):
        """numpy case at the parameter values theta (for a solver)."""
        rb, gb, ms = [float(x) for x in theta]
        c = cs.shock_sphere(self.n, mach=ms, x_shock=self.x_shock)
        c.gamma = [1.4, gb]
        c.prim[1, 0] = rb
        return c

    def prim(self, theta, dev):
        """Primitive states [N, NV, cells] as a differentiable function of theta."""
        rb, gb, ms = theta[0], theta[1], theta[2]
        one = torch.ones((), dtype=torch.float64, device=dev)
        rho1, u1, p1 = rankine_hugoniot(1.4 * one, one, one, ms)
        x = torch.tensor(cs.centres(self.n, self.base.lo, self.base.hi)[0].ravel(), device=dev)
        post = (x < self.x_shock).to(torch.float64)
        N, NV, cells = 2, self.dim + 2, int(np.prod(self.n))
        air = torch.zeros((NV, cells), dtype=torch.float64, device=dev)
        air[0] = post * rho1 + (1 - post)
        air[1] = post * u1
        air[NV - 1] = post * p1 + (1 - post)
        bub = torch.zeros((NV, cells), dtype=torch.float64, device=dev)
        bub[0] = rb * torch.ones(cells, dtype=torch.float64, device=dev)
        bub[NV - 1] = 1.0
        return torch.stack([air, bub])

    def eos(self, theta):
        gb = theta[1]
        z = torch.zeros((), dtype=torch.float64, device=theta.device)
        return torch.stack([torch.stack([1.4 + z, z]), torch.stack([gb, z])])

    def inflow(self, theta):
        one = torch.ones((), dtype=torch.float64, device=theta.device)
        rho1, u1, p1 = rankine_hugoniot(1.4 * one, one, one, theta[2])
        z = torch.zeros((), dtype=torch.float64, device=theta.device)
        inf = torch.zeros((3, 2, 5), dtype=torch.float64, device=theta.device)
        row = torch.stack([rho1, u1] + [z] * (self.dim - 1) + [p1] + [z] * (3 - self.dim))
        inf = inf.index_put((torch.tensor([0]), torch.tensor([0])), row.unsqueeze(0))
        return inf

    def conserved(self, prim, eos, alpha):
        """Q = alpha * cons(prim) of every material (zero where alpha = 0)."""
        N, NV = prim.shape[0], prim.shape[1]
        D = NV - 2
        gam = eos[:, 0].view(N, 1)
        pinf = eos[:, 1].view(N, 1)
        rho = prim[:, 0]
        vel = prim[:, 1:1 + D]
        p = prim[:, NV - 1]
        E = (p + gam * pinf) / (gam - 1.0) + 0.5 * rho * (vel * vel).sum(1)
        U = torch.cat([rho.unsqueeze(1), rho.unsqueeze(1) * vel, E.unsqueeze(1)], 1)
        return torch.where(alpha.unsqueeze(1) > 0, alpha.unsqueeze(1) * U, torch.zeros_like(U))


def mass_centroid_x(Q, m, x):
    """x of the centre of mass of material m."""
    rho = Q[m, 0]
    return (rho * x).sum() / rho.sum()


def wall_pressure(Q, eos, alpha, wall, farea):
    """sum over the wall-adjacent cells of sum_m alpha^m p^m times the face
    area (alpha^m p^m = (g-1)(Q_E - |Q_u|^2 / 2 Q_rho) - g pinf alpha^m)."""
    N, NV = Q.shape[0], Q.shape[1]
    D = NV - 2
    gam = eos[:, 0].view(N, 1)
    pinf = eos[:, 1].view(N, 1)
    q = Q[:, :, wall]
    rho = q[:, 0]
    mom2 = (q[:, 1:1 + D] ** 2).sum(1)
    safe = torch.where(rho > 0, rho, torch.ones_like(rho))
    ap = (gam - 1.0) * (q[:, NV - 1] - 0.5 * mom2 / safe) - gam * pinf * alpha[:, wall]
    ap = torch.where(rho > 0, ap, torch.zeros_like(ap))
    return ap.sum() * farea


def wall_pressure_rows(Q, eos, alpha_wall, wall, farea):
    """wall_pressure with the volume fractions of the wall cells only
    (alpha_wall [N, len(wall)]), for long runs that keep no full alpha."""
    N, NV = Q.shape[0], Q.shape[1]
    D = NV - 2
    gam = eos[:, 0].view(N, 1)
    pinf = eos[:, 1].view(N, 1)
    q = Q[:, :, wall]
    rho = q[:, 0]
    mom2 = (q[:, 1:1 + D] ** 2).sum(1)
    safe = torch.where(rho > 0, rho, torch.ones_like(rho))
    ap = (gam - 1.0) * (q[:, NV - 1] - 0.5 * mom2 / safe) - gam * pinf * alpha_wall
    ap = torch.where(rho > 0, ap, torch.zeros_like(ap))
    return ap.sum() * farea
