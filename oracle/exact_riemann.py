"""Exact Riemann solver for two stiffened gases (different gamma, pinf per
side) and the composed exact solution of the three-material shock tube.

Test infrastructure (pins the oracle). The stiffened-gas Riemann problem
reduces to the ideal-gas one in the shifted pressure p + pinf: the
Rankine-Hugoniot and isentrope relations are the textbook ones written in
that variable. The star pressure solves f_L(p) + f_R(p) + u_R - u_L = 0.
"""
from __future__ import annotations

import math

import numpy as np


class Side:
    def __init__(self, rho, u, p, gamma, pinf):
        self.rho, self.u, self.p, self.g, self.pi = float(rho), float(u), float(p), float(gamma), float(pinf)
        self.c = math.sqrt(self.g * (self.p + self.pi) / self.rho)

    def f(self, ps):
        """Velocity jump across the wave that connects this state to pressure ps."""
        g, pb, psb = self.g, self.p + self.pi, ps + self.pi
        if ps > self.p:
            A = 2.0 / ((g + 1.0) * self.rho)
            B = (g - 1.0) / (g + 1.0) * pb
            return (ps - self.p) * math.sqrt(A / (psb + B))
        return 2.0 * self.c / (g - 1.0) * ((psb / pb) ** ((g - 1.0) / (2.0 * g)) - 1.0)

    def df(self, ps):
        g, pb, psb = self.g, self.p + self.pi, ps + self.pi
        if ps > self.p:
            A = 2.0 / ((g + 1.0) * self.rho)
            B = (g - 1.0) / (g + 1.0) * pb
            return math.sqrt(A / (B + psb)) * (1.0 - (ps - self.p) / (2.0 * (B + psb)))
        return 1.0 / (self.rho * self.c) * (psb / pb) ** (-(g + 1.0) / (2.0 * g))

    def star_rho(self, ps):
        g, pb, psb = self.g, self.p + self.pi, ps + self.pi
        if ps > self.p:
            r = (g - 1.0) / (g + 1.0)
            return self.rho * (psb / pb + r) / (r * psb / pb + 1.0)
        return self.rho * (psb / pb) ** (1.0 / g)

    def shock_speed(self, ps, sign):
        g, pb, psb = self.g, self.p + self.pi, ps + self.pi
        return self.u + sign * self.c * math.sqrt((g + 1.0) / (2.0 * g) * psb / pb + (g - 1.0) / (2.0 * g))


class Riemann:
    """Exact solution of one Riemann problem; sample(xi) with xi = x/t."""

    def __init__(self, left: Side, right: Side):
        self.L, self.R = left, right
        du = right.u - left.u
        # bracket then Newton with bisection safeguard
        fa = lambda p: left.f(p) + right.f(p) + du
        a = -min(left.pi, right.pi) + 1e-12
        b = max(left.p, right.p, 1.0)
        while fa(b) < 0:
            b *= 2.0
        p = 0.5 * (left.p + right.p)
        if not (a < p < b):
            p = 0.5 * (a + b)
        for _ in range(200):
            fp = fa(p)
            if fp > 0:
                b = p
            else:
                a = p
            d = left.df(p) + right.df(p)
            pn = p - fp / d if d > 0 else 0.5 * (a + b)
            if not (a < pn < b):
                pn = 0.5 * (a + b)
            if abs(pn - p) <= 1e-15 * max(1.0, abs(p)):
                p = pn
                break
            p = pn
        self.ps = p
        self.us = 0.5 * (left.u + right.u) + 0.5 * (right.f(p) - left.f(p))
        self.rsl = left.star_rho(p)
        self.rsr = right.star_rho(p)

    def residual(self):
        return self.L.f(self.ps) + self.R.f(self.ps) + self.R.u - self.L.u

    def wave_speeds(self):
        """(leftmost, rightmost) signal speeds."""
        L, R, ps = self.L, self.R, self.ps
        sl = L.shock_speed(ps, -1.0) if ps > L.p else L.u - L.c
        sr = R.shock_speed(ps, +1.0) if ps > R.p else R.u + R.c
        return sl, sr

    def left_wave(self):
        """(kind, speed or (head, tail)) of the left-going wave."""
        L, ps = self.L, self.ps
        if ps > L.p:
            return "shock", L.shock_speed(ps, -1.0)
        cs = L.c * ((ps + L.pi) / (L.p + L.pi)) ** ((L.g - 1.0) / (2.0 * L.g))
        return "fan", (L.u - L.c, self.us - cs)

    def right_wave(self):
        R, ps = self.R, self.ps
        if ps > R.p:
            return "shock", R.shock_speed(ps, +1.0)
        cs = R.c * ((ps + R.pi) / (R.p + R.pi)) ** ((R.g - 1.0) / (2.0 * R.g))
        return "fan", (self.us + cs, R.u + R.c)

    def sample(self, xi):
        """(rho, u, p, side) at self-similar coordinate xi; side 0 = left material."""
        L, R = self.L, self.R
        if xi <= self.us:
            kind, sp = self.left_wave()
            if kind == "shock":
                return (L.rho, L.u, L.p, 0) if xi < sp else (self.rsl, self.us, self.ps, 0)
            head, tail = sp
            if xi <= head:
                return (L.rho, L.u, L.p, 0)
            if xi >= tail:
                return (self.rsl, self.us, self.ps, 0)
            g = L.g
            u = 2.0 / (g + 1.0) * (L.c + 0.5 * (g - 1.0) * L.u + xi)
            c = 2.0 / (g + 1.0) * (L.c + 0.5 * (g - 1.0) * (L.u - xi))
            rho = L.rho * (c / L.c) ** (2.0 / (g - 1.0))
            pb = (L.p + L.pi) * (c / L.c) ** (2.0 * g / (g - 1.0))
            return (rho, u, pb - L.pi, 0)
        kind, sp = self.right_wave()
        if kind == "shock":
            return (R.rho, R.u, R.p, 1) if xi > sp else (self.rsr, self.us, self.ps, 1)
        tail, head = sp
        if xi >= head:
            return (R.rho, R.u, R.p, 1)
        if xi <= tail:
            return (self.rsr, self.us, self.ps, 1)
        g = R.g
        u = 2.0 / (g + 1.0) * (-R.c + 0.5 * (g - 1.0) * R.u + xi)
        c = 2.0 / (g + 1.0) * (R.c - 0.5 * (g - 1.0) * (R.u - xi))
        rho = R.rho * (c / R.c) ** (2.0 / (g - 1.0))
        pb = (R.p + R.pi) * (c / R.c) ** (2.0 * g / (g - 1.0))
        return (rho, u, pb - R.pi, 1)


def rankine_hugoniot_residual(side: Side, rho2, u2, p2, s):
    """Mass, momentum and energy flux jumps across a discontinuity of speed s."""
    def flux(r, u, p):
        E = (p + side.g * side.pi) / (side.g - 1.0) + 0.5 * r * u * u
        return np.array([r * (u - s), r * u * (u - s) + p, E * (u - s) + p * u])
    return flux(side.rho, side.u, side.p) - flux(rho2, u2, p2)


def three_material_solution(states, gammas, pinfs, x1, x2, t):
    """Exact solution of A|B|C with interfaces x1 < x2, valid while only the
    first three wave interactions have occurred: RP1 at x1 (t=0), RP2 when
    RP1's right shock reaches x2, RP3 when RP2's reflected wave meets the A|B
    contact. Requires that B and C start in mechanical equilibrium.
    Returns a sampler x -> (rho, u, p, material) and the event times."""
    A = Side(*states[0], gammas[0], pinfs[0])
    B = Side(*states[1], gammas[1], pinfs[1])
    Cc = Side(*states[2], gammas[2], pinfs[2])
    assert abs(B.p - Cc.p) < 1e-15 and abs(B.u - Cc.u) < 1e-15
    rp1 = Riemann(A, B)
    k, s1 = rp1.right_wave()
    assert k == "shock"
    t1 = (x2 - x1) / s1
    Bs = Side(rp1.rsr, rp1.us, rp1.ps, gammas[1], pinfs[1])
    rp2 = Riemann(Bs, Cc)
    k2, s2 = rp2.left_wave()
    s2l = s2 if k2 == "shock" else s2[0]
    # reflected wave (its leading edge) meets the A|B contact x = x1 + us1 t
    t2 = (x2 - s2l * t1 - x1) / (rp1.us - s2l)
    xm = x1 + rp1.us * t2
    As = Side(rp1.rsl, rp1.us, rp1.ps, gammas[0], pinfs[0])
    Bss = Side(rp2.rsl, rp2.us, rp2.ps, gammas[1], pinfs[1])
    rp3 = Riemann(As, Bss)
    assert k2 == "shock", "the composition below assumes a reflected shock"
    # next event: RP3's right wave reaches RP2's contact
    _, s3r = rp3.wave_speeds()
    t3 = (x2 - rp2.us * t1 - xm + s3r * t2) / (s3r - rp2.us)
    assert t <= t3, "requested time is past the third interaction"
    assert t >= t2, "composition is written for t after the second interaction"

    def sample(x):
        xi1 = (x - x1) / t
        s3l, s3r_ = rp3.wave_speeds()
        x3l = xm + s3l * (t - t2)
        x3r = xm + s3r_ * (t - t2)
        xc2 = x2 + rp2.us * (t - t1)
        xs2 = x2 + (rp2.right_wave()[1] if rp2.right_wave()[0] == "shock" else rp2.right_wave()[1][1]) * (t - t1)
        if x < x3l:
            r, u, p, side = rp1.sample(xi1)
            return r, u, p, 0
        if x <= x3r:
            r, u, p, side = rp3.sample((x - xm) / (t - t2))
            return r, u, p, side
        if x < xc2:
            return Bss.rho, Bss.u, Bss.p, 1
        if x < xs2:
            r, u, p, side = rp2.sample((x - x2) / (t - t1))
            return r, u, p, 2
        return Cc.rho, Cc.u, Cc.p, 2

    return sample, dict(t1=t1, t2=t2, t3=t3, rp1=rp1, rp2=rp2, rp3=rp3)


def cell_average(sample, lo, hi, n, sub=64):
    """Cell averages of a sampled profile (sub-sampled midpoint rule)."""
    h = (hi - lo) / n
    out = np.zeros((n, 3))
    for i in range(n):
        xs = lo + (i + (np.arange(sub) + 0.5) / sub) * h
        vals = np.array([sample(x)[:3] for x in xs])
        out[i] = vals.mean(0)
    return out
