"""Seeded synthetic inputs shaped like the paper's test cases.

Initial data only: grid descriptors, material parameters, the regional level
set (unsigned distance ``phi`` and indicator ``chi``) and one primitive state
field per material. Nothing in this module computes any step of the method;
the CUDA path and the CPU oracle both take their inputs from here.

Array layouts (interior cells, x fastest):
  phi  float64 [nz, ny, nx] (squeezed to the grid's dimension)
  chi  int32   same shape
  prim float64 [N, D+2, cells]: (rho, u_0..u_{D-1}, p) of each material

Cases (the paper describes each analytically, so these stand in for its data):
  shock_tube_3   1D three-material shock tube (Sec. 3.1 / Table 1 style)
  triple_point   2D triple-point problem on [0,7]x[0,3] (Sec. 3.3)
  shock_bubbles  2D Mach-1.22 air shock on two gas bubbles (Sec. 3.5 style)
  batched_1d     256 seeded 1D multi-material Riemann problems
  shock_sphere   3D Mach-1.22 shock on one heavy sphere
  random_case    seeded random interface networks for parity tests
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

TRANSMISSIVE, REFLECTIVE, INFLOW = 0, 1, 2


@dataclasses.dataclass
class Case:
    name: str
    dim: int
    n: tuple                      # interior cells per axis (length dim)
    lo: tuple
    hi: tuple
    bc: list                      # [[lo, hi]] per axis
    gamma: list
    pinf: list
    phi: np.ndarray
    chi: np.ndarray
    prim: np.ndarray
    t_end: float
    inflow_prim: np.ndarray = None   # [3, 2, 5]
    inflow_mat: np.ndarray = None    # [3, 2]
    eos_kind: list = None            # per material: 0 stiffened gas, 1 Tait
    tait: list = None                # per material: (B, rho0, p0) of Tait's equation
    geom: int = 0                    # 0 Cartesian, 1 cylindrical (one dimension, x = radius)
    free_surface: tuple = None       # (material, rho, p0, t0, t1, p1): held ambient with pressure p(t)

    @property
    def nmat(self):
        return len(self.gamma)

    @property
    def nv(self):
        return self.dim + 2

    @property
    def cells(self):
        return int(np.prod(self.n))

    def params(self, **opts):
        """Plain dictionary of every run parameter (grid, EOS, options)."""
        ip = self.inflow_prim if self.inflow_prim is not None else np.zeros((3, 2, 5))
        im = self.inflow_mat if self.inflow_mat is not None else np.zeros((3, 2), np.int32)
        n3 = list(self.n) + [1] * (3 - self.dim)
        lo3 = list(self.lo) + [0.0] * (3 - self.dim)
        hi3 = list(self.hi) + [1.0] * (3 - self.dim)
        bc3 = [list(b) for b in self.bc] + [[0, 0]] * (3 - self.dim)
        kind = list(self.eos_kind) if self.eos_kind is not None else [0] * self.nmat
        tait = list(self.tait) if self.tait is not None else [(0.0, 0.0, 0.0)] * self.nmat
        p = dict(dim=self.dim, n=n3, lo=lo3, hi=hi3, bc=bc3, inflow_prim=np.asarray(ip, float),
                 inflow_mat=np.asarray(im, np.int32), nmat=self.nmat, gamma=list(self.gamma),
                 pinf=list(self.pinf), eos_kind=kind, tait=tait, geom=int(self.geom))
        fs = self.free_surface if self.free_surface is not None else (-1, 0.0, 0.0, 0.0, 0.0, 0.0)
        p.update(fs_mat=int(fs[0]), fs_rho=float(fs[1]), fs_p0=float(fs[2]), fs_t0=float(fs[3]),
                 fs_t1=float(fs[4]), fs_p1=float(fs[5]))
        p.update(default_options(self.dim))
        p.update(opts)
        return p


def default_options(dim):
    return dict(cfl=0.6, weno_eps=1e-6, mix_alpha=0.5, ext_sweeps=dim + 3, vel_sweeps=6,
                reinit_iters=6, scale_sep=1, reinit=1, scale_eps_h=0.0, phi_cap_h=8.0, rk_stages=3,
                literal_reduced=0, literal_normal=0, positivity=0)


def centres(n, lo, hi):
    """Cell-centre coordinate arrays, indexing 'ij' reversed to (z, y, x) order."""
    axes = [lo[d] + (np.arange(n[d]) + 0.5) * (hi[d] - lo[d]) / n[d] for d in range(len(n))]
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    return grids[::-1]  # x, y, z arrays of shape (nz, ny, nx) squeezed


def _uniform_prim(nmat, dim, cells, states):
    prim = np.zeros((nmat, dim + 2, cells))
    for m, s in enumerate(states):
        prim[m] = np.asarray(s, float)[:, None]
    return prim


def shock_tube_3(n=400):
    """Three materials A|B|C with interfaces at 0.4 and 0.6, transmissive ends."""
    (x,) = centres((n,), (0.0,), (1.0,))
    chi = np.where(x < 0.4, 0, np.where(x < 0.6, 1, 2)).astype(np.int32)
    phi = np.minimum(np.abs(x - 0.4), np.abs(x - 0.6))
    states = [(1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (0.5, 0.0, 0.1)]
    return Case("shock_tube_3", 1, (n,), (0.0,), (1.0,), [[TRANSMISSIVE, TRANSMISSIVE]],
                [1.4, 1.667, 1.4], [0.0, 0.0, 0.0], phi, chi, _uniform_prim(3, 1, n, states), 0.2)


def he_air_tube(n=200, gamma_right=1.667):
    """The paper's Case I (Sec. 3.1): helium | air | helium between walls, the
    air slab on [0.4, 0.6) as the text places it (its Table 1 prints 0.25 and
    0.5); states of Table 1, u = 0. gamma_right = 1.249 gives the
    helium-air-R22 variant of the table's footnote."""
    (x,) = centres((n,), (0.0,), (1.0,))
    chi = np.where(x < 0.4, 0, np.where(x < 0.6, 1, 2)).astype(np.int32)
    phi = np.minimum(np.abs(x - 0.4), np.abs(x - 0.6))
    states = [(0.125, 0.0, 0.1), (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)]
    return Case("he_air_tube", 1, (n,), (0.0,), (1.0,), [[REFLECTIVE, REFLECTIVE]],
                [1.667, 1.4, gamma_right], [0.0, 0.0, 0.0], phi, chi, _uniform_prim(3, 1, n, states), 0.1)


def triple_point(nx=896, ny=384):
    """Triple point on [0,7]x[0,3]: region 1 x<1, region 2 x>1 y<1.5, region 3
    x>1 y>1.5, all at rest, reflective walls (Sec. 3.3)."""
    x, y = centres((nx, ny), (0.0, 0.0), (7.0, 3.0))
    chi = np.where(x < 1.0, 0, np.where(y < 1.5, 1, 2)).astype(np.int32)
    phi = np.where(chi == 0, 1.0 - x, np.minimum(x - 1.0, np.abs(y - 1.5)))
    states = [(1.0, 0.0, 0.0, 1.0), (1.0, 0.0, 0.0, 0.1), (0.125, 0.0, 0.0, 0.1)]
    cells = nx * ny
    return Case("triple_point", 2, (nx, ny), (0.0, 0.0), (7.0, 3.0), [[REFLECTIVE] * 2, [REFLECTIVE] * 2],
                [1.5, 1.4, 1.5], [0.0, 0.0, 0.0], phi, chi.reshape(ny, nx), _uniform_prim(3, 2, cells, states), 5.0)


def normal_shock(gamma, rho0, p0, mach):
    """Post-shock state behind a shock moving into gas at rest (Rankine-Hugoniot)."""
    c0 = math.sqrt(gamma * p0 / rho0)
    s = mach * c0
    m2 = mach * mach
    p1 = p0 * (1.0 + 2.0 * gamma / (gamma + 1.0) * (m2 - 1.0))
    rho1 = rho0 * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    u1 = s * (1.0 - rho0 / rho1)
    return rho1, u1, p1, s


def shock_bubbles(nx=2048, ny=512, mach=1.22, x_shock=0.5):
    """Mach-1.22 air shock on a light (1.0, 0.5) and a heavy (1.8, 0.5) bubble
    of radius 0.25 in [0,3]x[0,1]; inflow left, transmissive right, walls."""
    x, y = centres((nx, ny), (0.0, 0.0), (3.0, 1.0))
    r = 0.25
    d1 = np.hypot(x - 1.0, y - 0.5) - r
    d2 = np.hypot(x - 1.8, y - 0.5) - r
    chi = np.where(d1 < 0, 1, np.where(d2 < 0, 2, 0)).astype(np.int32)
    phi = np.minimum(np.abs(d1), np.abs(d2))
    rho1, u1, p1, _ = normal_shock(1.4, 1.0, 1.0, mach)
    cells = nx * ny
    prim = np.zeros((3, 4, cells))
    post = (x.ravel() < x_shock)
    prim[0, 0] = np.where(post, rho1, 1.0)
    prim[0, 1] = np.where(post, u1, 0.0)
    prim[0, 3] = np.where(post, p1, 1.0)
    prim[1] = np.array([0.138, 0.0, 0.0, 1.0])[:, None]
    prim[2] = np.array([3.154, 0.0, 0.0, 1.0])[:, None]
    inflow = np.zeros((3, 2, 5))
    inflow[0, 0, :4] = (rho1, u1, 0.0, p1)
    imat = np.zeros((3, 2), np.int32)
    return Case("shock_bubbles", 2, (nx, ny), (0.0, 0.0), (3.0, 1.0), [[INFLOW, TRANSMISSIVE], [REFLECTIVE] * 2],
                [1.4, 1.648, 1.249], [0.0, 0.0, 0.0], phi, chi.reshape(ny, nx), prim, 1.2, inflow, imat)


# Tait's equation for water (Sec. 2.1) in the units of the air state rho = 1,
# p = 1: B = 3.31e8 Pa / 1e5 Pa, rho0 = 1000, p0 = 1
WATER_TAIT = (3310.0, 1000.0, 1.0)


def shock_helium_water(nx=1024, ny=256, mach=6.0, x_shock=0.5):
    """Mach-6 air shock on a helium bubble that then meets a water column
    (Sec. 3.6, Table 2 states; water by Tait's equation, gamma 7.15). The
    paper gives the geometry only in a figure: here the domain is [0,4]x[0,1]
    (its 4 x 1 root blocks), the helium bubble (radius 0.3) at (1.0, 0.5),
    the water column (radius 0.3) at (2.0, 0.5), the shock at x = 0.5; inflow
    left, transmissive right, walls top and bottom."""
    x, y = centres((nx, ny), (0.0, 0.0), (4.0, 1.0))
    d1 = np.hypot(x - 1.0, y - 0.5) - 0.3
    d2 = np.hypot(x - 2.0, y - 0.5) - 0.3
    chi = np.where(d1 < 0, 1, np.where(d2 < 0, 2, 0)).astype(np.int32)
    phi = np.minimum(np.abs(d1), np.abs(d2))
    rho1, u1, p1, _ = normal_shock(1.4, 1.0, 1.0, mach)
    cells = nx * ny
    prim = np.zeros((3, 4, cells))
    post = x.ravel() < x_shock
    prim[0, 0] = np.where(post, rho1, 1.0)
    prim[0, 1] = np.where(post, u1, 0.0)
    prim[0, 3] = np.where(post, p1, 1.0)
    prim[1] = np.array([0.138, 0.0, 0.0, 1.0])[:, None]
    prim[2] = np.array([1000.0, 0.0, 0.0, 1.0])[:, None]
    inflow = np.zeros((3, 2, 5))
    inflow[0, 0, :4] = (rho1, u1, 0.0, p1)
    return Case("shock_helium_water", 2, (nx, ny), (0.0, 0.0), (4.0, 1.0),
                [[INFLOW, TRANSMISSIVE], [REFLECTIVE] * 2], [1.4, 1.667, 7.15], [0.0, 0.0, 0.0],
                phi, chi.reshape(ny, nx), prim, 0.3, inflow, np.zeros((3, 2), np.int32),
                eos_kind=[0, 0, 1], tait=[(0.0, 0.0, 0.0), (0.0, 0.0, 0.0), WATER_TAIT])


ICF_DRIVE = (13.0, 0.04, 0.125, 0.5)   # p(t): 13 up to t = 0.04, linear to 0.5 at t = 0.125 (Sec. 3.2)


def icf_implosion(n=320, r1=0.6, r2=0.9, gamma1=5.0 / 3.0, gamma_ratio=1.0, t_end=0.3):
    """Case II (Sec. 3.2): one-dimensional cylindrical implosion on r in [0, 1].
    A light core (r < r1) inside a dense shell (r1 < r < r2); the ambient
    outside r2 is not solved and presses on the shell with the drive p(t).
    The paper takes its states from another work and prints none: core
    (0.05, 0, 0.1), shell (1, 0, 0.1), both gamma1 = 5/3 unless gamma_ratio
    (gamma2 / gamma1) is given; the ambient is held at density 1."""
    (x,) = centres((n,), (0.0,), (1.0,))
    chi = np.where(x < r1, 0, np.where(x < r2, 1, 2)).astype(np.int32)
    phi = np.minimum(np.abs(x - r1), np.abs(x - r2))
    p0 = ICF_DRIVE[0]
    states = [(0.05, 0.0, 0.1), (1.0, 0.0, 0.1), (1.0, 0.0, p0)]
    return Case("icf_implosion", 1, (n,), (0.0,), (1.0,), [[REFLECTIVE, TRANSMISSIVE]],
                [gamma1, gamma1 * gamma_ratio, gamma1], [0.0, 0.0, 0.0], phi, chi, _uniform_prim(3, 1, n, states),
                t_end, geom=1, free_surface=(2, 1.0) + ICF_DRIVE)


def icf_quarter_plane(n=64, r1=0.6, r2=0.9, t_end=0.1):
    """Case II's states on a two-dimensional Cartesian quarter plane [0, 1]^2
    (walls on the axes, transmissive outer sides): the same implosion without
    the axisymmetric metric, for cross-checks."""
    x, y = centres((n, n), (0.0, 0.0), (1.0, 1.0))
    r = np.sqrt(x ** 2 + y ** 2)
    chi = np.where(r < r1, 0, np.where(r < r2, 1, 2)).astype(np.int32)
    phi = np.minimum(np.abs(r - r1), np.abs(r - r2))
    states = [(0.05, 0.0, 0.0, 0.1), (1.0, 0.0, 0.0, 0.1), (1.0, 0.0, 0.0, ICF_DRIVE[0])]
    g = 5.0 / 3.0
    return Case("icf_quarter_plane", 2, (n, n), (0.0, 0.0), (1.0, 1.0),
                [[REFLECTIVE, TRANSMISSIVE], [REFLECTIVE, TRANSMISSIVE]], [g, g, g], [0.0, 0.0, 0.0],
                phi, chi, _uniform_prim(3, 2, n * n, states), t_end, free_surface=(2, 1.0) + ICF_DRIVE)


def icf_shell_study(n=1280, count=256, t_end=0.3):
    """Case II's study of the shell thickness (Sec. 3.2): instances with
    r2 - r1 spread over [0.05, 0.3] (r1 = 0.6, gamma2 / gamma1 = 1)."""
    return [icf_implosion(n, r1=0.6, r2=0.6 + 0.05 + 0.25 * k / max(count - 1, 1), t_end=t_end)
            for k in range(count)]


def water_pulse(n=400, amp=1e-4):
    """One-dimensional water at rest (Tait's equation) with a small Gaussian
    density pulse and the matching Tait pressure: linear acoustics."""
    (x,) = centres((n,), (0.0,), (1.0,))
    B, rho0, p0 = WATER_TAIT
    rho = rho0 * (1.0 + amp * np.exp(-((x - 0.5) / 0.03) ** 2))
    p = B * (rho / rho0) ** 7.15 - B + p0
    prim = np.stack([rho, np.zeros(n), p])[None]
    return Case("water_pulse", 1, (n,), (0.0,), (1.0,), [[TRANSMISSIVE, TRANSMISSIVE]], [7.15], [0.0],
                np.full(n, 10.0), np.zeros(n, np.int32), prim, 0.05, eos_kind=[1], tait=[WATER_TAIT])


def shock_sphere(n=(256, 128, 128), mach=1.22, x_shock=0.25):
    """3D Mach-1.22 air shock on a heavy sphere of radius 0.2 at (0.5,0.5,0.5)
    in [0,2]x[0,1]^2; inflow left, transmissive right, walls in y and z."""
    x, y, z = centres(n, (0.0, 0.0, 0.0), (2.0, 1.0, 1.0))
    d = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2) - 0.2
    chi = np.where(d < 0, 1, 0).astype(np.int32)
    phi = np.abs(d)
    rho1, u1, p1, _ = normal_shock(1.4, 1.0, 1.0, mach)
    cells = int(np.prod(n))
    prim = np.zeros((2, 5, cells))
    post = x.ravel() < x_shock
    prim[0, 0] = np.where(post, rho1, 1.0)
    prim[0, 1] = np.where(post, u1, 0.0)
    prim[0, 4] = np.where(post, p1, 1.0)
    prim[1] = np.array([3.154, 0, 0, 0, 1.0])[:, None]
    inflow = np.zeros((3, 2, 5))
    inflow[0, 0, :5] = (rho1, u1, 0.0, 0.0, p1)
    return Case("shock_sphere", 3, tuple(n), (0.0, 0.0, 0.0), (2.0, 1.0, 1.0),
                [[INFLOW, TRANSMISSIVE], [REFLECTIVE] * 2, [REFLECTIVE] * 2], [1.4, 1.249], [0.0, 0.0],
                phi, chi.reshape(n[2], n[1], n[0]), prim, 1.0, inflow, np.zeros((3, 2), np.int32))


def _loguniform(rng, a, b, size=None):
    return np.exp(rng.uniform(math.log(a), math.log(b), size))


def riemann_1d(rng, ncell=None, nmat=None):
    """One seeded 1D multi-material Riemann problem (cell count log-uniform in
    [200, 20000], 2-4 materials, interfaces uniform in (0.1, 0.9) at least 4
    cells apart; rho log-U[0.1,10], p log-U[0.01,100], u U[-1,1],
    gamma U[1.1,3], pinf U[0,5]); transmissive ends, t_end 0.1."""
    if ncell is None:
        ncell = int(round(math.exp(rng.uniform(math.log(200), math.log(20000)))))
    if nmat is None:
        nmat = int(rng.integers(2, 5))
    h = 1.0 / ncell
    while True:
        pos = np.sort(rng.uniform(0.1, 0.9, nmat - 1))
        if nmat == 2 or np.min(np.diff(pos)) >= 4 * h:
            break
    (x,) = centres((ncell,), (0.0,), (1.0,))
    chi = np.searchsorted(pos, x).astype(np.int32)
    phi = np.min(np.abs(x[:, None] - pos[None, :]), axis=1)
    rho = _loguniform(rng, 0.1, 10.0, nmat)
    p = _loguniform(rng, 0.01, 100.0, nmat)
    u = rng.uniform(-1.0, 1.0, nmat)
    gamma = rng.uniform(1.1, 3.0, nmat)
    pinf = rng.uniform(0.0, 5.0, nmat)
    states = [(rho[m], u[m], p[m]) for m in range(nmat)]
    return Case("riemann_1d", 1, (ncell,), (0.0,), (1.0,), [[TRANSMISSIVE, TRANSMISSIVE]], list(gamma),
                list(pinf), phi, chi, _uniform_prim(nmat, 1, ncell, states), 0.1)


def batched_1d(count=256, seed=20170403):
    rng = np.random.default_rng(seed)
    return [riemann_1d(rng) for _ in range(count)]


def random_case(dim, n, nmat, seed, kinds=("disc", "plane"), at_rest=False, p_equal=False):
    """Seeded random interface network: material 0 fills the box, then random
    discs/spheres and half-spaces of materials 1..nmat-1 are painted over it.
    phi is the distance to the nearest cell-centre-resolved interface,
    computed from the analytic shapes."""
    rng = np.random.default_rng(seed)
    lo = (0.0,) * dim
    hi = tuple(float(n[d]) / float(max(n)) for d in range(dim))
    X = centres(n, lo, hi)
    shape = X[0].shape
    chi = np.zeros(shape, np.int32)
    for m in range(1, nmat):
        kind = kinds[int(rng.integers(len(kinds)))]
        if kind == "disc":
            c = [rng.uniform(0.25, 0.75) * hi[d] for d in range(dim)]
            r = rng.uniform(0.12, 0.3) * min(hi)
            d = np.sqrt(sum((X[k] - c[k]) ** 2 for k in range(dim))) - r
        else:
            nrm = rng.normal(size=dim)
            nrm /= np.linalg.norm(nrm)
            off = rng.uniform(0.3, 0.7)
            d = sum(nrm[k] * (X[k] / hi[k] - 0.5) for k in range(dim)) - (off - 0.5)
            d = d * min(hi)
        chi = np.where(d < 0, m, chi)
    # unsigned distance to the interface network, taken as the set of
    # mid-points between face neighbours of different indicator
    phi = _distance_to_network(chi, [(hi[d] - lo[d]) / n[d] for d in range(dim)])
    gamma = list(rng.uniform(1.2, 2.5, nmat))
    pinf = list(rng.uniform(0.0, 2.0, nmat))
    prim = np.zeros((nmat, dim + 2, int(np.prod(n))))
    for m in range(nmat):
        rho = _loguniform(rng, 0.3, 3.0)
        p = 1.0 if p_equal else _loguniform(rng, 0.3, 3.0)
        vel = np.zeros(dim) if at_rest else rng.uniform(-0.3, 0.3, dim)
        prim[m] = np.array([rho, *vel, p])[:, None]
    bc = [[int(rng.integers(2)), int(rng.integers(2))] for _ in range(dim)]
    return Case(f"random_{dim}d_{nmat}m_{seed}", dim, tuple(n), lo, hi, bc, gamma, pinf, phi, chi, prim, 1.0)


def _distance_to_network(chi, h):
    """Unsigned distance from each cell centre to the set of mid-points between
    face-adjacent cells of different indicator (brute force; small grids)."""
    dim = chi.ndim
    pts = []
    idx = np.indices(chi.shape).reshape(dim, -1).T  # (z, y, x) order
    for ax in range(dim):
        a = np.take(chi, range(chi.shape[ax] - 1), axis=ax)
        b = np.take(chi, range(1, chi.shape[ax]), axis=ax)
        diff = np.argwhere(a != b).astype(float)
        diff[:, ax] += 0.5
        pts.append(diff)
    pts = np.concatenate(pts) if pts else np.zeros((0, dim))
    hs = np.array(h[::-1])  # (z, y, x) spacing
    if len(pts) == 0:
        return np.full(chi.shape, 8.0 * min(h))
    P = pts * hs
    C = idx * hs
    out = np.empty(len(C))
    for s in range(0, len(C), 4096):
        dd = C[s:s + 4096, None, :] - P[None, :, :]
        out[s:s + 4096] = np.sqrt((dd ** 2).sum(-1)).min(1)
    return out.reshape(chi.shape)


def scale_sep_demo(kind="filament", n=10):
    """Unit square, h = 0.1: a filament of thickness 1.2h between two
    materials, or a droplet of radius 1.5h touching an interface (Sec. 2.3.3)."""
    x, y = centres((n, n), (0.0, 0.0), (1.0, 1.0))
    h = 1.0 / n
    if kind == "filament":
        y0, y1 = 0.5 - 0.6 * h, 0.5 + 0.6 * h
        chi = np.where(y < y0, 0, np.where(y < y1, 2, 1)).astype(np.int32)
        phi = np.minimum(np.abs(y - y0), np.abs(y - y1))
    else:
        r = 1.5 * h
        cx, cy = 0.5, 0.5 + 0.5 * h
        dd = np.hypot(x - cx, y - cy) - r
        dl = y - 0.3
        chi = np.where(dd < 0, 2, np.where(dl < 0, 0, 1)).astype(np.int32)
        phi = np.minimum(np.abs(dd), np.abs(dl))
    prim = _uniform_prim(3, 2, n * n, [(1.0, 0, 0, 1.0), (0.5, 0, 0, 1.0), (2.0, 0, 0, 1.0)])
    return Case("scale_sep_" + kind, 2, (n, n), (0.0, 0.0), (1.0, 1.0), [[REFLECTIVE] * 2, [REFLECTIVE] * 2],
                [1.4, 1.4, 1.4], [0.0, 0.0, 0.0], phi, chi, prim, 1.0)
