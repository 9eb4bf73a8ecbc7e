"""ctypes wrapper around the plain FP64 C oracle (libmsf_oracle.so).

Test infrastructure only: tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline leg use it. The product path never imports this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "msf_oracle.c")
HDR = os.path.join(HERE, "msf_oracle.h")
LIB = os.path.join(HERE, "libmsf_oracle.so")
LIB_OMP = os.path.join(HERE, "libmsf_oracle_omp.so")
MAXM = 8
COUNTERS = ["cut", "multi", "corrected", "small", "mixfail", "merge", "oddball", "steps"]


def build(force=False, openmp=False):
    """Compile the oracle with gcc (no FMA contraction, no fast-math); with
    openmp=True the loops over cells run on all host cores (same results)."""
    out = LIB_OMP if openmp else LIB
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    if openmp:
        cmd.append("-fopenmp")
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(cmd + ["-o", tmp, SRC, "-lm"], check=True)
    os.replace(tmp, out)
    return out


class Params(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("n", C.c_int32 * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("bc", (C.c_int32 * 2) * 3), ("inflow_prim", ((C.c_double * 5) * 2) * 3),
        ("inflow_mat", (C.c_int32 * 2) * 3), ("nmat", C.c_int32),
        ("gamma", C.c_double * MAXM), ("pinf", C.c_double * MAXM),
        ("cfl", C.c_double), ("weno_eps", C.c_double), ("mix_alpha", C.c_double),
        ("ext_sweeps", C.c_int32), ("vel_sweeps", C.c_int32), ("reinit_iters", C.c_int32),
        ("scale_sep", C.c_int32), ("reinit", C.c_int32),
        ("scale_eps_h", C.c_double), ("phi_cap_h", C.c_double), ("rk_stages", C.c_int32),
        ("eos_kind", C.c_int32 * MAXM), ("tait_B", C.c_double * MAXM),
        ("tait_rho0", C.c_double * MAXM), ("tait_p0", C.c_double * MAXM),
        ("geom", C.c_int32), ("fs_mat", C.c_int32), ("fs_rho", C.c_double), ("fs_p0", C.c_double),
        ("fs_t0", C.c_double), ("fs_t1", C.c_double), ("fs_p1", C.c_double),
        ("literal_reduced", C.c_int32), ("literal_normal", C.c_int32), ("positivity", C.c_int32),
    ]


_libs = {}


def lib(openmp=False):
    if openmp not in _libs:
        L = C.CDLL(build(openmp=openmp))
        P = C.c_void_p
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        L.orc_create.restype = P
        L.orc_create.argtypes = [C.POINTER(Params)]
        L.orc_destroy.argtypes = [P]
        L.orc_set_levelset.argtypes = [P, dp, ip, dp]
        L.orc_step.argtypes = [P, C.c_int32, C.c_double]
        L.orc_get_state.argtypes = [P, dp, dp, dp, ip, dp]
        L.orc_set_state.argtypes = [P, dp, dp, ip, C.c_double]
        u8p = C.POINTER(C.c_uint8)
        L.orc_ncell.restype = C.c_long
        L.orc_ncell.argtypes = [P]
        L.orc_threads.restype = C.c_int
        L.orc_threads.argtypes = []
        L.orc_step_taped.argtypes = [P, C.c_double, dp, u8p, dp]
        L.orc_replay_step.argtypes = [P, dp, u8p, C.c_double]
        L.orc_set_conserved.argtypes = [P, dp]
        L.orc_mix_only.argtypes = [P]
        L.orc_scale_sep_only.argtypes = [P]
        L.orc_totals.argtypes = [P, dp, dp]
        L.orc_counters.argtypes = [P, C.POINTER(C.c_int64)]
        L.orc_last_dt.restype = C.c_double
        L.orc_last_dt.argtypes = [P]
        L.orc_error.argtypes = [P]
        L.orc_debug_field.argtypes = [P, C.c_int32, dp]
        L.orc_weno5.restype = C.c_double
        L.orc_weno5.argtypes = [C.c_double] * 6
        L.orc_hllc.argtypes = [dp, dp, dp, dp, dp, dp]
        for f in ("orc_seg_frac", "orc_tri_frac", "orc_tet_frac"):
            getattr(L, f).restype = C.c_double
        L.orc_seg_frac.argtypes = [C.c_double] * 2
        L.orc_tri_frac.argtypes = [C.c_double] * 3
        L.orc_tet_frac.argtypes = [C.c_double] * 4
        _libs[openmp] = L
    return _libs[openmp]


def threads(openmp=False):
    """Threads the oracle's loops over cells use."""
    return lib(openmp).orc_threads()


def make_params(p: dict) -> Params:
    s = Params()
    s.dim = p["dim"]
    for d in range(3):
        s.n[d] = int(p["n"][d])
        s.lo[d] = float(p["lo"][d])
        s.hi[d] = float(p["hi"][d])
        for side in range(2):
            s.bc[d][side] = int(p["bc"][d][side])
            s.inflow_mat[d][side] = int(p["inflow_mat"][d][side])
            for v in range(5):
                s.inflow_prim[d][side][v] = float(p["inflow_prim"][d][side][v])
    s.nmat = p["nmat"]
    for m in range(p["nmat"]):
        s.gamma[m] = p["gamma"][m]
        s.pinf[m] = p["pinf"][m]
        s.eos_kind[m] = int(p["eos_kind"][m])
        s.tait_B[m], s.tait_rho0[m], s.tait_p0[m] = (float(x) for x in p["tait"][m])
    for k in ("cfl", "weno_eps", "mix_alpha", "scale_eps_h", "phi_cap_h"):
        setattr(s, k, float(p[k]))
    for k in ("ext_sweeps", "vel_sweeps", "reinit_iters", "scale_sep", "reinit", "rk_stages"):
        setattr(s, k, int(p[k]))
    s.geom = int(p.get("geom", 0))
    s.fs_mat = int(p.get("fs_mat", -1))
    for k in ("fs_rho", "fs_p0", "fs_t0", "fs_t1", "fs_p1"):
        setattr(s, k, float(p.get(k, 0.0)))
    s.literal_reduced = int(p.get("literal_reduced", 0))
    s.literal_normal = int(p.get("literal_normal", 0))
    s.positivity = int(p.get("positivity", 0))
    return s


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


class Oracle:
    """One simulation instance on the CPU oracle."""

    def __init__(self, case, openmp=False, **opts):
        self.case = case
        self._L = lib(openmp)
        self.p = case.params(**opts)
        self._params = make_params(self.p)
        self.h = self._L.orc_create(C.byref(self._params))
        if not self.h:
            raise ValueError("oracle: invalid parameters")
        self.N, self.NV, self.cells = case.nmat, case.nv, case.cells
        phi = np.ascontiguousarray(case.phi, np.float64).ravel()
        chi = np.ascontiguousarray(case.chi, np.int32).ravel()
        prim = np.ascontiguousarray(case.prim, np.float64)
        self._L.orc_set_levelset(self.h, _dp(phi), _ip(chi), _dp(prim))

    def __del__(self):
        if getattr(self, "h", None):
            self._L.orc_destroy(self.h)
            self.h = None

    def step(self, n_steps, t_end=np.inf):
        return self._L.orc_step(self.h, int(n_steps), float(t_end))

    def state(self):
        Q = np.zeros((self.N, self.NV, self.cells))
        alpha = np.zeros((self.N, self.cells))
        phi = np.zeros(self.cells)
        chi = np.zeros(self.cells, np.int32)
        t = np.zeros(1)
        self._L.orc_get_state(self.h, _dp(Q), _dp(alpha), _dp(phi), _ip(chi), _dp(t))
        return dict(Q=Q, alpha=alpha, phi=phi, chi=chi, t=float(t[0]))

    def set_state(self, Q, phi, chi, t):
        Q = np.ascontiguousarray(Q, np.float64)
        phi = np.ascontiguousarray(phi, np.float64).ravel()
        chi = np.ascontiguousarray(chi, np.int32).ravel()
        self._L.orc_set_state(self.h, _dp(Q), _dp(phi), _ip(chi), float(t))

    def set_conserved(self, Q):
        """Replace the conserved state of the interior cells ([N][NV][cells])."""
        Q = np.ascontiguousarray(Q, np.float64)
        self._L.orc_set_conserved(self.h, _dp(Q))

    def mix_only(self):
        """The mixing pass alone on the current state and geometry."""
        self._L.orc_mix_only(self.h)

    def scale_sep_only(self):
        """The scale-separation pass alone on the current level set and geometry."""
        self._L.orc_scale_sep_only(self.h)

    def step_taped(self, t_end=np.inf):
        """One step that records its replay tape (the level set at the start of
        each stage and after the last level-set stage, and the time step);
        None when t >= t_end."""
        nc = self._L.orc_ncell(self.h)
        phi = np.zeros((4, nc))
        chi = np.zeros((4, nc), np.uint8)
        dt = np.zeros(1)
        rc = self._L.orc_step_taped(self.h, float(t_end), _dp(phi),
                                  chi.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(dt))
        if rc < 0:
            return None
        return dict(phi=phi, chi=chi, dt=float(dt[0]), err=rc)

    def replay_step(self, tape):
        """One step from the current conserved state with the interface
        evolution frozen to a tape of step_taped."""
        return self._L.orc_replay_step(self.h, _dp(tape["phi"]),
                                     tape["chi"].ctypes.data_as(C.POINTER(C.c_uint8)), float(tape["dt"]))

    def totals(self):
        tot = np.zeros((self.N, self.NV))
        led = np.zeros((self.N, self.NV))
        self._L.orc_totals(self.h, _dp(tot), _dp(led))
        return tot, led

    def counters(self):
        c = np.zeros(len(COUNTERS), np.int64)
        self._L.orc_counters(self.h, c.ctypes.data_as(C.POINTER(C.c_int64)))
        return dict(zip(COUNTERS, c.tolist()))

    def error(self):
        return self._L.orc_error(self.h)

    def last_dt(self):
        return self._L.orc_last_dt(self.h)

    def debug(self, which):
        sizes = {0: self.N, 1: self.N * self.NV, 2: self.N * self.NV, 3: 3, 4: 1, 5: 1, 6: 3 * self.N, 7: 3 * self.N}
        out = np.zeros(sizes[which] * self.cells)
        self._L.orc_debug_field(self.h, int(which), _dp(out))
        return out


def weno5(a, b, c, d, e, eps=1e-6):
    return lib().orc_weno5(a, b, c, d, e, eps)


def hllc(wl, wr, eosl, eosr):
    """Star velocity and pressure for w = (rho, u_n, p) and eos = (gamma,
    pinf[, kind]); kind 1 marks Tait's equation with pinf = B - p0."""
    us, ps = np.zeros(1), np.zeros(1)
    eosl = list(eosl) + [0.0] * (3 - len(eosl))
    eosr = list(eosr) + [0.0] * (3 - len(eosr))
    arrs = [np.asarray(x, np.float64) for x in (wl, wr, eosl, eosr)]
    lib().orc_hllc(*[_dp(a) for a in arrs], _dp(us), _dp(ps))
    return float(us[0]), float(ps[0])


def seg_frac(a, b):
    return lib().orc_seg_frac(a, b)


def tri_frac(a, b, c):
    return lib().orc_tri_frac(a, b, c)


def tet_frac(a, b, c, d):
    return lib().orc_tet_frac(a, b, c, d)
