"""Python binding of the msf C ABI (include/msf.h): argument marshalling only.

Every step of the method runs in the CUDA library libmsf.so built in this
package directory; there is no CPU fallback. Importing this module without
the built library raises ImportError.

The functions below carry the C names; ``Solver`` wraps one context. Arrays
may be numpy arrays (host) or torch CUDA tensors (device, passed by pointer);
torch is used only for device memory and the current stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmsf.so")

MSF_OK, MSF_EINVAL, MSF_ENOMEM, MSF_ECUDA, MSF_ENONFINITE, MSF_ENEGATIVE, MSF_EBAND, MSF_ETIMEOUT, MSF_ESTATE, \
    MSF_EUNSUPPORTED = range(10)
STATUS_NAMES = ["MSF_OK", "MSF_EINVAL", "MSF_ENOMEM", "MSF_ECUDA", "MSF_ENONFINITE", "MSF_ENEGATIVE", "MSF_EBAND",
                "MSF_ETIMEOUT", "MSF_ESTATE", "MSF_EUNSUPPORTED"]
MSF_HOST, MSF_DEVICE = 0, 1
MSF_FP64, MSF_FP32_BULK = 0, 1
MAXMAT = 8
NSTATS = 8
COUNTERS = ["cut", "multi", "corrected", "small", "mixfail", "merge", "oddball", "steps"]


class msf_grid(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n", C.c_int32 * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("bc", (C.c_int32 * 2) * 3), ("inflow_prim", ((C.c_double * 5) * 2) * 3),
                ("inflow_mat", (C.c_int32 * 2) * 3), ("geom", C.c_int32), ("free_surface", C.c_int32),
                ("fs_mat", C.c_int32), ("fs_rho", C.c_double), ("fs_p0", C.c_double), ("fs_t0", C.c_double),
                ("fs_t1", C.c_double), ("fs_p1", C.c_double)]


class msf_eos(C.Structure):
    _fields_ = [("gamma", C.c_double), ("pinf", C.c_double), ("kind", C.c_int32), ("tait_B", C.c_double),
                ("tait_rho0", C.c_double), ("tait_p0", C.c_double)]


MSF_EOS_STIFFENED, MSF_EOS_TAIT = 0, 1


def make_eos(p: dict, m: int) -> msf_eos:
    """EOS of material m from a case parameter dictionary (cases.Case.params)."""
    B, rho0, p0 = p["tait"][m]
    return msf_eos(p["gamma"][m], p["pinf"][m], int(p["eos_kind"][m]), B, rho0, p0)


class msf_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("cfl", C.c_double), ("weno_eps", C.c_double), ("mix_alpha", C.c_double),
                ("ext_sweeps", C.c_int32), ("vel_sweeps", C.c_int32), ("reinit_iters", C.c_int32),
                ("scale_sep", C.c_int32), ("reinit", C.c_int32), ("scale_eps_h", C.c_double),
                ("phi_cap_h", C.c_double), ("use_graph", C.c_int32), ("profile", C.c_int32),
                ("batch_mode", C.c_int32), ("stream", C.c_void_p), ("rk_stages", C.c_int32),
                ("literal_reduced", C.c_int32), ("literal_normal", C.c_int32), ("positivity", C.c_int32)]


class MsfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmsf.so is not built ({LIB_PATH}); run paper_1704_00519_gb300/build.py "
                          "(or __graft_entry__.build())")
    lib = C.CDLL(LIB_PATH)
    P, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32)
    sig = {
        "msf_default_options": ([C.c_int32, C.POINTER(msf_options)], C.c_int),
        "msf_create": ([C.POINTER(msf_grid), C.c_int32, C.c_int32, C.POINTER(msf_eos), C.POINTER(msf_options),
                        C.POINTER(C.c_void_p)], C.c_int),
        "msf_destroy": ([P], C.c_int),
        "msf_set_levelset": ([P, C.c_int32, P, P, P, C.c_int32], C.c_int),
        "msf_step": ([P, C.c_int32, C.c_double, C.c_int32], C.c_int),
        "msf_totals": ([P, C.c_int32, dp, dp], C.c_int),
        "msf_adjoint_step": ([P, P, P, P, dp, dp], C.c_int),
        "msf_tape_bytes": ([P, C.POINTER(C.c_int64)], C.c_int),
        "msf_step_taped": ([P, P, C.c_double], C.c_int),
        "msf_replay_step": ([P, P], C.c_int),
        "msf_set_conserved": ([P, C.c_int32, P, C.c_int32], C.c_int),
        "msf_get_state": ([P, C.c_int32, P, P, P, P, dp, C.c_int32], C.c_int),
        "msf_set_state": ([P, C.c_int32, P, P, P, C.c_double, C.c_int32], C.c_int),
        "msf_stats": ([P, C.POINTER(C.c_int64)], C.c_int),
        "msf_last_dt": ([P, C.c_int32, dp], C.c_int),
        "msf_debug_field": ([P, C.c_int32, C.c_int32, dp], C.c_int),
        "msf_launches_per_step": ([P, C.POINTER(C.c_int64)], C.c_int),
        "msf_profile_read": ([P, dp], C.c_int),
        "msf_batch_block_size": ([P, C.POINTER(C.c_int32)], C.c_int),
        "msf_instance_info": ([P, C.c_int32, dp, C.POINTER(C.c_int64), C.POINTER(C.c_int32)], C.c_int),
        "msf_cfl_dt_noalloc": ([P, C.c_int64, C.c_int32, C.POINTER(msf_eos), dp, C.c_double, P, P], C.c_int),
        "msf_fma_peak": ([C.c_int32, dp, P], C.c_int),
        "msf_last_error": ([P], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()

# the C entry points, under their own names
msf_default_options = _lib.msf_default_options
msf_create = _lib.msf_create
msf_destroy = _lib.msf_destroy
msf_set_levelset = _lib.msf_set_levelset
msf_step = _lib.msf_step
msf_totals = _lib.msf_totals
msf_adjoint_step = _lib.msf_adjoint_step
msf_tape_bytes = _lib.msf_tape_bytes
msf_step_taped = _lib.msf_step_taped
msf_replay_step = _lib.msf_replay_step
msf_set_conserved = _lib.msf_set_conserved
msf_get_state = _lib.msf_get_state
msf_set_state = _lib.msf_set_state
msf_stats = _lib.msf_stats
msf_last_dt = _lib.msf_last_dt
msf_debug_field = _lib.msf_debug_field
msf_launches_per_step = _lib.msf_launches_per_step
msf_profile_read = _lib.msf_profile_read
msf_batch_block_size = _lib.msf_batch_block_size
msf_instance_info = _lib.msf_instance_info
msf_cfl_dt_noalloc = _lib.msf_cfl_dt_noalloc
msf_fma_peak = _lib.msf_fma_peak


def fma_peak(precision, stream=None):
    """Measured FMA throughput (flop/s) of the current device's CUDA cores."""
    out = C.c_double()
    _check(msf_fma_peak(int(precision), C.byref(out), stream), None)
    return out.value
msf_last_error = _lib.msf_last_error


def lib():
    return _lib


def _check(status, ctx):
    if status != MSF_OK:
        raise MsfError(status, msf_last_error(ctx).decode())


def make_grid(p: dict) -> msf_grid:
    g = msf_grid()
    g.dim = int(p["dim"])
    for d in range(3):
        g.n[d] = int(p["n"][d])
        g.lo[d] = float(p["lo"][d])
        g.hi[d] = float(p["hi"][d])
        for s in range(2):
            g.bc[d][s] = int(p["bc"][d][s])
            g.inflow_mat[d][s] = int(p["inflow_mat"][d][s])
            for v in range(5):
                g.inflow_prim[d][s][v] = float(p["inflow_prim"][d][s][v])
    g.geom = int(p.get("geom", 0))
    fs = int(p.get("fs_mat", -1))
    g.free_surface = 1 if fs >= 0 else 0
    g.fs_mat = max(fs, 0)
    for k in ("fs_rho", "fs_p0", "fs_t0", "fs_t1", "fs_p1"):
        setattr(g, k, float(p.get(k, 0.0)))
    return g


def make_options(p: dict, precision=MSF_FP64, stream=None, use_graph=1, profile=0) -> msf_options:
    o = msf_options()
    _check(msf_default_options(int(p["dim"]), C.byref(o)), None)
    o.precision = int(precision)
    for k in ("cfl", "weno_eps", "mix_alpha", "scale_eps_h", "phi_cap_h"):
        setattr(o, k, float(p[k]))
    for k in ("ext_sweeps", "vel_sweeps", "reinit_iters", "scale_sep", "reinit", "rk_stages"):
        setattr(o, k, int(p[k]))
    o.literal_reduced = int(p.get("literal_reduced", 0))
    o.literal_normal = int(p.get("literal_normal", 0))
    o.positivity = int(p.get("positivity", 0))
    o.use_graph = int(use_graph)
    o.profile = int(profile)
    o.stream = stream
    return o


def _ptr(a, kind):
    """(pointer, mem) of a numpy array (host) or torch tensor (device or host)."""
    if hasattr(a, "data_ptr"):
        if a.dtype.itemsize != (8 if kind == "f8" else 4) or not a.is_contiguous():
            raise ValueError("tensor must be contiguous with the right dtype")
        return C.c_void_p(a.data_ptr()), (MSF_DEVICE if a.is_cuda else MSF_HOST), a
    arr = np.ascontiguousarray(a, dtype=np.float64 if kind == "f8" else np.int32)
    return C.c_void_p(arr.ctypes.data), MSF_HOST, arr


class Solver:
    """One context with one instance, built from a case (see cases.Case)."""

    def __init__(self, case, precision=MSF_FP64, stream=None, use_graph=1, profile=0, **opts):
        self.case = case
        self.p = case.params(**opts)
        self.N, self.NV, self.cells = case.nmat, case.nv, case.cells
        self._grid = make_grid(self.p)
        eos = (msf_eos * self.N)(*[make_eos(self.p, m) for m in range(self.N)])
        self._eos = eos
        self._opt = make_options(self.p, precision, stream, use_graph, profile)
        h = C.c_void_p()
        st = msf_create(C.byref(self._grid), 1, self.N, eos, C.byref(self._opt), C.byref(h))
        if st != MSF_OK:
            raise MsfError(st, msf_last_error(None).decode())
        self.h = h
        self.set_levelset(case.phi, case.chi, case.prim)

    def close(self):
        if getattr(self, "h", None):
            msf_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def set_levelset(self, phi, chi, prim):
        a, ma, ka = _ptr(phi, "f8")
        b, mb, kb = _ptr(chi, "i4")
        c, mc, kc = _ptr(prim, "f8")
        if not (ma == mb == mc):
            raise ValueError("phi, chi, prim must all be host or all device arrays")
        _check(msf_set_levelset(self.h, 0, a, b, c, ma), self.h)

    def step(self, n_steps, t_end=float("inf"), sync=True):
        _check(msf_step(self.h, int(n_steps), float(t_end), 1 if sync else 0), self.h)

    def state(self):
        Q = np.zeros((self.N, self.NV, self.cells))
        alpha = np.zeros((self.N, self.cells))
        phi = np.zeros(self.cells)
        chi = np.zeros(self.cells, np.int32)
        t = C.c_double()
        _check(msf_get_state(self.h, 0, C.c_void_p(Q.ctypes.data), C.c_void_p(alpha.ctypes.data),
                             C.c_void_p(phi.ctypes.data), C.c_void_p(chi.ctypes.data), C.byref(t), MSF_HOST), self.h)
        return dict(Q=Q, alpha=alpha, phi=phi, chi=chi, t=t.value)

    def get_state_device(self, Q):
        """Copy Q into a caller-owned device tensor (torch, float64, [N, NV, cells])."""
        _check(msf_get_state(self.h, 0, C.c_void_p(Q.data_ptr()), None, None, None, None, MSF_DEVICE), self.h)

    def get_alpha_device(self, alpha):
        """Copy the volume fractions into a caller-owned device tensor (torch,
        float64, [N, cells])."""
        _check(msf_get_state(self.h, 0, None, C.c_void_p(alpha.data_ptr()), None, None, None, MSF_DEVICE), self.h)

    def set_state(self, Q, phi, chi, t):
        a, ma, ka = _ptr(Q, "f8")
        b, mb, kb = _ptr(phi, "f8")
        c, mc, kc = _ptr(chi, "i4")
        _check(msf_set_state(self.h, 0, a, b, c, float(t), ma), self.h)

    def totals(self):
        tot = np.zeros((self.N, self.NV))
        led = np.zeros((self.N, self.NV))
        _check(msf_totals(self.h, 0, tot.ctypes.data_as(C.POINTER(C.c_double)),
                          led.ctypes.data_as(C.POINTER(C.c_double))), self.h)
        return tot, led

    def counters(self):
        c = (C.c_int64 * NSTATS)()
        _check(msf_stats(self.h, c), self.h)
        return dict(zip(COUNTERS, list(c)))

    def last_dt(self):
        dt = C.c_double()
        _check(msf_last_dt(self.h, 0, C.byref(dt)), self.h)
        return dt.value

    def launches_per_step(self):
        n = C.c_int64()
        _check(msf_launches_per_step(self.h, C.byref(n)), self.h)
        return n.value

    def flux_ms(self):
        out = (C.c_double * 3)()
        _check(msf_profile_read(self.h, out), self.h)
        return list(out)

    def debug(self, which):
        sizes = {0: self.N, 1: self.N * self.NV, 2: self.N * self.NV, 3: 3, 4: 1, 5: 1}
        out = np.zeros(sizes[which] * self.cells)
        _check(msf_debug_field(self.h, 0, int(which), out.ctypes.data_as(C.POINTER(C.c_double))), self.h)
        return out

    # ---- replay tapes and the adjoint step (frozen interface evolution)
    def tape_bytes(self):
        n = C.c_int64()
        _check(msf_tape_bytes(self.h, C.byref(n)), self.h)
        return n.value

    def new_tape(self):
        """A device buffer for one tape (torch uint8 tensor, 256-byte aligned)."""
        import torch
        nb = self.tape_bytes()
        buf = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
        off = (-buf.data_ptr()) % 256
        return buf[off:off + nb]

    def step_taped(self, tape, t_end=float("inf")):
        _check(msf_step_taped(self.h, C.c_void_p(tape.data_ptr()), float(t_end)), self.h)

    def replay_step(self, tape):
        _check(msf_replay_step(self.h, C.c_void_p(tape.data_ptr())), self.h)

    def set_conserved(self, Q):
        a, ma, ka = _ptr(Q, "f8")
        _check(msf_set_conserved(self.h, 0, a, ma), self.h)

    def adjoint_step(self, tape, lam_out):
        """(lam_in, d_eos [N, 2], d_inflow [3, 2, 5]) of one tape for the
        adjoint lam_out = dJ/dQ^{n+1} (torch float64 device [N, NV, cells])."""
        import torch
        lam_out = lam_out.contiguous()
        lam_in = torch.empty_like(lam_out)
        d_eos = np.zeros((self.N, 2))
        d_inf = np.zeros((3, 2, 5))
        _check(msf_adjoint_step(self.h, C.c_void_p(tape.data_ptr()), C.c_void_p(lam_out.data_ptr()),
                                C.c_void_p(lam_in.data_ptr()), d_eos.ctypes.data_as(C.POINTER(C.c_double)),
                                d_inf.ctypes.data_as(C.POINTER(C.c_double))), self.h)
        return lam_in, d_eos, d_inf


def pad_materials(case, nmat):
    """The same case with unused materials appended (EOS of an ideal gas, a
    resting unit state); they never appear in chi, so nothing changes."""
    import copy
    c = copy.copy(case)
    extra = nmat - case.nmat
    if extra <= 0:
        return c
    c.gamma = list(case.gamma) + [1.4] * extra
    c.pinf = list(case.pinf) + [0.0] * extra
    if case.eos_kind is not None:
        c.eos_kind = list(case.eos_kind) + [0] * extra
        c.tait = list(case.tait) + [(0.0, 0.0, 0.0)] * extra
    pad = np.zeros((extra, case.nv, case.cells))
    pad[:, 0] = 1.0
    pad[:, -1] = 1.0
    c.prim = np.concatenate([case.prim, pad], axis=0)
    return c


class Batch:
    """One context holding many instances of the same dimension (the batched
    form: one persistent launch per msf_step call for 1D instances)."""

    def __init__(self, cases, precision=MSF_FP64, batch_mode=0, stream=None, **opts):
        self.nmat = max(c.nmat for c in cases)
        self.cases = [pad_materials(c, self.nmat) for c in cases]
        self.n = len(cases)
        ps = [c.params(**opts) for c in self.cases]
        grids = (msf_grid * self.n)(*[make_grid(p) for p in ps])
        eos = (msf_eos * (self.n * self.nmat))(*[make_eos(p, m) for p in ps
                                                 for m in range(self.nmat)])
        self._keep = (grids, eos)
        self._opt = make_options(ps[0], precision, stream, 1, 0)
        self._opt.batch_mode = int(batch_mode)
        h = C.c_void_p()
        st = msf_create(grids, self.n, self.nmat, eos, C.byref(self._opt), C.byref(h))
        if st != MSF_OK:
            raise MsfError(st, msf_last_error(None).decode())
        self.h = h
        for i, c in enumerate(self.cases):
            phi = np.ascontiguousarray(c.phi, np.float64).ravel()
            chi = np.ascontiguousarray(c.chi, np.int32).ravel()
            prim = np.ascontiguousarray(c.prim, np.float64)
            _check(msf_set_levelset(h, i, C.c_void_p(phi.ctypes.data), C.c_void_p(chi.ctypes.data),
                                    C.c_void_p(prim.ctypes.data), MSF_HOST), h)

    def close(self):
        if getattr(self, "h", None):
            msf_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def step(self, n_steps, t_end=float("inf"), sync=True):
        _check(msf_step(self.h, int(n_steps), float(t_end), 1 if sync else 0), self.h)

    def state(self, i):
        c = self.cases[i]
        Q = np.zeros((self.nmat, c.nv, c.cells))
        alpha = np.zeros((self.nmat, c.cells))
        phi = np.zeros(c.cells)
        chi = np.zeros(c.cells, np.int32)
        t = C.c_double()
        _check(msf_get_state(self.h, int(i), C.c_void_p(Q.ctypes.data), C.c_void_p(alpha.ctypes.data),
                             C.c_void_p(phi.ctypes.data), C.c_void_p(chi.ctypes.data), C.byref(t), MSF_HOST), self.h)
        return dict(Q=Q, alpha=alpha, phi=phi, chi=chi, t=t.value)

    def totals(self, i):
        c = self.cases[i]
        tot = np.zeros((self.nmat, c.nv))
        led = np.zeros((self.nmat, c.nv))
        _check(msf_totals(self.h, int(i), tot.ctypes.data_as(C.POINTER(C.c_double)),
                          led.ctypes.data_as(C.POINTER(C.c_double))), self.h)
        return tot, led

    def info(self, i):
        t, steps, status = C.c_double(), C.c_int64(), C.c_int32()
        _check(msf_instance_info(self.h, int(i), C.byref(t), C.byref(steps), C.byref(status)), self.h)
        return t.value, steps.value, status.value

    def block_size(self):
        bs = C.c_int32()
        _check(msf_batch_block_size(self.h, C.byref(bs)), self.h)
        return bs.value

    def launches_per_step(self):
        n = C.c_int64()
        _check(msf_launches_per_step(self.h, C.byref(n)), self.h)
        return n.value
