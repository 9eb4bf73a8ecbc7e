"""The FP32 copy of the step state in the FP32-bulk form.

The flux update of the FP32-bulk form stages its bulk stencil states from an
FP32 copy of the state it reads. For stage 0 that copy is kept across steps:
written by the last update of the step before and refreshed on that step's
band after the band kernels changed those cells. It must equal Q^n rounded to
FP32 at every step start, so a run that keeps it must give the same bits as a
run whose copy is converted afresh from Q^n before every step
(msf_set_conserved converts the whole state).

The conversions themselves run on the integer pipes (the FP64 pipes are the
scarce unit on this GPU); they are checked here against the hardware
conversions on every binary32 pattern and on 2^28 binary64 patterns.
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import paper_1704_00519_gb300.cases as cs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def msf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00519_gb300 import build
    build.build()
    import paper_1704_00519_gb300.msf as m
    return m


def _run(msf, case, steps, fresh):
    """State, counters and the (step, status) of a device-detected failure
    (None if every step ran) of `steps` FP32-bulk steps."""
    import torch
    s = msf.Solver(case, precision=msf.MSF_FP32_BULK)
    Q = torch.empty((case.nmat, case.nv, case.cells), dtype=torch.float64, device="cuda")
    failed = None
    for k in range(steps):
        try:
            s.step(1, case.t_end)
        except msf.MsfError as e:
            failed = (k, e.status)
            break
        if fresh:
            s.get_state_device(Q)
            s.set_conserved(Q)
    st = s.state()
    counters = s.counters()
    s.close()
    return st, counters, failed


@pytest.mark.parametrize("maker,steps", [
    (lambda: cs.shock_sphere((48, 32, 32)), 25),
    (lambda: cs.triple_point(112, 48), 60),
    (lambda: cs.shock_bubbles(128, 48), 40),
    (lambda: cs.scale_sep_demo("droplet", n=10), 10),
    (lambda: cs.random_case(3, (14, 12, 11), 3, 4), 15),
    (lambda: cs.random_case(3, (14, 12, 11), 3, 3), 15),
    (lambda: cs.shock_tube_3(200), 60),
], ids=["sphere", "triple_point", "bubbles", "droplet", "random3d_s4", "random3d_s3", "tube1d"])
def test_kept_copy_equals_fresh_rounding(msf, maker, steps):
    case = maker()
    a, ca, fa = _run(msf, case, steps, fresh=False)
    b, cb, fb = _run(msf, case, steps, fresh=True)
    assert fa == fb
    assert a["t"] == b["t"]
    assert np.array_equal(a["chi"], b["chi"])
    assert np.array_equal(a["phi"], b["phi"])
    assert np.array_equal(a["Q"], b["Q"])
    assert ca == cb


@pytest.fixture(scope="module")
def conv_libs(tmp_path_factory):
    from paper_1704_00519_gb300 import build
    out = tmp_path_factory.mktemp("conv")
    libs = {}
    # the flags of the two kernel units: FP32-bulk (fast math) and strict FP64
    for name, flags in (("f32", ["-fmad=true", "-use_fast_math"]), ("f64", ["-fmad=false"])):
        so = str(out / f"conv_{name}.so")
        cmd = [build.nvcc(), *build.ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", *flags,
               os.path.join(HERE, "gpu_conversions.cu"), "-o", so]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        lib = C.CDLL(so)
        lib.conv_check.restype = C.c_int
        lib.conv_check.argtypes = [C.c_int, C.c_ulonglong, C.POINTER(C.c_ulonglong)]
        libs[name] = lib
    return libs


@pytest.mark.parametrize("unit", ["f32", "f64"])
def test_float_to_double_every_pattern(conv_libs, unit):
    out = (C.c_ulonglong * 3)()
    assert conv_libs[unit].conv_check(0, 0, out) == 0
    assert out[0] == 1 << 32
    assert out[1] == 0, f"first mismatch at float bits {out[2]:#010x}"


@pytest.mark.parametrize("unit", ["f32", "f64"])
def test_double_to_float_sign_and_order_tests(conv_libs, unit):
    count = 1 << 28
    out = (C.c_ulonglong * 3)()
    assert conv_libs[unit].conv_check(1, count, out) == 0
    assert out[0] == count
    assert out[1] == 0, f"first mismatch at double bits {out[2]:#018x}"
