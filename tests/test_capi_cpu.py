"""The C-ABI library loads and exports every entry point include/msf.h
declares; host-side validation needs no GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "msf.h")


@pytest.fixture(scope="module")
def msf():
    from paper_1704_00519_gb300 import build
    build.build()
    import paper_1704_00519_gb300.msf as m
    return m


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(msf_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("msf_create", "msf_set_levelset", "msf_step", "msf_totals", "msf_adjoint_step"):
        assert required in names


def test_library_exports_every_declared_symbol(msf):
    lib = C.CDLL(msf.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layout_matches_header(msf, tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include "msf.h"\nint main(){printf("%zu %zu %zu", sizeof(msf_grid),'
                   ' sizeof(msf_options), sizeof(msf_eos));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert [int(x) for x in out] == [C.sizeof(msf.msf_grid), C.sizeof(msf.msf_options), C.sizeof(msf.msf_eos)]


def test_default_options(msf):
    o = msf.msf_options()
    assert msf.msf_default_options(2, C.byref(o)) == msf.MSF_OK
    assert o.cfl == 0.6 and o.weno_eps == 1e-6 and o.ext_sweeps == 5
    assert msf.msf_default_options(4, C.byref(o)) == msf.MSF_EINVAL


def _args(msf, **over):
    import paper_1704_00519_gb300.cases as cs
    p = cs.shock_tube_3(20).params()
    q = dict(p)
    q.update(over)
    g = msf.make_grid(q)
    o = msf.make_options(p)
    for k in ("cfl", "ext_sweeps"):
        if k in over:
            setattr(o, k, over[k])
    eos = (msf.msf_eos * 3)(*[msf.msf_eos(1.4, 0.0)] * 3)
    return g, eos, o


@pytest.mark.parametrize("bad", [
    dict(n=[0, 1, 1]), dict(dim=0), dict(lo=[1.0, 0, 0], hi=[0.0, 1, 1]),
    dict(bc=[[5, 0], [0, 0], [0, 0]]), dict(cfl=0.0), dict(ext_sweeps=0),
    # axisymmetric grid below the axis, unknown geometry, free-surface ambient
    # out of range, without density, with a drive ramp that ends before it starts
    dict(geom=1, lo=[-0.5, 0.0, 0.0]), dict(geom=2), dict(fs_mat=7),
    dict(fs_mat=2, fs_rho=0.0, fs_p0=1.0, fs_t0=0.0, fs_t1=1.0, fs_p1=1.0),
    dict(fs_mat=2, fs_rho=1.0, fs_p0=1.0, fs_t0=1.0, fs_t1=0.5, fs_p1=1.0)])
def test_create_rejects_bad_arguments_on_host(msf, bad):
    g, eos, o = _args(msf, **bad)
    h = C.c_void_p()
    st = msf.msf_create(C.byref(g), 1, 3, eos, C.byref(o), C.byref(h))
    assert st == msf.MSF_EINVAL
    assert h.value is None
    assert msf.msf_last_error(None).decode()


def test_create_rejects_bad_eos_and_counts(msf):
    g, eos, o = _args(msf)
    h = C.c_void_p()
    assert msf.msf_create(C.byref(g), 1, 0, eos, C.byref(o), C.byref(h)) == msf.MSF_EINVAL
    assert msf.msf_create(C.byref(g), 1, 9, eos, C.byref(o), C.byref(h)) == msf.MSF_EINVAL
    bad = (msf.msf_eos * 3)(*[msf.msf_eos(1.0, 0.0)] * 3)
    assert msf.msf_create(C.byref(g), 1, 3, bad, C.byref(o), C.byref(h)) == msf.MSF_EINVAL
    assert msf.msf_create(None, 1, 3, eos, C.byref(o), C.byref(h)) == msf.MSF_EINVAL


def test_null_context_calls(msf):
    assert msf.msf_step(None, 1, 1.0, 1) == msf.MSF_EINVAL
    assert msf.msf_destroy(None) == msf.MSF_OK
    assert msf.msf_adjoint_step(None, None, None, None, None, None) == msf.MSF_EINVAL
    assert msf.msf_step_taped(None, None, 0.0) == msf.MSF_EINVAL
    assert msf.msf_replay_step(None, None) == msf.MSF_EINVAL
