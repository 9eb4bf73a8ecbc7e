"""Batched form: many independent 1D instances in one context, stepped by one
persistent launch (one CTA per instance). Each instance must reproduce its
single-instance GPU run and the oracle exactly in FP64, whatever CTA size the
autotuner picks, and the per-instance launch mode must agree as well."""
import numpy as np
import pytest

import paper_1704_00519_gb300.cases as cs
from oracle import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def msf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00519_gb300 import build
    build.build()
    import paper_1704_00519_gb300.msf as m
    return m


def _clean_batch(count, seed, lo=60, hi=420, steps=12, **opts):
    """Seeded Riemann problems that the oracle runs without a device error."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        c = cs.riemann_1d(rng, ncell=int(rng.integers(lo, hi)))
        o = orc.Oracle(c, **opts)
        if o.step(steps, c.t_end) == 0:
            out.append((c, o))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_instances_match_oracle(msf, precision):
    steps = 12
    pairs = _clean_batch(10, 7, steps=steps)
    cases = [c for c, _ in pairs]
    batch = msf.Batch(cases, precision=precision)
    batch.step(steps, 0.1)
    assert batch.block_size() in (128, 256, 512)
    assert batch.launches_per_step() == 1
    for i, (c, o) in enumerate(pairs):
        a, b = batch.state(i), o.state()
        Qa = a["Q"][:c.nmat]
        assert np.all(a["Q"][c.nmat:] == 0.0)
        assert a["t"] == pytest.approx(b["t"], rel=1e-14 if precision == 0 else 1e-5)
        if precision == 0:
            assert np.array_equal(Qa, b["Q"]), (i, np.abs(Qa - b["Q"]).max())
            assert np.array_equal(a["chi"], b["chi"])
            assert np.array_equal(a["phi"], b["phi"])
        else:
            ra, rb = Qa[:, 0].sum(0), b["Q"][:, 0].sum(0)
            assert np.abs(ra - rb).sum() / np.abs(rb).sum() <= 2e-5


def test_batched_equals_single_and_per_instance_modes(msf):
    steps = 10
    pairs = _clean_batch(6, 11, steps=steps)
    cases = [c for c, _ in pairs]
    batch = msf.Batch(cases)
    batch.step(steps, 0.1)
    seq = msf.Batch(cases, batch_mode=1)
    seq.step(steps, 0.1)
    for i, c in enumerate(cases):
        single = msf.Solver(msf.pad_materials(c, batch.nmat))
        single.step(steps, 0.1)
        a, b, s = batch.state(i), seq.state(i), single.state()
        assert np.array_equal(a["Q"], b["Q"])
        assert np.array_equal(a["Q"], s["Q"])
        ta, la = batch.totals(i)
        tb, lb = seq.totals(i)
        assert np.allclose(la, lb, rtol=1e-13, atol=1e-15)


def test_batched_conservation_and_end_time(msf):
    pairs = _clean_batch(8, 3, steps=30)
    cases = [c for c, _ in pairs]
    batch = msf.Batch(cases)
    tot0 = [batch.totals(i)[0] for i in range(len(cases))]
    batch.step(1000, 0.004)  # every instance stops at its own last clipped step
    for i in range(len(cases)):
        st = batch.state(i)
        assert st["t"] == 0.004
        tot, led = batch.totals(i)
        scale = max(np.abs(tot0[i]).sum(), np.abs(tot).sum())
        assert np.abs((tot - tot0[i] - led).sum(0)).max() / scale < 1e-12


def test_batched_rk2_matches_oracle(msf):
    """The persistent batched kernel with the two-stage TVD Runge-Kutta of
    Sec. 3: FP64 bit-identical to the oracle per instance."""
    steps = 10
    pairs = _clean_batch(8, 11, steps=steps, rk_stages=2)
    batch = msf.Batch([c for c, _ in pairs], precision=0, rk_stages=2)
    batch.step(steps, 0.1)
    for i, (c, o) in enumerate(pairs):
        a, b = batch.state(i), o.state()
        assert np.array_equal(a["Q"][:c.nmat], b["Q"]), i
        assert np.array_equal(a["phi"], b["phi"])


def test_batched_positivity_limiter_matches_oracle(msf):
    """The persistent batched kernel with the positivity limiter: FP64
    bit-identical to the oracle per instance, LeBlanc's problem among the
    instances (it runs to its end only with the limiter)."""
    from test_oracle_pins import _leblanc
    steps, t_end = 40, 6.0
    rng = np.random.default_rng(5)
    pairs = []
    while len(pairs) < 6:
        c = cs.riemann_1d(rng, ncell=int(rng.integers(60, 420)))
        o = orc.Oracle(c, positivity=1)
        if o.step(steps, t_end) == 0:
            pairs.append((c, o))
    lb = _leblanc(300)
    o = orc.Oracle(lb, positivity=1)
    assert o.step(steps, t_end) == 0
    pairs.append((lb, o))
    batch = msf.Batch([c for c, _ in pairs], precision=0, positivity=1)
    batch.step(steps, t_end)
    for i, (c, o) in enumerate(pairs):
        a, b = batch.state(i), o.state()
        assert np.array_equal(a["Q"][:c.nmat], b["Q"]), i
        assert np.array_equal(a["phi"], b["phi"])
