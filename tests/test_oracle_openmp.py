"""The OpenMP build of the oracle (used only to time the CPU baseline on all
host cores) gives the same bits as the plain build: its pragmas split loops
whose iterations write their own cells, flags and counters are atomic and the
sums keep their serial order."""
import os

import numpy as np
import pytest

import paper_1704_00519_gb300.cases as cs
from oracle import oracle as orc


@pytest.mark.parametrize("maker,steps", [
    (lambda: cs.shock_tube_3(400), 100000),
    (lambda: cs.triple_point(112, 48), 20),
    (lambda: cs.shock_bubbles(96, 32), 10),
    (lambda: cs.random_case(3, (12, 11, 10), 3, 2), 4),
    (lambda: cs.random_case(2, (40, 31), 4, 5), 10),
    (lambda: cs.icf_implosion(160), 60),
], ids=["tube", "triple", "bubbles_inflow", "random_3d", "random_2d_4mat", "icf_cylindrical"])
def test_openmp_build_gives_the_same_bits(maker, steps):
    if orc.threads(openmp=True) < 2:
        pytest.skip("one host core")
    case = maker()
    a = orc.Oracle(case)
    b = orc.Oracle(case, openmp=True)
    ea, eb = a.step(steps, case.t_end), b.step(steps, case.t_end)
    assert ea == eb
    sa, sb = a.state(), b.state()
    for k in ("Q", "alpha", "phi", "chi"):
        assert np.array_equal(sa[k], sb[k]), k
    assert sa["t"] == sb["t"]
    ta, tb = a.totals(), b.totals()
    assert np.array_equal(ta[0], tb[0]) and np.array_equal(ta[1], tb[1])
    assert a.counters() == b.counters()
