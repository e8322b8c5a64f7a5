"""Pins for the oracle's single-edge LOWD update (Algorithm 1's loop body).

Pinned against: the Fig. 1 worked example (tests/golden/fig1_update.txt), hand cases for
both clip branches, the tie case, the exact change of sum(l^2) derived in Sec. III-C, and
local optimality (no other feasible transfer lowers sum(l^2) further, Sec. III-C).
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig1_update.txt")


def _rows(path):
    with open(path) as f:
        return [list(map(float, ln.split())) for ln in f if ln.strip() and not ln.startswith("#")]


def test_fig1_worked_example(oracle_mod):
    for lu, lv, fu, fv, elu, elv, efu, efv, ed in _rows(GOLDEN):
        got = oracle_mod.lowd_update(lu, lv, fu, fv)
        assert got == (elu, elv, efu, efv, ed)


@pytest.mark.parametrize("lu,lv,fu,fv,exp", [
    # l_u > l_v, half the gap fits in f_e(u): d = (l_u - l_v)/2
    (5.0, 1.0, 3.0, 1.0, (3.0, 3.0, 1.0, 3.0, 2.0)),
    # l_u > l_v, f_e(u) smaller than half the gap: d = f_e(u) (clip)
    (5.0, 1.0, 0.5, 3.5, (4.5, 1.5, 0.0, 4.0, 0.5)),
    # l_u < l_v, half the gap fits in f_e(v)
    (1.0, 4.0, 0.25, 2.0, (2.5, 2.5, 1.75, 0.5, 1.5)),
    # l_u < l_v, clip at f_e(v)
    (1.0, 4.0, 1.75, 0.25, (1.25, 3.75, 2.0, 0.0, 0.25)),
    # tie: else-branch with d = min(0, f_e(v)) = 0, a no-op
    (2.0, 2.0, 0.5, 0.5, (2.0, 2.0, 0.5, 0.5, 0.0)),
    # edge already one-way toward the lower load: nothing to move
    (3.0, 1.0, 0.0, 1.0, (3.0, 1.0, 0.0, 1.0, 0.0)),
])
def test_clip_branches(oracle_mod, lu, lv, fu, fv, exp):
    assert oracle_mod.lowd_update(lu, lv, fu, fv) == exp


def test_sumsq_change_and_local_optimality(oracle_mod):
    rng = np.random.default_rng(7)
    for _ in range(2000):
        w = float(rng.uniform(0.1, 3.0))
        fu = float(rng.uniform(0, w)); fv = w - fu
        lu = fu + float(rng.uniform(0, 10)); lv = fv + float(rng.uniform(0, 10))
        nlu, nlv, nfu, nfv, d = oracle_mod.lowd_update(lu, lv, fu, fv)
        assert d >= 0
        # box and edge-sum constraints of the tighter dual (Sec. III-B)
        assert nfu >= 0 and nfv >= 0
        assert abs((nfu + nfv) - w) <= 1e-12 * w
        # loads move by exactly the split change
        assert abs((nlu - lu) - (nfu - fu)) <= 1e-12 * max(1, abs(lu))
        assert abs((nlv - lv) - (nfv - fv)) <= 1e-12 * max(1, abs(lv))
        # sum(l^2) falls by 2 d (|l_u - l_v| - d) >= 0 (Sec. III-C)
        before = lu * lu + lv * lv
        after = nlu * nlu + nlv * nlv
        gap = abs(lu - lv)
        assert abs((before - after) - 2 * d * (gap - d)) <= 1e-9 * max(1.0, before)
        assert after <= before + 1e-12 * before
        # no other feasible transfer t in [-f_e(v), f_e(u)] (u -> v positive) does better
        ts = np.linspace(-fv, fu, 257)
        alt = (lu - ts) ** 2 + (lv + ts) ** 2
        assert after <= alt.min() + 1e-9 * max(1.0, before)
