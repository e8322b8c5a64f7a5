"""The oracle's pass order (the circle colouring schedule) against what a proper edge
colouring must be: every class a matching, every edge in exactly one class, and on the
complete graph K_n the textbook round-robin counts (n - 1 perfect matchings for even n,
n matchings of (n - 1) / 2 edges for odd n)."""
import itertools

import numpy as np
import pytest

import synth


def _classes(order, offs):
    return [order[offs[c]:offs[c + 1]] for c in range(len(offs) - 1)]


def _is_matching(u, v, ids):
    ends = np.concatenate([u[ids], v[ids]])
    return np.unique(ends).shape[0] == ends.shape[0]


@pytest.mark.parametrize("n", list(range(2, 15)))
def test_complete_graph_round_robin(oracle_mod, n):
    pairs = np.array(list(itertools.combinations(range(n), 2)), np.int32)
    u, v = pairs[:, 0], pairs[:, 1]
    order, offs, col = oracle_mod.circle_order(n, u, v)
    assert np.array_equal(np.sort(order), np.arange(u.shape[0]))
    cls = _classes(order, offs)
    sizes = sorted(len(c) for c in cls if len(c))
    if n % 2 == 0:
        assert sizes == [n // 2] * (n - 1)
    else:
        assert sizes == [(n - 1) // 2] * n
    for c in cls:
        assert _is_matching(u, v, c)
        assert np.all(np.diff(c) > 0)          # by edge id inside a class


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_graph_classes_are_matchings(oracle_mod, seed):
    g = synth.erdos_renyi(301 + seed, 0.05, seed=seed)
    order, offs, col = oracle_mod.circle_order(g.n, g.u, g.v)
    assert np.array_equal(np.sort(order), np.arange(g.m))
    assert offs[-1] == g.m and np.all(np.diff(offs) >= 0)
    for c in range(len(offs) - 1):
        ids = order[offs[c]:offs[c + 1]]
        assert np.all(col[ids] == c)
        assert _is_matching(g.u, g.v, ids)


def test_order_inside_a_class_does_not_matter(oracle_mod):
    """A class is a matching, so shuffling inside classes leaves every pass unchanged."""
    g = synth.chung_lu(400, 3000, 2.3, seed=4)
    order, offs, _ = oracle_mod.circle_order(g.n, g.u, g.v)
    rng = np.random.default_rng(0)
    shuffled = order.copy()
    for c in range(len(offs) - 1):
        seg = shuffled[offs[c]:offs[c + 1]]
        rng.shuffle(seg)
        shuffled[offs[c]:offs[c + 1]] = seg
    s1 = oracle_mod.LowdState(g.n, g.u, g.v); s1.iterate(7, order=order)
    s2 = oracle_mod.LowdState(g.n, g.u, g.v); s2.iterate(7, order=shuffled)
    assert np.array_equal(s1.l, s2.l)
