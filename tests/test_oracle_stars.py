"""The hub-star block update in the oracle, pinned against what the paper's argument fixes.

A star update sets a hub's shares on a set of its edges to the exact minimiser of the sum of
squared loads over those shares with every other split fixed (the local optimality of
Sec. III-C taken over a block of edges instead of one edge).  Pins, none of which reuses the
water-filling formula: the KKT conditions of that convex problem; a one-leaf star is
Algorithm 1's edge update; many sequential Algorithm 1 passes over the star's edges converge
to the same loads; a hub-star pass conserves the total weight, never raises the sum of
squares, and converges to the exact locally-dense decomposition (min cut).
"""
import numpy as np
import pytest

import synth


def _random_star(rng, q):
    w = rng.uniform(0.2, 3.0, q)
    t = rng.uniform(0.0, 1.0, q) * w
    lh = rng.uniform(0.0, 40.0)
    l = rng.uniform(0.0, 40.0, q)
    return lh, l, w, t


@pytest.mark.parametrize("q", [1, 2, 3, 7, 40, 300])
def test_star_update_satisfies_kkt(oracle_mod, q):
    rng = np.random.default_rng(100 + q)
    for _ in range(20):
        lh, l, w, t = _random_star(rng, q)
        lh2, l2, t2, lam = oracle_mod.star_update(lh, l, w, t)
        scale = max(1.0, lh, l.max())
        assert abs(lh2 + l2.sum() - (lh + l.sum())) <= 1e-12 * scale * (q + 1)   # conservation
        assert np.all(t2 >= 0) and np.all(t2 <= w)
        assert abs(lh2 - lam) <= 1e-12 * scale * (q + 1)
        inner = (t2 > 0) & (t2 < w)
        assert np.all(np.abs(l2[inner] - lh2) <= 1e-11 * scale)            # balanced with the hub
        assert np.all(l2[t2 == 0] <= lh2 + 1e-11 * scale)                  # all to the leaf: leaf lower
        assert np.all(l2[t2 == w] >= lh2 - 1e-11 * scale)                  # all to the hub: leaf higher
        # never worse than the start: the minimiser over the shares
        assert lh2 ** 2 + (l2 ** 2).sum() <= lh ** 2 + (l ** 2).sum() + 1e-9 * scale ** 2


def test_one_leaf_star_is_algorithm_1(oracle_mod):
    rng = np.random.default_rng(7)
    for _ in range(200):
        lh, l, w, t = _random_star(rng, 1)
        lh2, l2, t2, _ = oracle_mod.star_update(lh, l, w, t)
        a, b, fa, fb, _ = oracle_mod.lowd_update(lh, l[0], t[0], w[0] - t[0])
        assert abs(a - lh2) <= 1e-12 * max(1, lh) and abs(b - l2[0]) <= 1e-12 * max(1, lh)
        assert abs(fa - t2[0]) <= 1e-12 * max(1, w[0])


@pytest.mark.parametrize("q", [2, 5, 12])
def test_sequential_passes_converge_to_the_star_update(oracle_mod, q):
    rng = np.random.default_rng(200 + q)
    lh, l, w, t = _random_star(rng, q)
    lh2, l2, _, _ = oracle_mod.star_update(lh, l, w, t)
    a, ls, ts = lh, l.copy(), t.copy()
    for _ in range(4000):
        for j in range(q):
            a, ls[j], ts[j], _, _ = oracle_mod.lowd_update(a, ls[j], ts[j], w[j] - ts[j])
    assert abs(a - lh2) <= 1e-7 * max(1, lh2)
    assert np.max(np.abs(ls - l2)) <= 1e-7 * max(1, lh2)


def _graphs():
    return [synth.chung_lu(300, 1500, 2.1, seed=3, block_size=12, block_p=0.7),
            synth.planted_background(200, 3.0, 20, 0.7, seed=6),
            synth.small_family("star", 30),
            synth.erdos_renyi(80, 0.2, seed=2)]


@pytest.mark.parametrize("gi", range(4))
def test_hub_star_structure_is_vertex_disjoint_and_complete(oracle_mod, gi):
    g = _graphs()[gi]
    deg = np.bincount(g.u, minlength=g.n) + np.bincount(g.v, minlength=g.n)
    tau = max(2, int(np.percentile(deg[deg > 0], 90)))
    plain, steps = oracle_mod.hub_star_structure(g.n, g.u, g.v, tau)
    seen = list(plain)
    hub = deg >= tau
    for st in steps:
        touched = []
        for h, es in st.items():
            assert hub[h]
            ends = np.concatenate([g.u[es], g.v[es]])
            leaves = ends[ends != h]
            assert leaves.shape[0] == es.shape[0] and not hub[leaves].any()
            touched += [h] + leaves.tolist()
            seen += es.tolist()
        assert len(touched) == len(set(touched))            # the stars of a step are disjoint
    assert sorted(seen) == list(range(g.m))                  # every edge in exactly one block
    star = hub[g.u] ^ hub[g.v]
    assert np.array_equal(np.sort(plain), np.nonzero(~star)[0])


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("gi", range(2))
def test_hub_star_passes_conserve_descend_and_converge(oracle_mod, gi, weighted):
    g = _graphs()[gi]
    w = synth.quantise_weights(np.random.default_rng(9).lognormal(0, 1, g.m)).astype(np.float64) if weighted else None
    deg = np.bincount(g.u, minlength=g.n) + np.bincount(g.v, minlength=g.n)
    tau = max(2, int(np.percentile(deg[deg > 0], 85)))
    plain, steps = oracle_mod.hub_star_structure(g.n, g.u, g.v, tau)
    assert len(steps) > 0
    po = plain[oracle_mod.level_order(g.n, g.u[plain], g.v[plain])[0]] if plain.shape[0] else plain
    st = oracle_mod.LowdState(g.n, g.u, g.v, w)
    total = st.l.sum()
    prev = (st.l ** 2).sum()
    for _ in range(60):
        st.iterate_hub_star(1, po, steps)
        cur = (st.l ** 2).sum()
        assert cur <= prev * (1 + 1e-12)
        assert abs(st.l.sum() - total) <= 1e-9 * total
        prev = cur
    st.iterate_hub_star(4000, po, steps)
    wu, scale = oracle_mod.weight_units(g.m, w)
    lstar, _, _ = oracle_mod.ldd_loads(g.n, g.u, g.v, wu, scale)
    assert np.max(np.abs(st.l - lstar)) <= 1e-6 * max(1.0, lstar.max())


def test_auto_hub_threshold_closed_forms(oracle_mod):
    # a star on q leaves: the centre alone has degree >= 2 (one node <= 1): tau = 2
    g = synth.small_family("star", 30)
    assert oracle_mod.auto_hub_threshold(g.n, g.u, g.v) == 2
    # a clique on 6 nodes: 6 nodes of degree 5 exceed the limit until no node qualifies
    g = synth.small_family("clique", 6)
    assert oracle_mod.auto_hub_threshold(g.n, g.u, g.v) == 8
    # a path: all degrees <= 2; 2^1 = 2 has n - 2 nodes of degree 2 > 1; 4 has none
    g = synth.small_family("path", 20)
    assert oracle_mod.auto_hub_threshold(g.n, g.u, g.v) == 4
    # schedule 1: the smallest power of two >= half the maximum degree
    g = synth.small_family("star", 30)                     # max degree 29: 16 (2 * 16 >= 29)
    assert oracle_mod.auto_hub_threshold(g.n, g.u, g.v, schedule=1) == 16
    g = synth.small_family("clique", 6)                    # max degree 5: 4
    assert oracle_mod.auto_hub_threshold(g.n, g.u, g.v, schedule=1) == 4
    g = synth.small_family("path", 20)                     # max degree 2: the minimum, 2
    assert oracle_mod.auto_hub_threshold(g.n, g.u, g.v, schedule=1) == 2


@pytest.mark.parametrize("gi", range(2))
def test_auto_hub_threshold_is_the_least_qualifying_power(oracle_mod, gi):
    g = _graphs()[gi]
    deg = np.bincount(g.u, minlength=g.n) + np.bincount(g.v, minlength=g.n)
    tau = oracle_mod.auto_hub_threshold(g.n, g.u, g.v)
    k = tau.bit_length() - 1
    assert tau == 1 << k and k >= 1
    assert (deg >= tau).sum() <= tau // 2
    if k > 1:
        assert (deg >= tau // 2).sum() > tau // 4
