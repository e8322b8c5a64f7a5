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


# ----------------------------------------------------------------------------- level order

def _fmix32(x):
    """MurmurHash3's 32-bit finaliser (Appleby), written from its published definition."""
    h = np.asarray(x, np.uint64) & np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(16)
    h = (h * np.uint64(0x85EBCA6B)) & np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(13)
    h = (h * np.uint64(0xC2B2AE35)) & np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(16)
    return h


def test_fmix32_known_values():
    # the finaliser maps 0 to 0 and is a bijection: no two of a range of ids collide
    assert int(_fmix32(0)) == 0
    assert np.unique(_fmix32(np.arange(1 << 16))).shape[0] == 1 << 16


def _key_sorted_adjacency(n, u, v):
    """Each node's edges by the key (max degree, min degree, fmix32(edge id)) of the level
    order."""
    deg = np.bincount(u, minlength=n) + np.bincount(v, minlength=n)
    hi = np.maximum(deg[u], deg[v])
    lo = np.minimum(deg[u], deg[v])
    rank = np.lexsort((_fmix32(np.arange(u.shape[0])), lo, hi))   # edge ids by ascending key
    pos = np.empty_like(rank)
    pos[rank] = np.arange(rank.shape[0])
    adj = [[] for _ in range(n)]
    for e in rank:
        adj[u[e]].append(int(e))
        adj[v[e]].append(int(e))
    return adj, rank


def _round_process(n, u, v):
    """The schedule's rounds written out literally: in round r every node with uncoloured
    edges designates the first uncoloured edge of its key-sorted list; every edge designated
    by both of its ends gets colour r."""
    adj, _ = _key_sorted_adjacency(n, u, v)
    m = u.shape[0]
    colour = np.full(m, -1)
    cur = [0] * n
    r = 0
    while (colour < 0).any():
        desig = {}
        for x in range(n):
            while cur[x] < len(adj[x]) and colour[adj[x][cur[x]]] >= 0:
                cur[x] += 1
            if cur[x] < len(adj[x]):
                desig[x] = adj[x][cur[x]]
        picked = [e for e in set(desig.values()) if desig.get(int(u[e])) == e and desig.get(int(v[e])) == e]
        assert picked, "a round that colours nothing"
        for e in picked:
            colour[e] = r
        r += 1
    return colour, r


def _level_graphs():
    gs = [synth.erdos_renyi(30, p, seed=s) for s, p in enumerate((0.1, 0.3, 0.6))]
    gs += [synth.chung_lu(80, 240, 2.1, seed=s, block_size=8, block_p=0.7) for s in range(3)]
    gs += [synth.small_family(k, 12, seed=1) for k in ("star", "path", "clique", "two_cliques", "tree", "cycle")]
    gs += [synth.planted_background(60, 3.0, 10, 0.8, seed=4)]
    return gs


@pytest.mark.parametrize("gi", range(13))
def test_level_order_equals_the_round_process(oracle_mod, gi):
    g = _level_graphs()[gi]
    order, offs, colour = oracle_mod.level_order(g.n, g.u, g.v)
    want, rounds = _round_process(g.n, g.u, g.v)
    assert np.array_equal(colour, want)
    assert offs.shape[0] - 1 == rounds
    # a proper colouring: every class a matching, every edge in exactly one class
    assert np.array_equal(np.sort(order), np.arange(g.m))
    for ids in _classes(order, offs):
        assert _is_matching(g.u, g.v, ids)
    # at least max degree classes
    deg = np.bincount(g.u, minlength=g.n) + np.bincount(g.v, minlength=g.n)
    assert rounds >= (deg.max() if g.m else 0)


@pytest.mark.parametrize("k", [1, 2, 5, 17])
def test_level_order_star(oracle_mod, k):
    star = synth.small_family("star", k + 1)
    _, offs, _ = oracle_mod.level_order(star.n, star.u, star.v)
    assert offs.shape[0] - 1 == k                    # Delta colours


def test_level_order_path_is_not_a_chain(oracle_mod):
    """A path's inner edges all have the same degree key; the scrambled tie-break keeps
    them from forming one chain of n - 2 levels (edge-id ties would)."""
    path = synth.small_family("path", 2000)
    _, offs, _ = oracle_mod.level_order(path.n, path.u, path.v)
    assert offs.shape[0] - 1 <= 20


def test_level_order_gives_the_key_order_pass(oracle_mod):
    """Visiting the classes in colour order is the same pass as visiting the edges one by
    one in key order: every update sees the same loads, so the FP64 states agree exactly."""
    g = synth.chung_lu(400, 2400, 2.1, seed=5, block_size=20, block_p=0.6)
    order, _, _ = oracle_mod.level_order(g.n, g.u, g.v)
    _, rank = _key_sorted_adjacency(g.n, g.u, g.v)
    a = oracle_mod.LowdState(g.n, g.u, g.v)
    b = oracle_mod.LowdState(g.n, g.u, g.v)
    a.iterate(7, order=order)
    b.iterate(7, order=rank.astype(np.int32))
    assert np.array_equal(a.l, b.l) and np.array_equal(a.fu, b.fu)
