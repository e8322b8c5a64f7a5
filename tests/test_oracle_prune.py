"""Pins for the oracle's input canonicalisation, degree order and Algorithm 2 (pruning).

Pinned against: numpy's own unique/argsort (library routines for the plain definitions
of a deduplicated edge list and a stable sort by degree); properties Theorem 3 and the
proof of Theorem 4 establish - every kept node has d_H(u) >= rho(H), rho(H) strictly
increases over rounds, the densest subgraph survives, and no node is removed that a
fixpoint test would keep; and Greedy (Algorithm 3) reaching the pruned graph exactly
where its density stops increasing (Theorem 4).
"""
from fractions import Fraction

import numpy as np
import pytest

import synth


def test_canonicalize_against_numpy_unique(oracle_mod):
    rng = np.random.default_rng(0)
    for trial in range(20):
        n = int(rng.integers(2, 60))
        m = int(rng.integers(0, 300))
        a = rng.integers(0, n, m); b = rng.integers(0, n, m)
        keep = a != b
        a, b = a[keep], b[keep]
        w = rng.uniform(0.5, 2, a.shape[0])
        u, v, ww, ndup = oracle_mod.canonicalize(n, a, b, w)
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        keys = lo.astype(np.int64) * n + hi
        uk, first = np.unique(keys, return_index=True)
        assert np.array_equal(u, lo[first]) and np.array_equal(v, hi[first])
        assert np.array_equal(ww, w[first])
        assert ndup == a.shape[0] - uk.shape[0]
    with pytest.raises(ValueError):
        oracle_mod.canonicalize(3, [0], [0])
    with pytest.raises(ValueError):
        oracle_mod.canonicalize(3, [0], [3])


@pytest.mark.parametrize("weighted", [False, True])
def test_degree_order_is_stable_sort(oracle_mod, weighted):
    g = synth.chung_lu(3000, 12000, 2.1, seed=4)
    w = None
    if weighted:
        w = synth.quantise_weights(np.random.default_rng(1).lognormal(0, 1, g.m)).astype(np.float64)
    wu, _ = oracle_mod.weight_units(g.m, w)
    deg = oracle_mod.degrees(g.n, g.u, g.v, wu)
    assert np.array_equal(deg, np.bincount(g.u, wu, g.n).astype(np.int64)
                          + np.bincount(g.v, wu, g.n).astype(np.int64))
    perm = oracle_mod.degree_order(deg, weighted)
    assert np.array_equal(perm, np.argsort(deg, kind="stable"))


def _prune_cases():
    out = []
    for seed in range(6):
        out.append(("chung_lu", seed, False))
        out.append(("chung_lu", seed, True))
        out.append(("planted", seed, False))
    return out


def _make(kind, seed, weighted):
    if kind == "chung_lu":
        g = synth.chung_lu(1500, 6000, 2.1 + 0.1 * seed, seed=seed, block_size=30, block_p=0.5)
    else:
        g = synth.planted_background(1500, 4.0, 40, 0.6, seed=seed)
    w = None
    if weighted:
        w = synth.quantise_weights(np.random.default_rng(seed).lognormal(0, 1, g.m)).astype(np.float64)
    return g, w


@pytest.mark.parametrize("kind,seed,weighted", _prune_cases())
def test_prune_properties(oracle_mod, kind, seed, weighted):
    g, w = _make(kind, seed, weighted)
    wu, scale = oracle_mod.weight_units(g.m, w)
    pr = oracle_mod.prune(g.n, g.u, g.v, wu, weighted)
    rr = pr["removal_round"]
    keep = rr < 0
    # the pruned graph H and its density
    ke = keep[g.u] & keep[g.v]
    W_H = int(wu[ke].sum()); N_H = int(keep.sum())
    assert (W_H, N_H) == (pr["W"], pr["N"])
    # fixpoint: every kept node has d_H(u) >= rho(H)
    dH = np.bincount(g.u[ke], wu[ke], g.n) + np.bincount(g.v[ke], wu[ke], g.n)
    assert np.all(dH[keep].astype(object) * N_H >= W_H)
    # rounds: each removed node had d < rho of the graph at the start of its round,
    # the density strictly increases from round to round (proof of Theorem 4)
    alive = np.ones(g.n, bool)
    prev = None
    for r in range(1, pr["rounds"] + 1):
        ea = alive[g.u] & alive[g.v]
        Wr = int(wu[ea].sum()); Nr = int(alive.sum())
        d = np.bincount(g.u[ea], wu[ea], g.n) + np.bincount(g.v[ea], wu[ea], g.n)
        below = alive & (d.astype(object) * Nr < Wr)
        assert np.array_equal(below, rr == r)           # exactly the nodes below the bound
        f = Fraction(Wr, Nr)
        if prev is not None:
            assert f > prev
        prev = f
        alive &= ~below
    assert np.array_equal(alive, keep)
    # Theorem 3: the maximal densest subgraph survives pruning
    rho, mask = oracle_mod.densest_flow(g.n, g.u, g.v, wu)
    assert np.all(keep[mask])
    assert Fraction(W_H, N_H) <= rho


@pytest.mark.parametrize("seed", range(8))
def test_prune_equals_greedy_at_first_non_increase(oracle_mod, seed):
    # Theorem 4: Greedy's remaining graph when its density first stops increasing is H.
    g = synth.chung_lu(400, 1600, 2.2, seed=seed, block_size=16, block_p=0.6)
    wu, _ = oracle_mod.weight_units(g.m, None)
    pr = oracle_mod.prune(g.n, g.u, g.v, wu, False)
    order, W_after = oracle_mod.greedy(g.n, g.u, g.v, wu)
    W_before = np.concatenate([[int(wu.sum())], W_after[:-1]])
    n_before = g.n - np.arange(g.n)
    for i in range(g.n - 1):
        # density before removal i vs after it
        if Fraction(int(W_after[i]), int(n_before[i] - 1)) <= Fraction(int(W_before[i]), int(n_before[i])):
            remaining = np.ones(g.n, bool); remaining[order[:i]] = False
            assert np.array_equal(remaining, pr["removal_round"] < 0)
            break
    else:
        pytest.fail("density never stopped increasing")


@pytest.mark.parametrize("weighted", [False, True])
def test_prune_keeps_exact_ties(oracle_mod, weighted):
    # Alg. 2 removes only nodes with d_H(u) < rho(H), strictly.
    if weighted:
        # triangle of unit weights + a separate edge of weight 3/4: rho = 3.75/5 = 0.75,
        # and the separate edge's ends have degree exactly 0.75
        u = np.array([0, 0, 1, 3], np.int32); v = np.array([1, 2, 2, 4], np.int32)
        w = np.array([1.0, 1.0, 1.0, 0.75])
        n = 5
    else:
        # 4-cycle + pendant node: W = N = 5, rho = 1, the pendant has degree exactly 1
        u = np.array([0, 1, 2, 0, 0], np.int32); v = np.array([1, 2, 3, 3, 4], np.int32)
        w = None
        n = 5
    wu, _ = oracle_mod.weight_units(u.shape[0], w)
    pr = oracle_mod.prune(n, u, v, wu, weighted)
    assert pr["rounds"] == 0 and np.all(pr["removal_round"] < 0)
    # one unit less on the pendant side tips it over: now it is removed in round 1
    if not weighted:
        u2 = np.array([0, 1, 2, 0, 0, 1], np.int32); v2 = np.array([1, 2, 3, 3, 4, 3], np.int32)
        pr = oracle_mod.prune(n, u2, v2, np.ones(6, np.int64), False)
        assert pr["removal_round"].tolist() == [-1, -1, -1, -1, 1]
