"""Pins for the oracle's Algorithm 1 (LOWD iterations) and its extraction.

Pinned against invariants the paper proves and exact solutions:
 - conservation sum(l) = sum(w) and the box 0 <= f_e(u) <= w_e (tighter dual, Sec. III-B);
 - sum(l^2) non-increasing per pass (Sec. III-C) and D_t = max l non-increasing (Thm. 1);
 - weak duality rho(S) <= rho* <= D_t for every iterate (Sec. III-B);
 - convergence of the loads to the exact LDD loads lambda_i (Thm. 2, Property 2), with
   lambda from brute force (tiny) or the min-cut solver (larger);
 - extraction on converged loads returns the maximal densest set B_1 (Sec. III-B);
 - the unweighted stopping certificate max l - rho(S) < 1/(n(n-1)) implies rho(S) = rho*;
 - extraction against a direct recount of every prefix density.
"""
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import brute


def _graph(kind, n, seed, weighted):
    return synth.small_family(kind, n, seed=seed, weighted=weighted)


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("seed", range(6))
def test_invariants_along_the_iteration(oracle_mod, seed, weighted):
    g = synth.chung_lu(300, 1500, 2.1, seed=seed, block_size=20, block_p=0.5)
    w = None
    if weighted:
        rng = np.random.default_rng(seed)
        w = synth.quantise_weights(np.exp(rng.normal(0, 1, g.m))).astype(np.float64)
    wu, scale = oracle_mod.weight_units(g.m, w)
    rho, _ = oracle_mod.densest_flow(g.n, g.u, g.v, wu)
    rho_f = float(rho) / scale
    st = oracle_mod.LowdState(g.n, g.u, g.v, w)
    wsum = float(st.w.sum())
    prev_ss, prev_D = np.inf, np.inf
    for t in range(60):
        ss = st.iterate(1, record_sumsq=True)[0]
        s, ss2, D = st.stats()
        assert abs(s - wsum) <= 1e-9 * wsum
        assert abs(ss - ss2) <= 1e-12 * ss2
        assert ss <= prev_ss * (1 + 1e-13)
        assert D <= prev_D * (1 + 1e-13)
        assert np.all(st.fu >= 0) and np.all(st.fv >= 0)
        assert np.allclose(st.fu + st.fv, st.w, rtol=1e-12, atol=0)
        S, WS = oracle_mod.extract(g.n, g.u, g.v, wu, st.l)
        rhoS = WS / scale / S.shape[0]
        assert rhoS <= rho_f * (1 + 1e-12)
        assert rho_f <= D * (1 + 1e-12)
        prev_ss, prev_D = ss, D


def _cases():
    out = []
    for seed in range(8):
        for kind in ("gnp0.25", "gnp0.5", "two_cliques", "tree"):
            for weighted in (False, True):
                out.append((kind, 6 + seed % 6, seed, weighted))
    return out


@pytest.mark.parametrize("kind,n,seed,weighted", _cases())
def test_converges_to_brute_force_ldd(oracle_mod, kind, n, seed, weighted):
    g = _graph(kind, n, seed, weighted)
    wu, scale = oracle_mod.weight_units(g.m, g.w)
    shell, lam = brute.ldd_brute(g.n, g.u, g.v, wu)
    lstar = np.array([float(lam[s - 1]) / scale for s in shell])
    st = oracle_mod.LowdState(g.n, g.u, g.v, None if g.w is None else g.w.astype(np.float64))
    st.iterate(4000)
    assert np.max(np.abs(st.l - lstar)) <= 1e-7 * max(1.0, lstar.max())
    S, WS = oracle_mod.extract(g.n, g.u, g.v, wu, st.l)
    assert S.tolist() == np.nonzero(shell == 1)[0].tolist()
    assert Fraction(WS, S.shape[0]) == lam[0]
    # Property 3 (one-way): an edge between shells gives nothing to the higher load
    hi_u = lstar[g.u] > lstar[g.v] + 1e-9
    hi_v = lstar[g.v] > lstar[g.u] + 1e-9
    assert np.all(st.fu[hi_u] <= 1e-6) and np.all(st.fv[hi_v] <= 1e-6)


def test_converges_to_min_cut_ldd_on_chung_lu(oracle_mod):
    g = synth.chung_lu(600, 3000, 2.1, seed=11, block_size=24, block_p=0.6)
    wu, scale = oracle_mod.weight_units(g.m, g.w)
    lstar, shell, lam = oracle_mod.ldd_loads(g.n, g.u, g.v, wu, scale)
    st = oracle_mod.LowdState(g.n, g.u, g.v)
    st.iterate(3000)
    assert np.max(np.abs(st.l - lstar)) <= 1e-4 * lstar.max()
    S, WS = oracle_mod.extract(g.n, g.u, g.v, wu, st.l)
    assert S.tolist() == np.nonzero(shell == 1)[0].tolist()


def test_unweighted_certificate(oracle_mod):
    # once max l - rho(S) < 1/(n(n-1)), S is a densest subgraph (Sec. III-B)
    for seed in range(5):
        g = synth.small_family("gnp0.3", 12, seed=seed)
        wu, _ = oracle_mod.weight_units(g.m, None)
        rho, _ = oracle_mod.densest_flow(g.n, g.u, g.v, wu)
        st = oracle_mod.LowdState(g.n, g.u, g.v)
        certified = False
        for t in range(3000):
            st.iterate(1)
            S, WS = oracle_mod.extract(g.n, g.u, g.v, wu, st.l)
            D = st.stats()[2]
            if D - WS / S.shape[0] < 1.0 / (g.n * (g.n - 1)):
                assert Fraction(WS, S.shape[0]) == rho
                certified = True
                break
        assert certified


def test_extract_matches_direct_prefix_recount(oracle_mod):
    rng = np.random.default_rng(3)
    for seed in range(30):
        n = int(rng.integers(2, 40))
        g = synth.small_family("gnp0.3", n, seed=seed, weighted=bool(seed % 2))
        wu, _ = oracle_mod.weight_units(g.m, g.w)
        # loads with many ties to exercise the (load, id) ordering
        loads = rng.integers(0, 4, size=n).astype(np.float64)
        S, WS = oracle_mod.extract(g.n, g.u, g.v, wu, loads)
        order = np.lexsort((np.arange(n), loads))[::-1]      # by (load, id) descending
        best_k, best = n, None
        for k in range(n, 0, -1):
            top = np.zeros(n, bool); top[order[:k]] = True
            Wk = int(wu[top[g.u] & top[g.v]].sum())
            f = Fraction(Wk, k)
            if best is None or f > best:
                best, best_k = f, k
        assert S.shape[0] == best_k
        assert sorted(S.tolist()) == sorted(order[:best_k].tolist())
        assert Fraction(WS, best_k) == best


def test_order_within_a_matching_does_not_matter(oracle_mod):
    # edges of a matching touch disjoint nodes, so their updates commute exactly
    g = synth.chung_lu(200, 800, 2.3, seed=2)
    m = g.m
    # greedy matching decomposition in edge-id order
    classes = []
    left = list(range(m))
    while left:
        used, cls, rest = set(), [], []
        for e in left:
            a, b = int(g.u[e]), int(g.v[e])
            if a in used or b in used:
                rest.append(e)
            else:
                used.update((a, b)); cls.append(e)
        classes.append(cls); left = rest
    o1 = np.concatenate([np.array(c) for c in classes]).astype(np.int32)
    o2 = np.concatenate([np.array(c[::-1]) for c in classes]).astype(np.int32)
    s1 = oracle_mod.LowdState(g.n, g.u, g.v); s1.iterate(20, order=o1)
    s2 = oracle_mod.LowdState(g.n, g.u, g.v); s2.iterate(20, order=o2)
    assert np.array_equal(s1.l, s2.l) and np.array_equal(s1.fu, s2.fu)
    s3 = oracle_mod.LowdState(g.n, g.u, g.v); s3.iterate(20)
    assert not np.array_equal(s1.l, s3.l)      # a different order gives other iterates


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_threaded_passes_equal_the_sequential_passes(oracle_mod, threads):
    """The all-cores timing variant (classes split over threads, a barrier per class) gives
    exactly the sequential oracle's state in the same order: the classes are matchings."""
    import synth
    g = synth.chung_lu(3000, 20000, 2.2, seed=31, block_size=30, block_p=0.5)
    w = synth.quantise_weights(np.random.default_rng(8).lognormal(0, 1, g.m)).astype(np.float64)
    for order, offs, _ in (oracle_mod.circle_order(g.n, g.u, g.v), oracle_mod.level_order(g.n, g.u, g.v)):
        a = oracle_mod.LowdState(g.n, g.u, g.v, w)
        b = oracle_mod.LowdState(g.n, g.u, g.v, w)
        a.iterate(6, order=order)
        b.iterate_threads(6, order, offs, threads)
        assert np.array_equal(a.l, b.l) and np.array_equal(a.fu, b.fu) and np.array_equal(a.fv, b.fv)
