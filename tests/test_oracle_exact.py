"""Pins for the oracle's exact solvers: min-cut densest subgraph and LDD.

Pinned against brute-force enumeration of every subset (Problem 1 and the LDD definition
of Sec. II, read straight off their definitions) on tiny graphs, and against closed forms:
a clique K_k has density (k-1)/2, a star or path on k nodes (k-1)/k, and two disjoint
equally dense cliques tie, so the maximal densest set is their union.
"""
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import brute


def _cases():
    out = []
    for seed in range(12):
        for kind in ("gnp0.2", "gnp0.45", "tree", "two_cliques", "star", "cycle", "path"):
            for weighted in (False, True):
                n = 5 + (seed * 3 + len(kind)) % 9
                out.append((kind, n, seed, weighted))
    return out


@pytest.mark.parametrize("kind,n,seed,weighted", _cases())
def test_flow_and_ldd_match_brute_force(oracle_mod, kind, n, seed, weighted):
    g = synth.small_family(kind, n, seed=seed, weighted=weighted)
    wu, _ = oracle_mod.weight_units(g.m, g.w)
    rho, mask = oracle_mod.densest_flow(g.n, g.u, g.v, wu)
    brho, bmask = brute.densest_brute(g.n, g.u, g.v, wu)
    assert rho == brho
    assert np.array_equal(mask, bmask)
    shell, lam = oracle_mod.ldd(g.n, g.u, g.v, wu)
    bshell, blam = brute.ldd_brute(g.n, g.u, g.v, wu)
    assert lam == blam
    assert np.array_equal(shell, bshell)
    # Property 2: lambda_1 > lambda_2 > ... and lambda_1 = rho*
    assert all(a > b for a, b in zip(lam, lam[1:]))
    assert lam[0] == rho


@pytest.mark.parametrize("k", [2, 3, 5, 8])
def test_closed_forms(oracle_mod, k):
    g = synth.small_family("clique", k)
    wu, _ = oracle_mod.weight_units(g.m, g.w)
    rho, mask = oracle_mod.densest_flow(g.n, g.u, g.v, wu)
    assert rho == Fraction(k - 1, 2) and mask.all()
    for kind in ("star", "path"):
        g = synth.small_family(kind, k)
        wu, _ = oracle_mod.weight_units(g.m, g.w)
        rho, mask = oracle_mod.densest_flow(g.n, g.u, g.v, wu)
        assert rho == Fraction(k - 1, k) and mask.all()


def test_tied_cliques_give_their_union(oracle_mod):
    # two disjoint K_5 (density 2 each) plus a pendant path: B_1 = both cliques
    pairs = [(i, j) for i in range(5) for j in range(i + 1, 5)]
    pairs += [(5 + i, 5 + j) for i in range(5) for j in range(i + 1, 5)]
    pairs += [(9, 10), (10, 11)]
    a = np.array(pairs)
    u = np.minimum(a[:, 0], a[:, 1]).astype(np.int32)
    v = np.maximum(a[:, 0], a[:, 1]).astype(np.int32)
    wu = np.ones(len(pairs), np.int64)
    rho, mask = oracle_mod.densest_flow(12, u, v, wu)
    assert rho == 2
    assert mask.tolist() == [True] * 10 + [False] * 2
    shell, lam = oracle_mod.ldd(12, u, v, wu)
    assert shell.tolist() == [1] * 10 + [2, 2]
    assert lam == [Fraction(2), Fraction(1)]


def test_flow_on_planted_block(oracle_mod):
    # sparse background (avg degree 4) + 64-node block at p=0.6: the block is far denser
    g = synth.planted_background(2000, 4.0, 64, 0.6, seed=5)
    wu, _ = oracle_mod.weight_units(g.m, g.w)
    rho, mask = oracle_mod.densest_flow(g.n, g.u, g.v, wu)
    assert set(g.block.tolist()) <= set(np.nonzero(mask)[0].tolist())
    # the block alone is a lower bound on rho*
    inb = np.zeros(g.n, bool); inb[g.block] = True
    wb = int(wu[inb[g.u] & inb[g.v]].sum())
    assert rho >= Fraction(wb, 64)
