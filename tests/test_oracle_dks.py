"""Corollary 1 in the oracle against exhaustive search: for every k the bound is at least
the densest k-subgraph density and the densest at-least-k subgraph density, with equality
when k is the size of some B_j (item 1)."""
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle.brute import _popcount, _subset_weights


def _brute_dks(n, u, v, wu):
    W = _subset_weights(n, u, v, wu)
    c = _popcount(n)
    dks = [Fraction(0)] * (n + 1)
    for s in range(1, 1 << n):
        k = int(c[s])
        f = Fraction(int(W[s]), k)
        if f > dks[k]:
            dks[k] = f
    dalks = [max(dks[k:]) for k in range(n + 1)]
    return dks, dalks


CASES = [("two_cliques", 12, 0), ("gnp0.3", 11, 1), ("gnp0.5", 10, 2), ("star", 9, 0)]


@pytest.mark.parametrize("fam,n,seed", CASES)
@pytest.mark.parametrize("weighted", [False, True])
def test_dks_bound_against_brute_force(oracle_mod, fam, n, seed, weighted):
    g = synth.small_family(fam, n, seed=seed)
    if g.m == 0:
        pytest.skip("no edges")
    wu = (np.random.default_rng(seed).integers(1, 9, g.m).astype(np.int64) if weighted
          else np.ones(g.m, np.int64))
    dks, dalks = _brute_dks(g.n, g.u, g.v, wu)
    shell, lam = oracle_mod.ldd(g.n, g.u, g.v, wu)
    ends = set(np.cumsum(np.bincount(shell, minlength=len(lam) + 1)[1:]).tolist())
    for k in range(1, g.n + 1):
        b, attained = oracle_mod.dks_bound(g.n, g.u, g.v, wu, k)
        assert attained == (k in ends)
        assert dks[k] <= b and dalks[k] <= b, (k, dks[k], dalks[k], b)
        if attained:
            assert dks[k] == b and dalks[k] == b, k
    # k = n: the bound is the whole graph's density
    assert oracle_mod.dks_bound(g.n, g.u, g.v, wu, g.n)[0] == Fraction(int(wu.sum()), g.n)


def test_dks_bound_rejects_k_out_of_range(oracle_mod):
    g = synth.small_family("two_cliques", 8)
    wu = np.ones(g.m, np.int64)
    for k in (0, g.n + 1):
        with pytest.raises(ValueError):
            oracle_mod.dks_bound(g.n, g.u, g.v, wu, k)


def test_library_bound_is_host_arithmetic_matching_the_oracle(oracle_mod):
    """lowd_ldd_dks_bound is plain host arithmetic on (lambda, shell_end): fed the oracle's
    exact decomposition it reproduces the oracle's bound (no GPU involved)."""
    from paper_2307_15969_gb300 import lowd as L
    from paper_2307_15969_gb300 import build
    build.build()
    g = synth.small_family("two_cliques", 14)
    wu = np.ones(g.m, np.int64)
    shell, lam = oracle_mod.ldd(g.n, g.u, g.v, wu)
    end = np.cumsum(np.bincount(shell, minlength=len(lam) + 1)[1:]).astype(np.int32)
    lamf = np.array([float(x) for x in lam])
    for k in range(1, g.n + 1):
        b, ex = L.lowd_ldd_dks_bound(lamf, end, k)
        bo, exo = oracle_mod.dks_bound(g.n, g.u, g.v, wu, k)
        assert ex == exo and abs(b - float(bo)) <= 1e-14 * float(bo)
    with pytest.raises(L.LowdError):
        L.lowd_ldd_dks_bound(lamf, end, 0)
    with pytest.raises(L.LowdError):
        L.lowd_ldd_dks_bound(lamf, end, g.n + 1)
