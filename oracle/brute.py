"""Exhaustive solvers for tiny graphs (n <= 16), used to pin the oracle.

TEST INFRASTRUCTURE ONLY.  These enumerate every node subset and read the answers
straight off the definitions: the density W(S)/|S| (Sec. II), Problem 1 (densest
subgraph) and the definition of the locally-dense decomposition (Sec. II).  Exact
integer / Fraction arithmetic throughout.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def _subset_weights(n, u, v, wu):
    """W(S) for every bitmask S in [0, 2^n)."""
    S = np.arange(1 << n, dtype=np.int64)
    W = np.zeros(1 << n, dtype=np.int64)
    for a, b, w in zip(np.asarray(u).tolist(), np.asarray(v).tolist(), np.asarray(wu).tolist()):
        mask = (1 << a) | (1 << b)
        W += np.where((S & mask) == mask, w, 0)
    return W


def _popcount(n):
    S = np.arange(1 << n, dtype=np.int64)
    c = np.zeros(1 << n, dtype=np.int64)
    for i in range(n):
        c += (S >> i) & 1
    return c


def densest_brute(n, u, v, wu):
    """rho* = max over non-empty S of W(S)/|S|, and the maximal maximiser (the union
    of all maximisers, itself a maximiser).  Returns (Fraction, bool mask)."""
    if n == 0:
        return Fraction(0), np.zeros(0, bool)
    W = _subset_weights(n, u, v, wu)
    k = _popcount(n)
    best = Fraction(0)
    for s in range(1, 1 << n):
        f = Fraction(int(W[s]), int(k[s]))
        if f > best:
            best = f
    union = 0
    for s in range(1, 1 << n):
        if int(W[s]) * best.denominator == best.numerator * int(k[s]):
            union |= s
    mask = np.array([(union >> i) & 1 for i in range(n)], bool)
    return best, mask


def ldd_brute(n, u, v, wu):
    """Locally-dense decomposition straight from its definition: B_0 = {}, B_i the
    maximal S strictly containing B_{i-1} maximising (W(S)-W(B_{i-1}))/|S \\ B_{i-1}|.
    Returns (shell index per node, 1-based; list of lambda_i Fractions)."""
    W = _subset_weights(n, u, v, wu)
    k = _popcount(n)
    full = (1 << n) - 1
    B = 0
    shells = np.zeros(n, np.int32)
    lams = []
    i = 0
    while B != full:
        i += 1
        best = None
        for s in range(1 << n):
            if (s & B) != B or s == B:
                continue
            f = Fraction(int(W[s] - W[B]), int(k[s] - k[B]))
            if best is None or f > best:
                best = f
        union = B
        for s in range(1 << n):
            if (s & B) != B or s == B:
                continue
            if Fraction(int(W[s] - W[B]), int(k[s] - k[B])) == best:
                union |= s
        for x in range(n):
            if (union >> x) & 1 and not (B >> x) & 1:
                shells[x] = i
        lams.append(best)
        B = union
    return shells, lams
