"""Helpers that compute the oracle's side of a parity check from the synthetic input alone
(nothing here reads a value produced by the CUDA path), plus the check that the GPU's
schedule has the oracle's colour classes in the oracle's order."""
import numpy as np


def oracle_graph(orc, g, prune):
    """The graph the passes run on: g canonicalised, then (if prune) Algorithm 2's core,
    relabelled by ascending id.  Returns (n, u, v, w or None, map to original ids)."""
    u, v, w, _ = orc.canonicalize(g.n, g.u, g.v, None if g.w is None else np.asarray(g.w, np.float64))
    if not prune:
        return g.n, u, v, w, np.arange(g.n, dtype=np.int32)
    wu, _ = orc.weight_units(u.shape[0], w)
    pr = orc.prune(g.n, u, v, wu, w is not None)
    keep = pr["removal_round"] < 0
    return orc.compact(g.n, u, v, w, keep)


def assert_same_schedule(orc, n, u, v, perm, offs, level=False):
    """The GPU's pass order (perm, class offsets) must visit the oracle's colour classes (the
    circle colouring, or with level=True the level order of the streamed schedule), as sets,
    in the same order (empty colours skipped); the order inside a class is free.  Returns the
    oracle's own order, which the oracle then replays."""
    order, _, colour = (orc.level_order if level else orc.circle_order)(n, u, v)
    perm = np.asarray(perm)
    offs = np.asarray(offs)
    m = np.asarray(u).shape[0]
    assert perm.shape[0] == m and np.array_equal(np.sort(perm), np.arange(m))
    sizes = np.diff(offs)
    assert offs[0] == 0 and offs[-1] == m and np.all(sizes > 0)
    cp = colour[perm]
    heads = cp[offs[:-1]]
    assert np.all(np.diff(heads) > 0)
    assert np.array_equal(cp, np.repeat(heads, sizes))
    return order
