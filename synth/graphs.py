"""Seeded synthetic graphs with the shapes of the paper's workloads.

The paper measures on public power-law graphs (social, rating and citation networks,
17 unweighted and 9 weighted; Section IV, Table II).  Those datasets are not available
here, so these generators stand in for them: Chung-Lu and R-MAT give power-law degree
sequences, and a planted block gives a known dense core.  Multiple edges and self-loops
are removed and direction is ignored, as the paper does with its datasets (Section IV,
"Datasets & Implementation").

Every generator returns a canonical edge list: ``u < v``, no duplicates, no loops,
sorted by ``(u, v)``, int32 ids.  Weighted graphs carry float32 weights that lie on
the 2^-20 grid (see :func:`quantise_weights`), so that weighted degree and density
sums are exact in 64-bit fixed point on every side that consumes them.

Randomness comes only from ``numpy.random.Generator(PCG64(seed))``; the draws are in
a fixed order, so a recipe gives the same graph on any machine with numpy >= 1.17.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

WEIGHT_GRID_BITS = 20
_GRID = float(2 ** WEIGHT_GRID_BITS)


@dataclass
class Graph:
    n: int
    u: np.ndarray            # int32 [m], u < v
    v: np.ndarray            # int32 [m]
    w: np.ndarray | None     # float32 [m] on the 2^-20 grid, or None for unit weights
    block: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.u.shape[0])

    @property
    def weighted(self) -> bool:
        return self.w is not None


def quantise_weights(x: np.ndarray) -> np.ndarray:
    """Put positive weights on the 2^-20 grid and return them as float32.

    q(x) = round-half-even(x * 2^20) / 2^20, clamped to at least 2^-20.  Below 16 every
    grid value is an exact float32; at 16 and above every float32 is already a multiple
    of 2^-20, so the float32 rounding of the grid value is itself on the grid.
    """
    x = np.asarray(x, dtype=np.float64)
    q = np.maximum(np.rint(x * _GRID), 1.0) / _GRID
    out = q.astype(np.float32)
    # float32 rounding above 16 keeps the value on the grid; check the claim cheaply.
    back = out.astype(np.float64) * _GRID
    if not np.all(back == np.rint(back)):
        raise AssertionError("quantised weight left the 2^-20 grid")
    return out


# ----------------------------------------------------------------------------- helpers

def _canonical(lo: np.ndarray, hi: np.ndarray):
    a = np.minimum(lo, hi).astype(np.int64)
    b = np.maximum(lo, hi).astype(np.int64)
    keep = a != b
    return a[keep], b[keep]


def _keys(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return (a.astype(np.uint64) << np.uint64(32)) | b.astype(np.uint64)


def _unkey(k: np.ndarray):
    return ((k >> np.uint64(32)).astype(np.int32),
            (k & np.uint64(0xFFFFFFFF)).astype(np.int32))


def _first_index(keys: np.ndarray) -> np.ndarray:
    """Index of the first occurrence of every distinct key (in ascending key order).

    Large arrays are split by the key's top bits into buckets that are deduplicated in
    parallel threads (numpy's sort releases the GIL); the result is the same set of first
    indices as one np.unique(keys, return_index=True)."""
    if keys.shape[0] < (1 << 22):
        return np.unique(keys, return_index=True)[1]
    import concurrent.futures as cf
    import os
    top = int(keys.max()).bit_length()
    shift = np.uint64(max(top - 6, 0))
    bucket = (keys >> shift).astype(np.uint8)            # at most 64 buckets
    idx = np.argsort(bucket, kind="stable")               # a stable radix sort on uint8
    counts = np.bincount(bucket, minlength=64)
    bounds = np.concatenate([[0], np.cumsum(counts)])

    def one(b):
        ids = idx[bounds[b]:bounds[b + 1]]               # ascending positions
        if ids.shape[0] == 0:
            return ids
        return ids[np.unique(keys[ids], return_index=True)[1]]

    workers = max(1, min(16, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        parts = list(ex.map(one, range(64)))
    return np.concatenate(parts)


def _first_unique(keys: np.ndarray, target: int | None):
    """Unique keys in order of first occurrence, cut to ``target`` if given."""
    first = _first_index(keys)
    if target is not None and first.shape[0] < target:
        return None
    order = np.sort(first)
    if target is not None:
        order = order[:target]
    return keys[order]


def _union_sorted(keys: np.ndarray, extra: np.ndarray) -> np.ndarray:
    """Sorted union of two arrays of distinct keys (np.union1d's result, by sort and merge)."""
    ks = np.sort(keys)
    ex = np.unique(extra)
    if ks.shape[0] and ex.shape[0]:
        pos = np.minimum(np.searchsorted(ks, ex), ks.shape[0] - 1)
        ex = ex[ks[pos] != ex]
    out = np.concatenate([ks, ex])
    out.sort()
    return out


def _add_block(rng, n: int, keys: np.ndarray, size: int, p: float):
    """Planted block: ``size`` nodes drawn without replacement, each pair kept w.p. p.

    Returns (all keys, block node ids, block keys)."""
    size = min(size, n)
    nodes = np.sort(rng.choice(n, size=size, replace=False)).astype(np.int64)
    iu, ju = np.triu_indices(size, k=1)
    keep = rng.random(iu.shape[0]) < p
    bkeys = _keys(nodes[iu[keep]], nodes[ju[keep]])
    return _union_sorted(keys, bkeys), nodes.astype(np.int32), bkeys


def _finish(n, keys, w_of_key=None, block=None, name=""):
    keys = np.sort(keys)
    u, v = _unkey(keys)
    w = None
    if w_of_key is not None:
        w = w_of_key(keys)
    return Graph(n=n, u=u, v=v, w=w,
                 block=block if block is not None else np.zeros(0, np.int32),
                 name=name)


# ----------------------------------------------------------------------------- models

def chung_lu(n: int, m: int, gamma: float, seed: int, block_size: int = 0,
             block_p: float = 0.0, name: str = "") -> Graph:
    """Chung-Lu power-law graph with exactly ``m`` unique background edges.

    Expected-degree weights (i+1)^(-1/(gamma-1)) are assigned over a seeded random
    label permutation; endpoints are drawn i.i.d. proportional to them; loops and
    repeats are dropped (first occurrence kept) until exactly ``m`` edges exist.  A
    planted block of ``block_size`` nodes with pair probability ``block_p`` is then
    added (union with the background)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    perm = rng.permutation(n)
    wt = np.arange(1, n + 1, dtype=np.float64) ** (-1.0 / (gamma - 1.0))
    p = np.empty(n)
    p[perm] = wt / wt.sum()
    cdf = np.cumsum(p)
    cdf[-1] = 1.0
    if m > n * (n - 1) // 2:
        raise ValueError("m exceeds the number of node pairs")
    keys = np.zeros(0, np.uint64)
    batch = max(1024, int(m * 1.3))
    for _ in range(1000):
        a = np.searchsorted(cdf, rng.random(batch), side="right")
        b = np.searchsorted(cdf, rng.random(batch), side="right")
        lo, hi = _canonical(np.minimum(a, n - 1), np.minimum(b, n - 1))
        keys = np.concatenate([keys, _keys(lo, hi)])
        got = _first_unique(keys, m)
        if got is not None:
            keys = got
            break
        keys = _first_unique(keys, None)
        batch = max(1024, int((m - keys.shape[0]) * 2.0))
    else:  # pragma: no cover
        raise RuntimeError("Chung-Lu sampling did not reach m unique edges")
    block = None
    if block_size > 0:
        keys, block, _ = _add_block(rng, n, keys, block_size, block_p)
    return _finish(n, keys, block=block, name=name)


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int,
         block_size: int = 0, block_p: float = 0.0, weighted: bool = False,
         block_weight_scale: float = 3.0, name: str = "") -> Graph:
    """R-MAT graph with exactly ``edge_factor * 2^scale`` unique undirected edges.

    Each sample descends ``scale`` levels, choosing quadrant (a, b, c, d=1-a-b-c) with one
    float32 uniform per level; labels are then permuted by a seeded permutation; loops
    are dropped and repeats removed keeping the first occurrence, sampling further
    batches until the target is met (the last batch is cut in generation order).

    Weighted: background weights are lognormal(0, 1) quantised to the 2^-20 grid; the
    planted block's edges get quantise(block_weight_scale * lognormal(0, 1)) and replace
    any background weight on the same pair."""
    n = 1 << scale
    target = edge_factor * n
    rng = np.random.Generator(np.random.PCG64(seed))
    perm = rng.permutation(n).astype(np.int64)
    t_ab = np.float32(a + b)
    t_a = np.float32(a)
    t_abc = np.float32(a + b + c)
    keys = np.zeros(0, np.uint64)
    batch = int(target * 1.15)
    chunk = 1 << 23
    for _ in range(100):
        parts = []
        for start in range(0, batch, chunk):
            cnt = min(chunk, batch - start)
            src = np.zeros(cnt, np.int64)
            dst = np.zeros(cnt, np.int64)
            for lvl in range(scale):
                r = rng.random(cnt, dtype=np.float32)
                sb = r >= t_ab
                db = ((r >= t_a) & (r < t_ab)) | (r >= t_abc)
                bit = np.int64(1) << np.int64(lvl)
                src |= sb.astype(np.int64) * bit
                dst |= db.astype(np.int64) * bit
            lo, hi = _canonical(perm[src], perm[dst])
            parts.append(_keys(lo, hi))
        keys = np.concatenate([keys] + parts)
        got = _first_unique(keys, target)
        if got is not None:
            keys = got
            break
        keys = _first_unique(keys, None)
        batch = int((target - keys.shape[0]) * 1.5) + 1024
    else:  # pragma: no cover
        raise RuntimeError("R-MAT sampling did not reach the target edge count")
    bkeys = np.zeros(0, np.uint64)
    block = None
    if block_size > 0:
        keys, block, bkeys = _add_block(rng, n, keys, block_size, block_p)
    w_of_key = None
    if weighted:
        keys = np.sort(keys)
        wbg = quantise_weights(np.exp(rng.normal(0.0, 1.0, keys.shape[0])))
        if bkeys.shape[0]:
            bk = np.sort(bkeys)
            wb = quantise_weights(block_weight_scale * np.exp(rng.normal(0.0, 1.0, bk.shape[0])))
            pos = np.searchsorted(keys, bk)
            wbg[pos] = wb

        def w_of_key(sorted_keys, _w=wbg):
            return _w

    return _finish(n, keys, w_of_key=w_of_key, block=block, name=name)


def erdos_renyi(n: int, p: float, seed: int, weighted: bool = False,
                block_size: int = 0, block_p: float = 0.0, name: str = "") -> Graph:
    """G(n, p) with an optional planted block; weights lognormal(0,1) on the grid."""
    rng = np.random.Generator(np.random.PCG64(seed))
    iu, ju = np.triu_indices(n, k=1)
    keep = rng.random(iu.shape[0]) < p
    keys = _keys(iu[keep], ju[keep])
    block = None
    if block_size > 0:
        keys, block, _ = _add_block(rng, n, keys, block_size, block_p)
    keys = np.sort(keys)
    w_of_key = None
    if weighted:
        w = quantise_weights(np.exp(rng.normal(0.0, 1.0, keys.shape[0])))

        def w_of_key(sorted_keys, _w=w):
            return _w
    return _finish(n, keys, w_of_key=w_of_key, block=block, name=name)


def planted_background(n: int, avg_degree: float, block_size: int, block_p: float,
                       seed: int, weighted: bool = False, name: str = "") -> Graph:
    """Sparse G(n, m) background (m = n*avg_degree/2 unique pairs) plus a planted block.

    With avg_degree 4 and a 64-node block at p=0.6 the block's density (~19) is far
    above anything the background reaches, so the densest subgraph contains it."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = int(round(n * avg_degree / 2))
    keys = np.zeros(0, np.uint64)
    while True:
        a = rng.integers(0, n, size=2 * m)
        b = rng.integers(0, n, size=2 * m)
        lo, hi = _canonical(a, b)
        keys = np.concatenate([keys, _keys(lo, hi)])
        got = _first_unique(keys, m)
        if got is not None:
            keys = got
            break
    keys, block, _ = _add_block(rng, n, keys, block_size, block_p)
    keys = np.sort(keys)
    w_of_key = None
    if weighted:
        w = quantise_weights(np.exp(rng.normal(0.0, 1.0, keys.shape[0])))

        def w_of_key(sorted_keys, _w=w):
            return _w
    return _finish(n, keys, w_of_key=w_of_key, block=block, name=name)


def _from_pairs(n, pairs, w=None, name=""):
    keys = np.zeros(0, np.uint64)
    if len(pairs):
        arr = np.asarray(pairs, dtype=np.int64)
        lo, hi = _canonical(arr[:, 0], arr[:, 1])
        keys = _keys(lo, hi)
    uniq, idx = np.unique(keys, return_index=True)
    ww = None
    if w is not None:
        ww = quantise_weights(np.asarray(w, np.float64)[idx])
    u, v = _unkey(uniq)
    return Graph(n=n, u=u, v=v, w=ww, name=name)


def small_family(kind: str, n: int, seed: int = 0, weighted: bool = False) -> Graph:
    """Small structured graphs for edge cases: empty, star, path, clique, two cliques
    joined by a path, disjoint cliques, random trees, and G(n, p) at several p."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pairs = []
    if kind == "empty":
        pass
    elif kind == "star":
        pairs = [(0, i) for i in range(1, n)]
    elif kind == "path":
        pairs = [(i, i + 1) for i in range(n - 1)]
    elif kind == "cycle":
        pairs = [(i, (i + 1) % n) for i in range(n)] if n >= 3 else []
    elif kind == "clique":
        pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    elif kind == "two_cliques":
        h = n // 2
        pairs = [(i, j) for i in range(h) for j in range(i + 1, h)]
        pairs += [(h + i, h + j) for i in range(n - h) for j in range(i + 1, n - h) if i < j]
        if h >= 1 and n - h >= 1:
            pairs.append((h - 1, h))
    elif kind == "tree":
        pairs = [(i, int(rng.integers(0, i))) for i in range(1, n)]
    elif kind.startswith("gnp"):
        p = float(kind[3:]) if len(kind) > 3 else 0.3
        for i in range(n):
            for j in range(i + 1, n):
                if rng.random() < p:
                    pairs.append((i, j))
    else:
        raise ValueError(kind)
    w = None
    if weighted and pairs:
        w = np.exp(rng.normal(0.0, 1.0, len(pairs)))
    return _from_pairs(n, pairs, w, name=f"{kind}-{n}-{seed}")


# ----------------------------------------------------------------------------- workloads

WORKLOADS = {
    # Chung-Lu n=10k, m=100k, gamma 2.1, seed 0, 64-node block p=0.6, unit weights.
    "chunglu_10k": dict(kind="chung_lu", n=10_000, m=100_000, gamma=2.1, seed=0,
                        block_size=64, block_p=0.6),
    # R-MAT scale 22, edge factor 16, (.57,.19,.19,.05), 256-node block p=0.5, unit.
    "rmat22": dict(kind="rmat", scale=22, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=2,
                   block_size=256, block_p=0.5, weighted=False),
    # R-MAT scale 24, edge factor 8, lognormal weights, 512-node block p=0.5 weights x3.
    "rmat24w": dict(kind="rmat", scale=24, edge_factor=8, a=0.57, b=0.19, c=0.19, seed=3,
                    block_size=512, block_p=0.5, weighted=True, block_weight_scale=3.0),
    # Smaller R-MAT cases of the same recipe (parity at sizes the oracle finishes fast).
    "rmat16": dict(kind="rmat", scale=16, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=12,
                   block_size=128, block_p=0.5, weighted=False),
    "rmat16w": dict(kind="rmat", scale=16, edge_factor=8, a=0.57, b=0.19, c=0.19, seed=13,
                    block_size=128, block_p=0.5, weighted=True, block_weight_scale=3.0),
    "rmat18": dict(kind="rmat", scale=18, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=14,
                   block_size=256, block_p=0.5, weighted=False),
    # Dense G(n, p) cores with the size and density of the pruned R-MAT cores (scale 22:
    # 9,109 nodes at density 0.156; scale 18: 4,048 nodes at 0.125): small cases of the
    # same sweep for profiling.
    "dense9110": dict(kind="gnp", n=9110, p=0.156, seed=22),
    "dense4096": dict(kind="gnp", n=4096, p=0.12, seed=1),
}


def batch_graph(g: int, seed_base: int = 1000, n_lo: int = 100, n_hi: int = 20000,
                d_lo: float = 4.0, d_hi: float = 32.0, gamma_lo: float = 2.1,
                gamma_hi: float = 2.8, block_frac: float = 0.05, block_p: float = 0.5) -> Graph:
    """Graph g of the batched workload: a Chung-Lu graph with n ~ U{n_lo..n_hi}, average
    degree ~ U[d_lo, d_hi], exponent ~ U[gamma_lo, gamma_hi] (drawn from seed
    seed_base + g), target m = round(n * d / 2), plus a planted block of round(block_frac*n)
    nodes at pair probability block_p."""
    rng = np.random.Generator(np.random.PCG64(seed_base + g))
    n = int(rng.integers(n_lo, n_hi + 1))
    d = float(rng.uniform(d_lo, d_hi))
    gamma = float(rng.uniform(gamma_lo, gamma_hi))
    m = min(int(round(n * d / 2)), n * (n - 1) // 4)
    bs = max(2, int(round(block_frac * n)))
    return chung_lu(n, m, gamma, seed=int(rng.integers(0, 2**31 - 1)), block_size=bs, block_p=block_p,
                    name=f"batch{seed_base}-{g}")


def batch(count: int, seed_base: int = 1000, **kw) -> list[Graph]:
    """The first ``count`` graphs of the batched workload (see :func:`batch_graph`)."""
    return [batch_graph(g, seed_base=seed_base, **kw) for g in range(count)]


def workload(name: str) -> Graph:
    spec = dict(WORKLOADS[name])
    kind = spec.pop("kind")
    if kind == "chung_lu":
        return chung_lu(name=name, **spec)
    if kind == "rmat":
        return rmat(name=name, **spec)
    if kind == "gnp":
        return erdos_renyi(name=name, **spec)
    raise ValueError(kind)
