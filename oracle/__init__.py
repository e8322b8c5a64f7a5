"""CPU oracle for LOWD with pruning and extraction (arXiv 2307.15969).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by
the CPU-baseline leg of ``bench.py``, never by the library.  The arithmetic lives in
``lowd_oracle.c`` (plain sequential C: double precision for Algorithm 1, exact integers
for weights, degrees and densities); this module compiles it with gcc and marshals
numpy arrays.  ``brute.py`` holds exhaustive solvers for tiny graphs.

Parity status of each function is stated in its docstring; every function is pinned by
``tests/test_oracle_*.py`` against closed forms, brute force, the exact min-cut solver,
or invariants the paper proves.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lowd_oracle.c")
_SRC_THREADS = os.path.join(_HERE, "lowd_threads.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblowd_oracle.so")
WEIGHT_SCALE = 1 << 20   # weighted graphs: integer units of 2^-20

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no target-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_THREADS))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC,
                               _SRC_THREADS, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.c_void_p
        i32, i64 = C.c_int32, C.c_int64
        lib.orc_canonicalize.restype = i64
        lib.orc_canonicalize.argtypes = [i32, i64, P, P, P, P, P, P, P]
        lib.orc_degrees.argtypes = [i32, i64, P, P, P, P]
        lib.orc_degree_order.argtypes = [i32, P, i32, P]
        lib.orc_prune.restype = i32
        lib.orc_prune.argtypes = [i32, i64, P, P, P, i32, P, P, P]
        lib.orc_lowd_update.restype = C.c_double
        lib.orc_lowd_update.argtypes = [P, P, P, P]
        lib.orc_lowd_init.argtypes = [i32, i64, P, P, P, P, P, P]
        lib.orc_lowd_iterate.argtypes = [i32, i64, P, P, P, i32, P, P, P, P]
        lib.orc_extract.restype = i32
        lib.orc_extract.argtypes = [i32, i64, P, P, P, P, P, P]
        lib.orc_greedy.argtypes = [i32, i64, P, P, P, P, P]
        lib.orc_densest_flow.restype = i32
        lib.orc_densest_flow.argtypes = [i32, i64, P, P, P, P, P, P]
        lib.orc_ldd.restype = i32
        lib.orc_ldd.argtypes = [i32, i64, P, P, P, P, P, P]
        lib.orc_load_stats.argtypes = [i32, P, P]
        lib.orc_lowd_iterate_threads.restype = i32
        lib.orc_lowd_iterate_threads.argtypes = [i32, i64, P, P, P, P, i32, i32, i32, P, P, P]
        lib.orc_star_update.restype = C.c_double
        lib.orc_star_update.argtypes = [i32, P, P, P, P]
        lib.orc_star_round.restype = i32
        lib.orc_star_round.argtypes = [i32, P, P, P, P, P, P, P, P, P]
        lib.orc_level_colouring.restype = i32
        lib.orc_level_colouring.argtypes = [i32, i64, P, P, P]
        _lib = lib
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ----------------------------------------------------------------------------- input

def canonicalize(n, u, v, w=None):
    """Undirected, loop-free, duplicate-free edges sorted by (lo, hi); a repeated pair
    keeps its first weight (Sec. IV: multiple edges and self-loops removed, direction
    ignored).  Raises ValueError on a self-loop or an id outside [0, n)."""
    lib = _load()
    u = _c(u, np.int32); v = _c(v, np.int32)
    m = u.shape[0]
    wd = None if w is None else _c(w, np.float64)
    ou = np.empty(max(m, 1), np.int32); ov = np.empty(max(m, 1), np.int32)
    ow = np.empty(max(m, 1), np.float64)
    ndup = np.zeros(1, np.int64)
    r = lib.orc_canonicalize(n, m, _p(u), _p(v), _p(wd), _p(ou), _p(ov), _p(ow), _p(ndup))
    if r == -1:
        raise ValueError("node id out of range")
    if r == -2:
        raise ValueError("self-loop")
    if r < 0:
        raise MemoryError
    return ou[:r].copy(), ov[:r].copy(), (None if w is None else ow[:r].copy()), int(ndup[0])


def weight_units(m: int, w) -> tuple[np.ndarray, int]:
    """Integer weight units and their scale: unit weights -> (1, scale 1); weighted ->
    (w * 2^20, scale 2^20), requiring every weight to lie on the 2^-20 grid."""
    if w is None:
        return np.ones(m, np.int64), 1
    x = np.asarray(w, np.float64) * WEIGHT_SCALE
    r = np.rint(x)
    if not np.all(r == x) or np.any(r <= 0):
        raise ValueError("weights must be positive multiples of 2^-20")
    return r.astype(np.int64), WEIGHT_SCALE


# ----------------------------------------------------------------------------- pruning

def degrees(n, u, v, wu):
    lib = _load()
    deg = np.zeros(n, np.int64)
    u = _c(u, np.int32); v = _c(v, np.int32); wu = _c(wu, np.int64)
    lib.orc_degrees(n, u.shape[0], _p(u), _p(v), _p(wu), _p(deg))
    return deg


def degree_order(deg, weighted: bool):
    """Nodes by degree ascending, ties by id (the counting sort of Sec. III-D)."""
    lib = _load()
    deg = _c(deg, np.int64)
    perm = np.empty(deg.shape[0], np.int32)
    lib.orc_degree_order(deg.shape[0], _p(deg), int(bool(weighted)), _p(perm))
    return perm


def prune(n, u, v, wu, weighted: bool):
    """Algorithm 2's pruning loop in synchronous rounds.  Returns
    dict(removal_round [n] (-1 kept, else 1-based round), rounds, W (units), N)."""
    lib = _load()
    u = _c(u, np.int32); v = _c(v, np.int32); wu = _c(wu, np.int64)
    if not weighted and u.shape[0] and not np.all(wu == 1):
        raise ValueError("unweighted pruning expects unit weights")
    rr = np.empty(n, np.int32)
    W = np.zeros(1, np.int64); N = np.zeros(1, np.int32)
    rounds = lib.orc_prune(n, u.shape[0], _p(u), _p(v), _p(wu), int(bool(weighted)),
                           _p(rr), _p(W), _p(N))
    if rounds < 0:
        raise MemoryError
    return dict(removal_round=rr, rounds=int(rounds), W=int(W[0]), N=int(N[0]))


def compact(n, u, v, w, keep_mask):
    """Sub-graph induced by the kept nodes: survivors relabelled by ascending original
    id, edges with both ends kept in their original order (Alg. 2: remove the pruned
    nodes and their edges).  Returns (n_H, u_H, v_H, w_H, map H-id -> original id)."""
    keep_mask = np.asarray(keep_mask, bool)
    ids = np.nonzero(keep_mask)[0].astype(np.int32)
    newid = np.full(n, -1, np.int64)
    newid[ids] = np.arange(ids.shape[0])
    ke = keep_mask[u] & keep_mask[v]
    uh = newid[np.asarray(u)[ke]].astype(np.int32)
    vh = newid[np.asarray(v)[ke]].astype(np.int32)
    wh = None if w is None else np.asarray(w)[ke]
    return int(ids.shape[0]), uh, vh, wh, ids


# ----------------------------------------------------------------------------- Algorithm 1

def lowd_update(lu, lv, fu, fv):
    """One application of Algorithm 1's loop body to an edge (u, v).
    Returns (lu, lv, fu, fv, d)."""
    lib = _load()
    a = np.array([lu, lv, fu, fv], np.float64)
    d = lib.orc_lowd_update(_p(a[0:]), _p(a[1:]), _p(a[2:]), _p(a[3:]))
    return float(a[0]), float(a[1]), float(a[2]), float(a[3]), float(d)


class LowdState:
    """Algorithm 1's state: the split vector f (f_e(u) and f_e(v) for every edge
    e = (u, v), u < v) and the node loads l."""

    def __init__(self, n, u, v, w=None):
        lib = _load()
        self.n = int(n)
        self.u = _c(u, np.int32)
        self.v = _c(v, np.int32)
        self.m = int(self.u.shape[0])
        self.w = np.ones(self.m) if w is None else _c(w, np.float64)
        self.fu = np.empty(self.m); self.fv = np.empty(self.m); self.l = np.empty(self.n)
        lib.orc_lowd_init(self.n, self.m, _p(self.u), _p(self.v), _p(self.w),
                          _p(self.fu), _p(self.fv), _p(self.l))
        self.iters = 0

    def iterate(self, T: int, order=None, record_sumsq: bool = False):
        """T passes of the edge loop in ``order`` (edge ids), default 0..m-1."""
        lib = _load()
        od = None if order is None else _c(order, np.int32)
        if od is not None and od.shape[0] != self.m:
            raise ValueError("order must list every edge once")
        ss = np.empty(max(T, 1)) if record_sumsq else None
        lib.orc_lowd_iterate(self.n, self.m, _p(self.u), _p(self.v), _p(od), int(T),
                             _p(self.fu), _p(self.fv), _p(self.l), _p(ss))
        self.iters += T
        return ss[:T] if record_sumsq else None

    def iterate_threads(self, T: int, order, class_offsets, threads: int):
        """T passes in ``order`` on ``threads`` host threads, one class at a time: the edges
        of class c are order[class_offsets[c]:class_offsets[c + 1]] and must form a matching
        (no two share a node), so the result equals iterate(T, order) exactly.  Used to time
        the oracle on all host cores (lowd_threads.c)."""
        lib = _load()
        od = _c(order, np.int32)
        off = _c(class_offsets, np.int64)
        if od.shape[0] != self.m or off[-1] != self.m:
            raise ValueError("order and class offsets must cover every edge once")
        r = lib.orc_lowd_iterate_threads(self.n, self.m, _p(self.u), _p(self.v), _p(od), _p(off),
                                         int(off.shape[0] - 1), int(T), int(threads),
                                         _p(self.fu), _p(self.fv), _p(self.l))
        if r != 0:
            raise RuntimeError("could not start the threads")
        self.iters += T

    def iterate_hub_star(self, T: int, plain_order, steps):
        """T hub-star passes (the hub-star block update): Algorithm 1 over the plain edges in
        plain_order, then every star step of `steps` (hub_star_structure): each star of the
        step is set to the exact minimiser of the sum of squared loads over its splits
        (star_update), the stars of a step being vertex-disjoint."""
        lib = _load()
        po = _c(plain_order, np.int32)
        hubs, beg, edges = [], [0], []
        for st in steps:
            for hub, es in st.items():
                hubs.append(int(hub))
                edges.extend(int(e) for e in es)
                beg.append(len(edges))
        hubs = np.asarray(hubs, np.int32)
        beg = np.asarray(beg, np.int64)
        edges = np.asarray(edges, np.int32)
        for _ in range(int(T)):
            if po.shape[0]:
                sub_u = self.u[po]
                sub_v = self.v[po]
                fu = self.fu[po].copy()
                fv = self.fv[po].copy()
                lib.orc_lowd_iterate(self.n, po.shape[0], _p(sub_u), _p(sub_v), None, 1,
                                     _p(fu), _p(fv), _p(self.l), None)
                self.fu[po] = fu
                self.fv[po] = fv
            if hubs.shape[0] and lib.orc_star_round(int(hubs.shape[0]), _p(hubs), _p(beg), _p(edges), _p(self.u),
                                                    _p(self.v), _p(self.w), _p(self.fu), _p(self.fv), _p(self.l)):
                raise MemoryError
        self.iters += T

    def stats(self):
        """(sum l, sum l^2, max l)."""
        lib = _load()
        out = np.zeros(3)
        lib.orc_load_stats(self.n, _p(self.l), _p(out))
        return float(out[0]), float(out[1]), float(out[2])


def circle_order(n, u, v):
    """The pass order of the parallel schedule, computed here from its definition.

    Algorithm 1 visits the edges one after another in any fixed order.  The GPU path
    groups them into the colour classes of the round-robin ("circle") tournament
    colouring of the complete graph on n nodes: with N' = n rounded up to even and
    P = N' - 1 (P = 1 when that is 0), edge {a, b}, a < b, has colour (a + b) mod P, or
    2a mod P when b = N' - 1.  Each class is a matching, so the order inside a class
    does not change the result of a pass; classes are visited in ascending colour.
    Returns (order, class_offsets[P + 1], colour): order lists edge ids class by class
    (by edge id inside a class).

    Parity pinned by tests/test_oracle_schedule.py: on K_n every class is a perfect (n
    even) or near-perfect (n odd) matching and every pair has exactly one colour; on
    random graphs every class is a matching."""
    u = np.asarray(u, np.int64)
    v = np.asarray(v, np.int64)
    a, b = np.minimum(u, v), np.maximum(u, v)
    Np = int(n) + (int(n) & 1)
    P = max(Np - 1, 1)
    colour = np.where(b == Np - 1, (2 * a) % P, (a + b) % P)
    order = np.argsort(colour, kind="stable").astype(np.int32)
    offs = np.searchsorted(colour[order], np.arange(P + 1)).astype(np.int64)
    return order, offs, colour


def level_order(n, u, v):
    """The pass order of the streamed schedule (graphs of any size), from its definition.

    Edges are ranked by the key (max(d_a, d_b), min(d_a, d_b), fmix32(edge id)), d the
    unweighted degree (light edges first; fmix32, MurmurHash3's 32-bit finaliser, a
    bijection, scrambles ties).  Visiting them in that order is one valid pass of Algorithm 1
    (the paper allows any order, Fig. 1 caption).  Its colour classes group the edges by
    level: colour(e) = 1 + max colour of the edges sharing an endpoint with e that come
    earlier in key order (0 if none).  Each class is a matching, and visiting the classes in
    ascending colour keeps the key order at every node, so it gives the same pass.
    Returns (order, class_offsets[C + 1], colour): order lists edge ids class by class, by
    edge id inside a class.

    Parity pinned by tests/test_oracle_schedule.py: the literal round process (every node
    designates its first uncoloured edge by key; an edge designated by both ends takes the
    round's colour) gives the same colours on random graphs; classes are matchings; stars,
    paths and cliques give their closed-form colour counts."""
    lib = _load()
    u = _c(u, np.int32); v = _c(v, np.int32)
    m = u.shape[0]
    colour = np.zeros(max(m, 1), np.int32)
    C = lib.orc_level_colouring(int(n), m, _p(u), _p(v), _p(colour))
    if C < 0:
        raise MemoryError
    colour = colour[:m]
    order = np.argsort(colour, kind="stable").astype(np.int32)
    offs = np.searchsorted(colour[order], np.arange(C + 1)).astype(np.int64)
    return order, offs, colour


def star_update(lh, l, w, t):
    """Exact minimisation of the sum of squared loads over the splits of one star (hub load
    lh, leaf loads l[j], edge weights w[j], t[j] = the hub's share f_e(h)), all other splits
    fixed: water filling, t_j = clip(B_j + w_j - lam, 0, w_j) with lam the hub's new load
    (lowd_oracle.c, orc_star_update).  Returns (lh, l, t, lam).

    Parity pinned by tests/test_oracle_stars.py: the KKT conditions of the star's quadratic
    program (interior shares leave the leaf at the hub's load, clipped ones on the right
    side of it); a one-leaf star equals Algorithm 1's edge update; many sequential passes of
    Algorithm 1 over the star's edges converge to the same loads."""
    lib = _load()
    l = _c(l, np.float64).copy()
    w = _c(w, np.float64)
    t = _c(t, np.float64).copy()
    lhv = np.array([lh], np.float64)
    lam = lib.orc_star_update(int(l.shape[0]), _p(lhv), _p(l), _p(w), _p(t))
    return float(lhv[0]), l, t, float(lam)


def hub_star_structure(n, u, v, tau: int):
    """The blocks of a hub-star pass, from their definition.  Hubs are the nodes of
    (unweighted) degree >= tau.  An edge with exactly one hub end is a star edge; every other
    edge is plain.  A leaf's star edges, ordered by its hub's degree (descending) then id,
    go to steps 0, 1, 2, ...; in step k the star edges grouped by hub form vertex-disjoint
    stars (one edge per leaf per step, hubs only as centres).  Returns (plain edge ids
    ascending, steps: list over k of dict hub -> array of star edge ids, ascending)."""
    u = np.asarray(u, np.int64)
    v = np.asarray(v, np.int64)
    m = u.shape[0]
    deg = np.bincount(u, minlength=n) + np.bincount(v, minlength=n)
    hub = deg >= tau
    star = hub[u] ^ hub[v]
    plain = np.nonzero(~star)[0].astype(np.int32)
    se = np.nonzero(star)[0]
    h = np.where(hub[u[se]], u[se], v[se])
    x = np.where(hub[u[se]], v[se], u[se])
    o = np.lexsort((h, -deg[h], x))            # by leaf, then hub degree desc, then hub id
    se, h, x = se[o], h[o], x[o]
    first = np.searchsorted(x, x, side="left")
    step = np.arange(se.shape[0]) - first
    steps = []
    for k in range(int(step.max()) + 1 if se.shape[0] else 0):
        sel = step == k
        hk, ek = h[sel], se[sel]
        d = {}
        for hh in np.unique(hk):
            d[int(hh)] = np.sort(ek[hk == hh]).astype(np.int32)
        steps.append(d)
    return plain, steps


def extract(n, u, v, wu, loads):
    """Algorithm 1's extraction.  Returns (S* ids ascending, W(S*) in units)."""
    lib = _load()
    u = _c(u, np.int32); v = _c(v, np.int32); wu = _c(wu, np.int64)
    l = _c(loads, np.float64)
    S = np.empty(max(n, 1), np.int32)
    Wb = np.zeros(1, np.int64)
    k = lib.orc_extract(n, u.shape[0], _p(u), _p(v), _p(wu), _p(l), _p(S), _p(Wb))
    if k < 0:
        raise MemoryError
    return S[:k].copy(), int(Wb[0])


# ----------------------------------------------------------------------------- exact solvers

def greedy(n, u, v, wu):
    """Algorithm 3 (Charikar's peeling).  Returns (removal order, W left after each)."""
    lib = _load()
    u = _c(u, np.int32); v = _c(v, np.int32); wu = _c(wu, np.int64)
    order = np.empty(n, np.int32); Wa = np.empty(n, np.int64)
    lib.orc_greedy(n, u.shape[0], _p(u), _p(v), _p(wu), _p(order), _p(Wa))
    return order, Wa


def densest_flow(n, u, v, wu):
    """Exact rho* (as a Fraction in weight units) and the maximal densest set B_1
    (bool mask), by min cuts (Goldberg's construction, Dinkelbach's iteration)."""
    lib = _load()
    u = _c(u, np.int32); v = _c(v, np.int32); wu = _c(wu, np.int64)
    inS = np.zeros(max(n, 1), np.int8)
    Wn = np.zeros(1, np.int64); kd = np.zeros(1, np.int64)
    k = lib.orc_densest_flow(n, u.shape[0], _p(u), _p(v), _p(wu), _p(inS), _p(Wn), _p(kd))
    if k < 0:
        raise OverflowError("min-cut capacities exceed 64 bits")
    return Fraction(int(Wn[0]), int(kd[0])), inS[:n].astype(bool)


def ldd(n, u, v, wu):
    """Exact locally-dense decomposition: shell index per node (1 = B_1) and the
    shell loads lambda_i as Fractions in weight units."""
    lib = _load()
    u = _c(u, np.int32); v = _c(v, np.int32); wu = _c(wu, np.int64)
    shell = np.zeros(max(n, 1), np.int32)
    num = np.zeros(max(n, 1), np.int64); den = np.zeros(max(n, 1), np.int64)
    k = lib.orc_ldd(n, u.shape[0], _p(u), _p(v), _p(wu), _p(shell), _p(num), _p(den))
    if k < 0:
        raise OverflowError("min-cut capacities exceed 64 bits")
    lam = [Fraction(int(num[i]), int(den[i])) for i in range(k)]
    return shell[:n].copy(), lam


def ldd_loads(n, u, v, wu, scale: int = 1):
    """The unique optimal loads l* (Properties 1-2): l*_x = lambda of x's shell."""
    shell, lam = ldd(n, u, v, wu)
    lamf = np.array([float(x) / scale for x in lam])
    return lamf[shell - 1] if n else np.zeros(0), shell, lam


def dks_bound(n, u, v, wu, k: int):
    """Corollary 1 from the exact decomposition: with |B_{j-1}| < k <= |B_j|, the bound
    (W(B_{j-1}) + (k - |B_{j-1}|) lambda_j) / k on the densest k-subgraph and at-least-k
    subgraph densities (reading: the corollary's lambda_i * |B_i| is lambda_i times the
    size of shell i, as its proof sums the loads of the k heaviest nodes).  Returns
    (Fraction in weight units, attained) where attained means k = |B_j|.

    Parity pinned by tests/test_oracle_dks.py against brute-force DkS and DalkS."""
    shell, lam = ldd(n, u, v, wu)
    sizes = np.bincount(shell, minlength=len(lam) + 1)[1:]
    if not 1 <= k <= int(sizes.sum()):
        raise ValueError("k out of range")
    prefix, prev = Fraction(0), 0
    for j, (sz, lj) in enumerate(zip(sizes.tolist(), lam)):
        if k <= prev + sz:
            return (prefix + (k - prev) * lj) / k, k == prev + sz
        prefix += lj * sz
        prev += sz
    raise AssertionError("unreachable")


# ----------------------------------------------------------------------------- full pipeline

def solve(n, u, v, w=None, T: int = 100, prune_first: bool = True, order=None):
    """Algorithm 2 with LOWD as the plug-in solver: prune, run T passes on the pruned
    graph, extract.  Returns a dict with the pruned graph, loads and S* (original ids)."""
    wu, scale = weight_units(u.shape[0], w)
    weighted = w is not None
    if prune_first:
        pr = prune(n, u, v, wu, weighted)
        keep = pr["removal_round"] < 0
    else:
        pr = None
        keep = np.ones(n, bool)
    nh, uh, vh, wh, idmap = compact(n, u, v, w, keep)
    st = LowdState(nh, uh, vh, None if wh is None else np.asarray(wh, np.float64))
    st.iterate(T, order=order)
    whu, _ = weight_units(uh.shape[0], wh)
    S, Wb = extract(nh, uh, vh, whu, st.l)
    return dict(prune=pr, n_H=nh, u_H=uh, v_H=vh, w_H=wh, map=idmap, state=st,
                S=idmap[S], W=Wb, k=int(S.shape[0]), scale=scale,
                rho=(Wb / scale / S.shape[0]) if S.shape[0] else 0.0)


def auto_hub_threshold(n, u, v, schedule: int = 2):
    """The automatic hub threshold of the hub-star pass.  Schedule 1: the smallest power of two
    p >= 2 with 2p >= the maximum (unweighted) degree.  Schedule 2: the smallest power of two
    2^k (k >= 1) such that at most 2^(k-1) nodes have degree >= 2^k (so at most half as many
    hubs as the threshold).  Returns an int (2^30 if no k up to 30 qualifies)."""
    deg = np.bincount(np.asarray(u, np.int64), minlength=n) + np.bincount(np.asarray(v, np.int64), minlength=n)
    if schedule == 1:
        dmax = int(deg.max()) if deg.shape[0] else 0
        p = 2
        while 2 * p < dmax and p < (1 << 30):
            p *= 2
        return p
    for k in range(1, 31):
        if int((deg >= (1 << k)).sum()) <= (1 << (k - 1)):
            return 1 << k
    return 1 << 30
