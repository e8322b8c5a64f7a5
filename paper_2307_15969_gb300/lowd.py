"""Python binding of the LOWD C ABI (include/lowd.h): argument marshalling only.

Every function has the C name and forwards to ``liblowd.so``; no step of the method runs
here.  Arrays may be numpy arrays (host mode) or CUDA torch tensors (device mode, chosen
by the first array given to :func:`lowd_load_graph`); outputs come back in the same mode.
The library must have been built (``python -m paper_2307_15969_gb300.build`` or
``__graft_entry__.build()``); if it is missing, loading fails with an error rather than
falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblowd.so")

LOWD_OK = 0
LOWD_ERR_INVALID_ARG = 1
LOWD_ERR_OUT_OF_MEMORY = 2
LOWD_ERR_CUDA = 3
LOWD_ERR_BAD_STATE = 4
LOWD_ERR_NOT_CONVERGED = 5
LOWD_ERR_INEXACT_WEIGHTS = 6
LOWD_ERR_TOO_LARGE = 7
LOWD_MEM_HOST = 0
LOWD_MEM_DEVICE = 1
LOWD_LOAD_ALLOW_INEXACT = 1

EXPORTED = (
    "lowd_load_graph", "lowd_prune", "lowd_iterate", "lowd_extract", "lowd_get_info",
    "lowd_get_graph", "lowd_get_splits", "lowd_set_splits", "lowd_get_loads",
    "lowd_get_prune_info", "lowd_get_edge_order", "lowd_free", "lowd_status_string",
    "lowd_last_error", "lowd_launch_count", "lowd_extract_noalloc",
    "lowd_batch_create", "lowd_batch_run", "lowd_batch_autotune", "lowd_batch_results",
    "lowd_batch_free", "lowd_batch_last_error", "lowd_batch_loads", "lowd_batch_core", "lowd_get_ldd",
    "lowd_ldd_dks_bound", "lowd_mpnn_param_count", "lowd_mpnn_create", "lowd_mpnn_set_params",
    "lowd_mpnn_get_params", "lowd_mpnn_bind", "lowd_mpnn_set_features", "lowd_mpnn_forward", "lowd_mpnn_backward", "lowd_mpnn_adam",
    "lowd_mpnn_read", "lowd_warm_start", "lowd_mpnn_last_error", "lowd_mpnn_free",
    "lowd_selftest_barrier_timeout",
)
LOWD_MPNN_SIGMA = 1
LOWD_MPNN_LOADS = 2
LOWD_MPNN_GRAD = 3
LOWD_MPNN_FEATURES = 4
LOWD_MPNN_PHI = 5
LOWD_BATCH_ORDER_AS_GIVEN = 1
LOWD_BATCH_ORDER_LARGEST_FIRST = 2


class lowd_options(C.Structure):
    _fields_ = [("check_every", C.c_int32), ("rel_tol", C.c_double),
                ("schedule", C.c_int32), ("rederive_every", C.c_int32), ("node_versions", C.c_int32),
                ("hub_stars", C.c_int32)]


class lowd_stats(C.Structure):
    _fields_ = [("iters_done", C.c_int32), ("checks_done", C.c_int32), ("sum_load", C.c_double),
                ("sum_load_sq", C.c_double), ("max_load", C.c_double), ("rho_best", C.c_double),
                ("best_size", C.c_int32), ("converged", C.c_int32)]


class lowd_info(C.Structure):
    _fields_ = [("n_orig", C.c_int32), ("n", C.c_int32), ("m_orig", C.c_int64), ("m", C.c_int64),
                ("duplicates", C.c_int64), ("weighted", C.c_int32), ("pruned", C.c_int32),
                ("classes", C.c_int32), ("schedule", C.c_int32), ("max_degree", C.c_int32),
                ("prune_rounds", C.c_int32), ("sweep_kernel", C.c_int32),
                ("sweep_edges_per_thread", C.c_int32), ("star_threshold", C.c_int32),
                ("star_steps", C.c_int32), ("stars", C.c_int32), ("star_edges", C.c_int64)]


class lowd_batch_options(C.Structure):
    _fields_ = [("passes", C.c_int32), ("ctas_per_sm", C.c_int32), ("threads", C.c_int32),
                ("order", C.c_int32)]


class LowdError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {lowd_status_string(status)} ({status})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


_lib = None


def load_library(path: str = LIB_PATH):
    """Load liblowd.so and declare its signatures.  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"liblowd.so not built at {path}: run paper_2307_15969_gb300.build.build()")
    lib = C.CDLL(path)
    P, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    lib.lowd_load_graph.restype = i32
    lib.lowd_load_graph.argtypes = [i32, i64, P, P, P, i32, i32, P, C.POINTER(P)]
    lib.lowd_prune.restype = i32
    lib.lowd_prune.argtypes = [P, C.POINTER(i32), C.POINTER(i64), C.POINTER(i32)]
    lib.lowd_iterate.restype = i32
    lib.lowd_iterate.argtypes = [P, i32, C.POINTER(lowd_options), C.POINTER(lowd_stats)]
    lib.lowd_extract.restype = i32
    lib.lowd_extract.argtypes = [P, P, C.POINTER(i32), C.POINTER(C.c_double), P]
    lib.lowd_get_ldd.restype = i32
    lib.lowd_get_ldd.argtypes = [P, C.c_double, P, P, P, C.POINTER(i32)]
    lib.lowd_ldd_dks_bound.restype = i32
    lib.lowd_ldd_dks_bound.argtypes = [i32, P, P, i32, C.POINTER(C.c_double), C.POINTER(i32)]
    lib.lowd_mpnn_param_count.restype = C.c_int64
    lib.lowd_mpnn_param_count.argtypes = []
    lib.lowd_mpnn_create.restype = i32
    lib.lowd_mpnn_create.argtypes = [P, C.POINTER(C.c_void_p)]
    lib.lowd_mpnn_set_params.restype = i32
    lib.lowd_mpnn_set_params.argtypes = [P, P, i32]
    lib.lowd_mpnn_get_params.restype = i32
    lib.lowd_mpnn_get_params.argtypes = [P, P, i32]
    lib.lowd_mpnn_bind.restype = i32
    lib.lowd_mpnn_bind.argtypes = [P, i32, C.c_int64, P, P, P, P, i32]
    lib.lowd_mpnn_set_features.restype = i32
    lib.lowd_mpnn_set_features.argtypes = [P, P, i32]
    lib.lowd_mpnn_forward.restype = i32
    lib.lowd_mpnn_forward.argtypes = [P, C.POINTER(C.c_double)]
    lib.lowd_mpnn_backward.restype = i32
    lib.lowd_mpnn_backward.argtypes = [P]
    lib.lowd_mpnn_adam.restype = i32
    lib.lowd_mpnn_adam.argtypes = [P, C.c_float, C.c_float, C.c_float, C.c_float]
    lib.lowd_mpnn_read.restype = i32
    lib.lowd_mpnn_read.argtypes = [P, i32, P, i32]
    lib.lowd_warm_start.restype = i32
    lib.lowd_warm_start.argtypes = [P, P]
    lib.lowd_mpnn_last_error.restype = C.c_char_p
    lib.lowd_mpnn_last_error.argtypes = [P]
    lib.lowd_mpnn_free.restype = None
    lib.lowd_mpnn_free.argtypes = [P]
    lib.lowd_get_info.restype = i32
    lib.lowd_get_info.argtypes = [P, C.POINTER(lowd_info)]
    lib.lowd_get_graph.restype = i32
    lib.lowd_get_graph.argtypes = [P, P, P, P]
    lib.lowd_get_splits.restype = i32
    lib.lowd_get_splits.argtypes = [P, P]
    lib.lowd_set_splits.restype = i32
    lib.lowd_set_splits.argtypes = [P, P]
    lib.lowd_get_loads.restype = i32
    lib.lowd_get_loads.argtypes = [P, P]
    lib.lowd_get_prune_info.restype = i32
    lib.lowd_get_prune_info.argtypes = [P, P, P]
    lib.lowd_get_edge_order.restype = i32
    lib.lowd_get_edge_order.argtypes = [P, P, P, C.POINTER(i32)]
    lib.lowd_free.restype = None
    lib.lowd_free.argtypes = [P]
    lib.lowd_status_string.restype = C.c_char_p
    lib.lowd_status_string.argtypes = [i32]
    lib.lowd_last_error.restype = C.c_char_p
    lib.lowd_last_error.argtypes = [P]
    lib.lowd_launch_count.restype = C.c_uint64
    lib.lowd_launch_count.argtypes = []
    lib.lowd_selftest_barrier_timeout.restype = i32
    lib.lowd_selftest_barrier_timeout.argtypes = [C.POINTER(i32)]
    lib.lowd_batch_create.restype = i32
    lib.lowd_batch_create.argtypes = [i32, P, P, P, P, i32, P, C.POINTER(P)]
    lib.lowd_batch_run.restype = i32
    lib.lowd_batch_run.argtypes = [P, C.POINTER(lowd_batch_options)]
    lib.lowd_batch_autotune.restype = i32
    lib.lowd_batch_autotune.argtypes = [P, i32, i32, C.POINTER(lowd_batch_options)]
    lib.lowd_batch_results.restype = i32
    lib.lowd_batch_results.argtypes = [P, P, P, P, P, P, P, P]
    lib.lowd_batch_core.restype = i32
    lib.lowd_batch_core.argtypes = [P, P]
    lib.lowd_batch_loads.restype = i32
    lib.lowd_batch_loads.argtypes = [P, P]
    lib.lowd_batch_last_error.restype = C.c_char_p
    lib.lowd_batch_last_error.argtypes = [P]
    lib.lowd_batch_free.restype = None
    lib.lowd_batch_free.argtypes = [P]
    lib.lowd_extract_noalloc.restype = i32
    lib.lowd_extract_noalloc.argtypes = [i32, i64, P, P, P, P, P, C.POINTER(i32), C.POINTER(C.c_double), P]
    _lib = lib
    return lib


def lowd_status_string(status: int) -> str:
    return load_library().lowd_status_string(int(status)).decode()


def lowd_launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load_library().lowd_launch_count())


def lowd_selftest_barrier_timeout():
    """The bounded grid barrier's expiry path (see include/lowd.h); returns (status, error word)."""
    bits = C.c_int32()
    s = load_library().lowd_selftest_barrier_timeout(C.byref(bits))
    return s, bits.value


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


class Handle:
    """An open LOWD handle (the C ``lowd_handle``) and the memory mode of its arrays."""

    def __init__(self, ptr: int, device: bool, n0: int, stream):
        self.ptr = C.c_void_p(ptr)
        self.device = device
        self.n0 = n0
        self.stream = stream

    def __del__(self):
        try:
            lowd_free(self)
        except Exception:
            pass

    def _check(self, status: int, where: str):
        if status != LOWD_OK:
            detail = load_library().lowd_last_error(self.ptr).decode() if self.ptr else ""
            raise LowdError(status, where, detail)

    # array helpers: allocate an output in this handle's memory mode
    def empty(self, n: int, dtype):
        if self.device:
            import torch
            td = {np.int32: torch.int32, np.float32: torch.float32}[dtype]
            return torch.empty(max(int(n), 1), dtype=td, device="cuda")
        return np.empty(max(int(n), 1), dtype=dtype)

    def ptr_of(self, a):
        if a is None:
            return None
        if self.device:
            if not _is_torch(a) or not a.is_cuda or not a.is_contiguous():
                raise ValueError("device-mode handles take contiguous CUDA tensors")
            return C.c_void_p(a.data_ptr())
        if not isinstance(a, np.ndarray) or not a.flags.c_contiguous:
            raise ValueError("host-mode handles take contiguous numpy arrays")
        return a.ctypes.data_as(C.c_void_p)


def lowd_load_graph(n: int, u, v, w=None, flags: int = 0, stream=None) -> Handle:
    """Load an undirected graph; numpy arrays give a host-mode handle, CUDA tensors a
    device-mode one.  ``stream`` is a torch.cuda.Stream (device mode; default: the
    current stream) or None (legacy default stream)."""
    lib = load_library()
    device = _is_torch(u)
    if device:
        import torch
        u = u.to(torch.int32).contiguous(); v = v.to(torch.int32).contiguous()
        if w is not None:
            w = w.to(torch.float32).contiguous()
        st = stream if stream is not None else torch.cuda.current_stream()
        sptr = C.c_void_p(st.cuda_stream)
        pu, pv = C.c_void_p(u.data_ptr()), C.c_void_p(v.data_ptr())
        pw = C.c_void_p(w.data_ptr()) if w is not None else None
        m = int(u.numel())
        keep = (u, v, w)
    else:
        u = np.ascontiguousarray(u, dtype=np.int32); v = np.ascontiguousarray(v, dtype=np.int32)
        if w is not None:
            w = np.ascontiguousarray(w, dtype=np.float32)
        st = stream
        sptr = C.c_void_p(stream.cuda_stream) if stream is not None else None
        pu, pv = u.ctypes.data_as(C.c_void_p), v.ctypes.data_as(C.c_void_p)
        pw = w.ctypes.data_as(C.c_void_p) if w is not None else None
        m = int(u.shape[0])
        keep = (u, v, w)
    if (v.numel() if device else v.shape[0]) != m or (w is not None and (w.numel() if device else w.shape[0]) != m):
        raise ValueError("u, v, w must have the same length")
    out = C.c_void_p()
    s = lib.lowd_load_graph(int(n), m, pu, pv, pw, LOWD_MEM_DEVICE if device else LOWD_MEM_HOST,
                            int(flags), sptr, C.byref(out))
    del keep
    if s != LOWD_OK:
        raise LowdError(s, "lowd_load_graph")
    return Handle(out.value, device, int(n), st)


def lowd_prune(h: Handle):
    """Algorithm 2's pruning; returns (n_kept, m_kept, rounds)."""
    nk, mk, r = C.c_int32(), C.c_int64(), C.c_int32()
    h._check(load_library().lowd_prune(h.ptr, C.byref(nk), C.byref(mk), C.byref(r)), "lowd_prune")
    return nk.value, mk.value, r.value


def lowd_iterate(h: Handle, k: int, check_every: int = 0, rel_tol: float = 0.0,
                 schedule: int = 0, allow_not_converged: bool = True, rederive_every: int = 0,
                 node_versions: bool = False, hub_stars: int = 0) -> dict:
    """k LOWD passes; returns the lowd_stats fields as a dict (plus 'status')."""
    o = lowd_options(int(check_every), float(rel_tol), int(schedule), int(rederive_every),
                     int(bool(node_versions)), int(hub_stars))
    st = lowd_stats()
    s = load_library().lowd_iterate(h.ptr, int(k), C.byref(o), C.byref(st))
    if s != LOWD_OK and not (allow_not_converged and s == LOWD_ERR_NOT_CONVERGED):
        h._check(s, "lowd_iterate")
    d = {f: getattr(st, f) for f, _ in lowd_stats._fields_}
    d["status"] = s
    return d


def lowd_extract(h: Handle, want_loads: bool = True):
    """Algorithm 1's extraction; returns (S* original ids ascending, rho*, loads [n_orig] or None)."""
    S = h.empty(h.n0, np.int32)
    loads = h.empty(h.n0, np.float32) if want_loads else None
    k = C.c_int32()
    rho = C.c_double()
    h._check(load_library().lowd_extract(h.ptr, h.ptr_of(S), C.byref(k), C.byref(rho),
                                         h.ptr_of(loads)), "lowd_extract")
    return S[:k.value], rho.value, (loads[:h.n0] if loads is not None else None)


def lowd_get_ldd(h: Handle, rel_tol: float = 1e-5):
    """Locally-dense decomposition of the current loads: (shell per original node, 0 =
    pruned; lambda per shell; |B_i| per shell)."""
    n = lowd_get_info(h)["n"]
    shell = h.empty(h.n0, np.int32)
    if h.device:
        import torch
        lam = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
        lamp = C.c_void_p(lam.data_ptr())
    else:
        lam = np.empty(max(n, 1), np.float64)
        lamp = lam.ctypes.data_as(C.c_void_p)
    end = h.empty(n, np.int32)
    ns = C.c_int32()
    h._check(load_library().lowd_get_ldd(h.ptr, float(rel_tol), h.ptr_of(shell), lamp, h.ptr_of(end),
                                         C.byref(ns)), "lowd_get_ldd")
    return shell[:h.n0], lam[:ns.value], end[:ns.value]


def lowd_ldd_dks_bound(lam, shell_end, k: int):
    """Corollary 1: (upper bound on the k-subgraph / at-least-k subgraph density, whether
    it is attained, i.e. k = |B_j|), from lowd_get_ldd's lambda and shell_end."""
    lam = np.ascontiguousarray(lam.cpu().numpy() if hasattr(lam, "cpu") else lam, np.float64)
    end = np.ascontiguousarray(shell_end.cpu().numpy() if hasattr(shell_end, "cpu") else shell_end, np.int32)
    b = C.c_double()
    ex = C.c_int32()
    s = load_library().lowd_ldd_dks_bound(int(lam.shape[0]), end.ctypes.data_as(C.c_void_p),
                                          lam.ctypes.data_as(C.c_void_p), int(k), C.byref(b), C.byref(ex))
    if s != LOWD_OK:
        raise LowdError(s, "lowd_ldd_dks_bound")
    return b.value, bool(ex.value)


def lowd_get_info(h: Handle) -> dict:
    info = lowd_info()
    h._check(load_library().lowd_get_info(h.ptr, C.byref(info)), "lowd_get_info")
    return {f: getattr(info, f) for f, _ in lowd_info._fields_}


def lowd_get_graph(h: Handle):
    m = lowd_get_info(h)["m"]
    u, v, w = h.empty(m, np.int32), h.empty(m, np.int32), h.empty(m, np.float32)
    h._check(load_library().lowd_get_graph(h.ptr, h.ptr_of(u), h.ptr_of(v), h.ptr_of(w)), "lowd_get_graph")
    return u[:m], v[:m], w[:m]


def lowd_get_splits(h: Handle):
    m = lowd_get_info(h)["m"]
    s = h.empty(m, np.float32)
    h._check(load_library().lowd_get_splits(h.ptr, h.ptr_of(s)), "lowd_get_splits")
    return s[:m]


def lowd_set_splits(h: Handle, s):
    if h.device:
        import torch
        s = s.to(torch.float32).contiguous()
    else:
        s = np.ascontiguousarray(s, dtype=np.float32)
    h._check(load_library().lowd_set_splits(h.ptr, h.ptr_of(s)), "lowd_set_splits")


def lowd_get_loads(h: Handle):
    n = lowd_get_info(h)["n"]
    l = h.empty(n, np.float32)
    h._check(load_library().lowd_get_loads(h.ptr, h.ptr_of(l)), "lowd_get_loads")
    return l[:n]


def lowd_get_prune_info(h: Handle):
    perm, rr = h.empty(h.n0, np.int32), h.empty(h.n0, np.int32)
    h._check(load_library().lowd_get_prune_info(h.ptr, h.ptr_of(perm), h.ptr_of(rr)), "lowd_get_prune_info")
    return perm[:h.n0], rr[:h.n0]


def lowd_get_edge_order(h: Handle):
    info = lowd_get_info(h)
    perm = h.empty(info["m"], np.int32)
    offs = h.empty(info["classes"] + 1, np.int32)
    c = C.c_int32()
    h._check(load_library().lowd_get_edge_order(h.ptr, h.ptr_of(perm), h.ptr_of(offs), C.byref(c)),
             "lowd_get_edge_order")
    return perm[:info["m"]], offs[:c.value + 1]


def lowd_extract_noalloc(n: int, u, v, w, loads, S=None, stream=None):
    """Allocation-free extraction on CUDA tensors (see include/lowd.h).  Returns
    (status, |S*|, rho*); S (int32 CUDA tensor of >= n entries) receives S* if given."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    k = C.c_int32()
    rho = C.c_double()

    def p(t):
        return None if t is None else C.c_void_p(t.data_ptr())
    s = load_library().lowd_extract_noalloc(int(n), int(u.numel()), p(u), p(v), p(w), p(loads), p(S),
                                            C.byref(k), C.byref(rho), C.c_void_p(st.cuda_stream))
    return s, k.value, rho.value


def lowd_free(h: Handle):
    if h is not None and h.ptr and h.ptr.value:
        load_library().lowd_free(h.ptr)
        h.ptr = C.c_void_p(None)


class Batch:
    """A batch of graphs (the C ``lowd_batch``), host mode: numpy in, numpy out."""

    def __init__(self, ptr, B, n_total):
        self.ptr = C.c_void_p(ptr)
        self.B = B
        self.n_total = n_total

    def __del__(self):
        try:
            lowd_batch_free(self)
        except Exception:
            pass


def lowd_batch_create(node_off, edge_off, u, v, stream=None) -> Batch:
    """Copy a batch: offsets [B+1] (int64) and local-id edges (int32), canonical per graph."""
    no = np.ascontiguousarray(node_off, dtype=np.int64)
    eo = np.ascontiguousarray(edge_off, dtype=np.int64)
    uu = np.ascontiguousarray(u, dtype=np.int32)
    vv = np.ascontiguousarray(v, dtype=np.int32)
    B = no.shape[0] - 1
    out = C.c_void_p()
    sptr = C.c_void_p(stream.cuda_stream) if stream is not None else None
    s = load_library().lowd_batch_create(B, no.ctypes.data_as(C.c_void_p), eo.ctypes.data_as(C.c_void_p),
                                         uu.ctypes.data_as(C.c_void_p), vv.ctypes.data_as(C.c_void_p),
                                         LOWD_MEM_HOST, sptr, C.byref(out))
    if s != LOWD_OK:
        raise LowdError(s, "lowd_batch_create")
    return Batch(out.value, B, int(no[-1]))


def lowd_batch_run(b: Batch, passes: int, ctas_per_sm: int = 0, threads: int = 0, order: int = 0):
    o = lowd_batch_options(int(passes), int(ctas_per_sm), int(threads), int(order))
    s = load_library().lowd_batch_run(b.ptr, C.byref(o))
    if s != LOWD_OK:
        raise LowdError(s, "lowd_batch_run", load_library().lowd_batch_last_error(b.ptr).decode())


def lowd_batch_autotune(b: Batch, passes: int, sample: int = 0) -> dict:
    o = lowd_batch_options()
    s = load_library().lowd_batch_autotune(b.ptr, int(passes), int(sample), C.byref(o))
    if s != LOWD_OK:
        raise LowdError(s, "lowd_batch_autotune", load_library().lowd_batch_last_error(b.ptr).decode())
    return {f: getattr(o, f) for f, _ in lowd_batch_options._fields_}


def lowd_batch_results(b: Batch) -> dict:
    rho = np.empty(b.B, np.float64)
    size, nc, mc, rr, st = (np.empty(b.B, np.int32) for _ in range(5))
    ins = np.empty(max(b.n_total, 1), np.uint8)
    P = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    s = load_library().lowd_batch_results(b.ptr, P(rho), P(size), P(ins), P(nc), P(mc), P(rr), P(st))
    if s != LOWD_OK:
        raise LowdError(s, "lowd_batch_results")
    return dict(rho=rho, S_size=size, in_S=ins[:b.n_total], n_core=nc, m_core=mc, rounds=rr, status=st)


def lowd_batch_loads(b: Batch) -> np.ndarray:
    """FP32 loads after the last run's passes, all graphs' nodes by local id."""
    out = np.empty(max(b.n_total, 1), np.float32)
    s = load_library().lowd_batch_loads(b.ptr, out.ctypes.data_as(C.c_void_p))
    if s != LOWD_OK:
        raise LowdError(s, "lowd_batch_loads", load_library().lowd_batch_last_error(b.ptr).decode())
    return out[:b.n_total]


def lowd_batch_core(b: Batch) -> np.ndarray:
    """1 for nodes that survived Algorithm 2 in the last run, all graphs by local id."""
    out = np.empty(max(b.n_total, 1), np.uint8)
    s = load_library().lowd_batch_core(b.ptr, out.ctypes.data_as(C.c_void_p))
    if s != LOWD_OK:
        raise LowdError(s, "lowd_batch_core", load_library().lowd_batch_last_error(b.ptr).decode())
    return out[:b.n_total]


def lowd_batch_free(b: Batch):
    if b is not None and b.ptr and b.ptr.value:
        load_library().lowd_batch_free(b.ptr)
        b.ptr = C.c_void_p(None)


# ----------------------------------------------------------------------------- warm-start network

class Mpnn:
    """The warm-start network (the C ``lowd_mpnn``); host-mode arrays (numpy)."""

    def __init__(self, ptr: int):
        self.ptr = C.c_void_p(ptr)
        self.n = 0
        self.m = 0

    def __del__(self):
        try:
            lowd_mpnn_free(self)
        except Exception:
            pass

    def _check(self, status: int, where: str):
        if status != LOWD_OK:
            detail = load_library().lowd_mpnn_last_error(self.ptr).decode() if self.ptr else ""
            raise LowdError(status, where, detail)


def _f32p(a):
    return a.ctypes.data_as(C.c_void_p)


def lowd_mpnn_param_count() -> int:
    return int(load_library().lowd_mpnn_param_count())


def lowd_mpnn_create(stream=None) -> Mpnn:
    out = C.c_void_p()
    sptr = C.c_void_p(stream.cuda_stream) if stream is not None else None
    s = load_library().lowd_mpnn_create(sptr, C.byref(out))
    if s != LOWD_OK:
        raise LowdError(s, "lowd_mpnn_create")
    return Mpnn(out.value)


def lowd_mpnn_set_params(net: Mpnn, params):
    p = np.ascontiguousarray(params, np.float32)
    if p.shape[0] != lowd_mpnn_param_count():
        raise ValueError("wrong parameter count")
    net._check(load_library().lowd_mpnn_set_params(net.ptr, _f32p(p), LOWD_MEM_HOST), "lowd_mpnn_set_params")


def lowd_mpnn_get_params(net: Mpnn) -> np.ndarray:
    p = np.empty(lowd_mpnn_param_count(), np.float32)
    net._check(load_library().lowd_mpnn_get_params(net.ptr, _f32p(p), LOWD_MEM_HOST), "lowd_mpnn_get_params")
    return p


def lowd_mpnn_bind(net: Mpnn, n: int, lo, hi, w=None, target=None):
    lo = np.ascontiguousarray(lo, np.int32)
    hi = np.ascontiguousarray(hi, np.int32)
    m = int(lo.shape[0])
    if hi.shape[0] != m:
        raise ValueError("lo, hi must have the same length")
    wa = None if w is None else np.ascontiguousarray(w, np.float32)
    ta = None if target is None else np.ascontiguousarray(target, np.float32)
    s = load_library().lowd_mpnn_bind(net.ptr, int(n), m, _f32p(lo), _f32p(hi),
                                      None if wa is None else _f32p(wa), None if ta is None else _f32p(ta),
                                      LOWD_MEM_HOST)
    net._check(s, "lowd_mpnn_bind")
    net.n, net.m = int(n), m


def lowd_mpnn_set_features(net: Mpnn, x):
    """Replace the bound graph's input features by x [n, 3]."""
    xa = np.ascontiguousarray(x, np.float32).reshape(-1)
    if xa.shape[0] != 3 * net.n:
        raise ValueError("features must be [n, 3]")
    net._check(load_library().lowd_mpnn_set_features(net.ptr, _f32p(xa), LOWD_MEM_HOST), "lowd_mpnn_set_features")


def lowd_mpnn_forward(net: Mpnn, with_loss: bool = True):
    loss = C.c_double()
    net._check(load_library().lowd_mpnn_forward(net.ptr, C.byref(loss) if with_loss else None), "lowd_mpnn_forward")
    return loss.value if with_loss else None


def lowd_mpnn_backward(net: Mpnn):
    net._check(load_library().lowd_mpnn_backward(net.ptr), "lowd_mpnn_backward")


def lowd_mpnn_adam(net: Mpnn, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    net._check(load_library().lowd_mpnn_adam(net.ptr, float(lr), float(beta1), float(beta2), float(eps)),
               "lowd_mpnn_adam")


def lowd_mpnn_read(net: Mpnn, what: int) -> np.ndarray:
    size = {LOWD_MPNN_SIGMA: net.m, LOWD_MPNN_LOADS: net.n, LOWD_MPNN_PHI: net.n,
            LOWD_MPNN_FEATURES: 3 * net.n, LOWD_MPNN_GRAD: lowd_mpnn_param_count()}[what]
    out = np.empty(max(size, 1), np.float32)
    net._check(load_library().lowd_mpnn_read(net.ptr, int(what), _f32p(out), LOWD_MEM_HOST), "lowd_mpnn_read")
    return out[:size]


def lowd_warm_start(h: Handle, net: Mpnn):
    """The network's splits on the handle's current graph become the LOWD state."""
    h._check(load_library().lowd_warm_start(h.ptr, net.ptr), "lowd_warm_start")


def lowd_mpnn_free(net: Mpnn):
    if net is not None and net.ptr and net.ptr.value:
        load_library().lowd_mpnn_free(net.ptr)
        net.ptr = C.c_void_p(None)
