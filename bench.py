"""Benchmark of the LOWD hot path on one GB300 (or N replicas under torchrun).

One step = the whole path on the R-MAT scale-22 graph (4,194,304 nodes, 67,125,322
unique undirected edges incl. a planted 256-node block at p=0.5, unit weights), inputs
resident in HBM: lowd_load_graph (validation + canonical check), lowd_prune (degrees,
counting sort, Algorithm 2 rounds, compaction to the dense core H), lowd_iterate(T)
(colouring + T LOWD passes over H) and lowd_extract (S*, rho*).  The metric is LOWD
edge-updates per second: m_H * T per step over the step's device time.

The same JSON line carries the other workloads as extra keys:
  unpruned   Algorithm 1 over the whole unpruned graph (rmat22, rmat24w) with the streamed
             schedule: edge-updates/s of the passes, the colouring time, the roofline
  rmat24w    the weighted scale-24 R-MAT graph through prune -> passes -> extract
  batch      4,096 independent Chung-Lu graphs in one persistent launch, CUDA-event timed,
             with a sample of graphs checked against the oracle's exact solution
  cpu_baseline  the oracle's passes on all host cores (colour classes split over threads)

  python bench.py [--gpus N] [--steps K] [--warmup W] [--iters T] [--impl lowd|reference]
                  [--legs main,unpruned,rmat24w,batch]

--impl reference times the CPU oracle (plain C, FP64) on this host on the same workload:
each step is a bounded sample of LOWD passes over the oracle's own pruned H.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "rmat22"
METRIC = "LOWD edge-updates/s"
UNIT = "edge-updates/s"
BYTES_PER_UPDATE = 16   # u, v int32 + split read + split write per edge-update (loads on chip)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _sweep_hash():
    """Hash of the staged sweep kernel's source: its layout, the kernel and its launcher."""
    with open(os.path.join(ROOT, "paper_2307_15969_gb300", "csrc", "sweep.cu")) as f:
        s = f.read()
    parts = []
    for a, b in (("struct TmaLayout {", "// The same staging as k_sweep_tma"),
                 ("cudaError_t launch_sweep_tma(", "\n}\n")):   # the launcher, to its closing brace
        i = s.find(a)
        j = s.find(b, i) if i >= 0 else -1
        if i < 0 or j < i:
            return "missing"
        parts.append(s[i:j])
    return hashlib.sha256("".join(parts).encode()).hexdigest()[:16]


def _sweep_record():
    """The committed ncu record of the staged sweep (DRAM bytes per pass, warp instructions
    per class), if it was taken on the current sweep kernel source."""
    p = os.path.join(ROOT, "profiles", "k_sweep_tma_rmat22_dram.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("sweep_cu_sha256_16") != _sweep_hash():
        return None
    return d


def _traffic_per_pass():
    d = _sweep_record()
    return float(d["dram_bytes_per_pass"]) if d else None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # raw samples go to a temporary file; the JSON line carries their summary
        self.path = os.path.join(os.environ.get("LOWD_BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for ln in f:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1])); mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_throughput(local_seconds: float, local_updates: float, ws: int, device=None):
    """Whole-job throughput of independent replicas (one per rank, no data exchange): the
    updates of every rank over the slowest rank's time.  Returns (value, max seconds)."""
    if ws <= 1:
        return local_updates / local_seconds, local_seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_seconds], dtype=torch.float64, device=device)
    u = torch.tensor([local_updates], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item())


def host_cores() -> int:
    """Host cores this process may use (nproc)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline_sample(g, T_target_s: float = 12.0, threads: int = 1):
    """The oracle as it stands on this host: its own pruning of G, then LOWD passes on H in
    the circle-colouring class order for roughly T_target_s seconds, on `threads` host
    threads (classes split over the threads, a barrier per class; one thread runs the plain
    sequential loop).  Returns (updates/s, dict)."""
    import oracle
    oracle.build()
    wu, _ = oracle.weight_units(g.m, g.w)
    pr = oracle.prune(g.n, g.u, g.v, wu, g.w is not None)
    keep = pr["removal_round"] < 0
    nh, uh, vh, wh, _ = oracle.compact(g.n, g.u, g.v, g.w, keep)
    st = oracle.LowdState(nh, uh, vh, None if wh is None else np.asarray(wh, np.float64))
    order, offs, _ = oracle.circle_order(nh, uh, vh)

    def passes(T):
        if threads > 1:
            st.iterate_threads(T, order, offs, threads)
        else:
            st.iterate(T, order=order)

    t0 = time.perf_counter()
    passes(1)
    one = time.perf_counter() - t0
    T = max(1, int(T_target_s / max(one, 1e-6)))
    t0 = time.perf_counter()
    passes(T)
    dt = time.perf_counter() - t0
    rate = uh.shape[0] * T / dt
    return rate, dict(n_H=nh, m_H=int(uh.shape[0]), passes=T, seconds=dt, threads=threads,
                      passes_fn=passes)


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import synth
    g = synth.workload(args.workload)
    cores = host_cores()
    # each step: a bounded sample of the workload (LOWD passes over the oracle's own H)
    rate0, info = cpu_baseline_sample(g, T_target_s=2.0, threads=cores)
    T = info["passes"]
    m_H = info["m_H"]
    for _ in range(args.warmup):
        info["passes_fn"](T)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        info["passes_fn"](T)
    dt = time.perf_counter() - t0
    value = m_H * T * args.steps / dt
    sample = (f"{args.steps} steps x {T} oracle LOWD passes over the oracle's pruned core H "
              f"(n={info['n_H']}, m={m_H}) of the {args.workload} graph; {cores} host threads, "
              f"colour classes split over the threads")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": g.n, "m": g.m, "n_H": info["n_H"],
                       "m_H": m_H, "passes_per_step": T},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- inputs made in the background

def _gen_batch(args_):
    import synth as _s
    lo, hi = args_
    out = []
    for gi in range(lo, hi):
        g = _s.batch_graph(gi)
        out.append((g.n, g.u, g.v))
    return out


def _gen_workload(name):
    import synth as _s
    g = _s.workload(name)
    return g.n, g.u, g.v, g.w


class Background:
    """Input generation in a spawn process pool, started before any GPU call: the batched
    workload's graphs and the weighted scale-24 R-MAT graph are made while the GPU works."""

    def __init__(self, batch_count: int, want_rmat24w: bool):
        import multiprocessing as mp
        procs = max(1, min(16, host_cores()))
        self.pool = mp.get_context("spawn").Pool(procs)
        self.r24 = self.pool.apply_async(_gen_workload, ("rmat24w",)) if want_rmat24w else None
        self.batch = None
        if batch_count > 0:
            step = max(1, (batch_count + procs * 4 - 1) // (procs * 4))
            chunks = [(lo, min(batch_count, lo + step)) for lo in range(0, batch_count, step)]
            self.batch = self.pool.map_async(_gen_batch, chunks)

    def rmat24w(self):
        import synth
        n, u, v, w = self.r24.get()
        return synth.Graph(n=n, u=u, v=v, w=w, name="rmat24w")

    def batch_inputs(self):
        gs = [x for part in self.batch.get() for x in part]
        node_off = np.concatenate([[0], np.cumsum([g[0] for g in gs])]).astype(np.int64)
        edge_off = np.concatenate([[0], np.cumsum([g[1].shape[0] for g in gs])]).astype(np.int64)
        u = np.concatenate([g[1] for g in gs]).astype(np.int32)
        v = np.concatenate([g[2] for g in gs]).astype(np.int32)
        return gs, node_off, edge_off, u, v

    def close(self):
        self.pool.close()
        self.pool.join()


# ----------------------------------------------------------------------------- GPU legs

def _events(torch, n=2):
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def _to_dev(torch, g, dev):
    du = torch.from_numpy(g.u).to(dev)
    dv = torch.from_numpy(g.v).to(dev)
    dw = torch.from_numpy(g.w).to(dev) if g.w is not None else None
    return du, dv, dw


def sweep_launch_seconds(torch, pkg, stream, h, T):
    """Device time of T passes alone: events around lowd_iterate(T) minus lowd_iterate(0)
    (the re-derivation of the loads both calls make), best of 3."""
    durs = {}
    for k in (T, 0):
        ev = []
        for _ in range(3):
            a, b = _events(torch)
            a.record(stream); pkg.lowd_iterate(h, k); b.record(stream); b.synchronize()
            ev.append(a.elapsed_time(b) / 1e3)
        durs[k] = min(ev)
    return max(durs[T] - durs[0], 1e-9)


def leg_unpruned(torch, pkg, stream, g, du, dv, dw, T, peak, peak_kind):
    """Algorithm 1 over the whole unpruned graph with the streamed schedule: the colouring
    (level order) is timed on its own, then T passes."""
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=du.device)
    flush.fill_(1.0)
    h = pkg.lowd_load_graph(g.n, du, dv, dw, stream=stream)
    a, b = _events(torch)
    a.record(stream)
    pkg.lowd_iterate(h, 0, schedule=2)     # schedule, streams, descriptors, initial loads
    b.record(stream)
    b.synchronize()
    prep_ms = a.elapsed_time(b)
    st0 = pkg.lowd_iterate(h, 0)
    sec = sweep_launch_seconds(torch, pkg, stream, h, T)
    st1 = pkg.lowd_iterate(h, 0)
    info = pkg.lowd_get_info(h)
    bpu = BYTES_PER_UPDATE + (4 if g.w is not None else 0)
    achieved = bpu * g.m * T / sec / 1e9
    C = info["classes"]
    out = {"workload": f"{g.name} unpruned", "n": g.n, "m": g.m, "max_degree": info["max_degree"],
           "classes": C, "passes": T, "value": g.m * T / sec, "unit": UNIT,
           "pass_ms": sec / T * 1e3, "ns_per_class": sec / T / max(C, 1) * 1e9,
           "colouring_ms": prep_ms, "sweep_kernel": info["sweep_kernel"],
           "sum_load_sq_before": st0["sum_load_sq"], "sum_load_sq_after": st1["sum_load_sq"],
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": None, "kernel": "k_sweep_stream",
                        "peak_kind": peak_kind, "bytes_per_update": bpu,
                        "chain": "Delta = classes per pass; a pass is at least one class-to-class "
                                 "dependency step per class"}}
    pkg.lowd_free(h)
    # the same graph with hub-star block updates (automatic threshold): fewer dependent steps
    # per pass (plain classes + star steps), each pass also a larger descent of sum l^2
    h = pkg.lowd_load_graph(g.n, du, dv, dw, stream=stream)
    a.record(stream)
    pkg.lowd_iterate(h, 0, schedule=2, hub_stars=1)
    b.record(stream)
    b.synchronize()
    prep_s = a.elapsed_time(b)
    sec_s = sweep_launch_seconds(torch, pkg, stream, h, T)
    st2 = pkg.lowd_iterate(h, 0)
    info = pkg.lowd_get_info(h)
    out["hub_stars"] = {"star_threshold": info["star_threshold"], "star_steps": info["star_steps"],
                        "stars": info["stars"], "star_edges": info["star_edges"],
                        "plain_classes": info["classes"] - info["star_steps"],
                        "dependent_steps_per_pass": info["classes"], "pass_ms": sec_s / T * 1e3,
                        "prepare_ms": prep_s, "sum_load_sq_after": st2["sum_load_sq"],
                        "passes_timed": T}
    pkg.lowd_free(h)
    del flush
    return out


def leg_weighted(torch, pkg, stream, g, T):
    """The weighted scale-24 R-MAT graph (lognormal weights on the 2^-20 grid, planted block
    with weights x3): load -> prune -> T passes -> extract, device time, inputs in HBM."""
    dev = torch.device("cuda", torch.cuda.current_device())
    du, dv, dw = _to_dev(torch, g, dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    times = []
    res = {}
    for it in range(3):
        flush.fill_(1.0)
        e = _events(torch, 5)
        e[0].record(stream)
        h = pkg.lowd_load_graph(g.n, du, dv, dw, stream=stream)
        e[1].record(stream)
        nk, mk, rounds = pkg.lowd_prune(h)
        e[2].record(stream)
        st = pkg.lowd_iterate(h, T, check_every=T, rel_tol=0.0)
        e[3].record(stream)
        S, rho, _ = pkg.lowd_extract(h, want_loads=False)
        e[4].record(stream)
        e[4].synchronize()
        info = pkg.lowd_get_info(h)
        pkg.lowd_free(h)
        times.append(e[0].elapsed_time(e[4]) / 1e3)
        res = dict(n_H=nk, m_H=mk, rounds=rounds, rho=rho, S=int(S.shape[0]), D=st["max_load"],
                   gap=(st["max_load"] - st["rho_best"]) / st["rho_best"] if st["rho_best"] > 0 else None,
                   classes=info["classes"], sweep_kernel=info["sweep_kernel"],
                   stages_ms={k: e[i].elapsed_time(e[i + 1]) for i, k in
                              enumerate(("load", "prune", "iterate", "extract"))})
    step = min(times)
    out = {"workload": "rmat24w", "n": g.n, "m": g.m, "passes": T, "value": res["m_H"] * T / step,
           "unit": UNIT, "step_ms": step * 1e3, "dtype": "f32 splits and pair loads; f64 checks",
           **res}
    peak, peak_kind = _peaks()
    out["unpruned"] = leg_unpruned(torch, pkg, stream, g, du, dv, dw, 5, peak, peak_kind)
    del du, dv, dw, flush
    return out


def leg_batch(torch, pkg, bg, T, check_count: int = 48):
    """Config 4: every graph through prune -> colour -> T passes -> extraction in one
    persistent launch replayed from a captured CUDA graph, timed with CUDA events on the
    batch's stream; a spread sample of graphs is checked against the oracle's exact
    solution (S* = the maximal densest set, rho* within 1e-9)."""
    import oracle
    gs, node_off, edge_off, u, v = bg.batch_inputs()
    stream = torch.cuda.Stream()
    b = pkg.lowd_batch_create(node_off, edge_off, u, v, stream=stream)
    t0 = time.perf_counter()
    tuned = pkg.lowd_batch_autotune(b, passes=T, sample=0)
    tune_s = time.perf_counter() - t0
    for _ in range(3):
        pkg.lowd_batch_run(b, passes=T)
    times = []
    for _ in range(5):
        a, e = _events(torch)
        a.record(stream)
        pkg.lowd_batch_run(b, passes=T)
        e.record(stream)
        e.synchronize()
        times.append(a.elapsed_time(e) / 1e3)
    res = pkg.lowd_batch_results(b)
    pkg.lowd_batch_free(b)
    ok = res["status"] == 0
    upd = int(res["m_core"][ok].astype(np.int64).sum()) * T
    step = statistics.median(times)
    # oracle check of a spread sample
    idx = np.unique(np.linspace(0, len(gs) - 1, check_count).astype(int))
    good = 0
    for i in idx:
        n_i, u_i, v_i = gs[i]
        rho, B1 = oracle.densest_flow(n_i, u_i, v_i, np.ones(u_i.shape[0], np.int64))
        mask = res["in_S"][node_off[i]:node_off[i + 1]].astype(bool)
        if ok[i] and abs(res["rho"][i] - float(rho)) <= 1e-9 * float(rho) and np.array_equal(mask, B1):
            good += 1
    peak, peak_kind = _peaks()
    achieved = BYTES_PER_UPDATE * upd / step / 1e9
    return {"workload": f"batch{len(gs)}", "graphs": len(gs), "nodes": int(node_off[-1]),
            "edges": int(edge_off[-1]), "core_nodes": int(res["n_core"][ok].sum()),
            "core_edges": int(res["m_core"][ok].sum()), "passes": T, "graphs_ok": int(ok.sum()),
            "value": upd / step, "unit": "core edge-updates/s", "graphs_per_s": len(gs) / step,
            "step_ms": step * 1e3, "timing": "CUDA events on the batch's stream around the graph replay",
            "schedule": tuned, "autotune_s": tune_s,
            "oracle_checked": {"graphs": int(idx.shape[0]), "matching": good,
                               "check": "S* = maximal densest set and rho* within 1e-9 of the exact min cut"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "kernel": "k_batch_lowd", "peak_kind": peak_kind,
                         "bytes_per_update": BYTES_PER_UPDATE,
                         "note": "whole launch (prune, colour, passes, extraction) over core updates"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--iters", type=int, default=200, help="LOWD passes per step")
    ap.add_argument("--impl", default="lowd", choices=["lowd", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--legs", default="main,unpruned,rmat24w,batch",
                    help="comma list of legs: main, unpruned, rmat24w, batch")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rho-max-passes", type=int, default=2000,
                    help="pass cap of the time-to-rho leg")
    ap.add_argument("--no-warm-start", action="store_true", help="skip the warm-start time-to-rho leg")
    ap.add_argument("--warm-params", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                          "paper_2307_15969_gb300", "warmstart_params.npy"))
    ap.add_argument("--batch-graphs", type=int, default=4096, help="graphs of the batched workload")
    ap.add_argument("--batch-iters", type=int, default=100, help="LOWD passes per graph of the batch leg")
    ap.add_argument("--unpruned-iters", type=int, default=10, help="passes of the unpruned streamed leg")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    legs = set(x.strip() for x in args.legs.split(",") if x.strip())

    ws, rank, local = _dist()
    bg = None
    if ws == 1 and rank == 0 and ({"rmat24w", "batch"} & legs):
        # start the input pool before the first GPU call
        bg = Background(args.batch_graphs if "batch" in legs else 0, "rmat24w" in legs)

    import torch
    import synth
    import paper_2307_15969_gb300 as pkg

    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    pkg.load_library()

    g = synth.workload(args.workload)
    du, dv, dw = _to_dev(torch, g, dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    T = args.iters

    def step(stats):
        h = pkg.lowd_load_graph(g.n, du, dv, dw, stream=stream)
        nk, mk, rounds = pkg.lowd_prune(h)
        st = pkg.lowd_iterate(h, T)
        S, rho, _ = pkg.lowd_extract(h, want_loads=False)
        info_ = pkg.lowd_get_info(h)
        stats.update(n_H=nk, m_H=mk, rounds=rounds, rho=rho, S=int(S.shape[0]),
                     classes=info_["classes"], sweep_kernel=info_["sweep_kernel"],
                     edges_per_thread=info_["sweep_edges_per_thread"])
        pkg.lowd_free(h)

    peak, peak_kind = _peaks()
    extra = {}
    with torch.cuda.stream(stream):
        info = {}
        for _ in range(max(args.warmup, 0)):
            step(info)
        stream.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks = Clocks(dev.index)
        clocks.start()
        times = []
        launches0 = pkg.lowd_launch_count()
        for _ in range(args.steps):
            flush.fill_(1.0)                       # evict L2 between timed steps
            e0, e1 = _events(torch)
            e0.record(stream)
            step(info)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        launches = pkg.lowd_launch_count() - launches0
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        ck = clocks.stop()

        m_H = info["m_H"]
        value, total = replica_throughput(sum(times), float(m_H * T * args.steps), ws, dev)

        # the dominant kernel: the one-CTA LOWD sweep on the core
        h = pkg.lowd_load_graph(g.n, du, dv, dw, stream=stream)
        pkg.lowd_prune(h)
        pkg.lowd_iterate(h, 1)
        sweep_s = sweep_launch_seconds(torch, pkg, stream, h, T)
        pkg.lowd_free(h)

        # per-stage device time of one step (events between the calls)
        stages = {}
        evs = _events(torch, 5)
        evs[0].record(stream)
        h = pkg.lowd_load_graph(g.n, du, dv, dw, stream=stream)
        evs[1].record(stream)
        pkg.lowd_prune(h)
        evs[2].record(stream)
        pkg.lowd_iterate(h, T)
        evs[3].record(stream)
        pkg.lowd_extract(h, want_loads=False)
        evs[4].record(stream)
        evs[4].synchronize()
        for i, nm in enumerate(("load", "prune", "iterate", "extract")):
            stages[nm] = evs[i].elapsed_time(evs[i + 1])
        pkg.lowd_free(h)

        # time to rho: passes until the certified relative gap (D - rho(S))/rho(S) <= 1e-6,
        # D = max load of the FP64 loads re-derived from the splits (an upper bound on
        # rho*), checked every `check` passes
        check = 10
        h = pkg.lowd_load_graph(g.n, du, dv, dw, stream=stream)
        t_a, t_b = _events(torch)
        t_a.record(stream)
        pkg.lowd_prune(h)
        st_rho = pkg.lowd_iterate(h, args.rho_max_passes, check_every=check, rel_tol=1e-6)
        t_b.record(stream)
        t_b.synchronize()
        time_to_rho = {"rel_gap": 1e-6, "converged": bool(st_rho["converged"]),
                       "passes": int(st_rho["iters_done"]), "ms": t_a.elapsed_time(t_b),
                       "check_every": check, "rho": st_rho["rho_best"], "D": st_rho["max_load"],
                       "includes": "prune + colouring + passes + FP64 checks with extraction"}
        pkg.lowd_free(h)

        # the same with the learned warm start: the network's splits replace the equal split
        # (features + three layers on the pruned core, inside the timed region)
        time_to_rho_warm = None
        if not args.no_warm_start and os.path.exists(args.warm_params):
            from paper_2307_15969_gb300 import warmstart
            net = pkg.lowd_mpnn_create()
            pkg.lowd_mpnn_set_params(net, warmstart.load_params(args.warm_params))
            h = pkg.lowd_load_graph(g.n, du, dv, dw, stream=stream)
            t_a.record(stream)
            pkg.lowd_prune(h)
            t_w = torch.cuda.Event(enable_timing=True)
            pkg.lowd_warm_start(h, net)
            t_w.record(stream)
            st_w = pkg.lowd_iterate(h, args.rho_max_passes, check_every=check, rel_tol=1e-6)
            t_b.record(stream)
            t_b.synchronize()
            time_to_rho_warm = {"rel_gap": 1e-6, "converged": bool(st_w["converged"]),
                                "passes": int(st_w["iters_done"]), "ms": t_a.elapsed_time(t_b),
                                "warm_start_ms": t_a.elapsed_time(t_w),
                                "check_every": check, "rho": st_w["rho_best"], "D": st_w["max_load"],
                                "params": os.path.basename(args.warm_params),
                                "includes": "prune + network inference + colouring + passes + FP64 checks"}
            pkg.lowd_free(h)
            pkg.lowd_mpnn_free(net)

        # the same with hub-star block updates (automatic threshold): per pass Algorithm 1 over
        # the plain edges, then every star's exact Sigma l^2 minimiser, from the equal split
        h = pkg.lowd_load_graph(g.n, du, dv, dw, stream=stream)
        t_a.record(stream)
        pkg.lowd_prune(h)
        st_s = pkg.lowd_iterate(h, args.rho_max_passes, check_every=check, rel_tol=1e-6, hub_stars=1)
        t_b.record(stream)
        t_b.synchronize()
        info_s = pkg.lowd_get_info(h)
        time_to_rho_stars = {"rel_gap": 1e-6, "converged": bool(st_s["converged"]),
                             "passes": int(st_s["iters_done"]), "ms": t_a.elapsed_time(t_b),
                             "check_every": check, "rho": st_s["rho_best"], "D": st_s["max_load"],
                             "star_threshold": info_s["star_threshold"], "star_steps": info_s["star_steps"],
                             "stars": info_s["stars"], "star_edges": info_s["star_edges"],
                             "plain_classes": info_s["classes"] - info_s["star_steps"],
                             "includes": "prune + star structure + colouring + passes + FP64 checks"}
        pkg.lowd_free(h)

        # end to end through the C ABI with pinned host buffers (copies inside the timing)
        hu = torch.from_numpy(g.u).pin_memory().numpy()
        hv = torch.from_numpy(g.v).pin_memory().numpy()
        hw = torch.from_numpy(g.w).pin_memory().numpy() if g.w is not None else None
        e2e_times = []
        for it in range(2):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = pkg.lowd_load_graph(g.n, hu, hv, hw, stream=stream)
            pkg.lowd_prune(h)
            pkg.lowd_iterate(h, T)
            S, rho, loads = pkg.lowd_extract(h, want_loads=True)
            pkg.lowd_free(h)
            e2e_times.append(time.perf_counter() - t0)
        e2e_s = min(e2e_times)
        h2d = int(g.u.nbytes + g.v.nbytes + (g.w.nbytes if g.w is not None else 0))
        d2h = int(4 * S.shape[0] + 4 * g.n + 8 * 4)

        if rank == 0 and ws == 1:
            if "unpruned" in legs:
                extra["unpruned"] = leg_unpruned(torch, pkg, stream, g, du, dv, dw, args.unpruned_iters,
                                                 peak, peak_kind)
            if "rmat24w" in legs:
                del flush
                g24 = bg.rmat24w()
                extra["rmat24w"] = leg_weighted(torch, pkg, stream, g24, 100)
                del g24
                torch.cuda.empty_cache()
            if "batch" in legs:
                extra["batch"] = leg_batch(torch, pkg, bg, args.batch_iters)
    if bg is not None:
        bg.close()

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    achieved = BYTES_PER_UPDATE * m_H * T / sweep_s / 1e9
    tpp = _traffic_per_pass()
    rec = _sweep_record()
    mhz = ck.get("sm_mhz") if isinstance(ck, dict) else None
    issue_floor = (rec["warp_instructions_per_class"] / 4.0 / (mhz * 1e6) * 1e9
                   if rec and rec.get("warp_instructions_per_class") and mhz else None)
    C = info["classes"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "n": g.n, "m": g.m, "n_H": info["n_H"], "m_H": m_H,
                   "prune_rounds": info["rounds"], "classes": C, "passes_per_step": T,
                   "rho_star_found": info["rho"], "S_size": info["S"],
                   "parallelism": "replicas" if ws > 1 else "single-gpu",
                   "l2": "flushed between timed steps (256 MB write); G's edge arrays (537 MB) exceed L2"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": (tpp * T if tpp is not None else None),
                     "kernel": "k_sweep_tma", "peak_kind": peak_kind,
                     "launch_ms": sweep_s * 1e3, "bytes_per_update": BYTES_PER_UPDATE,
                     "sweep_kernel": info["sweep_kernel"], "edges_per_thread": info["edges_per_thread"],
                     "chain": {"classes_per_pass": C, "ns_per_class": sweep_s / T / max(C, 1) * 1e9,
                               "issue_floor_ns_per_class": issue_floor,
                               "note": "each class waits for the previous one (Delta(H) >= n_H - 3 "
                                       "classes on this near-clique core): the pass is bound by the "
                                       "per-class chain on one SM, not by HBM; the issue floor is "
                                       "the class's warp instructions (ncu) over 4 schedulers at "
                                       "the sampled SM clock"}},
        "e2e": {"value": m_H * T / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3},
        "stages_ms": stages,
        "time_to_rho": time_to_rho,
        "time_to_rho_warm_start": time_to_rho_warm,
        "time_to_rho_hub_stars": time_to_rho_stars,
        "gpu_launches": int(launches),
        "gpu_launches_per_step": int(launches // max(args.steps, 1)),
        "clocks": ck,
    }
    line.update(extra)
    if ws == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        rate, cinfo = cpu_baseline_sample(g, threads=cores)
        rate1, cinfo1 = cpu_baseline_sample(g, threads=1)
        line["cpu_baseline"] = {
            "value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cinfo['passes']} oracle LOWD passes (FP64, plain C) over the oracle's own pruned "
                      f"core H (n={cinfo['n_H']}, m={cinfo['m_H']}) of {args.workload} in circle-colouring "
                      f"class order, classes split over {cores} host threads with a barrier per class, "
                      f"{cinfo['seconds']:.1f} s",
            "one_thread": {"value": rate1, "cores": 1, "passes": cinfo1["passes"],
                           "seconds": cinfo1["seconds"]}}
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
