"""Training and use of the learned warm start (the network behind ``lowd_mpnn_*`` and
``lowd_warm_start`` in include/lowd.h).

The training data are converged LOWD states the method itself produces: seeded synthetic
graphs of the batched workload's shape (Chung-Lu, n uniform in [100, 20000], average degree
in [4, 32], exponent 2.1-2.8, a planted block of 5% of n at p = 0.5) are pruned and run for
many passes by the batched kernel; each graph's pruned core with its loads is one training
example (the loads converge to the unique optimum of Properties 1-2, whatever the start).
Examples are packed into minibatches as disjoint unions (the network is local, so a union
is a batch) and trained with Adam on the GPU through the library's own forward and backward
kernels.  Every step runs in the library; this module only prepares arrays and loops.

Usage:
    python -m paper_2307_15969_gb300.warmstart --graphs 20000 --passes 3000 --epochs 6 \\
        --out paper_2307_15969_gb300/warmstart_params.npy
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

from . import lowd as L

PARAMS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "warmstart_params.npy")
HIDDEN, LAYERS, N_IN = 64, 3, 3


def load_params(path: str = PARAMS_PATH) -> np.ndarray:
    """The trained parameters shipped with the package (FP32, lowd_mpnn_param_count())."""
    p = np.load(path).astype(np.float32)
    if p.shape[0] != L.lowd_mpnn_param_count():
        raise ValueError(f"{path}: expected {L.lowd_mpnn_param_count()} parameters, found {p.shape[0]}")
    return p


def init_params(seed: int) -> np.ndarray:
    """He-uniform layer weights, zero biases, a small readout: a start near the equal split."""
    rng = np.random.default_rng(seed)
    parts = [rng.uniform(-1, 1, N_IN * HIDDEN) * np.sqrt(6.0 / N_IN), np.zeros(HIDDEN)]
    for _ in range(LAYERS):
        parts += [rng.uniform(-1, 1, HIDDEN * 2 * HIDDEN) * np.sqrt(6.0 / (2 * HIDDEN)), np.zeros(HIDDEN)]
    parts.append(rng.uniform(-1, 1, HIDDEN) * 0.01)
    return np.concatenate(parts).astype(np.float32)


def _one_graph(args):
    import synth
    g, seed_base = args
    gr = synth.batch_graph(g, seed_base=seed_base)
    return gr.n, gr.u, gr.v


def make_graphs(count: int, seed_base: int, workers: int = 0):
    """``count`` graphs of the batched workload's shape (graph g drawn from seed
    seed_base + g), generated by a spawn pool (start it before the first GPU call)."""
    jobs = [(g, seed_base) for g in range(count)]
    workers = workers or min(16, os.cpu_count() or 1)
    if workers <= 1:
        return [_one_graph(j) for j in jobs]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_one_graph, jobs, chunksize=8)


def converged_cores(graphs, passes: int, chunk: int = 2048, log=print):
    """Prune and iterate every graph with the batched kernel; return one example per graph
    with a non-empty core: dict(n, lo, hi, t) (core relabelled by ascending id, t = loads)."""
    out = []
    for c0 in range(0, len(graphs), chunk):
        part = graphs[c0:c0 + chunk]
        node_off = np.concatenate([[0], np.cumsum([g[0] for g in part])]).astype(np.int64)
        edge_off = np.concatenate([[0], np.cumsum([g[1].shape[0] for g in part])]).astype(np.int64)
        u = np.concatenate([g[1] for g in part]).astype(np.int32)
        v = np.concatenate([g[2] for g in part]).astype(np.int32)
        t0 = time.perf_counter()
        b = L.lowd_batch_create(node_off, edge_off, u, v)
        L.lowd_batch_run(b, passes=passes)
        res = L.lowd_batch_results(b)
        loads = L.lowd_batch_loads(b)
        core = L.lowd_batch_core(b).astype(bool)
        L.lowd_batch_free(b)
        for i, (n, gu, gv) in enumerate(part):
            if res["status"][i] != 0 or res["n_core"][i] < 2:
                continue
            mk = core[node_off[i]:node_off[i + 1]]
            newid = np.cumsum(mk) - 1
            ke = mk[gu] & mk[gv]
            out.append(dict(n=int(mk.sum()), lo=newid[gu[ke]].astype(np.int32), hi=newid[gv[ke]].astype(np.int32),
                            t=loads[node_off[i]:node_off[i + 1]][mk].astype(np.float32)))
        log(f"[warmstart] converged {len(part)} graphs ({passes} passes) in {time.perf_counter() - t0:.1f} s")
    return out


def union(examples):
    """Disjoint union of examples: (n, lo, hi, t)."""
    offs = np.concatenate([[0], np.cumsum([e["n"] for e in examples])])
    lo = np.concatenate([e["lo"] + o for e, o in zip(examples, offs)]).astype(np.int32)
    hi = np.concatenate([e["hi"] + o for e, o in zip(examples, offs)]).astype(np.int32)
    t = np.concatenate([e["t"] for e in examples]).astype(np.float32)
    return int(offs[-1]), lo, hi, t


def evaluate(net, examples, per_batch: int) -> float:
    """Mean minibatch loss of the current parameters (forward only)."""
    losses = []
    for i in range(0, len(examples), per_batch):
        n, lo, hi, t = union(examples[i:i + per_batch])
        L.lowd_mpnn_bind(net, n, lo, hi, None, t)
        losses.append(L.lowd_mpnn_forward(net))
    return float(np.mean(losses)) if losses else float("nan")


def train(examples, epochs: int = 6, per_batch: int = 32, lr: float = 2e-3, lr_min: float = 1e-4,
          seed: int = 0, val_frac: float = 0.05, log=print):
    """Adam on minibatches of ``per_batch`` examples, cosine learning-rate decay; the
    parameters with the best validation loss are returned with a training record."""
    rng = np.random.default_rng(seed)
    idx = rng.permutation(len(examples))
    nval = max(1, int(round(val_frac * len(examples))))
    val = [examples[i] for i in idx[:nval]]
    tr = [examples[i] for i in idx[nval:]]
    net = L.lowd_mpnn_create()
    L.lowd_mpnn_set_params(net, np.zeros(L.lowd_mpnn_param_count(), np.float32))
    base = evaluate(net, val, per_batch)                 # all splits equal: the paper's start
    p0 = init_params(seed)
    L.lowd_mpnn_set_params(net, p0)
    best, best_p = evaluate(net, val, per_batch), p0
    record = dict(equal_split_val_loss=base, init_val_loss=best, epochs=[])
    log(f"[warmstart] {len(tr)} training / {len(val)} validation cores; equal-split loss {base:.4f}, init {best:.4f}")
    steps = epochs * ((len(tr) + per_batch - 1) // per_batch)
    k = 0
    for ep in range(epochs):
        t0 = time.perf_counter()
        order = rng.permutation(len(tr))
        tl = []
        for i in range(0, len(tr), per_batch):
            n, lo, hi, t = union([tr[j] for j in order[i:i + per_batch]])
            L.lowd_mpnn_bind(net, n, lo, hi, None, t)
            tl.append(L.lowd_mpnn_forward(net))
            L.lowd_mpnn_backward(net)
            a = lr_min + 0.5 * (lr - lr_min) * (1 + np.cos(np.pi * k / max(1, steps)))
            L.lowd_mpnn_adam(net, float(a))
            k += 1
        cur = L.lowd_mpnn_get_params(net)
        vl = evaluate(net, val, per_batch)        # rebinds graphs only: parameters and Adam state stay
        if vl < best:
            best, best_p = vl, cur.copy()
        record["epochs"].append(dict(epoch=ep, train_loss=float(np.mean(tl)), val_loss=vl,
                                     seconds=time.perf_counter() - t0))
        log(f"[warmstart] epoch {ep}: train {np.mean(tl):.4f} val {vl:.4f} ({time.perf_counter() - t0:.1f} s)")
    record["best_val_loss"] = best
    L.lowd_mpnn_free(net)
    return best_p, record


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--graphs", type=int, default=20000)
    ap.add_argument("--seed-base", type=int, default=500000, help="graph g uses seed seed_base + g")
    ap.add_argument("--passes", type=int, default=3000)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--per-batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--out", default=PARAMS_PATH)
    ap.add_argument("--record", default=None, help="write the training record (JSON) here")
    a = ap.parse_args(argv)
    t0 = time.perf_counter()
    graphs = make_graphs(a.graphs, a.seed_base)           # spawn pool before any GPU call
    print(f"[warmstart] generated {len(graphs)} graphs in {time.perf_counter() - t0:.1f} s", flush=True)
    L.load_library()
    ex = converged_cores(graphs, a.passes)
    del graphs
    p, rec = train(ex, epochs=a.epochs, per_batch=a.per_batch, lr=a.lr)
    np.save(a.out, p)
    rec.update(graphs=a.graphs, seed_base=a.seed_base, passes=a.passes, per_batch=a.per_batch, lr=a.lr,
               cores=len(ex), seconds=time.perf_counter() - t0)
    if a.record:
        with open(a.record, "w") as f:
            json.dump(rec, f, indent=1)
    print(json.dumps({k: v for k, v in rec.items() if k != "epochs"}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
