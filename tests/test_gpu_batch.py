"""Batched LOWD (many graphs, one persistent launch) against the oracle, graph by graph.

Per graph: the pruning rounds and the pruned core's size (bit-exact against Algorithm 2 in
the oracle); after 1 and 9 passes the loads against the FP64 oracle replaying the
circle-colouring classes of its own pruned core; after 300 passes the densest set and density against the exact min-cut
solution (S* equal to the maximal densest set B_1, rho* within 1e-9 relative).  Also: the
autotuned and the captured-graph replays give the same results, and non-canonical input is
refused.
"""
import numpy as np
import pytest

import synth
from _oracle_side import oracle_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_15969_gb300 import build
    build.build()
    import paper_2307_15969_gb300 as pkg
    import oracle
    oracle.build()
    graphs = synth.batch(48, seed_base=5000, n_hi=3000)
    node_off = np.concatenate([[0], np.cumsum([g.n for g in graphs])]).astype(np.int64)
    edge_off = np.concatenate([[0], np.cumsum([g.m for g in graphs])]).astype(np.int64)
    u = np.concatenate([g.u for g in graphs]).astype(np.int32)
    v = np.concatenate([g.v for g in graphs]).astype(np.int32)
    ref = []
    for g in graphs:
        wu = np.ones(g.m, np.int64)
        pr = oracle.prune(g.n, g.u, g.v, wu, False)
        keep = pr["removal_round"] < 0
        rho, B1 = oracle.densest_flow(g.n, g.u, g.v, wu)
        ref.append(dict(rounds=pr["rounds"], n_core=int(keep.sum()),
                        m_core=int((keep[g.u] & keep[g.v]).sum()), rho=float(rho), B1=B1, keep=keep))
    return pkg, graphs, node_off, edge_off, u, v, ref


def _check(res, graphs, node_off, ref):
    for i, (g, r) in enumerate(zip(graphs, ref)):
        assert res["status"][i] == 0, i
        assert res["rounds"][i] == r["rounds"], i
        assert (res["n_core"][i], res["m_core"][i]) == (r["n_core"], r["m_core"]), i
        assert abs(res["rho"][i] - r["rho"]) <= 1e-9 * r["rho"], i
        mask = res["in_S"][node_off[i]:node_off[i + 1]].astype(bool)
        assert np.array_equal(mask, r["B1"]), i
        assert res["S_size"][i] == int(r["B1"].sum()), i


def test_batch_matches_oracle(setup):
    pkg, graphs, node_off, edge_off, u, v, ref = setup
    b = pkg.lowd_batch_create(node_off, edge_off, u, v)
    pkg.lowd_batch_run(b, passes=300)
    _check(pkg.lowd_batch_results(b), graphs, node_off, ref)
    pkg.lowd_batch_run(b, passes=300)          # replay of the captured launch
    _check(pkg.lowd_batch_results(b), graphs, node_off, ref)
    for per, thr, order in ((1, 256, 1), (2, 512, 2), (1, 1024, 2)):
        pkg.lowd_batch_run(b, passes=300, ctas_per_sm=per, threads=thr, order=order)
        _check(pkg.lowd_batch_results(b), graphs, node_off, ref)
    best = pkg.lowd_batch_autotune(b, passes=50, sample=16)
    assert best["ctas_per_sm"] in (1, 2) and best["threads"] in (256, 512, 1024)
    pkg.lowd_batch_run(b, passes=300)
    _check(pkg.lowd_batch_results(b), graphs, node_off, ref)
    pkg.lowd_batch_free(b)


@pytest.mark.parametrize("T", [1, 9])
def test_batch_same_order_loads(setup, T):
    """Loads after T passes: the oracle prunes, compacts and orders the core itself."""
    import oracle as orc
    pkg, graphs, node_off, edge_off, u, v, ref = setup
    b = pkg.lowd_batch_create(node_off, edge_off, u, v)
    for thr in (256, 1024):
        pkg.lowd_batch_run(b, passes=T, threads=thr)
        res = pkg.lowd_batch_results(b)
        lg = pkg.lowd_batch_loads(b)
        core = pkg.lowd_batch_core(b)
        for i, g in enumerate(graphs):
            assert res["status"][i] == 0, i
            nh, uh, vh, _, idmap = oracle_graph(orc, g, True)
            order, _, _ = orc.circle_order(nh, uh, vh)
            o = orc.LowdState(nh, uh, vh)
            o.iterate(T, order=order)
            li = lg[node_off[i]:node_off[i + 1]].astype(np.float64)
            assert np.all(li[~ref[i]["keep"]] == 0), i
            assert np.array_equal(core[node_off[i]:node_off[i + 1]].astype(bool), ref[i]["keep"]), i
            err = np.max(np.abs(li[idmap] - o.l)) if nh else 0.0
            assert err <= 1e-4 * max(1.0, o.l.max() if nh else 1.0), (i, T, thr, err)
    pkg.lowd_batch_free(b)


def test_batch_rejects_non_canonical_input(setup):
    pkg, graphs, node_off, edge_off, u, v, ref = setup
    u2, v2 = u.copy(), v.copy()
    u2[5], v2[5] = v2[5], u2[5]      # u > v
    with pytest.raises(pkg.LowdError):
        pkg.lowd_batch_create(node_off, edge_off, u2, v2)
    u3, v3 = u.copy(), v.copy()
    u3[6], v3[6] = u3[5], v3[5]      # a repeated pair
    with pytest.raises(pkg.LowdError):
        pkg.lowd_batch_create(node_off, edge_off, u3, v3)


@pytest.fixture(scope="module")
def top_of_range():
    """Graphs of the batched recipe at the top of its size range (n in [18,000, 20,000]:
    ~0.5 M edges, pruned cores of ~1,000 nodes and ~240 k edges, the largest the workload
    makes), interleaved with small ones so that uneven graphs share the launch."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    oracle.build()
    big = synth.batch(8, seed_base=7000, n_lo=18000, n_hi=20000)
    small = synth.batch(4, seed_base=7100, n_hi=600)
    graphs = [x for pair in zip(big[:4], small) for x in pair] + big[4:]
    node_off = np.concatenate([[0], np.cumsum([g.n for g in graphs])]).astype(np.int64)
    edge_off = np.concatenate([[0], np.cumsum([g.m for g in graphs])]).astype(np.int64)
    u = np.concatenate([g.u for g in graphs]).astype(np.int32)
    v = np.concatenate([g.v for g in graphs]).astype(np.int32)
    ref = []
    for g in graphs:
        wu = np.ones(g.m, np.int64)
        pr = oracle.prune(g.n, g.u, g.v, wu, False)
        keep = pr["removal_round"] < 0
        rho, B1 = oracle.densest_flow(g.n, g.u, g.v, wu)
        ref.append(dict(rounds=pr["rounds"], n_core=int(keep.sum()),
                        m_core=int((keep[g.u] & keep[g.v]).sum()), rho=float(rho), B1=B1, keep=keep))
    return graphs, node_off, edge_off, u, v, ref


def test_batch_top_of_size_range(setup, top_of_range):
    import oracle as orc
    pkg = setup[0]
    graphs, node_off, edge_off, u, v, ref = top_of_range
    assert max(g.n for g in graphs) >= 19000
    b = pkg.lowd_batch_create(node_off, edge_off, u, v)
    for per, thr in ((1, 1024), (2, 512)):
        pkg.lowd_batch_run(b, passes=400, ctas_per_sm=per, threads=thr)
        _check(pkg.lowd_batch_results(b), graphs, node_off, ref)
    # same-order loads after 2 passes (the oracle prunes, compacts and orders each core)
    pkg.lowd_batch_run(b, passes=2, ctas_per_sm=2, threads=512)
    res = pkg.lowd_batch_results(b)
    lg = pkg.lowd_batch_loads(b)
    for i, g in enumerate(graphs):
        assert res["status"][i] == 0, i
        nh, uh, vh, _, idmap = oracle_graph(orc, g, True)
        order, _, _ = orc.circle_order(nh, uh, vh)
        o = orc.LowdState(nh, uh, vh)
        o.iterate(2, order=order)
        li = lg[node_off[i]:node_off[i + 1]].astype(np.float64)
        err = np.max(np.abs(li[idmap] - o.l)) if nh else 0.0
        assert err <= 1e-4 * max(1.0, o.l.max() if nh else 1.0), (i, err)
    pkg.lowd_batch_free(b)
