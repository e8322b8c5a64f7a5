"""Hub-star passes on the GPU against the oracle's FP64 replay.

A hub-star pass runs Algorithm 1 over the plain edges (both ends hubs, or neither) in the
level order of their subgraph, then the star steps: every star of a step gets the exact
minimiser of the sum of squared loads over its splits (the local optimality of Sec. III-C
over a block of edges).  Checked here: the threshold (given, or the automatic rule computed
by the oracle from its definition), the step and star counts, the GPU's plain classes equal
to the oracle's level order of the plain subgraph and its star blocks equal to the oracle's
steps as edge sets; then T same-order passes against the oracle's FP64 replay within the
pair-load bar, conservation and the box constraint; and convergence to the exact densest
subgraph and decomposition.
"""
import numpy as np
import pytest

import synth
from _oracle_side import assert_same_schedule, oracle_graph
from test_gpu_parity import load_tol, per_node_converged_ok

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_15969_gb300 import build
    build.build()
    import paper_2307_15969_gb300 as p
    p.load_library()
    return p


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


# (graph, passes, hub_stars option, schedule asked for (0 = automatic: the shared-memory
# schedule for all of these))
CASES = {
    "cl300_auto": (lambda: synth.chung_lu(300, 1500, 2.1, seed=3, block_size=12, block_p=0.7), 30, 1, 0),
    "cl300_auto_s2": (lambda: synth.chung_lu(300, 1500, 2.1, seed=3, block_size=12, block_p=0.7), 30, 1, 2),
    "planted_tau8": (lambda: synth.planted_background(200, 3.0, 20, 0.7, seed=6), 30, 8, 0),
    "planted_tau8_s2": (lambda: synth.planted_background(200, 3.0, 20, 0.7, seed=6), 30, 8, 2),
    "star_all_star": (lambda: synth.small_family("star", 40), 5, 1, 0),
    "star_all_star_s2": (lambda: synth.small_family("star", 40), 5, 1, 2),
    "cl20k_auto": (lambda: synth.chung_lu(20000, 200000, 2.1, seed=5, block_size=60, block_p=0.5), 12, 1, 0),
    "cl20k_auto_s2": (lambda: synth.chung_lu(20000, 200000, 2.1, seed=5, block_size=60, block_p=0.5), 12, 1, 2),
    "cl20k_tau16": (lambda: synth.chung_lu(20000, 200000, 2.1, seed=5, block_size=60, block_p=0.5), 6, 16, 0),
    "dense_stars": (lambda: synth.chung_lu(6000, 600000, 2.0, seed=8, block_size=60, block_p=0.5), 4, 1, 0),
    "clique_no_hubs": (lambda: synth.small_family("clique", 12), 10, 1, 0),
}


def _load(torch, pkg, n, u, v, w):
    return pkg.lowd_load_graph(n, torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(),
                               None if w is None else torch.from_numpy(w.astype(np.float32)).cuda())


def _check_structure(orc, info, n, u, v, perm, offs, tau):
    """The GPU's blocks against the oracle's: returns (plain order as edge ids, steps)."""
    m = u.shape[0]
    plain, steps = orc.hub_star_structure(n, u, v, tau)
    mp = plain.shape[0]
    nstars = sum(len(s) for s in steps)
    assert info["star_threshold"] == (tau if mp < m else 0), info
    assert info["star_steps"] == len(steps) and info["stars"] == nstars, info
    assert info["star_edges"] == m - mp, info
    C = info["classes"]
    Cp = C - len(steps)
    assert offs.shape[0] == C + 1 and offs[Cp] == mp and offs[-1] == m
    if mp:
        inv = np.full(m, -1, np.int64)
        inv[plain] = np.arange(mp)
        sub = inv[perm[:mp]]
        assert np.all(sub >= 0)
        order = assert_same_schedule(orc, n, u[plain], v[plain], sub, offs[:Cp + 1],
                                     level=info["schedule"] == 2)
        plain_order = plain[order]
    else:
        plain_order = plain
    for k, st in enumerate(steps):
        blk = np.sort(perm[offs[Cp + k]:offs[Cp + k + 1]])
        want = np.sort(np.concatenate([np.asarray(e) for e in st.values()]))
        assert np.array_equal(blk, want), k
    return plain_order, steps


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("case", list(CASES))
def test_hub_star_passes_against_oracle(pkg, orc, case, weighted):
    import torch
    make, T, opt, sched = CASES[case]
    g = make()
    w0 = None
    if weighted:
        w0 = synth.quantise_weights(np.random.default_rng(len(case)).lognormal(0, 1, g.m)).astype(np.float64)
    n, u, v, w, _ = oracle_graph(orc, synth_graph(g, w0), False)
    h = _load(torch, pkg, n, u, v, w)
    pkg.lowd_iterate(h, T, hub_stars=opt, schedule=sched)
    info = pkg.lowd_get_info(h)
    assert info["schedule"] == (sched or 1), info
    if sched == 2:
        assert info["sweep_kernel"] == 4, info
    tau = opt if opt >= 2 else orc.auto_hub_threshold(n, u, v, schedule=info["schedule"])
    perm, offs = (x.cpu().numpy() for x in pkg.lowd_get_edge_order(h))
    plain_order, steps = _check_structure(orc, info, n, u, v, perm, offs, tau)
    o = orc.LowdState(n, u, v, w)
    o.iterate_hub_star(T, plain_order, steps)
    lg = pkg.lowd_get_loads(h).cpu().numpy().astype(np.float64)
    err = np.max(np.abs(lg - o.l)) / max(1.0, o.l.max())
    assert err <= load_tol(T, info["sweep_kernel"] or 1), (case, weighted, err)
    s = pkg.lowd_get_splits(h).cpu().numpy().astype(np.float64)
    wt = np.ones(u.shape[0]) if w is None else w
    assert np.all(s >= 0) and np.all(s <= wt)
    assert abs(lg.sum() - wt.sum()) <= 1e-6 * wt.sum()
    pkg.lowd_free(h)


def synth_graph(g, w):
    """g with weights w (None keeps it unweighted)."""
    import dataclasses
    return g if w is None else dataclasses.replace(g, w=w.astype(np.float32))


@pytest.mark.parametrize("weighted", [False, True])
def test_hub_star_passes_converge_to_the_densest_subgraph(pkg, orc, weighted):
    import torch
    # weighted: a smaller graph (the oracle's exact min cut on 2^-20 weight units is slow)
    g = (synth.chung_lu(6000, 60000, 2.1, seed=7, block_size=60, block_p=0.6) if weighted
         else synth.chung_lu(20000, 200000, 2.1, seed=7, block_size=80, block_p=0.6))
    w0 = None
    if weighted:
        w0 = synth.quantise_weights(np.random.default_rng(11).lognormal(0, 1, g.m)).astype(np.float64)
    n, u, v, w, _ = oracle_graph(orc, synth_graph(g, w0), False)
    wu, scale = orc.weight_units(u.shape[0], w)
    rho_star, B1 = orc.densest_flow(n, u, v, wu)
    lstar, _, _ = orc.ldd_loads(n, u, v, wu, scale)
    h = _load(torch, pkg, n, u, v, w)
    st = pkg.lowd_iterate(h, 6000, check_every=50, rel_tol=1e-6, hub_stars=1)
    assert st["converged"] == 1
    assert pkg.lowd_get_info(h)["star_edges"] > 0
    pkg.lowd_iterate(h, 2000)
    S, rho, _ = pkg.lowd_extract(h, want_loads=False)
    assert abs(rho - float(rho_star) / scale) <= 1e-9 * float(rho_star) / scale
    assert np.array_equal(S.cpu().numpy(), np.nonzero(B1)[0])
    lg = pkg.lowd_get_loads(h).cpu().numpy().astype(np.float64)
    ok = per_node_converged_ok(lg, lstar)
    assert np.all(ok), (int((~ok).sum()), float(np.max(np.abs(lg - lstar) / lstar)))
    pkg.lowd_free(h)


def test_negative_hub_stars_is_rejected(pkg):
    import torch
    g = synth.small_family("star", 10)
    h = _load(torch, pkg, g.n, g.u, g.v, None)
    with pytest.raises(Exception):
        pkg.lowd_iterate(h, 1, hub_stars=-1)
    pkg.lowd_free(h)
