"""Weighted graphs at full size: the R-MAT scale-24 graph with lognormal(0, 1) weights on the
2^-20 grid and a planted 512-node block with weights x3 (16.8 M nodes, 134.3 M edges).

Against the oracle: every node's removal round in Algorithm 2's weighted pruning (exact
integer degrees, Sec. III-D) and the pruned core's edges and weights, bit-exact; two
same-order passes on the core within the pair-load bar (1e-6 of the largest load) and the
sum of squared loads within 1e-9; converged, S* equal to the maximal densest set B_1 of the
exact min cut, rho* within 1e-9 relative and every load within 1e-4 relative of the exact
decomposition; and one pass of Algorithm 1 over the whole unpruned graph (streamed
schedule) against the oracle's FP64 replay of the level order.
"""
import numpy as np
import pytest

import synth
from _oracle_side import assert_same_schedule
from test_gpu_parity import load_tol, per_node_converged_ok

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
    g = synth.workload("rmat24w")
    w64 = g.w.astype(np.float64)
    wu, scale = oracle.weight_units(g.m, w64)
    pr = oracle.prune(g.n, g.u, g.v, wu, True)
    keep = pr["removal_round"] < 0
    core = oracle.compact(g.n, g.u, g.v, g.w, keep)
    return torch, pkg, oracle, g, pr, core, scale


def _load(torch, pkg, g):
    return pkg.lowd_load_graph(g.n, torch.from_numpy(g.u).cuda(), torch.from_numpy(g.v).cuda(),
                               torch.from_numpy(g.w).cuda())


def test_rmat24w_pruning_and_core_bit_exact(setup):
    torch, pkg, orc, g, pr, core, scale = setup
    h = _load(torch, pkg, g)
    nk, mk, rounds = pkg.lowd_prune(h)
    assert rounds == pr["rounds"]
    _, rr = pkg.lowd_get_prune_info(h)
    assert np.array_equal(rr.cpu().numpy(), pr["removal_round"])
    nh, uh, vh, wh, _ = core
    assert (nk, mk) == (nh, uh.shape[0])
    gu, gv, gw = (x.cpu().numpy() for x in pkg.lowd_get_graph(h))
    assert np.array_equal(gu, uh) and np.array_equal(gv, vh) and np.array_equal(gw, wh)
    # two passes in the oracle's own class order, FP64 replay
    st1 = pkg.lowd_iterate(h, 1)
    assert pkg.lowd_get_info(h)["sweep_kernel"] in (1, 5)
    order = assert_same_schedule(orc, nh, uh, vh, *(x.cpu().numpy() for x in pkg.lowd_get_edge_order(h)))
    st2 = pkg.lowd_iterate(h, 1)
    o = orc.LowdState(nh, uh, vh, wh.astype(np.float64))
    o.iterate(2, order=order)
    lg = pkg.lowd_get_loads(h).cpu().numpy().astype(np.float64)
    assert np.max(np.abs(lg - o.l)) <= load_tol(2, 1) * o.l.max()
    s64 = o.stats()
    assert abs(st2["sum_load_sq"] - s64[1]) <= 1e-9 * s64[1]
    assert st2["sum_load_sq"] <= st1["sum_load_sq"] * (1 + 1e-10)
    pkg.lowd_free(h)


def test_rmat24w_converged_densest_subgraph_and_loads(setup):
    torch, pkg, orc, g, pr, core, scale = setup
    nh, uh, vh, wh, idmap = core
    whu, _ = orc.weight_units(uh.shape[0], wh.astype(np.float64))
    rho_star, B1 = orc.densest_flow(nh, uh, vh, whu)          # on H: rho*(H) = rho*(G) (Thm. 3)
    lstar, _, _ = orc.ldd_loads(nh, uh, vh, whu, scale)
    h = _load(torch, pkg, g)
    pkg.lowd_prune(h)
    st = pkg.lowd_iterate(h, 4000, check_every=50, rel_tol=1e-6)
    assert st["converged"] == 1
    pkg.lowd_iterate(h, 1000)     # a certified 1e-6 gap bounds the top load; let the rest settle
    S, rho, _ = pkg.lowd_extract(h, want_loads=False)
    assert abs(rho - float(rho_star) / scale) <= 1e-9 * float(rho_star) / scale
    assert np.array_equal(S.cpu().numpy(), idmap[np.nonzero(B1)[0]])
    lg = pkg.lowd_get_loads(h).cpu().numpy().astype(np.float64)
    ok = per_node_converged_ok(lg, lstar)
    assert np.all(ok), (int((~ok).sum()), float(np.max(np.abs(lg - lstar) / lstar)))
    pkg.lowd_free(h)


def test_rmat24w_unpruned_streamed_pass(setup):
    torch, pkg, orc, g, pr, core, scale = setup
    h = _load(torch, pkg, g)
    pkg.lowd_iterate(h, 1)
    info = pkg.lowd_get_info(h)
    assert info["schedule"] == 2 and info["sweep_kernel"] == 4
    perm, offs = (x.cpu().numpy() for x in pkg.lowd_get_edge_order(h))
    order = assert_same_schedule(orc, g.n, g.u, g.v, perm, offs, level=True)
    o = orc.LowdState(g.n, g.u, g.v, g.w.astype(np.float64))
    o.iterate(1, order=order)
    lg = pkg.lowd_get_loads(h).cpu().numpy().astype(np.float64)
    assert np.max(np.abs(lg - o.l)) <= load_tol(1, 4) * o.l.max()
    st = pkg.lowd_iterate(h, 0)
    tot = float(g.w.astype(np.float64).sum())
    assert abs(st["sum_load"] - tot) <= 1e-9 * tot
    pkg.lowd_free(h)
