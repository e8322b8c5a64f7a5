"""Every LOWD pass kernel against the FP64 oracle, with the kernel that ran pinned.

lowd_iterate picks its pass kernel from the graph's schedule: the staged one-CTA sweep with
pair loads (kernel 1) with one, two or four edges per consumer thread by class size, the
register-ring sweep (kernel 2) when the staged layout's store ordering does not hold, the
simple sweep (kernel 3) for very few classes, and the streamed sweep (kernel 4) for graphs
whose loads do not fit shared memory; kernel 5 is kernel 1 with per-node versions in place of
the barrier after every class (classes of up to 992 edges).  Each case below is sized to
reach one variant,
unit and weighted, and checks lowd_get_info's record of it; the oracle replays its own
circle-colouring order (checked to be the GPU's classes) in FP64, and the loads must agree
within the bar of that kernel's arithmetic (Algorithm 1; pair loads 1e-6, single FP32 loads
1e-4 of the largest load, times sqrt(T/100) beyond 100 passes).
"""
import numpy as np
import pytest

import synth
from _oracle_side import assert_same_schedule
from test_gpu_parity import load_tol

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


# (graph, passes, node versions asked for, expected kernel, expected edges per thread
# (kernels 1 and 5))
CASES = {
    "simple_k6": (lambda: synth.small_family("clique", 6), 12, False, 3, 0),
    "ring_gnp60": (lambda: synth.erdos_renyi(60, 0.5, seed=61), 20, False, 2, 0),
    "versions_gnp60": (lambda: synth.erdos_renyi(60, 0.5, seed=61), 20, True, 5, 1),
    "versions_e1": (lambda: synth.erdos_renyi(1500, 0.5, seed=62), 6, True, 5, 1),
    "versions_sparse": (lambda: synth.chung_lu(4000, 30000, 2.3, seed=66, block_size=50, block_p=0.5),
                        30, True, 5, 1),
    "staged_e1": (lambda: synth.erdos_renyi(1500, 0.5, seed=62), 6, False, 1, 1),
    "staged_e2": (lambda: synth.erdos_renyi(2600, 0.95, seed=63), 4, False, 1, 2),
    "staged_e4": (lambda: synth.erdos_renyi(4400, 0.95, seed=64), 3, True, 1, 4),
}


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("case", list(CASES))
def test_pass_kernel_variant_against_oracle(pkg, orc, case, weighted):
    import torch
    make, T, versions, kern, E = CASES[case]
    g = make()
    w = None
    if weighted:
        w = synth.quantise_weights(np.random.default_rng(len(case)).lognormal(0, 1, g.m))
    h = pkg.lowd_load_graph(g.n, torch.from_numpy(g.u).cuda(), torch.from_numpy(g.v).cuda(),
                            None if w is None else torch.from_numpy(w).cuda())
    pkg.lowd_iterate(h, T, node_versions=versions)
    info = pkg.lowd_get_info(h)
    assert info["sweep_kernel"] == kern, info
    if kern in (1, 5):
        assert info["sweep_edges_per_thread"] == E, info
    perm, offs = (x.cpu().numpy() for x in pkg.lowd_get_edge_order(h))
    order = assert_same_schedule(orc, g.n, g.u, g.v, perm, offs)
    o = orc.LowdState(g.n, g.u, g.v, None if w is None else w.astype(np.float64))
    o.iterate(T, order=order)
    lg = pkg.lowd_get_loads(h).cpu().numpy().astype(np.float64)
    err = np.max(np.abs(lg - o.l)) / max(1.0, o.l.max())
    assert err <= load_tol(T, kern), (case, weighted, err)
    # conservation and the box constraint on the GPU's splits
    s = pkg.lowd_get_splits(h).cpu().numpy().astype(np.float64)
    wt = np.ones(g.m) if w is None else w.astype(np.float64)
    assert np.all(s >= 0) and np.all(s <= wt)
    assert abs(lg.sum() - wt.sum()) <= 1e-6 * wt.sum()
    pkg.lowd_free(h)
