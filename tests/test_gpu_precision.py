"""Precision of the FP32 sweep against the FP64 oracle on the weighted R-MAT recipe
(scale 16, edge factor 8, lognormal(0,1) weights on the 2^-20 grid, 128-node block with
weights x3).

The oracle replays, in FP64, the colour-class order it computes itself (checked to be
the GPU's classes in the GPU's order); the test bounds and prints the
relative load error max|l_gpu - l_64| / max l_64, the relative error of sum(l^2), and the
density gap, after 1, 10, 100 and 400 passes.  Pruning and the pruned graph are bit-exact;
the density reported for the extracted set is its exact density.
"""
import numpy as np
import pytest

import synth
from _oracle_side import assert_same_schedule

pytestmark = pytest.mark.gpu

# Same-order iterates: the pair-load sweep moves weight without rounding the loads, so the
# FP32 and FP64 runs differ only by the FP32 splits' rounding (<= 2^-24 w_e per update),
# which accumulates like a random walk over passes: 1e-6 of the largest load at up to 100
# passes, scaled by sqrt(T/100) beyond (measured 6e-8 at 1 pass, 3.4e-7 at 400).  The sum of
# squares is an FP64 sum of FP64 loads re-derived from those splits: 1e-9 relative (measured
# 6e-12 after 1 pass, 4e-15 after 400).
def load_tol(T):
    return 1e-6 * max(1.0, (T / 100.0) ** 0.5)


SUMSQ_TOL = 1e-9


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
    return torch, pkg, oracle, synth.workload("rmat16w")


def test_weighted_rmat_precision_against_fp64(setup, capsys):
    torch, pkg, orc, g = setup
    h = pkg.lowd_load_graph(g.n, torch.from_numpy(g.u).cuda(), torch.from_numpy(g.v).cuda(),
                            torch.from_numpy(g.w).cuda())
    nk, mk, rounds = pkg.lowd_prune(h)
    wu, scale = orc.weight_units(g.m, g.w)
    pr = orc.prune(g.n, g.u, g.v, wu, True)
    assert np.array_equal(pkg.lowd_get_prune_info(h)[1].cpu().numpy(), pr["removal_round"])
    keep = pr["removal_round"] < 0
    nh, uh, vh, wh, idmap = orc.compact(g.n, g.u, g.v, g.w, keep)
    gu, gv, gw = (x.cpu().numpy() for x in pkg.lowd_get_graph(h))
    assert np.array_equal(gu, uh) and np.array_equal(gv, vh) and np.array_equal(gw, wh)
    pkg.lowd_iterate(h, 1)
    assert pkg.lowd_get_info(h)["sweep_kernel"] in (1, 5)   # the staged pair-load sweep, weighted
    order = assert_same_schedule(orc, nh, uh, vh, *(x.cpu().numpy() for x in pkg.lowd_get_edge_order(h)))
    o = orc.LowdState(nh, uh, vh, wh.astype(np.float64))
    o.iterate(1, order=order)
    done = 1
    report = []
    whu, _ = orc.weight_units(uh.shape[0], wh)
    for T in (1, 10, 100, 400):
        if T > done:
            st = pkg.lowd_iterate(h, T - done)
            o.iterate(T - done, order=order)
            done = T
        else:
            st = pkg.lowd_iterate(h, 0)
        lg = pkg.lowd_get_loads(h).cpu().numpy().astype(np.float64)
        s64 = o.stats()
        lerr = np.max(np.abs(lg - o.l)) / o.l.max()
        qerr = abs(st["sum_load_sq"] - s64[1]) / s64[1]
        # the extracted set is valid: rho is its exact density W(S)/|S| (integer units)
        S, rho, _ = pkg.lowd_extract(h, want_loads=False)
        inS = np.zeros(g.n, bool)
        inS[S.cpu().numpy()] = True
        Sh = inS[idmap]
        WS = int(whu[Sh[uh] & Sh[vh]].sum())
        assert rho == WS / scale / int(Sh.sum())
        report.append((T, lerr, qerr, rho, st["max_load"]))
    with capsys.disabled():
        print(f"\n[precision] weighted rmat16w core n={nh} m={uh.shape[0]} (prune rounds {rounds})")
        for T, lerr, qerr, rho, D in report:
            print(f"[precision] passes={T:4d} load err {lerr:.2e}  sum-sq err {qerr:.2e}  "
                  f"rho(S)={rho:.6f}  D={D:.6f}  gap={(D - rho) / rho:.2e}")
    for T, lerr, qerr, rho, D in report:
        assert lerr <= load_tol(T), (T, lerr)
        assert qerr <= SUMSQ_TOL, (T, qerr)
    pkg.lowd_free(h)
