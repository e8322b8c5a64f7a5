"""Locally-dense decomposition export (lowd_get_ldd) against the exact decomposition.

On graphs whose exact shell loads are separated by more than the grouping tolerance, after
enough passes for the loads to converge (Theorem 2), every node's shell equals the one from
the oracle's min-cut decomposition (Sec. II, Definition of LDD) and each lambda_i equals the
exact shell density (Property 2) to double precision; Corollary 1's DkS/DalkS bounds read
off the export equal the oracle's.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

REL_TOL = 1e-3


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
    return torch, pkg, oracle


def _graphs():
    gs = [synth.planted_background(600, 4.0, 24, 0.6, seed=s) for s in range(3)]
    gs += [synth.chung_lu(400, 1600, 2.3, seed=s, block_size=16, block_p=0.6) for s in range(3)]
    gs += [synth.small_family("two_cliques", 30), synth.small_family("gnp0.1", 60, seed=2)]
    return gs


def test_ldd_export_matches_exact_decomposition(setup):
    torch, pkg, orc = setup
    tested = 0
    for g in _graphs():
        wu, scale = orc.weight_units(g.m, g.w)
        shell, lam = orc.ldd(g.n, g.u, g.v, wu)
        lf = np.array([float(x) / scale for x in lam])
        gaps = (lf[:-1] - lf[1:]) / lf[:-1] if lf.shape[0] > 1 else np.array([1.0])
        if gaps.min() < 4 * REL_TOL:
            continue           # shells closer than the grouping tolerance
        h = pkg.lowd_load_graph(g.n, torch.from_numpy(g.u).cuda(), torch.from_numpy(g.v).cuda())
        pkg.lowd_iterate(h, 4000)
        sh, lam_g, end = pkg.lowd_get_ldd(h, REL_TOL)
        sh = sh.cpu().numpy()
        lam_g = lam_g.cpu().numpy()
        assert lam_g.shape[0] == lf.shape[0], g.name
        assert np.array_equal(sh, shell), g.name
        assert np.allclose(lam_g, lf, rtol=1e-12, atol=0), g.name
        sizes = np.bincount(shell)[1:]
        assert np.array_equal(end.cpu().numpy(), np.cumsum(sizes)), g.name
        # Corollary 1 bounds from the exported decomposition against the oracle's
        for k in range(1, g.n + 1, max(1, g.n // 50)):
            b, ex = pkg.lowd_ldd_dks_bound(lam_g, end, k)
            bo, exo = orc.dks_bound(g.n, g.u, g.v, wu, k)
            assert ex == exo and abs(b - float(bo) / scale) <= 1e-12 * float(bo) / scale, (g.name, k)
        pkg.lowd_free(h)
        tested += 1
    assert tested >= 3
