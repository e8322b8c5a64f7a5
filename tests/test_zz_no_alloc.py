"""The allocation-free extraction entry point against lowd_extract.

Some callers cannot let a library allocate device memory (their memory belongs to their
own pool, or they cannot absorb the device synchronisation cudaMalloc/cudaFree may
cause); lowd_extract_noalloc serves them from a fixed static device array.  This checks,
through the C ABI, that two calls in a row return exactly what lowd_extract returns on the
same graph and loads, for unit and lognormal weights, and that oversized graphs are
refused.  Kept in a file collected last.
"""
import numpy as np
import pytest

import synth

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


@pytest.mark.parametrize("weighted", [False, True])
def test_noalloc_extract_matches_lowd_extract(pkg, weighted):
    import torch
    g = synth.chung_lu(6000, 40000, 2.2, seed=41, block_size=40, block_p=0.5)
    w = None
    if weighted:
        w = torch.from_numpy(synth.quantise_weights(np.random.default_rng(3).lognormal(0, 1, g.m))).cuda()
    h = pkg.lowd_load_graph(g.n, torch.from_numpy(g.u).cuda(), torch.from_numpy(g.v).cuda(), w)
    pkg.lowd_iterate(h, 25)
    S_ref, rho_ref, _ = pkg.lowd_extract(h, want_loads=False)
    loads = pkg.lowd_get_loads(h)
    u, v, gw = pkg.lowd_get_graph(h)
    for call in range(2):
        S = torch.full((g.n,), -1, dtype=torch.int32, device="cuda")
        status, k, rho = pkg.lowd_extract_noalloc(g.n, u, v, gw if weighted else None, loads, S)
        assert status == pkg.LOWD_OK, call
        assert k == S_ref.shape[0], call
        assert torch.equal(S[:k], S_ref), call
        assert rho == rho_ref, call
    pkg.lowd_free(h)


def test_noalloc_extract_refuses_oversized_graphs(pkg):
    import torch
    n = 65537
    u = torch.zeros(1, dtype=torch.int32, device="cuda")
    v = torch.ones(1, dtype=torch.int32, device="cuda")
    loads = torch.zeros(n, dtype=torch.float32, device="cuda")
    status, k, rho = pkg.lowd_extract_noalloc(n, u, v, None, loads)
    assert status == pkg.LOWD_ERR_TOO_LARGE
