"""The allocation-free extraction entry point against lowd_extract and the oracle.

Some callers cannot let a library allocate device memory (their memory belongs to their
own pool, or they cannot absorb the device synchronisation cudaMalloc/cudaFree may
cause); lowd_extract_noalloc serves them from a fixed static device array.  This checks,
through the C ABI, that two calls in a row return exactly what lowd_extract returns on the
same graph and loads, and the oracle's extraction on the same FP32 loads (S* equal, rho*
within 1e-9 relative), for unit and lognormal weights and at the largest accepted size;
that oversized graphs are refused; and that bad edges (an id out of range, a self-loop, a
non-finite weight) are reported as invalid arguments without being read past.  Kept in a
file collected last.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

MAX_NODES = 65536   # LOWD_NOALLOC_MAX_NODES


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


def _check_against_both(pkg, orc, h, n, weighted, passes):
    import torch
    if passes:
        pkg.lowd_iterate(h, passes)
    S_ref, rho_ref, _ = pkg.lowd_extract(h, want_loads=False)
    loads = pkg.lowd_get_loads(h)
    u, v, gw = pkg.lowd_get_graph(h)
    # the oracle's extraction on the same FP32 loads and edges
    un, vn = u.cpu().numpy(), v.cpu().numpy()
    wn = gw.cpu().numpy().astype(np.float64) if weighted else None
    wu, scale = orc.weight_units(un.shape[0], wn)
    So, Wo = orc.extract(n, un, vn, wu, loads.cpu().numpy().astype(np.float64))
    rho_o = Wo / scale / So.shape[0]
    for call in range(2):
        S = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        status, k, rho = pkg.lowd_extract_noalloc(n, u, v, gw if weighted else None, loads, S)
        assert status == pkg.LOWD_OK, call
        assert k == S_ref.shape[0], call
        assert torch.equal(S[:k], S_ref), call
        assert rho == rho_ref, call
        assert np.array_equal(S[:k].cpu().numpy(), So), call
        assert abs(rho - rho_o) <= 1e-9 * rho_o, call


@pytest.mark.parametrize("weighted", [False, True])
def test_noalloc_extract_matches_lowd_extract_and_oracle(pkg, orc, weighted):
    import torch
    g = synth.chung_lu(6000, 40000, 2.2, seed=41, block_size=40, block_p=0.5)
    w = None
    if weighted:
        w = torch.from_numpy(synth.quantise_weights(np.random.default_rng(3).lognormal(0, 1, g.m))).cuda()
    h = pkg.lowd_load_graph(g.n, torch.from_numpy(g.u).cuda(), torch.from_numpy(g.v).cuda(), w)
    _check_against_both(pkg, orc, h, g.n, weighted, 25)
    pkg.lowd_free(h)


def test_noalloc_extract_at_the_largest_accepted_size(pkg, orc):
    """n = 65,536, the size at which the scratch carve-up is closest to its limit; the
    equal-split loads (degree / 2) leave many exact ties, so the id tie-break is exercised."""
    import torch
    g = synth.chung_lu(MAX_NODES, 250000, 2.2, seed=43, block_size=60, block_p=0.5)
    h = pkg.lowd_load_graph(g.n, torch.from_numpy(g.u).cuda(), torch.from_numpy(g.v).cuda())
    _check_against_both(pkg, orc, h, g.n, False, 0)
    pkg.lowd_free(h)


def test_noalloc_extract_refuses_oversized_graphs(pkg):
    import torch
    n = MAX_NODES + 1
    u = torch.zeros(1, dtype=torch.int32, device="cuda")
    v = torch.ones(1, dtype=torch.int32, device="cuda")
    loads = torch.zeros(n, dtype=torch.float32, device="cuda")
    status, k, rho = pkg.lowd_extract_noalloc(n, u, v, None, loads)
    assert status == pkg.LOWD_ERR_TOO_LARGE


@pytest.mark.parametrize("bad", ["id_high", "id_negative", "self_loop", "nan_weight", "zero_weight",
                                 "inf_weight"])
def test_noalloc_extract_rejects_bad_edges(pkg, bad):
    """An edge the library would refuse at load time is skipped on the GPU and reported as
    LOWD_ERR_INVALID_ARG; a valid call right after it still gives the right answer."""
    import torch
    n = 6
    u = np.array([0, 1, 2, 3], np.int32)
    v = np.array([1, 2, 0, 4], np.int32)
    w = np.ones(4, np.float32)
    if bad == "id_high":
        v[3] = n + 1000
    elif bad == "id_negative":
        u[3] = -7
    elif bad == "self_loop":
        v[3] = 3
    elif bad == "nan_weight":
        w[1] = np.nan
    elif bad == "zero_weight":
        w[1] = 0.0
    else:
        w[2] = np.inf
    weighted = bad.endswith("weight")
    loads = torch.tensor([1.0, 1.0, 1.0, 0.5, 0.5, 0.0], dtype=torch.float32, device="cuda")
    tu, tv = torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()
    tw = torch.from_numpy(w).cuda() if weighted else None
    status, _, _ = pkg.lowd_extract_noalloc(n, tu, tv, tw, loads)
    assert status == pkg.LOWD_ERR_INVALID_ARG
    # the triangle {0, 1, 2} is the densest set of the valid graph
    ok_u = torch.tensor([0, 1, 2, 3], dtype=torch.int32, device="cuda")
    ok_v = torch.tensor([1, 2, 0, 4], dtype=torch.int32, device="cuda")
    S = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    status, k, rho = pkg.lowd_extract_noalloc(n, ok_u, ok_v, None, loads, S)
    assert status == pkg.LOWD_OK and k == 3 and rho == 1.0
    assert S[:3].cpu().tolist() == [0, 1, 2]
