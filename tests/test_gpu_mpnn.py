"""The warm-start network on the GPU (tcgen05 layer products, CUDA-core aggregation and
reductions) against the oracle in oracle/mpnn.py, which rounds to bfloat16 at the points
where the GPU stores bfloat16.  Graphs span several 128-row tiles with a ragged tail, a
single partial tile and an exact tile.

Bars: FP32 accumulation against FP64 (with identical bfloat16 storage points) differs by
parts in 1e6 (measured on the CPU with an FP32 emulation); rare rounding flips of a stored
bfloat16 value move single entries by one bfloat16 step.  The test bars are 1e-4 on the
features, splits, loads and loss and 1e-3 on the gradient norm, with room for both.
"""
import numpy as np
import pytest

from oracle import mpnn as omp

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


def _graph(n, m, seed, weighted):
    rng = np.random.default_rng(seed)
    # power-law-ish endpoint choice so degrees are uneven (a few high-degree rows)
    pr = 1.0 / np.arange(1, n + 1) ** 0.6
    pr /= pr.sum()
    pairs = set()
    while len(pairs) < m:
        a = rng.choice(n, 4 * m, p=pr)
        b = rng.integers(0, n, 4 * m)
        for x, y in zip(a.tolist(), b.tolist()):
            if x != y:
                pairs.add((min(x, y), max(x, y)))
            if len(pairs) >= m:
                break
    e = np.array(sorted(pairs), np.int32)
    w = rng.lognormal(0, 0.7, m).astype(np.float32).astype(np.float64) if weighted else None
    return n, e[:, 0], e[:, 1], w


def _params(seed, scale_q=0.5):
    p = omp.init_params(seed)
    W_in, b_in, Ws, bs, q = omp.unpack(p)
    rng = np.random.default_rng(seed + 7)
    b_in = rng.normal(0, 0.2, b_in.shape)
    bs = [rng.normal(0, 0.2, b.shape) for b in bs]
    q = rng.normal(0, scale_q, q.shape)
    return omp.pack(W_in, b_in, Ws, bs, q).astype(np.float32).astype(np.float64)


CASES = [(700, 6000, 1, True), (100, 900, 2, False), (128, 1500, 3, True), (1000, 30000, 4, False)]


@pytest.mark.parametrize("n,m,seed,weighted", CASES)
def test_forward_backward_against_oracle(pkg, n, m, seed, weighted):
    n, lo, hi, w = _graph(n, m, seed, weighted)
    wv = np.ones(lo.shape[0]) if w is None else w
    p = _params(seed)
    t = np.random.default_rng(seed + 50).uniform(0.5, 3.0, n) * (wv.sum() / n)
    net = pkg.lowd_mpnn_create()
    pkg.lowd_mpnn_set_params(net, p.astype(np.float32))
    pkg.lowd_mpnn_bind(net, n, lo, hi, None if w is None else w.astype(np.float32), t.astype(np.float32))
    loss = pkg.lowd_mpnn_forward(net)
    ref = omp.forward(p, n, lo, hi, wv, target=t.astype(np.float32).astype(np.float64), bf16=True)
    x = pkg.lowd_mpnn_read(net, pkg.LOWD_MPNN_FEATURES).reshape(n, 3)
    assert np.max(np.abs(x - ref["x"])) <= 1e-4 * max(1.0, np.abs(ref["x"]).max())
    sg = pkg.lowd_mpnn_read(net, pkg.LOWD_MPNN_SIGMA)
    assert np.max(np.abs(sg - ref["sigma"])) <= 1e-4
    ld = pkg.lowd_mpnn_read(net, pkg.LOWD_MPNN_LOADS)
    assert np.max(np.abs(ld - ref["loads"])) <= 1e-4 * ref["loads"].max()
    assert abs(loss - ref["loss"]) <= 1e-4 * ref["loss"]
    pkg.lowd_mpnn_backward(net)
    g = pkg.lowd_mpnn_read(net, pkg.LOWD_MPNN_GRAD).astype(np.float64)
    gr = omp.backward(p, ref)
    assert np.linalg.norm(g - gr) <= 1e-3 * np.linalg.norm(gr)
    # every parameter block on its own (embedding, each layer's W and b, readout)
    blocks = omp.unpack(np.arange(gr.shape[0], dtype=np.float64))
    idx = [blocks[0].ravel(), blocks[1], blocks[4]] + [W.ravel() for W in blocks[2]] + list(blocks[3])
    for ii in idx:
        ii = ii.astype(np.int64)
        assert np.linalg.norm(g[ii] - gr[ii]) <= 2e-3 * np.linalg.norm(gr[ii]) + 1e-7, ii[:3]
    pkg.lowd_mpnn_free(net)


def test_adam_step_against_oracle(pkg):
    n, lo, hi, w = _graph(400, 4000, 9, True)
    p = _params(9)
    t = np.random.default_rng(10).uniform(1.0, 5.0, n)
    net = pkg.lowd_mpnn_create()
    pkg.lowd_mpnn_set_params(net, p.astype(np.float32))
    pkg.lowd_mpnn_bind(net, n, lo, hi, w.astype(np.float32), t.astype(np.float32))
    pkg.lowd_mpnn_forward(net)
    pkg.lowd_mpnn_backward(net)
    lr = 1e-3
    pkg.lowd_mpnn_adam(net, lr)
    p1 = pkg.lowd_mpnn_get_params(net).astype(np.float64)
    ref = omp.forward(p, n, lo, hi, w, target=t.astype(np.float32).astype(np.float64), bf16=True)
    gr = omp.backward(p, ref)
    po, _, _ = omp.adam_step(p, gr, np.zeros_like(p), np.zeros_like(p), 1, lr)
    step_g, step_o = p1 - p, po - p
    # the first step is lr * g / (|g| + eps): equal where the gradient is clearly nonzero,
    # and never larger than lr anywhere
    clear = np.abs(gr) > 1e-3 * np.abs(gr).max()
    assert np.all(np.abs(step_g) <= lr * (1 + 1e-5) + 1e-7)
    assert np.max(np.abs(step_g[clear] - step_o[clear])) <= 1e-3 * lr + 1e-7
    pkg.lowd_mpnn_free(net)


def test_training_steps_reduce_the_loss(pkg):
    n, lo, hi, w = _graph(600, 5000, 11, False)
    # target: loads of a fixed split favouring the lower-degree end
    deg = np.bincount(lo, minlength=n) + np.bincount(hi, minlength=n)
    s = 1.0 / (1.0 + np.exp(np.log(deg[lo]) - np.log(deg[hi])))
    t = np.zeros(n)
    np.add.at(t, lo, s)
    np.add.at(t, hi, 1 - s)
    net = pkg.lowd_mpnn_create()
    pkg.lowd_mpnn_set_params(net, omp.init_params(12).astype(np.float32))
    pkg.lowd_mpnn_bind(net, n, lo, hi, None, t.astype(np.float32))
    first = pkg.lowd_mpnn_forward(net)
    for _ in range(60):
        pkg.lowd_mpnn_backward(net)
        pkg.lowd_mpnn_adam(net, 3e-3)
        last = pkg.lowd_mpnn_forward(net)
    assert last < 0.5 * first, (first, last)
    pkg.lowd_mpnn_free(net)


def test_invalid_graph_is_refused(pkg):
    net = pkg.lowd_mpnn_create()
    with pytest.raises(pkg.LowdError):
        pkg.lowd_mpnn_bind(net, 5, np.array([0, 3]), np.array([1, 2]))      # lo > hi
    with pytest.raises(pkg.LowdError):
        pkg.lowd_mpnn_bind(net, 5, np.array([0]), np.array([5]))            # hi out of range
    with pytest.raises(pkg.LowdError):
        pkg.lowd_mpnn_bind(net, 5, np.array([0]), np.array([1]), np.array([0.0]))  # weight 0
    with pytest.raises(pkg.LowdError):
        pkg.lowd_mpnn_forward(net)                                          # nothing bound
    pkg.lowd_mpnn_bind(net, 5, np.array([0]), np.array([1]))
    with pytest.raises(pkg.LowdError):
        pkg.lowd_mpnn_forward(net, with_loss=True)                          # no target
    pkg.lowd_mpnn_forward(net, with_loss=False)
    pkg.lowd_mpnn_free(net)


def test_warm_start_sets_the_predicted_splits_and_converges(pkg):
    import torch
    import oracle
    import synth
    oracle.build()
    g = synth.chung_lu(3000, 20000, 2.2, seed=21, block_size=30, block_p=0.5)
    p = _params(22, scale_q=0.3)
    net = pkg.lowd_mpnn_create()
    pkg.lowd_mpnn_set_params(net, p.astype(np.float32))
    h = pkg.lowd_load_graph(g.n, torch.from_numpy(g.u).cuda(), torch.from_numpy(g.v).cuda())
    pkg.lowd_prune(h)
    wu, _ = oracle.weight_units(g.m, None)
    pr = oracle.prune(g.n, g.u, g.v, wu, False)
    nh, uh, vh, _, idmap = oracle.compact(g.n, g.u, g.v, None, pr["removal_round"] < 0)
    pkg.lowd_warm_start(h, net)
    s = pkg.lowd_get_splits(h).cpu().numpy().astype(np.float64)
    ref = omp.forward(p, nh, uh, vh, np.ones(uh.shape[0]), bf16=True)
    assert np.max(np.abs(s - ref["sigma"])) <= 1e-4
    lg = pkg.lowd_get_loads(h).cpu().numpy().astype(np.float64)
    assert np.max(np.abs(lg - ref["loads"])) <= 1e-4 * ref["loads"].max()
    # the passes from this start reach the same optimum (Theorem 2 holds from any start)
    pkg.lowd_iterate(h, 3000, check_every=100, rel_tol=1e-9)
    S, rho, _ = pkg.lowd_extract(h)
    rho_star, B1 = oracle.densest_flow(g.n, g.u, g.v, wu)
    assert abs(rho - float(rho_star)) <= 1e-9 * float(rho_star)
    assert np.array_equal(S.cpu().numpy(), np.nonzero(B1)[0])
    pkg.lowd_free(h)
    pkg.lowd_mpnn_free(net)
