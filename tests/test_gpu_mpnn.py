"""The warm-start network on the GPU (tcgen05 layer products, CUDA-core aggregation and
reductions) against the oracle in oracle/mpnn.py, which rounds to bfloat16 at the points
where the GPU stores bfloat16.  Graphs span several 128-row tiles with a ragged tail, a
single partial tile and an exact tile.

Two kinds of bar, both derived from the arithmetic:
 - exact grid: integer input features, weights in {0, +-1} with four nonzeros per output
   row, integer biases and graphs whose degrees are 0, 4 or 8.  Every value before a
   bfloat16 rounding is then exact in FP32 and FP64 alike (means divide by a power of
   two; sums stay inside 24 bits), so both sides take every rounding decision identically
   although thousands of values do round.  What remains is FP32 rounding of the readout,
   the sigmoid and the backward sums: 1e-5 on the splits, loads and loss, 1e-3 on the
   gradient (the backward's own bfloat16 operand of the tensor cores can flip a rounding
   but does not feed a nonlinearity).
 - random parameters with computed features: FP32 and FP64 sums before a rounding differ
   in the last bits, and the flipped roundings cascade through the mean aggregation.  The
   oracle measures the size of that effect itself (bfloat16 storage against none); the
   GPU must stay within twice its maximum and within its median.
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


def _circulant(n, offs, base):
    e = set()
    for i in range(n):
        for k in offs:
            a, b = base + i, base + (i + k) % n
            e.add((min(a, b), max(a, b)))
    return e


def _grid_graph(n8, n4, n_iso, seed):
    """An 8-regular and a 4-regular circulant plus isolated nodes, ids shuffled; integer
    weights 1..4."""
    e = _circulant(n8, (1, 2, 3, 4), 0) | _circulant(n4, (1, 2), n8)
    e = np.array(sorted(e), np.int64)
    n = n8 + n4 + n_iso
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    a, b = perm[e[:, 0]], perm[e[:, 1]]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    o = np.lexsort((hi, lo))
    w = rng.integers(1, 5, lo.shape[0]).astype(np.float64)
    return n, lo[o].astype(np.int32), hi[o].astype(np.int32), w[o]


def _grid_params(seed):
    rng = np.random.default_rng(seed)
    H = omp.H
    W_in = rng.integers(-1, 2, (3, H)).astype(np.float64)
    b_in = rng.integers(-2, 3, H).astype(np.float64)
    Ws, bs = [], []
    for _ in range(omp.LAYERS):
        W = np.zeros((H, 2 * H))
        for j in range(H):
            W[j, rng.choice(2 * H, 4, replace=False)] = rng.choice([-1.0, 1.0], 4)
        Ws.append(W)
        bs.append(rng.integers(-2, 3, H).astype(np.float64))
    q = rng.normal(0, 0.02, H).astype(np.float32).astype(np.float64)
    return omp.pack(W_in, b_in, Ws, bs, q)


GRID = [(600, 90, 10, 1), (64, 36, 0, 2), (100, 28, 0, 3), (900, 100, 24, 4)]


def _net(pkg, p, n, lo, hi, w, t, x=None):
    net = pkg.lowd_mpnn_create()
    pkg.lowd_mpnn_set_params(net, p.astype(np.float32))
    pkg.lowd_mpnn_bind(net, n, lo, hi, None if w is None else w.astype(np.float32),
                       None if t is None else t.astype(np.float32))
    if x is not None:
        pkg.lowd_mpnn_set_features(net, x)
    return net


def _blocks(P):
    b = omp.unpack(np.arange(P, dtype=np.float64))
    return [b[0].ravel(), b[1], b[4]] + [W.ravel() for W in b[2]] + list(b[3])


@pytest.mark.parametrize("n8,n4,niso,seed", GRID)
def test_exact_grid_forward_backward(pkg, n8, n4, niso, seed):
    n, lo, hi, w = _grid_graph(n8, n4, niso, seed)
    x = np.random.default_rng(seed + 9).integers(0, 5, (n, 3)).astype(np.float64)
    p = _grid_params(seed)
    t = np.random.default_rng(seed + 50).uniform(0.5, 3.0, n).astype(np.float32).astype(np.float64) * 4
    net = _net(pkg, p, n, lo, hi, w, t, x)
    loss = pkg.lowd_mpnn_forward(net)
    ref = omp.forward(p, n, lo, hi, w, target=t, x=x, bf16=True)
    r64 = omp.forward(p, n, lo, hi, w, target=t, x=x, bf16=False)
    # the grid really rounds (storage changes the result), and both sides agree far below that
    eff = np.abs(ref["sigma"] - r64["sigma"]).max()
    assert eff > 1e-4
    sg = pkg.lowd_mpnn_read(net, pkg.LOWD_MPNN_SIGMA)
    assert np.max(np.abs(sg - ref["sigma"])) <= 1e-5
    phi = pkg.lowd_mpnn_read(net, pkg.LOWD_MPNN_PHI)
    assert np.max(np.abs(phi - ref["phi"])) <= 1e-5 * max(1.0, np.abs(ref["phi"]).max())
    ld = pkg.lowd_mpnn_read(net, pkg.LOWD_MPNN_LOADS)
    assert np.max(np.abs(ld - ref["loads"])) <= 1e-5 * ref["loads"].max()
    assert abs(loss - ref["loss"]) <= 1e-5 * ref["loss"]
    pkg.lowd_mpnn_backward(net)
    g = pkg.lowd_mpnn_read(net, pkg.LOWD_MPNN_GRAD).astype(np.float64)
    gr = omp.backward(p, ref)
    assert np.linalg.norm(g - gr) <= 1e-3 * np.linalg.norm(gr)
    for ii in _blocks(gr.shape[0]):
        ii = ii.astype(np.int64)
        assert np.linalg.norm(g[ii] - gr[ii]) <= 2e-3 * np.linalg.norm(gr[ii]) + 1e-9, ii[:3]
    pkg.lowd_mpnn_free(net)


def _graph(n, m, seed, weighted):
    """Uneven degrees: one endpoint drawn from a power law."""
    rng = np.random.default_rng(seed)
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


def _params(seed, scale_q=0.3):
    p = omp.init_params(seed)
    W_in, b_in, Ws, bs, q = omp.unpack(p)
    rng = np.random.default_rng(seed + 7)
    b_in = rng.normal(0, 0.2, b_in.shape)
    bs = [rng.normal(0, 0.2, b.shape) for b in bs]
    q = rng.normal(0, scale_q, q.shape)
    return omp.pack(W_in, b_in, Ws, bs, q).astype(np.float32).astype(np.float64)


CASES = [(700, 6000, 1, True), (100, 900, 2, False), (128, 1500, 3, True), (1000, 30000, 4, False)]


@pytest.mark.parametrize("n,m,seed,weighted", CASES)
def test_features_against_oracle(pkg, n, m, seed, weighted):
    n, lo, hi, w = _graph(n, m, seed, weighted)
    net = _net(pkg, _params(seed), n, lo, hi, w, None)
    x = pkg.lowd_mpnn_read(net, pkg.LOWD_MPNN_FEATURES).reshape(n, 3).astype(np.float64)
    ref = omp.features(n, lo, hi, np.ones(lo.shape[0]) if w is None else w)
    # FP32 logs and sums against FP64: a few units in the last place
    assert np.all(np.abs(x - ref) <= 1e-5 * np.maximum(1.0, np.abs(ref)))
    pkg.lowd_mpnn_free(net)


@pytest.mark.parametrize("n,m,seed,weighted", CASES)
def test_random_parameters_within_the_bf16_footprint(pkg, n, m, seed, weighted):
    n, lo, hi, w = _graph(n, m, seed, weighted)
    wv = np.ones(lo.shape[0]) if w is None else w
    p = _params(seed)
    t = (np.random.default_rng(seed + 50).uniform(0.5, 3.0, n) * (wv.sum() / n)).astype(np.float32).astype(np.float64)
    net = _net(pkg, p, n, lo, hi, w, t)
    loss = pkg.lowd_mpnn_forward(net)
    ref = omp.forward(p, n, lo, hi, wv, target=t, bf16=True)
    r64 = omp.forward(p, n, lo, hi, wv, target=t, bf16=False)
    sg = pkg.lowd_mpnn_read(net, pkg.LOWD_MPNN_SIGMA)
    d, e = np.abs(sg - ref["sigma"]), np.abs(ref["sigma"] - r64["sigma"])
    assert d.max() <= 2 * e.max() + 1e-6 and np.median(d) <= np.median(e) + 1e-6
    ld = pkg.lowd_mpnn_read(net, pkg.LOWD_MPNN_LOADS)
    d, e = np.abs(ld - ref["loads"]), np.abs(ref["loads"] - r64["loads"])
    assert d.max() <= 2 * e.max() + 1e-5 * ref["loads"].max() and np.median(d) <= np.median(e) + 1e-6 * ref["loads"].max()
    # the scalar loss sums signed rounding effects that cancel, so its own footprint is no
    # bound: check it against the GPU's loads (the reduction is pinned on the exact grid)
    ld64 = ld.astype(np.float64)
    assert abs(loss - np.sum((ld64 - t) ** 2) / np.sum(t * t)) <= 1e-5 * loss
    pkg.lowd_mpnn_backward(net)
    g = pkg.lowd_mpnn_read(net, pkg.LOWD_MPNN_GRAD).astype(np.float64)
    gr, g64 = omp.backward(p, ref), omp.backward(p, r64)
    assert np.linalg.norm(g - gr) <= 2 * np.linalg.norm(gr - g64) + 1e-3 * np.linalg.norm(gr)
    pkg.lowd_mpnn_free(net)


def test_adam_step_against_oracle(pkg):
    n, lo, hi, w = _grid_graph(300, 40, 4, 9)
    x = np.random.default_rng(19).integers(0, 5, (n, 3)).astype(np.float64)
    p = _grid_params(9)
    t = np.random.default_rng(10).uniform(1.0, 5.0, n).astype(np.float32).astype(np.float64)
    net = _net(pkg, p, n, lo, hi, w, t, x)
    pkg.lowd_mpnn_forward(net)
    pkg.lowd_mpnn_backward(net)
    lr = 1e-3
    pkg.lowd_mpnn_adam(net, lr)
    p1 = pkg.lowd_mpnn_get_params(net).astype(np.float64)
    gr = omp.backward(p, omp.forward(p, n, lo, hi, w, target=t, x=x, bf16=True))
    po, _, _ = omp.adam_step(p, gr, np.zeros_like(p), np.zeros_like(p), 1, lr)
    step_g, step_o = p1 - p, po - p
    # the first step is lr * g / (|g| + eps): equal where the gradient is clearly nonzero,
    # never larger than lr anywhere
    clear = np.abs(gr) > 1e-3 * np.abs(gr).max()
    assert clear.sum() > 1000
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
    net = _net(pkg, omp.init_params(12), n, lo, hi, None, t)
    first = pkg.lowd_mpnn_forward(net)
    for _ in range(60):
        pkg.lowd_mpnn_backward(net)
        pkg.lowd_mpnn_adam(net, 3e-3)
        last = pkg.lowd_mpnn_forward(net)
    assert last < 0.5 * first, (first, last)
    pkg.lowd_mpnn_free(net)


def test_invalid_input_is_refused(pkg):
    net = pkg.lowd_mpnn_create()
    with pytest.raises(pkg.LowdError):
        pkg.lowd_mpnn_forward(net)                                          # nothing bound
    with pytest.raises(pkg.LowdError):
        pkg.lowd_mpnn_bind(net, 5, np.array([0, 3]), np.array([1, 2]))      # lo > hi
    with pytest.raises(pkg.LowdError):
        pkg.lowd_mpnn_bind(net, 5, np.array([0]), np.array([5]))            # hi out of range
    with pytest.raises(pkg.LowdError):
        pkg.lowd_mpnn_bind(net, 5, np.array([0]), np.array([1]), np.array([0.0]))  # weight 0
    pkg.lowd_mpnn_bind(net, 5, np.array([0]), np.array([1]))
    with pytest.raises(pkg.LowdError):
        pkg.lowd_mpnn_forward(net, with_loss=True)                          # no target
    with pytest.raises(pkg.LowdError):
        pkg.lowd_mpnn_backward(net)                                         # no target
    pkg.lowd_mpnn_forward(net, with_loss=False)
    assert np.all(pkg.lowd_mpnn_read(net, pkg.LOWD_MPNN_SIGMA) == 0.5)    # zero parameters
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
    one = np.ones(uh.shape[0])
    ref = omp.forward(p, nh, uh, vh, one, bf16=True)
    r64 = omp.forward(p, nh, uh, vh, one, bf16=False)
    d, e = np.abs(s - ref["sigma"]), np.abs(ref["sigma"] - r64["sigma"])
    assert d.max() <= 2 * e.max() + 1e-6 and np.median(d) <= np.median(e) + 1e-6
    # loads re-derived from the splits: conservation
    lg = pkg.lowd_get_loads(h).cpu().numpy().astype(np.float64)
    assert abs(lg.sum() - uh.shape[0]) <= 1e-5 * uh.shape[0]
    # the passes from this start reach the same optimum (Theorem 2 holds from any start)
    pkg.lowd_iterate(h, 3000, check_every=100, rel_tol=1e-9)
    S, rho, _ = pkg.lowd_extract(h)
    rho_star, B1 = oracle.densest_flow(g.n, g.u, g.v, wu)
    assert abs(rho - float(rho_star)) <= 1e-9 * float(rho_star)
    assert np.array_equal(S.cpu().numpy(), np.nonzero(B1)[0])
    pkg.lowd_free(h)
    pkg.lowd_mpnn_free(net)
