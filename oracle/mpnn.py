"""CPU oracle of the learned warm start: a mean-aggregation message-passing network that
predicts each edge's initial split for Algorithm 1 (the paper initialises with the equal
split f_e(u) = f_e(v) = w_e / 2; any split in [0, w_e] is a valid start, since the
convergence argument of Theorem 2 does not depend on the start).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and never by the library.  Plain numpy in
float64; the forward pass, the loss and the backward pass follow the definitions below
term by term, with no fusion.  With ``bf16=True`` the values the GPU stores in bfloat16
(weights of the message-passing layers, node states h and means m, the layer gradients fed
to the tensor cores in the backward-data and weight-gradient products) are rounded to
bfloat16 (round to nearest even, through float32) at the same points; the backward pass
treats those roundings as the identity, as the GPU does.

Network (hidden width H = 64, L = 3 message-passing layers) on an undirected graph with
edges e = (lo, hi), lo < hi, weights w_e > 0; N(v) are v's neighbours, deg(v) = |N(v)|:
  inputs   x_v = (log(1 + d_v), mean_{e at v} log w_e, log(1 + sum_{u in N(v)} d_u)),
           d_v = sum_{e at v} w_e (the weighted degree)
  embed    h0_v = relu(x_v W_in + b_in)                        W_in [3, H]
  layer l  m_v = (1/deg v) sum_{u in N(v)} h_u  (0 if deg v = 0)
           h'_v = relu([h_v, m_v] W_l^T + b_l)                  W_l [H, 2H] (out, in)
  readout  phi_v = q . h3_v;  z_e = phi_lo - phi_hi;  sigma_e = 1 / (1 + exp(-z_e))
  split    f_e(lo) = sigma_e w_e,  f_e(hi) = (1 - sigma_e) w_e
  loads    l_v = sum_{e at v} f_e(v)
  loss     L = sum_v (l_v - t_v)^2 / sum_v t_v^2   (t: target loads)
Flat parameter vector (float32 on the GPU): W_in (3*H, row-major [in][out]), b_in (H),
then per layer W_l (H*2H, row-major [out][in]) and b_l (H), then q (H).

Parity pinned by tests/test_oracle_mpnn.py: gradients against central finite differences
(bf16=False), equal split at q = 0, antisymmetry under swapping an edge's ends,
equivariance under node relabelling, features against direct loops, and Adam's first step
in closed form.
"""
from __future__ import annotations

import numpy as np

H = 64
LAYERS = 3
N_IN = 3


def param_count(hidden: int = H, layers: int = LAYERS) -> int:
    return N_IN * hidden + hidden + layers * (hidden * 2 * hidden + hidden) + hidden


def unpack(p, hidden: int = H, layers: int = LAYERS):
    p = np.asarray(p, np.float64)
    o = 0
    W_in = p[o:o + N_IN * hidden].reshape(N_IN, hidden); o += N_IN * hidden
    b_in = p[o:o + hidden]; o += hidden
    Ws, bs = [], []
    for _ in range(layers):
        Ws.append(p[o:o + hidden * 2 * hidden].reshape(hidden, 2 * hidden)); o += hidden * 2 * hidden
        bs.append(p[o:o + hidden]); o += hidden
    q = p[o:o + hidden]; o += hidden
    assert o == p.shape[0]
    return W_in, b_in, Ws, bs, q


def pack(W_in, b_in, Ws, bs, q):
    parts = [np.ravel(W_in), np.ravel(b_in)]
    for W, b in zip(Ws, bs):
        parts += [np.ravel(W), np.ravel(b)]
    parts.append(np.ravel(q))
    return np.concatenate(parts).astype(np.float64)


def init_params(seed: int, hidden: int = H, layers: int = LAYERS) -> np.ndarray:
    """He-uniform weights, zero biases, small readout (a start near the equal split)."""
    rng = np.random.default_rng(seed)
    W_in = rng.uniform(-1, 1, (N_IN, hidden)) * np.sqrt(6.0 / N_IN)
    Ws = [rng.uniform(-1, 1, (hidden, 2 * hidden)) * np.sqrt(6.0 / (2 * hidden)) for _ in range(layers)]
    bs = [np.zeros(hidden) for _ in range(layers)]
    q = rng.uniform(-1, 1, hidden) * 0.01
    return pack(W_in, np.zeros(hidden), Ws, bs, q).astype(np.float32).astype(np.float64)


def round_bf16(x):
    """Round to bfloat16 (nearest, ties to even) through float32; returns float64."""
    f = np.asarray(x, np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def features(n, lo, hi, w):
    """x_v as defined in the module docstring, one node at a time from the edge list."""
    lo = np.asarray(lo, np.int64); hi = np.asarray(hi, np.int64); w = np.asarray(w, np.float64)
    d = np.zeros(n); slog = np.zeros(n); cnt = np.zeros(n)
    nbr = [[] for _ in range(n)]
    for a, b, we in zip(lo.tolist(), hi.tolist(), w.tolist()):
        d[a] += we; d[b] += we
        slog[a] += np.log(we); slog[b] += np.log(we)
        cnt[a] += 1; cnt[b] += 1
        nbr[a].append(b); nbr[b].append(a)
    two = np.array([sum(d[u] for u in nbr[v]) for v in range(n)]) if n else np.zeros(0)
    x = np.zeros((n, N_IN))
    x[:, 0] = np.log1p(d)
    x[:, 1] = np.where(cnt > 0, slog / np.maximum(cnt, 1), 0.0)
    x[:, 2] = np.log1p(two)
    return x


def _neighbour_mean(n, lo, hi, h):
    """m_v = mean of h over v's neighbours (0 for an isolated node)."""
    s = np.zeros_like(h)
    np.add.at(s, lo, h[hi])
    np.add.at(s, hi, h[lo])
    deg = np.bincount(lo, minlength=n) + np.bincount(hi, minlength=n)
    return s / np.maximum(deg, 1)[:, None], deg


def forward(params, n, lo, hi, w, target=None, x=None, bf16: bool = True):
    """The network, the split and (with a target) the loss.  Returns a dict with every
    intermediate the backward pass needs."""
    rb = round_bf16 if bf16 else (lambda a: np.asarray(a, np.float64))
    W_in, b_in, Ws, bs, q = unpack(params)
    lo = np.asarray(lo, np.int64); hi = np.asarray(hi, np.int64); w = np.asarray(w, np.float64)
    if x is None:
        x = features(n, lo, hi, w)
    a0 = x @ W_in + b_in
    h = [rb(np.maximum(a0, 0.0))]
    ms = []
    for W, b in zip(Ws, bs):
        m, deg = _neighbour_mean(n, lo, hi, h[-1])
        m = rb(m)
        ms.append(m)
        X = np.concatenate([h[-1], m], axis=1)
        a = X @ rb(W).T + b
        h.append(rb(np.maximum(a, 0.0)))
    phi = h[-1] @ q
    z = phi[lo] - phi[hi]
    sigma = 1.0 / (1.0 + np.exp(-z))
    loads = np.zeros(n)
    np.add.at(loads, lo, sigma * w)
    np.add.at(loads, hi, (1.0 - sigma) * w)
    out = dict(x=x, h=h, m=ms, phi=phi, z=z, sigma=sigma, loads=loads, lo=lo, hi=hi, w=w, n=n,
               bf16=bf16)
    if target is not None:
        t = np.asarray(target, np.float64)
        Z = float(np.sum(t * t))
        out["Z"] = Z
        out["target"] = t
        out["loss"] = float(np.sum((loads - t) ** 2) / Z) if Z > 0 else 0.0
    return out


def backward(params, fw):
    """Gradient of the loss with respect to the flat parameter vector, by the chain rule
    through every step of ``forward`` (roundings to bfloat16 passed straight through; the
    layer gradient is rounded where the GPU feeds it to the tensor cores)."""
    rb = round_bf16 if fw["bf16"] else (lambda a: np.asarray(a, np.float64))
    W_in, b_in, Ws, bs, q = unpack(params)
    n, lo, hi, w = fw["n"], fw["lo"], fw["hi"], fw["w"]
    t, Z = fw["target"], fw["Z"]
    g = 2.0 * (fw["loads"] - t) / Z                       # dL/dl_v
    s = fw["sigma"]
    delta = w * (g[lo] - g[hi]) * s * (1.0 - s)          # dL/dz_e
    psi = np.zeros(n)                                      # dL/dphi_v
    np.add.at(psi, lo, delta)
    np.add.at(psi, hi, -delta)
    dq = fw["h"][-1].T @ psi
    G = psi[:, None] * q[None, :]                          # dL/dh3
    dWs = [None] * len(Ws)
    dbs = [None] * len(Ws)
    deg = np.bincount(lo, minlength=n) + np.bincount(hi, minlength=n)
    for l in range(len(Ws) - 1, -1, -1):
        hl = fw["h"][l + 1]
        dA = G * (hl > 0)
        X = np.concatenate([fw["h"][l], fw["m"][l]], axis=1)
        dWs[l] = (X.T @ rb(dA)).T                          # [out][in]; dA enters the tensor cores
        dbs[l] = dA.sum(axis=0)
        dX = rb(dA) @ rb(Ws[l])
        dH, dM = dX[:, :H], dX[:, H:]
        dMs = dM / np.maximum(deg, 1)[:, None]
        Gp = dH.copy()
        np.add.at(Gp, lo, dMs[hi])
        np.add.at(Gp, hi, dMs[lo])
        G = Gp
    dA0 = G * (fw["h"][0] > 0)
    dW_in = fw["x"].T @ dA0
    db_in = dA0.sum(axis=0)
    return pack(dW_in, db_in, dWs, dbs, dq)


def adam_step(p, grad, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step (Kingma and Ba) with bias correction; t counts from 1.
    Returns (p, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
