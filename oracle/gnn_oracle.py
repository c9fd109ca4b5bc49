"""CPU FP64 oracle of the warm-start network for the local eigensolves.

TEST INFRASTRUCTURE ONLY (never imported by the CUDA path).  The paper has
no learned component; this network is the project's warm start for the local
eigenproblems of Eq. 3.1, and this module is the plain reference its GPU
forward and backward kernels are checked against.

Network on one subdomain with local matrix A_ii (n x n), lumped sums s_i and
n_I interior rows:
  edge weights   w_lk = (|a_lk| + |a_kl|) / (2 sqrt(|a_ll a_kk|)) for k != l when both a_lk and
                 a_kl are nonzero (and both diagonals are), else 0; W is symmetric
  node features  with d_l = |a_ll| and deg_l = sum_k w_lk:
                 x_l = [1, d_l / max d, clip(log(d_l / mean d) / 10, -1, 1),
                        [l is an overlap row], s_l / d_l, deg_l / 4]
                 (s_l: the lumped sums of Definition 3.1, 0 on interior rows; a zero d_l gives
                 x_l2 = -1 and x_l4 = 0)
  h_0 = relu(x W_in + b_in)                                   (6 -> 64)
  h_t = relu(h_{t-1} W_s,t + (W h_{t-1}) W_n,t + b_t), t = 1..3 (64 -> 64)
  p_0 = h_3 W_out                                             (64 -> 16)
  p_{k+1} = (1 - alpha) S p_k + alpha p_0, k < K, S = D^{-1/2} W D^{-1/2}, D = diag(W 1)
  Y = p_K
Loss against a target basis Z (n x m) of the wanted eigenspace:
  L = min_C (||Z - Y C||_F^2 + eps ||C||_F^2) / m,
which depends only on span(Y) (up to eps) and vanishes when span(Y) contains span(Z).
Weights are used rounded to bfloat16 (round to nearest even) in the forward pass.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

F_IN, WIDTH, LAYERS, OUT = 6, 64, 3, 16
K_PROP, ALPHA, EPS = 32, 0.1, 1e-6


def param_shapes() -> list:
    shapes = [("W_in", (F_IN, WIDTH)), ("b_in", (WIDTH,))]
    for t in range(1, LAYERS + 1):
        shapes += [(f"W_s{t}", (WIDTH, WIDTH)), (f"W_n{t}", (WIDTH, WIDTH)), (f"b_{t}", (WIDTH,))]
    shapes.append(("W_out", (WIDTH, OUT)))
    return shapes


def num_params() -> int:
    return int(sum(np.prod(s) for _, s in param_shapes()))


def unpack(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in param_shapes():
        k = int(np.prod(shape))
        out[name] = np.asarray(flat[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in param_shapes()])


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (f >> 16) & 1
    r = ((f + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def graph_and_features(Aii: np.ndarray, lump: np.ndarray, n_I: int) -> tuple:
    """Edge-weight matrix W (sparse, symmetric, zero diagonal), S = D^-1/2 W D^-1/2, features X."""
    A = np.asarray(Aii, dtype=np.float64)
    n = A.shape[0]
    d = np.abs(np.diag(A))
    mutual = (A != 0) & (A.T != 0) & (d[:, None] > 0) & (d[None, :] > 0)
    np.fill_diagonal(mutual, False)
    Wd = np.zeros((n, n))
    den = np.sqrt(np.outer(d, d))
    Wd[mutual] = (np.abs(A) + np.abs(A.T))[mutual] / (2.0 * den[mutual])
    W = sp.csr_matrix(Wd)
    deg = Wd.sum(axis=1)
    scale = np.where(deg > 0, 1.0 / np.sqrt(np.where(deg > 0, deg, 1.0)), 0.0)
    S = sp.diags(scale) @ W @ sp.diags(scale)
    X = np.zeros((n, F_IN))
    X[:, 0] = 1.0
    dmax, dmean = d.max(), d.mean()
    X[:, 1] = d / dmax if dmax > 0 else 0.0
    with np.errstate(divide="ignore"):
        X[:, 2] = np.where(d > 0, np.clip(np.log(d / dmean) / 10.0, -1.0, 1.0) if dmean > 0 else 0.0, -1.0)
    X[n_I:, 3] = 1.0
    X[:, 4] = np.where(d > 0, lump / np.where(d > 0, d, 1.0), 0.0)
    X[:, 5] = deg / 4.0
    return W.tocsr(), S.tocsr(), X


def propagate(S, p0: np.ndarray) -> np.ndarray:
    """K_PROP steps of p <- (1 - alpha) S p + alpha p0 from p = p0."""
    p = p0
    for _ in range(K_PROP):
        p = (1.0 - ALPHA) * (S @ p) + ALPHA * p0
    return p


def propagate_adjoint(S, g: np.ndarray) -> np.ndarray:
    """Gradient with respect to p0 of <propagate(S, p0), g> (S symmetric)."""
    acc = np.zeros_like(g)
    for _ in range(K_PROP):
        acc += ALPHA * g
        g = (1.0 - ALPHA) * (S.T @ g)
    return g + acc


def forward(params: dict, W, S, X, bf16: bool = True) -> dict:
    P = {k: (round_bf16(v) if bf16 and k.startswith("W") else v) for k, v in params.items()}
    c = {"X": X}
    pre = X @ P["W_in"] + P["b_in"]
    c["pre0"] = pre
    h = np.maximum(pre, 0.0)
    c["h0"] = h
    for t in range(1, LAYERS + 1):
        m = W @ h
        pre = h @ P[f"W_s{t}"] + m @ P[f"W_n{t}"] + P[f"b_{t}"]
        c[f"m{t}"], c[f"pre{t}"] = m, pre
        h = np.maximum(pre, 0.0)
        c[f"h{t}"] = h
    p0 = h @ P["W_out"]
    c["p0"], c["Y"], c["P"] = p0, propagate(S, p0), P
    return c


def loss_and_dY(Y: np.ndarray, Z: np.ndarray) -> tuple:
    m = Z.shape[1]
    G = Y.T @ Y + EPS * np.eye(Y.shape[1])
    C = np.linalg.solve(G, Y.T @ Z)
    R = Z - Y @ C
    L = (np.sum(R * R) + EPS * np.sum(C * C)) / m
    dY = -2.0 * R @ C.T / m
    return L, dY


def backward(c: dict, W, S, dY: np.ndarray) -> dict:
    P = c["P"]
    dp0 = propagate_adjoint(S, dY)
    grads = {"W_out": c[f"h{LAYERS}"].T @ dp0}
    dh = dp0 @ P["W_out"].T
    for t in range(LAYERS, 0, -1):
        dpre = dh * (c[f"pre{t}"] > 0)
        grads[f"W_s{t}"] = c[f"h{t - 1}"].T @ dpre
        grads[f"W_n{t}"] = c[f"m{t}"].T @ dpre
        grads[f"b_{t}"] = dpre.sum(axis=0)
        dh = dpre @ P[f"W_s{t}"].T + W.T @ (dpre @ P[f"W_n{t}"].T)
    dpre = dh * (c["pre0"] > 0)
    grads["W_in"] = c["X"].T @ dpre
    grads["b_in"] = dpre.sum(axis=0)
    return grads


def subdomain_loss_grad(flat: np.ndarray, Aii, lump, n_I, Z, bf16: bool = True) -> tuple:
    """Loss and flat gradient for one subdomain."""
    params = unpack(flat)
    W, S, X = graph_and_features(Aii, lump, n_I)
    c = forward(params, W, S, X, bf16)
    L, dY = loss_and_dY(c["Y"], Z)
    return L, pack(backward(c, W, S, dY)), c["Y"]


def init_params(seed: int) -> np.ndarray:
    """Reference initialisation (He-scaled normal weights, zero biases) from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = {}
    for name, shape in param_shapes():
        if name.startswith("b"):
            d[name] = np.zeros(shape)
        else:
            d[name] = rng.standard_normal(shape) * np.sqrt(2.0 / shape[0])
    return pack(d).astype(np.float32).astype(np.float64)


def sample_loss_grad(flat: np.ndarray, subdomains: list, bf16: bool = True) -> tuple:
    """Mean loss and mean gradient over the subdomains (Aii, lump, n_I, Z) that have a target (Z with >= 1 column)."""
    tot, g, cnt = 0.0, np.zeros_like(flat, dtype=np.float64), 0
    for Aii, lump, n_I, Z in subdomains:
        if Z.shape[1] == 0:
            continue
        L, gi, _ = subdomain_loss_grad(flat, Aii, lump, n_I, Z, bf16)
        tot += L
        g += gi
        cnt += 1
    return (tot / cnt, g / cnt) if cnt else (0.0, g)


def adam_step(theta, m, v, grad, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8) -> tuple:
    """One step of Adam (Kingma and Ba, 2015, Algorithm 1) with bias correction; t counts from 1."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
