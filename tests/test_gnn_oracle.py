"""Pins of the warm-start network's CPU oracle (oracle/gnn_oracle.py).

Each test checks the oracle against something it does not compute itself:
finite differences of the loss, closed forms of the propagation on
eigenvectors of S, hand-computed features of a 1D Laplacian, the two extreme
values of the subspace loss, torch's own bfloat16 rounding, and the
bias-corrected Adam recurrence unrolled by hand.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import a2ls_oracle as orc
from oracle import gnn_oracle as gnn
from workloads import config_c4, tiny_conv_diff


def _subdomain_inputs(seed=0, delta=1):
    prob = config_c4(seed, m=12, blocks=2) if seed >= 0 else tiny_conv_diff(m=12, nb=2)
    subs = orc.overlapping_subdomains(prob.A, prob.part, delta)
    out = []
    for sub in subs:
        Aii = orc.local_matrix(prob.A, sub)
        lump = np.zeros(sub.n_i)
        lump[sub.n_I:] = orc.lumped_row_sums(prob.A, sub)
        out.append((Aii, lump, sub.n_I))
    return out


def _orthonormal(n, m, seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, m)))
    return q


def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-8, 8, 4000),
                        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -1.0 - 2.0 ** -8, 0.0, -0.0])])
    x32 = x.astype(np.float32)
    ref = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(gnn.round_bf16(x32), ref)


def test_features_of_1d_laplacian():
    n = 6
    A = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    lump = np.zeros(n)
    lump[4:] = [0.0, 1.0]                     # pretend rows 4, 5 are overlap rows, 5 touches the outside
    W, S, X = gnn.graph_and_features(A, lump, n_I=4)
    Wd = W.toarray()
    for l in range(n - 1):
        assert Wd[l, l + 1] == pytest.approx(0.5) and Wd[l + 1, l] == pytest.approx(0.5)
    assert np.count_nonzero(Wd) == 2 * (n - 1)
    deg = np.array([0.5, 1, 1, 1, 1, 0.5])
    np.testing.assert_allclose(X[:, 0], 1.0)
    np.testing.assert_allclose(X[:, 1], 1.0)
    np.testing.assert_allclose(X[:, 2], 0.0, atol=1e-15)
    np.testing.assert_array_equal(X[:, 3], [0, 0, 0, 0, 1, 1])
    np.testing.assert_allclose(X[:, 4], [0, 0, 0, 0, 0, 0.5])
    np.testing.assert_allclose(X[:, 5], deg / 4)
    Sd = S.toarray()
    assert Sd[0, 1] == pytest.approx(0.5 / np.sqrt(0.5))
    assert Sd[2, 3] == pytest.approx(0.5)


def test_weights_symmetrised_and_one_sided_edges_dropped():
    A = np.array([[4.0, -1.0, -2.0], [-3.0, 4.0, 0.0], [0.0, 0.0, 1.0]])
    W, _, X = gnn.graph_and_features(A, np.zeros(3), n_I=3)
    Wd = W.toarray()
    assert Wd[0, 1] == pytest.approx((1.0 + 3.0) / (2.0 * 4.0)) and Wd[1, 0] == Wd[0, 1]
    assert Wd[0, 2] == 0.0 and Wd[2, 0] == 0.0   # a_02 != 0 but a_20 == 0
    assert X[2, 5] == 0.0
    assert X[2, 2] == pytest.approx(np.clip(np.log(1.0 / 3.0) / 10, -1, 1))


def test_propagation_on_eigenvectors_of_S():
    # path graph: W = tridiag(1, 0, 1) has eigenvectors sin(pi j k/(n+1)) with eigenvalues 2 cos(pi j/(n+1))
    n = 9
    Wd = np.eye(n, k=1) + np.eye(n, k=-1)
    deg = Wd.sum(axis=1)
    S = sp.csr_matrix(Wd / np.sqrt(np.outer(deg, deg)))
    lam, U = np.linalg.eigh(S.toarray())
    a, K = gnn.ALPHA, gnn.K_PROP
    for j in [0, 3, n - 1]:
        u = U[:, j]
        r = (1.0 - a) * lam[j]
        closed = r ** K + a * (1.0 - r ** K) / (1.0 - r)   # geometric series of the scalar recurrence
        np.testing.assert_allclose(gnn.propagate(S, u[:, None])[:, 0], closed * u, atol=1e-13)
    # the Perron vector D^1/2 1 (eigenvalue 1) is a fixed point
    v = np.sqrt(deg)[:, None]
    np.testing.assert_allclose(gnn.propagate(S, v), v, rtol=1e-13)


def test_propagation_adjoint():
    Aii, _, _ = _subdomain_inputs()[0]
    _, S, _ = gnn.graph_and_features(Aii, np.zeros(len(Aii)), len(Aii))
    rng = np.random.default_rng(3)
    p, q = rng.standard_normal((len(Aii), 4)), rng.standard_normal((len(Aii), 4))
    assert np.sum(gnn.propagate(S, p) * q) == pytest.approx(np.sum(p * gnn.propagate_adjoint(S, q)), rel=1e-12)


def test_loss_extremes_and_basis_invariance():
    rng = np.random.default_rng(4)
    n = 50
    Y = rng.standard_normal((n, gnn.OUT))
    # target inside span(Y): the loss is only the regulariser (tiny)
    Zin, _ = np.linalg.qr(Y[:, :5] @ rng.standard_normal((5, 3)))
    L, _ = gnn.loss_and_dY(Y, Zin)
    assert L < 1e-5
    # target orthogonal to span(Y): C = 0 and L = ||Z||^2 / m = 1 for orthonormal Z
    Q, _ = np.linalg.qr(np.hstack([Y, rng.standard_normal((n, 3))]))
    Zout = Q[:, gnn.OUT:gnn.OUT + 3]
    L, dY = gnn.loss_and_dY(Y, Zout)
    assert L == pytest.approx(1.0, rel=1e-12)
    assert np.abs(dY).max() < 1e-12
    # invariance under a change of basis of Y (up to the regulariser)
    Z = _orthonormal(n, 4, 5)
    M = rng.standard_normal((gnn.OUT, gnn.OUT)) + 4 * np.eye(gnn.OUT)
    assert gnn.loss_and_dY(Y @ M, Z)[0] == pytest.approx(gnn.loss_and_dY(Y, Z)[0], rel=1e-4)


@pytest.mark.parametrize("sub", [0, 3])
def test_gradient_matches_central_differences(sub):
    Aii, lump, n_I = _subdomain_inputs()[sub]
    Z = _orthonormal(len(Aii), 5, 6)
    theta = gnn.init_params(7)
    theta[gnn.num_params() - 1000:] *= 3.0  # larger output weights: a loss well away from 1
    L, g, _ = gnn.subdomain_loss_grad(theta, Aii, lump, n_I, Z, bf16=False)
    rng = np.random.default_rng(8)
    h = 1e-6
    offs, o = {}, 0
    for name, shape in gnn.param_shapes():
        offs[name] = (o, int(np.prod(shape)))
        o += offs[name][1]
    # directional derivatives: all parameters, then each parameter group alone
    dirs = [rng.standard_normal(theta.size)]
    for name, (o, k) in offs.items():
        d = np.zeros(theta.size)
        d[o:o + k] = rng.standard_normal(k)
        dirs.append(d)
    for d in dirs:
        d /= np.linalg.norm(d)
        Lp = gnn.subdomain_loss_grad(theta + h * d, Aii, lump, n_I, Z, bf16=False)[0]
        Lm = gnn.subdomain_loss_grad(theta - h * d, Aii, lump, n_I, Z, bf16=False)[0]
        fd = (Lp - Lm) / (2 * h)
        assert fd == pytest.approx(float(g @ d), rel=1e-5, abs=1e-9 * max(1.0, abs(L)))


def test_bf16_forward_uses_rounded_weights():
    """bfloat16 holds the weight matrices only: the biases (given values bfloat16 cannot hold
    here) stay in full precision."""
    Aii, lump, n_I = _subdomain_inputs()[1]
    d = gnn.unpack(gnn.init_params(9))
    rng = np.random.default_rng(12)
    for k in d:
        if k.startswith("b"):
            d[k] = 0.1 * rng.standard_normal(d[k].shape)
    theta = gnn.pack(d)
    W, S, X = gnn.graph_and_features(Aii, lump, n_I)
    c16 = gnn.forward(gnn.unpack(theta), W, S, X, bf16=True)
    rounded = gnn.unpack(theta)
    for k in rounded:
        if k.startswith("W"):
            rounded[k] = gnn.round_bf16(rounded[k])
    c64 = gnn.forward(rounded, W, S, X, bf16=False)
    np.testing.assert_array_equal(c16["Y"], c64["Y"])
    assert not np.array_equal(c16["Y"], gnn.forward(gnn.unpack(theta), W, S, X, bf16=False)["Y"])


def test_adam_two_steps_by_hand():
    theta = np.array([1.0, -2.0])
    g1, g2 = np.array([0.5, -1.0]), np.array([0.1, 2.0])
    lr = 0.01
    th, m, v = gnn.adam_step(theta, np.zeros(2), np.zeros(2), g1, 1, lr)
    # step 1: mhat = g1, vhat = g1^2, so every parameter moves by lr * sign(g1) (up to eps)
    np.testing.assert_allclose(th, theta - lr * np.sign(g1), rtol=1e-7)
    th2, _, _ = gnn.adam_step(th, m, v, g2, 2, lr)
    m2 = 0.9 * 0.1 * g1 + 0.1 * g2
    v2 = 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2
    step = lr * (m2 / (1 - 0.81)) / (np.sqrt(v2 / (1 - 0.999 ** 2)) + 1e-8)
    np.testing.assert_allclose(th2, th - step, rtol=1e-12)


def test_sample_loss_skips_subdomains_without_target():
    subs = _subdomain_inputs()[:2]
    theta = gnn.init_params(10)
    Z0 = _orthonormal(len(subs[0][0]), 3, 11)
    L1, g1 = gnn.sample_loss_grad(theta, [(*subs[0], Z0)])
    L2, g2 = gnn.sample_loss_grad(theta, [(*subs[0], Z0), (*subs[1], np.zeros((len(subs[1][0]), 0)))])
    assert L1 == L2
    np.testing.assert_array_equal(g1, g2)
