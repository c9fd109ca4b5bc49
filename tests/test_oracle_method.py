"""Pins for the oracle's eigenproblem, coarse space, preconditioners and GMRES.

Pins: the hand-derived 4-node example, closed forms (A^{-1} recovered in
the special cases of Section 2), the deflation invariant of Eq. 2.4, the
condition-number bound of Section 3.2, library eigen-solvers on the special
cases where they apply, and a brute-force Krylov least-squares check of GMRES.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import a2ls_oracle as O
from workloads import pde
from tests.golden_util import load, frac_array, frac_vector


def _golden_problem():
    g = load("laplace1d_n4.json")
    A = sp.csr_matrix(frac_array(g["A"]))
    return g, A, np.array(g["part"], dtype=np.int32)


def test_golden_ras_asm_operators():
    g, A, part = _golden_problem()
    P = O.setup(A, part, 1, nev=1, coarse=False)
    np.testing.assert_allclose(O.operator_matrix(P, "ras"), frac_array(g["M_ras"]), atol=1e-15)
    np.testing.assert_allclose(O.operator_matrix(P, "asm"), frac_array(g["M_asm"]), atol=1e-15)


def test_golden_gevp_and_coarse_operator():
    g, A, part = _golden_problem()
    P = O.setup(A, part, 1, nev=1, keep_local=True)
    for e, lam, vec in zip(P.eig, g["gevp_eigenvalues"], g["gevp_top_vector"]):
        np.testing.assert_allclose(np.sort(e.eigvals.real)[::-1], frac_vector(lam), atol=1e-14)
        assert e.kernel_dim == 0 and e.dimK == 0
        u = e.Z[:, 0] / e.Z[0, 0] * frac_vector(vec)[0]
        np.testing.assert_allclose(u, frac_vector(vec), atol=1e-13)
    for w, wg in zip(P.coarse.W, g["W_nev1"]):
        expect = frac_vector(wg) / math.sqrt(5.0)
        assert abs(abs(w[:, 0] @ expect) - 1.0) < 1e-14
    E = P.coarse.E
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(E)),
                               np.sort(np.linalg.eigvalsh(frac_array(g["E_times5"]) / 5)), atol=1e-14)


@pytest.mark.parametrize("case", range(5))
def test_golden_tau_selection(case):
    """Eq. 3.2 on the worked example: the pairs with |lambda| > 1/tau are kept (strictly), at most nev."""
    g, A, part = _golden_problem()
    c = g["tau_selection"][case]
    tau = float(Fraction(c["tau"]))
    kept = frac_vector(c["kept"]) if c["kept"] else np.zeros(0)
    P = O.setup(A, part, 1, nev=3, tau=tau, keep_local=True)
    for e, w, vec in zip(P.eig, P.coarse.W, g["gevp_top_vector"]):
        assert e.kernel_dim == 0
        np.testing.assert_allclose(np.sort(e.selected.real)[::-1], kept, atol=1e-13)
        assert w.shape[1] == len(kept)
        if len(kept) == 1:   # span(D_i u), u the eigenvector of 3
            u = frac_vector(vec) * np.array([1.0, 1.0, 0.0])
            u /= np.linalg.norm(u)
            assert abs(abs(w[:, 0] @ u) - 1.0) < 1e-13
        if len(kept) == 2:   # D_i [u v] spans the interior nodes
            np.testing.assert_allclose(w @ w.T, np.diag([1.0, 1.0, 0.0]), atol=1e-13)
    assert P.coarse.n0 == 2 * len(kept)


def test_single_subdomain_no_overlap_is_exact_inverse():
    """N = 1, delta = 0: M_RAS^{-1} = M_ASM^{-1} = A^{-1} (Eqs. 2.1, 2.3)."""
    P0 = pde.tiny_conv_diff(m=9, nb=1, overlap=0)
    P = O.setup(P0.A, P0.part, 0, nev=2, coarse=False)
    Ainv = np.linalg.inv(P0.A.toarray())
    for v in ("ras", "asm"):
        np.testing.assert_allclose(O.operator_matrix(P, v), Ainv, rtol=0, atol=1e-12)
    res = O.gmres(P0.A, lambda r: O.apply(P, r, "ras"), P0.b, rtol=1e-10)
    assert res.converged and res.iters == 1


@pytest.mark.parametrize("variant", ["deflated_ras", "deflated_asm"])
@pytest.mark.parametrize("maker", ["conv", "hpd"])
def test_full_coarse_space_gives_exact_inverse(maker, variant):
    """Boolean D and nev >= |Omega_Ii| make R_0^H square: M_deflated^{-1} = A^{-1} (Eq. 2.4)."""
    P0 = pde.tiny_conv_diff(m=8, nb=2) if maker == "conv" else pde.tiny_hpd_dd(m=8, nb=2)
    P = O.setup(P0.A, P0.part, 1, nev=100)
    assert P.coarse.n0 == P0.n
    np.testing.assert_allclose(O.operator_matrix(P, variant), np.linalg.inv(P0.A.toarray()),
                               rtol=0, atol=1e-10)


@pytest.mark.parametrize("maker", ["conv", "hpd"])
@pytest.mark.parametrize("pou", ["boolean", "multiplicity"])
def test_deflation_invariants(maker, pou):
    """M_deflated^{-1} A R_0^H = R_0^H, and R_0 (I - A R_0^H A_00^{-1} R_0) = 0 (Eq. 2.4)."""
    P0 = pde.tiny_conv_diff(m=12, nb=3) if maker == "conv" else pde.tiny_hpd_dd(m=12, nb=3)
    P = O.setup(P0.A, P0.part, 1, nev=3, pou=pou)
    Phi = P.coarse.Phi.toarray()
    assert Phi.shape[1] >= 27
    M = O.operator_matrix(P, "deflated_ras")
    A = P0.A.toarray()
    np.testing.assert_allclose(M @ A @ Phi, Phi, atol=1e-10)
    r = P0.b
    q = O.coarse_correction(P, r)
    np.testing.assert_allclose(Phi.T @ (r - A @ q), 0.0, atol=1e-12)


def test_ras_differs_from_asm_only_in_overlap_weighting():
    """With delta = 0 every D_i is the identity and RAS equals ASM (Eqs. 2.1, 2.3)."""
    P0 = pde.tiny_conv_diff(m=10, nb=2)
    P = O.setup(P0.A, P0.part, 0, nev=2, coarse=False)
    np.testing.assert_allclose(O.operator_matrix(P, "ras"), O.operator_matrix(P, "asm"), atol=1e-15)
    P1 = O.setup(P0.A, P0.part, 1, nev=2, coarse=False)
    assert not np.allclose(O.operator_matrix(P1, "ras"), O.operator_matrix(P1, "asm"))


def test_gevp_hpd_matches_generalized_eigh_in_full_space():
    """HPD case: the compressed pencil equals (Pi B Pi, C + V_K V_K^T) minus the zero modes."""
    P0 = pde.tiny_hpd_dd(m=12, nb=3, overlap=1)
    subs = O.overlapping_subdomains(P0.A, P0.part, 1)
    D = O.partition_of_unity(subs, P0.n)
    for s, d in zip(subs, D):
        Aii = O.local_matrix(P0.A, s)
        C = O.block_splitting(P0.A, s)
        e = O.local_gevp(Aii, C, d, nev=5)
        B = d[:, None] * Aii * d[None, :]
        w, V = np.linalg.eigh(C)
        tol = len(w) * np.finfo(float).eps * np.max(np.abs(w))
        VK = V[:, np.abs(w) <= tol]
        Pi = np.eye(len(w)) - VK @ VK.T
        ref = sla.eigh(Pi @ B @ Pi, C + VK @ VK.T, eigvals_only=True)
        ref = np.sort(ref)[::-1][:len(e.eigvals)]
        mine = np.sort(e.eigvals.real)[::-1]
        assert np.max(np.abs(e.eigvals.imag)) == 0.0 or np.max(np.abs(e.eigvals.imag)) < 1e-10 * np.max(np.abs(mine))
        np.testing.assert_allclose(mine[:8], ref[:8], rtol=1e-9)


def test_gevp_nonsymmetric_cross_check_and_residual():
    """Non-symmetric case: eigenvalues agree with a standard eig of C_R^{-1} B_R and
    every kept vector satisfies Pi (B u - lambda C u) = 0 with u orthogonal to ker(C)."""
    P0 = pde.tiny_conv_diff(m=12, nb=3, overlap=1)
    subs = O.overlapping_subdomains(P0.A, P0.part, 1)
    D = O.partition_of_unity(subs, P0.n)
    for s, d in zip(subs, D):
        Aii = O.local_matrix(P0.A, s)
        C = O.block_splitting(P0.A, s)
        B = d[:, None] * Aii * d[None, :]
        e = O.local_gevp(Aii, C, d, nev=4)
        U, sv, Vt = np.linalg.svd(C)
        r = int(np.sum(sv > len(sv) * np.finfo(float).eps * sv[0]))
        VR, VK = Vt[:r].T, Vt[r:].T
        ref = np.linalg.eigvals(np.linalg.solve(VR.T @ C @ VR, VR.T @ B @ VR))
        ref = ref[np.argsort(-np.abs(ref))]
        np.testing.assert_allclose(np.abs(e.eigvals[:6]), np.abs(ref[:6]), rtol=1e-9)
        assert e.dimK == VK.shape[1]
        # floating blocks: ker(C) = span(1) and D A D 1 != 0, so 1 is in the coarse space
        if e.dimK == 1:
            assert e.kernel_dim == 1
            k = e.Z[:, 0] / e.Z[0, 0]
            np.testing.assert_allclose(k, 1.0, atol=1e-10)
        lam = e.selected
        scale = np.linalg.norm(B, 2) + np.linalg.norm(C, 2)
        Pi = np.eye(len(d)) - VK @ VK.T
        j = 0
        col = e.kernel_dim
        while j < len(lam):
            if abs(lam[j].imag) > 0:
                u = e.Z[:, col] + 1j * e.Z[:, col + 1]
                col += 2
                j += 2
                l = lam[j - 2]
            else:
                u = e.Z[:, col]
                col += 1
                l = lam[j]
                j += 1
            res = np.linalg.norm(Pi @ (B @ u - l * (C @ u)))
            assert res <= 1e-9 * scale * abs(l) * np.linalg.norm(u)


def test_gevp_keeps_conjugate_partner():
    """A cut between a conjugate pair keeps both members (selection reading of Eq. 3.2)."""
    rot = np.array([[2.0, -3.0, 0.0], [3.0, 2.0, 0.0], [0.0, 0.0, 1.0]])  # eigenvalues 2 +- 3i, 1
    d = np.ones(3)
    e = O.local_gevp(rot, np.eye(3), d, nev=1)
    assert len(e.selected) == 2 and e.Z.shape[1] == 2
    np.testing.assert_allclose(sorted(e.selected.imag), [-3.0, 3.0], atol=1e-12)
    # the real basis spans the rotation plane
    np.testing.assert_allclose(np.abs(e.Z[2]), 0.0, atol=1e-14)


def test_condition_bound_hpd_dd():
    """Section 3.2: kappa(M_ASM,additive^{-1} A) <= (k_c+1)(2 + (2k_c+1) k_m / tau)."""
    for seed, tau in ((21, 0.3), (22, 0.1), (23, 0.5)):
        P0 = pde.tiny_hpd_dd(m=10, nb=3, overlap=1, seed=seed, contrast=1e4)
        P = O.setup(P0.A, P0.part, 1, nev=40, tau=tau)
        M = O.operator_matrix(P, "additive_asm")
        ev = np.linalg.eigvals(M @ P0.A.toarray())
        assert np.max(np.abs(ev.imag)) < 1e-8 * np.max(ev.real)
        kappa = np.max(ev.real) / np.min(ev.real)
        bound = O.condition_bound(P.subs, P0.n, tau)
        assert kappa <= bound, (kappa, bound)


def test_condition_bound_counts_by_hand():
    """Section 3.2's bound (k_c + 1)(2 + (2 k_c + 1) k_m / tau) with k_c and k_m counted by hand.

    4-node example (parts {0,1}, {2,3}, overlap 1): Omega_1 = {0,1,2} and Omega_2 = {1,2,3}
    intersect, so two colours; nodes 1 and 2 lie in both, so k_m = 2 and the bound is
    3 (2 + 10 / tau).  4 x 4 blocks of a 12 x 12 five-point grid, overlap 1: Omega_i reaches the
    first row or column of each edge neighbour's block, so diagonal neighbours share the corner
    node of the block between them (the overlap graph is the king's graph, four colours, and the
    greedy colouring in block order uses four); a corner node lies in its own subdomain and in the
    two whose blocks touch it, so k_m = 3 and the bound is 5 (2 + 27 / tau).
    """
    g, A, part = _golden_problem()
    subs = O.overlapping_subdomains(A, part, 1)
    assert O.coloring_number(subs) == 2 and O.multiplicity_number(subs, 4) == 2
    for tau in (0.1, 0.3, 0.5):
        assert O.condition_bound(subs, 4, tau) == pytest.approx(3.0 * (2.0 + 10.0 / tau), rel=1e-15)
    P0 = pde.tiny_conv_diff(m=12, nb=4, overlap=1)
    subs = O.overlapping_subdomains(P0.A, P0.part, 1)
    assert O.coloring_number(subs) == 4 and O.multiplicity_number(subs, 144) == 3
    for tau in (0.1, 0.3, 0.5):
        assert O.condition_bound(subs, 144, tau) == pytest.approx(5.0 * (2.0 + 27.0 / tau), rel=1e-15)


def test_coarse_space_improves_on_one_level():
    P0 = pde.tiny_hpd_dd(m=16, nb=4, overlap=1, contrast=1e4)
    P = O.setup(P0.A, P0.part, 1, nev=4)
    r1 = O.gmres(P0.A, lambda v: O.apply(P, v, "ras"), P0.b, rtol=1e-8)
    r2 = O.gmres(P0.A, lambda v: O.apply(P, v, "deflated_ras"), P0.b, rtol=1e-8)
    assert r1.converged and r2.converged and r2.iters < r1.iters


def _krylov_min_residual(A, M, b, k):
    """min_y ||b - A M^{-1} K_k y|| with K_k from QR of the explicit Krylov matrix."""
    cols = [b / np.linalg.norm(b)]
    for _ in range(k - 1):
        v = A @ M(cols[-1])
        cols.append(v / np.linalg.norm(v))
    Q, _ = np.linalg.qr(np.stack(cols, axis=1))
    AMQ = np.stack([A @ M(Q[:, j]) for j in range(k)], axis=1)
    y, *_ = np.linalg.lstsq(AMQ, b, rcond=None)
    return np.linalg.norm(b - AMQ @ y) / np.linalg.norm(b)


@pytest.mark.parametrize("flexible", [False, True])
def test_gmres_matches_brute_force_minimal_residual(flexible):
    P0 = pde.tiny_conv_diff(m=10, nb=2)
    P = O.setup(P0.A, P0.part, 1, nev=2)
    M = lambda v: O.apply(P, v)
    res = O.gmres(P0.A, M, P0.b, rtol=1e-14, restart=30, max_it=8, flexible=flexible)
    for k in range(1, 7):
        assert abs(res.history[k - 1] - _krylov_min_residual(P0.A, M, P0.b, k)) <= 1e-9
    # the iterate returned after 8 steps attains the minimal residual over the Krylov space
    assert not res.converged and res.iters == 8
    assert abs(res.relres - _krylov_min_residual(P0.A, M, P0.b, 8)) <= 1e-9


def test_gmres_distinct_eigenvalues_and_restart():
    """A diagonal matrix with 5 distinct eigenvalues: GMRES converges in at most 5 steps."""
    n = 50
    rng = np.random.Generator(np.random.PCG64(4))
    d = np.repeat([1.0, 2.0, 3.5, 7.0, 10.0], 10)
    A = sp.diags(d).tocsr()
    b = rng.uniform(-1, 1, n)
    res = O.gmres(A, None, b, rtol=1e-12)
    assert res.converged and res.iters <= 5
    # restarted: still converges, monotone estimated residuals within a cycle
    res2 = O.gmres(A, None, b, rtol=1e-10, restart=2, max_it=200)
    assert res2.converged and res2.relres <= 1e-10
    np.testing.assert_allclose(A @ res2.x, b, atol=1e-8)
