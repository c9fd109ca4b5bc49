"""Pins for the oracle-fast local eigensolve (Eqs. 3.1-3.2 by Arnoldi on the inverted pencil).

local_gevp_fast must reproduce the dense-QZ oracle local_gevp, itself pinned by the worked example
and the library eigen-solvers in test_oracle_method: the same selected eigenvalues (relative 1e-9)
and the same selected space (sine of the largest principal angle below 1e-9), with the same kernel
part, on the 2D convection-diffusion problem's 16 subdomains, on non-symmetric, HPD and tau-selected
tiny problems, and on a pencil whose cut splits a complex-conjugate pair.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import a2ls_oracle as O
from workloads import pde


def _sin_largest_angle(Z1, Z2):
    Q1 = np.linalg.qr(Z1)[0]
    Q2 = np.linalg.qr(Z2)[0]
    return np.linalg.norm(Q2 - Q1 @ (Q1.T @ Q2), 2)


def _compare(e, f):
    assert f.dimK == e.dimK and f.kernel_dim == e.kernel_dim
    assert f.Z.shape == e.Z.shape
    assert len(f.selected) == len(e.selected)
    if len(e.selected):
        np.testing.assert_allclose(np.sort_complex(f.selected), np.sort_complex(e.selected),
                                   rtol=1e-9, atol=0)
    if e.Z.shape[1]:
        assert _sin_largest_angle(e.Z, f.Z) < 1e-9


def _subdomain_cases(prob, pou="boolean", tau=None, nev=None):
    subs = O.overlapping_subdomains(prob.A, prob.part, prob.overlap)
    D = O.partition_of_unity(subs, prob.n, pou)
    for s, d in zip(subs, D):
        e = O.local_gevp(O.local_matrix(prob.A, s), O.block_splitting(prob.A, s), d, nev or prob.nev, tau)
        As, Ats = O.sparse_local_matrices(prob.A, s)
        f = O.local_gevp_fast(As, Ats, d, nev or prob.nev, tau)
        yield s, e, f


def test_sparse_local_matrices_match_dense():
    prob = pde.tiny_conv_diff(m=14, nb=2, overlap=2, nev=4)
    for s in O.overlapping_subdomains(prob.A, prob.part, 2):
        As, Ats = O.sparse_local_matrices(prob.A, s)
        np.testing.assert_array_equal(As.toarray(), O.local_matrix(prob.A, s))
        np.testing.assert_array_equal(Ats.toarray(), O.block_splitting(prob.A, s))


def test_fast_matches_dense_on_convection_diffusion_2d():
    """All 16 subdomains of the 64 x 64 convection-diffusion problem, 4 of them with a kernel."""
    kernels = 0
    for s, e, f in _subdomain_cases(pde.config_c1()):
        _compare(e, f)
        kernels += e.kernel_dim
    assert kernels == 4


@pytest.mark.parametrize("case", ["conv_diff_overlap2", "hpd_dd", "tau_0.3", "multiplicity"])
def test_fast_matches_dense_tiny(case):
    if case == "conv_diff_overlap2":
        it = _subdomain_cases(pde.tiny_conv_diff(m=20, nb=2, overlap=2, nev=5))
    elif case == "hpd_dd":
        it = _subdomain_cases(pde.tiny_hpd_dd(m=16, nb=2, overlap=1, nev=4))
    elif case == "tau_0.3":
        it = _subdomain_cases(pde.tiny_hpd_dd(m=16, nb=2, overlap=1, nev=20, seed=21, contrast=1e4), tau=0.3)
    else:
        it = _subdomain_cases(pde.tiny_conv_diff(m=20, nb=2, overlap=1, nev=5), pou="multiplicity")
    for _, e, f in it:
        _compare(e, f)


def test_fast_matches_dense_when_the_cut_splits_a_conjugate_pair():
    n = 80
    M = sp.random(n, n, density=0.1, random_state=np.random.RandomState(3)).toarray()
    M = M - 0.8 * M.T
    Aii = M + np.diag(np.abs(M).sum(1) + 0.1)
    C = Aii.copy()
    C[-10:, -10:] -= np.diag(np.abs(M[-10:]).sum(1) * 0.7)
    d = np.random.Generator(np.random.PCG64(7)).uniform(0.2, 1.0, n)
    d[-10:] = 0.3
    split = 0
    for nev in range(3, 14):
        e = O.local_gevp(Aii, C, d, nev)
        f = O.local_gevp_fast(sp.csr_matrix(Aii), sp.csr_matrix(C), d, nev)
        _compare(e, f)
        split += e.Z.shape[1] == nev + 1
    assert split >= 1   # at least one nev cuts a pair, which then keeps nev + 1 columns
