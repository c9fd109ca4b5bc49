"""The reading behind a2ls_options::static_pivoting, replayed on the CPU with the oracle's steps.

Unpivoted LU with a tiny pivot replaced by the subdomain's largest diagonal entry gives the factors of
A_ii + E (E diagonal, one entry per replacement).  The method built from such factors (the local
solves of Eq. 2.4 and the local eigenproblems of Eq. 3.1 on the perturbed splitting) is still a
preconditioner, and GMRES reaches the true residual 1e-8.  The matrix is the one of the GPU test:
convection-diffusion with a zero diagonal at each part's first interior node, which every
unpivoted local LU meets as its first pivot."""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import a2ls_oracle as O
from workloads import pde


def _zero_pivot_problem():
    m = 24
    A = pde.conv_diff_2d(m, 10.0, 0.3).tolil()
    part = pde.block_partition_2d(m, 3)
    for p in range(9):
        j = int(np.nonzero(part == p)[0].min())
        A[j, j] = 0.0
    A = sp.csr_matrix(A)
    A.sort_indices()
    return A, part, pde.rhs_uniform(A.shape[0], 2)


def _unpivoted_lu_with_replacement(M, tiny_rel=1e-14):
    """L U of M without row exchanges; a pivot at most tiny_rel * max|diag| becomes max|diag|.
    Returns L U (= M + E) and the number of replacements."""
    F = np.array(M, dtype=np.float64)
    n = F.shape[0]
    scale = np.abs(np.diag(F)).max()
    replaced = 0
    for k in range(n):
        if abs(F[k, k]) <= tiny_rel * scale:
            F[k, k] = scale
            replaced += 1
        F[k + 1:, k] /= F[k, k]
        F[k + 1:, k + 1:] -= np.outer(F[k + 1:, k], F[k, k + 1:])
    L = np.tril(F, -1) + np.eye(n)
    return L @ np.triu(F), replaced


def test_unpivoted_lu_meets_a_zero_pivot_that_partial_pivoting_avoids():
    A, part, _ = _zero_pivot_problem()
    subs = O.overlapping_subdomains(A, part, 1)
    for s in subs:
        Aii = O.local_matrix(A, s)
        assert Aii[0, 0] == 0.0  # the first pivot of the unpivoted LU
        lu, piv = sla.lu_factor(Aii)
        assert np.abs(np.diag(lu)).min() > 1e-3 * np.abs(np.diag(Aii)).max()  # nonsingular with pivoting
        F, replaced = _unpivoted_lu_with_replacement(Aii)
        assert replaced >= 1
        E = F - Aii
        assert np.count_nonzero(np.abs(E) > 1e-10 * np.abs(Aii).max()) == replaced  # diagonal only
        assert np.allclose(E - np.diag(np.diag(E)), 0.0, atol=1e-10 * np.abs(Aii).max())


def test_gmres_corrects_the_replaced_pivots():
    A, part, b = _zero_pivot_problem()
    ref = O.setup(A, part, 1, 4)
    exact = O.gmres(A, lambda v: O.apply(ref, v), b, rtol=1e-8)
    assert exact.converged
    subs, D = ref.subs, ref.D
    lus, W, replaced = [], [], 0
    for s, d in zip(subs, D):
        Aii = O.local_matrix(A, s)
        Atil = O.block_splitting(A, s)
        Ab, r1 = _unpivoted_lu_with_replacement(Aii)
        Cb, r2 = _unpivoted_lu_with_replacement(Atil)
        replaced += r1 + r2
        lus.append(sla.lu_factor(Ab))
        e = O.local_gevp(Aii, Cb, d, 4, None)
        W.append(O.orthonormal_columns(d[:, None] * e.Z))
    P = O.Preconditioner(A=A, subs=subs, D=D, local_lu=lus, coarse=O.coarse_space_from_W(A, subs, W), eig=[],
                         Aii=[], Atil=[])
    res = O.gmres(A, lambda v: O.apply(P, v), b, rtol=1e-8)
    assert replaced == 2 * len(subs)
    assert res.converged and np.linalg.norm(b - A @ res.x) <= 1e-8 * np.linalg.norm(b)
    # more iterations than with exact local factors (13), within the bound the GPU test uses
    assert exact.iters < res.iters <= 3 * exact.iters + 5
