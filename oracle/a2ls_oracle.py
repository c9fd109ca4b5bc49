"""CPU FP64 oracle for the algebraic two-level Schwarz preconditioner.

TEST INFRASTRUCTURE ONLY.  This module is a plain, slow, obviously correct
restatement of the method of Al Daas, Jolivet and Rees, "Efficient algebraic
two-level Schwarz preconditioner for sparse matrices" (arXiv 2201.02250),
written with numpy/scipy in float64.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import it; the CUDA library never does, and
the two share no code.

Every function names the passage it follows (section, definition, equation).
Readings taken where the paper is silent or ambiguous are marked READING.
All functions below are pinned by tests in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

EPS = np.finfo(np.float64).eps


# ---------------------------------------------------------------------------
# Section 2: algebraic overlap, restriction operators, partition of unity
# ---------------------------------------------------------------------------

def adjacency_lists(A: sp.spmatrix) -> list:
    """Neighbours of every node in the adjacency graph G(A) (Section 2).

    READING: for a non-symmetric pattern the graph of A + A^T is used (the
    paper partitions the symmetric part A^T + A, Section 4).  Self loops are
    removed.
    """
    P = (abs(A) + abs(A.T)).tocsr()
    P.sort_indices()
    out = []
    for j in range(P.shape[0]):
        nb = P.indices[P.indptr[j]:P.indptr[j + 1]]
        out.append(nb[nb != j])
    return out


@dataclass
class Subdomain:
    """Omega_i = [Omega_Ii, Omega_Gamma_i] (ordered concatenation, Notation, Section 2)."""
    interior: np.ndarray   # Omega_Ii, ascending
    gamma: np.ndarray      # Omega_Gamma_i, ascending

    @property
    def idx(self) -> np.ndarray:
        return np.concatenate([self.interior, self.gamma]).astype(np.int64)

    @property
    def n_i(self) -> int:
        return len(self.interior) + len(self.gamma)

    @property
    def n_I(self) -> int:
        return len(self.interior)


def overlapping_subdomains(A: sp.spmatrix, part: np.ndarray, delta: int) -> list:
    """Overlapping subdomains grown algebraically from a partition (Section 2).

    Omega_Gamma_i holds the nodes at distance one in G(A) from Omega_Ii.
    READING: an overlap of delta layers repeats that step delta times,
    Omega^(k) = Omega^(k-1) U adj(Omega^(k-1)), and Omega_Gamma_i is every node
    added in the process.  The interior is listed in ascending global order, the
    overlap layer by layer (the nodes added by step 1 ascending, then those of
    step 2, ...).  Section 2 defines Omega_Gamma_i as a set and Eqs. 2.3-2.4 use
    it only through R_i, so the method is invariant under any ordering of it.
    """
    nbrs = adjacency_lists(A)
    N = int(part.max()) + 1
    subs = []
    for i in range(N):
        interior = np.flatnonzero(part == i)
        member = set(interior.tolist())
        frontier = set(member)
        layers = []
        for _ in range(delta):
            new = set()
            for j in frontier:
                for k in nbrs[j]:
                    if k not in member:
                        new.add(int(k))
            member |= new
            frontier = new
            layers.extend(sorted(new))
        gamma = np.array(layers, dtype=np.int64)
        subs.append(Subdomain(interior.astype(np.int64), gamma))
    return subs


def restriction(sub: Subdomain, n: int) -> sp.csr_matrix:
    """R_i = I_n(Omega_i, :) (Section 2)."""
    idx = sub.idx
    return sp.csr_matrix((np.ones(len(idx)), (np.arange(len(idx)), idx)), shape=(len(idx), n))


def partition_of_unity(subs: list, n: int, kind: str = "boolean") -> list:
    """Non-negative diagonals D_i with sum_i R_i^T D_i R_i = I_n (Section 2).

    READING: the paper allows any such family.  "boolean" (the default) puts
    1 on Omega_Ii and 0 on Omega_Gamma_i; "multiplicity" puts 1/k(j) on every
    node j of Omega_i, with k(j) the number of subdomains containing j.
    """
    if kind == "boolean":
        return [np.concatenate([np.ones(s.n_I), np.zeros(s.n_i - s.n_I)]) for s in subs]
    if kind == "multiplicity":
        count = np.zeros(n)
        for s in subs:
            count[s.idx] += 1.0
        return [1.0 / count[s.idx] for s in subs]
    raise ValueError(kind)


# ---------------------------------------------------------------------------
# Section 3.1, Definition 3.1: local matrices and local block splitting
# ---------------------------------------------------------------------------

def local_matrix(A: sp.spmatrix, sub: Subdomain) -> np.ndarray:
    """A_ii = R_i A R_i^T as a dense matrix (Eq. 2.1)."""
    idx = sub.idx
    return A.tocsr()[idx][:, idx].toarray()


def lumped_row_sums(A: sp.spmatrix, sub: Subdomain) -> np.ndarray:
    """s_i(j) = sum of |entries| of row j of A_Gamma_c,i, j in Omega_Gamma_i (Definition 3.1).

    A_Gamma_c,i = A(Omega_Gamma_i, Omega_c_i) couples the overlap to the
    nodes outside Omega_i.
    """
    n = A.shape[0]
    outside = np.ones(n, dtype=bool)
    outside[sub.idx] = False
    Ar = abs(A.tocsr()[sub.gamma])
    return np.asarray(Ar[:, np.flatnonzero(outside)].sum(axis=1)).ravel()


def block_splitting(A: sp.spmatrix, sub: Subdomain) -> np.ndarray:
    """Local block splitting matrix A~_ii with lumping in the overlap (Definition 3.1).

    A~_ii = [[A_Ii, A_IGamma_i], [A_GammaI_i, A_Gamma_i - diag(s_i)]].
    """
    At = local_matrix(A, sub)
    s = lumped_row_sums(A, sub)
    nI = sub.n_I
    for j in range(len(s)):
        At[nI + j, nI + j] -= s[j]
    return At


def global_splitting(A: sp.spmatrix, sub: Subdomain) -> np.ndarray:
    """A~_i = R_i^T A~_ii R_i as a dense n x n matrix (Definition 3.1)."""
    n = A.shape[0]
    out = np.zeros((n, n))
    idx = sub.idx
    out[np.ix_(idx, idx)] = block_splitting(A, sub)
    return out


# ---------------------------------------------------------------------------
# Section 3.2: local generalized eigenproblem and coarse space
# ---------------------------------------------------------------------------

@dataclass
class LocalEigen:
    """Result of the local eigenproblem for one subdomain."""
    Z: np.ndarray               # n_i x m basis of the selected space (real)
    kernel_dim: int             # columns of Z spanning (L_i cap K_i)^{perp K_i}
    eigvals: np.ndarray         # all finite eigenvalues, sorted by |lambda| descending
    selected: np.ndarray        # the finite eigenvalues that were kept
    dimK: int                   # dim ker(A~_ii)


def _null_space(M: np.ndarray) -> tuple:
    """Right null basis and its orthogonal complement from the SVD.

    Singular values at or below n * eps * sigma_max count as zero.
    """
    U, sv, Vt = np.linalg.svd(M)
    tol = M.shape[0] * EPS * (sv[0] if len(sv) else 0.0)
    r = int(np.sum(sv > tol))
    return Vt[r:].T, Vt[:r].T


def local_gevp(Aii: np.ndarray, Atil: np.ndarray, d: np.ndarray, nev: int,
               tau: float | None = None) -> LocalEigen:
    """Local eigenproblem of Eq. 3.1 and the selection of Eq. 3.2.

    B = D_i A_ii D_i, C = A~_ii, K_i = ker(C), L_i = ker(B).
    Kernel part: (L_i cap K_i)^{perp K_i} = V_K * (right singular vectors of
    B V_K with non-zero singular value); these count as lambda = infinity.
    Finite part: Pi_i is taken as the orthogonal projector onto ker(C)^perp
    with basis V_R (READING: identical to the paper's projection on range(C)
    when C is Hermitian); the pencil is compressed to
    (V_R^T B V_R, V_R^T C V_R) and solved by dense QZ, u = V_R a.
    Selection (READING): eigenpairs are sorted by |lambda| descending,
    infinity first; with ``tau`` None the first ``nev`` are kept, otherwise
    those with |lambda| > 1/tau, capped at ``nev``.  If the cut splits a
    complex-conjugate pair the partner is kept as well.  A pair contributes
    the real basis [Re u, Im u].
    """
    B = (d[:, None] * Aii) * d[None, :]
    C = Atil
    VK, VR = _null_space(C)
    dimK = VK.shape[1]
    kernel_cols = _kernel_part(B, VK)
    kdim = kernel_cols.shape[1]
    Bc = VR.T @ B @ VR
    Cc = VR.T @ C @ VR
    lam, a = sla.eig(Bc, Cc)
    return _select_eigenpairs(lam, lambda j: VR @ a[:, j], kernel_cols, nev, tau, dimK)


def local_gevp_fast(Aii: sp.spmatrix, Atil: sp.spmatrix, d: np.ndarray, nev: int,
                    tau: float | None = None, seed: int = 0) -> LocalEigen:
    """Oracle-fast form of local_gevp for subdomains too large for dense QZ (Eqs. 3.1-3.2).

    The same compressed pencil (V_R^T B V_R, V_R^T C V_R), with B = D_i A_ii D_i and C = A~_ii kept
    sparse, and the same kernel part and selection.  Its largest-|lambda| eigenpairs are found by
    Arnoldi (ARPACK through scipy.sparse.linalg.eigs) on the operator T_R = C_R^{-1} B_R, the inverted
    form of the pencil, applied in the full local space: for u in range(V_R), T u = y solves
        [[C, V_K], [V_K^T, 0]] [y; s] = [B u; 0],
    i.e. V_R^T C y = V_R^T B u with y orthogonal to ker(C), which is V_R T_R V_R^T u (the bordered
    matrix is factored once by sparse LU).  T maps every vector into range(V_R), so its non-zero
    eigenvalues are those of T_R and their eigenvectors lie in range(V_R).  ker(C) comes from the
    dense SVD, as in local_gevp.  The start vector is a seeded uniform vector projected onto
    range(V_R).
    """
    import scipy.sparse.linalg as spla

    n = Aii.shape[0]
    Dm = sp.diags(d)
    B = (Dm @ sp.csr_matrix(Aii) @ Dm).tocsr()
    C = sp.csr_matrix(Atil)
    VK, _ = _null_space(C.toarray())
    dimK = VK.shape[1]
    kernel_cols = _kernel_part(B, VK)
    kdim = kernel_cols.shape[1]
    want = min(max(nev - kdim, 0), n - dimK)
    if want == 0:
        return _select_eigenpairs(np.zeros(0, dtype=complex), None, kernel_cols, nev, tau, dimK)
    K = sp.bmat([[C, sp.csr_matrix(VK)], [sp.csr_matrix(VK.T), None]], format="csc")
    lu = spla.splu(K)
    rhs = np.zeros(n + dimK)

    def T(u):
        rhs[:n] = B @ np.asarray(u).ravel()
        return lu.solve(rhs)[:n]

    rng = np.random.Generator(np.random.PCG64(seed))
    v0 = rng.uniform(-1.0, 1.0, n)
    v0 -= VK @ (VK.T @ v0)
    k = min(want + 2, n - dimK - 2)   # two more than kept, so that a pair cut at the end is seen
    if k < want + 1:
        raise ValueError("local_gevp_fast: subdomain too small for Arnoldi, use local_gevp")
    op = spla.LinearOperator((n, n), matvec=T, dtype=np.float64)
    lam, U = spla.eigs(op, k=k, which="LM", v0=v0, tol=1e-13, ncv=min(n - dimK - 1, max(2 * k + 1, 40)),
                       maxiter=100 * n)
    return _select_eigenpairs(lam, lambda j: U[:, j], kernel_cols, nev, tau, dimK)


def _fast_one(job: tuple) -> LocalEigen:
    Aii, Atil, d, nev, tau = job
    return local_gevp_fast(Aii, Atil, d, nev, tau)


def local_eigen_fast_many(A: sp.spmatrix, subs: list, D: list, nev: int, indices, tau: float | None = None,
                          workers: int = 1) -> list:
    """local_gevp_fast for the subdomains ``indices`` (in that order), optionally in a pool of
    ``workers`` processes started with spawn (one BLAS thread each)."""
    jobs = []
    for i in indices:
        Aii, Atil = sparse_local_matrices(A, subs[i])
        jobs.append((Aii, Atil, D[i], nev, tau))
    if workers <= 1:
        return [_fast_one(j) for j in jobs]
    import multiprocessing
    import os
    from concurrent.futures import ProcessPoolExecutor

    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"   # inherited by the spawned workers before they import numpy
    try:
        with ProcessPoolExecutor(max_workers=workers, mp_context=multiprocessing.get_context("spawn")) as ex:
            return list(ex.map(_fast_one, jobs, chunksize=1))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def sparse_local_matrices(A: sp.spmatrix, sub: Subdomain) -> tuple:
    """A_ii and A~_ii (Definition 3.1) as sparse matrices, for local_gevp_fast."""
    A = A.tocsr()
    idx = sub.idx
    Aii = A[idx][:, idx].tocsr()
    s = lumped_row_sums(A, sub)
    nI = sub.n_I
    At = Aii.tolil()
    for j in range(len(s)):
        At[nI + j, nI + j] -= s[j]
    return Aii, At.tocsr()


def _kernel_part(B, VK: np.ndarray) -> np.ndarray:
    """(L_i cap K_i)^{perp K_i} (Eq. 3.2): V_K times the right singular vectors of B V_K whose
    singular value is non-zero (above max(shape) * eps * ||B||_2)."""
    if VK.shape[1] == 0:
        return np.zeros((VK.shape[0], 0))
    BV = B @ VK
    _, sv, Vt = np.linalg.svd(BV)
    Bn = np.linalg.norm(B.toarray() if sp.issparse(B) else B, 2)
    tol = max(BV.shape) * EPS * max(Bn, 1e-300)
    r = int(np.sum(sv > tol))
    return VK @ Vt[:r].T


def _select_eigenpairs(lam: np.ndarray, vector, kernel_cols: np.ndarray, nev: int, tau, dimK: int) -> LocalEigen:
    """Selection of Eq. 3.2 from finite eigenvalues ``lam`` (any order) with eigenvectors ``vector(j)``.

    READING: sorted by |lambda| descending (the kernel part, lambda = infinity, first); the first
    nev - dim(kernel part) finite pairs are kept, or with tau > 0 only those with |lambda| > 1/tau
    among them; a complex-conjugate pair cut by the count keeps its partner; a pair contributes the
    real basis [Re u, Im u].
    """
    n = kernel_cols.shape[0]
    kdim = kernel_cols.shape[1]
    order = np.lexsort((-lam.imag, -np.abs(lam)))  # |lambda| descending, +imag first in a pair
    lam = lam[order]
    budget = min(max(nev - kdim, 0), len(lam))
    if tau is not None and tau > 0:
        budget = min(budget, int(np.sum(np.abs(lam) > 1.0 / tau)))
    take = budget
    if 0 < take < len(lam) and abs(lam[take - 1].imag) > 0:
        # include the conjugate partner if it was cut off
        partner = np.conj(lam[take - 1])
        if not np.any(np.isclose(lam[:take], partner, rtol=1e-12, atol=0)):
            take += 1
    cols = [kernel_cols]
    done = set()
    for j in range(take):
        if j in done:
            continue
        u = vector(order[j])
        if abs(lam[j].imag) > 0:
            # find the partner within the taken set and mark it
            for k in range(j + 1, take):
                if k not in done and np.isclose(lam[k], np.conj(lam[j]), rtol=1e-10, atol=0):
                    done.add(k)
                    break
            cols.append(np.stack([u.real, u.imag], axis=1))
        else:
            cols.append(u.real[:, None])
    Z = np.concatenate(cols, axis=1) if cols else np.zeros((n, 0))
    return LocalEigen(Z=Z, kernel_dim=kdim, eigvals=lam, selected=lam[:take], dimK=dimK)


def orthonormal_columns(W: np.ndarray, drop: float = 1e-12) -> np.ndarray:
    """Orthonormal basis of range(W) by column-pivoted QR.

    Columns whose |R_jj| falls below drop * max |R_jj| are dropped.
    """
    if W.shape[1] == 0:
        return W
    Q, R, _ = sla.qr(W, mode="economic", pivoting=True)
    dg = np.abs(np.diag(R))
    if dg.size == 0 or dg[0] == 0.0:
        return W[:, :0]
    keep = dg > drop * dg[0]
    return Q[:, keep]


@dataclass
class CoarseSpace:
    """Columns of R_0^H = [R_1^T D_1 Z_1 ... R_N^T D_N Z_N] (Section 3.2)."""
    W: list                     # per subdomain W_i = orth(D_i Z_i), n_i x m_i
    Phi: sp.csr_matrix          # n x n_0, block columns R_i^T W_i
    E: np.ndarray               # A_00 = R_0 A R_0^H (dense)
    E_lu: tuple                 # LU with partial pivoting

    @property
    def n0(self) -> int:
        return self.Phi.shape[1]


def assemble_phi(subs: list, W: list, n: int) -> sp.csr_matrix:
    """R_0^H = [R_1^T W_1 ... R_N^T W_N] as a sparse n x n_0 matrix."""
    blocks = [restriction(s, n).T @ sp.csr_matrix(w) for s, w in zip(subs, W)]
    if not blocks:
        return sp.csr_matrix((n, 0))
    return sp.hstack(blocks).tocsr()


def coarse_space_from_W(A: sp.spmatrix, subs: list, W: list) -> CoarseSpace:
    """Coarse operator A_00 = R_0 A R_0^H and its exact LU (Eq. 2.2, Section 4)."""
    n = A.shape[0]
    Phi = assemble_phi(subs, W, n)
    E = (Phi.T @ (A @ Phi)).toarray() if Phi.shape[1] else np.zeros((0, 0))
    E_lu = sla.lu_factor(E) if E.shape[0] else None
    return CoarseSpace(W=W, Phi=Phi, E=E, E_lu=E_lu)


# ---------------------------------------------------------------------------
# Section 2: the preconditioners (Eqs. 2.1 - 2.4)
# ---------------------------------------------------------------------------

@dataclass
class Preconditioner:
    """Everything the apply of Eqs. 2.1 - 2.4 needs."""
    A: sp.csr_matrix
    subs: list
    D: list
    local_lu: list
    coarse: CoarseSpace | None
    eig: list = field(default_factory=list)
    Aii: list = field(default_factory=list)
    Atil: list = field(default_factory=list)

    @property
    def n(self) -> int:
        return self.A.shape[0]


def setup(A: sp.spmatrix, part: np.ndarray, delta: int, nev: int, pou: str = "boolean",
          tau: float | None = None, coarse: bool = True, keep_local: bool = False) -> Preconditioner:
    """Full setup: overlap, local matrices, block splitting, local LU, eigenproblems, coarse operator."""
    A = A.tocsr()
    n = A.shape[0]
    subs = overlapping_subdomains(A, part, delta)
    D = partition_of_unity(subs, n, pou)
    local_lu, eig, Aiis, Atils, W = [], [], [], [], []
    for s, d in zip(subs, D):
        Aii = local_matrix(A, s)
        local_lu.append(sla.lu_factor(Aii))
        if coarse:
            Atil = block_splitting(A, s)
            e = local_gevp(Aii, Atil, d, nev, tau)
            eig.append(e)
            W.append(orthonormal_columns(d[:, None] * e.Z))
            if keep_local:
                Atils.append(Atil)
        if keep_local:
            Aiis.append(Aii)
    cs = coarse_space_from_W(A, subs, W) if coarse else None
    return Preconditioner(A=A, subs=subs, D=D, local_lu=local_lu, coarse=cs, eig=eig,
                          Aii=Aiis, Atil=Atils)


def with_coarse_basis(P: Preconditioner, W: list) -> Preconditioner:
    """Same preconditioner with a given coarse basis W_i per subdomain."""
    return Preconditioner(A=P.A, subs=P.subs, D=P.D, local_lu=P.local_lu,
                          coarse=coarse_space_from_W(P.A, P.subs, W), eig=P.eig)


def apply_asm(P: Preconditioner, r: np.ndarray) -> np.ndarray:
    """M_ASM^{-1} r = sum_i R_i^T A_ii^{-1} R_i r (Eq. 2.1)."""
    z = np.zeros(P.n)
    for s, lu in zip(P.subs, P.local_lu):
        idx = s.idx
        z[idx] += sla.lu_solve(lu, r[idx])
    return z


def apply_ras(P: Preconditioner, r: np.ndarray) -> np.ndarray:
    """M_RAS^{-1} r = sum_i R_i^T D_i A_ii^{-1} R_i r (Eq. 2.3)."""
    z = np.zeros(P.n)
    for s, d, lu in zip(P.subs, P.D, P.local_lu):
        idx = s.idx
        z[idx] += d * sla.lu_solve(lu, r[idx])
    return z


def coarse_correction(P: Preconditioner, r: np.ndarray) -> np.ndarray:
    """R_0^H A_00^{-1} R_0 r (Eq. 2.2)."""
    cs = P.coarse
    if cs is None or cs.n0 == 0:
        return np.zeros(P.n)
    g = cs.Phi.T @ r
    c = sla.lu_solve(cs.E_lu, g)
    return cs.Phi @ c


def apply(P: Preconditioner, r: np.ndarray, variant: str = "deflated_ras") -> np.ndarray:
    """Apply one of the preconditioners of Section 2.

    deflated_ras (default, Eq. 2.4, used in all of the paper's experiments):
        R_0^H A_00^{-1} R_0 r + M_RAS^{-1} (r - A R_0^H A_00^{-1} R_0 r)
    deflated_asm: the same with M_ASM^{-1}
    additive_ras / additive_asm: R_0^H A_00^{-1} R_0 r + M_star^{-1} r (Eq. 2.2)
    ras / asm: one-level (Eqs. 2.3, 2.1).
    """
    r = np.asarray(r, dtype=np.float64)
    one = apply_ras if variant.endswith("ras") else apply_asm
    if variant in ("ras", "asm"):
        return one(P, r)
    q = coarse_correction(P, r)
    if variant.startswith("additive"):
        return q + one(P, r)
    if variant.startswith("deflated"):
        return q + one(P, r - P.A @ q)
    raise ValueError(variant)


def operator_matrix(P: Preconditioner, variant: str = "deflated_ras") -> np.ndarray:
    """Dense M^{-1} by applying the preconditioner to the identity (tiny cases only)."""
    n = P.n
    return np.stack([apply(P, np.eye(n)[:, j], variant) for j in range(n)], axis=1)


# ---------------------------------------------------------------------------
# Section 4: right-preconditioned restarted GMRES and flexible GMRES
# ---------------------------------------------------------------------------

@dataclass
class GmresResult:
    x: np.ndarray
    iters: int
    relres: float            # true ||b - A x|| / ||b||
    converged: bool
    history: list            # estimated relative residual after every inner step


def gmres(A, M, b: np.ndarray, rtol: float = 1e-8, restart: int = 30, max_it: int = 1000,
          flexible: bool = False, x0: np.ndarray | None = None) -> GmresResult:
    """Right-preconditioned GMRES(restart) (Section 4), optionally flexible.

    Arnoldi with modified Gram-Schmidt on A M^{-1}; Givens rotations keep
    the least-squares residual.  READING (the paper states only restart 30,
    rtol 1e-8 and x0 = 0): the inner loop stops when the estimated residual
    is at most rtol * ||b||; the iterate is then formed and the true residual
    checked; the outer loop restarts until the true relative residual is at
    most rtol.  The iteration count is the total number of inner steps.  A
    happy breakdown is declared when h_{j+1,j} <= 1e-14 * ||A M^{-1} v_j||.
    With ``flexible`` the vectors z_j = M^{-1} v_j are kept and x = x0 + Z y.
    """
    Aop = (lambda v: A @ v)
    Mop = M if callable(M) else (lambda v: v)
    n = len(b)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return GmresResult(np.zeros(n), 0, 0.0, True, [])
    history = []
    iters = 0
    while True:
        r = b - Aop(x)
        beta = np.linalg.norm(r)
        if beta <= rtol * bnorm:
            return GmresResult(x, iters, beta / bnorm, True, history)
        if iters >= max_it:
            return GmresResult(x, iters, beta / bnorm, False, history)
        V = np.zeros((n, restart + 1))
        Zs = np.zeros((n, restart)) if flexible else None
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[:, 0] = r / beta
        k = 0
        for j in range(restart):
            z = Mop(V[:, j])
            if flexible:
                Zs[:, j] = z
            w = Aop(z)
            wnorm = np.linalg.norm(w)
            for i in range(j + 1):
                H[i, j] = np.dot(V[:, i], w)
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            breakdown = H[j + 1, j] <= 1e-14 * wnorm
            if not breakdown:
                V[:, j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            k = j + 1
            history.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= rtol * bnorm or breakdown or iters >= max_it:
                break
        y = sla.solve_triangular(H[:k, :k], g[:k])
        if flexible:
            x = x + Zs[:, :k] @ y
        else:
            x = x + Mop(V[:, :k] @ y)
        res = np.linalg.norm(b - Aop(x)) / bnorm
        if res <= rtol:
            return GmresResult(x, iters, res, True, history)
        if iters >= max_it:
            return GmresResult(x, iters, res, False, history)


# ---------------------------------------------------------------------------
# Section 3.2: the condition-number bound
# ---------------------------------------------------------------------------

def coloring_number(subs: list) -> int:
    """k_c: colours of a greedy colouring of the subdomain overlap graph.

    Two subdomains are neighbours when their overlapping sets intersect.
    READING: the bound is monotone in k_c, so any valid colouring (greedy
    in subdomain order) gives a valid bound.
    """
    sets = [set(s.idx.tolist()) for s in subs]
    colour = []
    for i, si in enumerate(sets):
        used = {colour[j] for j in range(i) if sets[j] & si}
        c = 0
        while c in used:
            c += 1
        colour.append(c)
    return max(colour) + 1 if colour else 0


def multiplicity_number(subs: list, n: int) -> int:
    """k_m: the largest number of overlapping subdomains sharing a row of A."""
    count = np.zeros(n, dtype=np.int64)
    for s in subs:
        count[s.idx] += 1
    return int(count.max())


def condition_bound(subs: list, n: int, tau: float) -> float:
    """(k_c + 1) (2 + (2 k_c + 1) k_m / tau) (Section 3.2)."""
    kc = coloring_number(subs)
    km = multiplicity_number(subs, n)
    return (kc + 1) * (2.0 + (2 * kc + 1) * km / tau)
