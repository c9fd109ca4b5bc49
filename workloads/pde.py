"""Synthetic PDE-shaped sparse matrices, partitions and right-hand sides.

All randomness comes from ``numpy.random.Generator(PCG64(seed))``:
structure (channels, region seeds and targets) from ``PCG64(seed + 100000)``
and right-hand sides from ``PCG64(seed)``.  Matrices are returned as
``scipy.sparse.csr_matrix`` with sorted int32 column indices and float64
values; partitions are int32 vectors with values ``0..N-1``.

The paper's own test problem is a SUPG-stabilised finite-element
convection-diffusion equation on FreeFEM meshes (Section 4, Eq. 4.1), which
cannot be rebuilt here; the finite-difference / finite-volume operators below
are members of the same PDE family (convection-diffusion and high-contrast
diffusion) on structured grids and stand in for those meshes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class Problem:
    """A sparse system together with the decomposition parameters."""
    name: str
    A: sp.csr_matrix
    part: np.ndarray
    overlap: int
    nev: int
    b: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.A.shape[0]

    @property
    def nparts(self) -> int:
        return int(self.part.max()) + 1


def _finish(rows, cols, vals, n) -> sp.csr_matrix:
    A = sp.coo_matrix((np.asarray(vals, dtype=np.float64),
                       (np.asarray(rows, dtype=np.int64), np.asarray(cols, dtype=np.int64))),
                      shape=(n, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    A.indptr = A.indptr.astype(np.int32)
    A.indices = A.indices.astype(np.int32)
    return A


def conv_diff_2d(m: int, beta: float, theta: float) -> sp.csr_matrix:
    """-Laplace(u) + b.grad(u) on the m x m interior grid of the unit square.

    h = 1/(m+1), node (i, j) -> k = j*m + i, b = beta*(cos theta, sin theta).
    The 5-point stencil is multiplied by h^2; convection is first-order
    upwind (h*|b_x| added to the diagonal and subtracted from the upwind
    neighbour).  Dirichlet boundary: off-grid neighbours are dropped.
    """
    h = 1.0 / (m + 1)
    bx, by = beta * math.cos(theta), beta * math.sin(theta)
    rows, cols, vals = [], [], []
    diag = 4.0 + h * (abs(bx) + abs(by))
    west = -1.0 - (h * bx if bx > 0 else 0.0)
    east = -1.0 - (h * -bx if bx < 0 else 0.0)
    south = -1.0 - (h * by if by > 0 else 0.0)
    north = -1.0 - (h * -by if by < 0 else 0.0)
    for j in range(m):
        for i in range(m):
            k = j * m + i
            rows.append(k); cols.append(k); vals.append(diag)
            if i > 0:
                rows.append(k); cols.append(k - 1); vals.append(west)
            if i < m - 1:
                rows.append(k); cols.append(k + 1); vals.append(east)
            if j > 0:
                rows.append(k); cols.append(k - m); vals.append(south)
            if j < m - 1:
                rows.append(k); cols.append(k + m); vals.append(north)
    return _finish(rows, cols, vals, m * m)


def _channel_rows(m: int, width: int, fraction: float, rng: np.random.Generator) -> list:
    """Start rows of non-overlapping horizontal channels, drawn by rejection."""
    count = math.ceil(fraction * m / width)
    starts: list = []
    tries = 0
    while len(starts) < count:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place channels")
        s = int(rng.integers(0, m - width + 1))
        if all(s + width <= t or t + width <= s for t in starts):
            starts.append(s)
    return sorted(starts)


def high_contrast_fv_2d(m: int, seed: int, width: int = 4, fraction: float = 0.1,
                        contrast: float = 1e6) -> tuple:
    """Cell-centred finite-volume diffusion -div(kappa grad u) on an m x m grid.

    kappa = 1, except on ceil(fraction*m/width) horizontal channels of
    ``width`` rows where kappa = ``contrast``.  The face transmissibility is
    the harmonic mean 2*ka*kb/(ka+kb); a Dirichlet boundary face contributes
    2*kappa_cell to the diagonal.  Cell (i, j) -> k = j*m + i.  The matrix is
    symmetric positive definite and diagonally dominant.
    Returns (A, kappa) with kappa of shape (m, m) indexed [j, i].
    """
    rng = np.random.Generator(np.random.PCG64(seed + 100000))
    kappa = np.ones((m, m))
    for s in _channel_rows(m, width, fraction, rng):
        kappa[s:s + width, :] = contrast
    rows, cols, vals = [], [], []
    for j in range(m):
        for i in range(m):
            k = j * m + i
            kc = kappa[j, i]
            d = 0.0
            for (ii, jj) in ((i - 1, j), (i + 1, j), (i, j - 1), (i, j + 1)):
                if 0 <= ii < m and 0 <= jj < m:
                    kn = kappa[jj, ii]
                    t = 2.0 * kc * kn / (kc + kn)
                    rows.append(k); cols.append(jj * m + ii); vals.append(-t)
                    d += t
                else:
                    d += 2.0 * kc
            rows.append(k); cols.append(k); vals.append(d)
    return _finish(rows, cols, vals, m * m), kappa


def gaussian_random_field(m: int, std: float, corr_len: float, seed: int) -> np.ndarray:
    """Stationary Gaussian random field on the m x m cell centres of the unit square.

    Gaussian covariance std^2 exp(-|d|^2 / (2 corr_len^2)), synthesised spectrally: white noise
    filtered in Fourier space by the square root of the covariance's spectral density on a
    doubled periodic grid, then cropped and rescaled to the requested standard deviation.
    """
    rng = np.random.Generator(np.random.PCG64(seed + 100000))
    M = 2 * m
    k = np.fft.fftfreq(M, d=1.0 / M)  # integer wavenumbers on the doubled (period 2) domain
    kx, ky = np.meshgrid(k, k, indexing="ij")
    # spectral density of the Gaussian covariance (period 2): exp(-(pi l)^2 |k|^2 / 2) up to a constant
    spec = np.exp(-0.5 * (np.pi * corr_len) ** 2 * (kx ** 2 + ky ** 2))
    noise = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    field = np.real(np.fft.ifft2(np.sqrt(spec) * noise))[:m, :m]
    field = (field - field.mean()) / max(field.std(), 1e-300)
    return std * field


def fv_diffusion_2d(kappa: np.ndarray) -> sp.csr_matrix:
    """Cell-centred finite-volume -div(kappa grad u) on a square grid, kappa[j, i] per cell,
    harmonic-mean face transmissibilities, Dirichlet faces 2 kappa (cell k = j*m + i)."""
    m = kappa.shape[0]
    rows, cols, vals = [], [], []
    for j in range(m):
        for i in range(m):
            k = j * m + i
            kc = kappa[j, i]
            d = 0.0
            for (ii, jj) in ((i - 1, j), (i + 1, j), (i, j - 1), (i, j + 1)):
                if 0 <= ii < m and 0 <= jj < m:
                    kn = kappa[jj, ii]
                    t = 2.0 * kc * kn / (kc + kn)
                    rows.append(k); cols.append(jj * m + ii); vals.append(-t)
                    d += t
                else:
                    d += 2.0 * kc
            rows.append(k); cols.append(k); vals.append(d)
    return _finish(rows, cols, vals, m * m)


def config_c4(seed: int, m: int = 256, blocks: int = 8) -> Problem:
    """Log-normal diffusion kappa = exp(g), g a Gaussian random field (std 2, correlation length
    0.05), on an m x m grid; blocks x blocks subdomains, overlap 2, nev = 10."""
    kappa = np.exp(gaussian_random_field(m, 2.0, 0.05, seed))
    A = fv_diffusion_2d(kappa)
    return Problem(f"c4_lognormal_{m}_s{seed}", A, block_partition_2d(m, blocks), 2, 10,
                   rhs_uniform(m * m, seed), {"grid": m, "blocks": blocks, "seed": seed})


def config_c5(seed: int = 5, nsys: int = 48, side_min: int = 64, side_max: int = 256, nrhs: int = 4) -> list:
    """Mixed batch of independent 2D convection-diffusion systems: grid side uniform in
    [side_min, side_max], Peclet number |b| uniform in [1, 500], angle uniform in [0, 2 pi),
    nb = clamp(ceil(side / 48), 3, 16) blocks per direction, overlap 1, nev 8, nrhs right-hand sides
    U(-1, 1) each (stored as rows of meta["B"])."""
    rng = np.random.Generator(np.random.PCG64(seed + 100000))
    out = []
    for k in range(nsys):
        side = int(rng.integers(side_min, side_max + 1))
        pe = float(rng.uniform(1.0, 500.0))
        theta = float(rng.uniform(0.0, 2.0 * math.pi))
        nb = min(16, max(3, math.ceil(side / 48)))
        A = conv_diff_2d(side, pe, theta)
        B = np.stack([rhs_uniform(side * side, seed * 1000 + 10 * k + r) for r in range(nrhs)])
        out.append(Problem(f"c5_sys{k}_{side}", A, block_partition_2d(side, nb), 1, 8, B[0],
                           {"grid": side, "peclet": pe, "theta": theta, "blocks": nb, "B": B}))
    return out


def conv_diff_3d(m: int, beta: float) -> sp.csr_matrix:
    """-Laplace(u) + b.grad(u) on the m^3 interior grid of the unit cube.

    h = 1/(m+1), node (i, j, l) -> k = (l*m + j)*m + i, coordinates
    ((i+1)h, (j+1)h, (l+1)h), b = beta*(-y, x, 0.3).  7-point stencil times
    h^2 with first-order upwinding chosen per node by the sign of b.
    """
    h = 1.0 / (m + 1)
    rows, cols, vals = [], [], []
    for l in range(m):
        for j in range(m):
            for i in range(m):
                k = (l * m + j) * m + i
                x, y = (i + 1) * h, (j + 1) * h
                b = (beta * -y, beta * x, beta * 0.3)
                rows.append(k); cols.append(k); vals.append(6.0 + h * sum(abs(c) for c in b))
                for axis, (coord, stride) in enumerate(((i, 1), (j, m), (l, m * m))):
                    c = b[axis]
                    lo = -1.0 - (h * c if c > 0 else 0.0)
                    hi = -1.0 - (h * -c if c < 0 else 0.0)
                    if coord > 0:
                        rows.append(k); cols.append(k - stride); vals.append(lo)
                    if coord < m - 1:
                        rows.append(k); cols.append(k + stride); vals.append(hi)
    return _finish(rows, cols, vals, m ** 3)


def block_partition_2d(m: int, nb: int) -> np.ndarray:
    """nb x nb contiguous blocks of an m x m grid (node k = j*m + i)."""
    i = np.arange(m)
    bi = (i * nb) // m
    part = (bi[:, None] * nb + bi[None, :])  # [j, i]
    return part.reshape(-1).astype(np.int32)


def block_partition_3d(m: int, nb: int) -> np.ndarray:
    """nb^3 contiguous blocks of an m^3 grid (node k = (l*m + j)*m + i)."""
    c = (np.arange(m) * nb) // m
    part = (c[:, None, None] * nb + c[None, :, None]) * nb + c[None, None, :]
    return part.reshape(-1).astype(np.int32)


def bfs_region_partition(A: sp.csr_matrix, nparts: int, tmin: int, tmax: int, seed: int) -> np.ndarray:
    """Uneven connected regions grown by simultaneous breadth-first search.

    Targets are drawn uniformly in [tmin, tmax] and rescaled to sum to n;
    region seeds are distinct random nodes.  Regions grow one node at a time
    in round-robin order until their target is met or their frontier is
    exhausted.  Connected groups of nodes left unclaimed join the smallest
    adjacent region when that keeps it within tmax; a larger group is shared
    among the regions around it, which grow into it one node at a time, the
    smallest region first.
    """
    n = A.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed + 100000))
    t = rng.uniform(tmin, tmax, nparts)
    t = np.maximum(1, np.floor(t * n / t.sum())).astype(np.int64)
    t[-1] += n - t.sum()
    indptr, indices = A.indptr, A.indices
    part = -np.ones(n, dtype=np.int64)
    seeds = rng.choice(n, size=nparts, replace=False)
    from collections import deque
    queues = []
    size = np.zeros(nparts, dtype=np.int64)
    for r, s in enumerate(seeds):
        part[s] = r
        size[r] = 1
        queues.append(deque([int(s)]))
    active = True
    while active:
        active = False
        for r in range(nparts):
            q = queues[r]
            while q and size[r] < t[r]:
                v = q[0]
                claimed = False
                for k in indices[indptr[v]:indptr[v + 1]]:
                    if part[k] < 0:
                        part[k] = r
                        size[r] += 1
                        q.append(int(k))
                        claimed = True
                        break
                if claimed:
                    active = True
                    break
                q.popleft()
    # leftovers: connected components of unclaimed nodes join the smallest neighbour
    for v in range(n):
        if part[v] >= 0:
            continue
        comp = [v]
        part[v] = -2
        stack = [v]
        nbr_regions = set()
        while stack:
            u = stack.pop()
            for k in indices[indptr[u]:indptr[u + 1]]:
                if part[k] == -1:
                    part[k] = -2
                    comp.append(int(k))
                    stack.append(int(k))
                elif part[k] >= 0:
                    nbr_regions.add(int(part[k]))
        target = min(nbr_regions, key=lambda r: (size[r], r))
        if size[target] + len(comp) <= tmax:
            for u in comp:
                part[u] = target
            size[target] += len(comp)
            continue
        in_comp = set(comp)
        for u in comp:
            part[u] = -1
        fronts = {r: deque() for r in sorted(nbr_regions)}
        for u in comp:
            for k in indices[indptr[u]:indptr[u + 1]]:
                if part[k] >= 0:
                    fronts[int(part[k])].append(int(k))
        left = len(comp)
        while left:
            claimed = False
            for r in sorted(fronts, key=lambda r: (size[r], r)):
                q = fronts[r]
                while q and not claimed:
                    v = q[0]
                    for k in indices[indptr[v]:indptr[v + 1]]:
                        if part[k] == -1 and int(k) in in_comp:
                            part[k] = r
                            size[r] += 1
                            q.append(int(k))
                            left -= 1
                            claimed = True
                            break
                    if not claimed:
                        q.popleft()
                if claimed:
                    break
            if not claimed:
                raise RuntimeError("unclaimed nodes left in a connected group")
    return part.astype(np.int32)


def rhs_uniform(n: int, seed: int) -> np.ndarray:
    """Right-hand side with i.i.d. U(-1, 1) entries from PCG64(seed)."""
    return np.random.Generator(np.random.PCG64(seed)).uniform(-1.0, 1.0, n)


def config_c1() -> Problem:
    """2D convection-diffusion, 64x64 grid (n = 4096), b = 50(cos pi/6, sin pi/6),
    4x4 block subdomains, overlap 1, nev = 8, seed 1."""
    m = 64
    A = conv_diff_2d(m, 50.0, math.pi / 6)
    return Problem("c1_convdiff2d_64", A, block_partition_2d(m, 4), 1, 8, rhs_uniform(m * m, 1),
                   {"grid": m, "blocks": 4, "seed": 1})


def config_c2() -> Problem:
    """High-contrast FV diffusion, 512x512 grid (n = 262144), 13 channels of
    4 rows at kappa = 1e6, 16x16 block subdomains, overlap 2, nev = 16, seed 2."""
    m = 512
    A, _ = high_contrast_fv_2d(m, seed=2)
    return Problem("c2_highcontrast2d_512", A, block_partition_2d(m, 16), 2, 16, rhs_uniform(m * m, 2),
                   {"grid": m, "blocks": 16, "seed": 2})


def config_c3(m: int = 96, nparts: int = 512, tmin: int = 800, tmax: int = 3000, seed: int = 3) -> Problem:
    """3D convection-diffusion on an m^3 grid with b = 100(-y, x, 0.3), uneven
    BFS-grown regions, overlap 1, nev = 12."""
    A = conv_diff_3d(m, 100.0)
    part = bfs_region_partition(A, nparts, tmin, tmax, seed)
    return Problem(f"c3_convdiff3d_{m}", A, part, 1, 12, rhs_uniform(m ** 3, seed),
                   {"grid": m, "nparts": nparts, "seed": seed})


def tiny_conv_diff(m: int = 12, nb: int = 2, overlap: int = 1, nev: int = 4,
                   beta: float = 50.0, theta: float = math.pi / 6, seed: int = 11) -> Problem:
    """Small 2D convection-diffusion case for fast oracle and parity tests."""
    A = conv_diff_2d(m, beta, theta)
    return Problem(f"tiny_convdiff2d_{m}", A, block_partition_2d(m, nb), overlap, nev,
                   rhs_uniform(m * m, seed), {"grid": m, "blocks": nb, "seed": seed})


def tiny_hpd_dd(m: int = 8, nb: int = 2, overlap: int = 1, nev: int = 4, seed: int = 12,
                contrast: float = 1e3) -> Problem:
    """Small high-contrast FV diffusion (HPD, diagonally dominant)."""
    rng = np.random.Generator(np.random.PCG64(seed + 100000))
    kappa = np.exp(rng.uniform(0.0, math.log(contrast), (m, m)))
    rows, cols, vals = [], [], []
    for j in range(m):
        for i in range(m):
            k = j * m + i
            kc = kappa[j, i]
            d = 0.0
            for (ii, jj) in ((i - 1, j), (i + 1, j), (i, j - 1), (i, j + 1)):
                if 0 <= ii < m and 0 <= jj < m:
                    kn = kappa[jj, ii]
                    tt = 2.0 * kc * kn / (kc + kn)
                    rows.append(k); cols.append(jj * m + ii); vals.append(-tt)
                    d += tt
                else:
                    d += 2.0 * kc
            rows.append(k); cols.append(k); vals.append(d)
    A = _finish(rows, cols, vals, m * m)
    return Problem(f"tiny_hpd_dd_{m}", A, block_partition_2d(m, nb), overlap, nev,
                   rhs_uniform(m * m, seed), {"grid": m, "blocks": nb, "seed": seed})


def random_dd_matrix(n: int, density: float, seed: int, symmetric: bool = True,
                     strict: float = 0.0) -> sp.csr_matrix:
    """Random sparse diagonally dominant matrix with a symmetric pattern.

    Off-diagonal values are drawn from N(0, 1) (both signs, so not an
    M-matrix); the diagonal equals the absolute row sum times (1 + strict),
    plus a tiny positive amount.  With ``symmetric`` the values are
    symmetric, giving a Hermitian positive (semi-)definite matrix.
    """
    rng = np.random.Generator(np.random.PCG64(seed + 100000))
    M = sp.random(n, n, density=density, random_state=rng, data_rvs=rng.standard_normal).tocsr()
    M = M - sp.diags(M.diagonal())
    if symmetric:
        M = (M + M.T) * 0.5
    else:
        P = (abs(M) + abs(M.T)) > 0
        M = M + 0.0 * P  # keep the pattern symmetric
        R = sp.random(n, n, density=1.0, random_state=rng, data_rvs=rng.standard_normal).multiply(P)
        M = (M + 0.5 * R).tocsr()
        M = M - sp.diags(M.diagonal())
    rowsum = np.asarray(abs(M).sum(axis=1)).ravel()
    A = M + sp.diags(rowsum * (1.0 + strict) + 1e-3)
    A = A.tocoo()
    return _finish(A.row, A.col, A.data, n)
