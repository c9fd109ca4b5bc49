"""Pins for the oracle's overlap, restriction, partition of unity and block splitting.

Each test checks the oracle against something other than itself: a
hand-derived fixture, a library routine (networkx BFS), a closed-form count
or an invariant stated in the paper (Section 2, Definition 3.1, Lemma 3.2).
"""
import networkx as nx
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import a2ls_oracle as O
from workloads import pde
from tests.golden_util import load, frac_array


def _laplace1d(n):
    return sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()


def test_golden_overlap_and_splitting():
    g = load("laplace1d_n4.json")
    A = sp.csr_matrix(frac_array(g["A"]))
    part = np.array(g["part"], dtype=np.int32)
    subs = O.overlapping_subdomains(A, part, g["overlap"])
    for s, (interior, gamma) in zip(subs, g["omega"]):
        assert s.interior.tolist() == interior
        assert s.gamma.tolist() == gamma
    for s, sv, At in zip(subs, g["s"], g["Atilde"]):
        np.testing.assert_array_equal(O.lumped_row_sums(A, s), [float(x) for x in sv])
        np.testing.assert_array_equal(O.block_splitting(A, s), frac_array(At))


@pytest.mark.parametrize("delta", [0, 1, 2, 3])
@pytest.mark.parametrize("case", ["tiny_conv", "bfs3d", "random", "one_sided"])
def test_overlap_matches_networkx_bfs(case, delta):
    if case == "tiny_conv":
        P = pde.tiny_conv_diff(m=10, nb=3)
        A, part = P.A, P.part
    elif case == "bfs3d":
        A = pde.conv_diff_3d(7, 100.0)
        part = pde.bfs_region_partition(A, 6, 30, 90, seed=5)
    elif case == "random":
        A = pde.random_dd_matrix(80, 0.04, seed=3)
        part = (np.arange(80) * 5 // 80).astype(np.int32)
    else:
        # every coupling one-sided (upper triangle only): the graph is that of A + A^T, not of A
        A = sp.triu(pde.random_dd_matrix(80, 0.04, seed=3)).tocsr()
        part = (np.arange(80) * 5 // 80).astype(np.int32)
    G = nx.Graph()  # undirected: an entry a_ij gives the edge {i, j}, the pattern of A + A^T
    G.add_nodes_from(range(A.shape[0]))
    Acoo = A.tocoo()
    G.add_edges_from((int(i), int(j)) for i, j in zip(Acoo.row, Acoo.col) if i != j)
    subs = O.overlapping_subdomains(A, part, delta)
    for i, s in enumerate(subs):
        interior = np.flatnonzero(part == i)
        G2 = G.copy()
        G2.add_node("src")
        G2.add_edges_from(("src", int(v)) for v in interior)
        dist = nx.single_source_shortest_path_length(G2, "src", cutoff=delta + 1)
        # Omega_Gamma layer by layer (distance from the interior), ascending within a layer
        expect = sorted((v for v, d in dist.items() if v != "src" and 2 <= d <= delta + 1),
                        key=lambda v: (dist[v], v))
        assert s.interior.tolist() == interior.tolist()
        assert s.gamma.tolist() == expect


def test_c1_subdomain_sizes_closed_form():
    """4x4 blocks of 16x16 with one layer: corner 256+32, edge 256+48, inner 256+64."""
    P = pde.config_c1()
    subs = O.overlapping_subdomains(P.A, P.part, 1)
    sizes = sorted(s.n_i for s in subs)
    assert sizes == [288] * 4 + [304] * 8 + [320] * 4
    assert sum(sizes) == 4864
    assert P.A.nnz == 20224


@pytest.mark.parametrize("kind", ["boolean", "multiplicity"])
def test_partition_of_unity_sums_to_identity(kind):
    """sum_i R_i^T D_i R_i = I_n (Section 2)."""
    P = pde.tiny_conv_diff(m=11, nb=3, overlap=2)
    subs = O.overlapping_subdomains(P.A, P.part, 2)
    D = O.partition_of_unity(subs, P.n, kind)
    total = np.zeros(P.n)
    for s, d in zip(subs, D):
        assert np.all(d >= 0)
        total[s.idx] += d
    if kind == "boolean":
        np.testing.assert_array_equal(total, np.ones(P.n))
    else:
        np.testing.assert_allclose(total, 1.0, rtol=0, atol=1e-15)


def test_restriction_is_identity_rows():
    P = pde.tiny_conv_diff(m=8, nb=2)
    subs = O.overlapping_subdomains(P.A, P.part, 1)
    for s in subs:
        R = O.restriction(s, P.n).toarray()
        np.testing.assert_array_equal(R, np.eye(P.n)[s.idx])
        np.testing.assert_array_equal(O.local_matrix(P.A, s), R @ P.A.toarray() @ R.T)


@pytest.mark.parametrize("seed", range(6))
def test_lemma_3_2_hpsd_splitting(seed):
    """Lemma 3.2: for HPD diagonally dominant A, A~_i and A - A~_i are HPSD."""
    n = 60
    A = pde.random_dd_matrix(n, 0.06, seed=seed, symmetric=True)
    part = (np.arange(n) * 4 // n).astype(np.int32)
    subs = O.overlapping_subdomains(A, part, 1 + seed % 2)
    Ad = A.toarray()
    scale = np.linalg.norm(Ad, 2)
    for s in subs:
        At = O.global_splitting(A, s)
        assert np.min(np.linalg.eigvalsh(At)) >= -1e-12 * scale
        assert np.min(np.linalg.eigvalsh(Ad - At)) >= -1e-12 * scale
        # the diagonal of A~_i given in the proof of Lemma 3.2
        diag = np.zeros(n)
        diag[s.interior] = Ad[s.interior, s.interior]
        diag[s.gamma] = Ad[s.gamma, s.gamma] - O.lumped_row_sums(A, s)
        np.testing.assert_allclose(np.diag(At), diag, rtol=0, atol=1e-13 * scale)


def test_splitting_zero_row_sums_for_floating_subdomain():
    """With zero row sums and non-positive couplings, lumping keeps zero row sums."""
    P = pde.tiny_conv_diff(m=12, nb=3, overlap=1)
    subs = O.overlapping_subdomains(P.A, P.part, 1)
    inner = subs[4]  # the middle block of a 3x3 layout touches no boundary
    At = O.block_splitting(P.A, inner)
    np.testing.assert_allclose(At @ np.ones(inner.n_i), 0.0, atol=1e-13)
