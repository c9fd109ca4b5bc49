"""The synthetic inputs have the structure their recipes state (no method arithmetic here)."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

from workloads import pde


def test_c3_regions_are_connected_and_within_the_size_range():
    """96^3 convection-diffusion, 512 BFS-grown regions with targets in [800, 3000]: every node is
    assigned, every region is connected, none exceeds 3000 nodes (enclosed pockets of unclaimed
    nodes are shared among the regions around them), and the regions cut short by their
    neighbours stay near the lower end."""
    prob = pde.config_c3()
    part = prob.part
    n = prob.A.shape[0]
    assert part.shape == (n,) and part.min() == 0 and part.max() == 511
    sizes = np.bincount(part, minlength=512)
    assert sizes.max() <= 3000 and sizes.min() >= 700, (sizes.min(), sizes.max())
    P = sp.csr_matrix(prob.A)
    order = np.argsort(part, kind="stable")
    starts = np.concatenate([[0], np.cumsum(sizes)])
    for r in range(512):
        nodes = order[starts[r]:starts[r + 1]]
        ncomp, _ = csg.connected_components(P[nodes][:, nodes], directed=False)
        assert ncomp == 1, r


def test_small_3d_partitions_are_connected_and_complete():
    """The small 3D partitions of the tests: every region is connected, non-empty, and the sizes
    add up to the grid."""
    for m, nparts, tmin, tmax, seed in ((7, 6, 30, 90, 5), (10, 8, 60, 180, 5), (12, 10, 60, 300, 11)):
        A = pde.conv_diff_3d(m, 100.0)
        part = pde.bfs_region_partition(A, nparts, tmin, tmax, seed)
        sizes = np.bincount(part, minlength=nparts)
        assert sizes.sum() == m ** 3 and sizes.min() > 0
        for r in range(nparts):
            nodes = np.flatnonzero(part == r)
            ncomp, _ = csg.connected_components(A[nodes][:, nodes], directed=False)
            assert ncomp == 1
