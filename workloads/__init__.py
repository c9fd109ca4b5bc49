"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package only builds inputs: sparse matrices in CSR form, partition
vectors and right-hand sides.  It contains none of the preconditioner's
arithmetic (no overlap growth, no local matrices, no eigenproblems, no
solves), so that the oracle and the GPU path can both consume it without
sharing any of the method's code.
"""
from .pde import (Problem, conv_diff_2d, high_contrast_fv_2d, conv_diff_3d,
                  block_partition_2d, block_partition_3d, bfs_region_partition,
                  rhs_uniform, config_c1, config_c2, config_c3, tiny_conv_diff,
                  tiny_hpd_dd, random_dd_matrix, gaussian_random_field,
                  fv_diffusion_2d, config_c4, config_c5)

__all__ = ["Problem", "conv_diff_2d", "high_contrast_fv_2d", "conv_diff_3d",
           "block_partition_2d", "block_partition_3d", "bfs_region_partition",
           "rhs_uniform", "config_c1", "config_c2", "config_c3", "tiny_conv_diff",
           "tiny_hpd_dd", "random_dd_matrix", "gaussian_random_field", "fv_diffusion_2d", "config_c4", "config_c5"]
