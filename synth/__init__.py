"""Seeded synthetic input generators shared by the oracle and the GPU path (no solver arithmetic)."""
from .kron import (CSR, KronFactors, assemble, batch_matrices, build, csr_from_dense, csr_from_scipy,
                   family_g, family_matrix, gaussian_block, kron_config, kron_factors, kron_matrix, named_factors,
                   laplacian_1d, laplacian_2d, learned_family, random_sparse_symmetric)
