"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This package holds none of the solver's arithmetic: it only draws matrices and
right-hand sides with the shapes and spectra of the paper's workloads (random
dense matrices with geometric singular values, prolate Toeplitz matrices,
Section 3) and of the two extra workloads (a dense 2-D convection-diffusion
operator and a batch of dense systems of uneven size).
"""
from .generators import (  # noqa: F401
    sigma_geometric,
    randsvd,
    randsvd_torch,
    prolate,
    prolate_torch,
    convdiff,
    rhs_uniform,
    normal_vector,
    batch_specs,
)
