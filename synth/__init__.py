"""Seeded synthetic inputs for the reservoir linear-solve path.

This package produces inputs only: grids, permeability fields, the 3x3-block
Jacobian of a seven-point two-point-flux discretisation, and right-hand sides.
It holds none of the solver arithmetic and imports neither the CUDA package
nor the CPU oracle; both of those consume what it generates.
"""
from .reservoir import (  # noqa: F401
    Problem, make_problem, perm_lognormal, perm_layered, perm_channelized,
    assemble_jacobian, accumulation_blocks, seven_point_pattern, nnzb_of, uniform01, std_normal,
    WORKLOADS, workload, batch_sizes, unet_init,
)
