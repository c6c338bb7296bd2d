"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This package only draws random numbers and lays them out as block-sparse (BSR)
arrays; it contains none of the solver's arithmetic.
"""
from .jacobian import (BSRMatrix, box_jacobian, grid_small, grid_spe10, perturb_values,
                       newton_sequence, random_rhs, poisson3d_bsr, chain_bsr, diagonal_bsr)

__all__ = ["BSRMatrix", "box_jacobian", "grid_small", "grid_spe10", "perturb_values",
           "newton_sequence", "random_rhs", "poisson3d_bsr", "chain_bsr", "diagonal_bsr"]
