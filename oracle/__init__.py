"""FP64 CPU oracle (test infrastructure only; never called by the CUDA library).

Pinned functions (see tests/test_oracle_pins.py): fd_weights, lap1d, eig1d,
kernel_f, apply_fL, dense_fL, vx_apply, exchange_energy, energy_gradient, ace, ace_apply,
multipole_moments, multipole_potential, rhs_multipole, apply_fL_multipole, lap1d_bloch,
apply_fL_bloch, vx_apply_kpoint, vx_kpoints, exchange_energy_kpoints.
"""
from .kron_oracle import (DIRICHLET, PERIODIC, UNSCREENED, SCREENED, Plan, fd_weights, lap1d, eig1d,
                          kernel_f, apply_fL, forward_transform, inverse_transform, fdiag_matrix,
                          dense_L, dense_fL, pair_list, vx_apply, exchange_energy, energy_gradient, ace, ace_apply,
                          expansion_centre, interior_points, exterior_points, multipole_moments,
                          multipole_potential, rhs_multipole, apply_fL_multipole, lap1d_bloch, BlochPlan,
                          forward_transform_bloch, inverse_transform_bloch, apply_fL_bloch, vx_apply_kpoint,
                          vx_kpoints, exchange_energy_kpoints)

__all__ = ["DIRICHLET", "PERIODIC", "UNSCREENED", "SCREENED", "Plan", "fd_weights", "lap1d", "eig1d",
           "kernel_f", "apply_fL", "forward_transform", "inverse_transform", "fdiag_matrix", "dense_L",
           "dense_fL", "pair_list", "vx_apply", "exchange_energy", "energy_gradient", "ace", "ace_apply",
           "expansion_centre", "interior_points", "exterior_points", "multipole_moments", "multipole_potential",
           "rhs_multipole", "apply_fL_multipole", "lap1d_bloch", "BlochPlan", "forward_transform_bloch",
           "inverse_transform_bloch", "apply_fL_bloch", "vx_apply_kpoint", "vx_kpoints", "exchange_energy_kpoints"]
