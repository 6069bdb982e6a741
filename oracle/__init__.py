"""FP64 CPU oracle (test infrastructure only; never called by the CUDA library).

Pinned functions (see tests/test_oracle_pins.py): fd_weights, lap1d, eig1d,
kernel_f, apply_fL, dense_fL, vx_apply, exchange_energy, energy_gradient, ace, ace_apply.
"""
from .kron_oracle import (DIRICHLET, PERIODIC, UNSCREENED, SCREENED, Plan, fd_weights, lap1d, eig1d,
                          kernel_f, apply_fL, forward_transform, inverse_transform, fdiag_matrix,
                          dense_L, dense_fL, pair_list, vx_apply, exchange_energy, energy_gradient, ace, ace_apply)

__all__ = ["DIRICHLET", "PERIODIC", "UNSCREENED", "SCREENED", "Plan", "fd_weights", "lap1d", "eig1d",
           "kernel_f", "apply_fL", "forward_transform", "inverse_transform", "fdiag_matrix", "dense_L",
           "dense_fL", "pair_list", "vx_apply", "exchange_energy", "energy_gradient", "ace", "ace_apply"]
