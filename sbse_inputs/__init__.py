"""Seeded synthetic model systems: the inputs shared by the FP64 oracle and the CUDA path.

This package builds the single-particle problem the method starts from (a closed-shell system of
2*N_occ electrons with real orbitals phi_s and eigenvalues eps_s of a zero-order Hamiltonian H0,
Sec. II, first paragraph of "Method"). It holds none of the method's own arithmetic (no
propagation, screening, contraction or exciton solve): in the paper the orbitals come from a DFT
code, here they come from diagonalising a Gaussian-well Hamiltonian on a periodic grid.
"""
from .model_system import (  # noqa: F401
    ModelSystem,
    PRESETS,
    batch_presets,
    box_sweep_presets,
    fno_presets,
    dense_eigensystem,
    gaussian_wells,
    local_potential,
    make_system,
    preset,
)
