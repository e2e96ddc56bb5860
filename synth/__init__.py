"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This package holds input generators only: atom positions, species, cells and
the seeded weights file of an Allegro model of a stated architecture.  It holds
none of the model's arithmetic (no basis, no harmonics, no tensor products, no
network evaluation), so the oracle and the CUDA path share no computation.
Random numbers come from numpy's PCG64 (`numpy.random.default_rng`).
"""
from .structures import (
    Structure,
    random_box,
    lattice_box,
    molecule_batch,
    SPECIES_NAMES,
    SPECIES_MASSES,
    SPECIES_Z,
    WATER_MIX,
    paper_pair_cutoffs,
)
from .weights import Arch, make_weights, weights_to_blob, blob_to_weights, ARCHS
from .configs import CONFIGS, make_config

__all__ = [
    "Structure",
    "random_box",
    "lattice_box",
    "molecule_batch",
    "SPECIES_NAMES",
    "SPECIES_MASSES",
    "WATER_MIX",
    "Arch",
    "make_weights",
    "weights_to_blob",
    "blob_to_weights",
    "ARCHS",
    "CONFIGS",
    "make_config",
]
