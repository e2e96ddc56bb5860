"""The named workloads: structure recipe + architecture + seeds.

c1      64 atoms, uniform random (min separation 0.9 A), periodic cube 8.62 A,
        2 species at 43:21; 1 layer, l_max=1, 8 channels.  Structure seed 0,
        weight seed 0.
c2      23,552 atoms, jittered lattice, periodic cube 61.74 A, water/protein mix;
        2 layers, l_max=2, 64 channels.  Seeds 1 / 1.
c3      2048 gas-phase molecules of 8-64 atoms (random walk); c2 architecture.
        Seeds 2 / 1.
c4      1,048,576 atoms, jittered lattice, periodic cube 218.9 A; c2 architecture.
        Seeds 3 / 1.
c4sub   4,096 atoms, periodic cube 34.48 A (same density), generated like c4.
c5      4,194,304 atoms, periodic cube 347.4 A; 3 layers, l_max=3, 128 channels.
"""
from __future__ import annotations

from .structures import random_box, lattice_box, molecule_batch
from .weights import ARCHS, make_weights

CONFIGS = {
    "c1": dict(kind="random", n=64, L=8.62, seed=0, arch="c1", wseed=0),
    "c2": dict(kind="lattice", n=23552, L=61.74, seed=1, arch="c2", wseed=1),
    "c3": dict(kind="molecules", n_mol=2048, seed=2, arch="c2", wseed=1),
    "c4": dict(kind="lattice", n=1048576, L=218.9, seed=3, arch="c2", wseed=1),
    "c4sub": dict(kind="lattice", n=4096, L=34.48, seed=3, arch="c2", wseed=1),
    "c5": dict(kind="lattice", n=4194304, L=347.4, seed=4, arch="c5", wseed=1),
}


def make_structure(name: str, **over):
    c = dict(CONFIGS[name])
    c.update(over)
    if c["kind"] == "random":
        return random_box(c["n"], c["L"], c["seed"])
    if c["kind"] == "lattice":
        return lattice_box(c["n"], c["L"], c["seed"])
    if c["kind"] == "molecules":
        return molecule_batch(c["n_mol"], c["seed"])
    raise KeyError(name)


def make_config(name: str, **over):
    """Returns (structure or list of structures, arch, weights dict)."""
    c = dict(CONFIGS[name])
    c.update(over)
    arch = ARCHS[c["arch"]]
    return make_structure(name, **over), arch, make_weights(arch, c["wseed"])
