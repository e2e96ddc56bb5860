"""Velocity-Verlet integration in float64 (Sec. "Problem Overview": MD integrates
Newton's equations with femtosecond time steps).

Units: positions in Angstrom, velocities in Angstrom/fs, masses in amu, forces
in eV/Angstrom, energies in eV.  1 eV/(Angstrom amu) = 9.648533212e-3 Angstrom/fs^2.
"""
from __future__ import annotations

import numpy as np

ACC_CONV = 9.648533212e-3          # (eV/A/amu) -> A/fs^2


def kinetic_energy(vel, masses) -> float:
    return float(0.5 * (np.asarray(masses)[:, None] * vel * vel).sum() / ACC_CONV)


def verlet_step(pos, vel, forces, masses, dt, force_fn):
    """One step: v += dt/2 a; x += dt v; F = force_fn(x); v += dt/2 a.  Returns (pos, vel, F, E)."""
    m = np.asarray(masses, dtype=np.float64)[:, None]
    vel = vel + 0.5 * dt * ACC_CONV * forces / m
    pos = pos + dt * vel
    E, F = force_fn(pos)
    vel = vel + 0.5 * dt * ACC_CONV * F / m
    return pos, vel, F, E
