"""Screened nuclear repulsion of the production potential (test infrastructure: the
oracle).  Sec. "Training details" adds a repulsive Ziegler-Biersack-Littmark (ZBL)
term to the potential and says nothing more; the readings taken here:

  * the universal ZBL pair energy
        E(r) = k_e Z_a Z_b / r * phi(r / a_s),   k_e = e^2 / (4 pi eps_0) = 14.399645 eV A,
        a_s  = 0.8854 a_0 / (Z_a^0.23 + Z_b^0.23),   a_0 = 0.529177 A,
        phi(x) = 0.18175 e^(-3.19980 x) + 0.50986 e^(-0.94229 x)
               + 0.28022 e^(-0.40290 x) + 0.02817 e^(-0.20162 x)
    (the universal screening function of Ziegler, Biersack and Littmark, "The
    Stopping and Range of Ions in Solids", 1985), Z the atomic numbers;
  * cut off smoothly by the model's polynomial envelope u(r / r_c) with the
    edge's cutoff (the ordered pair's when the model has a cutoff table);
  * each ordered edge (i, j) carries half of the pair energy, added to atom i's
    energy after the per-species scale and shift (a physical energy in eV, not
    a learned one).
"""
from __future__ import annotations

import torch

KE = 14.399645          # e^2 / (4 pi eps_0) in eV A
A0 = 0.529177           # Bohr radius in A
PHI_C = (0.18175, 0.50986, 0.28022, 0.02817)
PHI_D = (3.19980, 0.94229, 0.40290, 0.20162)


def screening(x: torch.Tensor) -> torch.Tensor:
    """The universal screening function phi(x)."""
    out = torch.zeros_like(x)
    for c, d in zip(PHI_C, PHI_D):
        out = out + c * torch.exp(-d * x)
    return out


def pair_energy(r: torch.Tensor, za: torch.Tensor, zb: torch.Tensor) -> torch.Tensor:
    """Unscreened-Coulomb-times-screening ZBL energy of pairs at distance r (eV)."""
    za = za.to(r.dtype)
    zb = zb.to(r.dtype)
    a_s = 0.8854 * A0 / (za ** 0.23 + zb ** 0.23)
    return KE * za * zb / r * screening(r / a_s)


def edge_energies(r: torch.Tensor, u: torch.Tensor, z_of_species, species, i, j) -> torch.Tensor:
    """Half the enveloped ZBL pair energy per ordered edge (i, j)."""
    z = torch.as_tensor(z_of_species, dtype=torch.int64)
    s = torch.as_tensor(species, dtype=torch.int64)
    zi = z[s[torch.as_tensor(i)]]
    zj = z[s[torch.as_tensor(j)]]
    return 0.5 * pair_energy(r, zi, zj) * u

