"""The Allegro model in float64 on the CPU (torch), forces and virial by autograd.

Follows Sec. "Allegro" (energy decomposition, Eq. 1), Sec. "Optimized tensor
product" (paths, fused path weights, scalar-only last layer), Sec.
"Mixed-precision calculations" (float64 final stage) and "Training details"
(8 Bessel functions, polynomial envelope, SiLU MLPs, linear embedding, linear
edge-energy MLP).  Every step is written as its plain definition; the only
library primitives are matmul, einsum and index_add.

Readings where the paper defers to the Allegro paper or is silent:
  * Bessel basis  B_n(r) = sqrt(2/r_c) sin(n pi r / r_c) / r, n = 1..n_bessel,
    frequencies fixed (not trained), shared by all species pairs.
  * Envelope  u(x) = 1 - (p+1)(p+2)/2 x^p + p(p+2) x^(p+1) - p(p+1)/2 x^(p+2),
    x = r / r_c, p = 6 (u(1) = u'(1) = u''(1) = 0).
  * Two-body input  [onehot(Z_i) | onehot(Z_j) | B(r_ij)];  x^0 = u * MLP_2(input).
  * MLPs have no biases; SiLU after every layer of the two-body and latent
    MLPs; embedding, env-weight and edge-energy maps are linear.
  * Embedding  w^0 = Lin_emb(x^0) in R^{C x (lmax+1)},  V^0_{u,lm} = w^0_{u,l} Y_lm.
  * Layer L:  w^L = Lin_env^L(x^{L-1});  Gamma^L_{i,u,lm} = nu sum_{k in N(i)} w^L_{ik,u,l} Y_lm(r_ik),
    nu = 1/sqrt(avg_num_neighbors);  V^L = sum_{a,b} W^L[a,b,c] V^{L-1}_a Gamma^L_{i,b}
    (channel-wise, the u index is shared);  x^L = u * MLP_L([x^{L-1} | V^L_{0e}]).
    No residual in the scalar track.
  * Edge energy  E_ij = MLP_E(x^{L_max});  E_i = sum_j E_ij;
    Etilde_i = sigma_{Z_i} E_i + mu_{Z_i};  E = sum_i Etilde_i  (float64).
  * Virial  W_ab = - sum_e d_{e,a} dE/dd_{e,b}.
  * Per-ordered-species-pair cutoffs (Sec. "Species-dependent cutoffs", values in
    "Training details"), when the architecture carries a table: edge (i, j) takes
    r_c = pair_rc[Z_i][Z_j] (row = centre species) in the neighbour rule, the
    Bessel basis and the envelope alike, so each pair's basis spans its own range
    and its terms vanish smoothly at its own cutoff.
  * ZBL repulsion (when the architecture lists atomic numbers): `oracle/zbl.py`.
"""
from __future__ import annotations

import math
from typing import Dict, Optional

import numpy as np
import torch

from . import so3, zbl

torch_f64 = torch.float64


def bessel(r: torch.Tensor, r_c: float, n: int) -> torch.Tensor:
    k = torch.arange(1, n + 1, dtype=r.dtype)
    return math.sqrt(2.0 / r_c) * torch.sin(k * math.pi * r[..., None] / r_c) / r[..., None]


def bessel_pair(r: torch.Tensor, r_c: torch.Tensor, n: int) -> torch.Tensor:
    """The Bessel basis with a per-edge cutoff r_c [E] (same formula as `bessel`)."""
    k = torch.arange(1, n + 1, dtype=r.dtype)
    rc = r_c[..., None]
    return torch.sqrt(2.0 / rc) * torch.sin(k * math.pi * r[..., None] / rc) / r[..., None]


def envelope(x: torch.Tensor, p: int) -> torch.Tensor:
    c0 = (p + 1.0) * (p + 2.0) / 2.0
    c1 = p * (p + 2.0)
    c2 = p * (p + 1.0) / 2.0
    u = 1.0 - c0 * x ** p + c1 * x ** (p + 1) - c2 * x ** (p + 2)
    return torch.where(x < 1.0, u, torch.zeros_like(u))


def silu(x: torch.Tensor) -> torch.Tensor:
    return x * torch.sigmoid(x)


class AllegroOracle:
    """FP64 Allegro.  `arch`, `weights` as produced by synth.weights."""

    def __init__(self, arch, weights: Dict[str, np.ndarray]):
        self.arch = arch
        t = lambda a: torch.tensor(np.asarray(a, dtype=np.float64))
        self.two_body = [t(weights[f"two_body.{k}"]) for k in range(len(arch.two_body))]
        self.embed = t(weights["embed"])
        self.env = [t(weights[f"env.{L}"]) for L in range(1, arch.n_layers + 1)]
        self.latent = [[t(weights[f"latent.{L}.{k}"]) for k in range(len(arch.latent))]
                       for L in range(1, arch.n_layers + 1)]
        self.edge = [t(weights[f"edge.{k}"]) for k in range(len(arch.edge) + 1)]
        self.sigma = t(weights["sigma"])
        self.mu = t(weights["mu"])
        self.irreps = so3.layer_irreps(arch.lmax, arch.n_layers)
        self.W = []
        for L in range(1, arch.n_layers + 1):
            W = so3.fused_path_tensor(weights[f"tp.{L}"], self.irreps[L - 1], self.irreps[L], arch.lmax)
            self.W.append(torch.tensor(W))
        self.nu = 1.0 / math.sqrt(arch.avg_num_neighbors)
        # l of each spherical-harmonic component, and of each V^0 component
        self.l_of_sh = torch.tensor([l for l in range(arch.lmax + 1) for _ in range(2 * l + 1)])

    # ------------------------------------------------------------------
    def edge_vectors(self, pos, cell, i, j, S):
        """d_e = (pos_j + off(S)) - pos_i, off = (S0 a + S1 b) + S2 c (same order as the neighbour rule)."""
        cell_t = torch.zeros(3, 3, dtype=torch_f64) if cell is None else torch.as_tensor(cell, dtype=torch_f64)
        S = torch.as_tensor(S, dtype=torch_f64)
        off = (S[:, 0:1] * cell_t[0] + S[:, 1:2] * cell_t[1]) + S[:, 2:3] * cell_t[2]
        return (pos[j] + off) - pos[i]

    def edge_energies(self, d, species, i, j, n_atoms, features=None):
        """Per-edge energies E_ij [E] from edge vectors d [E,3] (rows of each centre must be complete).

        If `features` is a dict, the intermediate x^L, w^L, Gamma^L and V^L are stored in it."""
        a = self.arch
        r = torch.sqrt((d * d).sum(-1))
        rhat = d / r[:, None]
        Z = torch.as_tensor(np.asarray(species), dtype=torch.int64)
        B, u = self._radial(r, Z, i, j)
        u = u[:, None]
        Y = so3.real_sh(a.lmax, rhat)                                    # [E, S]
        Zi = torch.nn.functional.one_hot(Z[torch.as_tensor(i)], a.n_species).to(torch_f64)
        Zj = torch.nn.functional.one_hot(Z[torch.as_tensor(j)], a.n_species).to(torch_f64)
        h = torch.cat([Zi, Zj, B], dim=1)
        for Wk in self.two_body:
            h = silu(self.linear(h, Wk))
        x = u * h                                                        # x^0
        C, lm = a.channels, a.lmax + 1
        w0 = self.linear(x, self.embed).view(-1, C, lm)
        V = w0[:, :, self.l_of_sh] * Y[:, None, :]                      # V^0 [E, C, S]
        i_t = torch.as_tensor(i)
        if features is not None:
            features.update(Y=Y, u=u, B=B, x0=x, w0=w0, V0=V)
        for L in range(1, a.n_layers + 1):
            wL = self.linear(x, self.env[L - 1]).view(-1, C, lm)
            contrib = wL[:, :, self.l_of_sh] * Y[:, None, :]
            Gam = torch.zeros(n_atoms, C, Y.shape[1], dtype=torch_f64).index_add_(0, i_t, contrib) * self.nu
            V = torch.einsum("eua,eub,abc->euc", V, Gam[i_t], self.W[L - 1])
            s = V[:, :, 0]                                               # the 0e component comes first
            h = torch.cat([x, s], dim=1)
            for Wk in self.latent[L - 1]:
                h = silu(self.linear(h, Wk))
            x = u * h
            if features is not None:
                features.update({f"w{L}": wL, f"Gamma{L}": Gam, f"V{L}": V, f"x{L}": x})
        e = x
        for Wk in self.edge:
            e = self.linear(e, Wk)
        return e[:, 0]

    def linear(self, x, W):
        """The bias-free linear layer x W^T of every MLP (one place, so a test can
        substitute a reduced-precision product)."""
        return x @ W.T

    def _radial(self, r, Z, i, j):
        """Bessel basis [E, n_bessel] and envelope [E] with each edge's cutoff."""
        a = self.arch
        if a.pair_rc is None:
            return bessel(r, a.r_c, a.n_bessel), envelope(r / a.r_c, a.p_env)
        rc = torch.tensor(a.pair_rc, dtype=torch_f64)[Z[torch.as_tensor(i)], Z[torch.as_tensor(j)]]
        return bessel_pair(r, rc, a.n_bessel), envelope(r / rc, a.p_env)

    def repulsion(self, d, species, i, j, n_atoms):
        """Per-atom ZBL energies [n] (zeros without atomic numbers in the architecture)."""
        if self.arch.zbl_z is None or len(i) == 0:
            return torch.zeros(n_atoms, dtype=torch_f64)
        r = torch.sqrt((d * d).sum(-1))
        Z = torch.as_tensor(np.asarray(species), dtype=torch.int64)
        _, u = self._radial(r, Z, i, j)
        ez = zbl.edge_energies(r, u, self.arch.zbl_z, species, i, j)
        return torch.zeros(n_atoms, dtype=torch_f64).index_add_(0, torch.as_tensor(i), ez)

    def energy(self, pos, species, cell, i, j, S, n_atoms=None):
        """Total energy and per-atom energies (float64)."""
        n = pos.shape[0] if n_atoms is None else n_atoms
        d = self.edge_vectors(pos, cell, i, j, S)
        Eij = self.edge_energies(d, species, i, j, n)
        Ei = torch.zeros(n, dtype=torch_f64).index_add_(0, torch.as_tensor(i), Eij)
        Z = torch.as_tensor(np.asarray(species), dtype=torch.int64)
        Et = self.sigma[Z] * Ei + self.mu[Z] + self.repulsion(d, species, i, j, n)
        return Et.sum(), Et

    def energy_forces(self, pos_np, species, cell, i, j, S, chunk_atoms: int = 2048,
                      centers: Optional[np.ndarray] = None):
        """E (sum over `centers`' atomic energies, all atoms by default), E_atom, F, virial.

        Works on chunks of centre atoms: each centre's energy depends only on
        its own row of edges (strict locality), so E and its gradient are sums
        of per-chunk terms.
        """
        pos_np = np.asarray(pos_np, dtype=np.float64)
        n = pos_np.shape[0]
        species = np.asarray(species)
        i = np.asarray(i); j = np.asarray(j); S = np.asarray(S)
        centers = np.arange(n) if centers is None else np.asarray(centers)
        F = np.zeros((n, 3)); Wv = np.zeros((3, 3)); E_atom = np.zeros(n); E_tot = 0.0
        row_start = np.searchsorted(i, np.arange(n + 1))
        Z = torch.as_tensor(species, dtype=torch.int64)
        for c0 in range(0, centers.size, chunk_atoms):
            cs = centers[c0:c0 + chunk_atoms]
            sel = np.concatenate([np.arange(row_start[c], row_start[c + 1]) for c in cs]) if cs.size else np.zeros(0, int)
            sel = sel.astype(np.int64)
            pos = torch.tensor(pos_np, requires_grad=True)
            d = self.edge_vectors(pos, cell, i[sel], j[sel], S[sel])
            if sel.size:
                Eij = self.edge_energies(d, species, i[sel], j[sel], n)
                Ei = torch.zeros(n, dtype=torch_f64).index_add_(0, torch.as_tensor(i[sel]), Eij)
                Er = self.repulsion(d, species, i[sel], j[sel], n)
            else:
                Ei = torch.zeros(n, dtype=torch_f64)
                Er = torch.zeros(n, dtype=torch_f64)
            cs_t = torch.as_tensor(cs)
            Et = self.sigma[Z[cs_t]] * Ei[cs_t] + self.mu[Z[cs_t]] + Er[cs_t]
            Ec = Et.sum()
            if sel.size:
                gpos, gd = torch.autograd.grad(Ec, [pos, d], allow_unused=True)
                F -= gpos.numpy()
                Wv -= (d.detach().numpy().T @ gd.numpy())
            E_atom[cs] = Et.detach().numpy()
            E_tot += float(Ec.detach())
        return E_tot, E_atom, F, Wv
