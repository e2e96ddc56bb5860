"""Seeded random weights of an Allegro model and their binary file format.

The paper's model is trained; no trained weights exist here, so every weight
is drawn from a seeded normal distribution: MLP matrices N(0, 1/fan_in) (bias
free), raw tensor-product path weights N(0, 1), per-species scale
sigma = 1 + 0.1 N(0,1) and shift mu = 10 N(0,1) eV.  Draw order is the order
of `weight_names(arch)`.

Architecture (Sec. "Allegro" and "Training details" of the paper): a two-body
MLP, a linear embedding, per layer an env-weight projection, a tensor-product
path-weight table and a latent MLP, then an edge-energy MLP.  Shapes are
[out, in] (row-major, `in` contiguous).

Binary format "ALGW" v1, little-endian:
    char[4] magic = "ALGW"; u32 version = 1
    f64 r_c; f64 avg_num_neighbors
    i32 n_species, n_bessel, p_env, lmax, n_layers, channels,
        n_two_body, n_latent, n_edge
    i32 two_body[n_two_body], latent[n_latent], edge[n_edge]
    then every array of `weight_names(arch)` in order, raw: f32 for matrices and
    path tables, f64 for sigma and mu.
"""
from __future__ import annotations

import struct
from dataclasses import dataclass, asdict
from typing import Dict, List, Optional, Tuple

import numpy as np

MAGIC = b"ALGW"
VERSION = 1


@dataclass(frozen=True)
class Arch:
    n_species: int
    lmax: int
    n_layers: int
    channels: int
    two_body: Tuple[int, ...]
    latent: Tuple[int, ...]
    edge: Tuple[int, ...]          # hidden widths of the edge-energy MLP; output width 1 is implied
    n_bessel: int = 8
    p_env: int = 6
    r_c: float = 4.0
    avg_num_neighbors: float = 27.0
    # cutoff per ordered (centre species, neighbour species) pair; None: r_c for every pair.
    # Not part of the weights blob (the float32 / BF16 library path takes one r_c).
    pair_rc: Optional[Tuple[Tuple[float, ...], ...]] = None
    # atomic number of each model species for the ZBL repulsion term; None: no ZBL term.
    # Not part of the weights blob (the library does not evaluate it yet).
    zbl_z: Optional[Tuple[int, ...]] = None

    @property
    def max_rc(self) -> float:
        """Largest cutoff of any ordered pair (the neighbour search radius)."""
        return max(max(row) for row in self.pair_rc) if self.pair_rc is not None else self.r_c

    @property
    def n_in_two_body(self) -> int:
        return 2 * self.n_species + self.n_bessel

    def latent_width(self, layer: int) -> int:
        """Width K_L of the scalar track after layer L (L = 0: two-body MLP)."""
        return self.two_body[-1] if layer == 0 else self.latent[-1]

    @property
    def n_w(self) -> int:
        """Width of the embedding / env-weight projections: channels x (lmax+1)."""
        return self.channels * (self.lmax + 1)


ARCHS: Dict[str, Arch] = {
    # 64-atom case: 1 layer, l_max=1, 8 channels, two-body [32], latent [32], edge 32->1
    "c1": Arch(n_species=2, lmax=1, n_layers=1, channels=8, two_body=(32,), latent=(32,), edge=()),
    # 23.5k / 1M-atom cases: 2 layers, l_max=2, 64 channels
    "c2": Arch(n_species=5, lmax=2, n_layers=2, channels=64, two_body=(64, 128, 256),
               latent=(256, 256), edge=(128,)),
    # the paper's production model (Sec. "Training details"): 2 layers of 64 tensor features,
    # l_max 2, two-body MLP [128, 256, 512, 1024], latent MLP [1024, 1024, 1024], edge MLP with
    # one hidden layer of 128, no nonlinearity; per-pair cutoffs and ZBL on the water/protein mix
    "paper": Arch(n_species=5, lmax=2, n_layers=2, channels=64, two_body=(128, 256, 512, 1024),
                  latent=(1024, 1024, 1024), edge=(128,)),
    # 4M-atom case: 3 layers, l_max=3, 128 channels, latent 2x512
    "c5": Arch(n_species=5, lmax=3, n_layers=3, channels=128, two_body=(64, 128, 512),
               latent=(512, 512), edge=(128,)),
}


def weight_shapes(arch: Arch) -> List[Tuple[str, tuple, str]]:
    """(name, shape, dtype) of every array, in draw and file order."""
    out = []
    fan = arch.n_in_two_body
    for k, w in enumerate(arch.two_body):
        out.append((f"two_body.{k}", (w, fan), "f32"))
        fan = w
    out.append(("embed", (arch.n_w, arch.latent_width(0)), "f32"))
    lm = arch.lmax + 1
    for L in range(1, arch.n_layers + 1):
        kin = arch.latent_width(L - 1)
        out.append((f"env.{L}", (arch.n_w, kin), "f32"))
        out.append((f"tp.{L}", (lm, 2, lm, 2, lm), "f32"))
        fan = kin + arch.channels
        for k, w in enumerate(arch.latent):
            out.append((f"latent.{L}.{k}", (w, fan), "f32"))
            fan = w
    fan = arch.latent_width(arch.n_layers)
    for k, w in enumerate(tuple(arch.edge) + (1,)):
        out.append((f"edge.{k}", (w, fan), "f32"))
        fan = w
    out.append(("sigma", (arch.n_species,), "f64"))
    out.append(("mu", (arch.n_species,), "f64"))
    return out


def weight_names(arch: Arch) -> List[str]:
    return [n for n, _, _ in weight_shapes(arch)]


def make_weights(arch: Arch, seed: int) -> Dict[str, np.ndarray]:
    """Draw all weights from numpy PCG64(seed) in file order."""
    rng = np.random.default_rng(seed)
    w: Dict[str, np.ndarray] = {}
    for name, shape, dt in weight_shapes(arch):
        if name.startswith("tp."):
            w[name] = rng.standard_normal(shape).astype(np.float32)
        elif name == "sigma":
            w[name] = (1.0 + 0.1 * rng.standard_normal(shape)).astype(np.float64)
        elif name == "mu":
            w[name] = (10.0 * rng.standard_normal(shape)).astype(np.float64)
        else:
            fan_in = shape[1]
            w[name] = (rng.standard_normal(shape) * np.sqrt(1.0 / fan_in)).astype(np.float32)
    return w


def weights_to_blob(arch: Arch, w: Dict[str, np.ndarray]) -> bytes:
    parts = [MAGIC, struct.pack("<I", VERSION), struct.pack("<dd", arch.r_c, arch.avg_num_neighbors)]
    parts.append(struct.pack("<9i", arch.n_species, arch.n_bessel, arch.p_env, arch.lmax,
                             arch.n_layers, arch.channels, len(arch.two_body), len(arch.latent),
                             len(arch.edge)))
    widths = list(arch.two_body) + list(arch.latent) + list(arch.edge)
    parts.append(struct.pack(f"<{len(widths)}i", *widths))
    for name, shape, dt in weight_shapes(arch):
        a = np.ascontiguousarray(w[name], dtype="<f4" if dt == "f32" else "<f8")
        assert a.shape == shape, (name, a.shape, shape)
        parts.append(a.tobytes())
    return b"".join(parts)


def blob_to_weights(blob: bytes):
    """Inverse of `weights_to_blob`: returns (arch, weights)."""
    if blob[:4] != MAGIC:
        raise ValueError("not an ALGW weights blob")
    (ver,) = struct.unpack_from("<I", blob, 4)
    if ver != VERSION:
        raise ValueError(f"unsupported ALGW version {ver}")
    r_c, ann = struct.unpack_from("<dd", blob, 8)
    hdr = struct.unpack_from("<9i", blob, 24)
    ns, nb, pe, lmax, nl, ch, n2, nlat, ned = hdr
    off = 24 + 36
    widths = struct.unpack_from(f"<{n2 + nlat + ned}i", blob, off)
    off += 4 * (n2 + nlat + ned)
    arch = Arch(n_species=ns, lmax=lmax, n_layers=nl, channels=ch,
                two_body=tuple(widths[:n2]), latent=tuple(widths[n2:n2 + nlat]),
                edge=tuple(widths[n2 + nlat:]), n_bessel=nb, p_env=pe, r_c=r_c,
                avg_num_neighbors=ann)
    w = {}
    for name, shape, dt in weight_shapes(arch):
        dtype = np.dtype("<f4" if dt == "f32" else "<f8")
        n = int(np.prod(shape))
        w[name] = np.frombuffer(blob, dtype=dtype, count=n, offset=off).reshape(shape).copy()
        off += n * dtype.itemsize
    if off != len(blob):
        raise ValueError("trailing bytes in ALGW blob")
    return arch, w


def arch_dict(arch: Arch) -> dict:
    return asdict(arch)
