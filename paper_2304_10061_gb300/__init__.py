"""GB300-native Allegro edge hot path (arXiv 2304.10061): Python binding.

`Allegro` wraps one context of liballegro_gb300.so (see include/allegro.h):
neighbour search, energy, per-atom energies, forces and virial, all computed
by the library's sm_103a kernels.  `AllegroEnergy` is a torch.autograd.Function
whose backward returns dE/dpos = -F from the hand-written adjoint.

Arrays may be numpy arrays or torch tensors, on the host or on the GPU; the
library detects which and copies as needed.  PyTorch provides device memory
and streams only.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import _lib

__all__ = ["Allegro", "AllegroError", "AllegroEnergy", "build"]


class AllegroError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_lib.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def build(force: bool = False, verbose: bool = False) -> str:
    from .build import build as _b
    return _b(force=force, verbose=verbose)


def _ptr(a) -> Optional[int]:
    """Raw pointer of a numpy array or torch tensor (contiguous), or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _as(a, dtype):
    """numpy views of the right dtype for host inputs; torch tensors are checked, not converted."""
    if a is None:
        return None
    if hasattr(a, "data_ptr") and not isinstance(a, np.ndarray):
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64, np.uint8: torch.uint8}[dtype]
        if a.dtype != want:
            raise TypeError(f"expected {want}, got {a.dtype}")
        return a.contiguous()
    return np.ascontiguousarray(a, dtype=dtype)


class Allegro:
    """One library context bound to one GPU and one model."""

    def __init__(self, weights_blob: bytes, species_map=None, r_c: float = 0.0, precision: str = "fp32",
                 device: int = 0):
        self._L = _lib.load()
        self._ctx = ctypes.c_void_p()
        blob = ctypes.create_string_buffer(bytes(weights_blob), len(weights_blob))
        smap = None if species_map is None else np.ascontiguousarray(species_map, dtype=np.int32)
        st = self._L.allegro_create(blob, len(weights_blob), None if smap is None else smap.ctypes.data,
                                    0 if smap is None else smap.size, float(r_c), _lib.PREC[precision],
                                    int(device), ctypes.byref(self._ctx))
        if st != 0:
            raise AllegroError(st, "allegro_create failed (see stderr)")
        self.precision = precision
        self.device = device
        self.n_atoms = 0
        self.n_edges = 0
        self.n_struct = 1

    def _check(self, st: int):
        if st != 0:
            raise AllegroError(st, self._L.allegro_last_error(self._ctx).decode())

    def close(self):
        if self._ctx:
            self._L.allegro_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_ptr: int):
        self._check(self._L.allegro_set_stream(self._ctx, ctypes.c_void_p(stream_ptr)))

    def reserve(self, atom_cap: int, edge_cap: int, fixed: bool = False, chunk_edges: int = 0):
        self._check(self._L.allegro_reserve(self._ctx, int(atom_cap), int(edge_cap), int(bool(fixed)),
                                            int(chunk_edges)))

    def set_pair_cutoffs(self, pair_rc=None):
        """Per-ordered-species-pair cutoffs [n_species][n_species] (row = centre species), or None
        for the model cutoff everywhere; rebuild the neighbour list afterwards."""
        if pair_rc is None:
            self._check(self._L.allegro_set_pair_cutoffs(self._ctx, None, 0))
            return
        t = np.ascontiguousarray(np.asarray(pair_rc, dtype=np.float64))
        if t.ndim != 2 or t.shape[0] != t.shape[1]:
            raise ValueError("pair_rc must be a square [n_species][n_species] table")
        self._check(self._L.allegro_set_pair_cutoffs(self._ctx, t.ctypes.data, int(t.shape[0])))

    def set_zbl(self, atomic_numbers=None):
        """ZBL repulsion with the atomic number of each model species (None removes it)."""
        if atomic_numbers is None:
            self._check(self._L.allegro_set_zbl(self._ctx, None, 0))
            return
        z = np.ascontiguousarray(np.asarray(atomic_numbers, dtype=np.int32))
        self._check(self._L.allegro_set_zbl(self._ctx, z.ctypes.data, int(z.size)))

    def neighbors(self, pos, types, cell=None, pbc=None) -> int:
        pos = _as(pos, np.float64)
        types = _as(types, np.int32)
        cell = _as(cell, np.float64)
        pbc = _as(pbc, np.uint8)
        n = int(pos.shape[0])
        ne = ctypes.c_int64(0)
        self._keep = (pos, types, cell, pbc)
        self._check(self._L.allegro_neighbors(self._ctx, n, _ptr(pos), _ptr(types), _ptr(cell), _ptr(pbc),
                                              ctypes.byref(ne)))
        self.n_atoms, self.n_edges, self.n_struct = n, int(ne.value), 1
        return self.n_edges

    def neighbors_local(self, n_local: int, pos, types, cell=None, pbc=None) -> int:
        """One sub-domain of a spatial decomposition: atoms [0, n_local) are centres, the
        rest ghosts (neighbours only)."""
        pos = _as(pos, np.float64)
        types = _as(types, np.int32)
        cell = _as(cell, np.float64)
        pbc = _as(pbc, np.uint8)
        n = int(pos.shape[0])
        ne = ctypes.c_int64(0)
        self._keep = (pos, types, cell, pbc)
        self._check(self._L.allegro_neighbors_local(self._ctx, int(n_local), n, _ptr(pos), _ptr(types), _ptr(cell),
                                                    _ptr(pbc), ctypes.byref(ne)))
        self.n_atoms, self.n_edges, self.n_struct = n, int(ne.value), 1
        return self.n_edges

    def neighbors_batched(self, offsets, pos, types, cells=None, pbc=None) -> int:
        offsets = _as(offsets, np.int64)
        pos = _as(pos, np.float64)
        types = _as(types, np.int32)
        cells = _as(cells, np.float64)
        pbc = _as(pbc, np.uint8)
        nb = int(offsets.shape[0]) - 1
        ne = ctypes.c_int64(0)
        self._keep = (offsets, pos, types, cells, pbc)
        self._check(self._L.allegro_neighbors_batched(self._ctx, nb, _ptr(offsets), _ptr(pos), _ptr(types),
                                                      _ptr(cells), _ptr(pbc), ctypes.byref(ne)))
        self.n_atoms, self.n_edges, self.n_struct = int(pos.shape[0]), int(ne.value), nb
        return self.n_edges

    def energy_forces(self, forces: bool = True, virial: bool = True, out: Optional[dict] = None,
                      device: Optional[str] = None) -> dict:
        """Returns dict(E [n_struct], E_atom [N], F [N,3], virial [n_struct,3,3]) as torch tensors
        (on `device`, default the context's GPU) or fills the arrays given in `out`."""
        import torch
        if out is None:
            dev = device or f"cuda:{self.device}"
            out = dict(E=torch.empty(self.n_struct, dtype=torch.float64, device=dev),
                       E_atom=torch.empty(self.n_atoms, dtype=torch.float64, device=dev))
            if forces:
                out["F"] = torch.empty(self.n_atoms, 3, dtype=torch.float64, device=dev)
            if virial:
                out["virial"] = torch.empty(self.n_struct, 3, 3, dtype=torch.float64, device=dev)
        self._check(self._L.allegro_energy_forces(self._ctx, _ptr(out["E"]), _ptr(out.get("E_atom")),
                                                  _ptr(out.get("F")), _ptr(out.get("virial"))))
        return out

    def md_verlet(self, pos, vel, types, masses, dt: float, n_steps: int, cell=None, pbc=None):
        """Velocity-Verlet MD on the GPU.  pos/vel are updated in place (numpy or torch,
        host or device).  Returns (E_pot [n_steps+1], E_kin [n_steps+1]) as numpy arrays."""
        types = _as(types, np.int32)
        masses = np.ascontiguousarray(masses, dtype=np.float64)
        cell = _as(cell, np.float64)
        pbc = _as(pbc, np.uint8)
        n = int(pos.shape[0])
        Ep = np.zeros(n_steps + 1)
        Ek = np.zeros(n_steps + 1)
        self._check(self._L.allegro_md_verlet(self._ctx, n, _ptr(pos), _ptr(vel), _ptr(types), masses.ctypes.data,
                                              masses.size, _ptr(cell), _ptr(pbc), float(dt), int(n_steps),
                                              Ep.ctypes.data, Ek.ctypes.data))
        self._sync_sizes()
        return Ep, Ek

    def _sync_sizes(self):
        """Atoms, edges and structures of the list the context holds."""
        na, ne, ns = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int32(0)
        self._check(self._L.allegro_list_size(self._ctx, ctypes.byref(na), ctypes.byref(ne), ctypes.byref(ns)))
        self.n_atoms, self.n_edges, self.n_struct = int(na.value), int(ne.value), int(ns.value)

    def set_autotune(self, enable: bool = True):
        """Launch-configuration autotuner (chunk size, fused layer pairs, epilogue warps) per shape bucket."""
        self._check(self._L.allegro_set_autotune(self._ctx, int(bool(enable))))

    def set_graphs(self, enable: bool = True):
        """Replay the evaluation as a CUDA graph while its shapes and buffers stay the same."""
        self._check(self._L.allegro_set_graphs(self._ctx, int(bool(enable))))

    def autotune_report(self) -> dict:
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        self._check(self._L.allegro_autotune_report(self._ctx, buf, len(buf)))
        return json.loads(buf.value.decode())

    def set_md_skin(self, skin: float):
        """Verlet skin (A) for md_verlet's neighbour reuse; 0 rebuilds every step."""
        self._check(self._L.allegro_set_md_skin(self._ctx, float(skin)))

    def md_rebuilds(self) -> int:
        """Neighbour-list builds made by the last md_verlet call."""
        n = ctypes.c_int64(0)
        self._check(self._L.allegro_md_rebuilds(self._ctx, ctypes.byref(n)))
        return int(n.value)

    def profile(self, enable: bool = True):
        self._check(self._L.allegro_profile(self._ctx, int(bool(enable))))

    def profile_report(self):
        """(per-kernel dict {name: {launches, ms, flops, bytes}}, total launches issued)."""
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        n = ctypes.c_int64(0)
        self._check(self._L.allegro_profile_report(self._ctx, buf, len(buf), ctypes.byref(n)))
        return json.loads(buf.value.decode() or "{}"), int(n.value)

    def get_neighbors(self):
        """(i, j, S) numpy int32 arrays of the last neighbour list (rows by ascending i)."""
        E = self.n_edges
        i = np.empty(E, np.int32)
        j = np.empty(E, np.int32)
        S = np.empty((E, 3), np.int32)
        self._check(self._L.allegro_get_neighbors(self._ctx, i.ctypes.data, j.ctypes.data, S.ctypes.data, E))
        return i, j, S


def _autograd():
    import torch

    class AllegroEnergy(torch.autograd.Function):
        """E = AllegroEnergy.apply(pos, model, types, cell, pbc): total energy (float64 scalar);
        backward gives dE/dpos = -F from the library's adjoint."""

        @staticmethod
        def forward(ctx, pos, model, types, cell=None, pbc=None):
            model.neighbors(pos.detach().contiguous(), types, cell, pbc)
            out = model.energy_forces(forces=True, virial=False, device=str(pos.device))
            ctx.save_for_backward(out["F"])
            return out["E"][0]

        @staticmethod
        def backward(ctx, gE):
            (F,) = ctx.saved_tensors
            return -F * gE, None, None, None, None

    return AllegroEnergy


class _Lazy:
    _cls = None

    def __getattr__(self, name):
        if _Lazy._cls is None:
            _Lazy._cls = _autograd()
        return getattr(_Lazy._cls, name)


AllegroEnergy = _Lazy()
