"""Benchmark of the Allegro edge hot path on GB300: atom-steps/s (E+F).

One step = neighbour rebuild + energy + forces + virial of the 1,048,576-atom
periodic water-density box (218.9 A, 2 layers, l_max 2, 64 channels) through the
C ABI, with BF16 MLP GEMMs on the tcgen05 tensor cores.  Inputs stay resident on
the GPU for `value`; `e2e` repeats the step with the positions in pinned host
memory and the results read back to pinned host memory every step.  The
float32 path is timed beside it (`fp32`), the FP64 CPU oracle on a 4,096-atom
sample of the same workload (`cpu_baseline`).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank evaluates its own replica (weak scaling, no
collective on the data path); the reported time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "atom-steps/s (E+F) per GB300 at 1M atoms, BF16-MLP vs FP32; force err vs FP64"
UNIT = "atom-steps/s"
WORKLOAD = ("1,048,576-atom periodic water-density box (218.9 A cube, jittered lattice, "
            "H/O/C/N/S mix), Allegro 2 layers, l_max 2, 64 channels, two-body [64,128,256], "
            "latent 2x256, edge 256->128->1, r_c 4 A, seeded random weights")


PAIR_NOTE = ", per-ordered-species-pair cutoffs (H-H 3.0, H-C 1.25, H-O 1.25, O-H 3.0 A, others 4.0 A)"


def _workload(args, s) -> str:
    """The workload string: the headline box, or what --config / --atoms / --pair-cutoffs selected."""
    note = PAIR_NOTE if getattr(args, "pair_cutoffs", False) else ""
    if args.config == "c4" and not args.atoms:
        return WORKLOAD + note
    L = float(abs(s.cell[0][0])) if s.cell is not None else 0.0
    return (f"{s.n_atoms:,}-atom periodic box ({L:.1f} A cube, config {args.config}), same model family and "
            "seeded random weights" + note)


def _pair_arch(args, arch):
    """The architecture with the paper's per-ordered-species-pair cutoff table when --pair-cutoffs is set."""
    if not getattr(args, "pair_cutoffs", False):
        return arch
    from dataclasses import replace
    from synth import paper_pair_cutoffs
    return replace(arch, pair_rc=paper_pair_cutoffs(default=arch.r_c))


def _edges(arch, s):
    """The oracle's neighbour list of `s` under the architecture's cutoff rule."""
    from oracle.neighbors import neighbor_list
    if arch.pair_rc is None:
        return neighbor_list(s.pos, s.cell, s.pbc, arch.r_c)
    return neighbor_list(s.pos, s.cell, s.pbc, arch.r_c, species=s.species, pair_rc=arch.pair_rc)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    import torch
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend=backend)
    return rank, ws, local, dist


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def reduce_max(x: float, dist=None, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (identity without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(atoms_per_rank: int, ms_per_step_local: float, world: int, dist=None, device=None):
    """Whole-job throughput: every rank evaluates its own replica, so the job
    processes world x atoms per step in the slowest rank's step time."""
    ms = reduce_max(ms_per_step_local, dist, device)
    return ms, atoms_per_rank * world / (ms * 1e-3)


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def _by_kernel(report: dict) -> dict:
    """Per-launch records are labelled '<kernel>/<which map>'; sum them per kernel."""
    out = {}
    for k, v in report.items():
        base = k.split("/")[0]
        a = out.setdefault(base, {"launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0})
        for f in a:
            a[f] += v[f]
    return out


def _traffic_per_launch(detail: dict, steps: int, n_edges: int):
    """DRAM traffic per GEMM launch from the committed ncu capture (bytes per edge per
    launch), scaled to this run's edges per launch (= edges / chunks per step)."""
    try:
        ref = json.load(open(os.path.join(ROOT, "profiles", "gemm_tc_traffic.json")))
        gem = [v for k, v in detail.items() if k.startswith("gemm_tc/")]
        chunks = gem[0]["launches"] / steps
        return ref["dram_bytes_per_edge_per_gemm_launch"] * n_edges / chunks
    except Exception:
        return None


def model_macs_per_edge(arch) -> int:
    """Forward multiply-adds per edge of every MLP of the model as the architecture
    defines it: two-body, embedding, per layer env weights and latent MLP, and the
    edge-energy MLP (the scope table's per-edge count; the library folds the linear
    edge MLP into one vector and forms the first two-body layer on the CUDA cores,
    so it executes fewer)."""
    macs, fan = 0, arch.n_in_two_body
    for w in arch.two_body:
        macs += fan * w
        fan = w
    macs += arch.latent_width(0) * arch.n_w                      # embedding
    for L in range(1, arch.n_layers + 1):
        kin = arch.latent_width(L - 1)
        macs += kin * arch.n_w                                   # env weights of layer L
        fan = kin + arch.channels
        for w in arch.latent:
            macs += fan * w
            fan = w
    fan = arch.latent_width(arch.n_layers)
    for w in tuple(arch.edge) + (1,):
        macs += fan * w
        fan = w
    return macs


def model_flops_per_edge(arch) -> float:
    """MLP FLOPs per edge of one energy + force evaluation: the forward and the
    input-gradient adjoint, each 2 FLOPs per multiply-add."""
    return 2.0 * 2.0 * model_macs_per_edge(arch)


def step_bytes_per_edge(arch, edges_per_atom: float, act_bytes: int = 2) -> float:
    """Algorithmic HBM bytes per edge of a whole step with fused, on-chip MLP
    activations: the CSR entry (16 B), the latents x^0..x^L kept for the adjoint
    (written once, read once), the per-atom environments and their adjoints
    (C S float32 per layer, two each) shared by the row's edges, and the edge
    force vector g_ij written and read (float32 x 3)."""
    S = (arch.lmax + 1) ** 2
    lat = sum(2.0 * arch.latent_width(L) * act_bytes for L in range(arch.n_layers + 1))
    per_atom = 2.0 * arch.n_layers * arch.channels * S * 4.0
    return 16.0 + lat + per_atom / max(edges_per_atom, 1e-9) + 24.0


def _roofline(report: dict, step_ms_total: float, steps: int = 1, n_edges: int = 0, arch=None,
              n_atoms: int = 0):
    """Dominant kernel (largest total time) of the timed region against its roofline.

    The MLP GEMMs (all "gemm_tc" launches together) are a dense contraction:
    bound "tensor", achieved = the model's MLP FLOPs per launch (the scope
    table's per-edge count x the edges one launch covers) / the launches'
    average CUDA-event duration, against the sustained BF16 peak (kernels timed
    inside a long step).  Other kernels: HBM, algorithmic bytes per launch
    against the measured copy bandwidth."""
    if not report:
        return None
    detail = report
    report = _by_kernel(report)
    name, r = max(report.items(), key=lambda kv: kv[1]["ms"])
    peaks = _peaks()
    tensor = name.startswith("gemm_tc")
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    tc_peak = peaks["bf16_tflops_sustained"] if peaks else 1700.0
    L = max(r["launches"], 1)
    ms_launch = r["ms"] / L
    share = {k: round(v["ms"] / max(step_ms_total, 1e-9), 4) for k, v in
             sorted(report.items(), key=lambda kv: -kv[1]["ms"])}
    out = {"kernel": name, "peak_source": "measured" if peaks else "fallback",
           "launches": r["launches"], "ms_per_launch": round(ms_launch, 5), "share_of_timed_region": share}
    if tensor and arch is not None and n_edges:
        fpe = model_flops_per_edge(arch)
        flops_launch = fpe * n_edges * steps / L
        achieved = flops_launch / (ms_launch * 1e-3) / 1e12
        traffic = _traffic_per_launch(detail, steps, n_edges)
        edges_launch = n_edges * steps / L
        s8d = step_bytes_per_edge(arch, n_edges / max(n_atoms, 1))
        out.update({"bound": "tensor", "achieved": round(achieved, 2), "peak": tc_peak, "unit": "TFLOP/s",
                    "frac": round(achieved / tc_peak, 4), "peak_kind": "bf16 sustained (of measured)",
                    "model_flops_per_edge": fpe, "edges_per_launch": round(edges_launch, 1),
                    "flops_per_launch": flops_launch,
                    "executed_flops_per_launch": r["flops"] / L,
                    "executed_tflops": round(r["flops"] / (r["ms"] * 1e-3) / 1e12, 2),
                    "traffic": traffic, "traffic_unit": "bytes per launch (DRAM read + write)",
                    "traffic_bytes_per_edge_per_step": (traffic * L / (n_edges * steps)) if traffic else None,
                    "decomposition_bytes_per_launch": r["bytes"] / L,
                    "decomposition_gbs": round(r["bytes"] / (r["ms"] * 1e-3) / 1e9, 1),
                    "step_bytes_per_edge": round(s8d, 1),
                    "wasted_traffic_ratio": round(traffic * L / (n_edges * steps) / s8d, 2) if traffic else None})
    elif tensor:
        achieved = r["flops"] / (r["ms"] * 1e-3) / 1e12
        out.update({"bound": "tensor", "achieved": round(achieved, 2), "peak": tc_peak, "unit": "TFLOP/s",
                    "frac": round(achieved / tc_peak, 4), "traffic": None})
    else:
        achieved = r["bytes"] / (r["ms"] * 1e-3) / 1e9
        out.update({"bound": "hbm", "achieved": round(achieved, 2), "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(achieved / hbm_peak, 4), "traffic": None,
                    "algorithmic_bytes_per_launch": r["bytes"] / L})
    if arch is not None and n_edges and n_atoms:
        s8d = step_bytes_per_edge(arch, n_edges / n_atoms)
        step_ms = step_ms_total / max(steps, 1)
        gbs = s8d * n_edges / (step_ms * 1e-3) / 1e9
        out["step_hbm"] = {"bytes_per_edge": round(s8d, 1), "achieved_gbs": round(gbs, 1), "peak": hbm_peak,
                           "frac": round(gbs / hbm_peak, 4),
                           "note": "whole step against the fused-activation byte budget"}
    out["kernels"] = {k: {"share": round(v["ms"] / max(step_ms_total, 1e-9), 4),
                          "GB/s": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1),
                          "frac_hbm": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9 / hbm_peak, 4)}
                      for k, v in sorted(report.items(), key=lambda kv: -kv[1]["ms"]) if not k.startswith("gemm")}
    out["gemm_detail"] = {k.split("/", 1)[1]: {
                              "share": round(v["ms"] / max(step_ms_total, 1e-9), 4),
                              "TFLOP/s": round(v["flops"] / (v["ms"] * 1e-3) / 1e12, 1),
                              "GB/s": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1)}
                          for k, v in sorted(detail.items(), key=lambda kv: -kv[1]["ms"]) if "/" in k}
    return out


def _force_errors(F, E, F0, E0) -> dict:
    import numpy as np
    rms = float(np.sqrt((F0 ** 2).mean()))
    return {"force_rms_err_over_rms_F": float(np.sqrt(((F - F0) ** 2).mean()) / rms),
            "force_max_err_over_rms_F": float(np.abs(F - F0).max() / rms),
            "E_rel_err": float(abs(E - E0) / abs(E0))}


def _cpu_baseline(arch, w, blob, precision_models: dict, timed_steps: int = 3):
    """FP64 oracle on a bounded sample (the 4,096-atom box of the same density and
    model): one untimed warm-up step, then `timed_steps` timed steps; and the GPU
    paths' force errors against it on that sample."""
    import numpy as np
    import torch
    from oracle.allegro import AllegroOracle
    from synth import make_config
    torch.set_num_threads(os.cpu_count() or 1)
    s, _, _ = make_config("c4sub")
    orc = AllegroOracle(arch, w)

    def step():
        i, j, S = _edges(arch, s)
        return (i,) + tuple(orc.energy_forces(s.pos, s.species, s.cell, i, j, S))

    i, E0, Ea0, F0, W0 = step()                      # warm-up (also the reference values)
    t0 = time.perf_counter()
    for _ in range(timed_steps):
        step()
    dt = (time.perf_counter() - t0) / timed_steps
    errs = {}
    for prec, m in precision_models.items():
        m.neighbors(s.pos, s.species, s.cell)
        out = m.energy_forces()
        errs[prec] = _force_errors(out["F"].cpu().numpy(), out["E"].item(), F0, E0)
    return {"value": s.n_atoms / dt, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"{timed_steps} timed steps after 1 warm-up (neighbours + E + F + virial) of the "
                      f"{s.n_atoms}-atom periodic box at the same density and model ({len(i)} edges), FP64 torch "
                      "on the host cores",
            "seconds_per_step": round(dt, 3)}, {"sample": "4,096-atom box, all atoms",
                                                "fp64_oracle_rms_F": float(np.sqrt((F0 ** 2).mean())), **errs}


def _pair_cutoff_run(args, make_model, pos, types, cell, out, N, steps: int):
    """The same box under the paper's per-ordered-species-pair cutoff table:
    step time and edges on the GPU, and the GPU paths' force errors against the
    FP64 oracle on the 4,096-atom sample under the same table."""
    import torch
    from dataclasses import replace
    from synth import make_config, paper_pair_cutoffs
    from oracle.allegro import AllegroOracle
    res = {}
    m = make_model(args.precision, pair=True)
    for _ in range(2):
        m.neighbors(pos, types, cell)
        m.energy_forces(out=out)
    torch.cuda.synchronize()
    st = m.stream
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(steps):
        m.neighbors(pos, types, cell)
        m.energy_forces(out=out)
    b.record(st)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    res.update({"ms_per_step": ms, "atom_steps_per_s": N / (ms * 1e-3), "edges": m.n_edges, "unit": UNIT,
                "table": "H-H 3.0, H-C 1.25, H-O 1.25, O-H 3.0 A, every other ordered pair 4.0 A"})
    if not args.skip_cpu:
        s, arch, w = make_config("c4sub")
        arch = replace(arch, pair_rc=paper_pair_cutoffs(default=arch.r_c))
        i, j, S = _edges(arch, s)
        E0, _, F0, _ = AllegroOracle(arch, w).energy_forces(s.pos, s.species, s.cell, i, j, S)
        for prec in (args.precision, "fp32"):
            mm = m if prec == args.precision else make_model(prec, pair=True)
            mm.neighbors(s.pos, s.species, s.cell)
            o = mm.energy_forces()
            res[f"force_err_vs_fp64_{prec}"] = _force_errors(o["F"].cpu().numpy(), o["E"].item(), F0, E0)
            if mm is not m:
                mm.close()
    m.close()
    return res


def _precision_matrix(args, local, stream):
    import numpy as np
    import torch
    from paper_2304_10061_gb300 import Allegro
    from synth import ARCHS, lattice_box, make_weights, weights_to_blob
    arch = ARCHS["c2"]
    w = make_weights(arch, 1)
    blob = weights_to_blob(arch, w)
    s = lattice_box(3072, (3072 / 0.1) ** (1.0 / 3.0), seed=7)
    dev = f"cuda:{local}"
    px = torch.tensor(s.pos, device=dev)
    tx = torch.tensor(s.species, dtype=torch.int32, device=dev)
    cx = torch.tensor(s.cell, device=dev)
    rows = {"tf32": "F64 final, F32 weights, TF32 compute", "fp32": "F64 final, F32 weights, F32 compute",
            "bf16": "F64 final, F32 master weights, BF16 compute"}
    res = {"atoms": s.n_atoms, "paper_relative_speed_A100": {"F64,F32,TF32": 1.0, "F64,F32,F32": 0.37,
                                                             "F32,F32,TF32": 0.98, "F32,F32,F32": 0.37,
                                                             "F64,F64,F64": 0.26}}
    F0 = E0 = None
    if not args.skip_cpu:
        from oracle.allegro import AllegroOracle
        i, j, S = _edges(arch, s)
        E0, _, F0, _ = AllegroOracle(arch, w).energy_forces(s.pos, s.species, s.cell, i, j, S)
    for prec, label in rows.items():
        m = Allegro(blob, precision=prec, device=local)
        m.set_stream(stream.cuda_stream)
        out = dict(E=torch.empty(1, dtype=torch.float64, device=dev),
                   E_atom=torch.empty(s.n_atoms, dtype=torch.float64, device=dev),
                   F=torch.empty(s.n_atoms, 3, dtype=torch.float64, device=dev),
                   virial=torch.empty(1, 3, 3, dtype=torch.float64, device=dev))
        for _ in range(3):
            m.neighbors(px, tx, cx)
            m.energy_forces(out=out)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(20):
            m.neighbors(px, tx, cx)
            m.energy_forces(out=out)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / 20
        rec = {"setting": label, "ms_per_step": ms, "atom_steps_per_s": s.n_atoms / (ms * 1e-3)}
        if F0 is not None:
            rec["force_err_vs_fp64"] = _force_errors(out["F"].cpu().numpy(), out["E"].item(), F0, E0)
        res[prec] = rec
        m.close()
    for prec in rows:
        res[prec]["relative_speed"] = res["tf32"]["ms_per_step"] / res[prec]["ms_per_step"]
    res["note"] = ("step = neighbour rebuild + E + F + virial; relative speed against the TF32 row as in the "
                   "paper's table; the all-float64 GPU row is not built (the FP64 path is the CPU oracle)")
    return res


def _paper_model(args, local, stream, n_atoms: int = 262144):
    """The paper's production architecture (2 layers, 64 channels, l_max 2, two-body
    [128, 256, 512, 1024], latent 3 x 1024, edge [128]) with its per-pair cutoffs and ZBL
    term, seeded random weights, on a water-density box: step time, throughput and the
    model's MLP FLOP rate, BF16 and TF32 (the paper's compute precision); force errors
    against the FP64 oracle on a 512-atom box of the same density."""
    import torch
    from dataclasses import replace
    from paper_2304_10061_gb300 import Allegro
    from synth import ARCHS, SPECIES_Z, lattice_box, make_weights, paper_pair_cutoffs, weights_to_blob
    arch = replace(ARCHS["paper"], pair_rc=paper_pair_cutoffs(), zbl_z=SPECIES_Z)
    w = make_weights(arch, 1)
    blob = weights_to_blob(arch, w)
    s = lattice_box(n_atoms, (n_atoms / 0.1) ** (1.0 / 3.0), seed=9)
    dev = f"cuda:{local}"
    px = torch.tensor(s.pos, device=dev)
    tx = torch.tensor(s.species, dtype=torch.int32, device=dev)
    cx = torch.tensor(s.cell, device=dev)
    res = {"atoms": s.n_atoms, "architecture": "2 layers, 64 channels, l_max 2, two-body [128,256,512,1024], "
                                               "latent [1024,1024,1024], edge [128], per-pair cutoffs, ZBL",
           "model_flops_per_edge": model_flops_per_edge(arch),
           "paper_context": "paper: 1,119,744-atom water on 64 A100 nodes (256 GPUs) at 20.3 steps/s, about "
                            "8.9e4 atom-steps/s per A100 (whole LAMMPS MD step, TF32)"}
    # force errors of the MLP precision: the ZBL term (exact up to float32 rounding) would dominate
    # RMS|F| at the lattice's closest contacts, so the error sample runs without it
    small = lattice_box(512, (512 / 0.1) ** (1.0 / 3.0), seed=10)
    ref = None
    if not args.skip_cpu:
        from oracle.allegro import AllegroOracle
        a0 = replace(arch, zbl_z=None)
        i, j, S = _edges(a0, small)
        ref = AllegroOracle(a0, w).energy_forces(small.pos, small.species, small.cell, i, j, S)
    for prec in ("bf16", "tf32"):
        m = Allegro(blob, precision=prec, device=local)
        m.set_stream(stream.cuda_stream)
        m.set_pair_cutoffs(arch.pair_rc)
        m.set_zbl(SPECIES_Z)
        out = dict(E=torch.empty(1, dtype=torch.float64, device=dev),
                   E_atom=torch.empty(s.n_atoms, dtype=torch.float64, device=dev),
                   F=torch.empty(s.n_atoms, 3, dtype=torch.float64, device=dev),
                   virial=torch.empty(1, 3, 3, dtype=torch.float64, device=dev))
        for _ in range(2):
            m.neighbors(px, tx, cx)
            m.energy_forces(out=out)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        K = 4
        a.record(stream)
        for _ in range(K):
            m.neighbors(px, tx, cx)
            m.energy_forces(out=out)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / K
        rec = {"ms_per_step": ms, "atom_steps_per_s": s.n_atoms / (ms * 1e-3), "edges": m.n_edges,
               "model_tflops_per_s": res["model_flops_per_edge"] * m.n_edges / (ms * 1e-3) / 1e12}
        if ref is not None:
            m.set_zbl(None)
            m.neighbors(small.pos, small.species, small.cell)
            o = m.energy_forces()
            rec["force_err_vs_fp64_512_atoms_no_zbl"] = _force_errors(o["F"].cpu().numpy(), o["E"].item(), ref[2],
                                                                      ref[0])
        res[prec] = rec
        m.close()
    return res


def _c5_run(args, local, stream, steps: int = 1):
    """The 4,194,304-atom configuration (3 layers, l_max 3, 128 channels, latent 2 x 512) in BF16:
    E + F + virial with a neighbour rebuild per step, the device memory the library holds, and
    the force error of the same architecture against the FP64 oracle on a 256-atom box."""
    import torch
    from paper_2304_10061_gb300 import Allegro
    from synth import lattice_box, make_config, weights_to_blob
    s, arch, w = make_config("c5")
    blob = weights_to_blob(arch, w)
    dev = f"cuda:{local}"
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info(local)
    px = torch.tensor(s.pos, device=dev)
    tx = torch.tensor(s.species, dtype=torch.int32, device=dev)
    cx = torch.tensor(s.cell, device=dev)
    out = dict(E=torch.empty(1, dtype=torch.float64, device=dev),
               E_atom=torch.empty(s.n_atoms, dtype=torch.float64, device=dev),
               F=torch.empty(s.n_atoms, 3, dtype=torch.float64, device=dev),
               virial=torch.empty(1, 3, 3, dtype=torch.float64, device=dev))
    m = Allegro(blob, precision="bf16", device=local)
    m.set_stream(stream.cuda_stream)
    m.neighbors(px, tx, cx)
    m.energy_forces(out=out)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        m.neighbors(px, tx, cx)
        m.energy_forces(out=out)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    free1, _ = torch.cuda.mem_get_info(local)
    res = {"atoms": s.n_atoms, "edges": m.n_edges, "precision": "bf16",
           "architecture": "3 layers, 128 channels, l_max 3, two-body [64,128,512], latent [512,512], edge [128]",
           "model_flops_per_edge": model_flops_per_edge(arch), "steps": steps, "ms_per_step": ms,
           "atom_steps_per_s": s.n_atoms / (ms * 1e-3),
           "model_tflops_per_s": model_flops_per_edge(arch) * m.n_edges / (ms * 1e-3) / 1e12,
           "device_gb_in_use": (free0 - free1) / 1e9, "device_gb_total": total / 1e9,
           "memory_note": "device memory in use after the step minus before the inputs were placed (inputs, outputs "
                          "and the library's buffers, which only grow, so this is the step's peak); edge activations "
                          "live for one chunk of centre rows at a time",
           "e_total": float(out["E"].item())}
    m.close()
    if not args.skip_fp8:
        m8 = Allegro(blob, precision="fp8", device=local)
        m8.set_stream(stream.cuda_stream)
        m8.neighbors(px, tx, cx)
        m8.energy_forces(out=out)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(steps):
            m8.neighbors(px, tx, cx)
            m8.energy_forces(out=out)
        b.record(stream)
        torch.cuda.synchronize()
        ms8 = a.elapsed_time(b) / steps
        res["fp8"] = {"ms_per_step": ms8, "atom_steps_per_s": s.n_atoms / (ms8 * 1e-3), "speedup_over_bf16": ms / ms8}
        m8.close()
    if not args.skip_cpu:
        from oracle.allegro import AllegroOracle
        small = lattice_box(256, (256 / 0.1) ** (1.0 / 3.0), seed=11)
        i, j, S = _edges(arch, small)
        ref = AllegroOracle(arch, w).energy_forces(small.pos, small.species, small.cell, i, j, S)
        for prec in ("bf16", "fp32") + (() if args.skip_fp8 else ("fp8",)):
            mm = Allegro(blob, precision=prec, device=local)
            mm.neighbors(small.pos, small.species, small.cell)
            o = mm.energy_forces()
            res[f"force_err_vs_fp64_256_atoms_{prec}"] = _force_errors(o["F"].cpu().numpy(), o["E"].item(), ref[2],
                                                                       ref[0])
            mm.close()
    return res


def run_reference(args):
    """The oracle as it stands, on the host cores: each step one bounded sample of the workload."""
    rank, ws, _, dist = _dist()
    if rank != 0:
        return
    import torch
    from oracle.allegro import AllegroOracle
    from synth import make_config
    torch.set_num_threads(os.cpu_count() or 1)
    s, arch, w = make_config("c4sub")
    arch = _pair_arch(args, arch)
    orc = AllegroOracle(arch, w)

    def step():
        i, j, S = _edges(arch, s)
        orc.energy_forces(s.pos, s.species, s.cell, i, j, S)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    v = s.n_atoms * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": _workload(args, s), "sample": "each step: the 4,096-atom box of the same density "
                                                       "and model (bounded sample for the CPU)"},
            "cpu_baseline": {"kind": "oracle", "cores": torch.get_num_threads(), "value": v, "unit": UNIT,
                             "sample": "4,096-atom box, neighbours + E + F + virial per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    rank, ws, local, dist = _dist()
    import __graft_entry__ as g
    if rank == 0:
        g.build()
    if dist is not None:
        dist.barrier()
    g.build()
    from paper_2304_10061_gb300 import Allegro
    from synth import make_config, weights_to_blob

    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    over = {}
    if args.atoms:   # same density as the configuration, scaled box
        from synth.configs import CONFIGS
        c = CONFIGS[args.config]
        over = dict(n=args.atoms, L=c["L"] * (args.atoms / c["n"]) ** (1.0 / 3.0))
    s, arch, w = make_config(args.config, **over)
    blob = weights_to_blob(arch, w)
    arch = _pair_arch(args, arch)
    N = s.n_atoms
    pos = torch.tensor(s.pos, device=dev)
    types = torch.tensor(s.species, dtype=torch.int32, device=dev)
    cell = torch.tensor(s.cell, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def make(prec, pair=False):
        m = Allegro(blob, precision=prec, device=local)
        m.set_stream(stream.cuda_stream)
        m.stream = stream
        if args.chunk_edges:
            m.reserve(0, 0, False, args.chunk_edges)
        if arch.pair_rc is not None:
            m.set_pair_cutoffs(arch.pair_rc)
        elif pair:
            from synth import paper_pair_cutoffs
            m.set_pair_cutoffs(paper_pair_cutoffs(default=arch.r_c))
        return m

    def timed(m, K, W, out):
        for _ in range(W):
            m.neighbors(pos, types, cell)
            m.energy_forces(out=out)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(K):
            m.neighbors(pos, types, cell)
            m.energy_forces(out=out)
        b.record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        return a.elapsed_time(b) / K

    def dev_out():
        return dict(E=torch.empty(1, dtype=torch.float64, device=dev),
                    E_atom=torch.empty(N, dtype=torch.float64, device=dev),
                    F=torch.empty(N, 3, dtype=torch.float64, device=dev),
                    virial=torch.empty(1, 3, 3, dtype=torch.float64, device=dev))

    # ---- BF16 path, inputs resident (the headline) ----
    m = make(args.precision)
    out = dev_out()
    for _ in range(args.warmup):
        m.neighbors(pos, types, cell)
        m.energy_forces(out=out)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    m.profile(True)
    launches0 = m.profile_report()[1]
    ms = timed(m, args.steps, 0, out)
    report, launches1 = m.profile_report()
    m.profile(False)
    clk = clocks.stop()
    n_edges = m.n_edges
    ms_max, value = aggregate(N, ms, ws, dist, dev)

    # ---- energy + forces + virial alone on a fixed neighbour list, eager and CUDA-graph replay ----
    ef_only = {}
    for graphs in (False, True):
        m.set_graphs(graphs)
        m.neighbors(pos, types, cell)
        for _ in range(3):
            m.energy_forces(out=out)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        kf = max(1, min(args.steps, 5))
        a.record(stream)
        for _ in range(kf):
            m.energy_forces(out=out)
        b.record(stream)
        torch.cuda.synchronize()
        msf = a.elapsed_time(b) / kf
        ef_only["graph_replay" if graphs else "eager"] = {"ms_per_step": msf, "atom_steps_per_s": N / (msf * 1e-3)}
    m.set_graphs(False)
    ef_only["note"] = "energy + forces + virial on the list built once (no neighbour rebuild in the step)"

    # ---- end to end: pinned host inputs, host outputs, every step ----
    hpos = torch.tensor(s.pos).pin_memory()
    htypes = torch.tensor(s.species, dtype=torch.int32).pin_memory()
    hcell = torch.tensor(s.cell).pin_memory()
    hout = dict(E=torch.empty(1, dtype=torch.float64).pin_memory(),
                E_atom=torch.empty(N, dtype=torch.float64).pin_memory(),
                F=torch.empty(N, 3, dtype=torch.float64).pin_memory(),
                virial=torch.empty(1, 3, 3, dtype=torch.float64).pin_memory())
    ke = max(1, min(args.steps, 5))
    m.neighbors(hpos, htypes, hcell)
    m.energy_forces(out=hout)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        m.neighbors(hpos, htypes, hcell)
        m.energy_forces(out=hout)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / ke
    e2e_max = reduce_max(e2e_s, dist, dev)
    h2d = N * 3 * 8 + N * 4 + 9 * 8
    d2h = 8 + N * 8 + N * 3 * 8 + 9 * 8

    # ---- float32 path beside it ----
    fp32 = None
    if not args.skip_fp32:
        m32 = make("fp32")
        ms32 = timed(m32, max(1, min(args.steps, args.fp32_steps)), 1, dev_out())
        fp32 = {"value": N * ws / (ms32 * 1e-3), "unit": UNIT, "ms_per_step": ms32,
                "bf16_speedup_over_fp32": ms32 / ms}
    else:
        m32 = None

    # ---- FP8 (E4M3 MLP GEMMs, per-tensor scales) beside it ----
    fp8 = None
    m8 = None
    if args.precision == "bf16" and not args.skip_fp8:
        m8 = make("fp8")
        ms8 = timed(m8, max(1, min(args.steps, 5)), 1, dev_out())
        fp8 = {"value": N * ws / (ms8 * 1e-3), "unit": UNIT, "ms_per_step": ms8, "speedup_over_bf16": ms / ms8,
               "note": "MLP GEMMs with E4M3 operands (tcgen05 kind::f8f6f4), float32 accumulation, per-tensor "
                       "power-of-two scales, bf16 activations; evaluated through the generic row path"}

    # ---- context workloads: batched uneven molecules, and an MD run with 1 fs steps ----
    extra = {}
    if not args.skip_extra:
        from synth import molecule_batch, lattice_box
        from synth.structures import pack
        import numpy as np
        mols = molecule_batch(2048, seed=2)
        mpos, mspec, moffs = pack(mols)
        bt, bt_ef, tuned = {}, {}, {}
        for prec in (args.precision, "fp32"):
            # the batched-inference configuration: launch configuration autotuned on the first
            # evaluation of the shape, then the evaluation replayed as one CUDA graph
            mb = make(prec)
            mb.set_autotune(True)
            mb.set_graphs(True)
            mb.neighbors_batched(moffs, mpos, mspec)
            for _ in range(3):                       # tune, capture, replay
                mb.energy_forces()
            torch.cuda.synchronize()
            nrep = 10
            t0 = time.perf_counter()
            for _ in range(nrep):                    # whole step: host inputs, list rebuild, E + F + virial
                mb.neighbors_batched(moffs, mpos, mspec)
                mb.energy_forces()
            torch.cuda.synchronize()
            bt[prec] = len(mpos) * nrep / (time.perf_counter() - t0)
            t0 = time.perf_counter()
            for _ in range(nrep):                    # E + F + virial on the list built once
                mb.energy_forces()
            torch.cuda.synchronize()
            bt_ef[prec] = len(mpos) * nrep / (time.perf_counter() - t0)
            rep = mb.autotune_report()
            tuned[prec] = {"configuration": rep["current"], "graph_replays": rep["graph_replays"],
                           "kernels_per_graph": rep["graph_kernels"]}
            ne = mb.n_edges
            mb.close()
        extra["batched_2048_molecules"] = {
            "atoms": int(len(mpos)), "edges": int(ne), "unit": UNIT, args.precision: bt[args.precision],
            "fp32": bt["fp32"],
            "ef_only": {args.precision: bt_ef[args.precision], "fp32": bt_ef["fp32"]},
            "autotuned": tuned,
            "note": "2048 gas-phase molecules of 8-64 atoms in one packed edge list, per-molecule E/F/virial; "
                    "autotuned launch configuration, evaluation replayed as a CUDA graph; the step rebuilds "
                    "the list from host inputs each time, ef_only evaluates the list built once"}
        s2, _, _ = make_config("c2")
        masses = np.array([1.008, 15.999, 12.011, 14.007, 32.06])
        rng = np.random.default_rng(0)
        vel = rng.normal(size=(s2.n_atoms, 3)) * np.sqrt(0.0257 * 9.648533212e-3 / masses[s2.species][:, None])
        md = {}
        for skin in (0.0, 1.0):
            mm = make(args.precision)
            mm.set_md_skin(skin)
            p2, v2 = s2.pos.copy(), vel.copy()
            mm.md_verlet(p2, v2, s2.species, masses, 1.0, 2, cell=s2.cell)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            nmd = 20
            Ep, Ek = mm.md_verlet(p2, v2, s2.species, masses, 1.0, nmd, cell=s2.cell)
            torch.cuda.synchronize()
            dt_md = time.perf_counter() - t0
            md[f"skin_{skin:g}A"] = {"timesteps_per_s": nmd / dt_md, "atom_steps_per_s": s2.n_atoms * nmd / dt_md,
                                     "list_builds": mm.md_rebuilds(),
                                     "energy_drift_eV_per_atom":
                                         float(abs((Ep[-1] + Ek[-1]) - (Ep[0] + Ek[0])) / s2.n_atoms)}
            mm.close()
        extra["md_23552_atoms"] = {"dt_fs": 1.0, "steps": nmd, **md,
                                   "note": "velocity Verlet on the GPU, host inputs once per run; skin 0: neighbour "
                                           "rebuild every step; skin 1 A: exact list filtered from a candidate list "
                                           "at r_c + skin, rebuilt when an atom moved skin/2"}
        # the smaller named workloads (E + F + virial with a neighbour rebuild per step), both precisions
        for name, label in (("c2", "c2_23552_atoms"), ("c1", "c1_64_atoms")):
            sx, ax, wx = make_config(name)
            bx = weights_to_blob(ax, wx)
            px = torch.tensor(sx.pos, device=dev)
            tx = torch.tensor(sx.species, dtype=torch.int32, device=dev)
            cx = torch.tensor(sx.cell, device=dev)
            rec = {"atoms": sx.n_atoms, "unit": UNIT}
            for prec in (args.precision, "fp32"):
                mx = Allegro(bx, precision=prec, device=local)
                mx.set_stream(stream.cuda_stream)
                ox = dict(E=torch.empty(1, dtype=torch.float64, device=dev),
                          E_atom=torch.empty(sx.n_atoms, dtype=torch.float64, device=dev),
                          F=torch.empty(sx.n_atoms, 3, dtype=torch.float64, device=dev),
                          virial=torch.empty(1, 3, 3, dtype=torch.float64, device=dev))
                for _ in range(3):
                    mx.neighbors(px, tx, cx)
                    mx.energy_forces(out=ox)
                torch.cuda.synchronize()
                kx = 20 if name == "c2" else 50
                ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ea.record(stream)
                for _ in range(kx):
                    mx.neighbors(px, tx, cx)
                    mx.energy_forces(out=ox)
                eb.record(stream)
                torch.cuda.synchronize()
                msx = ea.elapsed_time(eb) / kx
                rec["edges"] = mx.n_edges
                rec[prec] = {"ms_per_step": msx, "atom_steps_per_s": sx.n_atoms / (msx * 1e-3)}
                mx.close()
            extra[label] = rec
        # Table IV of the paper on GB300: relative speed of the precision settings on a 3,072-atom
        # water-density box (float64 final sums throughout; weights and activations float32 for the
        # TF32 and FP32 rows), and each setting's force error against the FP64 oracle
        extra["table_iv_3072_atoms"] = _precision_matrix(args, local, stream)
        # the paper's production architecture (1024-wide MLPs, per-pair cutoffs, ZBL)
        extra["paper_model_262144_atoms"] = _paper_model(args, local, stream)
        # the largest configuration: 3 layers, l_max 3, 128 channels on 4,194,304 atoms
        extra["c5_4194304_atoms"] = _c5_run(args, local, stream)
        # the headline box under the paper's per-ordered-species-pair cutoffs
        if arch.pair_rc is None:
            extra["pair_cutoffs_1M_atoms" if args.config == "c4" and not args.atoms else "pair_cutoffs"] = \
                _pair_cutoff_run(args, make, pos, types, cell, out, N, max(1, min(args.steps, 5)))

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"bf16": "bf16", "tf32": "tf32", "fp8": "e4m3"}.get(args.precision, "f32"), "data": "synthetic",
            "config": {"workload": _workload(args, s), "atoms": N, "edges": n_edges,
                       "step": "neighbour rebuild + E + F + virial, float64 reductions",
                       "l2": "inputs larger than L2 (edge arrays of several GB per step)",
                       "parallelism": f"replicas x{ws}"},
            "clocks": clk,
            "e2e": {"value": N * ws / e2e_max, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches1 - launches0),
            "roofline": _roofline(report, ms * args.steps, args.steps, n_edges, arch, N)}
    line["ef_only"] = ef_only
    if fp32:
        line["fp32"] = fp32
    if fp8:
        line["fp8"] = fp8
    line.update(extra)
    if rank == 0 and ws == 1 and not args.skip_cpu:
        models = {args.precision: m}
        if m32 is not None:
            models["fp32"] = m32
        if m8 is not None:
            models["fp8"] = m8
        cpu, ferr = _cpu_baseline(arch, w, blob, models)
        line["cpu_baseline"] = cpu
        line["force_err_vs_fp64"] = ferr
    if rank == 0:
        print(json.dumps(line), flush=True)
    m.close()
    if m32 is not None:
        m32.close()
    if m8 is not None:
        m8.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c4")
    ap.add_argument("--atoms", type=int, default=0, help="scale the configuration's box to this many atoms "
                                                           "(same density; lattice configurations)")
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32", "tf32", "fp8"])
    ap.add_argument("--fp32-steps", type=int, default=3)
    ap.add_argument("--skip-fp32", action="store_true")
    ap.add_argument("--skip-fp8", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--chunk-edges", type=int, default=0, help="edges per model pass (0 = automatic)")
    ap.add_argument("--skip-extra", action="store_true", help="skip the batched-molecule and MD context runs")
    ap.add_argument("--pair-cutoffs", action="store_true",
                    help="per-ordered-species-pair cutoffs of the paper's production model (H-H 3.0, H-C 1.25, "
                         "H-O 1.25, O-H 3.0 A, every other pair the model cutoff)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
