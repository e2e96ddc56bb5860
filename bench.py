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


def _roofline(report: dict, step_ms_total: float, steps: int = 1, n_edges: int = 0):
    """Dominant kernel (largest total time) of the timed region against its roofline."""
    if not report:
        return None
    detail = report
    report = _by_kernel(report)
    name, r = max(report.items(), key=lambda kv: kv[1]["ms"])
    peaks = _peaks()
    tensor = name.startswith("gemm_tc")
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    tc_peak = peaks["bf16_tflops_sustained"] if peaks else 1700.0
    tc_ctx = None
    bound = "hbm"
    if tensor:
        # the MLP GEMMs' arithmetic intensity (algorithmic FLOPs per algorithmic byte)
        # decides which roof binds them: below the ridge point it is HBM
        intensity = r["flops"] / max(r["bytes"], 1.0)
        ridge = tc_peak * 1e12 / (hbm_peak * 1e9)
        tflops = r["flops"] / (r["ms"] * 1e-3) / 1e12
        tc_ctx = {"achieved_tflops": round(tflops, 2), "peak_tflops": tc_peak, "frac": round(tflops / tc_peak, 4),
                  "arithmetic_intensity_flop_per_byte": round(intensity, 1),
                  "ridge_flop_per_byte": round(ridge, 1)}
        bound = "tensor" if intensity >= ridge else "hbm"
    if bound == "tensor":
        peak, achieved, unit = tc_peak, r["flops"] / (r["ms"] * 1e-3) / 1e12, "TFLOP/s"
    else:
        peak, achieved, unit = hbm_peak, r["bytes"] / (r["ms"] * 1e-3) / 1e9, "GB/s"
    share = {k: round(v["ms"] / max(step_ms_total, 1e-9), 4) for k, v in
             sorted(report.items(), key=lambda kv: -kv[1]["ms"])}
    return {"kernel": name, "bound": bound, "achieved": round(achieved, 2), "peak": peak, "unit": unit,
            "frac": round(achieved / peak, 4), "peak_source": "measured" if peaks else "fallback",
            "traffic": _traffic_per_launch(detail, steps, n_edges) if tensor else None,
            "traffic_unit": "bytes per launch (DRAM read + write)",
            "algorithmic_bytes_per_launch": r["bytes"] / max(r["launches"], 1),
            "launches": r["launches"], "ms_per_launch": round(r["ms"] / max(r["launches"], 1), 5),
            "tensor": tc_ctx,
            "share_of_timed_region": share,
            "gemm_detail": {k.split("/", 1)[1]: {
                                                 "share": round(v["ms"] / max(step_ms_total, 1e-9), 4),
                                                 "TFLOP/s": round(v["flops"] / (v["ms"] * 1e-3) / 1e12, 1),
                                                 "GB/s": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1)}
                            for k, v in sorted(detail.items(), key=lambda kv: -kv[1]["ms"]) if "/" in k}}


def _cpu_baseline(arch, w, blob, precision_models: dict):
    """FP64 oracle on a bounded sample (the 4,096-atom box of the same density and model),
    and the GPU paths' force errors against it on that sample."""
    import numpy as np
    import torch
    from oracle.allegro import AllegroOracle
    from synth import make_config
    torch.set_num_threads(os.cpu_count() or 1)
    s, _, _ = make_config("c4sub")
    t0 = time.perf_counter()
    i, j, S = _edges(arch, s)
    E0, Ea0, F0, W0 = AllegroOracle(arch, w).energy_forces(s.pos, s.species, s.cell, i, j, S)
    dt = time.perf_counter() - t0
    errs = {}
    rms = float(np.sqrt((F0 ** 2).mean()))
    for prec, m in precision_models.items():
        m.neighbors(s.pos, s.species, s.cell)
        out = m.energy_forces()
        F = out["F"].cpu().numpy()
        errs[prec] = {"force_rms_err_over_rms_F": float(np.sqrt(((F - F0) ** 2).mean()) / rms),
                      "force_max_err_over_rms_F": float(np.abs(F - F0).max() / rms),
                      "E_rel_err": float(abs(out["E"].item() - E0) / abs(E0))}
    return {"value": s.n_atoms / dt, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"1 step (neighbours + E + F + virial) of the {s.n_atoms}-atom periodic box at the "
                      f"same density and model ({len(i)} edges), FP64 torch on the host cores",
            "seconds": round(dt, 3)}, {"sample": "4,096-atom box, all atoms", "fp64_oracle_rms_F": rms, **errs}


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

    def make(prec):
        m = Allegro(blob, precision=prec, device=local)
        m.set_stream(stream.cuda_stream)
        if args.chunk_edges:
            m.reserve(0, 0, False, args.chunk_edges)
        if arch.pair_rc is not None:
            m.set_pair_cutoffs(arch.pair_rc)
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

    # ---- context workloads: batched uneven molecules, and an MD run with 1 fs steps ----
    extra = {}
    if not args.skip_extra:
        from synth import molecule_batch, lattice_box
        from synth.structures import pack
        import numpy as np
        mols = molecule_batch(2048, seed=2)
        mpos, mspec, moffs = pack(mols)
        bt = {}
        for prec in (args.precision, "fp32"):
            mb = make(prec)
            mb.neighbors_batched(moffs, mpos, mspec)
            mb.energy_forces()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(3):
                mb.neighbors_batched(moffs, mpos, mspec)
                mb.energy_forces()
            torch.cuda.synchronize()
            bt[prec] = len(mpos) * 3 / (time.perf_counter() - t0)
            ne = mb.n_edges
            mb.close()
        extra["batched_2048_molecules"] = {
            "atoms": int(len(mpos)), "edges": int(ne), "unit": UNIT, args.precision: bt[args.precision],
            "fp32": bt["fp32"], "note": "2048 gas-phase molecules of 8-64 atoms in one packed edge list, "
                                        "per-molecule E/F/virial; host inputs each step"}
        s2, _, _ = make_config("c2")
        masses = np.array([1.008, 15.999, 12.011, 14.007, 32.06])
        rng = np.random.default_rng(0)
        vel = rng.normal(size=(s2.n_atoms, 3)) * np.sqrt(0.0257 * 9.648533212e-3 / masses[s2.species][:, None])
        mm = make(args.precision)
        p2 = s2.pos.copy()
        mm.md_verlet(p2, vel, s2.species, masses, 1.0, 2, cell=s2.cell)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nmd = 10
        Ep, Ek = mm.md_verlet(p2, vel, s2.species, masses, 1.0, nmd, cell=s2.cell)
        torch.cuda.synchronize()
        dt_md = time.perf_counter() - t0
        mm.close()
        extra["md_23552_atoms"] = {"dt_fs": 1.0, "steps": nmd, "timesteps_per_s": nmd / dt_md,
                                   "atom_steps_per_s": s2.n_atoms * nmd / dt_md,
                                   "energy_drift_eV_per_atom": float(abs((Ep[-1] + Ek[-1]) - (Ep[0] + Ek[0])) / s2.n_atoms),
                                   "note": "velocity Verlet on the GPU, neighbour rebuild every step"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16" if args.precision == "bf16" else "f32", "data": "synthetic",
            "config": {"workload": _workload(args, s), "atoms": N, "edges": n_edges,
                       "step": "neighbour rebuild + E + F + virial, float64 reductions",
                       "l2": "inputs larger than L2 (edge arrays of several GB per step)",
                       "parallelism": f"replicas x{ws}"},
            "clocks": clk,
            "e2e": {"value": N * ws / e2e_max, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches1 - launches0),
            "roofline": _roofline(report, ms * args.steps, args.steps, n_edges)}
    if fp32:
        line["fp32"] = fp32
    line.update(extra)
    if rank == 0 and ws == 1 and not args.skip_cpu:
        models = {args.precision: m}
        if m32 is not None:
            models["fp32"] = m32
        cpu, ferr = _cpu_baseline(arch, w, blob, models)
        line["cpu_baseline"] = cpu
        line["force_err_vs_fp64"] = ferr
    if rank == 0:
        print(json.dumps(line), flush=True)
    m.close()
    if m32 is not None:
        m32.close()
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
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--fp32-steps", type=int, default=3)
    ap.add_argument("--skip-fp32", action="store_true")
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
