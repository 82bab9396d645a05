"""Benchmark of the qNEP force call on one GB300 (or N replicas under torchrun).

Default workload (the batched form): 512 LLZO-shaped cells of 192-1536 atoms under
64 candidate parameter vectors, every (structure, candidate) force call (energy,
forces, charges; Ewald per cell) in one persistent launch replayed from a CUDA
graph.  value = atom-evaluations per second.  The line also carries the plain
FP32 single-structure path on the same structures, the precision form (BF16 /
TF32 network on the tensor cores) against FP32 on 8000 waters with PPPM, the
item kernel's roofline (CUDA events around it) and the FP64 oracle on the host.

Single-structure workloads (--workload batio3 | water_pppm, --precision): one full
force call per step (forces, virial, BEC, polarization).  Inputs are resident in
HBM; L2 is flushed (a 512 MB write) between timed steps, outside the timed events.
The JSON line carries value, roofline (dominant kernel against the measured peak), cpu_baseline
(the FP64 oracle on the host cores), e2e (host buffers, copies inside the timed region), clocks
(nvidia-smi samples during the timed region) and gpu_launches.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "qNEP force-call atom-steps/s on 1 GB300 (mixed/batched vs FP32) at stated error"
UNIT = "atom-steps/s"
WORKLOADS = {
    "batio3": ("BaTiO3 10x10x10 perovskite, 5000 atoms, 3 species; NEP 6/4 A, n_max 4/4, basis 8, l_max 4 + "
               "4-body, 30 tanh units x 2 outputs; Ewald alpha 0.3, r_c 6 A, k_max 2.230 (1e-6), mode 1; "
               "forces + virial + BEC + polarization, FP32 path"),
    "water_pppm": ("liquid water 8000 H2O (24,000 atoms) at 1.0 g/cm3, 2 species; same descriptor / network; "
                   "PPPM mesh 64^3, order 5, alpha 0.3, r_c 6 A, mode 1; forces + virial + BEC + polarization, "
                   "FP32 path"),
}
WORKLOADS["llzo_batch"] = (
    "512 LLZO-shaped cells (Li/La/Zr/O 7:3:2:12, 1x1x1..2x2x2 supercells of a random 12.97 A 192-atom cell, "
    "192-1536 atoms, N(0, 0.1 A) moves) x 64 candidate parameter vectors N(0, 0.1), 4 species; same descriptor / "
    "network; Ewald per cell alpha 0.3, r_c 6 A, k_max 2.230, mode 1; energy, forces and charges per "
    "(structure, candidate), FP32 path, one persistent launch")
WORKLOADS["mgwater_nve"] = (
    "Mg-water interface: hcp Mg slab (a 3.21, c 5.21 A, 15 layers) under 60 A of water at 1.0 g/cm3, "
    "112 x 65 orthohexagonal cells, ~1.0 M atoms, 3 species; same descriptor; network BF16 on the tensor "
    "cores; PPPM mesh 256 x 256 x 384, order 5, alpha 0.3, r_c 6 A, mode 1; NVE velocity Verlet 0.5 fs "
    "from 300 K Maxwell-Boltzmann; a step = one MD step (force call + two half kicks + drift)")
WORKLOAD = WORKLOADS["batio3"]
WORKLOADS["field_response"] = (
    "external-field force F^ext_i = E . Z_i and polarization current Pdot = sum_i Z_i v_i (Sec. II.D) over "
    "4,194,304 atoms: Born effective charges [N][3][3], velocities and forces [N][3] float32 (252 MB, > L2), "
    "one qnep_field_response launch per step")


def _config(name):
    from paper_2601_19034_gb300 import workloads
    return {"batio3": workloads.config_batio3, "water_pppm": workloads.config_water_pppm,
            "llzo_batch": workloads.config_llzo_batch}[name]()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self, sm_max_default: float) -> dict:
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else sm_max_default,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _reduce_max(x: float, device=None) -> float:
    """Max over the ranks of the job (the timing rule); the identity on one process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _batch_seed(rank: int) -> int:
    """Each rank of a multi-GPU batched run evaluates its own batch (independent structures)."""
    return 1003 + 7919 * rank


def _ewald_kcount(box, kmax):
    """Half-space k vectors with |k| < kmax (for the algorithmic operation count), k = 2 pi H^-1 n
    for the cell with rows H (any cell; |n_d| <= kmax |a_d| / 2 pi)."""
    box = np.asarray(box, dtype=np.float64)
    nmax = [int(math.floor(kmax * np.linalg.norm(box[d]) / (2 * math.pi))) for d in range(3)]
    g = np.meshgrid(*[np.arange(-m, m + 1) for m in nmax], indexing="ij")
    n = np.stack([x.ravel() for x in g], 1)
    k = 2 * math.pi * n @ np.linalg.inv(box).T
    k2 = (k * k).sum(1)
    return int(((k2 > 0) & (k2 < kmax * kmax)).sum()) // 2


# DRAM bytes (read + write) of the batched item kernel per atom-evaluation, from one ncu
# capture of the current kernel (tensor-core form) on the first 160 structures x 64
# candidates (10.330 GB read + 7.348 GB written for 6,709,248 atom-evaluations; the traffic grows
# with the atom-evaluations).  Set to None when the item kernel changes until it is captured again.
ITEM_DRAM_BYTES_PER_EVAL = (10.329806e9 + 7.348257e9) / 6709248
ITEM_DRAM_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_batch_items launch on the "
                    "first 160 structures x 64 candidates, scaled by atom-evaluations")


def _time_single(model, sysm, dev, steps, warmup, flush, want=None):
    """CUDA-graph replay of one force call; L2 flushed between calls; event-timed ms per call."""
    import torch
    want = want or {}
    pos = torch.tensor(sysm.positions, device=dev)
    typ = torch.tensor(sysm.types, device=dev)
    model.reserve(sysm.n_atoms, sysm.box)
    out = model.compute(pos, typ, sysm.box, **want)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        for _ in range(3):
            model.compute_into(pos, typ, sysm.box, out, stream=stream.cuda_stream)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        model.compute_into(pos, typ, sysm.box, out, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    for _ in range(warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
            graph.replay()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.zero_()
            starts[k].record(stream)
            graph.replay()
            ends[k].record(stream)
    torch.cuda.synchronize()
    return float(np.median([a.elapsed_time(b) for a, b in zip(starts, ends)])), out


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2601_19034_gb300 import workloads
    from paper_2601_19034_gb300.qnep import QNEP, parse_scalars

    world, rank, local = _dist()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sysm, hp, params, elec = _config(args.workload)
    n = sysm.n_atoms
    model = QNEP(hp, params, elec, precision=args.precision)
    pos = torch.tensor(sysm.positions, device=dev)
    typ = torch.tensor(sysm.types, device=dev)
    model.reserve(n, sysm.box)
    # capacity check (and list growth) before capture
    out = model.compute(pos, typ, sysm.box)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(3):
            model.compute_into(pos, typ, sysm.box, out, stream=stream.cuda_stream)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        model.compute_into(pos, typ, sysm.box, out, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
            graph.replay()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    peaks, peak_kind = _peaks()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.zero_()
                starts[k].record(stream)
                graph.replay()
                ends[k].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = float(sum(step_ms))
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * n * args.steps / (total_ms * 1e-3)

    # parity spot-check of the timed graph's output (energy per atom, finite forces)
    sc = parse_scalars(out["scalars"])
    status = int(sc["status"])

    # per-stage device times (events on the launching stream), eager launches
    model.set_profiling(True)
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            model.compute_into(pos, typ, sysm.box, out, stream=stream.cuda_stream)
    stages, calls = model.stage_times()
    model.set_profiling(False)
    stage_avg = {k: v / max(calls, 1) for k, v in stages.items()}

    # end to end: host buffers through the C ABI (copies in and out timed)
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        model.compute_host(sysm.positions, sysm.types, sysm.box)
        dt = time.perf_counter() - t
        if k >= args.warmup:
            e2e_ms.append(dt * 1e3)
    h2d = n * 3 * 4 + n * 4
    d2h = 20 * 8 + n * 3 * 4 + n * 9 * 4 + n * 4

    clocks = clk.summary(peaks.get("sm_max_mhz", 2070.0))
    line = None
    if rank == 0:
        roof = _roofline(stage_avg, sysm, hp, elec, clocks, peaks, peak_kind) if elec.kind == "ewald" else \
            _roofline_generic(stage_avg, sysm, clocks, peaks)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 reductions)", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "atoms": n, "l2": "flushed between steps (512 MB write)",
                       "launch": "CUDA graph replay of one qnep_compute", "parallelism": "replicas" if world > 1
                       else "single GPU", "wall_s": wall},
            "stage_ms": stage_avg,
            "roofline": roof,
            "e2e": {"value": n / (statistics.median(e2e_ms) * 1e-3) * world, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": statistics.median(e2e_ms)},
            "gpu_launches": KERNELS_PER_CALL * args.steps,
            "clocks": clocks,
            "device_status": status,
            "energy_per_atom": sc["energy"] / n,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = _cpu_baseline(sysm, hp, params, elec, reps=1)
    if world > 1:
        dist.destroy_process_group()
    return line


def _fp32_peak(mhz):
    """FP32 FMA peak (TFLOP/s) of the current device at the sampled SM clock, and how it was formed."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count \
        if torch.cuda.is_available() else 152
    return sms * 128 * 2 * mhz * 1e6 / 1e12, f"derived: {sms} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz (sampled)"


# kernels of one Ewald force call with forces + BEC (warp-per-atom path): k_bin, k_scan,
# k_fill, k_order, k_nbr_desc_coop, k_real (second stream), k_sk (with its fused
# finalisation), k_field_k, k_desc_bwd_coop, k_finalize
KERNELS_PER_CALL = 10


def _roofline(stage_avg, sysm, hp, elec, clocks, peaks, peak_kind):
    """Roofline of the dominant kernel from its live CUDA-event duration."""
    name = max(stage_avg, key=stage_avg.get)
    ms = stage_avg[name]
    n = sysm.n_atoms
    nk = _ewald_kcount(sysm.box, elec.kmax)
    mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak, peak_src = _fp32_peak(mhz)
    if name in ("field_kspace", "ewald_structure_factor"):
        # algorithmic FP32 work: per (atom, half-space k) one complex multiply-accumulate
        # for S(k) (8 flop) or potential + force (16 flop)
        flop = n * nk * (16 if name == "field_kspace" else 8)
        achieved = flop / (ms * 1e-3) / 1e12
        return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": None, "ms": ms,
                "peak_source": peak_src,
                "work": f"{n} atoms x {nk} half-space k"}
    flop = n * FLOP_PER_ATOM.get(name, 0)
    achieved = flop / (ms * 1e-3) / 1e12
    return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak, "traffic": None, "ms": ms,
            "peak_source": peak_src}


def _roofline_generic(stage_avg, sysm, clocks, peaks):
    # the dominant stage among those with an algorithmic operation count (the descriptor kernels)
    counted = {k: v for k, v in stage_avg.items() if k in FLOP_PER_ATOM} or stage_avg
    name = max(counted, key=counted.get)
    ms = stage_avg[name]
    mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak, peak_src = _fp32_peak(mhz)
    flop = sysm.n_atoms * FLOP_PER_ATOM.get(name, 0)
    achieved = flop / (ms * 1e-3) / 1e12
    return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak, "traffic": None, "ms": ms,
            "peak_source": peak_src}


# algorithmic FP32 flop per atom of the descriptor kernels at the BaTiO3 neighbour counts (68 list and
# 18 angular entries per atom): forward radial 68 x 30 + angular 18 x 230 + network 3 x 900; backward
# radial 68 x 40 + angular 18 x 2 x 700
FLOP_PER_ATOM = {"descriptor_forward": 18000, "descriptor_backward": 45000}


def _cpu_baseline(sysm, hp, params, elec, reps=1):
    import torch

    from oracle import forcecall
    cores = torch.get_num_threads()
    t = time.perf_counter()
    for _ in range(reps):
        forcecall.force_call(sysm.positions.astype(np.float64), sysm.box, sysm.types, hp, params, elec)
    dt = (time.perf_counter() - t) / reps
    return {"value": sysm.n_atoms / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps} full force call(s) of the same workload (FP64 oracle, torch CPU threads={cores})"}


def run_reference(args):
    """The FP64 oracle timed on the host cores on this workload (rank 0 only)."""
    world, rank, _ = _dist()
    if rank != 0:
        return None
    import torch

    from oracle import forcecall
    from paper_2601_19034_gb300 import workloads
    cores = torch.get_num_threads()
    if args.workload == "llzo_batch":
        return _reference_batch(args, world, cores)
    if args.workload == "field_response":
        # bounded sample: 262,144 atoms of the same synthetic Z and v per step
        from oracle import field
        n = 262144
        rng = np.random.default_rng(7)
        z = rng.normal(size=(n, 3, 3)).astype(np.float32)
        v = (rng.normal(size=(n, 3)) * 0.02).astype(np.float32)
        e = np.array([0.12, 0.05, -0.33])
        times = []
        for k in range(args.warmup + args.steps):
            t = time.perf_counter()
            field.electric_force(z, e)
            field.polarization_current(z, v)
            if k >= args.warmup:
                times.append(time.perf_counter() - t)
        value = n * len(times) / sum(times)
        return {"impl": "reference", "metric": "qNEP field response (E.Z_i, sum_i Z_i v_i) atoms/s",
                "value": value, "unit": "atoms/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": sum(times) / len(times) * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOADS["field_response"]},
                "cpu_baseline": {"value": value, "unit": "atoms/s", "cores": cores, "kind": "oracle",
                                 "sample": f"each step the oracle's two contractions over {n} atoms"},
                "e2e": {"value": value, "unit": "atoms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if args.workload == "mgwater_nve":
        # bounded sample: each step one force call of a 3297-atom slab of the same construction
        sy0, hp, params, _ = workloads.config_mg_water(nx=6, ny=4)
        sysm = workloads.mg_water_interface(6, 4, seed=77)
        elec = workloads.Elec(mode=1, kind="pppm", mesh=(20, 24, 100), order=5)
        times = []
        for k in range(args.warmup + args.steps):
            t = time.perf_counter()
            forcecall.force_call(sysm.positions.astype(np.float64), sysm.box, sysm.types, hp, params, elec,
                                 want_bec=False)
            if k >= args.warmup:
                times.append(time.perf_counter() - t)
        value = sysm.n_atoms * len(times) / sum(times)
        return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(times) / len(times) * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": WORKLOADS["mgwater_nve"]},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": f"each step one force call of a {sysm.n_atoms}-atom slab"},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    sysm, hp, params, elec = _config(args.workload)
    times = []
    for k in range(args.warmup + args.steps):
        t = time.perf_counter()
        forcecall.force_call(sysm.positions.astype(np.float64), sysm.box, sysm.types, hp, params, elec)
        dt = time.perf_counter() - t
        if k >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = sysm.n_atoms * len(times) / total
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / len(times) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload], "atoms": sysm.n_atoms},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "each step one full force call of the workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# kernels of one batched call: k_batch_sort, k_batch_lists, k_batch_items
BATCH_KERNELS_PER_CALL = 3


def _batch_flop(systems, hp, elec, n_cand):
    """Algorithmic FP32 flop of one batched call (per (atom, candidate) counts below).

    Neighbour counts are the density estimates 4/3 pi r_c^3 rho of each structure.
    Per (atom, candidate): descriptor contractions 2 S (K_R N_R + K_A N_A N_lm),
    network 2 (N_neu N_des) x 3 (forward, dU/dD, dq/dD), radial backward 24 per pair,
    angular backward 840 per pair, real space 8 per pair, Ewald 14 per half-space k.
    """
    S = hp.n_species
    total = 0.0
    for sy in systems:
        vol = abs(float(np.linalg.det(np.asarray(sy.box, dtype=np.float64))))
        rho = sy.n_atoms / vol
        n_r = 4.0 / 3.0 * math.pi * hp.rc_radial ** 3 * rho
        n_a = 4.0 / 3.0 * math.pi * hp.rc_angular ** 3 * rho
        nk = _ewald_kcount(sy.box, elec.kmax)
        per = (2 * S * (hp.basis_radial * hp.n_radial + hp.basis_angular * hp.n_angular * 24)
               + 6 * hp.n_neurons * hp.n_des + 24 * n_r + 840 * n_a + 8 * n_r + 14 * nk)
        total += sy.n_atoms * n_cand * per
    return total


# DRAM bytes of one k_field_response launch (forces + Pdot, 4,194,304 atoms) from the ncu capture of
# the current kernel (dram__bytes_read.sum / write.sum): 211.97 MB read + 30.22 MB written (the rest of
# the 50 MB of forces is still in L2 when the kernel ends); None whenever the kernel changes
FIELD_DRAM_BYTES = 211.97e6 + 30.22e6
FIELD_BYTES_PER_ATOM = 36 + 12 + 12      # read Z and v, write F^ext


def _time_field_response(dev, flush, peaks, reps):
    """qnep_field_response (forces and Pdot) on FIELD_RESPONSE_ATOMS atoms; HBM roofline.

    CUDA events on torch's current stream, which the call launches on; L2 flushed
    before every timed call.  Returns the roofline object and the call times (ms).
    """
    import torch

    from paper_2601_19034_gb300 import workloads
    from paper_2601_19034_gb300.qnep import field_response

    n = workloads.FIELD_RESPONSE_ATOMS
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    z = torch.randn(n, 3, 3, device=dev, generator=g)
    v = torch.randn(n, 3, device=dev, generator=g) * 0.02
    f = torch.empty(n, 3, device=dev)
    pdot = torch.empty(3, dtype=torch.float64, device=dev)
    efield = (0.12, 0.05, -0.33)
    for _ in range(3):
        field_response(z, efield, v, forces=f, pdot=pdot)
    torch.cuda.synchronize()
    cur = torch.cuda.current_stream(dev)

    def timed(flush_between):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        for k in range(reps):
            if flush_between:
                flush.zero_()
            starts[k].record(cur)
            field_response(z, efield, v, forces=f, pdot=pdot)
            ends[k].record(cur)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in zip(starts, ends)]

    # the inputs (252 MB) exceed the 129 MB L2, so consecutive calls are timed without a flush; a
    # 512 MB write between calls leaves up to 129 MB of dirty lines whose write-back then falls
    # inside the next call (reported beside it)
    times = timed(False)
    flushed = timed(True)
    ms = float(np.median(times))
    algo = n * FIELD_BYTES_PER_ATOM
    achieved = algo / (ms * 1e-3) / 1e9
    peak = peaks["hbm_gbs"]
    del z, v, f
    return {"kernel": "k_field_response", "atoms": n, "bound": "hbm", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "ms": ms, "traffic": FIELD_DRAM_BYTES,
            "work": f"{algo} algorithmic bytes per launch ({FIELD_BYTES_PER_ATOM} B per atom: Z 36, v 12, F 12)",
            "timing": "median of CUDA-event times of consecutive single calls (memset of Pdot + one kernel); "
                      "inputs larger than L2, no flush",
            "ms_after_write_flush": float(np.median(flushed))}, times


def _time_snes_step(b, graph, stream, out, off, params, dev, reps):
    """Median time (ms) of one training iteration on the device: randn, sample, set_params,
    batched call (graph replay), loss (weights 1, 1, 0, 1e-6), SNES update."""
    import torch

    from paper_2601_19034_gb300.qnep import batch_loss, snes_sample, snes_update

    c, p = params.shape
    mu = torch.tensor(params.mean(0), dtype=torch.float32, device=dev)
    sigma = torch.full((p,), 0.01, dtype=torch.float32, device=dev)
    noise = torch.empty(c, p, dtype=torch.float32, device=dev)
    z = torch.empty(c, p, dtype=torch.float32, device=dev)
    off_d = torch.tensor(np.asarray(off, dtype=np.int32), device=dev)
    with torch.cuda.stream(stream):
        graph.replay()
        e_ref = out["energy"][0].clone()
        f_ref = out["forces"][0].clone()
    loss = torch.empty(c, dtype=torch.float64, device=dev)
    terms = torch.empty(c, 4, dtype=torch.float64, device=dev)
    names = ("normal_deviates", "snes_sample", "set_params", "batched_call", "batch_loss", "snes_update")
    times, parts = [], {k: [] for k in names}
    with torch.cuda.stream(stream):
        for k in range(reps + 2):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
            ev[0].record(stream)
            noise.normal_()
            ev[1].record(stream)
            snes_sample(mu, sigma, noise, out=z, stream=stream.cuda_stream)
            ev[2].record(stream)
            b.set_params(z, stream=stream.cuda_stream)
            ev[3].record(stream)
            graph.replay()
            ev[4].record(stream)
            batch_loss(out["energy"], out["forces"], e_ref, f_ref, off_d, z, (1.0, 1.0, 0.0, 1e-6), loss=loss,
                       terms=terms, stream=stream.cuda_stream)
            ev[5].record(stream)
            snes_update(loss, noise, mu, sigma, stream=stream.cuda_stream)
            ev[6].record(stream)
            ev[6].synchronize()
            if k >= 2:
                times.append(ev[0].elapsed_time(ev[6]))
                for q, name in enumerate(names):
                    parts[name].append(ev[q].elapsed_time(ev[q + 1]))
    b.set_params(torch.tensor(params, dtype=torch.float32, device=dev), stream=stream.cuda_stream)
    stream.synchronize()
    ms = float(np.median(times))
    stage_ms = {k: float(np.median(v)) for k, v in parts.items()}
    # the loss pass streams the candidates' forces once (12 B per atom and candidate); the reference
    # forces (12 B per atom) are re-read per candidate from L2, the energies and parameters are small
    n_total = int(out["forces"].shape[1])
    loss_bytes = c * n_total * 12 + n_total * 12 + c * (len(off) - 1) * 8 + c * p * 4
    loss_gbs = loss_bytes / (stage_ms["batch_loss"] * 1e-3) / 1e9
    hbm = _peaks()[0]["hbm_gbs"]
    return {"ms": ms, "stage_ms": stage_ms, "loss_best": float(loss.min().item()),
            "batch_loss_roofline": {"kernel": "k_batch_loss (+ memset, k_loss_finalize)", "bound": "hbm",
                                    "achieved": loss_gbs, "peak": hbm, "unit": "GB/s", "frac": loss_gbs / hbm,
                                    "work": f"{loss_bytes} algorithmic bytes per call"},
            "what": "normal deviates + qnep_snes_sample + qnep_batch_set_params + batched call (graph replay) "
                    "+ qnep_batch_loss + qnep_snes_update, CUDA events on the call's stream, median"}


def _time_plain_single(hp, params0, elec, systems, dev, stream, flush):
    """Single-structure FP32 calls (forces + charges) on the given structures, candidate 0."""
    import torch
    from paper_2601_19034_gb300.qnep import QNEP
    models, graphs, outs = {}, [], []
    eager_ms = 0.0
    for sy in systems:
        key = tuple(np.round(np.diag(sy.box), 6))
        if key not in models:
            models[key] = QNEP(hp, params0, elec)
            models[key].reserve(max(x.n_atoms for x in systems), sy.box)
        m = models[key]
        p1, t1 = torch.tensor(sy.positions, device=dev), torch.tensor(sy.types, device=dev)
        o1 = m.compute(p1, t1, sy.box, bec=False, virial=False)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(3):
            m.compute_into(p1, t1, sy.box, o1)
        ev1.record()
        ev1.synchronize()
        eager_ms += ev0.elapsed_time(ev1) / 3
        with torch.cuda.stream(stream):
            m.compute_into(p1, t1, sy.box, o1, stream=stream.cuda_stream)
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            m.compute_into(p1, t1, sy.box, o1, stream=stream.cuda_stream)
        graphs.append(g)
        outs.append((p1, t1, o1))
    torch.cuda.synchronize()
    times = []
    for k in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.zero_()
            e0.record(stream)
            for g in graphs:
                g.replay()
            e1.record(stream)
        e1.synchronize()
        if k:
            times.append(e0.elapsed_time(e1))
    for m in models.values():
        m.close()
    atoms = int(sum(sy.n_atoms for sy in systems))
    ms = float(np.median(times))
    return {"value": atoms / (ms * 1e-3), "unit": UNIT, "ms": ms,
            "eager_value": atoms / (eager_ms * 1e-3), "eager_ms": eager_ms,
            "what": f"single-structure qnep_compute (forces + charges), one call per structure on the first "
                    f"{len(systems)} structures, candidate 0: each call a CUDA graph (one model per box shape), "
                    f"replayed back to back after one L2 flush (median of 3); eager calls beside it"}


def _time_with_virial(b, pos_d, typ_d, off, boxes, stream, flush, steps, evals, bec=False):
    """The headline batched call with the per-(candidate, structure) virial as well (and, with
    bec, the per-atom Born effective charges and the uncorrected total charges: every input of
    the full training loss)."""
    import torch
    out = b.outputs(len(off) - 1, pos_d.shape[0], pos_d.device, virial=True, bec=bec, total_charge=bec,
                    polarization=bec)
    b.compute_into(pos_d, typ_d, off, boxes, out)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        b.compute_into(pos_d, typ_d, off, boxes, out, stream=stream.cuda_stream)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        b.compute_into(pos_d, typ_d, off, boxes, out, stream=stream.cuda_stream)
    ts = []
    for k in range(steps + 3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.zero_()
            e0.record(stream)
            g.replay()
            e1.record(stream)
        e1.synchronize()
        if k >= 3:
            ts.append(e0.elapsed_time(e1))
    ms = float(np.median(ts))
    what = ("the same graph-replayed batched call writing energies, forces, charges and the 3x3 virial "
            "of every (candidate, structure) (qnep_batch_compute_outputs)")
    if bec:
        what += (", the 3x3 Born effective charge of every atom, the polarization and the total charge before "
                 "the correction of every (candidate, structure)")
    del out, g
    return {"ms_per_step": ms, "value": evals / (ms * 1e-3), "unit": UNIT, "what": what}


def _time_other_contraction(hp, params, elec, pos_d, typ_d, off, boxes, stream, flush, contract, steps, evals):
    """The same batched call with the other descriptor contraction (graph replay, L2 flushed)."""
    import torch
    from paper_2601_19034_gb300.qnep import QNEPBatch
    b2 = QNEPBatch(hp, params, elec)
    b2.set_contraction(contract)
    b2.set_config(8, "largest_first")
    out2 = b2.compute(pos_d, typ_d, off, boxes)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        b2.compute_into(pos_d, typ_d, off, boxes, out2, stream=stream.cuda_stream)
    stream.synchronize()
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2, stream=stream):
        b2.compute_into(pos_d, typ_d, off, boxes, out2, stream=stream.cuda_stream)
    ts = []
    for k in range(steps + 3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.zero_()
            e0.record(stream)
            g2.replay()
            e1.record(stream)
        e1.synchronize()
        if k >= 3:
            ts.append(e0.elapsed_time(e1))
    b2.set_profiling(True)
    for _ in range(4):
        with torch.cuda.stream(stream):
            flush.zero_()
            b2.compute_into(pos_d, typ_d, off, boxes, out2, stream=stream.cuda_stream)
    st2, calls2 = b2.stage_times()
    b2.close()
    ms = float(np.median(ts))
    return {"contraction": contract, "ms_per_step": ms, "value": evals / (ms * 1e-3), "unit": UNIT,
            "item_kernel_ms": st2["items"] / max(calls2, 1),
            "what": "same batch, warps 8, largest first, CUDA graph replay, L2 flushed, median"}


_CHUNKS = {}


def _time_atom_virial(dev, flush, steps):
    """Cost of the per-atom virial (the entry scatter, the static pair terms and the per-atom k-space
    term; with PPPM its six more inverse FFTs): the single-structure call on BaTiO3 5000 (Ewald) and
    on 8000 waters (PPPM 64^3), with and without W_i, graph replay, L2 flushed.  Never raises: a
    failure is reported in the leg."""
    from paper_2601_19034_gb300.qnep import QNEP
    res = {"what": "single-structure force call (forces, virial, BEC, P) with and without the per-atom virial"}
    for name in ("batio3", "water_pppm"):
        m = None
        try:
            sysm, hp, par, el = _config(name)
            m = QNEP(hp, par, el)
            base, _ = _time_single(m, sysm, dev, steps, 3, flush)
            av, _ = _time_single(m, sysm, dev, steps, 3, flush, want=dict(atom_virial=True))
            res[name] = {"atoms": sysm.n_atoms, "ms_per_call": base, "ms_per_call_with_atom_virial": av,
                         "cost": av / base - 1.0, "value_with_atom_virial": sysm.n_atoms / (av * 1e-3),
                         "unit": UNIT}
        except Exception as exc:   # noqa: BLE001  (a side measurement never ends the bench line)
            res[name] = {"error": f"{type(exc).__name__}: {exc}"}
        finally:
            if m is not None:
                m.close()
    return res


def _general_cells(systems, seed=11):
    """The structures with their cells sheared into the restricted form (every entry below the
    diagonal non-zero) and then turned by one random rotation: fully general cells with the same
    fractional coordinates."""
    from paper_2601_19034_gb300 import workloads
    rng = np.random.default_rng(seed)
    r, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(r) < 0:
        r[:, 0] = -r[:, 0]
    shear = np.array([[0.0, 0.0, 0.0], [0.1, 0.0, 0.0], [-0.05, 0.07, 0.0]])
    out = []
    for s_ in systems:
        box = np.asarray(s_.box, dtype=np.float64)
        cell = box + shear * np.diag(box)[:, None]
        frac = np.asarray(s_.positions, dtype=np.float64) @ np.linalg.inv(box)
        out.append(workloads.System(((frac @ cell) @ r.T).astype(np.float32), s_.types, cell @ r.T, s_.species))
    return out


def _time_general_cells(hp, params, elec, systems, dev, stream, flush, steps, evals, contract, config,
                        ortho_ms):
    """General (triclinic) cells: the batched call on the same structures in fully general cells
    (the restricted form inside the call, outputs turned back), and the single-structure call on
    BaTiO3 5000 in a sheared cell, each against its orthorhombic form.  Never raises."""
    import torch

    from paper_2601_19034_gb300.qnep import QNEP, QNEPBatch, stack_structures
    res = {"what": "cells sheared (b_x = 0.1 b_y, c_x = -0.05 c_z, c_y = 0.07 c_z) and turned by one random "
                   "rotation, same fractional coordinates"}
    g = None
    try:
        turned = _general_cells(systems)
        pos, typ, off, boxes = stack_structures(turned)
        pos_d, typ_d = torch.tensor(pos, device=dev), torch.tensor(typ, device=dev)
        g = QNEPBatch(hp, params, elec)
        g.set_contraction(contract)
        g.set_config(*config)
        out = g.compute(pos_d, typ_d, off, boxes)
        with torch.cuda.stream(stream):
            g.compute_into(pos_d, typ_d, off, boxes, out, stream=stream.cuda_stream)
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            g.compute_into(pos_d, typ_d, off, boxes, out, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        ms = []
        for k in range(3 + steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                graph.replay()
                b_.record(stream)
            torch.cuda.synchronize()
            if k >= 3:
                ms.append(a.elapsed_time(b_))
        status = g.sync_status()
        del graph
        med = float(np.median(ms))
        res["batched"] = {"ms_per_step": med, "value": evals / (med * 1e-3), "unit": UNIT,
                          "vs_orthorhombic": ortho_ms / med, "device_status": status}
    except Exception as exc:   # noqa: BLE001  (a side measurement never ends the bench line)
        res["batched"] = {"error": f"{type(exc).__name__}: {exc}"}
    finally:
        if g is not None:
            g.close()
    m = None
    try:
        sysm, hp_b, par_b, el_b = _config("batio3")
        m = QNEP(hp_b, par_b, el_b)
        ortho, _ = _time_single(m, sysm, dev, steps, 3, flush)
        m.close()
        m = QNEP(hp_b, par_b, el_b)
        sheared = _general_cells([sysm])[0]
        general, _ = _time_single(m, sheared, dev, steps, 3, flush)
        res["single_batio3_5000"] = {"ms_per_call_orthorhombic": ortho, "ms_per_call_general": general,
                                     "vs_orthorhombic": ortho / general}
    except Exception as exc:   # noqa: BLE001
        res["single_batio3_5000"] = {"error": f"{type(exc).__name__}: {exc}"}
    finally:
        if m is not None:
            m.close()
    return res


def _ewald_chunks(box, kmax):
    """Chunks of 8 wave vectors of the half-space k-set (orthorhombic box): per (n1, n2) column
    the contiguous n3 range with 0 < |k| < kmax, split into chunks of 8 (cached per box shape)."""
    key = (tuple(np.round(np.diag(box), 9)), kmax)
    if key not in _CHUNKS:
        _CHUNKS[key] = _ewald_chunks_of(np.diag(box), kmax)
    return _CHUNKS[key]


def _ewald_chunks_of(lengths, kmax):
    nmax = [int(math.floor(kmax * ln / (2 * math.pi))) for ln in lengths]
    chunks = 0
    for n1 in range(0, nmax[0] + 1):
        for n2 in range(-nmax[1], nmax[1] + 1):
            n3s = [n3 for n3 in range(-nmax[2], nmax[2] + 1)
                   if (n1 > 0 or (n1 == 0 and (n2 > 0 or (n2 == 0 and n3 > 0))))
                   and 0 < sum((2 * math.pi * m / ln) ** 2 for m, ln in zip((n1, n2, n3), lengths)) < kmax * kmax]
            if n3s:
                chunks += (n3s[-1] - n3s[0] + 8) // 8
    return chunks


def _tensor_roofline(systems, hp, elec, n_cand, item_ms, peaks, contract="bf16x3"):
    """Tensor-pipe share of the batched item kernel: its three tcgen05.mma kind::f16 contractions.

    Useful work (real data only, the products of the hi / lo splits counted), per (atom, candidate):
    the angular descriptor contraction 2 x 5 n x 24 lm x 9 S per product (three BF16 products, one
    for the BF16 form); the k-space potential and field 4 outputs x 2 x 2 per real half-space k and
    the structure factor 2 x 2 per real k, three FP16 products each.  Issued work adds the padding
    of the MMA shapes: descriptor M 256 / K 48 / N 128 per 5-atom tile; field M 128 atoms x N 128 x
    K 16 per (128-atom tile, chunk of 8 wave vectors); structure factor M 128 x N 32 x K 32 per
    (32-atom tile, window of 8 chunks).
    """
    S = hp.n_species
    atoms = sum(sy.n_atoms for sy in systems)
    groups = (n_cand + 31) // 32
    prod = 3 if contract == "bf16x3" else 1
    useful_d = prod * 2 * 5 * 24 * 9 * S * atoms * n_cand
    issued_d = prod * 2 * 256 * 48 * (128 / 5.0) * atoms * groups
    useful_k = issued_k = 0.0
    for sy in systems:
        nk = _ewald_kcount(sy.box, elec.kmax)
        nch = _ewald_chunks(sy.box, elec.kmax)
        useful_k += 3 * (16 + 4) * sy.n_atoms * n_cand * nk
        issued_k += groups * 3 * (math.ceil(sy.n_atoms / 128) * nch * 2 * 128 * 128 * 16
                                  + math.ceil(sy.n_atoms / 32) * math.ceil(nch / 8) * 2 * 2 * 128 * 32 * 16)
    useful, issued = useful_d + useful_k, issued_d + issued_k
    peak = peaks["bf16_tflops"]
    ach = useful / (item_ms * 1e-3) / 1e12
    return {"kernel": "k_batch_items (tcgen05.mma kind::f16: descriptor contraction, k-space field, S(k))",
            "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
            "work": f"{useful:.4g} useful / {issued:.4g} issued tensor flop per launch (descriptor {useful_d:.3g}, "
                    f"k space {useful_k:.3g} useful; {contract} descriptor products, FP16x3 k space)",
            "note": "averaged over the whole item kernel; the contractions are three phases of it (the kernel as a "
                    "whole is bound by the FP32 pipes, see roofline)",
            "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst, cuBLAS bf16; FP16 has the same kind::f16 rate)"}


def run_batch(args):
    """Batched form: every (candidate, structure) pair of the LLZO batch in one persistent launch."""
    import torch

    from paper_2601_19034_gb300.qnep import QNEP, QNEPBatch, stack_structures

    import torch.distributed as dist
    from paper_2601_19034_gb300 import workloads

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        # the batch partitions into independent items: every rank evaluates its own batch of
        # the same shape (weak scaling); only the timing barrier and the max-over-ranks reduction
        # cross ranks, there is no collective in the data path
        dist.init_process_group("nccl")
    systems, hp, params, elec = workloads.config_llzo_batch(seed=_batch_seed(rank))
    if args.structures:
        systems = systems[:args.structures]
    if args.candidates:
        params = params[:args.candidates]
    n_cand = params.shape[0]
    pos, typ, off, boxes = stack_structures(systems)
    n_total = int(off[-1])
    pos_d, typ_d = torch.tensor(pos, device=dev), torch.tensor(typ, device=dev)
    b = QNEPBatch(hp, params, elec)
    b.set_contraction(args.contract)
    out = b.compute(pos_d, typ_d, off, boxes)          # lists sized, status checked
    tune_ms = b.autotune(pos_d, typ_d, off, boxes, reps=2, out=out)
    warps, order = b.config()
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        b.compute_into(pos_d, typ_d, off, boxes, out, stream=stream.cuda_stream)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        b.compute_into(pos_d, typ_d, off, boxes, out, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
            graph.replay()
    torch.cuda.synchronize()
    peaks, peak_kind = _peaks()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.zero_()
                starts[k].record(stream)
                graph.replay()
                ends[k].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    step_ms = [s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)]
    ms_per_step = _reduce_max(float(sum(step_ms)), dev) / args.steps
    evals = n_total * n_cand
    value = world * evals / (ms_per_step * 1e-3)
    status = b.sync_status()

    clocks = clk.summary(peaks.get("sm_max_mhz", 2070.0))
    mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak, peak_src = _fp32_peak(mhz)
    flop = _batch_flop(systems, hp, elec, n_cand)

    # the item kernel alone: CUDA events around it on the launching stream (eager calls)
    b.set_profiling(True)
    for _ in range(min(args.steps, 5) + 1):
        with torch.cuda.stream(stream):
            flush.zero_()
            b.compute_into(pos_d, typ_d, off, boxes, out, stream=stream.cuda_stream)
    stage, calls = b.stage_times()
    b.set_profiling(False)
    item_ms = stage["items"] / max(calls, 1)
    prep_ms = stage["prepass"] / max(calls, 1)
    other = {c: _time_other_contraction(hp, params, elec, pos_d, typ_d, off, boxes, stream, flush, c,
                                        min(args.steps, 10), evals)
             for c in ("fp32", "bf16x3", "bf16") if c != args.contract}
    for c, v in other.items():
        v["speedup_vs_fp32_contraction"] = (other["fp32"]["ms_per_step"] if "fp32" in other else ms_per_step) \
            / v["ms_per_step"]
    other["note"] = ("fp32 and bf16x3 meet the FP32-path tolerances against the FP64 oracle; bf16 (one product) "
                     "is the reduced-precision form, within the mixed-path bounds (tests/test_gpu_batch.py)")

    # external-field response from the Born effective charges (Sec. II.D), its own HBM roofline
    field_roof, _ = _time_field_response(dev, flush, peaks, min(args.steps, 20))

    # precision form on liquid water (8000 H2O, PPPM 64^3): FP32 vs BF16 / TF32 network
    mixed = {"workload": WORKLOADS["water_pppm"]}
    sy_w, hp_w, par_w, el_w = _config("water_pppm")
    for prec in ("fp32", "bf16", "tf32"):
        mw = QNEP(hp_w, par_w, el_w, precision=prec)
        ms_w, _ = _time_single(mw, sy_w, dev, min(args.steps, 20), 3, flush)
        mixed[prec] = {"ms_per_call": ms_w, "value": sy_w.n_atoms / (ms_w * 1e-3), "unit": UNIT}
        mw.close()
    for prec in ("bf16", "tf32"):
        mixed[f"speedup_{prec}_vs_fp32"] = mixed[prec]["value"] / mixed["fp32"]["value"]
    mixed["errors_vs_oracle"] = "per-output bounds against the FP64 oracle in tests/test_gpu_precision.py"
    # and on the ~1.0 M-atom Mg-water interface (PPPM 256 x 256 x 384), the configuration that names
    # the mixed-precision network: the MD force call (forces and charges), FP32 vs BF16 network
    sy_m, hp_m, par_m, el_m = workloads.config_mg_water()
    large = {"workload": WORKLOADS["mgwater_nve"], "atoms": sy_m.n_atoms, "outputs": "forces, charges"}
    for prec in ("fp32", "bf16"):
        mm = QNEP(hp_m, par_m, el_m, precision=prec)
        ms_m, _ = _time_single(mm, sy_m, dev, min(args.steps, 10), 3, flush, want=dict(bec=False, virial=False))
        large[prec] = {"ms_per_call": ms_m, "value": sy_m.n_atoms / (ms_m * 1e-3), "unit": UNIT}
        mm.close()
    large["speedup_bf16_vs_fp32"] = large["bf16"]["value"] / large["fp32"]["value"]
    large["errors_vs_oracle"] = ("BF16 network against the FP32 path at this size: force RMSE <= 5e-3 eV/A "
                                 "(tests/test_gpu_nve.py); per-output bounds in tests/test_gpu_precision.py")
    mixed["mgwater_1m"] = large

    # plain FP32 single-structure path on the same structures (candidate 0; one call per structure):
    # every call captured in its own CUDA graph (one model per box shape, so no call rebuilds its
    # k-tables), the 64 graphs replayed back to back; the eager calls are reported beside it
    plain = _time_plain_single(hp, params[0], elec, systems[:64], dev, stream, flush)

    # end to end through the C ABI's host-buffer entry point (qnep_batch_compute_host): positions
    # and types from pinned host memory in, energies, forces and charges back to pinned host
    # memory, stream synchronised, every step
    pos_h = torch.tensor(pos).pin_memory()
    typ_h = torch.tensor(typ).pin_memory()
    out_h = {"energy": torch.empty(n_cand, len(systems), dtype=torch.float64).pin_memory(),
             "forces": torch.empty(n_cand, n_total, 3, dtype=torch.float32).pin_memory(),
             "charges": torch.empty(n_cand, n_total, dtype=torch.float32).pin_memory()}
    e2e_ms = []
    for k in range(args.warmup + min(args.steps, 10)):
        torch.cuda.synchronize()
        t = time.perf_counter()
        b.compute_host(pos_h, typ_h, off, boxes, out_h, stream=stream.cuda_stream)
        dt = time.perf_counter() - t
        if k >= args.warmup:
            e2e_ms.append(dt * 1e3)
    d2h = sum(v.numel() * v.element_size() for v in out_h.values())
    # the same call with the per-(candidate, structure) virial (graph replay, L2 flushed)
    with_virial = _time_with_virial(b, pos_d, typ_d, off, boxes, stream, flush, min(args.steps, 10), evals)
    with_bec = _time_with_virial(b, pos_d, typ_d, off, boxes, stream, flush, min(args.steps, 10), evals, bec=True)

    # one device-resident SNES iteration around the same call (Sec. II.E): normal deviates,
    # sampling, parameter upload, the batched call (graph replay), the loss against reference
    # energies and forces (here candidate 0's outputs), the update of (mu, sigma)
    snes = _time_snes_step(b, graph, stream, out, off, params, dev, min(args.steps, 10))
    # the same iteration on fixed training structures with their geometry kept between generations
    # (qnep_batch_set_static_geometry: the first call builds it, the captured call holds the item
    # kernel only); the headline above runs the pre-pass in every call
    b.set_static_geometry(True)
    with torch.cuda.stream(stream):
        b.compute_into(pos_d, typ_d, off, boxes, out, stream=stream.cuda_stream)
    stream.synchronize()
    g_static = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_static, stream=stream):
        b.compute_into(pos_d, typ_d, off, boxes, out, stream=stream.cuda_stream)
    snes_static = _time_snes_step(b, g_static, stream, out, off, params, dev, min(args.steps, 10))
    snes_static["what"] = ("as snes_step, with qnep_batch_set_static_geometry: the candidate-independent pre-pass "
                           "built once for the fixed training structures, each iteration's batched call the item "
                           "kernel alone")
    b.set_static_geometry(False)
    del g_static
    # side measurements of the scope table's further rows, last so that nothing above depends on them
    atom_virial = _time_atom_virial(dev, flush, min(args.steps, 20))
    general = _time_general_cells(hp, params, elec, systems, dev, stream, flush, min(args.steps, 10), evals,
                                  args.contract, (warps, order), ms_per_step)
    line = None
    if rank == 0:
        achieved = flop / (ms_per_step * 1e-3) / 1e12
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 reductions)", "data": "synthetic",
            "config": {"workload": WORKLOADS["llzo_batch"], "structures": len(systems), "candidates": n_cand,
                       "atoms": n_total, "atom_evaluations_per_step": evals,
                       "l2": "flushed between steps (512 MB write); working set > L2",
                       "launch": "CUDA graph replay of one qnep_batch_compute (pre-pass + persistent item kernel)",
                       "autotuned": {"warps": warps, "order": order, "ms": tune_ms},
                       "contraction": args.contract,
                       "parallelism": f"{world} ranks, one batch each (no data-path collective)" if world > 1
                       else "single GPU", "wall_s": wall},
            "roofline": {"kernel": "k_batch_items", "bound": "alu", "achieved": flop / (item_ms * 1e-3) / 1e12,
                         "peak": fp32_peak, "unit": "TFLOP/s", "frac": flop / (item_ms * 1e-3) / 1e12 / fp32_peak,
                         "traffic": ITEM_DRAM_BYTES_PER_EVAL * evals
                         if (ITEM_DRAM_BYTES_PER_EVAL and args.contract == "bf16x3") else None,
                         "traffic_unit": "bytes per launch",
                         "traffic_source": ITEM_DRAM_SOURCE, "ms": item_ms, "prepass_ms": prep_ms,
                         "peak_source": peak_src,
                         "work": f"{flop:.4g} algorithmic flop per launch (whole batch)",
                         "whole_call_frac": achieved / fp32_peak},
            "roofline_tensor": _tensor_roofline(systems, hp, elec, n_cand, item_ms, peaks, args.contract)
            if args.contract != "fp32" else None,
            "contraction_compare": other,
            "mixed": mixed,
            "field_response": field_roof,
            "snes_step": dict(snes, batched_call_ms=ms_per_step),
            "snes_step_static_geometry": snes_static,
            "plain_fp32": dict(plain, speedup_batched_vs_plain=value / plain["value"]),
            "with_virial": with_virial,
            "with_bec": with_bec,
            "atom_virial": atom_virial,
            "general_cells": general,
            "e2e": {"value": evals / (statistics.median(e2e_ms) * 1e-3) * world, "unit": UNIT,
                    "h2d_bytes_per_step": n_total * 16, "d2h_bytes_per_step": d2h,
                    "ms_per_step": statistics.median(e2e_ms),
                    "entry_point": "qnep_batch_compute_host (C ABI, host buffers): positions + types in; "
                                   "energies, forces and charges of every (candidate, structure) back"},
            "gpu_launches": BATCH_KERNELS_PER_CALL * args.steps,
            "clocks": clocks,
            "device_status": status,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = _cpu_baseline_batch(systems, hp, params, elec)
    b.close()
    if world > 1:
        dist.destroy_process_group()
    return line


def _cpu_baseline_batch(systems, hp, params, elec):
    """Oracle on a bounded sample: the two smallest structures under one candidate."""
    import torch

    from oracle import forcecall
    cores = torch.get_num_threads()
    order = np.argsort([sy.n_atoms for sy in systems])[:2]
    t = time.perf_counter()
    atoms = 0
    for s_ in order:
        sy = systems[s_]
        forcecall.force_call(sy.positions.astype(np.float64), sy.box, sy.types, hp, params[0], elec,
                             want_bec=False)
        atoms += sy.n_atoms
    dt = time.perf_counter() - t
    return {"value": atoms / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{atoms} atom-evaluations: the 2 smallest structures x 1 candidate (FP64 oracle, "
                      f"torch CPU threads={cores})"}


def _reference_batch(args, world, cores):
    """Oracle steps on the batch workload: each step one (smallest structure, candidate) pair."""
    from oracle import forcecall
    systems, hp, params, elec = _config("llzo_batch")
    small = [i for i in np.argsort([sy.n_atoms for sy in systems])]
    times, atoms = [], 0
    for k in range(args.warmup + args.steps):
        sy = systems[small[k % 8]]
        t = time.perf_counter()
        forcecall.force_call(sy.positions.astype(np.float64), sy.box, sy.types, hp, params[k % params.shape[0]],
                             elec, want_bec=False)
        dt = time.perf_counter() - t
        if k >= args.warmup:
            times.append(dt)
            atoms += sy.n_atoms
    total = sum(times)
    value = atoms / total
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / len(times) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS["llzo_batch"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "each step one (structure, candidate) pair of the batch, the 8 smallest "
                                       "structures in turn"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def model_precision(args):
    """Network precision of the large-scale NVE workload: the precision form (BF16) unless asked otherwise."""
    return args.precision if args.precision != "fp32" else "bf16"


def run_nve(args):
    """Large-scale form: NVE velocity Verlet on the ~1 M-atom Mg-water interface."""
    import torch

    from paper_2601_19034_gb300 import workloads
    from paper_2601_19034_gb300.qnep import QNEP, nve

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.mg_cells:   # a narrower slab of the same construction (profiling), mesh scaled to keep h
        nx, ny = (int(x) for x in args.mg_cells.split(","))
        mesh = (2 * max(4, round(128 * nx / 112)), 2 * max(4, round(128 * ny / 65)), 384)
        sysm, hp, params, elec = workloads.config_mg_water(nx=nx, ny=ny, mesh=mesh)
    else:
        sysm, hp, params, elec = workloads.config_mg_water()
    n = sysm.n_atoms
    masses = workloads.species_masses(workloads.MGWATER_SPECIES)
    v0 = workloads.maxwell_boltzmann(masses[sysm.types], 300.0).astype(np.float32)
    model = QNEP(hp, params, elec, precision=model_precision(args))
    model.set_skin(args.skin)
    pos = torch.tensor(sysm.positions, device=dev)
    vel = torch.tensor(v0, device=dev)
    typ = torch.tensor(sysm.types, device=dev)
    model.compute(pos, typ, sysm.box, bec=False)          # lists sized, status checked
    nve(model, pos, vel, typ, masses, sysm.box, 0.5, args.warmup)
    torch.cuda.synchronize()
    peaks, peak_kind = _peaks()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0.record()
        _, en = nve(model, pos, vel, typ, masses, sysm.box, 0.5, args.steps)
        e1.record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    status = model.sync_status()
    rebuilds = model.skin_rebuilds() if args.skin > 0 else None
    ms = e0.elapsed_time(e1)
    ms_per_step = ms / args.steps
    # the same run with the lists rebuilt at every force call (skin 0), continuing from this state
    compare = None
    if args.skin > 0:
        model.set_skin(0.0)
        ksk = min(args.steps, 20)
        nve(model, pos, vel, typ, masses, sysm.box, 0.5, 2)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record()
        nve(model, pos, vel, typ, masses, sysm.box, 0.5, ksk)
        c1.record()
        c1.synchronize()
        compare = {"skin_A": 0.0, "steps": ksk, "ms_per_step": c0.elapsed_time(c1) / ksk,
                   "value": n * ksk / (c0.elapsed_time(c1) * 1e-3),
                   "what": "the same NVE run with the neighbour lists rebuilt at every force call"}
        model.set_skin(args.skin)
    value = world * n * args.steps / (ms * 1e-3)
    e = en.cpu().numpy()
    etot = e.sum(1)
    tps = np.arange(len(etot)) * 0.5e-3
    drift = float(np.polyfit(tps, (etot - etot[0]) / n, 1)[0] * 1e3) if len(etot) > 2 else None
    # the precision form against the FP32 network on the same run (same skin, same state)
    prec_cmp = None
    if model_precision(args) != "fp32":
        m32 = QNEP(hp, params, elec, precision="fp32")
        m32.set_skin(args.skin)
        p32, v32 = pos.clone(), vel.clone()
        m32.compute(p32, typ, sysm.box, bec=False)
        nve(m32, p32, v32, typ, masses, sysm.box, 0.5, 2)
        kp = min(args.steps, 20)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record()
        nve(m32, p32, v32, typ, masses, sysm.box, 0.5, kp)
        c1.record()
        c1.synchronize()
        m32.close()
        ms32 = c0.elapsed_time(c1) / kp
        prec_cmp = {"network": model_precision(args), "ms_per_step": ms_per_step, "fp32_network_ms_per_step": ms32,
                    "speedup_vs_fp32_network": ms32 / ms_per_step, "steps_fp32": kp,
                    "accuracy": "BF16 network against the FP32 path at 1 M atoms: force RMSE <= 5e-3 eV/A "
                                "(tests/test_gpu_nve.py)"}
    # per-stage device times of one force call (library stage timers)
    model.set_profiling(True)
    for _ in range(3):
        model.compute(pos, typ, sysm.box, bec=False)
    stages, calls = model.stage_times()
    model.set_profiling(False)
    stage_avg = {k: v / max(calls, 1) for k, v in stages.items()}
    # end to end: state from pinned host memory, the run, energies back
    pos_h = torch.tensor(sysm.positions).pin_memory()
    vel_h = torch.tensor(v0).pin_memory()
    ksteps = min(args.steps, 10)
    torch.cuda.synchronize()
    t = time.perf_counter()
    pos.copy_(pos_h, non_blocking=True)
    vel.copy_(vel_h, non_blocking=True)
    _, en2 = nve(model, pos, vel, typ, masses, sysm.box, 0.5, ksteps)
    en_h = en2.cpu()
    e2e_s = time.perf_counter() - t
    clocks = clk.summary(peaks.get("sm_max_mhz", 2070.0))
    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (network bf16 on tensor cores, FP64 reductions)", "data": "synthetic",
            "config": {"workload": WORKLOADS["mgwater_nve"], "atoms": n, "dt_fs": 0.5,
                       "l2": "inputs larger than L2 (1 M atoms, 25 M-point meshes)",
                       "launch": "qnep_nve_run: per step kick+drift, force call, kick+FP64 kinetic energy; "
                                 "neighbour lists kept with a Verlet skin (rebuilt on the device when an atom "
                                 "has moved more than skin / 2)",
                       "parallelism": "replicas" if world > 1 else "single GPU", "wall_s": wall},
            "mixed": prec_cmp,
            "skin": {"skin_A": args.skin, "rebuilds": rebuilds,
                     "force_calls": args.steps + args.warmup + 2, "no_skin": compare},
            "nve": {"drift_mev_per_atom_ps": drift, "steps": args.steps,
                    "drift_first_100fs_mev_per_atom_ps": float(np.polyfit(tps[:201], (etot[:201] - etot[0]) / n, 1)[0]
                                                               * 1e3) if len(etot) > 2 else None,
                    "max_abs_dE_per_atom_eV": float(np.abs(etot - etot[0]).max() / n),
                    "temperature_K": [float(e[0, 1] / n / (1.5 * 8.617333e-5)),
                                      float(e[-1, 1] / n / (1.5 * 8.617333e-5))],
                    "note": "random-parameter potential: no short-range repulsion; atoms fall into its wells "
                            "(T rises, pairs approach ~0.1 A) and the error grows after ~150 fs"},
            "stage_ms": stage_avg,
            "roofline": _roofline_generic(stage_avg, sysm, clocks, peaks),
            "e2e": {"value": n * ksteps / e2e_s * world, "unit": UNIT, "h2d_bytes_per_step": n * 24 // ksteps,
                    "d2h_bytes_per_step": int(en_h.numel() * 8 // ksteps), "ms_per_step": e2e_s * 1e3 / ksteps},
            "gpu_launches": None,
            "clocks": clocks,
            "device_status": status,
        }
        if not args.no_cpu_baseline:
            from oracle import forcecall
            small = workloads.mg_water_interface(6, 4, seed=77)
            el_s = workloads.Elec(mode=1, kind="pppm", mesh=(20, 24, 100), order=5)
            tc = time.perf_counter()
            forcecall.force_call(small.positions.astype(np.float64), small.box, small.types, hp, params, el_s,
                                 want_bec=False)
            dtc = time.perf_counter() - tc
            line["cpu_baseline"] = {"value": small.n_atoms / dtc, "unit": UNIT, "cores": torch.get_num_threads(),
                                    "kind": "oracle", "sample": f"one force call of a {small.n_atoms}-atom "
                                    "Mg-water slab of the same construction (FP64 oracle, PPPM)"}
    model.close()
    return line


def run_field(args):
    """Field response alone (profiling and its own line): forces + Pdot per step."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peaks, peak_kind = _peaks()
    with ClockSampler(0) as clk:
        roof, times = _time_field_response(dev, flush, peaks, args.steps)
    from paper_2601_19034_gb300 import workloads
    n = workloads.FIELD_RESPONSE_ATOMS
    ms = float(sum(times)) / len(times)
    return {"metric": "qNEP field response (E.Z_i, sum_i Z_i v_i) atoms/s", "value": n / (ms * 1e-3),
            "unit": "atoms/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 Pdot sum)",
            "data": "synthetic", "config": {"workload": WORKLOADS["field_response"],
                                            "l2": "inputs larger than L2 (252 MB per step), no flush"},
            "roofline": dict(roof, peak_source=peak_kind), "gpu_launches": args.steps,
            "clocks": clk.summary(peaks.get("sm_max_mhz", 2070.0))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="llzo_batch", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "tf32"],
                    help="single-structure workloads: network precision")
    ap.add_argument("--contract", default="bf16x3", choices=["fp32", "bf16x3", "bf16"],
                    help="llzo_batch: descriptor contraction on the FP32 pipes or on the tensor cores (BF16x3)")
    ap.add_argument("--structures", type=int, default=0, help="llzo_batch: first N structures only (profiling)")
    ap.add_argument("--candidates", type=int, default=0, help="llzo_batch: first C candidates only (profiling)")
    ap.add_argument("--skin", type=float, default=1.0, help="mgwater_nve: Verlet skin of the neighbour lists (A)")
    ap.add_argument("--mg-cells", default="", help="mgwater_nve: NX,NY orthohexagonal cells instead of 112,65 "
                                                   "(profiling on a smaller slab)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        line = run_reference(args)
    elif args.workload == "llzo_batch":
        line = run_batch(args)
    elif args.workload == "field_response":
        line = run_field(args)
    elif args.workload == "mgwater_nve":
        line = run_nve(args)
    else:
        line = run_ours(args)
    if line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
