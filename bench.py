"""Benchmark of the q-LSKUM hot path on GB300: point-iterations per second.

One step = one pseudo-time iteration of Algorithm 1 over the whole cloud: the
local time step, four SSP-RK stages of {q-variables, q-derivatives with two
inner iterations, flux residual, state update} and the residue. Workload: the
synthetic NACA 0012 O-cloud with 10M points (5658 x 1768, shuffled input
order), M = 0.63, alpha = 2 deg, FP64, started from a developed (non-uniform
everywhere) state. Inputs (the 12 GB device working set) are far larger than
L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (oracle/) on the host cores instead, on
a bounded sample of the same workload. With N > 1 (torchrun) every rank runs
an independent replica on its own GPU (the solver has no data-path exchange
on one cloud per GPU); the reference arm runs on rank 0 only.

Prints one JSON line on rank 0.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "q-LSKUM point-iterations/s (FP64 vs mixed vs batched), % of HBM roofline"
UNIT = "point-iterations/s"
WORKLOAD_POINTS = 10_000_000
MACH, ALPHA = 0.63, 2.0
VARIANTS = ("mixed", "batched64_mixed", "batched64_fp64", "fp64_split_flux_ablation",
            "ragged16_mixed")
SAMPLE_POINTS = 2_500_000  # CPU-oracle sample: an inner region of the workload cloud


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(points_requested: int, world: int, flux_split: bool = False,
                    mach: float = MACH, alpha: float = ALPHA) -> dict:
    """The `config` both arms report: the NACA 0012 cloud of about
    `points_requested` points (its exact size from the generator's grid)."""
    from paper_2108_07031_gb300 import cloud as Cl
    n_c, n_r = Cl.cloud_dims(points_requested)
    n = n_c * n_r
    cond = "" if (mach, alpha) == (MACH, ALPHA) else f"-M{mach:g}-a{alpha:g}"
    return {"workload": f"naca0012-o-cloud-{n}pts-fp64" + cond
            + ("-split-flux-kernels" if flux_split else ""),
            "points": n, "mach": mach, "alpha_deg": alpha, "inner_iters": 2, "rk_stages": 4,
            "cfl": 0.2, "parallelism": f"replicas{world}",
            "l2": "inputs larger than L2 (device working set ~17 GB), no flush",
            "initial_state": "developed: seeded smooth perturbation of the free stream at every "
                             "point"}


def max_over_ranks(x: float, dist) -> float:
    """Maximum of a per-rank float over all ranks (the job's wall time is its
    slowest rank's); the identity without a process group."""
    if dist is None:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units processed by all ranks (each rank does the same work: weak
    scaling, replicas) per second of the slowest rank."""
    return world * units_per_rank / seconds


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _cloud(n_points: int, shuffle: bool = True):
    from paper_2108_07031_gb300 import cloud as Cl
    n_c, n_r = Cl.cloud_dims(n_points)
    cache = os.environ.get("LSKUM_CLOUD_CACHE", os.path.join(tempfile.gettempdir(), "lskum_clouds"))
    fn = os.path.join(cache, f"naca_{n_c}x{n_r}_s{int(shuffle)}.npz")
    if os.path.exists(fn):
        try:
            z = np.load(fn)
            return Cl.Cloud(xy=z["xy"], normals=z["normals"], flags=z["flags"],
                            nbr_offsets=z["off"], nbr_idx=z["idx"], n_c=n_c, n_r=n_r,
                            k=z["k"], l=z["l"])
        except Exception:
            pass
    c = Cl.naca0012_cloud(n_c, n_r, shuffle=shuffle)
    try:
        os.makedirs(cache, exist_ok=True)
        tmp = fn + f".{os.getpid()}.npz"
        np.savez(tmp, xy=c.xy, normals=c.normals, flags=c.flags, off=c.nbr_offsets,
                 idx=c.nbr_idx, k=c.k, l=c.l)
        os.replace(tmp, fn)
    except OSError:
        pass
    return c


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        try:
            self.out.flush()
            with open(self.out.name) as f:
                rows = [r.strip().split(", ") for r in f if r.strip()]
        except OSError:
            rows = []
        finally:
            try:
                os.unlink(self.out.name)
            except OSError:
                pass
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _fp64_peak():
    """FP64 pipe throughput and FP64 library-call costs measured live by the probe."""
    from paper_2108_07031_gb300 import build as B
    try:
        out = subprocess.run([B.PROBE], capture_output=True, text=True, timeout=120, check=True)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:  # the probe is a measurement aid; report without it
        return {"error": str(e)}


# Per-unit figures of the FP64 flux/update kernel (k_flux), from one ncu
# capture of a stage launch on the 600,138-point cloud (8,338,298 neighbour
# entries): 1.0688e9 DFMA, 0.2379e9 DADD and 0.5728e9 DMUL thread
# instructions (predicated on) = 2.948e9 FP64 flops = 353.6 flops per
# neighbour entry (225.4 FP64 instructions), and 438.0 MB of DRAM traffic
# = 729.8 bytes per point.
# Units of one launch: neighbour entries (flops) and points (bytes); both
# scale in proportion with the cloud size. With this instruction mix a
# saturated FP64 pipe reaches (2 DFMA + DADD + DMUL) / (2 (DFMA + DADD +
# DMUL)) = 0.784 of the FMA peak (every FP64 instruction takes one issue
# slot of the pipe).
FLUX_FP64_FLOPS_PER_NEIGHBOUR = 353.6
FLUX_FP64_INSTR_PER_NEIGHBOUR = 225.4  # DFMA + DADD + DMUL
FLUX_DRAM_BYTES_PER_POINT = 729.8
FLUX_FRAC_CEILING = 0.784
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12  # 1.2586
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # 80.55: 128 FP32 lanes per SM
ALGORITHMIC_BYTES_PER_POINT_ITERATION = 4600.0  # minimal passes, gathers from cache

# The variants' dominant flux kernels, per neighbour entry (x condition) and
# per point (x condition), from one ncu capture each of a 600,138-point
# launch (thread-level predicated-on FP32 / FP64 instructions, DRAM bytes):
#   mixed: k_flux_mx, FP32 flops (2 FFMA + FADD + FMUL) per entry; its FP64
#          epilogue (state update, q-variables) is per point;
#   split: the four k_flux_part launches and k_stage_split of one stage.
#   mixed: 0.7822e9 FFMA + 1.0223e9 FMUL + 0.5091e9 FADD = 3.096e9 FP32 flops
#          = 371.3 per entry (plus 57 FP64 instructions per point), 277.0 MB
#          of DRAM traffic = 461.6 bytes per point;
#   split: 1.4516e9 DFMA + 0.2950e9 DADD + 0.8724e9 DMUL over the five
#          launches of a stage = 4.071e9 FP64 flops = 488.2 per entry,
#          1353.9 MB = 2256 bytes per point.
FLUX_MX_FP32_FLOPS_PER_NEIGHBOUR = 371.3
FLUX_MX_DRAM_BYTES_PER_POINT = 461.6
FLUX_SPLIT_FP64_FLOPS_PER_NEIGHBOUR = 488.2
FLUX_SPLIT_DRAM_BYTES_PER_POINT = 2257.0


def layout_bytes_per_point_iteration(mixed: bool, entries_per_point: float, inner: int = 2) -> float:
    """Compulsory DRAM bytes of one iteration (4 RK stages) per point of the
    library's device layout: every slot-major per-neighbour stream and
    per-point record read or written once per pass, the neighbours'
    gathered records served from cache. E = neighbour entries per point.
      FP64  first-order sweep: (4 + 8 + 8) E + q 32 + count 4 + (q_x, q_y) 64
            inner sweep:       (4 + 32) E + per-point sums 32 + derivatives
                               64 in, 64 first-order, 64 out + count 4
            flux + update:     (4 + 4 x 8) E + flag 1 + count 4 + normal 16
                               + q 32 + derivatives 64 + U 32 in, 32 out
                               + next q 32 + 26 (time step, U0: stage mean)
      mixed first-order sweep: (4 + 8) E + q pair 32 + count 4 + out 32
            inner sweep:       (4 + 8) E + coordinate pair 16 + 32 in,
                               32 first-order, 32 out + count 4
            flux + update:     (4 + 16) E + 1 + 4 + 16 + q pair 32
                               + derivatives 32 + U 64 + next q 32 + 26"""
    E = entries_per_point
    if mixed:
        per_stage = (12 * E + 68) + inner * (12 * E + 116) + (20 * E + 207)
    else:
        per_stage = (20 * E + 100) + inner * (36 * E + 228) + (36 * E + 239)
    return 4.0 * per_stage


def run_ours(args, rank, world, local):
    import torch

    from paper_2108_07031_gb300 import cloud as Cl
    from paper_2108_07031_gb300 import lskum as L

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    cloud = _cloud(args.points)
    n = cloud.n
    stream = torch.cuda.Stream()
    solver = L.Solver.from_cloud(cloud, flux_split=1 if args.flux_split else 0)
    solver.set_stream(stream.cuda_stream)
    solver.set_freestream(args.mach, args.alpha)
    # time a developed flow: a smooth seeded perturbation of the free stream at
    # every point, so no neighbour pair has equal modified states (the flux
    # kernel skips such pairs exactly; a uniform start would time that skip)
    solver.set_state(Cl.perturbed_state(cloud, args.mach, args.alpha))
    info = solver.info()

    # warm-up (also captures the iteration graph)
    solver.step(args.warmup)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # timed region: K iterations, per-kernel CUDA events on the solver's stream
    solver.profile(True)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        start.record(stream)
        solver.step(args.steps)
        launches = solver.last_launch_count()
        end.record(stream)
        barrier()
    ms = start.elapsed_time(end)
    flux_ms, flux_n = solver.kernel_time(L.KERNEL_FLUX)
    kt = {name: solver.kernel_time(k) for name, k in (("flux", L.KERNEL_FLUX),
                                                       ("ls_first", L.KERNEL_LS_FIRST),
                                                       ("ls_inner", L.KERNEL_LS_INNER),
                                                       ("residue", L.KERNEL_REDUCE))}
    solver.profile(False)
    clocks = clk.summary()
    t_max = max_over_ranks(ms, dist)
    value = whole_job_rate(n * args.steps, world, t_max * 1e-3)

    # end to end through the C ABI with host buffers: H2D of the state,
    # one iteration, D2H of the residue, every step
    W0 = solver.get_state()
    pinned = torch.from_numpy(W0).pin_memory()
    e2e_steps = max(1, min(args.steps, 5))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.set_state_ptr(pinned.data_ptr())
        solver.step(1)
        _ = solver.residual_norm()
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_t = max_over_ranks(e2e_s, dist)
    e2e_value = whole_job_rate(n * e2e_steps, world, e2e_t)
    # the same, for a caller that consumes the field: the state is also read
    # back (lskum_get_state, into pinned host memory) every step
    out_pinned = torch.empty_like(pinned).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.set_state_ptr(pinned.data_ptr())
        solver.step(1)
        _ = solver.residual_norm()
        solver.get_state_ptr(out_pinned.data_ptr())
    barrier()
    e2e_state_t = max_over_ranks(time.perf_counter() - t0, dist)
    e2e_state_value = whole_job_rate(n * e2e_steps, world, e2e_state_t)

    result = None
    config = workload_config(args.points, world, args.flux_split, args.mach, args.alpha)
    assert config["points"] == n
    if rank == 0:
        peaks = _fp64_peak()
        nnz = int(cloud.nbr_offsets[-1])
        flux_launch_ms = flux_ms / max(flux_n, 1)
        achieved = FLUX_FP64_FLOPS_PER_NEIGHBOUR * nnz / (flux_launch_ms * 1e-3) / 1e12
        # ALU-bound kernel: the peak derived from unit counts and clocks,
        # 152 SMs x 2 FP64 FMA per SM per clock x 2 flops x 2.07 GHz
        peak = FP64_PEAK_TFLOPS
        mp, mp_kind = _peaks()
        cpu = cpu_baseline(args) if not args.no_cpu_baseline else None
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "ours",
            "config": config,
            "max_neighbours": info["max_neighbours"],
            "roofline": {
                "kernel": "k_flux (flux residual + SSP-RK stage update, FP64)", "bound": "alu",
                "unit": "TFLOP/s", "achieved": achieved, "peak": peak,
                "frac": (achieved / peak) if peak else None,
                "traffic": FLUX_DRAM_BYTES_PER_POINT * n,
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk/SM x 2 flops x 2.07 GHz "
                               "(maximum SM clock)",
                "measured_fma_peak": peaks.get("fp64_fma_tflops"),
                "measured_fma_peak_source": "pure-DFMA probe (pipe_peaks) run live on this GPU",
                "flops_per_launch": FLUX_FP64_FLOPS_PER_NEIGHBOUR * nnz,
                "frac_ceiling_at_instruction_mix": FLUX_FRAC_CEILING,
                # the pipe's own bound: FP64 instructions issued per second
                # against 152 SMs x 2 per clock x 2.07 GHz
                "fp64_issue_frac": (FLUX_FP64_INSTR_PER_NEIGHBOUR * nnz / (flux_launch_ms * 1e-3))
                                   / (FP64_PEAK_TFLOPS * 1e12 / 2) if flux_launch_ms else None,
                "launch_ms": flux_launch_ms,
                "traffic_note": "ncu dram bytes of a 0.6M-point launch scaled by points",
                "hbm_frac_of_measured_whole_step": {
                    "algorithmic": (ALGORITHMIC_BYTES_PER_POINT_ITERATION * n
                                    / (t_max / args.steps * 1e-3)) / (mp["hbm_gbs"] * 1e9),
                    "layout": (layout_bytes_per_point_iteration(False, nnz / n) * n
                               / (t_max / args.steps * 1e-3)) / (mp["hbm_gbs"] * 1e9),
                    "layout_bytes_per_point_iteration":
                        layout_bytes_per_point_iteration(False, nnz / n),
                    "peak_gbs": mp["hbm_gbs"], "peak_kind": mp_kind},
            },
            "kernel_ms": {k: {"total_ms": v[0], "launches": v[1]} for k, v in kt.items()},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * 32,
                    "d2h_bytes_per_step": 8, "steps": e2e_steps,
                    "with_state_readback": {"value": e2e_state_value, "unit": UNIT,
                                            "h2d_bytes_per_step": n * 32,
                                            "d2h_bytes_per_step": n * 32 + 8}},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
    solver.close()
    if args.variants:
        from paper_2108_07031_gb300 import cloud as Cl
        want = set(VARIANTS) if args.variants == "all" else set(args.variants.split(","))
        unknown = want - set(VARIANTS)
        if unknown:
            raise SystemExit(f"unknown variants {sorted(unknown)}; known: {', '.join(VARIANTS)}")
        variants = {}
        if "mixed" in want:
            variants["mixed"] = time_variant(args, cloud, L.MIXED, 1, stream, barrier, dist,
                                             f"{n}-point cloud, one condition, block sizes autotuned",
                                             autotune=True)
        if want & {"batched64_mixed", "batched64_fp64"}:
            c06 = _cloud(600_000)
            mach, alpha = Cl.conditions(64)
        if "batched64_mixed" in want:
            variants["batched64_mixed"] = time_variant(
                args, c06, L.MIXED, 64, stream, barrier, dist,
                "64 seeded conditions (M ~ U[0.3,0.8], alpha ~ U[-4,6] deg) on the 600,138-point "
                "cloud, condition-innermost, block size autotuned", conditions=(mach, alpha),
                autotune=True)
        if "batched64_fp64" in want:
            variants["batched64_fp64"] = time_variant(
                args, c06, L.FP64, 64, stream, barrier, dist,
                "the same 64 conditions in FP64", conditions=(mach, alpha), autotune=True)
        if "fp64_split_flux_ablation" in want:
            variants["fp64_split_flux_ablation"] = time_variant(
                args, cloud, L.FP64, 1, stream, barrier, dist,
                f"{n}-point cloud, FP64, the paper's kernel splitting (four split-flux kernels "
                "and a stage kernel per stage)", split=True)
        if "ragged16_mixed" in want:
            packed, sizes = _ragged_cloud()
            variants["ragged16_mixed"] = time_variant(
                args, packed, L.MIXED, 1, stream, barrier, dist,
                f"16 clouds of {min(sizes)}-{max(sizes)} points packed into one launch "
                f"({packed.n} points)", autotune=True)
        if result is not None:
            for v in variants.values():
                v["speedup_vs_fp64"] = v["value"] / value
            result["variants"] = variants
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return result


def _ragged_cloud():
    from paper_2108_07031_gb300 import cloud as Cl
    sizes = Cl.ragged_sizes(16)
    members = [_cloud(n) for n in sizes]
    packed, _ = Cl.pack(members)
    return packed, [m.n for m in members]


def time_variant(args, cloud, precision, n_cond, stream, barrier, dist, what,
                 conditions=None, autotune=False, split=False):
    """Same timed region as the headline for another precision / batch shape."""
    import torch

    from paper_2108_07031_gb300 import cloud as Cl
    from paper_2108_07031_gb300 import lskum as L
    s = L.Solver.from_cloud(cloud, precision=precision, n_conditions=n_cond,
                            flux_split=1 if split else 0)
    s.set_stream(stream.cuda_stream)
    if conditions is None:
        s.set_freestream(args.mach, args.alpha)
        W = Cl.perturbed_state(cloud, args.mach, args.alpha)
    else:
        s.set_conditions(*conditions)
        W = np.stack([Cl.perturbed_state(cloud, m, a) for m, a in zip(*conditions)])
    s.set_state(W)
    del W
    block = list(s.autotune(1)) if autotune else [128, 128]
    s.step(args.warmup)
    s.profile(True)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    barrier()
    start.record(stream)
    s.step(args.steps)
    launches = s.last_launch_count()
    end.record(stream)
    barrier()
    ms = start.elapsed_time(end)
    kt = {name: s.kernel_time(k) for name, k in (("flux", L.KERNEL_FLUX),
                                                  ("ls_first", L.KERNEL_LS_FIRST),
                                                  ("ls_inner", L.KERNEL_LS_INNER),
                                                  ("residue", L.KERNEL_REDUCE))}
    s.profile(False)
    s.close()
    world = dist.get_world_size() if dist is not None else 1
    t_max = max_over_ranks(ms, dist)
    value = whole_job_rate(cloud.n * n_cond * args.steps, world, t_max * 1e-3)
    mixed = precision == L.MIXED
    return {"workload": what, "precision": "mixed" if mixed else "fp64",
            "points": cloud.n, "conditions": n_cond, "block_size": {"flux": block[0], "q_derivatives": block[1]},
            "autotune_space": ({"flux": [128, 256], "q_derivatives": [128, 256]} if autotune
                               else None),
            "value": value, "unit": "point-condition-iterations/s" if n_cond > 1 else UNIT,
            "ms_per_step": t_max / args.steps, "gpu_launches": int(launches),
            "kernel_ms": {k: {"total_ms": v[0], "launches": v[1]} for k, v in kt.items()},
            "roofline": variant_roofline(mixed, split, kt["flux"], int(cloud.nbr_offsets[-1]),
                                         cloud.n, n_cond, t_max / args.steps)}


def variant_roofline(mixed: bool, split: bool, flux_time, nnz: int, n: int, n_cond: int,
                     ms_per_step: float) -> dict:
    """Roofline of a variant's dominant kernel (the flux kernel: FP32 issue
    for the mixed path, the FP64 pipe otherwise) and the HBM fraction of its
    whole step, both from the live CUDA-event times of the timed region."""
    flux_ms, flux_n = flux_time
    launch_s = flux_ms / max(flux_n, 1) * 1e-3
    if mixed:
        kernel, per_entry, per_point = ("k_flux_mx (mixed-precision flux residual + stage update)",
                                        FLUX_MX_FP32_FLOPS_PER_NEIGHBOUR, FLUX_MX_DRAM_BYTES_PER_POINT)
        peak, peak_src = FP32_PEAK_TFLOPS, "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz"
    elif split:
        kernel, per_entry, per_point = ("k_flux_part x 4 + k_stage_split (one stage, FP64)",
                                        FLUX_SPLIT_FP64_FLOPS_PER_NEIGHBOUR,
                                        FLUX_SPLIT_DRAM_BYTES_PER_POINT)
        peak, peak_src = FP64_PEAK_TFLOPS, "derived: 152 SMs x 2 FP64 FMA/clk/SM x 2 flops x 2.07 GHz"
    else:
        kernel, per_entry, per_point = ("k_flux (flux residual + SSP-RK stage update, FP64)",
                                        FLUX_FP64_FLOPS_PER_NEIGHBOUR, FLUX_DRAM_BYTES_PER_POINT)
        peak, peak_src = FP64_PEAK_TFLOPS, "derived: 152 SMs x 2 FP64 FMA/clk/SM x 2 flops x 2.07 GHz"
    achieved = per_entry * nnz * n_cond / launch_s / 1e12 if per_entry else None
    mp, mp_kind = _peaks()
    hbm = mp["hbm_gbs"] * 1e9
    step_s = ms_per_step * 1e-3
    layout = layout_bytes_per_point_iteration(mixed, nnz / n)
    return {"kernel": kernel, "bound": "alu", "unit": "TFLOP/s", "achieved": achieved,
            "peak": peak, "frac": achieved / peak if achieved else None, "peak_source": peak_src,
            "launch_ms": launch_s * 1e3,
            "traffic": per_point * n * n_cond if per_point else None,
            "traffic_note": "ncu dram bytes of a 0.6M-point launch, scaled by points x conditions",
            "hbm_frac_of_measured_whole_step": {
                "algorithmic": ALGORITHMIC_BYTES_PER_POINT_ITERATION * n * n_cond / step_s / hbm,
                "layout": layout * n * n_cond / step_s / hbm,
                "layout_bytes_per_point_iteration": layout,
                "peak_gbs": mp["hbm_gbs"], "peak_kind": mp_kind}}


def inner_region(cloud, n_target: int, mach: float = MACH, alpha: float = ALPHA):
    """The inner layers of `cloud` (generator layers 0..L, L the first layer at
    which the region holds `n_target` points) as a cloud of its own, with the
    state to time on it. Stencils reach two layers out, so every point below
    layer L - 1 keeps its whole stencil; layers L - 1 and L are held at the
    given state (far-field flag), so the region is the same problem at the
    same resolution on a bounded part of the cloud."""
    from paper_2108_07031_gb300 import cloud as Cl
    counts = np.cumsum(np.bincount(cloud.l, minlength=cloud.n_r))
    L = int(min(np.searchsorted(counts, n_target), cloud.n_r - 1))
    members = np.flatnonzero(cloud.l <= L)
    local = np.full(cloud.n, -1, dtype=np.int64)
    local[members] = np.arange(members.size)
    off, idx = cloud.nbr_offsets, cloud.nbr_idx
    nb = [local[idx[off[i]:off[i + 1]]] for i in members]
    nb = [a[a >= 0] for a in nb]
    new_off = np.zeros(members.size + 1, dtype=np.int32)
    new_off[1:] = np.cumsum([a.size for a in nb])
    flags = cloud.flags[members].copy()
    normals = cloud.normals[members].copy()
    rim = cloud.l[members] >= L - 1
    flags[rim] = Cl.FLAG_OUTER
    d = cloud.xy[members][rim] - np.array(Cl.FAR_FIELD_CENTRE)
    normals[rim] = d / np.hypot(d[:, 0], d[:, 1])[:, None]
    region = Cl.Cloud(xy=cloud.xy[members], normals=normals, flags=flags, nbr_offsets=new_off,
                      nbr_idx=np.concatenate(nb).astype(np.int32), n_c=cloud.n_c, n_r=L + 1,
                      k=cloud.k[members], l=cloud.l[members])
    W = Cl.perturbed_state(cloud, mach, alpha)[members]
    return region, W, L


def _oracle_region(args):
    """The oracle on the inner region of the workload's own cloud."""
    from oracle import oracle as O
    cloud = _cloud(args.points)
    region, W, L = inner_region(cloud, SAMPLE_POINTS, args.mach, args.alpha)
    return O, O.OracleCloud.from_cloud(region), W, region.n, L, cloud.n


def _region_sample_text(n, L, n_all, what):
    return (f"{what} of the FP64 CPU oracle on the inner {L + 1} layers of the workload's own "
            f"{n_all}-point cloud ({n} points, the two outermost layers held), from the same kind "
            f"of developed state")


def cpu_baseline(args):
    O, oc, W, n, L, n_all = _oracle_region(args)
    t0 = time.perf_counter()
    _, _, st = O.iterate(oc, W, 2)
    rate = n * 2 / (time.perf_counter() - t0)
    if st != 0:
        raise RuntimeError(f"oracle sample diverged at iteration {st}")
    return {"value": rate, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": _region_sample_text(n, L, n_all, "2 iterations")}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    O, oc, W, n, L, n_all = _oracle_region(args)
    for _ in range(args.warmup):
        W, _, st = O.iterate(oc, W, 1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        W, _, st = O.iterate(oc, W, 1)
        times.append(time.perf_counter() - t0)
        if st != 0:  # a diverged iteration stops early: its time is not a step
            raise RuntimeError("oracle sample diverged")
    total = sum(times)
    value = n * args.steps / total
    cores = O.num_threads()
    sample = _region_sample_text(n, L, n_all, f"1 iteration per step, on {cores} host cores,")
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        # the arms share the workload's config; the points this arm actually
        # iterates (a bounded inner region of that cloud) are named here
        "config": workload_config(args.points, world, mach=args.mach, alpha=args.alpha),
        "timed_points": n,
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": cores,
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--points", type=int, default=WORKLOAD_POINTS)
    ap.add_argument("--mach", type=float, default=MACH)
    ap.add_argument("--alpha", type=float, default=ALPHA, help="angle of attack, degrees")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--flux-split", action="store_true",
                    help="run the headline with the split flux kernels (profiling the ablation)")
    ap.add_argument("--variants", default="all",
                    help="comma-separated variants to time after the headline (default all: "
                         + ", ".join(VARIANTS) + ")")
    ap.add_argument("--no-variants", dest="variants", action="store_const", const="",
                    help="time the headline only")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)  # at least three untimed warm-up steps
    args.steps = max(args.steps, 1)
    rank, world, local = _dist()
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        res = run_ours(args, rank, world, local)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
