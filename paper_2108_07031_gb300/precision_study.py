"""Mixed precision against FP64 on large clouds.

  python -m paper_2108_07031_gb300.precision_study --points 10000000 --iters 200 \
      [--mach 0.85 --alpha 1.0] [--cfl 0.2] [--option wall_factor=1] [--out precision_study.json]

Runs the same iterations from the free stream in both precisions on one
NACA 0012 cloud (shuffled input order, the benchmark's family) and reports
the lift and drag of both, the norm-wise state difference, the residue
histories and the time per iteration of each. If the state turns
non-physical (the solver's DIVERGED status), the run stops, records the
iteration window, and the comparison uses the last state snapshot before it
(the same iteration in both precisions, checked). The FP64 path is the one the
parity tests hold to the FP64 CPU oracle; at these sizes the oracle itself
would need hours per thousand iterations.
"""

from __future__ import annotations

import argparse
import json
import time

import numpy as np


def _run(cloud, precision, mach, alpha, iters, chunk, cfl, snapshot_every, options):
    """Runs `iters` iterations from the free stream. Returns the forces, the
    residue history, the time per iteration and the state at the last
    snapshot (every `snapshot_every` chunks, and at the end); if the state
    turns non-physical, the iteration window where it did and the last
    snapshot before it."""
    import torch

    from . import lskum as L
    t0 = time.perf_counter()
    with L.Solver.from_cloud(cloud, precision=precision, cfl=cfl, **options) as s:
        t_create = time.perf_counter() - t0
        s.set_freestream(mach, alpha)
        s.step(2)  # warm-up: builds the iteration graph
        s.set_freestream(mach, alpha)
        torch.cuda.synchronize()
        hist, t_iter = [], 0.0
        done, n_chunk, diverged = 0, 0, None
        snap = {"iteration": 0, "W": s.get_state(), "cl": 0.0, "cd": 0.0}
        while done < iters:
            k = min(chunk, iters - done)
            t0 = time.perf_counter()
            try:
                s.step(k)
            except L.LskumError as e:
                if e.code != L.ERR_DIVERGED:
                    raise
                diverged = [done, done + k]
                break
            r = s.residual_norm()
            t_iter += time.perf_counter() - t0
            done += k
            n_chunk += 1
            hist.append((done, r))
            if n_chunk % snapshot_every == 0 or done == iters:
                cl, cd = s.forces()
                snap = {"iteration": done, "W": s.get_state(), "cl": cl, "cd": cd}
    out = {"cl": snap["cl"], "cd": snap["cd"], "compared_iteration": snap["iteration"],
           "hist": hist, "seconds_per_iteration": t_iter / max(done, 1),
           "create_seconds": t_create, "diverged_between": diverged}
    return out, snap["W"]


def parse_options(items) -> dict:
    """NAME=VALUE strings into solver option keywords: a value with a decimal
    point or an exponent is a float, anything else an int."""
    options = {}
    for kv in items:
        name, sep, value = kv.partition("=")
        if not sep or not name:
            raise ValueError(f"expected NAME=VALUE, got {kv!r}")
        options[name] = float(value) if any(ch in value for ch in ".eE") else int(value)
    return options


def main():
    from . import cloud as Cl
    from . import lskum as L

    ap = argparse.ArgumentParser()
    ap.add_argument("--points", type=int, default=10_000_000)
    ap.add_argument("--iters", type=int, default=200)
    ap.add_argument("--chunk", type=int, default=50)
    ap.add_argument("--snapshot-every", type=int, default=1,
                    help="chunks between state snapshots (the comparison falls back to the "
                         "last one if the state turns non-physical)")
    ap.add_argument("--mach", type=float, default=0.85)
    ap.add_argument("--alpha", type=float, default=1.0)
    ap.add_argument("--cfl", type=float, default=0.2)
    ap.add_argument("--option", action="append", default=[], metavar="NAME=VALUE",
                    help="a solver option for both precisions (lskum_options field), "
                         "e.g. wall_factor=1 or order=1; repeatable")
    ap.add_argument("--out", default="precision_study.json")
    args = ap.parse_args()
    options = parse_options(args.option)

    n_c, n_r = Cl.cloud_dims(args.points)
    t0 = time.perf_counter()
    cloud = Cl.naca0012_cloud(n_c, n_r, shuffle=True)
    t_cloud = time.perf_counter() - t0
    out = {"points": cloud.n, "n_c": n_c, "n_r": n_r, "mach": args.mach, "alpha_deg": args.alpha,
           "iterations": args.iters, "cfl": args.cfl, "options": options,
           "cloud_seconds": t_cloud}
    r64, W64 = _run(cloud, L.FP64, args.mach, args.alpha, args.iters, args.chunk, args.cfl,
                    args.snapshot_every, options)
    rmx, Wmx = _run(cloud, L.MIXED, args.mach, args.alpha, args.iters, args.chunk, args.cfl,
                    args.snapshot_every, options)
    scale = np.abs(W64).max(axis=0)
    out["fp64"] = r64
    out["mixed"] = rmx
    out["state_normwise_diff"] = float((np.abs(Wmx - W64).max(axis=0) / scale).max())
    out["dcl"] = abs(rmx["cl"] - r64["cl"])
    out["dcd"] = abs(rmx["cd"] - r64["cd"])
    if r64["compared_iteration"] != rmx["compared_iteration"]:
        raise RuntimeError("the two precisions stopped at different iterations: "
                           f"{r64['diverged_between']} vs {rmx['diverged_between']}")
    h64 = dict(r64["hist"])
    hmx = dict(rmx["hist"])
    it = r64["compared_iteration"]
    out["compared_iteration"] = it
    out["residue_rel_diff_at_compared"] = abs(hmx[it] - h64[it]) / h64[it] if it in h64 else None
    out["speedup_mixed"] = r64["seconds_per_iteration"] / rmx["seconds_per_iteration"]
    out["mixed_point_iterations_per_s"] = cloud.n / rmx["seconds_per_iteration"]
    out["fp64_point_iterations_per_s"] = cloud.n / r64["seconds_per_iteration"]
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: v for k, v in out.items() if not isinstance(v, dict)}), flush=True)


if __name__ == "__main__":
    main()
