"""Mixed precision against FP64 on large clouds.

  python -m paper_2108_07031_gb300.precision_study --points 10000000 --iters 200 \
      [--mach 0.85 --alpha 1.0] [--out precision_study.json]

Runs the same iterations from the free stream in both precisions on one
NACA 0012 cloud (shuffled input order, the benchmark's family) and reports
the lift and drag of both, the norm-wise state difference, the residue
histories and the time per iteration of each. The FP64 path is the one the
parity tests hold to the FP64 CPU oracle; at these sizes the oracle itself
would need hours per thousand iterations.
"""

from __future__ import annotations

import argparse
import json
import time

import numpy as np


def _run(cloud, precision, mach, alpha, iters, chunk):
    import torch

    from . import lskum as L
    t0 = time.perf_counter()
    with L.Solver.from_cloud(cloud, precision=precision) as s:
        t_create = time.perf_counter() - t0
        s.set_freestream(mach, alpha)
        s.step(2)  # warm-up: builds the iteration graph
        s.set_freestream(mach, alpha)
        torch.cuda.synchronize()
        hist, t_iter = [], 0.0
        done = 0
        while done < iters:
            k = min(chunk, iters - done)
            t0 = time.perf_counter()
            s.step(k)
            r = s.residual_norm()
            t_iter += time.perf_counter() - t0
            done += k
            hist.append((done, r))
        cl, cd = s.forces()
        W = s.get_state()
    return {"cl": cl, "cd": cd, "hist": hist, "seconds_per_iteration": t_iter / iters,
            "create_seconds": t_create}, W


def main():
    from . import cloud as Cl
    from . import lskum as L

    ap = argparse.ArgumentParser()
    ap.add_argument("--points", type=int, default=10_000_000)
    ap.add_argument("--iters", type=int, default=200)
    ap.add_argument("--chunk", type=int, default=50)
    ap.add_argument("--mach", type=float, default=0.85)
    ap.add_argument("--alpha", type=float, default=1.0)
    ap.add_argument("--out", default="precision_study.json")
    args = ap.parse_args()

    n_c, n_r = Cl.cloud_dims(args.points)
    t0 = time.perf_counter()
    cloud = Cl.naca0012_cloud(n_c, n_r, shuffle=True)
    t_cloud = time.perf_counter() - t0
    out = {"points": cloud.n, "n_c": n_c, "n_r": n_r, "mach": args.mach, "alpha_deg": args.alpha,
           "iterations": args.iters, "cloud_seconds": t_cloud}
    r64, W64 = _run(cloud, L.FP64, args.mach, args.alpha, args.iters, args.chunk)
    rmx, Wmx = _run(cloud, L.MIXED, args.mach, args.alpha, args.iters, args.chunk)
    scale = np.abs(W64).max(axis=0)
    out["fp64"] = r64
    out["mixed"] = rmx
    out["state_normwise_diff"] = float((np.abs(Wmx - W64).max(axis=0) / scale).max())
    out["dcl"] = abs(rmx["cl"] - r64["cl"])
    out["dcd"] = abs(rmx["cd"] - r64["cd"])
    out["residue_rel_diff_last"] = abs(rmx["hist"][-1][1] - r64["hist"][-1][1]) / r64["hist"][-1][1]
    out["speedup_mixed"] = r64["seconds_per_iteration"] / rmx["seconds_per_iteration"]
    out["mixed_point_iterations_per_s"] = cloud.n / rmx["seconds_per_iteration"]
    out["fp64_point_iterations_per_s"] = cloud.n / r64["seconds_per_iteration"]
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: v for k, v in out.items() if not isinstance(v, dict)}), flush=True)


if __name__ == "__main__":
    main()
