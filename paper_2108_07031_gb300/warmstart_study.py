"""Warm-start study: train the surrogate on converged solutions from the
batched solver and measure what it gains over the free-stream start.

  python -m paper_2108_07031_gb300.warmstart_study [--out results.json]

Cloud: the NACA 0012 cloud of --cloud points (default 128 x 40 = 5,120).
Training: --train seeded conditions (default 256), M ~ U[0.3, 0.8],
alpha ~ U[-4, 6] deg, each solved by the batched mixed-precision solver (64
conditions per launch, CFL 0.8: the converged state does not depend on the
pseudo-time step) to a 7-order residue drop. Network: the 6-layer,
width-256 BF16 tensor-core MLP, Adam with a cosine schedule; with
--ensemble K, K networks from different seeds whose predicted states are
averaged. Evaluation: 32 held-out conditions (another seed), each
solved from the free stream and from the network's prediction (whose
far-field points keep the exact free stream: they are boundary data) at the
configuration's CFL 0.2 (--eval-cfl); reported: iterations until the residue
is 1e-6 of the free-stream start's first residue, and the converged Cl/Cd of
both.
"""

from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np


def main():
    import torch

    from . import cloud as Cl
    from . import lskum as L
    from . import surrogate as S

    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="warmstart_study.json")
    ap.add_argument("--cloud", default="128x40", help="n_c x n_r of the NACA 0012 cloud")
    ap.add_argument("--data-iters", type=int, default=40_000,
                    help="iteration budget per batch of training solves")
    ap.add_argument("--train", type=int, default=256)
    ap.add_argument("--test", type=int, default=32)
    ap.add_argument("--epochs", type=int, default=240)
    ap.add_argument("--ensemble", type=int, default=1,
                    help="networks trained from different seeds; the prediction is their mean state")
    ap.add_argument("--eval-cfl", type=float, default=0.2)
    ap.add_argument("--eval-iters", type=int, default=60_000)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--proj-scales", default="1,1,1,1,1,1,1,1",
                    help="standard deviations of the 8 Fourier projections")
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--features", default="fourier", choices=["fourier", "wall"],
                    help="network inputs: the library's Fourier encoding, or wall-loop "
                         "position harmonics (surrogate.wall_features)")
    ap.add_argument("--data-cache", default="",
                    help="file (.npy) to keep the converged training states in between runs")
    ap.add_argument("--save-states", default="",
                    help="file (.npz) for the held-out conditions' final states of both starts")
    args = ap.parse_args()
    prec = L.MIXED if args.precision == "mixed" else L.FP64
    log = lambda m: print(m, flush=True)  # noqa: E731

    n_c, n_r = (int(v) for v in args.cloud.lower().split("x"))
    cloud = Cl.naca0012_cloud(n_c, n_r)
    wd = S.wall_distance(cloud)
    m_tr, a_tr = Cl.conditions(args.train, seed=2021)
    m_te, a_te = Cl.conditions(args.test, seed=4242)
    t0 = time.time()
    if args.data_cache and os.path.exists(args.data_cache):
        W_tr, it_tr = np.load(args.data_cache), []
    else:
        W_tr, it_tr = S.converged_solutions(cloud, m_tr, a_tr, tol=1e-7,
                                            max_iters=args.data_iters)
        if args.data_cache:
            np.save(args.data_cache, W_tr)
    t_data = time.time() - t0
    log(f"training data: {args.train} conditions in {t_data:.1f} s (iterations per batch {it_tr})")

    raw = np.concatenate(S.raw_inputs(cloud, wd, m_tr, a_tr))
    T = np.concatenate([S.targets(W_tr[k], m_tr[k], a_tr[k]) for k in range(args.train)])
    scales = [float(v) for v in args.proj_scales.split(",")]
    arc = S.wall_arc(cloud) if args.features == "wall" else None
    Td = torch.from_numpy(T).cuda()
    nets, losses = [], []
    t0 = time.time()
    for e in range(args.ensemble):
        net = S.MLP(capacity=16384, seed=e, proj=S.projection(scales=scales))
        if arc is None:
            feats = net.features(torch.from_numpy(raw).cuda())
        else:
            feats = torch.from_numpy(np.concatenate(
                [S.wall_features(cloud, wd, arc, m_tr[k], a_tr[k], net.proj)
                 for k in range(args.train)])).cuda()
        losses_e = S.train(net, feats, Td, epochs=args.epochs, batch=args.batch, lr=2e-3,
                           lr_final=2e-5, seed=e, log=log)
        nets.append(net)
        losses.append(losses_e)
        del feats
    t_train = time.time() - t0

    # held-out: both starts in one batched solve each (32 conditions)
    n = args.test
    nc = 1 << int(np.ceil(np.log2(n)))
    pred, fallback = [], 0
    for k in range(n):
        Ws = [S.predict_state(net, cloud, wd, m_te[k], a_te[k], arc=arc) for net in nets]
        Ws = [w for w in Ws if w is not None]
        W = np.mean(Ws, axis=0) if Ws else None
        if W is None:
            fallback += 1
            W = np.tile(S.freestream(m_te[k], a_te[k]), (cloud.n, 1))
        pred.append(W)
    # prediction error against the reference solutions computed below
    results = {}
    chunk = 100
    for mode in ("cold", "warm"):
        with L.Solver.from_cloud(cloud, precision=prec, cfl=args.eval_cfl, n_conditions=nc) as s:
            mm = np.concatenate([m_te, np.repeat(m_te[-1:], nc - n)])
            aa = np.concatenate([a_te, np.repeat(a_te[-1:], nc - n)])
            s.set_conditions(mm, aa)
            if mode == "cold":
                s.step(2)
                r_first = s.residual_norm()[:n].copy()
                s.set_conditions(mm, aa)
            else:
                W0 = np.concatenate([np.stack(pred), np.repeat(np.stack(pred)[-1:], nc - n, 0)])
                s.set_state(W0)
            hist = []
            t0 = time.time()
            for _ in range(args.eval_iters // chunk):
                s.step(chunk)
                hist.append(s.residual_norm()[:n].copy())
            cl, cd = s.forces()
            W_end = s.get_state()[:n]
            results[mode] = {"hist": np.array(hist), "cl": cl[:n], "cd": cd[:n], "W": W_end,
                             "time": time.time() - t0}
    thr = 1e-6 * r_first
    def first_below(h):
        ok = h < thr[None, :]
        return np.where(ok.any(0), chunk * (1 + ok.argmax(0)), -1)
    it_cold = first_below(results["cold"]["hist"])
    it_warm = first_below(results["warm"]["hist"])
    both = (it_cold > 0) & (it_warm > 0)
    saving = 1 - it_warm[both] / it_cold[both]
    pred_err = [float(np.abs(pred[k] - results["cold"]["W"][k]).max() /
                      np.abs(results["cold"]["W"][k]).max()) for k in range(n)]
    out = {
        "cloud_points": cloud.n, "train_conditions": args.train, "test_conditions": n,
        "eval_cfl": args.eval_cfl, "precision": args.precision, "proj_scales": scales,
        "features": args.features,
        "epochs": args.epochs,
        "data_seconds": t_data, "train_seconds": t_train,
        "ensemble": args.ensemble,
        "loss_first": losses[0][0], "loss_last": [l[-1] for l in losses], "fallbacks": fallback,
        "iterations_cold": it_cold.tolist(), "iterations_warm": it_warm.tolist(),
        "converged_both": int(both.sum()),
        "saving_mean": float(saving.mean()) if saving.size else None,
        "saving_median": float(np.median(saving)) if saving.size else None,
        "saving_min": float(saving.min()) if saving.size else None,
        "cl_cold": results["cold"]["cl"].tolist(), "cl_warm": results["warm"]["cl"].tolist(),
        "cd_cold": results["cold"]["cd"].tolist(), "cd_warm": results["warm"]["cd"].tolist(),
        "dcl_abs_mean": float(np.mean(np.abs(results["warm"]["cl"] - results["cold"]["cl"]))),
        "dcd_abs_mean": float(np.mean(np.abs(results["warm"]["cd"] - results["cold"]["cd"]))),
        "dcl_abs_max": float(np.max(np.abs(results["warm"]["cl"] - results["cold"]["cl"]))),
        "dcd_abs_max": float(np.max(np.abs(results["warm"]["cd"] - results["cold"]["cd"]))),
        "residue_first_cold": r_first.tolist(),
        "residue_after_100_cold": results["cold"]["hist"][0].tolist(),
        "residue_after_100_warm": results["warm"]["hist"][0].tolist(),
        "residue_end_cold": results["cold"]["hist"][-1].tolist(),
        "residue_end_warm": results["warm"]["hist"][-1].tolist(),
        "eval_iters": args.eval_iters,
        "prediction_rel_err_max_mean": float(np.mean(pred_err)),
        "mach": m_te.tolist(), "alpha": a_te.tolist(),
    }
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    if args.save_states:
        np.savez(args.save_states, cold=results["cold"]["W"], warm=results["warm"]["W"],
                 mach=m_te, alpha=a_te)
    log(json.dumps({k: v for k, v in out.items() if not isinstance(v, list)}))


if __name__ == "__main__":
    main()
