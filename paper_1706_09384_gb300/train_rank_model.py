"""Trains the rank predictor on ranks the method itself produces.

Training set: unit-cube surface clouds (R2 sequence, seeded) with
n_c in {16384, 32768, 65536}, k_s in {2, 4, 8, 16, 32}, eps in {1e-3, 1e-4, 1e-5},
U kernel, leaf 64, eta 3; every admissible block of every build is one sample
(features and ACA rank, see include/hm.h).  Usage:

    python -m paper_1706_09384_gb300.train_rank_model OUT.npy [--steps N]
    python -m paper_1706_09384_gb300.train_rank_model --eval [WEIGHTS.npy]

--eval builds the 262144-point cube-surface cloud at k_s = 24 (U kernel,
eps 1e-4, leaf 64, eta 3) with and without the model and prints, for each,
the ACA batches, re-runs after overflow, workspace and build times, and
whether the ranks agree.
"""
import argparse
import json
import time

import numpy as np

from . import hm, inputs, rank_model


def collect(ncs=(16384, 32768, 65536), kss=(2.0, 4.0, 8.0, 16.0, 32.0), epss=(1e-3, 1e-4, 1e-5),
            leaf=64, eta=3.0, seed=0):
    F, T, info = [], [], []
    q = 0
    for nc in ncs:
        for ks in kss:
            for eps in epss:
                pts, _ = inputs.cube_surface(nc, seed=seed + q)
                rho, lam, mu, om = inputs.material(ks)
                t0 = time.time()
                H = hm.HMatrix.build(pts, None, rho, lam, mu, om, "U", eps, eta, leaf)
                f, t = H.rank_samples()
                F.append(f)
                T.append(t)
                info.append(dict(nc=nc, ks=ks, eps=eps, blocks=len(t), build_s=time.time() - t0))
                H.free()
                q += 1
    return np.concatenate(F), np.concatenate(T), info


def evaluate(P, nc=262144, ks=24.0, seed=99):
    import torch
    pts, _ = inputs.cube_surface(nc, seed=seed)
    rho, lam, mu, om = inputs.material(ks)
    out, blocks = {"n_c": nc, "kappa_s": ks}, []
    for use in (False, True):
        torch.cuda.synchronize()
        t0 = time.time()
        H = hm.HMatrix.build(pts, None, rho, lam, mu, om, "U", 1e-4, 3.0, 64,
                             opts=hm.hm_opts_default(rank_model=P if use else None))
        torch.cuda.synchronize()
        s = H.stats()
        out["binned" if use else "unbinned"] = {
            "build_s": time.time() - t0, "aca_ms": s["device_ms"]["aca"],
            "recompress_ms": s["device_ms"]["recompress"], "aca_batches": s["aca_batches"],
            "overflow_reruns": s["aca_overflow_reruns"],
            "workspace_total_GB": s["aca_workspace_total_bytes"] / 1e9,
            "workspace_peak_GB": s["aca_workspace_peak_bytes"] / 1e9,
            "rank_aca_mean": s["rank_aca_mean"], "rank_aca_max": s["rank_aca_max"]}
        b = H.blocks()
        blocks.append((b["rank_aca"].copy(), b["rank"].copy()))
        if not use:
            f, t = H.rank_samples()
        H.free()
    out["ranks_equal"] = bool(all(np.array_equal(a, b) for a, b in zip(blocks[0], blocks[1])))
    pred = rank_model.predict(P, f) * P[13] + P[12]
    out["rank_mae"] = float(np.abs(3 * np.expm1(pred) - 3 * np.expm1(t)).mean())
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("out", nargs="?")
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--eval", action="store_true")
    args = ap.parse_args()
    if args.eval:
        P = rank_model.load(args.out) if args.out else rank_model.load()
        print(json.dumps(evaluate(P)))
        return
    F, T, info = collect()
    P, losses = rank_model.train(F, T, steps=args.steps, batch=4096, lr=2e-3, seed=args.seed)
    np.save(args.out, P)
    pred = rank_model.predict(P, F) * P[13] + P[12]
    rank_true = 3 * np.expm1(T)
    rank_pred = 3 * np.expm1(pred)
    print(json.dumps({"samples": int(len(T)), "builds": info,
                      "loss_first100": float(losses[:100].mean()),
                      "loss_last100": float(losses[-100:].mean()),
                      "rank_mae": float(np.abs(rank_pred - rank_true).mean()),
                      "rank_true_mean": float(rank_true.mean())}))


if __name__ == "__main__":
    main()
