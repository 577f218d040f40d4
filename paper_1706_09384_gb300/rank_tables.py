"""Rank statistics of the H-matrix on the paper's sphere meshes (vertex clouds
of the subdivided icosahedron, N_c = 10 * 4^l + 2), for a comparison with the
rank tables of Sec. 7.2 and the growth of the ranks with the frequency
(Sec. 8: about flat in N_c at fixed omega, growing with omega at fixed
points per wavelength).  Point kernel U (or T), rho = mu = 1, lambda = 2,
eta = 3, eps = 1e-4, N_leaf = 100 as in Sec. 7 (--leaf to change it).  Prints
one JSON line per build:
min / mean / max ACA and recompressed ranks of the admissible blocks, overall
and per level of the row cluster.

    python -m paper_1706_09384_gb300.rank_tables [--levels 3 4 5 6] [--omegas 3 14]
                                                  [--ppw 10] [--kernel U] [--leaf 100]
"""
import argparse
import json
import math
import time

import numpy as np

from . import hm, inputs


def rank_stats(H):
    blk = H.blocks()
    _, cl = H.tree()
    adm = blk[blk["admissible"] == 1]
    out = {"blocks": int(len(blk)), "admissible": int(len(adm))}
    if len(adm) == 0:
        return out
    for key in ("rank_aca", "rank"):
        v = adm[key].astype(np.int64)
        out[key] = {"min": int(v.min()), "mean": float(v.mean()), "max": int(v.max())}
    lev = cl["level"][adm["tau"]]
    out["by_level"] = {int(l): {"n": int((lev == l).sum()),
                                "rank_aca_max": int(adm["rank_aca"][lev == l].max()),
                                "rank_max": int(adm["rank"][lev == l].max()),
                                "rank_mean": float(adm["rank"][lev == l].mean())}
                       for l in sorted(set(lev.tolist()))}
    return out


def run(level, omega, kernel="U", eps=1e-4, leaf=100):
    pts, nrm = inputs.icosphere(level)
    t0 = time.time()
    H = hm.HMatrix.build(pts, nrm if kernel == "T" else None, 1.0, 2.0, 1.0, omega, kernel, eps,
                         3.0, leaf)
    res = {"level": level, "n_c": len(pts), "omega": omega, "kappa_s": omega,
           "points_per_wavelength": 2 * math.pi / omega / math.sqrt(4 * math.pi / len(pts)),
           "kernel": kernel, "leaf": leaf, "build_s": time.time() - t0}
    res.update(rank_stats(H))
    H.free()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--levels", type=int, nargs="+", default=[3, 4, 5, 6])
    ap.add_argument("--omegas", type=float, nargs="+", default=[3.0, 14.0])
    ap.add_argument("--ppw", type=float, default=10.0,
                    help="also run every level at this many points per S-wavelength")
    ap.add_argument("--kernel", default="U", choices=["U", "T"])
    ap.add_argument("--leaf", type=int, default=100, help="N_leaf (the paper uses 100)")
    args = ap.parse_args()
    for level in args.levels:
        for om in args.omegas:
            print(json.dumps(run(level, om, args.kernel, leaf=args.leaf)), flush=True)
    if args.ppw > 0:
        for level in args.levels:
            n = 10 * 4 ** level + 2
            h = math.sqrt(4 * math.pi / n)  # mean spacing on the unit sphere
            print(json.dumps(run(level, 2 * math.pi / (args.ppw * h), args.kernel, leaf=args.leaf)),
                  flush=True)


if __name__ == "__main__":
    main()
