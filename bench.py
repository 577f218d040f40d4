"""Benchmark of the H-matrix hot path on GB300 (one JSON line on stdout).

Workload (default): 65 536 Fibonacci points on the unit sphere, k_s = 16
(rho = mu = 1, lambda = 2), U kernel, leaf 64, eta = 3, eps = 1e-4, FP32
complex storage with FP64 Green's tensors, seeded N(0,1) complex RHS.

One step = the whole hot path over the workload: H-matrix build (cluster
tree, block partition, near-field Green's tensors, batched vector ACA,
QR/SVD recompression, storage layout), `--matvecs` H-matrix-vector products
and a GMRES(100) solve to 1e-6.  The matrix carries the quadrature weights
w_j = 4 pi / n_c of the collocation matrix (Sec. 4), which keeps the system
well conditioned (without them GMRES stalls at this size).  `value` is the H-matvec throughput in GB/s (algorithmic bytes of
the stored H-matrix plus x and y per product / device time of the products);
`build_s` is the device-synchronised build time per step.  The stored
H-matrix (~8.5 GB) is far larger than L2, so no flush is needed between
products.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (every S-th block of the same partition), on the host cores.
Multi-GPU (torchrun): independent replicas, one per rank (weak scaling).
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("H-matvec GB/s (% HBM peak) + build s, mixed vs plain GPU form at rel.err≤3ε")

WORKLOADS = {
    "sphere65536_ks16_U": dict(nc=65536, ks=16.0, kernel="U", leaf=64, eta=3.0, eps=1e-4),
    "sphere16384_ks16_U": dict(nc=16384, ks=16.0, kernel="U", leaf=64, eta=3.0, eps=1e-4),
    "sphere1536_ks4_U": dict(nc=1536, ks=4.0, kernel="U", leaf=32, eta=3.0, eps=1e-4),
}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def kernel_profile(kernel_file, kernel_name):
    """The committed ncu summary of a kernel (profiles/traffic.json), only if the
    kernel source is unchanged since the capture (sha256 of the .cu file)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    src = os.path.join(ROOT, "paper_1706_09384_gb300", "csrc", kernel_file)
    if not os.path.exists(p) or not os.path.exists(src):
        return None
    d = json.load(open(p)).get(kernel_name)
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()
    return d if d and d.get("source_sha256") == h else None


def kernel_traffic(kernel_file, kernel_name, alg_bytes=None):
    """DRAM bytes per launch from a committed ncu summary, only if the kernel
    source is unchanged since the capture (sha256 of the .cu file): the
    recorded DRAM bytes per algorithmic byte of the captured launch times this
    launch's algorithmic bytes (the captured case is smaller than the bench's
    where a full-size capture would hold too much device memory)."""
    d = kernel_profile(kernel_file, kernel_name)
    if not d:
        return None
    if "dram_per_alg_byte" in d and alg_bytes:
        return d["dram_per_alg_byte"] * alg_bytes
    return d.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None
        self.skip = 0

    def __enter__(self):
        # the sampler is started and its first sample awaited before the timed
        # region begins: nvidia-smi's start-up (driver and NVML initialisation)
        # then cannot stall the timed work; that first sample is not counted
        self.skip = 0
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        if self.p:
            t0 = time.time()
            while time.time() - t0 < 10.0 and self.p.poll() is None:
                self.f.flush()
                with open(self.f.name) as g:
                    self.skip = sum(1 for _ in g)
                if self.skip:
                    break
                time.sleep(0.02)
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        try:
            for q, line in enumerate(open(self.f.name)):
                parts = [x.strip() for x in line.split(",")]
                if q >= self.skip and len(parts) >= 9:
                    rows.append(parts)
        finally:
            os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(num(r[2]) or 0 for r in rows), "reasons": reasons,
                "samples": len(rows)}


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v):
    """The slowest rank's time (replicas: the job ends when the last one does)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, bytes_per_product, products_per_rank, max_ms):
    """GB/s of the whole job: the products of all ranks over the slowest rank's time."""
    return world * bytes_per_product * products_per_rank / (max_ms * 1e-3) / 1e9


def cpu_baseline(wl, budget_s=20.0):
    """The oracle, as it stands, on a bounded sample of the workload: every
    S-th block of the same partition is built (OpenMP over blocks), then the
    oracle's serial H-matvec over those blocks is timed.  Returns GB/s counted
    with the same algorithmic bytes as the GPU (complex64 entries + x, y)."""
    import oracle as O
    from paper_1706_09384_gb300 import inputs
    pts = inputs.fibonacci_sphere(wl["nc"])
    rho, lam, mu, om = inputs.material(wl["ks"])
    pb = O.problem(rho, lam, mu, om, wl["kernel"])
    stride = 97 if wl["nc"] > 10000 else 1
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    H = O.HMatrix(pb, pts, None, wl["eps"], wl["eta"], wl["leaf"], True, stride, threads)
    build_s = time.perf_counter() - t0
    blk, ra, r = H.blocks()
    cl = H.clusters()
    sz = cl["end"] - cl["begin"]
    m, n = 3 * sz[blk["tau"]], 3 * sz[blk["sigma"]]
    built = r >= 0
    ent = np.where(blk["admissible"] == 1, r * (m + n), m * n)[built].sum()
    nbytes = 8 * ent + 2 * 16 * 3 * wl["nc"]
    x = inputs.random_rhs(3 * wl["nc"], seed=0)
    H.matvec(x)
    reps, t = 0, 0.0
    while t < min(budget_s, 10.0) and reps < 20:
        t1 = time.perf_counter()
        H.matvec(x)
        t += time.perf_counter() - t1
        reps += 1
    return {"value": nbytes * reps / t / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": ("every %d-th block of the %d-point partition (%d of %d blocks) built by the "
                       "oracle on %d threads in %.1f s; oracle H-matvec (serial, FP64) over those "
                       "blocks timed %d times" % (stride, wl["nc"], int(built.sum()), len(blk),
                                                  threads, build_s, reps)),
            "build_threads": threads, "sample_build_s": build_s}


def workload_config(args, wl, form, world):
    """The workload as both arms report it (the reference arm times the oracle
    on a sample of the same workload)."""
    return {"workload": args.workload, "n_c": wl["nc"], "kappa_s": wl["ks"],
            "kernel": wl["kernel"], "leaf": wl["leaf"], "eta": wl["eta"], "eps": wl["eps"],
            "weights": "4 pi / n_c (W_y of Sec. 4)",
            "storage": ("bf16-complex, one fp32 scale per block and factor for U and V, "
                        "dense blocks unscaled (products); fp32 for refinement residuals")
            if form == "mixed" else "fp32-complex",
            "form": form, "rank_model": 1 if form == "mixed" else 0,
            "green": "fp64", "matvecs_per_step": args.matvecs,
            "gmres": "GMRES(100) to 1e-6, FP64 vectors",
            "parallelism": "replicas" if world > 1 else "1gpu",
            "l2": "no flush: every product streams the whole stored operator (GBs) >> 129 MB L2"}


def run_reference(args, wl, world, rank):
    if rank != 0:
        return
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(wl)
    t0 = time.perf_counter()
    info = None
    for _ in range(args.steps):
        info = cpu_baseline(wl)
        vals.append(info["value"])
    wall = time.perf_counter() - t0
    v = statistics.median(vals)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(args, wl, args.form, world),
           "cpu_baseline": {"kind": "oracle", "cores": info["cores"], "sample": info["sample"],
                            "value": v, "unit": "GB/s"},
           "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


FP64_PEAK_TFLOPS = 1.25  # GB300 nominal dense FP64 rate (no measured FP64 peak is available)
# nominal issue rates from the unit counts and the maximum SM clock (152 SMs, 2.07 GHz):
# 128 FP32 lanes per SM, and the FP64 rate above as 2 DFMA per SM and clock
FP32_INST_PER_S = 152 * 128 * 2.07e9
FP64_DFMA_PER_S = FP64_PEAK_TFLOPS * 1e12 / 2.0
# FP64 instructions of one Green's tensor evaluation in FP64 (green.cuh, with the
# column weights), counted from the source: every FP64 add, multiply and fused
# multiply-add once, products and sums fused wherever the source allows, and the
# square root, the divisions and each sine/cosine call once (they expand to more
# instructions), so a lower bound.  U: distance and direction 13, the two
# Helmholtz derivative sets 58, F 8, psi and chi 11, the nine entries 24, the
# weights 18; T: the same up to psi and chi, then the derivatives of psi and chi,
# the three coefficients and the nine entries 126, the weights 18.
GREEN_FP64_INST = {"U": 132, "T": 234}
# FP64 instructions of the ACA per Green's tensor evaluation besides the tensor:
# the residual's nine double-float sums subtracted part by part (4 adds per
# complex entry) and the double-float copies of the new factor entries of that
# point (9 per point and rank-3 step, one subtraction per real part)
ACA_FP64_PER_EVAL = 9 * 4 + 9 * 2


def dense_rows(hm, kernel, mat, pts_t, nrm_t, w_t, pidx, X):
    """Rows 3 i + a (i in pidx) of A X for the exact matrix A (block (i, j) =
    K(x_i, x_j) w_j, i != j, FP64 Green's tensors of the library's
    hm_green_eval; block (i, i) = I3), X (3 n_c, nrhs) complex128 on the GPU.
    Returns (rows, A[rows] X)."""
    import torch
    rho, lam, mu, om = mat
    n = pts_t.shape[0]
    Xp = X.reshape(n, 3, -1)
    out = []
    k = hm.HM_KERNEL_U if kernel == "U" else hm.HM_KERNEL_T
    for i in pidx:
        xi = pts_t[i].expand(n, 3).contiguous()
        G = hm.hm_green_eval(k, rho, lam, mu, om, xi, pts_t, nrm_t)  # (n, 3, 3), I3 at j = i
        wj = w_t.clone()
        wj[i] = 1.0
        out.append(torch.einsum("jab,jbs->as", G * wj[:, None, None], Xp))
    rows = np.array([3 * i + a for i in pidx for a in range(3)])
    return rows, torch.cat(out, 0)


def product_relerr(y, rows, yd):
    """||y[rows] - yd|| / ||yd|| (per column for a block of right-hand sides)."""
    d = (y[rows] - yd).reshape(len(rows), -1)
    ref = yd.reshape(len(rows), -1)
    return (d.norm(dim=0) / ref.norm(dim=0)).cpu().numpy()


def run_gpu(args, wl, world, rank, local):
    import torch
    from paper_1706_09384_gb300 import hm, inputs
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    st = torch.cuda.current_stream()
    pts = inputs.fibonacci_sphere(wl["nc"])
    rho, lam, mu, om = inputs.material(wl["ks"])
    # quadrature weights W_y (Sec. 4): area per point of the unit sphere
    weights = np.full(wl["nc"], 4 * math.pi / wl["nc"])
    form = args.form
    # the mixed form is the learned-batched one: the trained rank predictor sizes
    # each block's ACA workspace and bins blocks of similar predicted rank
    from paper_1706_09384_gb300 import rank_model
    model = rank_model.load() if form == "mixed" else None
    # the autotuner's cache (launch parameters of the product per GPU and workload
    # class): the first build sweeps the candidates, later builds read the cache
    tune_cache = os.path.join(ROOT, "paper_1706_09384_gb300", "_build", "tune_cache.txt")
    os.makedirs(os.path.dirname(tune_cache), exist_ok=True)
    opts = hm.hm_opts_default(weights=weights, rank_model=model, tune_cache=tune_cache,
                              storage=hm.HM_STORE_BF16 if form == "mixed" else hm.HM_STORE_FP32)
    x = torch.from_numpy(inputs.random_rhs(3 * wl["nc"], seed=rank)).to(dev)
    y = torch.empty_like(x)

    def build():
        return hm.HMatrix.build(pts, None, rho, lam, mu, om, wl["kernel"], wl["eps"], wl["eta"],
                                wl["leaf"], opts=opts)

    H = None
    tune_first = None
    for _ in range(args.warmup):
        if H is not None:
            H.free()
        H = build()
        tune_first = tune_first or H.stats()["tune"]
        for _ in range(args.matvecs):
            H.matvec(x, y)
        H.gmres(x, restart=100, tol=1e-6, maxit=2000, check=False)
    if H is None:
        H = build()
    torch.cuda.synchronize()
    stats = H.stats()
    alg = stats["matvec_alg_bytes"]
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    build_ms, mv_ms, gm_ms, gm_it, gm_rr, aca_ms, rec_ms, aca_fl = [], [], [], [], [], [], [], []
    aca_fl64, aca_fldf, aca_ev = [], [], []
    gm_prod = []
    launches0 = hm.hm_kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t_start = ev()
        t_start.record(st)
        for _ in range(args.steps):
            H.free()
            b0, b1 = ev(), ev()
            b0.record(st)
            H = build()
            b1.record(st)
            m0, m1 = ev(), ev()
            m0.record(st)
            for _ in range(args.matvecs):
                H.matvec(x, y)
            m1.record(st)
            g0, g1 = ev(), ev()
            g0.record(st)
            _, it, rr, gst = H.gmres(x, restart=100, tol=1e-6, maxit=2000, check=False)
            g1.record(st)
            torch.cuda.synchronize()
            build_ms.append(b0.elapsed_time(b1))
            mv_ms.append(m0.elapsed_time(m1))
            gm_ms.append(g0.elapsed_time(g1))
            gm_it.append(it)
            gm_rr.append(rr)
            sd = H.stats()
            aca_ms.append(sd["device_ms"]["aca"])
            rec_ms.append(sd["device_ms"]["recompress"])
            aca_fl.append(sd["aca_flops"])
            aca_fl64.append(sd["aca_flops_fp64"])
            aca_fldf.append(sd["aca_flops_df"])
            aca_ev.append(sd["aca_green_evals"])
            gm_prod.append(sd["gmres_last"])
        t_end = ev()
        t_end.record(st)
        torch.cuda.synchronize()
    barrier(world)
    total_ms = max_over_ranks(world, t_start.elapsed_time(t_end))
    mv_total = max_over_ranks(world, sum(mv_ms))
    launches = hm.hm_kernel_launches() - launches0
    value = whole_job_value(world, alg, args.matvecs * args.steps, mv_total)
    # accuracy of the timed product: sampled rows of the exact operator (FP64
    # Green's tensors of the library's hm_green_eval), 64 points = 192 rows
    pts_t = torch.from_numpy(pts).to(dev)
    w_t = torch.from_numpy(weights).to(dev)
    mat = (rho, lam, mu, om)
    pidx = np.sort(np.random.default_rng(7).choice(wl["nc"], 64, replace=False))
    H.matvec(x, y)
    rows, yd = dense_rows(hm, wl["kernel"], mat, pts_t, None, w_t, pidx, x.reshape(-1, 1))
    relerr = float(product_relerr(y.reshape(-1, 1), rows, yd)[0])
    # per-kernel roofline of the product (phase 2), events on the launching stream
    prof = H.profile_matvec(reps=10)
    peak, peak_kind = measured_peaks()
    ph2 = prof["bytes"]["phase2"] / (prof["ms"]["phase2"] * 1e-3) / 1e9
    kname = "mv16s_kernel<2>" if form == "mixed" else "mv_phase2"
    roof_mv = {"bound": "hbm", "kernel": kname, "achieved": ph2, "peak": peak,
               "peak_kind": peak_kind, "unit": "GB/s", "frac": ph2 / peak,
               "traffic": kernel_traffic("matvec.cu", kname, prof["bytes"]["phase2"]),
               "alg_bytes_per_launch": prof["bytes"]["phase2"],
               "ms_per_launch": prof["ms"]["phase2"], "kernels_ms": prof["ms"]}
    # the product for a block of 32 right-hand sides on the tensor cores (mixed form)
    block = None
    if form == "mixed":
        pm = H.profile_matvec_multi(reps=10)
        tb = sum(pm["ms"].values())
        tk = pm["ms"]["phase1"] + pm["ms"]["phase2"]
        block = {"nrhs": hm.HM_NRHS_BLOCK, "kernels": "mvc_phase1 / mvc_phase2 (persistent; TMA "
                 "128-byte-swizzled tiles, tcgen05.mma kind::f16 BF16 x BF16, FP32 accumulators in "
                 "TMEM)", "ms": pm["ms"], "alg_bytes": pm["bytes"],
                 "achieved_GBps": pm["bytes"] / (tk * 1e-3) / 1e9,
                 "frac": pm["bytes"] / (tk * 1e-3) / 1e9 / peak, "peak": peak,
                 "per_rhs_ms": tb / hm.HM_NRHS_BLOCK,
                 "speedup_vs_one_vector_products": statistics.mean(mv_ms) / args.matvecs
                 * hm.HM_NRHS_BLOCK / tb}
    # the dominant kernel of a step: the FP64 vector ACA of the build
    aca_t = statistics.mean(aca_ms)
    per_step = {"aca_kernel": aca_t, "recompression": statistics.mean(rec_ms),
                "h_matvec": statistics.mean(mv_ms), "gmres": statistics.mean(gm_ms)}
    # ALU roofline of the ACA.  Its arithmetic runs on two pipes that work side
    # by side: the FP32 pipes take the double-float multiply-adds (residuals,
    # norm-update cross terms, Gram blocks: 48 FP32 instructions per complex
    # multiply-add), the FP64 pipe the Green's tensors, the residual's rounding,
    # the double-float copies and the factor columns (4 DFMA per complex
    # multiply-add).  Each pipe's minimum time at its nominal rate; the kernel
    # can be no faster than the busier pipe, so t_min = max of the two and
    # frac = t_min / the measured time (each pipe's own fraction beside it).
    f64 = statistics.mean(aca_fl64)
    fdf = statistics.mean(aca_fldf)
    evals = statistics.mean(aca_ev)
    fp64_inst = evals * (GREEN_FP64_INST[wl["kernel"]] + ACA_FP64_PER_EVAL) + f64 / 8.0 * 4.0
    t32 = (fdf / 8.0 * 48.0) / FP32_INST_PER_S
    t64 = fp64_inst / FP64_DFMA_PER_S
    t_min = max(t32, t64)
    t_aca = aca_t * 1e-3
    prof_aca = kernel_profile("aca.cu", "aca_kernel")
    roofline = {"bound": "alu", "kernel": "aca_kernel", "achieved": (f64 + fdf) / t_aca / 1e12,
                "peak": (f64 + fdf) / t_min / 1e12, "peak_kind": "derived: nominal unit counts "
                "and clock (152 SMs x 128 FP32 lanes, 2 DFMA per SM and clock, 2.07 GHz); "
                "the busier pipe's minimum time",
                "unit": "TFLOP/s", "frac": t_min / t_aca,
                "pipes": {"fp32": {"t_min_ms": 1e3 * t32, "frac": t32 / t_aca,
                                   "work": "double-float multiply-adds, 48 FP32 instructions each"},
                          "fp64": {"t_min_ms": 1e3 * t64, "frac": t64 / t_aca,
                                   "instructions": fp64_inst, "green_evals": evals,
                                   "per_eval": GREEN_FP64_INST[wl["kernel"]] + ACA_FP64_PER_EVAL}},
                "traffic": (prof_aca["bytes_per_model_flop"] * (f64 + fdf)) if prof_aca else None,
                "alg_fp64_flops_per_launch": f64, "double_float_flops_per_launch": fdf,
                "ms_per_step": aca_t, "t_min_ms": 1e3 * t_min, "profile": prof_aca,
                "note": "ACA device time per build; model per rank-3 step: double-float 9k(m+n) "
                        "residuals + 9k(m+n) cross terms + 27(m+n) Gram blocks (FP32 pipes), "
                        "m+n FP64 Green's tensors with the residual rounding and the factor "
                        "copies, FP64 27m factor columns (FP64 pipe); the flops count 8 per "
                        "complex multiply-add; traffic = the ncu DRAM bytes per model flop of "
                        "the committed 16384-point capture times this launch's model flops"}
    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    xh = torch.empty(3 * wl["nc"], dtype=torch.complex128).pin_memory()
    xh.copy_(x.cpu())
    yh = torch.empty_like(xh).pin_memory()
    lib = hm.lib()
    sp = hm._stream_ptr(None)
    for _ in range(2):
        lib.hm_matvec_host(H.h, 1, xh.data_ptr(), yh.data_ptr(), sp)
    torch.cuda.synchronize()
    reps = max(5, args.matvecs)
    t0 = time.perf_counter()
    for _ in range(reps):
        lib.hm_matvec_host(H.h, 1, xh.data_ptr(), yh.data_ptr(), sp)
    e2e_s = (time.perf_counter() - t0) / reps
    nb = 16 * 3 * wl["nc"]
    out = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16c" if form == "mixed" else "c64", "data": "synthetic",
        "config": workload_config(args, wl, form, world),
        "streamed_gb_per_product": alg / 1e9,
        "product_relerr_vs_dense_rows": {
            "value": relerr, "rows": int(len(rows)), "eps": wl["eps"], "three_eps": 3 * wl["eps"],
            "note": ("relative error of the timed product on 192 sampled rows of the exact FP64 "
                     "operator; BF16 storage rounds every entry (unit roundoff 2^-8), so the mixed "
                     "product's error is of that order; the 3 eps of the metric holds for the "
                     "plain form's product and for the refined GMRES solutions of both forms")},
        "pct_hbm_peak": 100.0 * value / peak,
        "build_s": statistics.mean(build_ms) / 1e3,
        "matvec_ms": statistics.mean(mv_ms) / args.matvecs,
        "gmres": {"iters": gm_it[-1], "relres": gm_rr[-1], "ms": statistics.mean(gm_ms),
                  "products": gm_prod[-1]},
        "step_device_ms": per_step,
        "hmatrix": {k: stats[k] for k in ("blocks", "dense_blocks", "lowrank_blocks", "C_sp",
                                          "rank_aca_max", "rank_max", "tau_H", "stored_bytes",
                                          "matvec_alg_bytes")},
        "build_ms_phases": stats["ms"],
        "tune": {"first_build": tune_first, "timed_builds": stats["tune"]["source"],
                 "nstage": stats["tune"]["nstage"], "item_bytes": stats["tune"]["item_bytes"]},
        "roofline": roofline,
        "roofline_matvec": roof_mv,
        "e2e": {"value": alg / e2e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": nb,
                "d2h_bytes_per_step": nb, "api": "hm_matvec_host (pinned host buffers)"},
        "gpu_launches": launches,
        "clocks": clocks.summary(),
    }
    if block:
        out["block_product_32rhs"] = block
    if form == "mixed" and not args.no_compare:
        # the plain form on the same workload, once, outside the timed steps
        H.free()
        H = None
        popts = hm.hm_opts_default(weights=weights, tune_cache=tune_cache)
        b0, b1 = ev(), ev()
        b0.record(st)
        Hp = hm.HMatrix.build(pts, None, rho, lam, mu, om, wl["kernel"], wl["eps"], wl["eta"],
                              wl["leaf"], opts=popts)
        b1.record(st)
        for _ in range(3):
            Hp.matvec(x, y)
        m0, m1 = ev(), ev()
        m0.record(st)
        for _ in range(args.matvecs):
            Hp.matvec(x, y)
        m1.record(st)
        g0, g1 = ev(), ev()
        g0.record(st)
        _, pit, prr, _ = Hp.gmres(x, restart=100, tol=1e-6, maxit=2000, check=False)
        g1.record(st)
        torch.cuda.synchronize()
        palg = Hp.stats()["matvec_alg_bytes"]
        pmv = m0.elapsed_time(m1) / args.matvecs
        Hp.matvec(x, y)
        prel = float(product_relerr(y.reshape(-1, 1), rows, yd)[0])
        pgm = Hp.stats()["gmres_last"]
        out["plain"] = {"value": palg / (pmv * 1e-3) / 1e9, "unit": "GB/s",
                        "pct_hbm_peak": 100.0 * palg / (pmv * 1e-3) / 1e9 / peak,
                        "matvec_ms": pmv, "build_s": b0.elapsed_time(b1) / 1e3,
                        "gmres": {"iters": pit, "relres": prr, "ms": g0.elapsed_time(g1),
                                  "products": pgm},
                        "product_relerr_vs_dense_rows": prel,
                        "tune": Hp.stats()["tune"],
                        "stored_bytes": Hp.stats()["stored_bytes"]}
        out["mixed_vs_plain"] = {"matvec_speedup": pmv / out["matvec_ms"],
                                 "gmres_speedup_at_1e-6": g0.elapsed_time(g1) / out["gmres"]["ms"]}
        Hp.free()
    if H is not None:
        H.free()
        H = None
    if not args.no_extra and args.workload == "sphere65536_ks16_U":
        out["fp32_far_green"] = fp32_switch_build(hm, torch, pts, weights, mat, wl, opts_kw={
            "weights": weights, "rank_model": model,
            "storage": hm.HM_STORE_BF16 if form == "mixed" else hm.HM_STORE_FP32})
        out["mixed_vs_plain_T"] = mixed_vs_plain_T(hm, torch, pts, weights, mat, wl, model, tune_cache, x)
        out["multi_rhs_131072_T"] = multi_rhs_workload(hm, torch, dev, peak)
        out["batch_16_problems"] = batch_workload(hm, torch, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl)
    if rank == 0:
        print(json.dumps(out), flush=True)


def mixed_vs_plain_T(hm, torch, pts, weights, mat, wl, model, tune_cache, x):
    """Mixed against plain form at equal GMRES residual 1e-6 on the same sphere
    with the traction kernel T (normals of the sphere), where GMRES needs tens of
    iterations: the fast products dominate the solve, the refinement's accurate
    products are diluted."""
    from paper_1706_09384_gb300 import inputs
    rho, lam, mu, om = mat
    nrm = inputs.sphere_normals(pts)
    res = {"kernel": "T", "n_c": wl["nc"], "kappa_s": wl["ks"], "eps": wl["eps"]}
    st = torch.cuda.current_stream()
    y = torch.empty_like(x)
    for name, opts in (("mixed", hm.hm_opts_default(weights=weights, rank_model=model, tune_cache=tune_cache,
                                                    storage=hm.HM_STORE_BF16)),
                       ("plain", hm.hm_opts_default(weights=weights, tune_cache=tune_cache))):
        H = hm.HMatrix.build(pts, nrm, rho, lam, mu, om, "T", wl["eps"], wl["eta"], wl["leaf"], opts=opts)
        for _ in range(3):
            H.matvec(x, y)
        H.gmres(x, restart=100, tol=1e-6, maxit=2000, check=False)  # warm-up solve
        m0, m1, g0, g1 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
        m0.record(st)
        for _ in range(10):
            H.matvec(x, y)
        m1.record(st)
        g0.record(st)
        _, it, rr, _ = H.gmres(x, restart=100, tol=1e-6, maxit=2000, check=False)
        g1.record(st)
        torch.cuda.synchronize()
        res[name] = {"matvec_ms": m0.elapsed_time(m1) / 10, "gmres": {"iters": it, "relres": rr,
                     "ms": g0.elapsed_time(g1), "products": H.stats()["gmres_last"]}}
        H.free()
    res["matvec_speedup"] = res["plain"]["matvec_ms"] / res["mixed"]["matvec_ms"]
    res["gmres_speedup_at_1e-6"] = res["plain"]["gmres"]["ms"] / res["mixed"]["gmres"]["ms"]
    return res


def fp32_switch_build(hm, torch, pts, weights, mat, wl, opts_kw):
    """The same build with Green's tensors in FP32 where k_s r >= 1
    (hm_opts.fp64_switch_ksr): build seconds and ACA ranks against the FP64 build."""
    rho, lam, mu, om = mat
    res = {}
    for name, sw in (("fp64", float("inf")), ("fp32_beyond_ksr_1", 1.0)):
        o = hm.hm_opts_default(fp64_switch_ksr=sw, **opts_kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H = hm.HMatrix.build(pts, None, rho, lam, mu, om, wl["kernel"], wl["eps"], wl["eta"],
                             wl["leaf"], opts=o)
        torch.cuda.synchronize()
        st = H.stats()
        res[name] = {"build_s": time.perf_counter() - t0, "aca_device_ms": st["device_ms"]["aca"],
                     "near_field_ms": st["ms"]["near_field"], "rank_aca_mean": st["rank_aca_mean"],
                     "rank_mean": st["rank_mean"]}
        H.free()
    return res


def multi_rhs_workload(hm, torch, dev, peak):
    """131 072 Fibonacci points, k_s = 16, T kernel with outward normals, 32
    plane-wave right-hand sides (P and S waves), BF16 storage with per-block
    scales, the tensor-core block product inside lockstep GMRES(100) with
    refinement to 1e-6; per right-hand side: the residual of the exact FP64
    operator on 96 sampled rows, and the block product's error on those rows."""
    from paper_1706_09384_gb300 import inputs
    nc, ks, eps = 131072, 16.0, 1e-4
    pts = inputs.fibonacci_sphere(nc)
    nrm = inputs.sphere_normals(pts)
    rho, lam, mu, om = inputs.material(ks)
    w = np.full(nc, 4 * math.pi / nc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    H = hm.HMatrix.build(pts, nrm, rho, lam, mu, om, "T", eps, 3.0, 64,
                         opts=hm.hm_opts_default(weights=w, storage=hm.HM_STORE_BF16))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    B = torch.from_numpy(np.ascontiguousarray(inputs.plane_wave_rhs(pts, ks / 2, ks, 32, seed=0))
                         ).to(dev)
    t0 = time.perf_counter()
    X, it, rr, st = H.gmres_multi(B, restart=100, tol=1e-6, maxit=2000, check=False)
    torch.cuda.synchronize()
    gm_s = time.perf_counter() - t0
    gm = H.stats()["gmres_last"]
    pm = H.profile_matvec_multi(reps=10)
    tk = pm["ms"]["phase1"] + pm["ms"]["phase2"]
    pts_t, nrm_t = torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev)
    w_t = torch.from_numpy(w).to(dev)
    pidx = np.sort(np.random.default_rng(3).choice(nc, 32, replace=False))
    rows, AX = dense_rows(hm, "T", (rho, lam, mu, om), pts_t, nrm_t, w_t, pidx, X)
    res_exact = ((B[rows] - AX).norm(dim=0) / B[rows].norm(dim=0)).cpu().numpy()
    Xr = torch.from_numpy(inputs.random_rhs(3 * nc, nrhs=32, seed=5)).to(dev)
    Y = H.matvec(Xr)
    rows, Yd = dense_rows(hm, "T", (rho, lam, mu, om), pts_t, nrm_t, w_t, pidx, Xr)
    perr = product_relerr(Y, rows, Yd)
    alg = H.stats()["stored_bytes"]
    H.free()
    return {"n_c": nc, "kappa_s": ks, "kernel": "T", "nrhs": 32, "eps": eps,
            "storage": "bf16 + per-block fp32 scales", "build_s": build_s,
            "stored_gb": alg / 1e9, "gmres_s": gm_s, "gmres_products": gm,
            "iters_max": int(np.max(it)), "relres_max": float(np.max(rr)), "status": int(st),
            "exact_operator_residual_rows": {"max": float(res_exact.max()),
                                             "median": float(np.median(res_exact)),
                                             "rows": int(len(rows))},
            "block_product": {"ms": pm["ms"], "alg_bytes": pm["bytes"],
                              "achieved_GBps": pm["bytes"] / (tk * 1e-3) / 1e9,
                              "frac": pm["bytes"] / (tk * 1e-3) / 1e9 / peak,
                              "relerr_vs_dense_rows_max": float(perr.max()),
                              "relerr_vs_dense_rows_median": float(np.median(perr))}}


def batch_workload(hm, torch, dev):
    """16 independent problems (n_c 4 096 - 131 072; sphere, cube and ellipsoid
    surfaces; k_s ~ U[2, 24]; U or T; weights area / n_c; eps = 1e-4, FP32
    storage), built by one batch build (shared ACA and recompression
    launches), joined into one block-diagonal operator (hm_batch_join) and
    solved by lockstep GMRES(100) to 1e-6, one per problem, one product of all
    problems per Arnoldi step (at most 500 steps): wall time of the build, the
    join and the solve, per-problem results; the same solves one problem at a
    time for comparison."""
    from paper_1706_09384_gb300 import inputs
    P = inputs.batch_problems(16, seed=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Hs = hm.HMatrix.build_batch([dict(p, eta=3.0, leaf_size=64) for p in P], eps=1e-4)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    J = hm.HMatrix.join(Hs)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    b = torch.from_numpy(np.concatenate([inputs.random_rhs(3 * len(p["points"]), seed=100 + q)
                                         for q, p in enumerate(P)])).to(dev)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    _, it, rr, st = J.gmres_batch(b, restart=100, tol=1e-6, maxit=500, check=False)
    torch.cuda.synchronize()
    t4 = time.perf_counter()
    steps = J.stats()["gmres_last"]
    J.free()
    per = [{"n_c": len(p["points"]), "shape": p["shape"], "kernel": p["kernel"],
            "kappa_s": round(p["ks"], 3), "iters": int(it[q]), "relres": float(rr[q])}
           for q, p in enumerate(P)]
    # one problem at a time (each GMRES on its own handle)
    off = 0
    torch.cuda.synchronize()
    t5 = time.perf_counter()
    for p, H in zip(P, Hs):
        n = 3 * len(p["points"])
        H.gmres(b[off:off + n], restart=100, tol=1e-6, maxit=500, check=False)
        off += n
    torch.cuda.synchronize()
    t6 = time.perf_counter()
    for H in Hs:
        H.free()
    return {"problems": 16, "points": int(sum(len(p["points"]) for p in P)),
            "build_s": t1 - t0, "join_s": t2 - t1, "solve_lockstep_s": t4 - t3,
            "lockstep_products": steps, "total_s": (t2 - t0) + (t4 - t3),
            "solve_one_by_one_s": t6 - t5,
            "converged": int(sum(r["relres"] <= 1e-6 for r in per)), "per_problem": per}


def run_hlu(nc):
    """The H-LU direct solver (Sec. 3.2) on the n_c-point sphere, U kernel at
    omega = 4, eps = eps_LU = 1e-4, leaf 32: host wall time of the
    factorisation (its recursion is driven from the host), of one solve, and
    the residual of that solve with the H-matrix product."""
    import torch
    from paper_1706_09384_gb300 import hm, inputs
    hm.lib()
    pts = inputs.fibonacci_sphere(nc)
    w = np.full(nc, 4 * np.pi / nc)
    H = hm.HMatrix.build(pts, None, 1.0, 2.0, 1.0, 4.0, "U", 1e-4, 3.0, 32,
                         opts=hm.hm_opts_default(weights=w))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    H.lu_factor(1e-4)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    b = torch.from_numpy(inputs.random_rhs(3 * nc, seed=1)).cuda()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    x = H.lu_solve(b)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    relres = (torch.linalg.vector_norm(b - H.matvec(x)) / torch.linalg.vector_norm(b)).item()
    sec, entries, launches = H.lu_info()
    st = H.stats()
    print(json.dumps({
        "metric": "H-LU factorisation time (Sec. 3.2)", "value": t1 - t0, "unit": "s",
        "higher_is_better": False, "n_gpus": 1, "dtype": "f64c", "data": "synthetic",
        "config": {"workload": "sphere%d_U_hlu" % nc, "n_c": nc, "kernel": "U", "omega": 4.0,
                   "leaf": 32, "eta": 3.0, "eps": 1e-4, "eps_lu": 1e-4},
        "solve_s": t3 - t2, "relres": relres, "gpu_launches": launches,
        "lu_entries": entries, "N_s": st["N_s"]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--matvecs", type=int, default=20)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="sphere65536_ks16_U", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--form", default="mixed", choices=["mixed", "plain"],
                    help="mixed: BF16 storage (per-chunk scale) for the products, FP32-stored "
                         "operator for the refinement residuals; plain: FP32 storage")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the untimed plain-form comparison run")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the untimed extra workloads (FP32 far-field build, 131 072-point "
                         "T with 32 plane waves, the 16-problem batch)")
    ap.add_argument("--hlu", type=int, default=0,
                    help="instead of the step: time the H-LU direct solver on this many points")
    args = ap.parse_args()
    if args.hlu:
        run_hlu(args.hlu)
        return
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        run_reference(args, wl, world, rank)
        return
    world, rank, local = dist_setup(args.gpus)
    run_gpu(args, wl, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
