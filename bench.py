"""Benchmark of the H^2 matrix-vector product on GB300 (one JSON line on stdout).

Workload (default): 2D exponential covariance exp(-r/0.1), n = 2^20 uniform
points in the unit square, leaf size m = 64, 4x4 Chebyshev bases (k = 16),
admissibility eta = 0.9, x ~ N(0,1), FP64 plain form, nv = 1. The matrix
(about 15 GB) is far larger than the 129 MB L2, so every timed product streams
it from HBM; no L2 flush is needed between steps.

A step is one y = A^H x through the C ABI (all phases: projection, upsweep,
coupling, downsweep, dense blocks + expansion). value = paper bytes streamed
per step (U, V, E, F, S, D; the paper's Sec. 4.6 bandwidth metric) times steps
on all ranks / max elapsed time over ranks.

--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import h2gen  # noqa: E402

METRIC = "H^2 matvec HBM GB/s & vectors/s at n=2^20 (FP64 vs mixed @ rel err ≤1e-4)"
WORKLOADS = {
    "2d_n1M": "2D exp(-r/0.1) covariance H^2 matvec, n=2^20 uniform points, m=64, k=16 (4x4 Chebyshev), eta=0.9, FP64",
    "2d_n4096": "2D exp(-r/0.1) covariance H^2 matvec, n=4096 uniform points, m=32, k=16, eta=0.9, FP64",
    "2d_n256k": "2D exp(-r/0.1) covariance H^2 matvec, n=2^18 uniform points, m=64, k=16, eta=0.9, FP64",
    "3d_n512k": "3D exp(-r/0.2) covariance H^2 matvec, n=2^19 uniform points in the unit cube, m=64, k=64 (4x4x4 Chebyshev), "
                "eta=0.9, FP64",
    "3d_n64k": "3D exp(-r/0.2) covariance H^2 matvec, n=2^16 uniform points in the unit cube, m=64, k=64 (4x4x4 Chebyshev), "
               "eta=0.9, FP64",
    "3d_n1M_kc": "3D exp(-r/0.2) covariance H^2 matvec, n=2^20 uniform points in the unit cube, m=64, k=64 (4x4x4 "
                 "Chebyshev), eta=0.9, int16 + per-block f32 scale (S none: evaluated from the kernel), f32 bases",
    "3d_n4M_gen": "3D Matern-3/2 (length 0.1) covariance H^2 matvec, n=2^22 uniform points in the unit cube, m=64, "
                  "k=64 (4x4x4 Chebyshev), eta=0.7, fp16 + per-block f32 scale (S none: evaluated from the kernel; "
                  "D generated and quantized on the device from the points)",
    "compress_2d": "algebraic compression (Sec. 5: orthogonalization, basis generation, truncation, projection) of the "
                   "2D exp(-r/0.1) covariance H^2 matrix, n=2^20 uniform points, m=64, k=64 (8x8 Chebyshev), eta=0.9, "
                   "FP64, relative threshold 1e-7",
    "build_2d": "construction on the GPU (Sec. 4.6: KD tree, boxes, Chebyshev nodes, dual traversal, FP64 U, E, S, D) "
                "of the 2D exp(-r/0.1) covariance H^2 matrix, n=2^20 uniform points, m=64, k=16, eta=0.9",
    "build_3d": "construction on the GPU (Sec. 4.6; structure, U and E) of the 3D Matern-3/2 (length 0.1) covariance "
                "H^2 matrix, n=2^22 uniform points in the unit cube, m=64, k=64, eta=0.7",
    "compress_2d_small": "algebraic compression (Sec. 5) of the 2D exp(-r/0.1) covariance H^2 matrix, n=2^16 uniform "
                         "points, m=64, k=64 (8x8 Chebyshev), eta=0.9, FP64, relative threshold 1e-7",
    "compress_3d": "algebraic compression (Sec. 5) of the 3D exp(-r/0.2) covariance H^2 matrix, n=2^18 uniform points "
                   "in the unit cube, m=64, k=64 (4x4x4 Chebyshev), eta=0.9, FP64, relative threshold 1e-3",
    "batch256": "256 independent 2D exp(-r/0.1) covariance H^2 matvecs, n log-uniform in [2^12, 2^17], m=32, k=16, "
                "eta=0.9, nv in {1, 4, 16}, fp16 storage + f32 arithmetic, one graph-captured batched product",
}


def replica_config(workload: str, rank: int) -> dict:
    """Weak scaling: every rank multiplies its own independent matrix of the same workload (seed per rank)."""
    workload = {"3d_n1M_kc": "3d_n1M", "3d_n4M_gen": "3d_n4M"}.get(workload, workload)
    if workload not in h2gen.CONFIGS:
        return {}
    cfg = dict(h2gen.CONFIGS[workload])
    cfg["seed"] = cfg["seed"] + 1000 * rank
    return cfg


def max_over_ranks(value: float, dist, device) -> float:
    """The slowest rank's time (the job's time); identity without a process group."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / seconds


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            import tempfile

            fd, self.path = tempfile.mkstemp(prefix="h2_clocks_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        rows = []
        with open(self.path) as f:
            for ln in f:
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows)}


# DRAM bytes (read + write) of one dense-stream launch over its algorithmic bytes, from full ncu captures
# of the 2D n=2^18 workload (FP64, and int16 codes with FP32 bases); the traffic grows with the leaf
# count, so the ratio carries over to the n=2^20 launch
TRAFFIC_RATIO = {("fp64", False): 3184266039 / 3178496000, ("int16", True): 794616064 / 788584800}
TRAFFIC_KERNEL = {("fp64", False): "k_dense_stream", ("int16", True): "k_dense_stream_m"}  # the kernel those counters belong to

# FP32 instructions per double-float product a * x (split entry times split vector entry): the exact
# product p, e (2), the two cross terms (2), TwoSum of the running sum (6), the small-part sum (2)
DF_FP32_OPS = 12
FP32_LANES_PER_SM = 128


def dense_kernel_bytes(info: dict, A, nv: int, storage: str = "fp64", bases_fp32: bool = False) -> int:
    """Algorithmic bytes of one launch of the dense phase's kernel. FP64 form (D blocks and the fused
    leaf expansion): D and U once, x read once, y written once (8 bytes), the leaf yhat read once.
    Precision form on the CUDA cores (D blocks only; the expansion runs in the downsweep): D codes
    and one 4-byte scale per block, x once (FP32), y written once (8 bytes). Tensor-core pass (D
    blocks with the fused expansion): D codes and U codes with their scales, x once, y once, yhat."""
    nDval = int(A.D_valoff[-1])
    if storage == "fp64":
        return 8 * (nDval + A.n * A.k) + 8 * A.n * nv * 2 + 8 * A.leaves * A.k * nv
    if dense_kernel_name(A, nv, storage, bases_fp32) == "k_dense_stream_m":
        return 2 * nDval + 4 * A.nD + 4 * A.n * nv + 8 * A.n * nv
    u_bytes = 4 if bases_fp32 else 2
    return (2 * nDval + u_bytes * A.n * A.k + 4 * (A.nD + A.leaves) + 4 * A.n * nv + 8 * A.n * nv
            + 4 * A.leaves * A.k * nv)


def sm_count(dev) -> int:
    import torch

    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def df_peak_products(dev) -> float:
    """Peak double-float products per second on the FP32 pipes: 128 FP32 lanes per SM x SMs x the
    measured maximum SM clock / 12 FP32 instructions per product."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    mhz = 2070.0
    if os.path.exists(p):
        with open(p) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    return FP32_LANES_PER_SM * sm_count(dev) * mhz * 1e6 / DF_FP32_OPS


FP64_FMA_PER_SM_CYCLE = 2   # GB300: 152 SMs x 2 FP64 FMA per cycle x 2.07 GHz x 2 = 1.26 TFLOP/s (nominal 1.25)


def fp64_peak_flops(dev) -> float:
    """FP64 FLOP/s: 2 FP64 FMA per SM per cycle x SMs x the measured maximum SM clock x 2 flops."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    mhz = 2070.0
    if os.path.exists(p):
        with open(p) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    return 2.0 * FP64_FMA_PER_SM_CYCLE * sm_count(dev) * mhz * 1e6


def compress_kernel_flops(A, K: int) -> dict:
    """FP64 flops each compression kernel computes, counted from what it does per unit:
    k_project (the orthogonalization's, with upper triangular T): two K x K x K products with one
    triangular factor per coupling block (2 K^2 (K + 1));
    k_basis_gen: per coupling block the Householder reduction of K stacked rows against the
    triangular factor (per column j, a dot product and an update of K rows for the K - j - 1
    later columns: 4 K sum_j (K - j - 1) = 2 K^2 (K - 1)), per node R_parent E^T (K^2 (K + 1))
    and the QR of that K x K product (4 K^3 / 3)."""
    nodes = (2 << A.q) - 1
    return {"k_project": 2 * K * K * (K + 1) * A.nS,
            "k_basis_gen": 2 * K * K * (K - 1) * A.nS + (nodes - 1) * (K * K * (K + 1) + 4 * K ** 3 // 3)}


COMPRESS = {
    "compress_2d": dict(cfg=dict(dim=2, n=1 << 20, m=64, p=8, eta=0.9, kernel="exp", ell=0.1, seed=2), eps=1e-7,
                        oracle_n=1 << 14),
    "compress_3d": dict(cfg=dict(dim=3, n=1 << 18, m=64, p=4, eta=0.9, kernel="exp", ell=0.2, seed=3), eps=1e-3,
                        oracle_n=1 << 13),
    # the small line of the default run: the 2D problem at n = 2^16
    "compress_2d_small": dict(cfg=dict(dim=2, n=1 << 16, m=64, p=8, eta=0.9, kernel="exp", ell=0.1, seed=2),
                              eps=1e-7, oracle_n=1 << 13),
}


def compress_line(h2, dev, name: str, steps: int, warmup: int, cpu: bool = True) -> dict:
    """Time h2_compress_run on one of COMPRESS's workloads (inputs resident on the device, CUDA
    events on the stream), then: level ranks, memory of the low-rank part before and after, the
    FP64 product before and after, the errors of the paper's compression tables (Sec. 5.6) on
    sampled rows, the dominant kernel's roofline against the FP64 peak, and the compression
    oracle on a smaller matrix of the same family (host cores)."""
    import torch

    spec = COMPRESS[name]
    cfg, eps = spec["cfg"], spec["eps"]
    t0 = time.perf_counter()
    A = h2gen.generate(**cfg)
    gen_s = time.perf_counter() - t0
    cp = h2.Compressor.from_generator(A)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(1, warmup)):
        cp.run(eps, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            cp.run(eps, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    cp.profile(True)
    cp.run(eps, stream=stream)
    phases, launches = cp.profile_read()
    cp.profile(False)
    K, ru, rv = cp.result()
    inf = cp.info()
    U2, E2, S2 = cp.read("U"), cp.read("E"), cp.read("S")
    cp.close()
    nodes = (2 << A.q) - 1

    def lr_bytes(k):
        return 8 * (A.n * k + (nodes - 1) * k * k + A.nS * k * k)

    # the FP64 product before and after compression (1 vector x ~ U[0, 1], as the paper's tables)
    M1 = h2.H2Matrix.from_generator(A)
    M2 = h2.H2Matrix(n=A.n, depth=A.q, rank=K, leaf_offset=A.leaf_offset, U=U2, E=E2, S_rowptr=A.S_rowptr,
                     S_colidx=A.S_colidx, S_val=S2, D_rowptr=A.D_rowptr, D_colidx=A.D_colidx, D_val=A.D_val)
    x_np = h2gen.vectors(61, A.n, 1, dist="uniform")
    x = torch.from_numpy(np.ascontiguousarray(x_np.T)).to(dev).t()
    hmv = {}
    ys = {}
    for tag, M in (("before", M1), ("after", M2)):
        y = torch.empty((1, A.n), dtype=torch.float64, device=dev).t()
        for _ in range(3):
            M.matvec(x, y, stream=stream)
        reps = 20
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            M.matvec(x, y, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        hmv[tag] = round(e0.elapsed_time(e1) / reps, 4)
        ys[tag] = y[:, 0].cpu().numpy()
    M1.close()
    M2.close()
    rng = np.random.default_rng(11)
    rows = np.sort(rng.choice(A.n, size=min(A.n, 4096), replace=False))
    ax = A.exact_matvec_rows(rows, x_np)[:, 0]
    e_h1 = float(np.linalg.norm(ax - ys["before"][rows]) / np.linalg.norm(ax))
    e_h2 = float(np.linalg.norm(ax - ys["after"][rows]) / np.linalg.norm(ax))
    e_12 = float(np.linalg.norm(ys["after"] - ys["before"]) / np.linalg.norm(ys["before"]))
    flops = compress_kernel_flops(A, A.k)
    kern = {"k_project": phases["project"], "k_basis_gen": phases["basis_generation"]}
    top = max(kern, key=kern.get)
    peak = fp64_peak_flops(dev)
    ach = flops[top] / (kern[top] * 1e-3)
    out = {"workload": WORKLOADS.get(name, name), "n": A.n, "k": A.k, "q": A.q, "nS": A.nS, "eps": eps,
           "ms_per_compression": round(ms, 3), "points_per_s": round(A.n / (ms * 1e-3), 1),
           "phase_ms": {k: round(v, 3) for k, v in phases.items()}, "launches": launches,
           "ranks_per_level": ru, "uniform_rank": K, "jacobi_sweeps": {"max": inf["max_sweeps"],
                                                                     "mean": round(inf["total_sweeps"] / nodes, 2)},
           "lowrank_bytes_before": lr_bytes(A.k), "lowrank_bytes_after": lr_bytes(K),
           "hmv_ms_before": hmv["before"], "hmv_ms_after": hmv["after"],
           "rel_err_compressed_vs_original": e_12,
           "rel_err_vs_exact_before_sampled": e_h1, "rel_err_vs_exact_after_sampled": e_h2,
           "error_sample": f"{rows.size} random rows, x ~ U[0,1]",
           "roofline": {"kernel": top, "bound": "alu", "achieved": round(ach / 1e12, 4), "peak": round(peak / 1e12, 4),
                        "unit": "TFLOP/s (FP64)", "frac": round(ach / peak, 4),
                        "peak_derivation": f"{FP64_FMA_PER_SM_CYCLE} FP64 FMA per SM per cycle x {sm_count(dev)} SMs "
                                           "x max SM clock x 2",
                        "flops_per_launch_total": flops[top], "kernel_ms": round(kern[top], 3)},
           "device_bytes": inf["device_bytes"], "generate_s": round(gen_s, 1), "clocks": clk.summary()}
    if cpu:
        import oracle
        from oracle import compress as oc

        B = h2gen.generate(**dict(cfg, n=spec["oracle_n"]))
        t1 = time.perf_counter()
        oc.compress(B, eps)
        sec = time.perf_counter() - t1
        out["cpu_baseline"] = {"value": round(B.n / sec, 1), "unit": "points/s", "cores": oracle.threads(),
                               "kind": "oracle", "sample": f"the same family at n={B.n}, one compression "
                                                           f"({sec:.2f} s; numpy, plain loops over nodes and blocks)"}
    return out


COMPRESS_METRIC = "H^2 algebraic compression throughput (points/s) and time, Sec. 5"
BUILD = {"build_2d": ("2d_n1M", ("U", "E", "S", "D")), "build_3d": ("3d_n4M", ("U", "E"))}


def reference_build(args):
    """The construction oracle (oracle/construct.py, plain numpy) on a bounded sample of the workload's family:
    the structure (cluster tree, boxes, dual traversal) of 2^14 points."""
    import oracle
    from oracle import construct

    name, _ = BUILD[args.workload]
    cfg = dict(h2gen.CONFIGS[name])
    nb = 1 << 14
    pts = h2gen.uniform(cfg["seed"], (nb, cfg["dim"]))
    times = []
    for _ in range(max(1, min(args.steps, 3))):
        t = time.perf_counter()
        perm, lo, q = construct.cluster_tree(pts, cfg["m"])
        bmin, bmax = construct.node_boxes(pts[perm], lo, q)
        construct.dual_traversal(bmin, bmax, q, cfg["eta"])
        times.append(time.perf_counter() - t)
    sec = statistics.median(times)
    val = round(nb / sec, 1)
    print(json.dumps({"impl": "reference", "metric": "H^2 construction on the GPU (points/s), Sec. 4.6", "value": val,
                      "unit": "points/s", "n_gpus": 1, "steps": len(times), "warmup": 0,
                      "ms_per_step": round(sec * 1e3, 1), "higher_is_better": True, "scaling": "weak",
                      "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": WORKLOADS[args.workload], "sample_n": nb},
                      "cpu_baseline": {"value": val, "unit": "points/s", "cores": 1, "kind": "oracle",
                                       "sample": f"structure of {nb} points of the family ({len(times)} runs)"},
                      "e2e": {"value": val, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


def build_main(h2, args, dev, world, rank):
    """--workload build_2d / build_3d: the construction on the GPU (h2_build) as the main line, timed over
    a few builds (CUDA events inside the library), with the host generator's time as context."""
    import torch

    name, values = BUILD[args.workload]
    cfg = dict(h2gen.CONFIGS[name])
    t0 = time.perf_counter()
    A = h2gen.generate(**cfg, values=False)
    host_s = time.perf_counter() - t0
    pts = h2gen.uniform(A.seed, (A.n, A.dim))
    steps, warm = max(1, min(args.steps, 5)), max(1, min(args.warmup, 3))
    for _ in range(warm):
        h2.Built(pts, m=A.m, p=A.p, eta=A.eta, kernel=A.kernel, ell=A.ell, values=values).close()
    times = []
    with ClockSampler(dev.index) as clk:
        for _ in range(steps):
            B = h2.Built(pts, m=A.m, p=A.p, eta=A.eta, kernel=A.kernel, ell=A.ell, values=values)
            times.append(B.times())
            same = np.array_equal(B.read("S_colidx"), A.S_colidx) and np.array_equal(B.read("perm"), A.perm)
            B.close()
    ms = {k: statistics.median(t[k] for t in times) for k in times[0]}
    total = sum(ms.values())
    out = {"metric": "H^2 construction on the GPU (points/s), Sec. 4.6", "value": round(A.n / (total * 1e-3), 1),
           "unit": "points/s", "n_gpus": world, "steps": steps, "warmup": warm, "ms_per_step": round(total, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload], "n": A.n, "nS": A.nS, "nD": A.nD, "values": list(values),
                      "parallelism": "1 GPU"},
           "phase_ms": {k: round(v, 3) for k, v in ms.items()}, "structure_equals_generator": bool(same),
           "host_generator_structure_s": round(host_s, 2), "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(out), flush=True)


def reference_compress(args):
    """The compression oracle (numpy, FP64) on a bounded sample of the workload's family."""
    import oracle
    from oracle import compress as oc

    spec = COMPRESS[args.workload]
    B = h2gen.generate(**dict(spec["cfg"], n=spec["oracle_n"]))
    oc.compress(B, spec["eps"])   # warm
    times = []
    for _ in range(max(1, min(args.steps, 3))):
        t = time.perf_counter()
        oc.compress(B, spec["eps"])
        times.append(time.perf_counter() - t)
    sec = statistics.median(times)
    val = round(B.n / sec, 1)
    sample = f"the same family at n={B.n} (the workload has n={spec['cfg']['n']}), {len(times)} compressions"
    print(json.dumps({"impl": "reference", "metric": COMPRESS_METRIC, "value": val, "unit": "points/s",
                      "n_gpus": 1, "steps": len(times), "warmup": 1, "ms_per_step": round(sec * 1e3, 1),
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": {"workload": WORKLOADS[args.workload], "sample_n": B.n},
                      "cpu_baseline": {"value": val, "unit": "points/s", "cores": oracle.threads(), "kind": "oracle",
                                       "sample": sample},
                      "e2e": {"value": val, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


def compress_main(h2, args, dev, world, rank):
    """--workload compress_2d / compress_3d: the compression as the main line (points per second)."""
    steps, warm = max(1, min(args.steps, 5)), max(1, min(args.warmup, 3))
    c = compress_line(h2, dev, args.workload, steps, warm)
    out = {"metric": COMPRESS_METRIC, "value": c["points_per_s"],
           "unit": "points/s", "n_gpus": world, "steps": steps, "warmup": warm,
           "ms_per_step": c["ms_per_compression"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": c["workload"], "n": c["n"], "k": c["k"], "eps": c["eps"],
                      "l2": "coupling blocks (%.1f GB) >> 129 MB L2: no flush needed" % (c["lowrank_bytes_before"] / 1e9),
                      "parallelism": "1 GPU"},
           "gpu_launches": c["launches"] * steps, "roofline": c["roofline"],
           "clocks": c["clocks"], "compression": c}
    if "cpu_baseline" in c:
        out["cpu_baseline"] = c["cpu_baseline"]
    if rank == 0:
        print(json.dumps(out), flush=True)


def construction_line(h2, A, values=("U", "E", "S", "D")) -> dict:
    """Build the workload's matrix on the GPU (h2_build: KD tree, boxes, Chebyshev nodes, dual traversal,
    FP64 values) from the generator's points and compare its structure with the host generator's."""
    import oracle
    from oracle import construct

    pts = h2gen.uniform(A.seed, (A.n, A.dim))
    t0 = time.perf_counter()
    B = h2.Built(pts, m=A.m, p=A.p, eta=A.eta, kernel=A.kernel, ell=A.ell, values=values)
    wall = time.perf_counter() - t0
    t = B.times()
    same = (np.array_equal(B.read("perm"), A.perm) and np.array_equal(B.read("S_colidx"), A.S_colidx)
            and np.array_equal(B.read("S_rowptr"), A.S_rowptr) and np.array_equal(B.read("D_colidx"), A.D_colidx)
            and np.array_equal(B.read("D_rowptr"), A.D_rowptr))
    out = {"n": A.n, "dim": A.dim, "nS": B.nS, "nD": B.nD, "values": list(values),
           "gpu_ms": {k: round(v, 3) for k, v in t.items()}, "gpu_total_ms": round(sum(t.values()), 3),
           "call_s": round(wall, 3), "device_bytes": B.device_bytes, "structure_equals_generator": bool(same)}
    B.close()
    # the construction oracle (plain numpy, one thread of loops) on a bounded sample of the family
    nb = 1 << 12
    pts_s = h2gen.uniform(A.seed, (nb, A.dim))
    t1 = time.perf_counter()
    perm, lo, q = construct.cluster_tree(pts_s, A.m)
    bmin, bmax = construct.node_boxes(pts_s[perm], lo, q)
    construct.dual_traversal(bmin, bmax, q, A.eta)
    sec = time.perf_counter() - t1
    out["cpu_baseline"] = {"value": round(nb / sec, 1), "unit": "points/s (structure)", "cores": 1, "kind": "oracle",
                           "sample": f"oracle/construct.py structure at n={nb} ({sec:.2f} s)"}
    out["gpu_points_per_s_structure"] = round(A.n / ((t["tree_ms"] + t["blocks_ms"]) * 1e-3), 1)
    return out


def dense_kernel_name(A, nv: int, storage: str, bases_fp32: bool) -> str:
    """The kernel of the dense phase: the FP64 stream, or in the precision form the tensor-core
    kernel (16-bit fp16 / bf16 codes and bases, k a multiple of 16, every leaf 64 points, 8 or
    more vectors) or else the CUDA-core stream."""
    if storage == "fp64":
        return "k_dense_stream"
    panel = (storage in ("fp16", "bf16") and not bases_fp32 and A.k % 16 == 0 and A.k <= 64
             and bool(np.all(np.diff(np.asarray(A.leaf_offset)) == 64)))
    return "k_dense_tc" if panel and nv >= 8 else "k_dense_stream_m"


def run_oracle_baseline(A, x, budget_s: float = 12.0):
    """Time the FP64 oracle (as it stands) on the host cores over about budget_s seconds."""
    import oracle

    oracle.matvec(A, x)  # warm
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.matvec(A, x)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= 200:
            break
    return el / reps, reps, oracle.threads()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="h2", choices=["h2", "reference"])
    ap.add_argument("--workload", default="2d_n1M", choices=sorted(WORKLOADS))
    ap.add_argument("--nv", type=int, default=1)
    ap.add_argument("--no-extras", action="store_true", help="skip the nv=16 line, e2e and the CPU baseline")
    ap.add_argument("--storage", default="fp64", choices=["fp64", "fp16", "bf16", "int16"],
                    help="storage form of the timed product (the extras always use fp64 and list the scaled forms)")
    ap.add_argument("--bases-fp32", action="store_true", help="scaled forms: keep U, V, E, F in FP32")
    ap.add_argument("--coupling", default="stored", choices=["stored", "kernel"],
                    help="scaled forms: coupling blocks stored, or evaluated from the kernel in every product")
    ap.add_argument("--no-batch", action="store_true", help="extras without the batched-workload line")
    ap.add_argument("--batch-count", type=int, default=256, help="--workload batch256: members of the batch (the "
                    "first ones of the 256-member workload; fewer for profiling)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    cfg = replica_config(args.workload, rank)
    hbm, peak_kind = peaks()

    if args.impl == "reference":
        if rank != 0:
            return
        return reference_arm(args, cfg, world)

    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank if world > 1 else 0)
    torch.cuda.set_device(dev)
    import paper_1902_01829_gb300 as h2

    if args.workload == "batch256":
        return batch_main(h2, args, dev, dist, world, rank, hbm, peak_kind)
    if args.workload in COMPRESS:
        return compress_main(h2, args, dev, world, rank)
    if args.workload in BUILD:
        return build_main(h2, args, dev, world, rank)
    if args.workload in LARGE:
        return large_main(h2, args, cfg, dev, dist, world, rank, LARGE[args.workload])
    A = h2gen.generate(**cfg)
    M = h2.H2Matrix.from_generator(A, storage=args.storage, bases_fp32=args.bases_fp32, coupling=args.coupling)
    info = M.info()
    nv = args.nv
    x_np = h2gen.vectors(77 + rank, A.n, nv)
    x = torch.from_numpy(np.ascontiguousarray(x_np.T)).to(dev).t()
    y = torch.empty((nv, A.n), dtype=torch.float64, device=dev).t()
    stream = torch.cuda.current_stream(dev)

    def step(nvv=None, xx=None, yy=None):
        M.matvec(x if xx is None else xx, y if yy is None else yy, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # correctness of this run's output (not timed): every row against the oracle
    import oracle

    y_ref = oracle.matvec(A, x_np)
    rel_err = oracle.rel_l2(y.cpu().numpy(), y_ref)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # The FP64 form runs its phases in order: per-phase events inside the timed region give the dense
    # kernel's duration live. A scaled form runs its dense phase beside the tree phases (events
    # between phases would serialize them), so it is timed plain and its phases are timed after.
    live_phases = args.storage == "fp64"
    M.profile(live_phases)
    M.profile_read()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        barrier()
    if live_phases:
        phase_ms, launches = M.profile_read()
        M.profile(False)
    else:
        M.profile(True)
        M.profile_read()
        for _ in range(args.steps):
            step()
        phase_ms, launches = M.profile_read()
        M.profile(False)
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    ms_step = ms / args.steps
    gbs = job_rate(info["paper_bytes"], world, ms_step * 1e-3) / 1e9
    vps = job_rate(nv, world, ms_step * 1e-3)

    # roofline of the dominant kernel (dense blocks + leaf expansion), timed live above
    dense_ms = phase_ms["dense_expand"] / args.steps
    dbytes = dense_kernel_bytes(info, A, nv, args.storage, args.bases_fp32)
    achieved = dbytes / (dense_ms * 1e-3) / 1e9
    kname = dense_kernel_name(A, nv, args.storage, args.bases_fp32)
    roofline = {"kernel": kname + " (dense blocks + leaf expansion)", "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "traffic": (round(TRAFFIC_RATIO[(args.storage, args.bases_fp32)] * dbytes)
                            if (args.storage, args.bases_fp32) in TRAFFIC_RATIO and nv == 1
                            and TRAFFIC_KERNEL[(args.storage, args.bases_fp32)] == kname else None),
                "duration_source": ("CUDA events between phases inside the timed region" if live_phases else
                                    "CUDA events between phases, separate run of the same steps"),
                "bytes_per_launch": dbytes,
                "phase_share": {k: round(v / max(sum(phase_ms.values()), 1e-9), 4) for k, v in phase_ms.items()}}

    out = {"metric": METRIC, "value": round(gbs, 1), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None,
           "dtype": ("f64 (stored) / double-float (computed)" if args.storage == "fp64" else
                     f"{args.storage} + per-block f32 scale (stored{', f32 bases' if args.bases_fp32 else ''}) / f32 (computed)"),
           "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload], "n": A.n, "nv": nv, "q": A.q, "k": A.k,
                      "coupling": args.coupling,
                      "nS": A.nS, "nD": A.nD, "paper_bytes": info["paper_bytes"],
                      "l2": "matrix (%.1f GB) >> 129 MB L2: no flush needed" % (info["paper_bytes"] / 1e9),
                      "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
           "vectors_per_s": round(vps, 2), "rel_err_vs_oracle": rel_err,
           "gpu_launches": int(launches), "roofline": roofline,
           "frac_of_nominal_8TBs": round(gbs / world / 8000.0, 4)}

    clocks = clk.summary()
    out["clocks"] = clocks

    if not args.no_extras:
        # end to end through the public C ABI with host buffers (pinned), copies inside the timed region
        xh = torch.empty((nv, A.n), dtype=torch.float64, pin_memory=True)
        xh.copy_(torch.from_numpy(np.ascontiguousarray(x_np.T)))
        yh = torch.empty((nv, A.n), dtype=torch.float64, pin_memory=True)
        xh_np, yh_np = xh.numpy().T, yh.numpy().T
        for _ in range(2):
            M.matvec_host(xh_np, yh_np, stream=stream)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            M.matvec_host(xh_np, yh_np, stream=stream)
        el = max_over_ranks(time.perf_counter() - t0, dist, dev)
        e2e_step = el / args.steps
        out["e2e"] = {"value": round(info["paper_bytes"] * world / e2e_step / 1e9, 1), "unit": "GB/s",
                      "ms_per_step": round(e2e_step * 1e3, 4), "vectors_per_s": round(nv * world / e2e_step, 2),
                      "h2d_bytes_per_step": 8 * A.n * nv, "d2h_bytes_per_step": 8 * A.n * nv,
                      "rel_err_vs_oracle": oracle.rel_l2(yh_np, y_ref)}

        # 16 right-hand sides per product (the workload's second vector count)
        x16_np = h2gen.vectors(177 + rank, A.n, 16)
        x16 = torch.from_numpy(np.ascontiguousarray(x16_np.T)).to(dev).t()
        y16 = torch.empty((16, A.n), dtype=torch.float64, device=dev).t()
        for _ in range(3):
            M.matvec(x16, y16, stream=stream)
        steps16 = max(3, args.steps // 4)
        barrier()
        e0.record(stream)
        for _ in range(steps16):
            M.matvec(x16, y16, stream=stream)
        e1.record(stream)
        barrier()
        ms16 = e0.elapsed_time(e1) / steps16
        out["nv16"] = {"ms_per_step": round(ms16, 4), "vectors_per_s": round(16 * world / (ms16 * 1e-3), 1),
                       "GBs": round(info["paper_bytes"] * world / (ms16 * 1e-3) / 1e9, 1),
                       "rel_err_vs_oracle": oracle.rel_l2(y16.cpu().numpy(), oracle.matvec(A, x16_np))}
        if args.storage == "fp64":
            # at 16 vectors the FP64 form's dense phase is bound by double-float arithmetic on the FP32
            # pipes, not by HBM: products per second of its kernel against that peak
            M.profile(True)
            M.profile_read()
            for _ in range(steps16):
                M.matvec(x16, y16, stream=stream)
            ph16, _ = M.profile_read()
            M.profile(False)
            d16_ms = ph16["dense_expand"] / steps16
            prods = 16 * (int(A.D_valoff[-1]) + A.n * A.k)
            peak = df_peak_products(dev)
            ach = prods / (d16_ms * 1e-3)
            hbm_frac = dense_kernel_bytes(info, A, 16) / (d16_ms * 1e-3) / 1e9 / hbm
            out["nv16"]["roofline"] = {
                "kernel": "k_dense_stream (dense blocks + leaf expansion, 16 vectors)", "bound": "alu",
                "achieved": round(ach / 1e12, 4), "peak": round(peak / 1e12, 4), "unit": "T double-float products/s",
                "frac": round(ach / peak, 4), "hbm_frac": round(hbm_frac, 4),
                "peak_derivation": f"{FP32_LANES_PER_SM} FP32 lanes x {sm_count(dev)} SMs x max SM clock / "
                                   f"{DF_FP32_OPS} FP32 instructions per product",
                "products_per_launch": prods, "kernel_ms": round(d16_ms, 4)}

        # precision form (per-block scaled 16-bit S and D; U, V, E, F in FP32 or 16-bit) at several vector counts
        out["mixed"] = mixed_lines(h2, A, info, dev, stream, y_ref, x_np, args.steps, world, rank)

        # the coupling blocks evaluated from the kernel at the interpolation points (none stored)
        out["kernel_coupling"] = kernel_coupling_lines(h2, A, dev, stream, y_ref, x_np, args.steps, world)

        # many independent matrices of uneven size in one batched, graph-captured product
        if not args.no_batch:
            out["batch"] = batch_line(h2, dev, args.steps, world, rank, hbm)

        # algebraic compression (Sec. 5) of the 2D 8x8-Chebyshev problem at n = 2^16
        out["compression"] = compress_line(h2, dev, "compress_2d_small", 3, 1, cpu=(rank == 0 and world == 1))

        # construction of this workload's matrix on the GPU (Sec. 4.6), FP64 values included
        out["construction"] = construction_line(h2, A)

        if rank == 0 and world == 1:
            sec, reps, cores = run_oracle_baseline(A, x_np)
            out["cpu_baseline"] = {"value": round(info["paper_bytes"] / sec / 1e9, 2), "unit": "GB/s",
                                   "cores": cores, "kind": "oracle",
                                   "sample": f"full workload, nv={nv}, {reps} products ({sec * 1e3:.1f} ms each)",
                                   "vectors_per_s": round(nv / sec, 2)}

    if rank == 0:
        print(json.dumps(out), flush=True)
    M.close()
    if dist is not None:
        dist.destroy_process_group()


# (storage, bases_fp32): int16 with FP32 bases meets 1e-4; fp16 / bf16 with 16-bit bases run the dense
# phase on the tensor cores for passes of 8 or more vectors (64-point leaves)
MIXED_FORMS = [("int16", True), ("fp16", True), ("fp16", False), ("bf16", False)]
MIXED_NV = [1, 8, 32, 64]
MIXED_F32_FORMS = [("int16", True), ("fp16", False)]   # also timed with FP32 vectors


def mixed_lines(h2, A, info64, dev, stream, y_ref, x_np, steps, world, rank):
    """Time the precision form on the same matrix: GB/s of its own stored bytes, vectors/s, error vs the FP64 oracle."""
    import oracle
    import torch

    xw_np = np.asfortranarray(np.concatenate([x_np, h2gen.vectors(911 + rank, A.n, max(MIXED_NV) - 1)], axis=1))
    ref2 = np.concatenate([y_ref, oracle.matvec(A, xw_np[:, 1:2])], axis=1)  # FP64 oracle, first two columns
    xw = torch.from_numpy(np.ascontiguousarray(xw_np.T)).to(dev).t()
    lines = []
    for form, bases in MIXED_FORMS:
        M = h2.H2Matrix.from_generator(A, storage=form, bases_fp32=bases)
        mb = M.info()["paper_bytes"]
        for nv in MIXED_NV:
            X = xw[:, :nv]
            Y = torch.empty((nv, A.n), dtype=torch.float64, device=dev).t()
            tuned = M.tune(X, Y, stream=stream)  # launch parameters chosen by timing (h2_tune)
            for _ in range(3):
                M.matvec(X, Y, stream=stream)
            M.check(stream)
            k = max(3, steps // (1 + nv // 8))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(k):
                M.matvec(X, Y, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / k
            yy = Y[:, :min(nv, 2)].cpu().numpy()
            err = oracle.rel_l2(yy, ref2[:, :yy.shape[1]])
            lines.append({"storage": form, "bases_fp32": bases, "nv": nv, "xy": "f64", "tuned": tuned,
                          "ms_per_step": round(ms, 4), "GBs": round(mb * world / (ms * 1e-3) / 1e9, 1),
                          "vectors_per_s": round(nv * world / (ms * 1e-3), 1),
                          "stored_bytes": mb, "rel_err_vs_fp64_oracle": err})
            if (form, bases) in MIXED_F32_FORMS and nv in (1, max(MIXED_NV)):
                # the same product with FP32 vectors (h2_matvec_f32): half the vector bytes
                X32 = X.float().t().contiguous().t()
                Y32 = torch.empty((nv, A.n), dtype=torch.float32, device=dev).t()
                for _ in range(3):
                    M.matvec_f32(X32, Y32, stream=stream)
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(k):
                    M.matvec_f32(X32, Y32, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ms32 = e0.elapsed_time(e1) / k
                yy = Y32[:, :min(nv, 2)].cpu().numpy().astype(np.float64)
                lines.append({"storage": form, "bases_fp32": bases, "nv": nv, "xy": "f32", "tuned": tuned,
                              "ms_per_step": round(ms32, 4), "GBs": round(mb * world / (ms32 * 1e-3) / 1e9, 1),
                              "vectors_per_s": round(nv * world / (ms32 * 1e-3), 1), "stored_bytes": mb,
                              "rel_err_vs_fp64_oracle": oracle.rel_l2(yy, ref2[:, :yy.shape[1]])})
        M.close()
    return lines


def kernel_coupling_lines(h2, A, dev, stream, y_ref, x_np, steps, world, form="int16", bases=True, nvs=(1, 16, 64)):
    """The precision form with its coupling blocks evaluated in every product from the kernel at the
    interpolation points (h2_create_kernel_coupling) next to the same form with the blocks stored:
    time per product, the coupling phase, stored bytes, error vs the FP64 oracle (first column)."""
    import oracle
    import torch

    xw = torch.from_numpy(np.ascontiguousarray(
        np.concatenate([x_np, h2gen.vectors(913, A.n, max(nvs) - 1)], axis=1).T)).to(dev).t()
    lines = []
    for coupling in ("kernel", "stored"):
        M = h2.H2Matrix.from_generator(A, storage=form, bases_fp32=bases, coupling=coupling)
        info = M.info()
        for nv in nvs:
            X = xw[:, :nv]
            Y = torch.empty((nv, A.n), dtype=torch.float64, device=dev).t()
            M.tune(X, Y, stream=stream)
            for _ in range(3):
                M.matvec(X, Y, stream=stream)
            M.check(stream)
            k = max(3, steps // (1 + nv // 8))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(k):
                M.matvec(X, Y, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / k
            M.profile(True)  # the coupling phase alone (profiled products keep the phases in order)
            M.profile_read()
            for _ in range(k):
                M.matvec(X, Y, stream=stream)
            phase, _ = M.profile_read()
            M.profile(False)
            lines.append({"coupling": coupling, "storage": form, "bases_fp32": bases, "nv": nv,
                          "ms_per_step": round(ms, 4), "coupling_ms": round(phase["coupling"] / k, 4),
                          "vectors_per_s": round(nv * world / (ms * 1e-3), 1), "stored_bytes": info["paper_bytes"],
                          "device_bytes": info["device_bytes"],
                          "rel_err_vs_fp64_oracle": oracle.rel_l2(Y[:, :1].cpu().numpy(), y_ref[:, :1])})
        M.close()
    return lines


def batch_line(h2, dev, steps, world, rank, hbm, count=256, storage="fp16", timed_barrier=None):
    """The batched workload: 256 independent 2D exp(-r/0.1) matrices, n log-uniform in [2^12, 2^17],
    m=32, k=16, nv_i drawn from {1, 4, 16}, fp16 storage with per-block scales, FP32 arithmetic.
    One product of every member = one graph replay (one launch per phase for the whole batch).
    Reported: stored bytes streamed per second, vectors/s, member products/s; the same products
    as a loop of one h2_matvec per member, for comparison; the error of sampled members."""
    import oracle
    import torch
    from oracle import quant

    t_build = time.perf_counter()
    spec = h2gen.batch_workload(count=count, seed=40 + rank)
    ns = [kw["n"] for kw, _ in spec]
    sample = sorted({int(np.argmin(ns)), int(np.argmax(ns))})
    Ms, xs, ys, keep = [], [], [], {}
    for i, (kw, nv) in enumerate(spec):
        A = h2gen.generate(**kw)
        Ms.append(h2.H2Matrix.from_generator(A, storage=storage))
        x = h2gen.vectors(3000 + i, A.n, nv)
        xs.append(torch.from_numpy(np.ascontiguousarray(x.T)).to(dev).t())
        ys.append(torch.empty((nv, A.n), dtype=torch.float64, device=dev).t())
        if i in sample:
            keep[i] = (A, x)
        else:
            A.free()
    B = h2.H2Batch(Ms)
    t_build = time.perf_counter() - t_build
    stored = sum(M.info()["paper_bytes"] for M in Ms)
    vecs = sum(nv for _, nv in spec)
    t_tune = time.perf_counter()
    tuned = B.tune(xs, ys)  # launch parameters chosen by timing (h2_batch_tune)
    t_tune = time.perf_counter() - t_tune
    args = B.prepare(xs, ys)
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        for _ in range(3):
            B.matvec_prepared(args, s)
    s.synchronize()
    B.check(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        B.matvec_prepared(args, s)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    k = max(5, steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cur = torch.cuda.current_stream(dev)
    if timed_barrier is not None:
        timed_barrier.barrier()
    torch.cuda.synchronize()
    e0.record(cur)
    for _ in range(k):
        g.replay()
    e1.record(cur)
    if timed_barrier is not None:
        timed_barrier.barrier()
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / k, timed_barrier, dev)
    B.check(s)
    # per-phase split (events between the phase launches; outside the timed graph replays)
    B.profile(True)
    B.profile_read()
    for _ in range(3):
        B.matvec_prepared(args, cur)
    phase_ms, _ = B.profile_read()
    B.profile(False)
    errs = {}
    for i, (A, x) in keep.items():
        y = ys[i].cpu().numpy()
        errs[str(A.n)] = {"vs_fp64_oracle": oracle.rel_l2(y, oracle.matvec(A, x)),
                          "vs_quantized_oracle": oracle.rel_l2(y, oracle.matvec(A, x, **quant.dequantized_arrays(A, storage)))}
    # the same products one handle at a time (no graph)
    loop_k = max(3, k // 4)
    for M, x, y in zip(Ms, xs, ys):
        M.matvec(x, y, stream=cur)
    torch.cuda.synchronize()
    e0.record(cur)
    for _ in range(loop_k):
        for M, x, y in zip(Ms, xs, ys):
            M.matvec(x, y, stream=cur)
    e1.record(cur)
    torch.cuda.synchronize()
    loop_ms = e0.elapsed_time(e1) / loop_k
    info = B.info()
    del g
    B.close()
    for M in Ms:
        M.close()
    gbs = stored * world / (ms * 1e-3) / 1e9
    return {"workload": f"{count} 2D exp(-r/0.1) matrices, n log-uniform in [2^12, 2^17] (sum {sum(ns)}), m=32, k=16, "
                        f"eta=0.9, nv in {{1, 4, 16}} (sum {vecs}), {storage} + per-block f32 scale, f32 arithmetic",
            "ms_per_step": round(ms, 4), "GBs": round(gbs, 1), "frac_of_hbm": round(gbs / world / hbm, 4),
            "vectors_per_s": round(vecs * world / (ms * 1e-3), 1),
            "matvecs_per_s": round(count * world / (ms * 1e-3), 1), "stored_bytes": stored,
            "l2": "batch (%.1f GB) >> 129 MB L2: no flush needed" % (stored / 1e9),
            "launches_per_step": info["launches_per_pass"], "tree_jobs": info["tree_jobs"],
            "dense_items": info["dense_items"], "graph": True, "tuned": tuned, "tune_s": round(t_tune, 2),
            "phase_ms": {key: round(v / 3, 4) for key, v in phase_ms.items()},
            "one_handle_at_a_time_ms": round(loop_ms, 4), "rel_err_sampled": errs,
            "build_s": round(t_build, 1)}


def batch_main(h2, args, dev, dist, world, rank, hbm, peak_kind):
    """--workload batch256: the batched product alone, as the main line."""
    import torch

    with ClockSampler(dev.index) as clk:
        b = batch_line(h2, dev, args.steps, world, rank, hbm, count=args.batch_count, timed_barrier=dist)
    out = {"metric": METRIC, "value": b["GBs"], "unit": "GB/s", "n_gpus": world, "steps": max(5, args.steps),
           "warmup": args.warmup, "ms_per_step": b["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "fp16 + per-block f32 scale (stored) / f32 (computed)", "data": "synthetic",
           "config": {"workload": WORKLOADS["batch256"], "l2": b["l2"],
                      "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
           "vectors_per_s": b["vectors_per_s"], "gpu_launches": b["launches_per_step"] * max(5, args.steps),
           "batch": b, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(out), flush=True)
    torch.cuda.synchronize()
    if dist is not None:
        dist.destroy_process_group()


# Workloads that one GPU holds only with the coupling blocks evaluated from the kernel in every product
# (and, for the largest, the dense blocks generated on the device): their FP64 values are never made.
LARGE = {
    "3d_n1M_kc": dict(storage="int16", bases_fp32=True, dense="stored", nvs=(1, 8, 32, 64), leaves=16,
                      dtype="int16 + per-block f32 scale (stored), f32 bases / f32 (computed)"),
    "3d_n4M_gen": dict(storage="fp16", bases_fp32=False, dense="generated", nvs=(1, 32), leaves=8,
                       dtype="fp16 + per-block f32 scale (stored) / f32 (computed)"),
}


def large_main(h2, args, cfg, dev, dist, world, rank, spec):
    """--workload 3d_n1M_kc: the 3D k = 64 workload at n = 2^20 (int16 codes + FP32 bases, nv in
    {1, 8, 32, 64}); --workload 3d_n4M_gen: the 3D Matern-3/2 workload at n = 2^22, eta = 0.7 (fp16
    codes, nv in {1, 32}), its dense blocks generated on the device. Both evaluate the coupling blocks
    from the kernel. The error is taken on sampled rows against the exact kernel matrix, as the paper
    measures its large problems (Sec. 4.6)."""
    import torch

    t0 = time.perf_counter()
    gen = spec["dense"] == "generated"
    A = h2gen.generate(**cfg, coupling_values=False, dense_values=not gen)
    t_host = time.perf_counter() - t0
    t0 = time.perf_counter()
    built = None
    if gen:
        # the whole matrix from the points on the GPU (h2_build), then a handle that evaluates the coupling
        # blocks and generates the dense blocks on the device (h2_create_built)
        built = h2.Built(h2gen.uniform(A.seed, (A.n, A.dim)), m=A.m, p=A.p, eta=A.eta, kernel=A.kernel, ell=A.ell,
                         values=("U", "E"))
        M = built.matrix(storage=spec["storage"], bases_fp32=spec["bases_fp32"], coupling="kernel", dense="generated")
    else:
        M = h2.H2Matrix.from_generator(A, storage=spec["storage"], bases_fp32=spec["bases_fp32"], coupling="kernel",
                                       dense=spec["dense"])
    build_s = time.perf_counter() - t0
    A.D_val = None  # the device holds the codes; free the host copy
    info = M.info()
    rng = np.random.default_rng(7 + rank)
    leaves = rng.choice(A.leaves, size=spec["leaves"], replace=False)
    rows = np.concatenate([np.arange(A.leaf_offset[i], A.leaf_offset[i + 1]) for i in sorted(leaves)])
    nv_max = max(spec["nvs"])
    x_np = h2gen.vectors(51 + rank, A.n, nv_max)
    xw = torch.from_numpy(np.ascontiguousarray(x_np.T)).to(dev).t()
    exact = A.exact_matvec_rows(rows, x_np[:, :1])
    from oracle import rows as oracle_rows  # the checks below run outside the timed regions

    ref64 = oracle_rows.sampled_rows(A, x_np[:, :1], sorted(leaves))
    lines = []
    with ClockSampler(dev.index) as clk:
        for nv in spec["nvs"]:
            X = xw[:, :nv]
            Y = torch.empty((nv, A.n), dtype=torch.float64, device=dev).t()
            tuned = M.tune(X, Y)
            for _ in range(3):
                M.matvec(X, Y)
            M.check()
            k = max(3, args.steps // (1 + nv // 4))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()
            e0.record()
            for _ in range(k):
                M.matvec(X, Y)
            e1.record()
            torch.cuda.synchronize()
            ms = max_over_ranks(e0.elapsed_time(e1) / k, dist, dev)
            M.profile(True)  # per-phase times from a separate run (profiled products keep the phases in order)
            M.profile_read()
            for _ in range(k):
                M.matvec(X, Y)
            phase, launches = M.profile_read()
            M.profile(False)
            yr = Y[:, 0].cpu().numpy()[rows]
            err = float(np.linalg.norm(yr - exact[:, 0]) / np.linalg.norm(exact[:, 0]))
            err64 = float(np.linalg.norm(yr - ref64[:, 0]) / np.linalg.norm(ref64[:, 0]))
            lines.append({"nv": nv, "tuned": tuned, "ms_per_step": round(ms, 4),
                          "GBs": round(info["paper_bytes"] * world / (ms * 1e-3) / 1e9, 1),
                          "vectors_per_s": round(nv * world / (ms * 1e-3), 1),
                          "phase_ms": {key: round(v / k, 4) for key, v in phase.items()},
                          "launches_per_step": int(launches) // k,
                          "rel_err_vs_fp64_oracle_sampled_rows": err64,
                          "rel_err_vs_exact_kernel_sampled_rows": err})
    head = lines[0]
    out = {"metric": METRIC, "value": head["GBs"], "unit": "GB/s", "n_gpus": world, "steps": args.steps,
           "warmup": 3, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": spec["dtype"], "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload], "n": A.n, "q": A.q, "k": A.k, "nS": A.nS, "nD": A.nD,
                      "paper_bytes": info["paper_bytes"], "device_bytes": info["device_bytes"],
                      "l2": "matrix (%.1f GB) >> 129 MB L2: no flush needed" % (info["paper_bytes"] / 1e9),
                      "error_sample": f"{rows.size} rows of {spec['leaves']} random leaves, first vector: against "
                                      "the FP64 H^2 oracle (the same matrix in FP64) and against the exact kernel "
                                      "matrix (adds the H^2 approximation error)",
                      "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
           "vectors_per_s": max(l["vectors_per_s"] for l in lines), "gpu_launches": head["launches_per_step"] * args.steps,
           "rel_err_vs_fp64_oracle": max(l["rel_err_vs_fp64_oracle_sampled_rows"] for l in lines),
           "lines": lines, "build_s": round(build_s, 1), "host_structure_s": round(t_host, 1), "clocks": clk.summary()}
    if built is not None:
        out["construction"] = {"gpu_ms": {k: round(v, 2) for k, v in built.times().items()},
                               "source": "h2_build (structure, U, E on the GPU) + h2_create_built",
                               "handle_s": round(build_s, 1), "host_generator_s": round(t_host, 1)}
        built.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    M.close()
    if dist is not None:
        dist.destroy_process_group()


def reference_arm(args, cfg, world):
    """The FP64 CPU oracle, timed as it stands on the host cores, same workload and metric."""
    import oracle

    if args.workload == "batch256":
        return reference_batch(args, world)
    if args.workload in COMPRESS:
        return reference_compress(args)
    if args.workload in BUILD:
        return reference_build(args)
    if args.workload in LARGE:
        print(json.dumps({"impl": "reference", "unavailable": "the FP64 oracle needs the stored coupling values "
                          "(126 GB at n=2^20, 960 GB at n=2^22) that this workload never makes (it evaluates them "
                          "from the kernel)"}), flush=True)
        return
    A = h2gen.generate(**dict(h2gen.CONFIGS[args.workload]))
    x = h2gen.vectors(77, A.n, args.nv)
    paper_bytes = 8 * (2 * A.n * A.k + 2 * (A.n_nodes - 1) * A.k * A.k + A.nS * A.k * A.k + int(A.D_valoff[-1]))
    for _ in range(max(1, min(args.warmup, 2))):
        oracle.matvec(A, x)
    steps = args.steps
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle.matvec(A, x)
    el = time.perf_counter() - t0
    sec = el / steps
    val = round(paper_bytes / sec / 1e9, 2)
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": world, "steps": steps,
           "warmup": args.warmup, "ms_per_step": round(sec * 1e3, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOADS[args.workload], "n": A.n, "nv": args.nv, "paper_bytes": paper_bytes},
           "vectors_per_s": round(args.nv / sec, 2),
           "cpu_baseline": {"value": val, "unit": "GB/s", "cores": oracle.threads(), "kind": "oracle",
                            "sample": f"full workload, nv={args.nv}, {steps} products"},
           "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def fp16_stored_bytes(A) -> int:
    """Bytes of a matrix in the scaled 16-bit form: 2 per entry of U, V, E, F, S, D plus a 4-byte scale per block."""
    kk = A.k * A.k
    entries = 2 * A.n * A.k + 2 * (A.n_nodes - 1) * kk + A.nS * kk + int(A.D_valoff[-1])
    blocks = 2 * A.leaves + 2 * (A.n_nodes - 1) + A.nS + A.nD
    return 2 * entries + 4 * blocks


def reference_batch(args, world):
    """The FP64 oracle on a bounded sample of the batched workload (the first members, in order, each
    with its own vector count), reported in the batched line's unit (stored 16-bit bytes per second)."""
    import oracle

    spec = h2gen.batch_workload()
    sample, total = [], 0
    for kw, nv in spec:  # about 1.5e6 points of work per step
        A = h2gen.generate(**kw)
        sample.append((A, h2gen.vectors(3000 + len(sample), A.n, nv), nv))
        total += A.n * nv
        if total >= 1_500_000:
            break
    stored = sum(fp16_stored_bytes(A) for A, _, _ in sample)
    vecs = sum(nv for _, _, nv in sample)
    for A, x, _ in sample[:2]:
        oracle.matvec(A, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for A, x, _ in sample:
            oracle.matvec(A, x)
    sec = (time.perf_counter() - t0) / args.steps
    val = round(stored / sec / 1e9, 3)
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(sec * 1e3, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOADS["batch256"], "sample_members": len(sample), "stored_bytes": stored},
           "vectors_per_s": round(vecs / sec, 2),
           "cpu_baseline": {"value": val, "unit": "GB/s", "cores": oracle.threads(), "kind": "oracle",
                            "sample": f"first {len(sample)} of 256 members ({vecs} vectors) per step"},
           "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
