"""Benchmark: adaptive randomized column ID (Algorithm 1 of arXiv:2310.09417) on
GB300.

Default line: the 40000 x 10000 FP64 workload (A = U diag(s) V^T with the
polynomial spectrum s_j = (1+j)^-2, sketch block b = 64, relative tolerance
1e-10) on the FP64-accurate tensor-core path (sketch, Schur GEMM and block
update as exact BF16 digit products on tcgen05; LU, X and norms in FP64).

One step = one complete adaptive ID (every step of the hot path: Gaussian rows,
sketch GEMM, Schur complement and its FP64 norm, stop test, LUPP, re-blocking,
interpolation matrix) on inputs resident in HBM.  The metric is throughput in
algorithmic GFLOP/s at the fixed relative error; ms_per_step is the ID time.

The same run times the other forms the metric compares ("forms"), each with its
own CUDA events, roofline fraction, e2e and error: plain FP64 on the same
matrix (the baseline), the FP32-accurate tensor-core path, BF16 and FP8 mixed
precision on the 100000 x 20000 matrix, the predictor-seeded BF16 run and the
batched kernel blocks.  The cpu_baseline leg runs the oracle on the first
rounds of Algorithm 1 over the same full-size matrix and compares its
skeletons, estimates and pivots with the GPU's ("parity").

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--forms auto|all|none]
                  [--impl reference]

Multi-GPU: one ID does not shard across GPUs here, so N ranks run N
independent replicas (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ID time & GFLOP/s at fixed rel. error; mixed/batched/learned vs plain FP64"
UNIT = "GFLOP/s"

WORKLOADS = {
    # name: (m, n, spectrum kind, kwargs, dtype, rel tol, block)
    "adaptive_poly_f32": (40000, 10000, "poly", {}, "f32", 1e-6, 64),
    "adaptive_step_f32": (40000, 10000, "step", {"rank": 600, "floor": 1e-9}, "f32", 1e-6, 64),
    # FP32 A, LU and X with the FP32-accurate sketch on the BF16 tensor cores (3 digit slices)
    "adaptive_poly_f32emu": (40000, 10000, "poly", {}, "f32emu", 1e-6, 64),
    "adaptive_step_f32emu": (40000, 10000, "step", {"rank": 600, "floor": 1e-9}, "f32emu", 1e-6, 64),
    "adaptive_poly_f64": (40000, 10000, "poly", {}, "f64", 1e-10, 64),
    "adaptive_step_f64": (40000, 10000, "step", {"rank": 600, "floor": 1e-9}, "f64", 1e-10, 64),
    # FP64 A, LU and X with the FP64-accurate sketch on the BF16 tensor cores (exact digit
    # slices of A, Omega on the grid 2^-11)
    "adaptive_poly_f64emu": (40000, 10000, "poly", {}, "f64emu", 1e-10, 64),
    "adaptive_step_f64emu": (40000, 10000, "step", {"rank": 600, "floor": 1e-9}, "f64emu", 1e-10, 64),
    # the sparse-sign sketch of Sec. 5.1 (zeta = 8) on the same FP64 matrix: the gather-add
    # reads A once per pass in FP64; the Schur GEMM and block update stay on the tensor cores
    "adaptive_poly_f64emu_sparse": (40000, 10000, "poly", {}, "f64emu", 1e-10, 64),
    "adaptive_poly_f64_sparse": (40000, 10000, "poly", {}, "f64", 1e-10, 64),
    "small_poly_f64emu_sparse": (16384, 4096, "poly", {}, "f64emu", 1e-10, 64),
    "adaptive_poly_f32_sparse": (40000, 10000, "poly", {}, "f32", 1e-6, 64),
    "mixed_bf16_tol3e-2_sparse": (100000, 20000, "lowrank", {"rank": 1500, "noise": 1e-4}, "bf16", 3e-2, 64),
    # reduced sizes of the same families, for profiler captures (inputs still > L2)
    "small_poly_f64": (16384, 4096, "poly", {}, "f64", 1e-10, 64),
    "small_poly_f32": (16384, 4096, "poly", {}, "f32", 1e-6, 64),
    "small_poly_f64emu": (16384, 4096, "poly", {}, "f64emu", 1e-10, 64),
    "small_poly_f32emu": (16384, 4096, "poly", {}, "f32emu", 1e-6, 64),
    # mixed precision: A stored in BF16 = Gaussian factor product of rank 1500 + 1e-4 noise,
    # sketch on the tensor cores (BF16 x BF16 -> FP32), LU in FP32, norms in FP64
    "mixed_bf16": (100000, 20000, "lowrank", {"rank": 1500, "noise": 1e-4}, "bf16", 1e-3, 64),
    "mixed_bf16_tol3e-3": (100000, 20000, "lowrank", {"rank": 1500, "noise": 1e-4}, "bf16", 3e-3, 64),
    "mixed_bf16_tol3e-2": (100000, 20000, "lowrank", {"rank": 1500, "noise": 1e-4}, "bf16", 3e-2, 64),
    "small_mixed_bf16": (32768, 8192, "lowrank", {"rank": 600, "noise": 1e-4}, "bf16", 1e-3, 64),
    # the same matrix quantised to FP8 E4M3 with power-of-two scales per 128-row block;
    # E4M3 sketch on the tensor cores (kind::f8f6f4), LU in FP32.  The E4M3 rounding
    # (about 2.6e-2 relative) is part of the stored matrix
    "mixed_fp8": (100000, 20000, "lowrank", {"rank": 1500, "noise": 1e-4}, "fp8", 1e-3, 64),
    "mixed_fp8_tol5e-2": (100000, 20000, "lowrank", {"rank": 1500, "noise": 1e-4}, "fp8", 5e-2, 64),
    "small_mixed_fp8": (32768, 8192, "lowrank", {"rank": 600, "noise": 1e-4}, "fp8", 5e-2, 64),
    # batched: 4096 off-diagonal blocks exp(-|x-y|^2/h^2), h = 0.3, of a k-d tree over 2^20 uniform
    # points in the unit cube (leaves of at most 1024 points, sizes 64..1024), one persistent launch
    "batched_kernel_f64": (2 ** 20, 4096, "kernel", {"leaf_max": 1024, "h": 0.3}, "f64", 1e-8, 32),
    "batched_kernel_f32": (2 ** 20, 4096, "kernel", {"leaf_max": 1024, "h": 0.3}, "f32", 1e-8, 32),
    # the same batch at a tolerance FP32 can certify (at 1e-8 every FP32 problem runs to its rank cap)
    "batched_kernel_f32_tol1e-5": (2 ** 20, 4096, "kernel", {"leaf_max": 1024, "h": 0.3}, "f32", 1e-5, 32),
    "small_batched_kernel_f64": (2 ** 16, 512, "kernel", {"leaf_max": 512, "h": 0.3}, "f64", 1e-8, 32),
    # fixed rank (randLUPP, Sec. 3.1): 2000 x 2000 FP64, s_j = 10^(-j/20), U and V Haar, one
    # sketch of l = 120 Gaussian rows, k = 100 skeleton columns, the estimate from the l - k extra
    # rows; plain FP64 and the FP64-accurate tensor-core sketch.  A is 32 MB (inside L2): L2 is
    # flushed before every timed ID
    "fixed_f64": (2000, 2000, "fixed", {"k": 100, "l": 120}, "f64", None, 64),
    "fixed_f64emu": (2000, 2000, "fixed", {"k": 100, "l": 120}, "f64emu", None, 64),
}
DEFAULT_WORKLOAD = "adaptive_poly_f64emu"
# Peaks of the plain-ALU paths, from unit counts x maximum SM clock (2070 MHz):
# FP32: 152 SMs x 128 FMA lanes x 2 flops; FP64: the 1.25 TFLOP/s GB300 rate.
ALU_PEAK_TFLOPS = {"f32": 152 * 128 * 2 * 2.070e9 / 1e12, "f64": 1.25}
# Measured copy bandwidth of the GB300s (fallback: the recipe's 6.8 TB/s).
try:
    PEAKS = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
except (OSError, ValueError):
    PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# DRAM bytes per sketch launch (dram__bytes_read.sum + dram__bytes_write.sum) from the ncu
# captures summarised under profiles/, scaled to the full size by the A bytes read.
# DRAM bytes (read + write) per launch of the dominant kernel, from ncu captures (the
# 16384 x 4096 captures of the FP64-accurate and sparse-sign sketches scaled by m n to
# 40000 x 10000: their traffic grows in proportion)
PROFILED_TRAFFIC = {"adaptive_poly_f64": 3.40e9, "adaptive_step_f64": 3.40e9,
                    "adaptive_poly_f64emu": 5.75e9, "adaptive_step_f64emu": 5.75e9,
                    "adaptive_poly_f64emu_sparse": 3.40e9, "adaptive_poly_f64_sparse": 3.40e9}


def algorithmic_flops(m: int, n: int, k: int, b: int) -> float:
    """Flops the method must perform for a rank-k ID with block b: the sketch of
    k + b rows (incl. the last estimation block), per round the triangular solve,
    Schur update and panel LU at rank tb, and the final interpolation solve."""
    f = 2.0 * m * n * (k + b)
    tb = 0
    while tb < k:
        f += b * tb * tb + 2.0 * (n - tb) * tb * b + (n - tb) * b * b
        tb += b
    f += float(k) * k * (n - k)
    return f


def make_input(name, device, seed=2310_09417 + 1):
    import torch

    from paper_2310_09417_gb300 import workloads as W
    m, n, kind, kw, dt, _, _ = WORKLOADS[name]
    if kind == "lowrank":
        # A^T = G2^T G1^T + noise (n x m row-major == A column-major), rounded to BF16
        g = torch.Generator(device=device)
        g.manual_seed(seed)
        r = kw["rank"]
        G1t = torch.randn(r, m, generator=g, device=device, dtype=torch.float32)
        G2t = torch.randn(n, r, generator=g, device=device, dtype=torch.float32)
        torch.backends.cuda.matmul.allow_tf32 = False
        At = torch.empty((n, m), dtype=torch.bfloat16, device=device)
        for j0 in range(0, n, 2048):  # bounded temporaries
            blk = G2t[j0:j0 + 2048] @ G1t
            blk += kw["noise"] * torch.randn(blk.shape, generator=g, device=device, dtype=torch.float32)
            At[j0:j0 + 2048] = blk.to(torch.bfloat16)
            del blk
        del G1t, G2t
        torch.cuda.synchronize()
        if dt == "fp8":
            from paper_2310_09417_gb300 import binding as B
            A8 = B.quantize_fp8(At.t(), pow2=True)
            del At
            torch.cuda.synchronize()
            return A8
        return At.t()
    if kind == "fixed":
        At = W.spectral_matrix_torch(m, n, W.spectrum("geometric", min(m, n)), seed, torch.float64, device)
        torch.cuda.synchronize()
        return At.t()
    s = W.spectrum(kind, n, **kw)
    dtype = torch.float32 if dt in ("f32", "f32emu") else torch.float64
    if dt in ("f32", "f32emu"):
        # U, V from an FP32 QR; the product in FP32 (TF32 off): the rounding of A
        # (~6e-8 relative) is far below the 1e-6 tolerance
        torch.backends.cuda.matmul.allow_tf32 = False
        g = torch.Generator(device=device)
        g.manual_seed(seed)

        def haar(rows, cols):
            G = torch.randn(rows, cols, generator=g, device=device, dtype=torch.float32)
            Q, R = torch.linalg.qr(G)
            d = torch.sign(torch.diagonal(R))
            d[d == 0] = 1
            return Q * d
        U = haar(m, n)
        V = haar(n, n)
        At = (V * torch.as_tensor(s, dtype=torch.float32, device=device)) @ U.T
        del U, V
    else:
        At = W.spectral_matrix_torch(m, n, s, seed, torch.float64, device)
    torch.cuda.synchronize()
    return At.t()  # (m, n) column-major view


def host_f64(A):
    """A (a column-major device tensor or an FP8Matrix) as an FP64 Fortran-order host
    array of the values the ID works on (FP8: the decoded values times the scales)."""
    import numpy as np
    import torch
    if hasattr(A, "scale"):
        m = A.shape[0]
        s = A.scale.repeat_interleave(128, dim=0)[:m]
        At = (A.data.float() * s).t().contiguous()
    else:
        At = A.t().contiguous()
    out = np.asfortranarray(At.double().cpu().numpy().T)
    del At
    torch.cuda.empty_cache()
    return out


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # RANDID_CLOCKS_DIR keeps the raw samples; by default they go to the temp directory
        out = os.environ.get("RANDID_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, "randid_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def ref_rounds(args, name):
    """Rounds of the oracle sample: about 1.7e11 flops of sketch (4 s on 16 Grace cores)."""
    if args.ref_rounds > 0:
        return args.ref_rounds
    m, n, _, _, _, _, b = WORKLOADS[name]
    return int(min(8, max(1, round(1.7e11 / (2.0 * m * n * b)))))


def on_grid(Om):
    """Omega as the FP64-accurate tensor-core path defines it: the Gaussian rounded
    to the grid 2^-11 and clipped at |q| <= 16383."""
    import numpy as np
    return np.clip(np.rint(Om * 2048.0), -16383.0, 16383.0) / 2048.0


def cpu_oracle_sample(A_host_f64, name, seed, rounds=6):
    """The FP64 oracle as it stands, on the first `rounds` rounds of Algorithm 1
    over the full matrix (the run stops at k_max = rounds * b), with the Gaussian
    rows of `seed` (on the grid 2^-11 for the FP64-accurate tensor-core path).
    Returns (GFLOP/s, seconds, threads, description, oracle result)."""
    import oracle
    _, _, _, _, dt, tol, b = WORKLOADS[name]
    m, n = A_host_f64.shape  # the workload's size on a GPU machine; reduced without a GPU
    kmax = rounds * b
    if is_sparse(name):
        Om = oracle.sparse_sign_rows(seed, 0, rounds + 1, b, m)
    else:
        Om = oracle.gaussian_rows(seed, 0, (rounds + 1) * b, m)
        if dt == "f64emu":
            Om = on_grid(Om)
    t0 = time.perf_counter()
    r = oracle.id_adaptive(A_host_f64, Om, b, tol * 1.0, kmax=kmax)
    dt_s = time.perf_counter() - t0
    k = r["k"]
    flops = algorithmic_flops(m, n, k, b)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    desc = ("oracle (plain C, FP64, OpenMP) on the first %d rounds of Algorithm 1 over the whole "
            "%dx%d matrix (k_max = %d), %.1f s" % (rounds, m, n, kmax, dt_s))
    return flops / dt_s / 1e9, dt_s, threads, desc, r


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on a bounded sample of the same workload."""
    if rank != 0:
        return
    import numpy as np
    import torch

    name = args.workload
    m, n, kind, kw, dt, tol, b = WORKLOADS[name]
    dev = torch.device("cuda", 0) if torch.cuda.is_available() else None
    if kind == "kernel":
        run_reference_batched(args, name, dev)
        return
    if kind == "fixed":
        run_reference_fixed(args, name, dev, world)
        return
    if dev is not None:
        A = make_input(name, dev)
        A_host = host_f64(A)
        del A
    else:  # no GPU: same family, host generation at reduced size
        from paper_2310_09417_gb300 import workloads as W
        A_host = W.spectral_matrix(m // 10, n // 10, W.spectrum(kind, n // 10, **kw), 1)
    rounds = ref_rounds(args, name)
    times, vals = [], []
    for i in range(args.warmup + args.steps):
        v, sec, threads, desc, _ = cpu_oracle_sample(A_host, name, seed=2310_09417 + i, rounds=rounds)
        if i >= args.warmup:
            times.append(sec)
            vals.append(v)
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(name, None),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_fixed(args, name, dev, world):
    """Reference arm for the fixed-rank workload: the oracle's whole fixed-rank ID of
    the same matrix with the same Gaussian rows, once per step."""
    import oracle
    from paper_2310_09417_gb300 import workloads as W
    m, n, kind, kw, dt, _, b = WORKLOADS[name]
    k, l = kw["k"], kw["l"]
    oracle.build()
    if dev is not None:
        A = make_input(name, dev)
        A_host = host_f64(A)
        del A
    else:  # no GPU: the same family generated on the host
        A_host = W.spectral_matrix(m, n, W.spectrum("geometric", min(m, n)), 1)
    Om = oracle.gaussian_rows(2310_09417, 0, l, m)
    if dt == "f64emu":
        Om = on_grid(Om)
    flops = fixed_flops(m, n, k, l, b)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.id_fixed_rank(A_host, Om, k)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    sec = statistics.mean(times)
    value = flops / sec / 1e9
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    desc = "oracle (plain C, FP64, OpenMP) on the whole fixed-rank ID, %.1f ms" % (sec * 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec, "us_per_id": 1e6 * sec,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": name, "m": m, "n": n, "k": k, "l": l, "block": b,
                                            "spectrum": "s_j = 10^(-j/20)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_batched(args, name, dev):
    """Reference arm for the batched workload: the oracle, one block after another,
    on the largest blocks of the batch (about 8 s per step)."""
    import numpy as np

    import oracle
    from paper_2310_09417_gb300 import workloads as W
    npts, count, kind, kw, dt, tol, b = WORKLOADS[name]
    pts, leaves, pairs = W.kernel_block_pairs(npts, count, 2310_09417 + 3, leaf_max=kw["leaf_max"], size_min=64)
    pairs = sorted(pairs, key=lambda p: -len(leaves[p[0]]) * len(leaves[p[1]]))
    times, vals, used = [], [], 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        fl, used = 0.0, 0
        for a, c in pairs:
            A = W.gaussian_kernel_block(pts, leaves[a], leaves[c], h=kw["h"])
            mm, nn = A.shape
            Om = oracle.gaussian_rows(2310_09417, 0, oracle.rows_needed(nn, b, m=mm), mm)
            r = oracle.id_adaptive(A, Om, b, tol * oracle.fro_norm(A))
            fl += algorithmic_flops(mm, nn, r["k"], b)
            used += 1
            if time.perf_counter() - t0 > 8.0:
                break
        sec = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(sec)
            vals.append(fl / sec / 1e9)
    value = statistics.mean(vals)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    desc = "oracle (plain C, FP64, OpenMP) on the %d largest of the %d blocks per step" % (used, count)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(name, None),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(name, res):
    m, n, kind, kw, dt, tol, b = WORKLOADS[name]
    if kind == "kernel":
        return {"workload": name, "points": m, "blocks": n, "kernel": "exp(-|x-y|^2/h^2), h = %s" % kw["h"],
                "tree": "k-d tree, widest side split at U[0.3,0.7], leaves <= %d points" % kw["leaf_max"],
                "block_sizes": "m, n in [64, %d]" % kw["leaf_max"], "block": b, "rel_tol": tol,
                "precision": "%s sketch, LU and X; FP64 norms" % dt.upper(),
                "omega": "Philox4x64-10 Gaussian, generated inside the kernel",
                "l2": "inputs larger than L2 (the batch is %s)" % (res if res else "several GB"),
                "parallelism": "one persistent launch, CTA per problem; replicas across GPUs"}
    spec = {"poly": "s_j = (1+j)^-2", "step": "rank 600 at 1, then 1e-9",
            "lowrank": "G1 G2 (Gaussian factors, rank %s) + %s N(0,1) noise, stored in %s"
                       % (kw.get("rank"), kw.get("noise"), "FP8 E4M3" if dt == "fp8" else "BF16")}[kind]
    if name.startswith("small_"):
        spec += " (reduced size for profiling)"
    el = {"f32": 4, "f32emu": 4, "f64": 8, "f64emu": 8, "bf16": 2, "fp8": 1}[dt]
    prec = {"f64": "FP64 sketch, LU and X", "f32": "FP32 sketch, LU and X",
            "f64emu": "FP64 A, LU and X; FP64-accurate sketch, Schur GEMM and block update on the BF16 tensor cores "
                      "(7 exact 8-bit digit slices per operand, Omega on the grid 2^-11 in 2 digits, exact FP32 "
                      "chunk sums, int64 totals)",
            "f32emu": "FP32 A, LU and X; FP32-accurate sketch on the BF16 tensor cores (3 exact 8-bit digit slices "
                      "of A and of Omega, exact FP32 chunk sums, int64 totals)",
            "bf16": "BF16 A and Omega, tensor-core sketch with FP32 accumulation, FP32 LU and X, FP64 norms",
            "fp8": "FP8 E4M3 A with power-of-two FP32 scales per 128-row block (quantised from the BF16 matrix), "
                   "E4M3 Omega, tcgen05 kind::f8f6f4 sketch with FP32 accumulation, FP32 LU and X, FP64 norms"}[dt]
    if is_sparse(name):
        prec = ("FP64 A, LU and X; sparse-sign gather-add sketch in FP64" +
                ("; FP64-accurate Schur GEMM and block update on the BF16 tensor cores (7 exact 8-bit digit slices "
                 "per operand)" if dt == "f64emu" else "; FP64 SIMT Schur GEMM and block update"))
    c = {"workload": name, "m": m, "n": n, "spectrum": spec, "block": b, "rel_tol": tol,
         "precision": prec,
         "omega": ("sparse sign (Sec. 5.1), zeta = 8 nonzeros +-sqrt(b/8) per column of each block, Philox4x64-10 "
                   "counters, generated on the device; the sketch is a gather-add in A's precision"
                   if is_sparse(name) else "Philox4x64-10 Gaussian, generated on the device"
                   + (", rounded to the grid 2^-11" if dt == "f64emu" else "")),
         "l2": "inputs larger than L2 (A is %.1f GB)" % (m * n * el / 1e9),
         "parallelism": "replicas (one ID per GPU)"}
    if res is not None:
        c.update({"k": res.k, "rounds": res.rounds, "passes": res.passes})
    return c


def make_batch(name, device, seed=2310_09417 + 3, rank=0, world=1):
    """The kernel blocks of the batched workload (column-major CUDA tensors).  With
    world > 1 the batch holds count * world blocks of the same tree, and this rank
    builds only its share of a size-balanced assignment (greedy LPT on the sketch
    cost 2 m n (k + b), k estimated as min(m, n, 64)): every rank runs about
    `count` blocks, with no collective on the data path.  Returns (blocks, info)."""
    import torch

    from paper_2310_09417_gb300 import shard
    from paper_2310_09417_gb300 import workloads as W
    npts, count, kind, kw, dt, _, b = WORKLOADS[name]
    total = count * world
    pts, leaves, pairs = W.kernel_block_pairs(npts, total, seed, leaf_max=kw["leaf_max"], size_min=64)
    info = {"blocks_total": len(pairs)}
    if world > 1:
        costs = [shard.problem_cost(len(leaves[a]), len(leaves[c]), min(len(leaves[a]), len(leaves[c]), 64), b)
                 for a, c in pairs]
        parts = shard.assign(costs, world)
        info.update({"blocks_this_rank": len(parts[rank]), "load_imbalance": shard.imbalance(costs, parts),
                     "assignment": "greedy LPT on 2 m n (min(m, n, 64) + b)"})
        pairs = [pairs[i] for i in parts[rank]]
    P = torch.from_numpy(pts).to(device)
    idx = [torch.from_numpy(l).to(device) for l in leaves]
    dtype = torch.float64 if dt == "f64" else torch.float32
    h2 = kw["h"] ** 2
    As = []
    for a, c in pairs:
        d2 = torch.cdist(P[idx[c]], P[idx[a]]) ** 2  # n x m row-major == m x n column-major
        As.append(torch.exp(-d2 / h2).to(dtype).t())
    torch.cuda.synchronize()
    return As, info


def measure_batched(B, name, dev, steps, warmup, seed, *, e2e=True, cpu_baseline=False, errors=False,
                    max_over_ranks=None, barrier=None, rank=0, world=1):
    """One persistent launch per step over the whole batch of kernel blocks.
    Returns the form's measurements (ms per step, GFLOP/s, roofline, e2e, the
    ranks, and with `errors` each block's relative error evaluated in FP64)."""
    import torch

    max_over_ranks = max_over_ranks or (lambda x: x)
    barrier = barrier or (lambda: None)
    npts, count, kind, kw, dt, tol, b = WORKLOADS[name]
    As, shard_info = make_batch(name, dev, rank=rank, world=world)
    xdt = torch.float64 if dt == "f64" else torch.float32
    outs = [(torch.empty(min(A.shape), dtype=torch.int64, device=dev),
             torch.empty((A.shape[1], min(A.shape)), dtype=xdt, device=dev)) for A in As]
    nbytes = sum(A.numel() * A.element_size() for A in As)
    stream = torch.cuda.current_stream(dev)
    import ctypes
    mats = (B.IdMatrix * len(As))(*[B._matrix(a) for a in As])
    o = B._opts(As[0], block=b, tol=tol, relative=True, k_max=0, k0=0, blocks_per_pass=1, seed=seed, omega=None,
                profile=False)
    nb = ctypes.c_size_t(0)
    B.load().id_batched_workspace_size(len(As), mats, ctypes.byref(o), ctypes.byref(nb))
    ws = torch.empty(nb.value, dtype=torch.uint8, device=dev)

    def step():
        return B.id_batched(As, tol, block=b, seed=seed, outs=outs, workspace=ws, stream=stream)
    for _ in range(max(warmup, 1)):
        res = step()
    torch.cuda.synchronize()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_gpu(dev)) as clk:
        ev0.record(stream)
        for _ in range(steps):
            res = step()
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / steps)
    flops = sum(algorithmic_flops(A.shape[0], A.shape[1], r.k, b) for A, r in zip(As, res))
    ks = [r.k for r in res]
    peak = ALU_PEAK_TFLOPS[dt]
    achieved = flops / (ms * 1e-3) / 1e12
    out = {"workload": name, "ms_per_step": ms, "value": flops / (ms * 1e-3) / 1e9, "unit": UNIT,
           "steps": steps, "warmup": warmup, "flops": flops, "ids": len(As),
           "roofline": {"bound": "alu", "kernel": "k_batched (one persistent launch per step, %s FMA)" % dt,
                        "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                        "traffic": None, "timing": "CUDA events around the whole step (descriptor upload, graph "
                                                   "replay of the persistent kernel, result copy)",
                        "peak_source": "derived: %s" % ("152 SMs x 128 FP32 lanes x 2 x 2.07 GHz" if dt == "f32"
                                                         else "GB300 FP64 rate 1.25 TFLOP/s")},
           "result": {"k_mean": sum(ks) / len(ks), "k_max": max(ks), "k_min": min(ks),
                      "statuses": sorted(set(r.status for r in res)), "batch_gb": round(nbytes / 1e9, 2),
                      "ids_per_s": len(As) / (ms * 1e-3), "shard": shard_info},
           "gpu_launches": 2 * steps, "clocks": clk.summary()}
    if errors:
        # each block's ||A - A(:,J)X||_F / ||A||_F evaluated in FP64 (harness check, not timed)
        rel = []
        for A, r in zip(As, res):
            A64 = A.double()
            E = A64 - A64[:, r.J] @ r.X.double()
            rel.append(float(torch.linalg.norm(E) / torch.linalg.norm(A64)))
        out["result"].update({"rel_err_max": max(rel), "rel_err_mean": sum(rel) / len(rel),
                              "met_tol": sum(1 for e in rel if e <= tol), "tol": tol})
    if e2e:
        hosts = [torch.empty((A.shape[1], A.shape[0]), dtype=A.dtype, pin_memory=True) for A in As]
        for h, A in zip(hosts, As):
            h.copy_(A.t())
        devs = [torch.empty_like(h, device=dev) for h in hosts]
        xh = [torch.empty_like(X, device="cpu", pin_memory=True) for _, X in outs]

        def e2e_step():
            for h, d in zip(hosts, devs):
                d.copy_(h, non_blocking=True)
            r = B.id_batched([d.t() for d in devs], tol, block=b, seed=seed, outs=outs, workspace=ws,
                             stream=stream)
            for x, (_, X) in zip(xh, outs):
                x.copy_(X, non_blocking=True)
            return r
        for _ in range(max(warmup, 1)):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        e_ms = max_over_ranks(e0.elapsed_time(e1) / steps)
        out["e2e"] = {"value": flops / (e_ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": e_ms,
                      "h2d_bytes_per_step": nbytes,
                      "d2h_bytes_per_step": sum(x.numel() * x.element_size() for x in xh)}
        del hosts, devs, xh
    if cpu_baseline:
        import numpy as np

        import oracle
        t0 = time.perf_counter()
        fl = 0.0
        used = 0
        for A in As:  # the largest blocks first, until ~8 s of oracle work
            Ah = np.asfortranarray(A.t().contiguous().double().cpu().numpy().T)
            mm, nn = Ah.shape
            Om = oracle.gaussian_rows(seed, 0, oracle.rows_needed(nn, b, m=mm), mm)
            r = oracle.id_adaptive(Ah, Om, b, tol * oracle.fro_norm(Ah))
            fl += algorithmic_flops(mm, nn, r["k"], b)
            used += 1
            if time.perf_counter() - t0 > 8.0:
                break
        dtc = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": fl / dtc / 1e9, "unit": UNIT,
                               "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count())), "kind": "oracle",
                               "sample": "oracle (plain C, FP64, OpenMP) on the first %d of the %d blocks, %.1f s"
                                         % (used, len(As), dtc)}
    del As, outs, ws
    torch.cuda.empty_cache()
    return out


def run_batched(args, rank, world, dev, barrier, max_over_ranks, sum_over_ranks):
    from paper_2310_09417_gb300 import binding as B
    name = args.workload
    seed = 2310_09417 + 100 * rank
    r = measure_batched(B, name, dev, args.steps, args.warmup, seed, e2e=not args.no_e2e,
                        cpu_baseline=rank == 0 and world == 1 and not args.no_cpu_baseline,
                        max_over_ranks=max_over_ranks, barrier=barrier, rank=rank, world=world)
    # whole job: the work of every rank (replicas with their own seeds) over the slowest rank's time
    flops_all = sum_over_ranks(r["flops"])
    value = flops_all / (r["ms_per_step"] * 1e-3) / 1e9
    if r.get("e2e"):
        r["e2e"]["value"] = flops_all / (r["e2e"]["ms_per_step"] * 1e-3) / 1e9
    if rank == 0:
        cfg = config_dict(name, None)
        cfg.update({k: r["result"][k] for k in ("k_mean", "k_max", "k_min", "batch_gb")})
        if world > 1:
            cfg["parallelism"] = ("sharded: %d blocks over %d ranks by a size-balanced assignment, no collective on "
                                  "the data path" % (r["result"]["shard"]["blocks_total"], world))
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_LABEL.get(WORKLOADS[name][4], "f64"),
                "data": "synthetic", "config": cfg, "roofline": r["roofline"],
                "cpu_baseline": r.get("cpu_baseline"), "e2e": r.get("e2e"), "gpu_launches": r["gpu_launches"],
                "clocks": r["clocks"], "result": r["result"]}
        print(json.dumps(line), flush=True)


def over_ranks(x: float, op: str, world: int, device) -> float:
    """x reduced over the ranks of the default process group, op "max" or "sum",
    as one FP64 value on `device` (a CUDA device under NCCL, the CPU under gloo);
    x itself on a single rank."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op={"max": dist.ReduceOp.MAX, "sum": dist.ReduceOp.SUM}[op])
    return float(t.item())


def local_gpu(dev):
    return dev.index


DTYPE_LABEL = {
    "f64": "f64",
    "f32": "f32",
    "f64emu": "f64 (FP64-accurate: sketch, Schur GEMM and block update as exact bf16 digit products on tcgen05 "
              "with fp32/int64 sums; LU, X and norms in f64)",
    "f32emu": "f32 (FP32-accurate sketch as exact bf16 digit products on tcgen05; LU and X in f32)",
    "bf16": "bf16 (sketch on tcgen05, fp32 accumulation), f32 (LU, X), f64 (norms)",
    "fp8": "fp8 e4m3 (sketch on tcgen05, fp32 accumulation), f32 (LU, X), f64 (norms)",
}


def sketch_roofline(name, m, n, b, passes, blocks, sk_ms, sk_launches):
    """Roofline of the dominant kernel, the sketch (+ its split-K reduction), from the
    library's per-phase CUDA events on the launching stream.  The method's own work
    per ID: A read once per pass in its storage precision, plus one Omega block
    and one sketch block per block of rows (bytes), and 2 m n rows multiply-adds
    (flops; on the digit-sliced paths every FP64 / FP32 product is 14 / 6 BF16
    digit products).  The bound is the larger of bytes / HBM bandwidth and tensor
    flops / tensor peak; frac = that time / the measured time.  A pass that
    sketches many blocks (the predictor) moves from the HBM to the tensor bound."""
    dt = WORKLOADS[name][4]
    rows = blocks * b
    t = sk_ms * 1e-3
    if is_sparse(name):
        esz = {"f64": 8, "f64emu": 8, "f32": 4, "f32emu": 4, "bf16": 2}[dt]
        # A once per pass, the lists of the pass's blocks (2 bytes per nonzero: zeta
        # per column of A and block), the sketch block written
        byts = esz * m * n * passes + 2.0 * 8 * m * rows / b + esz * n * rows
        achieved = byts / t / 1e9
        return {"bound": "hbm", "kernel": "k_sparse_gather (sparse-sign gather-add, zeta = 8; lists from "
                "k_sparse_csr) + split-K reduce", "achieved": achieved, "peak": PEAKS["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / PEAKS["hbm_gbs"], "traffic": PROFILED_TRAFFIC.get(name),
                "algorithmic_bytes_per_step": byts, "sketch_launches_per_step": sk_launches,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    if dt in ("f64", "f32"):
        fl = 2.0 * m * n * rows
        achieved = fl / t / 1e12
        peak = ALU_PEAK_TFLOPS[dt]
        return {"bound": "alu", "kernel": "k_sgemm_gather (sketch Y = Omega A, %s FMA) + split-K reduce" % dt,
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": PROFILED_TRAFFIC.get(name), "sketch_launches_per_step": sk_launches,
                "peak_source": "derived: %s" % ("152 SMs x 128 FP32 lanes x 2 x 2.07 GHz" if dt == "f32"
                                                 else "GB300 FP64 rate 1.25 TFLOP/s")}
    bf16_peak = PEAKS.get("bf16_tflops_sustained", PEAKS["bf16_tflops"])
    extra = {}
    if dt == "bf16":
        byts = 2.0 * m * n * passes + (2.0 * m + 4.0 * n) * rows
        tfl, tpeak = 2.0 * m * n * rows, bf16_peak
        kern = "k_sketch_tc_bf16 (tcgen05 + TMA) + split-K reduce"
    elif dt == "fp8":
        nbs = (m + 127) // 128
        byts = (1.0 * m * n + 4.0 * nbs * n) * passes + (1.0 * m + 4.0 * n) * rows
        tfl, tpeak = 2.0 * m * n * rows, 2.0 * bf16_peak
        kern = "k_sketch_tc_fp8 (tcgen05 kind::f8f6f4 + TMA, block scales) + split-K reduce"
    elif dt == "f32emu":
        byts = 4.0 * m * n * passes + (4.0 * m + 4.0 * n) * rows
        tfl, tpeak = 6 * 2.0 * m * n * rows, bf16_peak
        kp = (m + 63) // 64 * 64
        stream = 6.0 * kp * n * passes + (16.0 * kp + 4.0 * n) * rows + 10.0 * m * n
        extra = {"stream_bytes": stream, "frac_of_stream": stream / t / 1e9 / PEAKS["hbm_gbs"]}
        kern = "k_sketch_f32emu (tcgen05 + TMA, exact digit slices) + Omega slicing + split-K reduce"
    else:  # f64emu
        byts = 8.0 * m * n * passes + (8.0 * m + 8.0 * n) * rows
        tfl, tpeak = 14 * 2.0 * m * n * rows, bf16_peak
        mp = (m + 7) // 8 * 8
        stream = 14.0 * mp * n * passes + (4.0 * mp + 8.0 * n) * rows + 30.0 * m * n
        extra = {"stream_bytes": stream, "frac_of_stream": stream / t / 1e9 / PEAKS["hbm_gbs"],
                 "note": "frac counts the method's 8 bytes per element of A per pass; the kernel streams 14 "
                         "(seven BF16 digit slices), see stream_bytes"}
        kern = "k_sketch_f64emu (tcgen05 + TMA, exact digit slices) + split-K reduce + digit preparation"
    t_hbm = byts / (PEAKS["hbm_gbs"] * 1e9)
    t_tc = tfl / (tpeak * 1e12)
    if t_hbm >= t_tc:
        r = {"bound": "hbm", "achieved": byts / t / 1e9, "peak": PEAKS["hbm_gbs"], "unit": "GB/s",
             "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    else:
        r = {"bound": "tensor", "achieved": tfl / t / 1e12, "peak": tpeak, "unit": "TFLOP/s",
             "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)%s"
                            % (" x 2, the nominal FP8 : BF16 ratio" if dt == "fp8" else "")}
    r.update({"kernel": kern, "frac": max(t_hbm, t_tc) / t, "frac_hbm": t_hbm / t, "frac_tensor": t_tc / t,
              "traffic": PROFILED_TRAFFIC.get(name), "algorithmic_bytes_per_step": byts,
              "tensor_flops_per_step": tfl, "sketch_launches_per_step": sk_launches}, **extra)
    return r


def fixed_flops(m: int, n: int, k: int, l: int, b: int) -> float:
    """Flops of a rank-k fixed-rank ID from l sketch rows: the sketch, per block of
    pivots the triangular solve, Schur update and panel LU, the estimate rows'
    Schur product and the interpolation solve."""
    f = 2.0 * m * n * l
    tb = 0
    while tb < k:
        w = min(b, k - tb)
        f += w * tb * tb + 2.0 * (n - tb) * tb * w + (n - tb) * w * w
        tb += w
    f += 2.0 * (n - k) * k * (l - k) + float(k) * k * (n - k)
    return f


def run_fixed(args, rank, world, dev, barrier, max_over_ranks, sum_over_ranks):
    """The fixed-rank workload: `steps` IDs of the 2000 x 2000 matrix, each timed with
    its own CUDA events after an L2 flush (A fits in L2); the headline is the time
    per ID in microseconds.  e2e: A copied in from pinned host memory and J, X
    copied back inside each timed interval.  cpu_baseline / parity: the oracle's
    fixed-rank ID on the same matrix and the same Gaussian rows (on the grid 2^-11
    for the tensor-core path): J compared bit for bit, the relative errors of both
    IDs and the estimates."""
    import numpy as np
    import torch

    from paper_2310_09417_gb300 import binding as B
    name = args.workload
    m, n, kind, kw, dt, _, b = WORKLOADS[name]
    k, l = kw["k"], kw["l"]
    A = make_input(name, dev)
    seed = 2310_09417 + 100 * rank
    sprec = B.F64_EMU if dt == "f64emu" else None
    opts = B._opts(A, block=b, tol=0.0, relative=False, k_max=k, k0=0, blocks_per_pass=1, seed=seed, omega=None,
                   profile=True, sketch_prec=sprec)
    ws = torch.empty(B.workspace_size(A, opts, l), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # larger than the 129 MB L2

    def one(A_in, profile=True):
        return B.id_fixed_rank(A_in, k, l, block=b, seed=seed, profile=profile, workspace=ws, stream=stream,
                               sketch_prec=sprec)

    def timed(steps, fn):
        evs = []
        out = None
        for i in range(steps):
            flush.fill_(i & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(c) for a, c in evs) / steps, out

    for _ in range(max(args.warmup, 1)):
        one(A)
    torch.cuda.synchronize()
    barrier()
    results = []
    with ClockSampler(local_gpu(dev)) as clk:
        ms, _ = timed(args.steps, lambda: results.append(one(A)))
    barrier()
    ms = max_over_ranks(ms)
    res = results[-1]
    flops = fixed_flops(m, n, k, l, b)
    sk_ms = sum(r.phase_ms["sketch"] for r in results) / args.steps
    roof = sketch_roofline(name, m, n, b, 1, l / b, sk_ms, res.phase_launches["sketch"])
    tot = max(1e-9, sum(res.phase_ms.values()))
    roof.update({"phase_ms_per_step": {q: round(v, 4) for q, v in res.phase_ms.items()},
                 "phase_share": {q: round(v / tot, 4) for q, v in res.phase_ms.items()},
                 "timing": "library CUDA events on the launching stream around each phase, inside the timed "
                           "region"})
    e2e = None
    if not args.no_e2e:
        A_host = torch.empty((n, m), dtype=torch.float64, pin_memory=True)
        A_host.copy_(A.t())
        A_dev = torch.empty((n, m), dtype=torch.float64, device=dev)
        X_host = torch.empty((n, k), dtype=torch.float64, pin_memory=True)
        J_host = torch.empty(k, dtype=torch.int64, pin_memory=True)

        def e2e_step():
            A_dev.copy_(A_host, non_blocking=True)
            r = one(A_dev.t(), profile=False)
            X_host.copy_(r.X.t(), non_blocking=True)  # the (n x k) buffer behind X
            J_host.copy_(r.J, non_blocking=True)
        for _ in range(max(args.warmup, 1)):
            e2e_step()
        torch.cuda.synchronize()
        e_ms, _ = timed(args.steps, e2e_step)
        e_ms = max_over_ranks(e_ms)
        e2e = {"value": sum_over_ranks(flops) / (e_ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": e_ms,
               "us_per_id": e_ms * 1e3, "h2d_bytes_per_step": m * n * 8, "d2h_bytes_per_step": k * n * 8 + 8 * k}
    cpu, parity = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        A64 = host_f64(A)
        Om = oracle.gaussian_rows(seed, 0, l, m)
        if dt == "f64emu":
            Om = on_grid(Om)
        t0 = time.perf_counter()
        reps = 0
        while True:
            r = oracle.id_fixed_rank(A64, Om, k)
            reps += 1
            if time.perf_counter() - t0 > 2.0:
                break
        sec = (time.perf_counter() - t0) / reps
        threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        cpu = {"value": flops / sec / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "oracle (plain C, FP64, OpenMP) on the whole fixed-rank ID of the same matrix and the "
                         "same Gaussian rows, %d repetitions, %.1f ms each" % (reps, sec * 1e3)}
        Jg = res.J.cpu().numpy()
        Xg = res.X.double().cpu().numpy()
        nA = oracle.fro_norm(A64)
        eg = oracle.id_residual(A64, Jg, Xg) / nA
        eo = oracle.id_residual(A64, r["J"], r["X"]) / nA
        est_d = abs(res.est_err - r["est"]) / max(abs(r["est"]), 1e-300)
        parity = {"J_identical": bool(np.array_equal(Jg, r["J"])), "J_mismatches": int(np.sum(Jg != r["J"])),
                  "rel_error_gpu": eg, "rel_error_oracle": eo, "rel_error_diff": abs(eg - eo) / eo,
                  "estimate_rel_diff": est_d,
                  "bar": "J bit-exact; relative errors within 1e-10 of each other; estimate within 1e-10"}
        parity["pass"] = bool(parity["J_identical"] and parity["rel_error_diff"] <= 1e-10 and est_d <= 1e-10)
    if rank == 0:
        line = {"metric": METRIC, "value": sum_over_ranks(flops) / (ms * 1e-3) / 1e9, "unit": UNIT,
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "us_per_id": ms * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPE_LABEL[dt], "data": "synthetic",
                "config": {"workload": name, "m": m, "n": n, "spectrum": "s_j = 10^(-j/20)", "k": k, "l": l,
                           "block": b, "precision": ("FP64 A, LU and X; FP64-accurate sketch on the BF16 tensor "
                                                     "cores" if dt == "f64emu" else "FP64 sketch, LU and X"),
                           "omega": "Philox4x64-10 Gaussian, generated on the device"
                                    + (", rounded to the grid 2^-11" if dt == "f64emu" else ""),
                           "l2": "A is 32 MB (inside L2): L2 flushed (256 MB written) before every timed ID",
                           "parallelism": "replicas (one ID per GPU)"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": sum(r.launches for r in results), "clocks": clk.summary(),
                "result": {"k": res.k, "status": res.status,
                           "est_err_rel": res.est_err / res.norm_A if res.norm_A > 0 else 0.0,
                           "gflop_per_id": flops / 1e9}, "parity": parity}
        print(json.dumps(line), flush=True)


def is_sparse(name):
    """Workloads sketched with the sparse-sign matrix (Sec. 5.1) instead of Gaussian rows."""
    return name.endswith("_sparse")


def sampled_rel_error(A, J, X, norm_A, rows=4096, seed=5):
    """||A - A(:,J) X||_F / ||A||_F estimated in FP64 from a uniform sample of the
    rows of A (the squared error is a sum over rows, so (m/rows) times the
    sample's sum is unbiased).  A harness evaluation, not part of the timed ID."""
    import torch
    m, n = A.shape
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    I = torch.randperm(m, generator=g)[: min(rows, m)].to(X.device)
    if hasattr(A, "scale"):  # FP8: decoded values times the block scales
        rowsA = A.data.t()[:, I].float().t() * A.scale.t()[:, I // 128].t()
    else:
        rowsA = A.t()[:, I].t()
    R = rowsA.double()
    E = R - R[:, J] @ X.double()
    return float(torch.linalg.norm(E)) * math.sqrt(m / len(I)) / norm_A


def measure_adaptive(B, name, A, dev, steps, warmup, seed, *, e2e=True, predictor=None, max_pass_rows=0,
                     max_over_ranks=None, barrier=None, want_pivots=False, blocks_per_pass=0):
    """Time `steps` complete adaptive IDs of A (inputs resident in HBM) after
    `warmup` untimed ones; then, unless e2e is False, the same ID through the C ABI
    with A copied in from pinned host memory and J, X copied back inside the timed
    region.  Returns the measurements and the last result."""
    import torch

    max_over_ranks = max_over_ranks or (lambda x: x)
    barrier = barrier or (lambda: None)
    m, n, kind, kw, dt, tol, b = WORKLOADS[name]
    kmax = min(m, n)
    xdt = torch.float64 if dt in ("f64", "f64emu") else torch.float32
    sprec = {"f64emu": B.F64_EMU, "f32emu": B.F32_EMU}.get(dt)
    J = torch.empty(kmax, dtype=torch.int64, device=dev)
    Xbuf = torch.empty((n, kmax), dtype=xdt, device=dev)
    okind = B.OMEGA_SPARSE_SIGN if is_sparse(name) else B.OMEGA_GAUSSIAN
    opts = B._opts(A, block=b, tol=tol, relative=True, k_max=kmax, k0=0, blocks_per_pass=blocks_per_pass, seed=seed,
                   omega=None, profile=True, sketch_prec=sprec, omega_kind=okind)
    if predictor is not None:
        opts.predictor = predictor.data_ptr()
        opts.max_pass_rows = max_pass_rows
    ws = torch.empty(B.workspace_size(A, opts), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(profile=True, pivots=False):
        return B.id_adaptive(A, tol, block=b, relative=True, k_max=kmax, seed=seed, profile=profile,
                             workspace=ws, out=(J, Xbuf), stream=stream, sketch_prec=sprec, pivots=pivots,
                             predictor=predictor, max_pass_rows=max_pass_rows, omega_kind=okind,
                             blocks_per_pass=blocks_per_pass)

    for _ in range(max(warmup, 1)):
        res = step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    with ClockSampler(local_gpu(dev)) as clk:
        ev0.record(stream)
        for _ in range(steps):
            results.append(step())
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / steps)
    res = results[-1]
    flops = algorithmic_flops(m, n, res.k, b)
    sk_ms = sum(r.phase_ms["sketch"] for r in results) / steps
    # blocks of sketch rows the ID used: one per round plus the first (a seeded pass may
    # draw a few more that go unused; they are not counted)
    blocks = max(res.passes, res.rounds + 1)
    roof = sketch_roofline(name, m, n, b, res.passes, blocks, sk_ms, res.phase_launches["sketch"])
    tot = max(1e-9, sum(res.phase_ms.values()))
    roof.update({"phase_ms_per_step": {k: round(v, 3) for k, v in res.phase_ms.items()},
                 "phase_share": {k: round(v / tot, 4) for k, v in res.phase_ms.items()},
                 "timing": "library CUDA events on the launching stream around each phase, inside the timed "
                           "region"})
    out = {"workload": name, "ms_per_step": ms, "value": flops / (ms * 1e-3) / 1e9, "unit": UNIT,
           "steps": steps, "warmup": warmup, "flops": flops, "roofline": roof,
           "gpu_launches": sum(r.launches for r in results), "clocks": clk.summary(),
           "result": {"k": res.k, "rounds": res.rounds, "passes": res.passes, "status": res.status,
                      "est_err_rel": res.est_err / res.norm_A if res.norm_A > 0 else 0.0,
                      "gflop_per_id": flops / 1e9}}
    if want_pivots:  # an untimed run that also returns the pivots |U(i,i)|
        pres = step(profile=False, pivots=True)
        out["pivots"] = pres.pivots.double().cpu().numpy()
        out["J_host"] = pres.J.cpu().numpy()
        out["trace"] = list(pres.trace)
    if e2e:
        is8 = hasattr(A, "scale")
        if is8:  # the E4M3 bytes (row stride ld) and the block scales travel
            ldq = A.data.stride(1)
            A_host = torch.empty((n, ldq), dtype=torch.uint8, pin_memory=True)
            A_host.copy_(A.data.view(torch.uint8).t().as_strided((n, ldq), (ldq, 1)))
            S_host = torch.empty(A.scale.t().shape, dtype=torch.float32, pin_memory=True)
            S_host.copy_(A.scale.t())
            A_dev = torch.empty((n, ldq), dtype=torch.uint8, device=dev)
            S_dev = torch.empty(S_host.shape, dtype=torch.float32, device=dev)
            A_in = B.FP8Matrix(A_dev.view(torch.float8_e4m3fn)[:, :m].t(), S_dev.t())
        else:
            A_host = torch.empty((n, m), dtype=A.dtype, pin_memory=True)
            A_host.copy_(A.t())
            A_dev = torch.empty((n, m), dtype=A.dtype, device=dev)
            A_in = A_dev.t()
        X_host = torch.empty((n, kmax), dtype=xdt, pin_memory=True)
        J_host = torch.empty(kmax, dtype=torch.int64, pin_memory=True)

        def e2e_step():
            A_dev.copy_(A_host, non_blocking=True)
            if is8:
                S_dev.copy_(S_host, non_blocking=True)
            r = B.id_adaptive(A_in, tol, block=b, relative=True, k_max=kmax, seed=seed, profile=False,
                              workspace=ws, out=(J, Xbuf), stream=stream, sketch_prec=sprec,
                              predictor=predictor, max_pass_rows=max_pass_rows, omega_kind=okind,
                              blocks_per_pass=blocks_per_pass)
            kk = r.k
            X_host[:, :kk].copy_(Xbuf[:, :kk], non_blocking=True)
            J_host[:kk].copy_(J[:kk], non_blocking=True)
            return r
        for _ in range(max(warmup, 1)):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            r = e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        e_ms = max_over_ranks(e0.elapsed_time(e1) / steps)
        xel = torch.empty((), dtype=xdt).element_size()
        h2d = A_host.numel() * A_host.element_size() + (S_host.numel() * 4 if is8 else 0)
        out["e2e"] = {"value": flops / (e_ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": e_ms,
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": r.k * n * xel + 8 * r.k}
        del A_host, A_dev, X_host, A_in
    out["_res"] = res
    out["_bufs"] = (J, Xbuf)
    del ws
    return out


def public(form):
    """A form's measurements without the in-memory objects."""
    return {k: v for k, v in form.items() if not k.startswith("_") and k not in ("pivots", "J_host", "trace")}


def parity_with_oracle(main, A, name, seed, rounds):
    """The oracle on the first `rounds` rounds of Algorithm 1 over the same full-size
    matrix and the same Gaussian rows; compares the GPU's first rounds*b skeletons
    (bit-exact), the estimates E^(t) and the pivots |U(i,i)|.  Returns the
    cpu_baseline entry and the parity entry."""
    import numpy as np
    A_host64 = host_f64(A)
    v, sec, threads, desc, r = cpu_oracle_sample(A_host64, name, seed=seed, rounds=rounds)
    del A_host64
    kk = r["k"]
    Jg = main["J_host"][:kk]
    nA = main["_res"].norm_A
    tr_o = np.asarray(r["trace"])
    tr_g = np.asarray(main["trace"][: len(tr_o)])
    nt = min(len(tr_o), len(tr_g))
    tr_d = (float(np.max(np.abs(tr_g[:nt] - tr_o[:nt]) / (np.abs(tr_o[:nt]) + 1e-13 * nA))) if nt else 0.0)
    pv_o = np.asarray(r["pivots"][:kk])
    pv_g = main["pivots"][:kk]
    pv_d = float(np.max(np.abs(pv_g - pv_o) / np.maximum(np.abs(pv_o), 1e-300)))
    par = {"oracle_rounds": rounds, "skeletons_compared": int(kk),
           "J_prefix_identical": bool(np.array_equal(Jg, r["J"])),
           "J_prefix_mismatches": int(np.sum(Jg != r["J"])),
           "estimates_compared": int(nt), "estimate_max_rel_diff": tr_d,
           "pivots_max_rel_diff": pv_d,
           "bar": "J bit-exact; E within 1e-9 relative (+1e-13 ||A||_F); pivots within 1e-9 relative"}
    par["pass"] = bool(par["J_prefix_identical"] and tr_d <= 1e-9 and pv_d <= 1e-9)
    cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc}
    return cpu, par


def run_forms(B, dev, main, A, seed, args):
    """The forms the metric compares on the same GB300, each timed with its own
    CUDA events: plain FP64 on the same matrix, the FP32-accurate tensor-core path,
    the BF16 and FP8 mixed-precision paths, the predictor-seeded BF16 path and the
    batched path.  Each carries ms per ID, GFLOP/s, its dominant kernel's
    roofline fraction, e2e, and its error (against the oracle where it can run,
    else evaluated in FP64 on a row sample)."""
    import torch

    forms = {}
    fs, fw = args.form_steps, args.form_warmup
    # plain FP64 on the same A: the metric's baseline
    base = measure_adaptive(B, "adaptive_poly_f64", A, dev, max(1, fs - 1), 1, seed, e2e=False)
    fb = public(base)
    fb["result"]["note"] = ("plain FP64 sketch with the unrounded Gaussian rows; the headline's rows are on "
                            "the grid 2^-11, so the two skeletons are each checked against the oracle, not "
                            "against each other")
    forms["adaptive_poly_f64"] = fb
    plain = fb["value"]
    del base
    torch.cuda.empty_cache()
    # FP32-accurate sketch on the tensor cores: the same matrix rounded to FP32
    A32 = A.t().float().t()
    f = measure_adaptive(B, "adaptive_poly_f32emu", A32, dev, fs, fw, seed)
    forms["adaptive_poly_f32emu"] = public(f)
    forms["adaptive_poly_f32emu"]["config_note"] = "the headline's FP64 matrix rounded to FP32"
    del f, A32
    torch.cuda.empty_cache()
    # mixed precision: BF16 A (100000 x 20000), tolerance 3e-2 (stops just after the signal)
    Ab = make_input("mixed_bf16_tol3e-2", dev)
    f = measure_adaptive(B, "mixed_bf16_tol3e-2", Ab, dev, fs + 2, fw, seed)
    r = f["_res"]
    f["result"]["rel_err_sampled"] = sampled_rel_error(Ab, r.J, r.X, r.norm_A)
    fpub = public(f)
    forms["mixed_bf16_tol3e-2"] = fpub
    # the same run seeded by the learned rank predictor
    from paper_2310_09417_gb300 import predictor as P
    params = P.load(os.path.join(ROOT, "paper_2310_09417_gb300", "data", "rank_predictor.f32"), device=dev)
    g = measure_adaptive(B, "mixed_bf16_tol3e-2", Ab, dev, fs + 2, fw, seed, predictor=params, max_pass_rows=4096)
    gr = g["_res"]
    gp = public(g)
    gp["result"]["identical_to_plain"] = bool(gr.k == r.k and torch.equal(g["_bufs"][0][:gr.k], f["_bufs"][0][:r.k])
                                              and torch.equal(g["_bufs"][1][:, :gr.k], f["_bufs"][1][:, :r.k]))
    gp["result"]["passes_plain"] = r.passes
    gp["result"]["ms_saved_vs_plain"] = fpub["ms_per_step"] - gp["ms_per_step"]
    forms["mixed_bf16_tol3e-2_predictor"] = gp
    del f, g
    torch.cuda.empty_cache()
    # FP8 E4M3 storage with per-128-row block scales, tolerance 1e-3
    A8 = B.quantize_fp8(Ab, pow2=True)
    del Ab
    torch.cuda.empty_cache()
    f = measure_adaptive(B, "mixed_fp8", A8, dev, fs, fw, seed)
    forms["mixed_fp8"] = public(f)
    del f, A8
    torch.cuda.empty_cache()
    # batched: 4096 kernel blocks in one persistent launch per step
    forms["batched_kernel_f64"] = measure_batched(B, "batched_kernel_f64", dev, fs, fw, seed, errors=True)
    for k, v in forms.items():
        v["gflops_over_plain_f64"] = v["value"] / plain
        if k.startswith("adaptive_poly"):
            v["speedup_over_plain_f64_same_matrix"] = forms["adaptive_poly_f64"]["ms_per_step"] / v["ms_per_step"]
    return forms


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-rounds", type=int, default=0, help="oracle rounds per sample (0: sized to ~4 s)")
    ap.add_argument("--parity-rounds", type=int, default=7,
                    help="oracle rounds of the full-size parity check in the cpu_baseline leg")
    ap.add_argument("--forms", default="auto", choices=["auto", "all", "none"],
                    help="time the other forms the metric compares (auto: with the default workload on one GPU)")
    ap.add_argument("--form-steps", type=int, default=3)
    ap.add_argument("--blocks-per-pass", type=int, default=0,
                    help="sketch blocks per pass over A (0: the library's choice); J, X, k do not depend on it")
    ap.add_argument("--form-warmup", type=int, default=2)
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        return over_ranks(x, "max", world, dev)

    def sum_over_ranks(x: float) -> float:
        return over_ranks(x, "sum", world, dev)

    from paper_2310_09417_gb300 import binding as B
    from paper_2310_09417_gb300 import build
    build.build()
    B.load()

    name = args.workload
    if WORKLOADS[name][2] in ("kernel", "fixed"):
        (run_batched if WORKLOADS[name][2] == "kernel" else run_fixed)(args, rank, world, dev, barrier,
                                                                        max_over_ranks, sum_over_ranks)
        if world > 1:
            dist.destroy_process_group()
        return
    m, n, kind, kw, dt, tol, b = WORKLOADS[name]
    A = make_input(name, dev)
    seed = 2310_09417 + 100 * rank
    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    main_r = measure_adaptive(B, name, A, dev, args.steps, args.warmup, seed, e2e=not args.no_e2e,
                              max_over_ranks=max_over_ranks, barrier=barrier, want_pivots=want_cpu,
                              blocks_per_pass=args.blocks_per_pass)
    res = main_r["_res"]
    # whole job: every rank's ID (own seed) over the slowest rank's time
    flops_all = sum_over_ranks(main_r["flops"])
    value = flops_all / (main_r["ms_per_step"] * 1e-3) / 1e9
    if main_r.get("e2e"):
        main_r["e2e"]["value"] = flops_all / (main_r["e2e"]["ms_per_step"] * 1e-3) / 1e9

    cpu, parity = None, None
    if want_cpu:
        rounds = args.parity_rounds if kind in ("poly", "step") else ref_rounds(args, name)
        cpu, parity = parity_with_oracle(main_r, A, name, seed, rounds)

    forms = None
    if args.forms == "all" or (args.forms == "auto" and name == DEFAULT_WORKLOAD and world == 1):
        forms = run_forms(B, dev, main_r, A, seed, args)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": main_r["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_LABEL[dt], "data": "synthetic",
                "config": config_dict(name, res), "roofline": main_r["roofline"], "cpu_baseline": cpu,
                "e2e": main_r.get("e2e"), "gpu_launches": main_r["gpu_launches"], "clocks": main_r["clocks"],
                "result": main_r["result"], "parity": parity}
        if forms is not None:
            line["forms"] = forms
            base = forms["adaptive_poly_f64"]
            line["plain_f64_same_matrix"] = {"ms_per_step": base["ms_per_step"], "value": base["value"],
                                             "k": base["result"]["k"],
                                             "speedup": base["ms_per_step"] / main_r["ms_per_step"]}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
