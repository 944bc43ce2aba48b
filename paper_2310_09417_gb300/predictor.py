"""Learned rank predictor for the adaptive ID: data, training and evaluation.

The network (see include/randid.h, "learned rank predictor") maps features of
the first sketch block -- the leading LUPP pivot magnitudes, which track the
spectrum (Remark 1 of arXiv:2310.09417) -- plus log m, log n and log tol to the
log2 of the rank that Algorithm 1 returns.  id_adaptive uses the prediction
only to sketch the blocks up to the predicted rank in fewer passes over A; the
plain loop still performs every stop test, so J, X and k do not change.

Everything numeric runs in the CUDA library: labels come from runs of the
method (id_batched, which also returns the pivots), features from
id_rank_features, training from id_mlp_loss_grad and id_mlp_adam.  PyTorch only
holds the tensors.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np
import torch

from . import binding as B

FAMILIES = ("exponential", "polynomial", "step", "kernel")


# ---------------------------------------------------------------- problems
def _spectrum(family, n, rng):
    j = np.arange(n, dtype=np.float64)
    if family == "exponential":
        return np.exp(-j / (n * 10 ** rng.uniform(-2.0, -0.5)))
    if family == "polynomial":
        return (1.0 + j) ** (-rng.uniform(0.75, 3.0))
    if family == "step":
        r = int(n * rng.uniform(0.05, 0.6))
        s = np.full(n, 10 ** rng.uniform(-12, -3))
        s[:r] = 1.0
        return s
    raise ValueError(family)


def generate_problems(count, families, seed, device, dims=(256, 2048), dtype=torch.float64):
    """`count` seeded test matrices (column-major CUDA tensors) drawn from the
    given families with n log-uniform in `dims` and m = n x U[1, 3]."""
    rng = np.random.default_rng(seed)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    out = []
    for i in range(count):
        fam = families[i % len(families)]
        n = int(round(math.exp(rng.uniform(math.log(dims[0]), math.log(dims[1])))))
        m = int(n * rng.uniform(1.0, 3.0))
        if fam == "kernel":
            h = rng.uniform(0.1, 0.6)
            sep = rng.uniform(0.0, 2.0)
            X = torch.rand(m, 3, generator=g, device=device, dtype=torch.float64)
            Y = torch.rand(n, 3, generator=g, device=device, dtype=torch.float64)
            Y[:, 0] += sep
            At = torch.exp(-torch.cdist(Y, X) ** 2 / (h * h))
        else:
            s = torch.as_tensor(_spectrum(fam, n, rng), device=device)
            U, _ = torch.linalg.qr(torch.randn(m, n, generator=g, device=device, dtype=torch.float32))
            V, _ = torch.linalg.qr(torch.randn(n, n, generator=g, device=device, dtype=torch.float32))
            At = (V.double() * s) @ U.double().T
        out.append((At.to(dtype).t(), fam))
    return out


# ---------------------------------------------------------------- labels and features
def label(problems, tols, seed=1, block=32):
    """Run the method on every problem at every relative tolerance (one batched
    launch per tolerance).  Returns features (N x 35, CUDA float32), targets
    log2 k (N, CUDA float32) and a record per sample."""
    feats, targs, recs = [], [], []
    As = [A for A, _ in problems]
    for tol in tols:
        res = B.id_batched(As, tol, block=block, seed=seed, pivots=True)
        for (A, fam), r in zip(problems, res):
            if r.status < 0 or r.k < 1:
                continue
            m, n = A.shape
            feats.append(B.rank_features(r.pivots[:32].contiguous(), m, n, tol))
            targs.append(math.log2(r.k))
            recs.append({"family": fam, "m": m, "n": n, "tol": tol, "k": r.k})
    x = torch.stack(feats)
    y = torch.tensor(targs, dtype=torch.float32, device=x.device)
    return x, y, recs


# ---------------------------------------------------------------- labels at scale
def sketch_equivalent(family, n, rng, g, device):
    """A matrix whose sketches have the distribution of those of an m x n matrix
    A = U diag(s) V^T (U with orthonormal columns, Haar): Omega A = (Omega U)
    diag(s) V^T and Omega U is Gaussian, so the n x n matrix diag(s) V^T (with
    N(0,1) sketch rows of length n) gives the same estimates, ranks and pivots in
    distribution without forming A.  V comes from an FP32 QR of a Gaussian
    matrix; the matrix is stored in FP64, column-major."""
    s = torch.as_tensor(_spectrum(family, n, rng), device=device)
    V, _ = torch.linalg.qr(torch.randn(n, n, generator=g, device=device, dtype=torch.float32))
    At = (V.double() * s).contiguous()  # (A')^T = V diag(s), row-major: A' column-major
    del V
    return At.t()


def ranks_from_trace(trace, norm_a, tols, block, cap):
    """The rank Algorithm 1 returns at each relative tolerance, from the estimates
    E^(t) of one run at a tighter tolerance: the loop stops at the first t with
    E^(t) <= tol ||A||_F and returns k = t b (the estimates do not depend on tol);
    a tolerance the trace never meets gives the rank cap."""
    out = []
    for tol in tols:
        k = cap
        for t, e in enumerate(trace, start=1):
            if e <= tol * norm_a:
                k = min(t * block, cap)
                break
        out.append(k)
    return out


def label_large(count, families, seed, device="cuda", dims=(512, 20000), tols=None, block=64,
                log_every=0):
    """`count` problems with n log-uniform in `dims`, m = n U[1, 3] (recorded for the
    features; spectral families run on the sketch-equivalent n x n matrix, kernel
    blocks on the m x n matrix itself), one run of the
    FP64-accurate tensor-core path at the tightest tolerance each; labels for every
    tolerance from its estimates.  Returns features, targets log2 k and records."""
    tols = tols or [10.0 ** -e for e in (2, 3, 4, 5, 6, 7, 8, 9)]
    rng = np.random.default_rng(seed)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    feats, targs, recs = [], [], []
    t0 = time.perf_counter()
    for i in range(count):
        fam = families[i % len(families)]
        n = int(round(math.exp(rng.uniform(math.log(dims[0]), math.log(dims[1])))))
        m = int(n * rng.uniform(1.0, 3.0))
        if fam == "kernel":  # a Gaussian kernel block between two point clouds, formed on the device
            h = rng.uniform(0.1, 0.6)
            sep = rng.uniform(0.0, 2.0)
            X = torch.rand(m, 3, generator=g, device=device, dtype=torch.float64)
            Y = torch.rand(n, 3, generator=g, device=device, dtype=torch.float64)
            Y[:, 0] += sep
            A = torch.exp(-torch.cdist(Y, X) ** 2 / (h * h)).t()
            del X, Y
        else:
            A = sketch_equivalent(fam, n, rng, g, device)
        r = B.id_adaptive(A, min(tols), block=block, seed=seed + i, pivots=True, trace_cap=n // block + 2,
                          sketch_prec=B.F64_EMU)
        n_cap = min(A.shape)
        ks = ranks_from_trace(r.trace, r.norm_A, tols, block, n_cap)
        piv = r.pivots[:32].contiguous()
        for tol, k in zip(tols, ks):
            feats.append(B.rank_features(piv, m, n, tol))
            targs.append(math.log2(k))
            recs.append({"family": fam, "m": m, "n": n, "tol": tol, "k": k})
        del A, r
        if log_every and (i + 1) % log_every == 0:
            print("labelled %d / %d problems (%.0f s)" % (i + 1, count, time.perf_counter() - t0), flush=True)
    x = torch.stack(feats)
    y = torch.tensor(targs, dtype=torch.float32, device=x.device)
    return x, y, recs


def tall_bf16(D, tall):
    """The (tall n) x n BF16 matrix [D; D; ...; D] / sqrt(tall), column-major with
    an even leading dimension: its Gram matrix is D^T D, so it has D's singular
    values and right singular vectors (left ones [U; ...; U] / sqrt(tall), again
    orthonormal), and its Gaussian sketches have the distribution of D's."""
    n = D.shape[0]
    m = tall * n
    ld = -(-m // 8) * 8
    buf = torch.zeros((n, ld), dtype=torch.bfloat16, device=D.device)
    Dt = (D * (1.0 / math.sqrt(tall))).t().to(torch.bfloat16)
    for c in range(tall):
        buf[:, c * n:(c + 1) * n] = Dt
    return buf[:, :m].t()


def evaluate_large(params, count, family, seed, tols=(1e-4, 1e-8), device="cuda", dims=(4096, 20000), block=64,
                   max_pass_rows=4096, precision="f64emu", tall=1):
    """Held-out evaluation at scale: plain loop vs predictor-seeded loop on the
    same matrices, wall time by CUDA events.  precision "f64emu": FP64 A on the
    FP64-accurate tensor-core path (one CTA per 64 sketch rows and column tile,
    so a pass of many blocks costs about as much as as many passes of one);
    "bf16": the matrix rounded to BF16 with the FP32 LU, whose sketch reads A once
    per pass however many blocks the pass holds (tolerances above BF16's 2^-8),
    stacked `tall` times (tall_bf16) to the shape of the 100000 x 20000
    configuration.  The seeded loop saves passes over A, not rounds: each block is
    still factored on its own, and the plain loop's automatic passes of eight blocks
    already read A once per eight blocks."""
    if precision not in ("f64emu", "bf16"):
        raise ValueError("precision must be 'f64emu' or 'bf16'")
    rng = np.random.default_rng(seed)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    rows = {t: [] for t in tols}
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(dims[0]), math.log(dims[1])))))
        A = sketch_equivalent(family, n, rng, g, device)
        if precision == "bf16":
            A = tall_bf16(A, tall)
        for tol in tols:
            kw = dict(block=block, seed=seed + i)
            if precision == "f64emu":
                kw["sketch_prec"] = B.F64_EMU
            B.id_adaptive(A, tol, **kw)  # warm-up (workspace, tuned launches)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            a = B.id_adaptive(A, tol, **kw)
            e1.record()
            s = B.id_adaptive(A, tol, predictor=params, max_pass_rows=max_pass_rows, **kw)
            e2.record()
            torch.cuda.synchronize()
            same = a.k == s.k and torch.equal(a.J, s.J) and bool(torch.equal(a.X, s.X))
            thr = tol * a.norm_A
            rows[tol].append({"family": family, "n": n, "k": a.k, "passes_plain": a.passes,
                              "passes_seeded": s.passes, "identical": same,
                              "ms_plain": e0.elapsed_time(e1), "ms_seeded": e1.elapsed_time(e2),
                              "miss_plain": a.status & B.WARN_TOL_NOT_MET != 0 and a.est_err > thr,
                              "miss_seeded": s.status & B.WARN_TOL_NOT_MET != 0 and s.est_err > thr})
        del A
    return rows


def run_large(out_dir=None, train_count=2500, eval_count=12, held_out="step", seed=31, steps=3000,
              device="cuda", log_every=100):
    """The predictor at scale: 2500 problems x 8 tolerances = 20000 labelled runs
    of the method over n in [512, 20000] (three families; `held_out` set aside),
    training by the library's kernels, and the held-out evaluation at scale."""
    train_fams = [f for f in FAMILIES if f != held_out]
    t0 = time.perf_counter()
    x, y, recs = label_large(train_count, train_fams, seed, device, log_every=log_every)
    t_label = time.perf_counter() - t0
    t0 = time.perf_counter()
    params, hist = train(x, y, steps=steps, log_every=max(1, steps // 10))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    pred = B.mlp_forward(params, x)
    rmse = float(torch.sqrt(torch.mean((pred - y) ** 2)).item())
    report = {"train_samples": int(x.shape[0]), "train_problems": train_count, "dims": [512, 20000],
              "families_train": train_fams, "family_held_out": held_out, "label_s": t_label, "train_s": t_train,
              "rmse_log2k_train": rmse, "loss_history": hist}
    ev = evaluate_large(params, eval_count, held_out, seed + 7, device=device)
    for tol, rows in ev.items():
        report["held_out_tol_%g" % tol] = summarize(rows)
    if out_dir:
        os.makedirs(out_dir, exist_ok=True)
        save(params, os.path.join(out_dir, "rank_predictor.f32"), {"held_out": held_out, "dims": [512, 20000]})
        with open(os.path.join(out_dir, "predictor_report.json"), "w") as f:
            json.dump(report, f, indent=1)
    return params, report


# ---------------------------------------------------------------- training
def init_params(x, y, seed=0):
    """Xavier-scaled weights and the standardisation of the training data."""
    n = B.mlp_param_count()
    g = torch.Generator(device=x.device)
    g.manual_seed(seed)
    p = torch.zeros(n, dtype=torch.float32, device=x.device)
    In, H = B.MLP_IN, B.MLP_HIDDEN
    off = 0
    for rows, cols in ((H, In), (H, 1), (H, H), (H, 1), (1, H), (1, 1)):
        size = rows * cols
        if cols > 1 or rows == 1 and cols == H:
            fan = cols
            p[off:off + size] = torch.randn(size, generator=g, device=x.device) / math.sqrt(fan)
        off += size
    mu = x.mean(dim=0)
    sd = x.std(dim=0).clamp_min(1e-3)
    p[off:off + In] = mu
    p[off + In:off + 2 * In] = sd
    p[off + 2 * In] = y.mean()
    p[off + 2 * In + 1] = y.std().clamp_min(1e-3)
    return p


def train(x, y, steps=1500, lr=2e-3, batch=512, seed=0, log_every=0):
    """Adam on the mean squared error of log2 k; returns (params, loss history)."""
    p = init_params(x, y, seed)
    nt = B.MLP_TRAINABLE
    m1 = torch.zeros(nt, dtype=torch.float32, device=x.device)
    m2 = torch.zeros(nt, dtype=torch.float32, device=x.device)
    grad = torch.empty(nt, dtype=torch.float32, device=x.device)
    g = torch.Generator(device=x.device)
    g.manual_seed(seed + 1)
    hist = []
    N = x.shape[0]
    for step in range(1, steps + 1):
        idx = torch.randint(0, N, (min(batch, N),), generator=g, device=x.device)
        loss, _ = B.mlp_loss_grad(p, x[idx], y[idx], grad)
        B.mlp_adam(p, grad, m1, m2, step, lr)
        if log_every and step % log_every == 0:
            hist.append((step, float(loss.item())))
    return p, hist


def save(params, path, meta=None):
    """Parameters as raw little-endian float32 plus a JSON side file."""
    params.detach().cpu().numpy().astype("<f4").tofile(path)
    with open(path + ".json", "w") as f:
        json.dump(dict(meta or {}, count=int(params.numel()), layout="see include/randid.h"), f, indent=1)


def load(path, device="cuda"):
    a = np.fromfile(path, dtype="<f4")
    return torch.from_numpy(a).to(device)


# ---------------------------------------------------------------- evaluation
def evaluate(params, problems, tol, block=64, max_pass_rows=4096, seed=3):
    """Plain loop vs predictor-seeded loop on each problem: passes over A, wall
    time, whether the results are identical, and the tolerance-miss rate (the
    estimate at the returned rank above tol while k < min(m, n))."""
    rows = []
    for A, fam in problems:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        a = B.id_adaptive(A, tol, block=block, seed=seed)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        s = B.id_adaptive(A, tol, block=block, seed=seed, predictor=params, max_pass_rows=max_pass_rows)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        same = a.k == s.k and torch.equal(a.J, s.J) and bool(torch.equal(a.X, s.X))
        thr = tol * a.norm_A
        rows.append({"family": fam, "m": A.shape[0], "n": A.shape[1], "k": a.k,
                     "passes_plain": a.passes, "passes_seeded": s.passes, "identical": same,
                     "ms_plain": 1e3 * (t1 - t0), "ms_seeded": 1e3 * (t2 - t1),
                     "miss_plain": a.status & B.WARN_TOL_NOT_MET != 0 and a.est_err > thr,
                     "miss_seeded": s.status & B.WARN_TOL_NOT_MET != 0 and s.est_err > thr})
    return rows


def summarize(rows):
    n = len(rows)
    pp = sum(r["passes_plain"] for r in rows)
    ps = sum(r["passes_seeded"] for r in rows)
    return {"problems": n, "passes_plain": pp, "passes_seeded": ps,
            "passes_saved_frac": 1.0 - ps / max(pp, 1),
            "all_identical": all(r["identical"] for r in rows),
            "miss_rate_plain": sum(r["miss_plain"] for r in rows) / max(n, 1),
            "miss_rate_seeded": sum(r["miss_seeded"] for r in rows) / max(n, 1),
            "ms_plain": sum(r["ms_plain"] for r in rows), "ms_seeded": sum(r["ms_seeded"] for r in rows)}


def run(out_dir=None, train_count=480, eval_count=40, held_out="step", seed=11, device="cuda", steps=1500):
    """Train on three families, evaluate on the held-out fourth; returns a report."""
    train_fams = [f for f in FAMILIES if f != held_out]
    tols = [10.0 ** -e for e in (2, 3, 4, 5, 6, 7, 8, 9, 10)]
    t0 = time.perf_counter()
    probs = generate_problems(train_count, train_fams, seed, device)
    x, y, recs = label(probs, tols)
    del probs
    t_label = time.perf_counter() - t0
    t0 = time.perf_counter()
    params, hist = train(x, y, steps=steps, log_every=max(1, steps // 10))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    pred = B.mlp_forward(params, x)
    rmse_train = float(torch.sqrt(torch.mean((pred - y) ** 2)).item())
    held = generate_problems(eval_count, [held_out], seed + 1, device)
    report = {"train_samples": int(x.shape[0]), "families_train": train_fams, "family_held_out": held_out,
              "label_s": t_label, "train_s": t_train, "rmse_log2k_train": rmse_train, "loss_history": hist}
    for tol in (1e-4, 1e-8):
        rows = evaluate(params, held, tol)
        report["held_out_tol_%g" % tol] = summarize(rows)
    if out_dir:
        os.makedirs(out_dir, exist_ok=True)
        save(params, os.path.join(out_dir, "rank_predictor.f32"), {"held_out": held_out})
        with open(os.path.join(out_dir, "predictor_report.json"), "w") as f:
            json.dump(report, f, indent=1)
    return params, report


if __name__ == "__main__":
    import sys
    out = sys.argv[1] if len(sys.argv) > 1 else None
    if len(sys.argv) > 2 and sys.argv[2] == "large":
        _, rep = run_large(out_dir=out)
    else:
        _, rep = run(out_dir=out)
    print(json.dumps({k: v for k, v in rep.items() if k != "loss_history"}, indent=1))
