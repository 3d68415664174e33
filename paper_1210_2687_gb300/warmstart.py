"""Training and evaluation of the learned warm start (include/admm_warmstart.h).

The network is trained on the GPU by the library's own kernels, on solutions
that this ADMM itself computes: for each synthetic TV problem the solver runs
from u0 = d0 = 0 to rel-x < 1e-5 and its (x*, d1*, d2*) is the target. At
solve time the prediction feeds admm_deconv_warm_start and the solver runs
to the same stop rule as from a cold start (Theorem 1: any start converges),
so the plain ADMM still decides the result.

    python -m paper_1210_2687_gb300.warmstart train        # writes weights/warmstart_tv.npz
    python -m paper_1210_2687_gb300.warmstart eval --weights weights.npz --count 64
    python -m paper_1210_2687_gb300.warmstart export       # weights/warmstart_tv.bin for admm_warmstart_load

Training problems (256 x 256): an image from the piecewise-constant law
(20 rectangles / disks) or the textured law with probability 1/2; a kernel
from the batched workload's law (box, Gaussian or motion, side 5..25);
missing fraction U[0, 0.5] inside the valid region; BSNR 40 dB. Evaluation
problems (512 x 512): the piecewise-constant law scaled to 512 (disk radius
up to 128), 9 x 9 box, valid region only, BSNR 40 dB. Both use lambda = 1e-3
with mu2 = 10 lambda, mu1 = 3 mu2: the network sees no lambda, so it is
trained for the weight it is evaluated with.

Argument marshalling and data handling only: every step of the solver and
of the network runs in the library's kernels.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

import numpy as np

from . import Cnn, Plan, admm_deconv_get_state, admm_warmstart_load, solve_batch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth as S  # noqa: E402  (seeded input generators)

LAM = 1e-3
TOL = 1e-5
MAX_ITERS = 5000
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "warmstart_tv.npz")
WEIGHTS_BIN = os.path.splitext(WEIGHTS)[0] + ".bin"


def mu():
    return S.default_mu(LAM)


# --------------------------------------------------------------------------
# problems
# --------------------------------------------------------------------------
def training_problem(seed: int, size: int = 256):
    g = S.rng(seed)
    if g.uniform() < 0.5:
        x = S.shapes_image(size, size, g, 20, rmax=size / 4.0)
    else:
        x = S.textured_image(size, size, g)
    psf, _ = S.config4_psf(g)
    missing = float(g.uniform(0.0, 0.5))
    keep = (g.uniform(0.0, 1.0, size=(size, size)) >= missing).astype(np.uint8)
    ybar, mask, _ = S.observe(x, psf, keep, 40.0, g, fast=True)
    return ybar.astype(np.float32), mask, psf


def eval_problem(seed: int, size: int = 512):
    g = S.rng(seed)
    x = S.shapes_image(size, size, g, 20, rmax=16.0 * size / 64.0)
    psf = S.psf_box(9)
    ybar, mask, _ = S.observe(x, psf, None, 40.0, g, fast=True)
    return x, ybar.astype(np.float32), mask, psf


def _gen(args):
    kind, seed, size = args
    return training_problem(seed, size) if kind == "train" else eval_problem(seed, size)


def generate(kind: str, seeds, size: int, procs: int | None = None):
    """Problems for `seeds`, drawn in a spawn pool (safe before or after CUDA
    is initialised in this process)."""
    procs = procs or min(16, os.cpu_count() or 1)
    jobs = [(kind, int(s), size) for s in seeds]
    main = sys.modules.get("__main__")
    spawnable = getattr(main, "__spec__", None) is not None or os.path.exists(getattr(main, "__file__", "") or "")
    if procs <= 1 or len(jobs) < 8 or not spawnable:
        return [_gen(j) for j in jobs]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_gen, jobs, chunksize=max(1, len(jobs) // (4 * procs)))


def isnr(x_true, ybar, x_hat, region):
    r = region.astype(bool)
    return 10.0 * math.log10(np.sum((x_true[r] - ybar[r]) ** 2) / np.sum((x_true[r] - x_hat[r]) ** 2))


# --------------------------------------------------------------------------
# solver-generated targets
# --------------------------------------------------------------------------
def solve_targets(probs, torch, chunk: int = 512):
    """Cold solves of every problem; returns device tensors ybar (N, H, W),
    mask (N, H, W), state (N, H, W, 4) = (x*, d1*, d2h*, d2v*), and the mean
    iteration count."""
    N = len(probs)
    H, W = probs[0][0].shape
    n = H * W
    mu1, mu2 = mu()
    ybar = torch.empty((N, H, W), dtype=torch.float32, device="cuda")
    mask = torch.empty((N, H, W), dtype=torch.uint8, device="cuda")
    state = torch.empty((N, H, W, 4), dtype=torch.float32, device="cuda")
    iters = []
    for c0 in range(0, N, chunk):
        part = probs[c0:c0 + chunk]
        plans = [Plan(H, W, psf, LAM, mu1, mu2, "tv", stop="rel_x", tol=TOL, max_iters=MAX_ITERS, check_every=10)
                 for _, _, psf in part]
        for j, (y, m, _) in enumerate(part):
            ybar[c0 + j].copy_(torch.from_numpy(y))
            mask[c0 + j].copy_(torch.from_numpy(m))
        xs = [state[c0 + j, :, :, 0].clone() for j in range(len(part))]
        res = solve_batch(plans, [ybar[c0 + j] for j in range(len(part))], [mask[c0 + j] for j in range(len(part))],
                          xs)
        d = torch.empty(3 * n, dtype=torch.float32, device="cuda")
        for j, pl in enumerate(plans):
            admm_deconv_get_state(pl.handle, d.data_ptr())
            state[c0 + j, :, :, 0] = xs[j]
            state[c0 + j, :, :, 1] = d[:n].view(H, W)
            state[c0 + j, :, :, 2:] = d[n:].view(H, W, 2)
            pl.close()
        iters += [r.iters for r in res]
    torch.cuda.synchronize()
    return ybar, mask, state, float(np.mean(iters))


# --------------------------------------------------------------------------
# training
# --------------------------------------------------------------------------
def prepare(count=20000, size=256, seed=0, log=print):
    """Training set: generated problems, their cold solutions as targets
    (x*, d1* / s1, d2h* / s2, d2v* / s2) on the device, and the scales."""
    import torch
    t0 = time.time()
    probs = generate("train", range(10_000_000 + seed, 10_000_000 + seed + count), size)
    t_gen = time.time() - t0
    t0 = time.time()
    ybar, mask, state, mean_it = solve_targets(probs, torch)
    del probs
    t_solve = time.time() - t0
    log(json.dumps({"generated": count, "gen_s": t_gen, "solve_s": t_solve, "mean_target_iters": mean_it}))
    mu1, mu2 = mu()
    # output scales: x as is, d2 by its bound lambda / mu2, d1 by its RMS
    s1 = float(torch.sqrt(torch.mean(state[..., 1].double() ** 2)).item())
    scales = np.array([1.0, max(s1, 1e-6), LAM / mu2, 0.0], dtype=np.float32)
    state[..., 1] /= scales[1]
    state[..., 2:] /= scales[2]
    meta = {"count": count, "size": size, "seed": seed, "lam": LAM, "mu1": mu1, "mu2": mu2,
            "mean_target_iters": mean_it, "gen_s": t_gen, "solve_s": t_solve}
    return {"ybar": ybar, "mask": mask, "target": state, "scales": scales, "meta": meta}


def fit(data, epochs=4, batch=16, lr=1e-3, cw=(1.0, 1.0, 1.0, 1.0), seed=0, log=print):
    """Adam with a cosine step size from lr to 1e-5 over all steps."""
    import torch
    ybar, mask, target = data["ybar"], data["mask"], data["target"]
    N = ybar.shape[0]
    H, W = ybar.shape[1:]
    rng = np.random.Generator(np.random.PCG64(seed))
    net = Cnn(batch * H * W, training=True)
    net.set_params(_init_params(seed))
    steps = epochs * (N // batch)
    t0 = time.time()
    step = 0
    hist = []
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(N)).cuda()
        for b0 in range(0, N - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            yb, mb, tb = ybar[idx].contiguous(), mask[idx].contiguous(), target[idx].contiguous()
            lr_t = 1e-5 + 0.5 * (lr - 1e-5) * (1.0 + math.cos(math.pi * step / max(1, steps)))
            want = step % 500 == 0 or step == steps - 1
            L = net.train_step(yb, mb, tb, cw, lr_t, want_loss=want)
            if want:
                hist.append((step, L))
                log(json.dumps({"step": step, "epoch": ep, "loss": L, "lr": lr_t}))
            step += 1
    torch.cuda.synchronize()
    meta = dict(data["meta"], epochs=epochs, batch=batch, lr=lr, cw=list(cw), train_s=time.time() - t0,
                steps=steps, loss_history=hist)
    params = net.get_params()
    net.close()
    return params, meta


def train(count=20000, epochs=4, batch=16, lr=1e-3, cw=(1.0, 1.0, 1.0, 1.0), size=256, seed=0, log=print):
    data = prepare(count, size, seed, log)
    params, meta = fit(data, epochs, batch, lr, cw, seed, log)
    return params, data["scales"], meta


def _init_params(seed):
    """He-normal weights, zero biases, last layer scaled by 0.1."""
    g = np.random.Generator(np.random.PCG64(seed + 7))
    out = []
    shapes = [(32, 2)] + [(32, 32)] * 6 + [(4, 32)]
    for li, (co, ci) in enumerate(shapes):
        std = math.sqrt(2.0 / (9.0 * ci)) * (0.1 if li == len(shapes) - 1 else 1.0)
        out.append((g.standard_normal((co, ci, 3, 3)) * std).ravel())
        out.append(np.zeros(co))
    return np.concatenate(out).astype(np.float32)


def save(path, params, scales, meta):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    np.savez(path, params=params.astype(np.float32), scales=scales.astype(np.float32),
             meta=np.array(json.dumps(meta)))


def load(path=WEIGHTS):
    z = np.load(path)
    return z["params"].astype(np.float32), z["scales"].astype(np.float32), json.loads(str(z["meta"]))


def export_binary(params, scales, path=WEIGHTS_BIN):
    """The weights file of admm_warmstart_load (include/admm_deconv.h): magic
    "ADMMCNN1", int32 version 1, int32 0, int64 parameter count, float32
    scales[4], float32 parameters; little-endian."""
    params = np.ascontiguousarray(params, dtype="<f4")
    scales = np.ascontiguousarray(np.resize(np.asarray(scales, dtype="<f4"), 4))
    with open(path, "wb") as f:
        f.write(b"ADMMCNN1")
        f.write(np.array([1, 0], dtype="<i4").tobytes())
        f.write(np.array([params.size], dtype="<i8").tobytes())
        f.write(scales.tobytes())
        f.write(params.tobytes())
    return path


# --------------------------------------------------------------------------
# evaluation: cold vs warm start to the same stop rule
# --------------------------------------------------------------------------
def evaluate(params, scales, count=64, size=512, seed=0, check_every=1, probs=None, api_weights=None):
    import torch
    if probs is None:
        probs = generate("eval", range(20_000_000 + seed, 20_000_000 + seed + count), size)
    count = len(probs)
    H = W = size
    n = H * W
    mu1, mu2 = mu()
    ys = [torch.from_numpy(p[1]).cuda() for p in probs]
    ms = [torch.from_numpy(p[2]).cuda() for p in probs]
    plans = [Plan(H, W, p[3], LAM, mu1, mu2, "tv", stop="rel_x", tol=TOL, max_iters=MAX_ITERS,
                  check_every=check_every) for p in probs]
    xc = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in probs]
    xw = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in probs]
    net = Cnn(min(count, 16) * n)
    net.set_params(params)
    yb = torch.stack(ys)
    mb = torch.stack(ms)
    x0 = torch.empty((count, H, W), dtype=torch.float32, device="cuda")
    d0 = torch.empty((count, 3 * n), dtype=torch.float32, device="cuda")
    # warm-up of both paths (graphs, attributes), then timed runs
    solve_batch(plans, ys, ms, xc)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    e[0].record()
    rc = solve_batch(plans, ys, ms, xc)
    e[1].record()
    torch.cuda.synchronize()
    dcold = torch.empty((count, 3 * n), dtype=torch.float32, device="cuda")
    for j, pl in enumerate(plans):
        admm_deconv_get_state(pl.handle, dcold[j].data_ptr())
    e[4].record()
    for c0 in range(0, count, 16):
        net.predict_start(yb[c0:c0 + 16], mb[c0:c0 + 16], scales, x0[c0:c0 + 16], d0[c0:c0 + 16])
    for j, pl in enumerate(plans):
        pl.warm_start(x0[j], d0[j])
    e[2].record()
    rw = solve_batch(plans, ys, ms, xw)
    e[3].record()
    torch.cuda.synchronize()
    api = None
    if api_weights is not None:
        # the same warm start through the library's own path: the weights file
        # loaded by admm_warmstart_load, the network run inside solve_batch
        xa = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in probs]
        admm_warmstart_load(api_weights)
        try:
            solve_batch(plans, ys, ms, xa, use_warmstart=True)   # warm-up (the network's buffers)
            ea = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ea[0].record()
            ra = solve_batch(plans, ys, ms, xa, use_warmstart=True)
            ea[1].record()
            torch.cuda.synchronize()
        finally:
            admm_warmstart_load(None)
        api = {"images_per_s": count / (ea[0].elapsed_time(ea[1]) * 1e-3),
               "iters_mean": float(np.mean([r.iters for r in ra])),
               "x_equal_to_manual_start": all(bool(torch.equal(a, b)) for a, b in zip(xa, xw))}
    # prediction error against the cold solution, relative L2 per field
    xs = torch.stack(xc)

    def rel(a, b):
        return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))

    pred_err = {"x": rel(x0, xs), "d1": rel(d0[:, :n], dcold[:, :n]), "d2": rel(d0[:, n:], dcold[:, n:])}
    cold_s = e[0].elapsed_time(e[1]) * 1e-3
    warm_s = e[2].elapsed_time(e[3]) * 1e-3
    cnn_s = e[4].elapsed_time(e[2]) * 1e-3
    ic = np.array([r.iters for r in rc], dtype=np.float64)
    iw = np.array([r.iters for r in rw], dtype=np.float64)
    dis = []
    for j, p in enumerate(probs):
        vm = S.valid_mask(H, W, *p[3].shape)
        a = isnr(p[0], p[1].astype(np.float64), xc[j].cpu().numpy().astype(np.float64), vm)
        b = isnr(p[0], p[1].astype(np.float64), xw[j].cpu().numpy().astype(np.float64), vm)
        dis.append((a, b))
    dis = np.array(dis)
    for pl in plans:
        pl.close()
    return {
        "problems": count, "size": size, "check_every": check_every,
        "cold_iters_mean": float(ic.mean()), "warm_iters_mean": float(iw.mean()),
        "iters_ratio": float(ic.mean() / iw.mean()),
        "cold_converged": int(sum(r.converged for r in rc)), "warm_converged": int(sum(r.converged for r in rw)),
        "cold_images_per_s": count / cold_s, "warm_images_per_s": count / (warm_s + cnn_s),
        "cnn_ms_per_image": 1e3 * cnn_s / count,
        "cold_isnr_db": float(dis[:, 0].mean()), "warm_isnr_db": float(dis[:, 1].mean()),
        "isnr_diff_db_max_abs": float(np.abs(dis[:, 1] - dis[:, 0]).max()),
        "prediction_rel_err": pred_err,
        **({"api_warm": api} if api is not None else {}),
    }


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--count", type=int, default=20000)
    t.add_argument("--epochs", type=int, default=12)
    t.add_argument("--batch", type=int, default=16)
    t.add_argument("--lr", type=float, default=2e-3)
    t.add_argument("--seed", type=int, default=0)
    t.add_argument("--out", default=WEIGHTS)
    t.add_argument("--eval-count", type=int, default=32)
    t.add_argument("--cw", type=float, nargs=4, default=(1.0, 1.0, 1.0, 1.0))
    x = sub.add_parser("export")
    x.add_argument("--weights", default=WEIGHTS)
    x.add_argument("--out", default=WEIGHTS_BIN)
    v = sub.add_parser("eval")
    v.add_argument("--weights", default=WEIGHTS)
    v.add_argument("--count", type=int, default=64)
    v.add_argument("--check-every", type=int, default=1)
    a = ap.parse_args(argv)
    if a.cmd == "train":
        params, scales, meta = train(a.count, a.epochs, a.batch, a.lr, tuple(a.cw), seed=a.seed)
        if a.eval_count > 0:
            meta["eval"] = evaluate(params, scales, a.eval_count)
        save(a.out, params, scales, meta)
        export_binary(params, scales, os.path.splitext(a.out)[0] + ".bin")
        print(json.dumps({k: v for k, v in meta.items() if k != "loss_history"}), flush=True)
    elif a.cmd == "export":
        params, scales, _ = load(a.weights)
        print(export_binary(params, scales, a.out))
    else:
        params, scales, meta = load(a.weights)
        print(json.dumps(evaluate(params, scales, a.count, check_every=a.check_every)), flush=True)


if __name__ == "__main__":
    main()
