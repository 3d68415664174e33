"""Benchmark: batched TV-MD deconvolution + inpainting at 512 x 512, solved
to a relative change of x below 1e-5.

One step = one call of admm_deconv_solve_batch over a batch of synthetic
512 x 512 problems (19 x 19 Gaussian sigma 3 and 15-px / 30 degree motion
blur, BSNR 40 and 60 dB, valid region AND 60% of interior pixels kept), each
run from u0 = d0 = 0 until ||x_k - x_{k-1}|| / ||x_k|| < 1e-5 (at most 5000
iterations). The batch's working set (~11 MB per problem) is larger than L2.

Prints one JSON line. `value` = ADMM iterations per second summed over the
batch (device-resident inputs); `e2e` = the same through the C ABI with host
buffers (host->device and device->host copies inside the timed region).
`--impl reference` times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth as S  # noqa: E402

METRIC = "ADMM iters/s and images/s to tol at fixed ISNR; fraction of HBM roofline"
H = W = 512
TOL = 1e-5
MAX_ITERS = 5000
CHECK_EVERY = 10
COMBOS = [("gauss", 40), ("motion", 40), ("gauss", 60), ("motion", 60)]
STEADY_ITERS = 40
TUNING_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_1210_2687_gb300", "tuning.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=256, help="problems per step per GPU")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the frame-prior workload")
    ap.add_argument("--frame-only", action="store_true", help="only the frame-prior workload (profiler captures)")
    ap.add_argument("--frame-sizes", default="1024,2048,fs1024",
                    help="frame workloads to run: sides, 'fs' prefix for the synthesis formulation")
    ap.add_argument("--frame-iters", type=int, default=500, help="fixed iterations of the frame workloads")
    ap.add_argument("--frame-no-accuracy", action="store_true", help="skip the frame workloads' solve to tolerance")
    ap.add_argument("--frame-batch", type=int, default=1,
                    help="problems per solve in the frame workloads' throughput leg (copies of the image)")
    ap.add_argument("--uneven-only", action="store_true", help="only the batched uneven workload")
    ap.add_argument("--warm-only", action="store_true", help="only the learned warm-start comparison")
    ap.add_argument("--cg-only", action="store_true", help="only the mask-decoupling vs Reeves-Sorel comparison")
    ap.add_argument("--oracle-only", action="store_true", help="only the CPU oracle timing table")
    ap.add_argument("--steady-only", action="store_true",
                    help="only the fixed-iteration pass with every slot busy (for profiler captures)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the default launch configurations instead of the autotuner's")
    ap.add_argument("--retune", action="store_true", help="autotune even if the tuning cache has the class")
    ap.add_argument("--tv-tuning", default=None,
                    help="row_variant,col_variant,slot_ctas,lanes for the 512^2 TV class instead of the autotuner's "
                         "(profiler captures of a known configuration)")
    return ap.parse_args()


def tune_class(ad, torch, args, size_h, size_w, reg, levels=4, problems=0):
    """Launch configuration of a size class: the autotuner's choice (from the
    tuning cache in the user's cache directory when it holds this GPU and
    class, else measured now and added to it), or the defaults."""
    if args.no_autotune:
        cfg = ad.admm_deconv_get_tuning(size_h, size_w, reg, levels)
        cfg["source"] = "default"
        return cfg
    cfg = ad.autotune_cached(size_h, size_w, reg, levels, path=TUNING_CACHE,
                             device_name=torch.cuda.get_device_name(), retune=args.retune, problems=problems)
    trials = cfg.pop("trials", None)
    if trials:
        cfg["trials"] = len(trials)
        cfg["trial_table"] = [[t["rows_per_strip"], t["walk_depth"], t["row_threads"], t["col_block"],
                               t["col_min_ctas"], t["col_persistent"], t["slot_ctas"], t["lanes"],
                               round(t["us_per_iter"], 3)] for t in trials]
        cfg["us_per_iter_default"] = next((t["us_per_iter"] for t in trials if t["row_variant"] == 0
                                           and t["col_variant"] == 0 and t["slot_ctas"] == 0
                                           and t["lanes"] == 0), None)
    return cfg


def kernel_names(cfg, size_h, size_w):
    """Names of the TV row-phase and column-phase kernels of a configuration."""
    mb = f",{cfg['col_min_ctas']}" if cfg.get("col_min_ctas") else ""
    col = "col_phase_pers" if cfg.get("col_persistent") else "col_phase"
    if cfg.get("col_persistent"):
        mb = ""
    return (f"row_phase_tv<{size_w},{cfg['rows_per_strip']},{cfg['walk_depth']},{cfg['row_threads']}>",
            f"{col}<{size_h},{cfg['col_block']}{mb}>")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_over_ranks(seconds, work, device=None):
    """Whole-job figures of a replicated run: the slowest rank's time and the
    work summed over ranks (one process per GPU, no data-path collective;
    this is bookkeeping after the timed region)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds), float(work)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def make_batch(batch, rank):
    probs = []
    for i in range(batch):
        blur, bsnr = COMBOS[i % len(COMBOS)]
        probs.append(S.config2_problem(seed=1000 * rank + i, blur=blur, bsnr=bsnr))
    return probs


def bytes_per_pixel_iter():
    """Algorithmic HBM bytes per pixel and iteration of each phase (FP32).
    Row phase: half spectra in and out (8 + 8), d1 and d2 read and written
    (8 + 16), M^T y read (4; the observation mask is folded into it), x_prev
    for the rel-x rule (read + write once per CHECK_EVERY iterations).
    Column phase: half spectra in and out (8 + 8) and Lambda, K over the half
    spectrum (6)."""
    half = (W // 2 + 1) / W
    row = 8 + 8 + 8 + 16 + 4 + 8.0 / CHECK_EVERY
    col = (16 + 16 + 8 + 4) * half
    return row, col


def device_sources_sha256():
    """Digest of the device-code sources of the TV kernels (iteration
    kernels, FFT, configuration list), which ties a stored ncu traffic figure
    to the kernels it was measured on."""
    import hashlib
    h = hashlib.sha256()
    for f in ("kernels.cuh", "fft.cuh", "variants.cuh"):
        with open(os.path.join(ROOT, "paper_1210_2687_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def isnr_db(x_true, ybar, x_hat, region):
    """ISNR over the boolean region: 10 log10(||x - ybar||^2 / ||x - x_hat||^2)
    (the figure of merit of Sec. V; accuracy context, outside timed regions)."""
    r = region.astype(bool)
    num = float(np.sum((x_true[r] - ybar[r]) ** 2))
    den = float(np.sum((x_true[r] - x_hat[r]) ** 2))
    return 10.0 * math.log10(num / den)


def read_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to BENCH_CLOCKS_DIR (default: the system's temporary directory)
        import tempfile
        self.path = os.path.join(os.environ.get("BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 7:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx = float(parts[1])
                except ValueError:
                    continue
                for n, v in zip(names, parts[3:7]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        except OSError:
            return None
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cufft_comparison(torch, probs, iters, x_ref, stream):
    """The same TV-MD iteration written with torch.fft (cuFFT) and torch
    elementwise operations over the whole batch, timed for comparison only
    (it is not the product path): per iteration two forward and two inverse
    real 2-D FFTs (X^ = K (mu1 conj(Lambda) Z1^ + mu2 (D^T delta)^),
    x = F^-1 X^, A x = F^-1 Lambda X^), the mask prox and d1 update
    (eq. new_line, Alg. 3 line 8) and the vector-soft TV prox and d2 update
    (Alg. 3 lines 9-11). Returns its iterations per second and the relative
    L2 difference of its x from `x_ref` (this library's x after the same
    number of iterations from the same cold start)."""
    dev = x_ref[0].device
    B = len(probs)
    f32 = torch.float32
    lam = torch.tensor([p.lam for p in probs], dtype=torch.float64, device=dev).view(B, 1, 1)
    mu1 = torch.tensor([p.mu1 for p in probs], dtype=torch.float64, device=dev).view(B, 1, 1)
    mu2 = torch.tensor([p.mu2 for p in probs], dtype=torch.float64, device=dev).view(B, 1, 1)
    # Lambda: DFT of each kernel with its centre moved to (0, 0)
    ker = torch.zeros((B, H, W), dtype=torch.float64, device=dev)
    for b, p in enumerate(probs):
        kh, kw = p.psf.shape
        k = torch.zeros((H, W), dtype=torch.float64)
        k[:kh, :kw] = torch.from_numpy(p.psf.astype(np.float64))
        ker[b] = torch.roll(k, shifts=(-(kh // 2), -(kw // 2)), dims=(0, 1)).to(dev)
    lam_hat = torch.fft.rfft2(ker)
    kr = torch.arange(H, dtype=torch.float64, device=dev).view(H, 1)
    kc = torch.arange(W // 2 + 1, dtype=torch.float64, device=dev).view(1, -1)
    dd = 4.0 * torch.sin(math.pi * kc / W) ** 2 + 4.0 * torch.sin(math.pi * kr / H) ** 2
    kinv = (1.0 / (mu1 * lam_hat.abs() ** 2 + mu2 * dd)).to(f32)
    lam_hat = lam_hat.to(torch.complex64)
    obs = torch.stack([torch.from_numpy(p.mask.astype(bool)) for p in probs]).to(dev)
    yb = torch.stack([torch.from_numpy(p.ybar.astype(np.float32)) for p in probs]).to(dev)
    m1, m2 = mu1.to(f32), mu2.to(f32)
    tau = (lam / mu2).to(f32)
    inv1 = (1.0 / (1.0 + mu1)).to(f32)

    def run():
        d1 = torch.zeros((B, H, W), dtype=f32, device=dev)
        d2h, d2v = torch.zeros_like(d1), torch.zeros_like(d1)
        z1, dh, dv = torch.zeros_like(d1), torch.zeros_like(d1), torch.zeros_like(d1)
        x = None
        for _ in range(iters):
            dtd = (torch.roll(dh, 1, 2) - dh) + (torch.roll(dv, 1, 1) - dv)
            xh = kinv * (m1 * torch.conj(lam_hat) * torch.fft.rfft2(z1) + m2 * torch.fft.rfft2(dtd))
            x = torch.fft.irfft2(xh, s=(H, W))
            ax = torch.fft.irfft2(lam_hat * xh, s=(H, W))
            s1 = ax - d1
            u1 = torch.where(obs, (yb + m1 * s1) * inv1, s1)
            d1 = d1 - (ax - u1)
            gh = torch.roll(x, -1, 2) - x
            gv = torch.roll(x, -1, 1) - x
            sh, sv = gh - d2h, gv - d2v
            sc = torch.clamp(1.0 - tau * torch.rsqrt(sh * sh + sv * sv), min=0.0)
            uh, uv = sc * sh, sc * sv
            d2h = d2h - (gh - uh)
            d2v = d2v - (gv - uv)
            z1, dh, dv = u1 + d1, uh + d2h, uv + d2v
        return x

    with torch.cuda.stream(stream):
        run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x = run()
        e1.record(stream)
        torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3
    xr = torch.stack(list(x_ref))
    rel = float(torch.linalg.norm((x - xr).flatten()) / torch.linalg.norm(xr.flatten()))
    return {"iters_per_s": B * iters / sec, "problems": B, "iters": iters, "rel_l2_vs_library": rel,
            "what": "torch.fft (cuFFT) rfft2/irfft2 + torch elementwise ops, same iteration, same batch"}


FRAME_ITERS = 500
TV_ALG_BYTES = 67.0      # TV-MD: d (3 planes) in and out 24, M^T y and mask 5, Lambda and K 6, two complex round trips 32
FRAME_ALG_BYTES = 155.0  # FA-MD, 4 levels: d (14 planes) in and out 112, 5, 6, 32


def frame_secondary(ad, torch, stream, args):
    """Frame-prior (FA-MD) workload: 4-level undecimated Haar, 13 x 13
    uniform blur, valid region, BSNR 50 dB, 1024^2 and 2048^2 (and the
    synthesis formulation FS-MD at 1024^2), a fixed 500
    iterations (throughput); kernel time per phase from a profiled pass; and
    the same problem solved to rel-x < 1e-5 (checked every 10 iterations)
    for accuracy: iterations and ISNR. The fraction of the HBM roofline is
    taken on the method's algorithmic bytes per pixel and iteration, 155 for
    the 13-band frame prior: d1 and d2 (14 planes) read and written (112),
    M^T y and the mask (5), Lambda and K over the half spectrum (6), and two
    complex round trips between the row and column phases (32). The kernels
    themselves move more (the zeta2 re-read by the synthesis with its halo,
    the x and zeta1 scratch planes): column phase 22.1, row side 28 (inverse
    rows) + 116 (analysis tile: x, zeta2 in and out, the state bits) + 56
    (synthesis tile: zeta2, w) + 16 (forward rows); FS-MD's analysis tile
    also reads the previous w (+4; its previous zeta2 is the state it reads
    anyway). That figure is
    reported beside it, and the extra bytes count as overhead, not work. With
    --frame-batch B > 1 the throughput leg solves B copies of the image in
    one call (key suffix _xB; iterations/s counts problem-iterations)."""
    out = {}
    FRAME_ITERS = args.frame_iters
    cases = []
    for tok in args.frame_sizes.split(","):
        tok = tok.strip()
        cases.append(("haar_synthesis", int(tok[2:])) if tok.startswith("fs") else ("haar", int(tok)))
    for reg, size in cases:
        p = S.config3_problem(0, size, lam=S.FS_FRAME_LAMBDA) if reg == "haar_synthesis" else S.config3_problem(0, size)
        n = size * size
        B = max(1, args.frame_batch)
        tune = tune_class(ad, torch, args, size, size, "haar", 4, problems=B)
        plans = [ad.Plan(size, size, p.psf, p.lam, p.mu1, p.mu2, reg, stop="iters", max_iters=FRAME_ITERS)
                 for _ in range(B)]
        y = torch.from_numpy(p.ybar.astype(np.float32)).to("cuda")
        m = torch.from_numpy(p.mask).to("cuda")
        xs = [torch.empty((size, size), dtype=torch.float32, device="cuda") for _ in range(B)]
        x = xs[0]

        def run():
            ad.solve_batch(plans, [y] * B, [m] * B, xs, stream=stream)

        run()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run()
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3 / B      # per problem
        ad.admm_deconv_profile(True)
        run()
        pf = ad.admm_deconv_profile(False)
        pf_row_ms, pf_col_ms = pf.row_ms / B, pf.col_ms / B
        # synthesis form: the analysis tile also reads the previous w
        row_b = 28.0 + 116.0 + 56.0 + 16.0 + (4.0 if reg == "haar_synthesis" else 0.0)
        col_b = 44.0 * (size // 2 + 1) / size
        alg_b = FRAME_ALG_BYTES
        peak, _ = read_peak()
        key = f"{'fs' if reg == 'haar_synthesis' else 'fa'}_md_{size}" + (f"_x{B}" if B > 1 else "")
        out[key] = {
            "iters_per_s": FRAME_ITERS / sec,
            # whole iteration: the method's algorithmic bytes over the timed solve
            "iteration_gbs": FRAME_ITERS * n * alg_b / sec / 1e9,
            "iteration_frac": FRAME_ITERS * n * alg_b / sec / 1e9 / peak,
            "alg_bytes_per_px_iter": alg_b,
            # the same with the bytes the kernels move (their overhead included)
            "iteration_frac_kernel_bytes": FRAME_ITERS * n * (row_b + col_b) / sec / 1e9 / peak,
            "row_side_gbs": FRAME_ITERS * n * row_b / (pf_row_ms * 1e-3) / 1e9,
            "col_phase_gbs": FRAME_ITERS * n * col_b / (pf_col_ms * 1e-3) / 1e9,
            "bytes_per_px_iter": {"row_side": row_b, "col_phase": col_b},
            "problems_per_solve": B,
            "tuning": tune}
        for pl in plans:
            pl.close()
        if args.frame_no_accuracy:
            continue
        acc = ad.Plan(size, size, p.psf, p.lam, p.mu1, p.mu2, reg, stop="rel_x", tol=TOL, max_iters=MAX_ITERS,
                      check_every=CHECK_EVERY)
        r = ad.solve(acc, y, m, x, stream)
        torch.cuda.synchronize()
        vm = S.valid_mask(size, size, *p.psf.shape)
        out[key]["to_tolerance"] = {
            "iters": int(r.iters), "converged": int(r.converged), "rel_x": r.rel_x,
            "isnr_db": isnr_db(p.x_true, p.ybar, x.cpu().numpy().astype(np.float64), vm)}
        acc.close()
    return out


UNEVEN_COUNT = 256


def uneven_secondary(ad, torch, stream, args, count=UNEVEN_COUNT):
    """Batched uneven workload: ``count`` problems (seed 0) with sides drawn
    from {128, 256, 384 (solved on the exact 384 x 384 domain), 512, 1024},
    box / Gaussian / motion kernels of side 5..25, missing fraction
    U[0, 0.5], TV or 4-level Haar, BSNR 40 dB, all in one solve_batch call to
    rel-x < 1e-5, checked every CHECK_EVERY iterations as in the headline
    workload (the algorithmic bytes per iteration, 67 and 155 B/px, assume
    that rate; a problem retires at the first check that meets the rule).
    Time to tolerance per problem comes from its device-clock start and
    retirement stamps."""
    t_gen = time.perf_counter()
    probs = S.config4_batch(0, count, pad=False)
    t_gen = time.perf_counter() - t_gen
    # launch configuration of every size class (before the plans are made)
    tunings = {}
    for key in sorted({(p.ybar.shape[0], p.reg) for p in probs}):
        if key[0] & (key[0] - 1):
            tunings[f"{key[0]}_{key[1]}"] = "mixed-radix kernels on the exact domain (one configuration)"
            continue
        cfg = tune_class(ad, torch, args, key[0], key[0], key[1], 4)
        tunings[f"{key[0]}_{key[1]}"] = [cfg["rows_per_strip"], cfg["walk_depth"], cfg["row_threads"],
                                         cfg["col_block"], cfg["slot_ctas"], cfg.get("source")]
    plans, ys, ms, xs = [], [], [], []
    for p in probs:
        N = p.ybar.shape[0]
        plans.append(ad.Plan(N, N, p.psf, p.lam, p.mu1, p.mu2, p.reg, stop="rel_x", tol=TOL,
                             max_iters=MAX_ITERS, check_every=CHECK_EVERY))
        ys.append(torch.from_numpy(p.ybar.astype(np.float32)).to("cuda"))
        ms.append(torch.from_numpy(p.mask).to("cuda"))
        xs.append(torch.empty((N, N), dtype=torch.float32, device="cuda"))
    ad.solve_batch(plans, ys, ms, xs, stream=stream)          # warm-up: graphs, attributes
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = ad.solve_batch(plans, ys, ms, xs, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3
    done = np.array([r.t_done_ms for r in res])
    solve = np.array([r.t_done_ms - r.t_start_ms for r in res])
    iters = np.array([r.iters for r in res])
    px_iters = sum(int(r.iters) * p.ybar.size for r, p in zip(res, probs))
    # algorithmic bytes of every problem-iteration, each on its (padded) domain
    alg_bytes = sum(int(r.iters) * p.ybar.size * (TV_ALG_BYTES if p.reg == "tv" else FRAME_ALG_BYTES)
                    for r, p in zip(res, probs))
    peak, _ = read_peak()
    # where the work is: per size class and prior, problems, mean iterations
    # and the share of the algorithmic bytes
    classes = {}
    for r, p in zip(res, probs):
        c = classes.setdefault(f"{p.ybar.shape[0]}_{p.reg}", {"problems": 0, "iters": 0, "bytes": 0.0})
        c["problems"] += 1
        c["iters"] += int(r.iters)
        c["bytes"] += int(r.iters) * p.ybar.size * (TV_ALG_BYTES if p.reg == "tv" else FRAME_ALG_BYTES)
    class_table = {k: {"problems": v["problems"], "iters_mean": v["iters"] / v["problems"],
                       "alg_bytes_share": v["bytes"] / alg_bytes} for k, v in sorted(classes.items())}
    isnr = []
    for p, x in zip(probs, xs):
        n = p.meta["window"]
        N = p.ybar.shape[0]
        vm = np.zeros((N, N), dtype=np.uint8)
        vm[:n, :n] = S.valid_mask(n, n, *p.psf.shape)
        isnr.append(isnr_db(p.x_true, p.ybar, x.cpu().numpy().astype(np.float64), vm))
    for pl in plans:
        pl.close()
    return {
        "workload": f"{count} problems, sides {{128,256,384,512,1024}} (384 exact), box/gauss/motion 5..25, "
                    "missing U[0,0.5], TV or Haar, BSNR 40, rel-x < 1e-5 checked every "
                    f"{CHECK_EVERY} iterations",
        "images_per_s": count / sec,
        "iters_per_s": float(iters.sum()) / sec,
        "mpix_iters_per_s": px_iters / sec / 1e6,
        "hbm_gbs_algorithmic": alg_bytes / sec / 1e9,
        "hbm_frac": alg_bytes / sec / 1e9 / peak,
        "hbm_frac_note": "67 B/px (TV) or 155 B/px (4-level Haar) per iteration on each problem's domain",
        "wall_s": sec,
        "converged": int(sum(r.converged for r in res)),
        "iters_mean": float(iters.mean()),
        "iters_p50": float(np.percentile(iters, 50)),
        "iters_max": int(iters.max()),
        "latency_ms_p50": float(np.percentile(done, 50)),
        "latency_ms_p99": float(np.percentile(done, 99)),
        "time_to_tol_ms_p50": float(np.percentile(solve, 50)),
        "time_to_tol_ms_p99": float(np.percentile(solve, 99)),
        "isnr_db_mean": float(np.mean(isnr)),
        "input_generation_s": t_gen,
        "classes": class_table,
        "tuning": tunings,
    }


CG_ITERS = 200


def cg_secondary(ad, torch, stream, batch=64):
    """Mask decoupling against the Reeves-Sorel method (the paper's MD vs CG
    comparison, Table IV: 256 x 256 domain, 19 x 19 uniform blur, the valid
    region observed, i.e. 238 x 238, BSNR 40 dB): device time per iteration
    of TV-MD, TV-CG, FA-MD and FA-CG for one image and for a batch of
    `batch` images (fixed 200 iterations), and each method's iterations and
    time to the paper's stop rule (relative change of the objective < 1e-4)
    on one image with its ISNR."""
    size = 256
    psf = S.psf_box(19)
    probs = []
    for i in range(batch):
        g = S.rng(5000 + i)
        x = S.shapes_image(size, size, g, 20, rmax=size / 4.0) if i % 2 == 0 else S.textured_image(size, size, g)
        ybar, mask, _ = S.observe(x, psf, None, 40.0, g)
        probs.append((x, ybar.astype(np.float32), mask))
    lam = {"tv": 2e-4, "haar": 2e-4}
    ys = [torch.from_numpy(p[1]).cuda() for p in probs]
    ms = [torch.from_numpy(p[2]).cuda() for p in probs]
    xs = [torch.empty((size, size), dtype=torch.float32, device="cuda") for _ in probs]
    vm = S.valid_mask(size, size, 19, 19)

    def timed(plans, k):
        ad.solve_batch(plans, ys[:k], ms[:k], xs[:k], stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ad.solve_batch(plans, ys[:k], ms[:k], xs[:k], stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3

    out = {"workload": "256x256 domain, 19x19 uniform blur, valid region (238x238 observed), BSNR 40, "
                       f"lambda 2e-4; {CG_ITERS} iterations; batch {batch}"}
    for prior in ("tv", "haar"):
        mu1, mu2 = S.default_mu(lam[prior])
        row = {}
        for method in ("md", "cg"):
            reg = prior if method == "md" else prior + "_cg"
            r = {}
            for k in (1, batch):
                plans = [ad.Plan(size, size, psf, lam[prior], mu1, mu2, reg, max_iters=CG_ITERS) for _ in range(k)]
                sec = timed(plans, k)
                r[f"us_per_iter_batch{k}"] = sec / CG_ITERS * 1e6
                r[f"us_per_problem_iter_batch{k}"] = sec / (CG_ITERS * k) * 1e6
                for pl in plans:
                    pl.close()
            acc = ad.Plan(size, size, psf, lam[prior], mu1, mu2, reg, stop="rel_obj", tol=1e-4, max_iters=MAX_ITERS)
            ad.solve(acc, ys[0], ms[0], xs[0], stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = ad.solve(acc, ys[0], ms[0], xs[0], stream)
            e1.record(stream)
            torch.cuda.synchronize()
            r["to_rel_obj_1e-4"] = {"iters": int(res.iters), "converged": int(res.converged),
                                    "ms": e0.elapsed_time(e1),
                                    "isnr_db": isnr_db(probs[0][0], probs[0][1],
                                                       xs[0].cpu().numpy().astype(np.float64), vm)}
            acc.close()
            row[method] = r
        row["cg_over_md_per_iter_single"] = row["cg"]["us_per_iter_batch1"] / row["md"]["us_per_iter_batch1"]
        row["cg_over_md_per_iter_batch"] = (row["cg"][f"us_per_iter_batch{batch}"]
                                            / row["md"][f"us_per_iter_batch{batch}"])
        row["cg_over_md_time_to_tol"] = row["cg"]["to_rel_obj_1e-4"]["ms"] / row["md"]["to_rel_obj_1e-4"]["ms"]
        out[prior] = row
    out["paper"] = "MD 1.6-1.8x faster per iteration, 1.5-2x in total (Sec. V, Table IV; MATLAB, Core i5)"
    return out


CNN_FLOP_PER_PX = 2 * 9 * (2 * 32 + 6 * 32 * 32 + 32 * 4)   # eight 3x3 convolutions
# HBM bytes per pixel of one forward: the input kernel (M^T y 4 + mask 1 in,
# one plane of 8 BF16 channels out 16), layer 0 (16 in, 64 out), six
# 32-channel layers (64 in, 64 out each), the last layer (64 in, 4 FP32
# channels out 16)
CNN_BYTES_PER_PX = (4 + 1 + 16) + (16 + 64) + 6 * (64 + 64) + (64 + 16)


def warm_secondary(ad, torch, stream, count=32):
    """Learned warm start against the cold start on unseen 512^2 problems
    (piecewise-constant law, 9 x 9 box, valid region, BSNR 40, lambda 1e-3),
    both to rel-x < 1e-5; and the network's forward throughput on the tensor
    cores (16 images of 512^2, FLOPs of the eight convolutions)."""
    import paper_1210_2687_gb300.warmstart as WS
    params, scales, meta = WS.load()
    ev = WS.evaluate(params, scales, count=count, seed=1, api_weights=WS.WEIGHTS_BIN)
    n = 16
    net = ad.Cnn(n * 512 * 512)
    net.set_params(params)
    g = np.random.default_rng(0)
    y = torch.from_numpy(g.uniform(size=(n, 512, 512)).astype(np.float32)).cuda()
    m = torch.ones((n, 512, 512), dtype=torch.uint8, device="cuda")
    out = torch.empty((n, 512, 512, 4), dtype=torch.float32, device="cuda")
    for _ in range(3):
        net.forward(y, m, out, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    e0.record(stream)
    for _ in range(reps):
        net.forward(y, m, out, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3 / reps
    tflops = CNN_FLOP_PER_PX * n * 512 * 512 / sec / 1e12
    net.close()
    peak, _ = read_peak()
    hbm = CNN_BYTES_PER_PX * n * 512 * 512 / sec / 1e9
    ev["cnn_forward"] = {"images": n, "size": 512, "ms": sec * 1e3, "tflops": tflops,
                         "hbm_gbs": hbm, "hbm_frac": hbm / peak, "bytes_per_px": CNN_BYTES_PER_PX,
                         "note": "all 8 convolutions on tcgen05.mma (two TMEM accumulators) fed by "
                                 "double-buffered TMA halo boxes of 160-byte rows (activations in planes of "
                                 "8 channels); 9 launches per forward; each layer reads and writes its "
                                 "activations in HBM"}
    ev["trained"] = {k: meta[k] for k in ("count", "epochs", "lr", "train_s", "steps") if k in meta}
    return ev


_ORACLE_TIMING = r"""
import json, os, resource, sys, time
sys.path.insert(0, sys.argv[1])
import numpy as np
import oracle as O
import synth as S
size, reg, budget, min_it, max_it = int(sys.argv[2]), sys.argv[3], float(sys.argv[4]), int(sys.argv[5]), int(sys.argv[6])
if reg == "tv":
    p = S.config1_problem(0) if size == 64 else S.config2_problem(0, "gauss", 40, size=size)
else:
    p = S.config3_problem(0, size)
H, W = p.ybar.shape
st = O.State.zeros(H, W, reg)
otf = O.psf_otf(p.psf, H, W)
den = O.tv_denominator_diag(p.psf, H, W, p.mu1, p.mu2) if reg == "tv" else None
r0 = resource.getrusage(resource.RUSAGE_SELF)
t0 = time.perf_counter()
n = 0
while n < max_it and (n < min_it or time.perf_counter() - t0 < budget):
    if reg == "tv":
        st = O.tvmd_step(st, p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, otf, den)
    else:
        st = O.famd_step(st, p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, 4, otf)
    n += 1
dt = time.perf_counter() - t0
r1 = resource.getrusage(resource.RUSAGE_SELF)
cpu = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
print(json.dumps({"iters": n, "seconds": dt, "iters_per_s": n / dt, "cpu_util": cpu / dt}))
"""


def oracle_timing(cores):
    """The FP64 oracle timed as it stands on the host cores, in fresh
    processes whose BLAS thread count is set by the environment: one thread,
    and all `cores` the process may run on. Sizes 64^2 and 512^2 run TV-MD
    (the 64^2 and 512^2 workloads), 1024^2 and 2048^2 FA-MD (the frame
    workload; at least 5 iterations). One thread is timed at 64^2 and 512^2
    only (at 2048^2 one FP64 iteration of the oracle's matrix DFTs takes
    minutes on one core). `cpu_util` = CPU time / wall time of the loop."""
    cases = [(64, "tv", 3.0, 5, 10 ** 6), (512, "tv", 6.0, 3, 10 ** 6),
             (1024, "haar", 0.0, 5, 5), (2048, "haar", 0.0, 5, 5)]
    out = {"cores_available": cores, "runs": []}
    for threads in (1, cores):
        env = dict(os.environ)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[k] = str(threads)
        for size, reg, budget, lo, hi in cases:
            if threads == 1 and size > 512:
                continue
            r = subprocess.run([sys.executable, "-c", _ORACLE_TIMING, ROOT, str(size), reg, str(budget), str(lo),
                                str(hi)], capture_output=True, text=True, env=env, timeout=1200)
            if r.returncode != 0:
                out["runs"].append({"size": size, "reg": reg, "threads": threads, "error": r.stderr[-300:]})
                continue
            d = json.loads(r.stdout.strip().splitlines()[-1])
            d.update({"size": size, "reg": reg, "threads": threads})
            out["runs"].append(d)
    return out


def cpu_baseline_oracle(probs, seconds=12.0):
    """The FP64 oracle as it stands on one 512^2 problem of the workload,
    iterating until about `seconds` of CPU time; iterations per second."""
    import oracle as O
    p = probs[0]
    st = O.State.zeros(H, W, "tv")
    otf = O.psf_otf(p.psf, H, W)
    den = O.tv_denominator_diag(p.psf, H, W, p.mu1, p.mu2)
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < seconds:
        st = O.tvmd_step(st, p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, otf, den)
        n += 1
    dt = time.perf_counter() - t0
    return n / dt, n, dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import resource
    cores = len(os.sched_getaffinity(0))
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    w0 = time.perf_counter()
    probs = make_batch(1, 0)
    per_step = []
    iters_step = 0
    for s in range(args.warmup + args.steps):
        v, n, dt = cpu_baseline_oracle(probs, seconds=3.0)
        if s >= args.warmup:
            per_step.append((n, dt))
            iters_step = n
    tot_n = sum(n for n, _ in per_step)
    tot_t = sum(t for _, t in per_step)
    value = tot_n / tot_t
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    util = ((r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)) / (time.perf_counter() - w0)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * tot_t / max(1, len(per_step)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "tv_md_512x512_inpaint40_gauss19_motion15_relx1e-5",
                   "sample": f"{iters_step} oracle iterations on one 512x512 problem per step"},
        "cpu_baseline": {"value": value, "unit": "iters/s", "cores": cores, "kind": "oracle",
                         "sample": f"TV-MD FP64 oracle (matrix DFTs on the host's BLAS), one 512x512 problem, "
                                   f"~3 s per step, CPU utilisation {util:.1f} cores"},
        "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    if args.oracle_only:      # host only (no GPU work)
        print(json.dumps({"oracle_timing": oracle_timing(len(os.sched_getaffinity(0)))}), flush=True)
        return
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1210_2687_gb300 as ad

    dev = torch.device("cuda", local)
    if args.frame_only:
        print(json.dumps({"secondary": frame_secondary(ad, torch, torch.cuda.current_stream(), args)}), flush=True)
        return
    if args.warm_only:
        print(json.dumps({"warm_start": warm_secondary(ad, torch, torch.cuda.current_stream())}), flush=True)
        return
    if args.cg_only:
        print(json.dumps({"md_vs_cg_256": cg_secondary(ad, torch, torch.cuda.current_stream())}), flush=True)
        return
    if args.uneven_only:
        print(json.dumps({"uneven_batch": uneven_secondary(ad, torch, torch.cuda.current_stream(), args)}), flush=True)
        return
    if args.tv_tuning:
        rv, cv, sc, ln = (int(v) for v in args.tv_tuning.split(","))
        ad.admm_deconv_set_tuning({"H": H, "W": W, "reg": ad.ADMM_REG_TV, "haar_levels": 0, "row_variant": rv,
                                   "col_variant": cv, "slot_ctas": sc, "lanes": ln})
        tune = ad.admm_deconv_get_tuning(H, W, "tv")
        tune["source"] = "given"
    else:
        tune = tune_class(ad, torch, args, H, W, "tv")
    row_kernel, col_kernel = kernel_names(tune, H, W)
    probs = make_batch(args.batch, rank)
    n = H * W
    plans = [ad.Plan(H, W, p.psf, p.lam, p.mu1, p.mu2, "tv", stop="rel_x", tol=TOL,
                     max_iters=MAX_ITERS, check_every=CHECK_EVERY) for p in probs]
    ys = [torch.from_numpy(p.ybar.astype(np.float32)).to(dev) for p in probs]
    ms = [torch.from_numpy(p.mask).to(dev) for p in probs]
    xs = [torch.empty((H, W), dtype=torch.float32, device=dev) for _ in probs]
    stream = torch.cuda.current_stream()

    if args.steady_only:
        fixed = [ad.Plan(H, W, p.psf, p.lam, p.mu1, p.mu2, "tv", max_iters=STEADY_ITERS) for p in probs]
        ad.solve_batch(fixed, ys, ms, xs, stream=stream)
        ad.admm_deconv_profile(True)
        ad.solve_batch(fixed, ys, ms, xs, stream=stream)
        pf = ad.admm_deconv_profile(False)
        row_b, col_b = bytes_per_pixel_iter()
        its = STEADY_ITERS * len(fixed)
        print(json.dumps({"steady_state": {
            "problems": len(fixed), "iters": STEADY_ITERS, "kernels": [row_kernel, col_kernel],
            "row_phase_gbs": its * n * row_b / (pf.row_ms * 1e-3) / 1e9,
            "col_phase_gbs": its * n * col_b / (pf.col_ms * 1e-3) / 1e9,
            "iters_per_s": its / ((pf.row_ms + pf.col_ms) * 1e-3)}}), flush=True)
        return

    def step():
        return ad.solve_batch(plans, ys, ms, xs, stream=stream)

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---- timed region: device-resident inputs, normal operation ----
    ad.admm_deconv_profile(False)
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        total_iters = 0
        for _ in range(args.steps):
            res = step()
            total_iters += sum(r.iters for r in res)
        ev1.record(stream)
        torch.cuda.synchronize()
        launches = ad.admm_deconv_profile(False).kernel_launches
        ms_total = ev0.elapsed_time(ev1)
        barrier()

        # ---- end to end through the C ABI with host buffers ----
        yh = [torch.from_numpy(p.ybar.astype(np.float32)).pin_memory() for p in probs]
        mh = [torch.from_numpy(p.mask).pin_memory() for p in probs]
        xh = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in probs]
        # the same warm-up as the device-resident steps (the first calls on
        # freshly pinned buffers pay their first-touch costs)
        for _ in range(args.warmup):
            ad.solve_batch(plans, yh, mh, xh, stream=stream)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        e2e_iters = 0
        e2e_steps_ms = []
        for _ in range(args.steps):
            ts = time.perf_counter()
            r2 = ad.solve_batch(plans, yh, mh, xh, stream=stream)
            e2e_iters += sum(r.iters for r in r2)
            e2e_steps_ms.append((time.perf_counter() - ts) * 1e3)
        torch.cuda.synchronize()
        e2e_sec = time.perf_counter() - t0
        e2e_sec, e2e_iters = reduce_over_ranks(e2e_sec, e2e_iters, dev)
    barrier()

    # ---- second timed pass of the same steps with per-phase CUDA events on
    # the solve's stream: the kernels' own durations for the roofline ----
    ad.admm_deconv_profile(True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    prof = ad.admm_deconv_profile(False)
    my_iters = total_iters
    ms_total, total_iters = reduce_over_ranks(ms_total, total_iters, dev)
    sec = ms_total / 1000.0
    value = total_iters / sec
    images_per_s = args.batch * world * args.steps / sec

    # ---- ISNR of the last solve (accuracy context) ----
    isnrs = []
    for p, x in zip(probs, xs):
        vm = S.valid_mask(H, W, *p.psf.shape)
        isnrs.append(isnr_db(p.x_true, p.ybar, x.cpu().numpy().astype(np.float64), vm))

    # ---- roofline of the dominant kernel ----
    row_b, col_b = bytes_per_pixel_iter()
    img_iters = my_iters          # this rank's kernels ran this rank's image-iterations
    # the profiled pass ran the same steps: the same image-iterations per kernel
    row_gbs = img_iters * n * row_b / (prof.row_ms * 1e-3) / 1e9 if prof.row_ms > 0 else 0.0
    col_gbs = img_iters * n * col_b / (prof.col_ms * 1e-3) / 1e9 if prof.col_ms > 0 else 0.0
    peak, peak_kind = read_peak()
    dom = row_kernel if prof.row_ms >= prof.col_ms else col_kernel
    ach = row_gbs if prof.row_ms >= prof.col_ms else col_gbs

    # ---- steady state (untimed for `value`): every slot busy for a fixed
    # number of iterations, the kernels' own bandwidth without the batch tail
    steady = None
    cufft = None
    if rank == 0:
        fixed = [ad.Plan(H, W, p.psf, p.lam, p.mu1, p.mu2, "tv", max_iters=STEADY_ITERS) for p in probs[:32]]
        ad.solve_batch(fixed, ys[:32], ms[:32], xs[:32], stream=stream)
        ad.admm_deconv_profile(True)
        ad.solve_batch(fixed, ys[:32], ms[:32], xs[:32], stream=stream)
        pf = ad.admm_deconv_profile(False)
        its = STEADY_ITERS * len(fixed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ad.solve_batch(fixed, ys[:32], ms[:32], xs[:32], stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        steady = {"problems": len(fixed), "iters": STEADY_ITERS,
                  "row_phase_gbs": its * n * row_b / (pf.row_ms * 1e-3) / 1e9,
                  "col_phase_gbs": its * n * col_b / (pf.col_ms * 1e-3) / 1e9,
                  "iters_per_s_kernels_alone": its / ((pf.row_ms + pf.col_ms) * 1e-3),
                  "iters_per_s": its / (e0.elapsed_time(e1) * 1e-3)}
        cufft = cufft_comparison(torch, probs[:32], STEADY_ITERS, xs[:32], stream)
        for f in fixed:
            f.close()
    # DRAM bytes per launch from the committed ncu capture (bytes per pixel
    # there) scaled to the pixels an average launch of this pass processed
    # (null when the device sources have changed since the capture)
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    launches_dom = prof.row_launches if dom == row_kernel else prof.col_launches
    if os.path.exists(tpath) and launches_dom > 0:
        try:
            tj = json.load(open(tpath))
            if tj.get("_device_sources_sha256") == device_sources_sha256():
                traffic = tj[dom]["bytes_per_px"] * n * img_iters / launches_dom
        except Exception:
            traffic = None

    secondary = None
    if rank == 0 and not args.no_secondary:
        secondary = frame_secondary(ad, torch, stream, args)
        secondary["uneven_batch"] = uneven_secondary(ad, torch, stream, args)
        secondary["warm_start"] = warm_secondary(ad, torch, stream)
        secondary["md_vs_cg_256"] = cg_secondary(ad, torch, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = len(os.sched_getaffinity(0))
        ot = oracle_timing(cores)
        all512 = next((r for r in ot["runs"] if r["size"] == 512 and r["threads"] == cores and "iters" in r), None)
        if all512 is not None:
            cpu = {"value": all512["iters_per_s"], "unit": "iters/s", "cores": cores, "kind": "oracle",
                   "sample": f"{all512['iters']} TV-MD iterations of the FP64 oracle on one 512x512 problem "
                             f"({all512['seconds']:.1f} s, BLAS threads = {cores}, "
                             f"CPU utilisation {all512['cpu_util']:.1f} cores)",
                   "timing_table": ot}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "tv_md_512x512_inpaint40_gauss19_motion15_relx1e-5",
                       "batch_per_gpu": args.batch, "H": H, "W": W, "tol_rel_x": TOL,
                       "check_every": CHECK_EVERY, "max_iters": MAX_ITERS,
                       "l2": "inputs larger than L2 (~11 MB per problem x batch)",
                       "slots": "automatic (continuous batching: queued problems start as others retire)",
                       "parallelism": f"replicas x{world}"},
            "images_per_s": images_per_s,
            "tuning": tune,
            "iters_per_image_mean": total_iters / (args.batch * world * args.steps),
            "isnr_db_mean": float(np.mean(isnrs)),
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": ach / peak,
                         "traffic": traffic,
                         "bytes_per_px_iter": {"row_phase": row_b, "col_phase": col_b},
                         "row_phase_gbs": row_gbs, "col_phase_gbs": col_gbs,
                         "row_ms": prof.row_ms, "col_ms": prof.col_ms,
                         # the whole iteration (both phases, all lanes overlapped) over
                         # the timed region: algorithmic bytes of every image-iteration
                         # the job ran / wall time (fraction of the peak of all GPUs)
                         "iteration_gbs": total_iters * n * (row_b + col_b) / sec / 1e9,
                         "iteration_frac": total_iters * n * (row_b + col_b) / sec / 1e9 / (peak * world),
                         "steady_state": steady},
            "cufft_comparison": cufft,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_iters / e2e_sec, "unit": "iters/s", "ms_per_step": e2e_steps_ms,
                    "h2d_bytes_per_step": args.batch * (4 * n + n),
                    "d2h_bytes_per_step": args.batch * 4 * n},
            "gpu_launches": int(launches),
            "secondary": secondary,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
