"""Seeded synthetic inputs for the unknown-boundary deconvolution workloads.

This module is the one piece shared by the FP64 oracle's tests and the CUDA
path's tests and benchmark. It holds no arithmetic of the ADMM method itself:
it draws test images, blur kernels, observation masks and noise, and forms the
observation the way the paper's experiments describe it (Sec. V): the blur is
applied to the full unknown image and only the *valid* region -- the pixels
whose blurred value does not depend on anything outside the image -- is kept,
then white Gaussian noise at a prescribed BSNR is added to the observed pixels.

The valid-region convolution below is a direct sum over kernel taps on the
non-periodic image; it is independent of both the oracle's operators and the
CUDA kernels, so it doubles as an outside check of the periodic model
y = M A x + n of Sec. IV-A.

All randomness comes from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "rng",
    "shapes_image",
    "value_noise",
    "textured_image",
    "psf_box",
    "psf_gaussian",
    "psf_motion",
    "psf_disk",
    "valid_mask",
    "conv_valid",
    "Problem",
    "observe",
    "config1_problem",
    "config2_problem",
    "config3_problem",
    "conv_valid_fft",
    "fft_domain",
    "config4_problem",
    "config4_batch",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


# --------------------------------------------------------------------------
# images
# --------------------------------------------------------------------------
def shapes_image(H: int, W: int, g: np.random.Generator, n_shapes: int = 20,
                 rmax: float | None = None) -> np.ndarray:
    """Piecewise-constant image in [0, 1]: a U[0,1] background with
    ``n_shapes`` axis-aligned rectangles or disks (equal odds) painted in
    order, each with a U[0,1] intensity. Rectangle corners are U[0, size);
    disk centres are U[0, size) and radii U[2, rmax] (rmax defaults to a
    quarter of the smaller side)."""
    if rmax is None:
        rmax = max(2.0, min(H, W) / 4.0)
    img = np.full((H, W), g.uniform(0.0, 1.0), dtype=np.float64)
    rr, cc = np.mgrid[0:H, 0:W]
    for _ in range(n_shapes):
        kind = g.integers(0, 2)
        val = g.uniform(0.0, 1.0)
        if kind == 0:
            r0, r1 = np.sort(g.uniform(0, H, size=2))
            c0, c1 = np.sort(g.uniform(0, W, size=2))
            sel = (rr >= r0) & (rr <= r1) & (cc >= c0) & (cc <= c1)
        else:
            cr = g.uniform(0, H)
            ccn = g.uniform(0, W)
            rad = g.uniform(2.0, rmax)
            sel = (rr - cr) ** 2 + (cc - ccn) ** 2 <= rad * rad
        img[sel] = val
    return img


def value_noise(H: int, W: int, g: np.random.Generator, octaves: int = 4,
                base_period: int = 64, persistence: float = 0.5) -> np.ndarray:
    """Smooth 'Perlin-like' texture: a sum of ``octaves`` lattice value-noise
    layers (random values on a grid of spacing base_period / 2**o, smoothstep
    interpolated), amplitude multiplied by ``persistence`` per octave,
    rescaled to [0, 1]."""
    out = np.zeros((H, W), dtype=np.float64)
    amp = 1.0
    for o in range(octaves):
        period = max(1, base_period >> o)
        gh = H // period + 2
        gw = W // period + 2
        lat = g.uniform(0.0, 1.0, size=(gh, gw))
        r = np.arange(H) / period
        c = np.arange(W) / period
        r0 = np.floor(r).astype(int)
        c0 = np.floor(c).astype(int)
        fr = r - r0
        fc = c - c0
        sr = fr * fr * (3 - 2 * fr)
        sc = fc * fc * (3 - 2 * fc)
        v00 = lat[r0[:, None], c0[None, :]]
        v01 = lat[r0[:, None], c0[None, :] + 1]
        v10 = lat[r0[:, None] + 1, c0[None, :]]
        v11 = lat[r0[:, None] + 1, c0[None, :] + 1]
        top = v00 + (v01 - v00) * sc[None, :]
        bot = v10 + (v11 - v10) * sc[None, :]
        out += amp * (top + (bot - top) * sr[:, None])
        amp *= persistence
    lo, hi = out.min(), out.max()
    return (out - lo) / max(hi - lo, 1e-12)


def textured_image(H: int, W: int, g: np.random.Generator) -> np.ndarray:
    """0.6 x piecewise-constant (20 shapes, radius up to a quarter side)
    + 0.4 x 4-octave value noise (base period 64 px), clamped to [0, 1]."""
    pc = shapes_image(H, W, g, 20, rmax=max(2.0, min(H, W) / 4.0))
    tx = value_noise(H, W, g, 4, 64, 0.5)
    return np.clip(0.6 * pc + 0.4 * tx, 0.0, 1.0)


# --------------------------------------------------------------------------
# blur kernels (odd side, centre at (side//2, side//2), unit sum)
# --------------------------------------------------------------------------
def psf_box(side: int) -> np.ndarray:
    assert side % 2 == 1
    return np.full((side, side), 1.0 / (side * side))


def psf_gaussian(side: int, sigma: float) -> np.ndarray:
    assert side % 2 == 1
    h = side // 2
    t = np.arange(-h, h + 1, dtype=np.float64)
    k = np.exp(-(t[:, None] ** 2 + t[None, :] ** 2) / (2.0 * sigma * sigma))
    return k / k.sum()


def psf_motion(length: float, angle_deg: float, side: int | None = None,
               supersample: int = 64) -> np.ndarray:
    """Linear motion blur: a centred segment of ``length`` pixels at
    ``angle_deg`` (counter-clockwise from the +column axis), supersampled
    ``supersample`` times per pixel of length and splatted bilinearly."""
    if side is None:
        side = int(math.ceil(length))
        side += 1 - side % 2
    assert side % 2 == 1
    h = side // 2
    k = np.zeros((side, side))
    ns = max(2, int(round(length * supersample)))
    t = (np.arange(ns) + 0.5) / ns - 0.5
    ang = math.radians(angle_deg)
    cs = h + t * (length - 1.0) * math.cos(ang)
    rs = h - t * (length - 1.0) * math.sin(ang)
    r0 = np.floor(rs).astype(int)
    c0 = np.floor(cs).astype(int)
    fr = rs - r0
    fc = cs - c0
    for dr, dc, wgt in ((0, 0, (1 - fr) * (1 - fc)), (0, 1, (1 - fr) * fc),
                        (1, 0, fr * (1 - fc)), (1, 1, fr * fc)):
        rr = np.clip(r0 + dr, 0, side - 1)
        cc = np.clip(c0 + dc, 0, side - 1)
        np.add.at(k, (rr, cc), wgt)
    return k / k.sum()


def psf_disk(side: int, radius: float | None = None, supersample: int = 8) -> np.ndarray:
    """Out-of-focus blur: area coverage of a disk, supersampled per pixel."""
    assert side % 2 == 1
    h = side // 2
    if radius is None:
        radius = h + 0.5
    s = (np.arange(supersample) + 0.5) / supersample - 0.5
    t = np.arange(-h, h + 1, dtype=np.float64)
    rr = (t[:, None, None, None] + s[None, None, :, None])
    cc = (t[None, :, None, None] + s[None, None, None, :])
    k = ((rr ** 2 + cc ** 2) <= radius * radius).mean(axis=(2, 3))
    return k / k.sum()


# --------------------------------------------------------------------------
# observation
# --------------------------------------------------------------------------
def valid_mask(H: int, W: int, psf_h: int, psf_w: int) -> np.ndarray:
    """uint8 mask of the pixels whose blurred value uses only pixels inside
    the H x W image: rows l_r..H-1-l_r, columns l_c..W-1-l_c (Sec. IV-A)."""
    lr, lc = psf_h // 2, psf_w // 2
    m = np.zeros((H, W), dtype=np.uint8)
    if H - 2 * lr > 0 and W - 2 * lc > 0:
        m[lr:H - lr, lc:W - lc] = 1
    return m


def conv_valid(x: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """Non-periodic 2-D convolution of x with psf, returned on the full H x W
    grid; only the valid region (see valid_mask) is meaningful, the rest is 0.
    out[r, c] = sum_{a,b} psf[a+lr, b+lc] * x[r-a, c-b]."""
    H, W = x.shape
    ph, pw = psf.shape
    lr, lc = ph // 2, pw // 2
    out = np.zeros((H, W))
    Hv, Wv = H - 2 * lr, W - 2 * lc
    if Hv <= 0 or Wv <= 0:
        return out
    acc = np.zeros((Hv, Wv))
    for a in range(-lr, lr + 1):
        for b in range(-lc, lc + 1):
            wgt = psf[a + lr, b + lc]
            if wgt == 0.0:
                continue
            acc += wgt * x[lr - a:lr - a + Hv, lc - b:lc - b + Wv]
    out[lr:lr + Hv, lc:lc + Wv] = acc
    return out


@dataclass
class Problem:
    """One synthetic deconvolution instance on the full H x W domain."""
    x_true: np.ndarray          # float64 H x W
    psf: np.ndarray             # float64, odd sides, unit sum
    ybar: np.ndarray            # float64 H x W: observed values, 0 elsewhere
    mask: np.ndarray            # uint8 H x W: 1 = observed
    sigma: float                # noise standard deviation
    lam: float
    mu1: float
    mu2: float
    reg: str = "tv"             # "tv" or "haar"
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.x_true.shape


def conv_valid_fft(x: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """conv_valid through a zero-padded (linear, not periodic) FFT product:
    the same valid-region values up to rounding, at O(n log n) for the large
    kernels of the batched workload."""
    H, W = x.shape
    ph, pw = psf.shape
    lr, lc = ph // 2, pw // 2
    out = np.zeros((H, W))
    Hv, Wv = H - 2 * lr, W - 2 * lc
    if Hv <= 0 or Wv <= 0:
        return out
    fh, fw = H + ph - 1, W + pw - 1
    full = np.fft.irfft2(np.fft.rfft2(x, (fh, fw)) * np.fft.rfft2(psf, (fh, fw)), (fh, fw))
    # full[i, j] = sum psf[a', b'] x[i - a', j - b']; the valid output at
    # (r, c) is full[r + lr, c + lc] for r in [lr, H - lr)
    out[lr:lr + Hv, lc:lc + Wv] = full[2 * lr:2 * lr + Hv, 2 * lc:2 * lc + Wv]
    return out


def observe(x: np.ndarray, psf: np.ndarray, keep: np.ndarray | None,
            bsnr_db: float, g: np.random.Generator, fast: bool = False):
    """Blur x (valid region only), drop the pixels outside ``keep`` and add
    white Gaussian noise whose variance gives the requested BSNR
    = 10 log10(var(blurred observed pixels) / sigma^2)."""
    H, W = x.shape
    vm = valid_mask(H, W, *psf.shape)
    mask = vm if keep is None else (vm & keep.astype(np.uint8))
    blurred = conv_valid_fft(x, psf) if fast else conv_valid(x, psf)
    obs = mask.astype(bool)
    v = blurred[obs].var() if obs.any() else 0.0
    sigma = math.sqrt(v / (10.0 ** (bsnr_db / 10.0))) if v > 0 else 0.0
    noise = g.standard_normal((H, W)) * sigma
    ybar = np.where(obs, blurred + noise, 0.0)
    return ybar, mask, sigma


def default_mu(lam: float):
    """Penalty rule: mu2 = 10 lambda as in Sec. V; the printed mu1 rule is
    garbled and stated for an unknown intensity scale, and the penalties only
    change the speed of convergence (Theorem 1), so mu1 = min(1, 3 mu2), the
    fastest of the oracle sweep on [0, 1]-scaled images."""
    mu2 = 10.0 * lam
    return min(1.0, 3.0 * mu2), mu2


def config1_problem(seed: int = 0) -> Problem:
    """64 x 64 piecewise-constant image, 9 x 9 box blur, valid region only,
    BSNR 40 dB, TV, lambda = 1e-3, mu2 = 1e-2, mu1 = 1."""
    g = rng(seed)
    x = shapes_image(64, 64, g, 20, rmax=16.0)
    psf = psf_box(9)
    ybar, mask, sigma = observe(x, psf, None, 40.0, g)
    return Problem(x, psf, ybar, mask, sigma, 1e-3, 1.0, 1e-2, "tv",
                   {"config": "tv64_box9_bsnr40"})


# lambda per (blur, BSNR) for the 512 x 512 TV inpainting workload: the best
# converged oracle ISNR on one 128 x 128 calibration image (seed 1000) over
# {1e-5, 3e-5, 1e-4, 3e-4, 1e-3, 3e-3}, among the values whose run met
# rel-x < 1e-5 within 3000 iterations; the paper tuned lambda per condition
# for the best ISNR (Sec. V). oracle/calibrate_lambda.py
CONFIG2_LAMBDA = {("gauss", 40): 1e-5, ("gauss", 60): 1e-5,
                  ("motion", 40): 3e-5, ("motion", 60): 1e-5}


def config2_problem(seed: int = 0, blur: str = "gauss", bsnr: int = 40,
                    size: int = 512, missing: float = 0.4) -> Problem:
    """size^2 textured image; 19x19 Gaussian (sigma 3) or 15-px motion blur at
    30 degrees; valid region AND Bernoulli(1 - missing) kept interior pixels;
    BSNR 40 or 60 dB; TV."""
    g = rng(seed)
    x = textured_image(size, size, g)
    psf = psf_gaussian(19, 3.0) if blur == "gauss" else psf_motion(15.0, 30.0, 15)
    keep = (g.uniform(0.0, 1.0, size=(size, size)) >= missing).astype(np.uint8)
    ybar, mask, sigma = observe(x, psf, keep, float(bsnr), g)
    lam = CONFIG2_LAMBDA[(blur, int(bsnr))]
    mu1, mu2 = default_mu(lam)
    return Problem(x, psf, ybar, mask, sigma, lam, mu1, mu2, "tv",
                   {"config": f"tv{size}_{blur}_bsnr{bsnr}_miss{missing}"})


# lambda of the synthesis prior (FS-MD) on the frame workload, by the same rule
# (best converged oracle ISNR) on one 128 x 128 calibration image of that
# workload (13 x 13 box, valid region, 50 dB); oracle/calibrate_lambda.py,
# run with `frame`. On that image every lambda from 1e-5 to 1e-1 leaves the
# synthesis prior's ISNR below zero (best -1.45 dB at 3e-3); the analysis
# prior's best converged value there is 3e-5 (14.0 dB), next to this
# workload's 5e-5.
FS_FRAME_LAMBDA = 3e-3


def config3_problem(seed: int = 0, size: int = 1024, lam: float = 5e-5) -> Problem:
    """size^2 textured image, 13 x 13 uniform blur, valid region only,
    BSNR 50 dB, 4-level undecimated Haar analysis prior."""
    g = rng(seed)
    x = textured_image(size, size, g)
    psf = psf_box(13)
    ybar, mask, sigma = observe(x, psf, None, 50.0, g)
    mu1, mu2 = default_mu(lam)
    return Problem(x, psf, ybar, mask, sigma, lam, mu1, mu2, "haar",
                   {"config": f"haar{size}_box13_bsnr50"})


# --------------------------------------------------------------------------
# batched uneven workload
# --------------------------------------------------------------------------
CONFIG4_SIZES = (128, 256, 384, 512, 1024)

# lambda per (regularizer, blur family) at BSNR 40, by the same rule on one
# 128 x 128 calibration image per family (box 13, Gaussian 17 sigma 2.5,
# motion 15 px at 30 degrees, 25 % missing); oracle/calibrate_lambda.py
CONFIG4_LAMBDA = {("tv", "box"): 3e-5, ("tv", "gauss"): 1e-5, ("tv", "motion"): 3e-5,
                  ("haar", "box"): 1e-4, ("haar", "gauss"): 1e-4, ("haar", "motion"): 1e-4}


def fft_domain(n: int) -> int:
    """Smallest power of two >= n (at least 64): the unknown domain a side of
    n pixels is solved on. The extra rows and columns are more unknown
    boundary, never observed (Sec. IV-A: the domain only has to hold the
    image and the kernel support)."""
    d = 64
    while d < n:
        d *= 2
    return d


def config4_psf(g: np.random.Generator):
    """One kernel from the batched workload's law: box (odd side 5..21),
    Gaussian (sigma U[1, 4], side 2 ceil(3 sigma) + 1) or motion (length
    U{5..25} at angle U[0, 180) degrees, odd side >= length), each with
    probability 1/3. Returns (psf, family)."""
    kind = int(g.integers(3))
    if kind == 0:
        side = 2 * int(g.integers(2, 11)) + 1
        return psf_box(side), "box"
    if kind == 1:
        sigma = float(g.uniform(1.0, 4.0))
        return psf_gaussian(2 * math.ceil(3.0 * sigma) + 1, sigma), "gauss"
    length = int(g.integers(5, 26))
    angle = float(g.uniform(0.0, 180.0))
    return psf_motion(float(length), angle, length + 1 - length % 2), "motion"


def config4_problem(g: np.random.Generator, size: int | None = None, reg: str | None = None,
                    pad: bool = True) -> Problem:
    """One problem of the batched uneven workload: side uniform over
    CONFIG4_SIZES, kernel from config4_psf, missing fraction U[0, 0.5],
    TV or 4-level Haar with probability 1/2, BSNR 40 dB, textured image.
    With pad = True a side that is not a power of two is embedded in the
    padded domain fft_domain(side): the image sits in the top-left corner and
    the padding is unobserved; meta["window"] is the image's side, x_true is
    zero on the padding. With pad = False the problem keeps its own side
    (solved on the exact domain). The random draws do not depend on pad."""
    if size is None:
        size = CONFIG4_SIZES[int(g.integers(len(CONFIG4_SIZES)))]
    psf, family = config4_psf(g)
    missing = float(g.uniform(0.0, 0.5))
    r = ("tv" if g.uniform() < 0.5 else "haar")
    reg = reg or r
    x = textured_image(size, size, g)
    keep = (g.uniform(0.0, 1.0, size=(size, size)) >= missing).astype(np.uint8)
    ybar, mask, sigma = observe(x, psf, keep, 40.0, g, fast=True)
    N = fft_domain(size) if pad else size
    if N != size:
        xp = np.zeros((N, N))
        yp = np.zeros((N, N))
        mp = np.zeros((N, N), dtype=np.uint8)
        xp[:size, :size] = x
        yp[:size, :size] = ybar
        mp[:size, :size] = mask
        x, ybar, mask = xp, yp, mp
    lam = CONFIG4_LAMBDA[(reg, family)]
    mu1, mu2 = default_mu(lam)
    return Problem(x, psf, ybar, mask, sigma, lam, mu1, mu2, reg,
                   {"config": f"{reg}{size}_{family}{psf.shape[0]}_miss{missing:.2f}",
                    "window": size, "family": family, "missing": missing})


def config4_batch(seed: int = 0, count: int = 256, sizes=None, pad: bool = True) -> list:
    """``count`` problems of the batched uneven workload from one stream;
    ``sizes`` (optional) restricts the side law to a subset; ``pad`` as in
    config4_problem."""
    g = rng(seed)
    out = []
    for _ in range(count):
        size = None
        if sizes is not None:
            size = sizes[int(g.integers(len(sizes)))]
        out.append(config4_problem(g, size, pad=pad))
    return out
