"""Plain FP64 CPU oracle for mask-decoupled ADMM deconvolution (TV-MD, FA-MD).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this
package; only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it. It shares no code with the CUDA path.

It follows M. S. C. Almeida and M. A. T. Figueiredo, "Deconvolving Images with
Unknown Boundaries Using the Alternating Direction Method of Multipliers":

* observation model  y = M A x + n                     (Sec. IV-A, eq. model_unknown_BC)
* ADMM-2 (Algorithm 2) with the mask-decoupled g1 of eq. g_1_uBC, whose prox is
  eq. prox_g_1_uBC
* TV-MD  = Algorithm 3 (ADMM-TV) with line 7 replaced by eq. new_line (Sec. IV-D)
* FA-MD  = Algorithm 2 with H1 = A, H2 = P, x-step eqs. invAnalysis/invAnalysisp1
  and the soft threshold of eq. soft (Sec. IV-C)
* FS-MD  = Algorithm 2 on the synthesis formulation (Sec. IV-B, eq.
  unconstrained_synthesis_uBC): unknown theta, x = P^T theta, H1 = A P^T,
  H2 = I, line 4 by eq. inverse_synth2
* TV-CG, FA-CG = the Reeves-Sorel variants (Sec. IV-D and IV-C, "Using the
  Reeves-Sorel technique"): H1 = M A with g1(u) = 1/2 ||y - u||^2, the x-step
  inverse applied as C - C B^T (B C B^T - I)^{-1} B C (eqs. ReevesTV, reeves3)
  with one conjugate-gradient iteration per outer iteration, warm-started
  from the previous one (Sec. IV-B, "Using the Reeves-Sorel technique")

Conventions (readings of points the paper leaves open; each is listed with
its justification in the design notes):

* DFT: the oracle's own, written out as its definition: the 2-D DFT of an
  H x W array is F_H X F_W with the DFT matrices F_N[j, k] = exp(-2 pi i j k / N)
  (unnormalised forward), and the inverse is conj(F_H) X conj(F_W) / (H W).
  U of eq. DFT_fact is the unitary version; the diagonal ratios of eq.
  fast_inversion are unchanged. No FFT library is used.
* A is periodic convolution on the full domain with the kernel centred at
  (0, 0):  (A x)[r,c] = sum_{a,b} h[a+l_r, b+l_c] x[(r-a) mod H, (c-b) mod W].
* D^h, D^v are forward periodic differences:
  (D^h x)[r,c] = x[r,(c+1) mod W] - x[r,c],  (D^v x)[r,c] = x[(r+1) mod H,c] - x[r,c].
* P is the 4-level undecimated (a-trous) 2-D Haar frame with periodic wrap;
  level j filters with h = [1/2, 1/2] and g = [1/2, -1/2] at taps {0, 2^j}
  along each axis. Each level emits three detail bands and passes the
  low-low band on; the last low-low band is kept: 3 L + 1 bands. P^T P = I.
* vector-soft maps 0 to 0 (Sec. III-C); soft(v, t) = sign(v) max(|v| - t, 0).
* Variants beyond the paper's two priors: anisotropic TV (the l1 norm of each
  difference component; its prox is eq. soft per component) and the frame
  prior with the last low-low band unpenalised (its prox is the identity).

Every function below is written to be checked by eye against the equation
it cites, not for speed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "dft2", "idft2", "psf_otf", "A_fft", "At_fft", "A_direct", "At_direct",
    "Dh", "Dv", "DhT", "DvT", "tv_denominator_diag",
    "haar_analysis", "haar_synthesis", "haar_nbands", "haar_band_spectra",
    "soft", "vsoft", "mask_prox",
    "objective_tv", "objective_haar", "objective_synthesis",
    "State", "tvmd_step", "famd_step", "fsmd_step", "tvcg_step", "facg_step", "solve",
    "isnr", "snr",
]


# --------------------------------------------------------------------------
# the discrete Fourier transform (Sec. III-C: U and U* of eq. DFT_fact, up to
# the 1/sqrt(n) normalisation), by its definition
# --------------------------------------------------------------------------
_DFT_CACHE: dict = {}


def _dft_matrix(N: int) -> np.ndarray:
    """F_N[j, k] = exp(-2 pi i j k / N); the exponent is reduced as (j k mod N)
    so that every entry is one of the N exact N-th roots of unity."""
    F = _DFT_CACHE.get(N)
    if F is None:
        jk = np.mod(np.outer(np.arange(N), np.arange(N)), N)
        F = np.exp(-2j * np.pi * jk / N)
        _DFT_CACHE[N] = F
    return F


def dft2(x: np.ndarray) -> np.ndarray:
    """X[kr, kc] = sum_{r, c} x[r, c] exp(-2 pi i (kr r / H + kc c / W))."""
    H, W = x.shape
    return _dft_matrix(H) @ np.asarray(x, dtype=np.complex128) @ _dft_matrix(W)


def idft2(X: np.ndarray) -> np.ndarray:
    """x[r, c] = (1 / (H W)) sum_{kr, kc} X[kr, kc] exp(+2 pi i (kr r / H + kc c / W))."""
    H, W = X.shape
    return (np.conj(_dft_matrix(H)) @ np.asarray(X, dtype=np.complex128) @ np.conj(_dft_matrix(W))) / (H * W)


# --------------------------------------------------------------------------
# circulant operators (Sec. III-C, eq. DFT_fact: A = U* Lambda U)
# --------------------------------------------------------------------------
def _centred_kernel(psf: np.ndarray, H: int, W: int) -> np.ndarray:
    """The blur kernel laid out on the H x W torus with its centre at (0,0)."""
    ph, pw = psf.shape
    lr, lc = ph // 2, pw // 2
    k = np.zeros((H, W))
    for a in range(-lr, lr + 1):
        for b in range(-lc, lc + 1):
            k[a % H, b % W] += psf[a + lr, b + lc]
    return k


def psf_otf(psf: np.ndarray, H: int, W: int) -> np.ndarray:
    """Lambda: the DFT of the convolution kernel (diagonal of eq. DFT_fact)."""
    return dft2(_centred_kernel(psf, H, W))


def A_fft(x: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """A x = U* Lambda U x (eq. DFT_fact)."""
    H, W = x.shape
    return np.real(idft2(psf_otf(psf, H, W) * dft2(x)))


def At_fft(x: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """A^T x = U* conj(Lambda) U x."""
    H, W = x.shape
    return np.real(idft2(np.conj(psf_otf(psf, H, W)) * dft2(x)))


def A_direct(x: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """Periodic convolution by its definition, one kernel tap at a time."""
    ph, pw = psf.shape
    lr, lc = ph // 2, pw // 2
    out = np.zeros_like(x, dtype=np.float64)
    for a in range(-lr, lr + 1):
        for b in range(-lc, lc + 1):
            # x[(r-a) mod H, (c-b) mod W] is np.roll(x, (a, b))
            out += psf[a + lr, b + lc] * np.roll(x, (a, b), axis=(0, 1))
    return out


def At_direct(x: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """Adjoint of A_direct: periodic correlation with the same taps."""
    ph, pw = psf.shape
    lr, lc = ph // 2, pw // 2
    out = np.zeros_like(x, dtype=np.float64)
    for a in range(-lr, lr + 1):
        for b in range(-lc, lc + 1):
            out += psf[a + lr, b + lc] * np.roll(x, (-a, -b), axis=(0, 1))
    return out


# --------------------------------------------------------------------------
# TV differences (Sec. III-C: D_i = horizontal and vertical differences,
# periodic BC)
# --------------------------------------------------------------------------
def Dh(x):
    return np.roll(x, -1, axis=1) - x


def Dv(x):
    return np.roll(x, -1, axis=0) - x


def DhT(p):
    return np.roll(p, 1, axis=1) - p


def DvT(p):
    return np.roll(p, 1, axis=0) - p


def tv_denominator_diag(psf, H, W, mu1, mu2):
    """Diagonal of eq. fast_inversion: mu1|Lambda|^2 + mu2|Delta^h|^2 + mu2|Delta^v|^2,
    with Delta^h, Delta^v the DFTs of the difference kernels."""
    lam = psf_otf(psf, H, W)
    eh = np.zeros((H, W)); eh[0, 0] = -1.0; eh[0, (-1) % W] += 1.0   # D^h x = e_h (*) x
    ev = np.zeros((H, W)); ev[0, 0] = -1.0; ev[(-1) % H, 0] += 1.0
    dh = dft2(eh)
    dv = dft2(ev)
    return mu1 * np.abs(lam) ** 2 + mu2 * np.abs(dh) ** 2 + mu2 * np.abs(dv) ** 2


# --------------------------------------------------------------------------
# undecimated Haar Parseval frame (Sec. V: redundant Haar frame, 4 levels;
# Sec. III-B requires P^T P = I)
# --------------------------------------------------------------------------
def haar_nbands(levels: int) -> int:
    return 3 * levels + 1


def _lo(v, s, axis):
    return 0.5 * (v + np.roll(v, -s, axis=axis))


def _hi(v, s, axis):
    return 0.5 * (v - np.roll(v, -s, axis=axis))


def _loT(v, s, axis):
    return 0.5 * (v + np.roll(v, s, axis=axis))


def _hiT(v, s, axis):
    return 0.5 * (v - np.roll(v, s, axis=axis))


def haar_analysis(x: np.ndarray, levels: int = 4) -> np.ndarray:
    """P x as an array (3 L + 1, H, W). Band order for level j: [rows low /
    columns high, rows high / columns low, rows high / columns high]; the
    final band is the low-low approximation. 'columns high' means the
    high-pass acts along the column index (axis 1)."""
    bands = []
    a = np.asarray(x, dtype=np.float64)
    for j in range(levels):
        s = 1 << j
        lo_c = _lo(a, s, 1)
        hi_c = _hi(a, s, 1)
        bands.append(_lo(hi_c, s, 0))
        bands.append(_hi(lo_c, s, 0))
        bands.append(_hi(hi_c, s, 0))
        a = _lo(lo_c, s, 0)
    bands.append(a)
    return np.stack(bands)


def haar_synthesis(c: np.ndarray, levels: int = 4) -> np.ndarray:
    """P^T c, the adjoint of haar_analysis."""
    a = c[3 * levels].copy()
    for j in reversed(range(levels)):
        s = 1 << j
        b0, b1, b2 = c[3 * j], c[3 * j + 1], c[3 * j + 2]
        lo_c = _loT(a, s, 0) + _hiT(b1, s, 0)
        hi_c = _loT(b0, s, 0) + _hiT(b2, s, 0)
        a = _loT(lo_c, s, 1) + _hiT(hi_c, s, 1)
    return a


# --------------------------------------------------------------------------
# proximity operators
# --------------------------------------------------------------------------
def soft(v, tau):
    """eq. soft: sign(v) * max(|v| - tau, 0), componentwise."""
    return np.sign(v) * np.maximum(np.abs(v) - tau, 0.0)


def vsoft(vh, vv, tau):
    """vector-soft of Sec. III-C applied per pixel to (vh, vv), with 0/0 = 0:
    v / ||v|| * max(||v|| - tau, 0)."""
    nrm = np.sqrt(vh * vh + vv * vv)
    scale = np.where(nrm > tau, (nrm - tau) / np.where(nrm > 0, nrm, 1.0), 0.0)
    return scale * vh, scale * vv


def mask_prox(v, ybar, mask, mu1):
    """eq. prox_g_1_uBC: (M^T M + mu1 I)^{-1} (M^T y + mu1 v); M^T M = diag(mask),
    M^T y = ybar (observations zero-extended to the full domain)."""
    m = mask.astype(np.float64)
    return (m * ybar + mu1 * v) / (m + mu1)


# --------------------------------------------------------------------------
# objectives (eq. unconstrained_TV_uBC and eq. unconstrained_analysis_uBC)
# --------------------------------------------------------------------------
def objective_tv(x, ybar, mask, psf, lam, aniso=False):
    """Isotropic TV: lam sum_i ||(Dh x, Dv x)_i||; anisotropic (aniso=True):
    lam sum_i (|Dh x|_i + |Dv x|_i)."""
    m = mask.astype(np.float64)
    r = m * (ybar - A_fft(x, psf))
    gh, gv = Dh(x), Dv(x)
    reg = np.abs(gh) + np.abs(gv) if aniso else np.sqrt(gh ** 2 + gv ** 2)
    return 0.5 * float(np.sum(r * r)) + lam * float(np.sum(reg))


def objective_synthesis(theta, ybar, mask, psf, lam):
    """Frame synthesis prior (FS, eq. unconstrained_synthesis_uBC):
    1/2 ||M(y - A W theta)||^2 + lam ||theta||_1 with W = P^T."""
    m = mask.astype(np.float64)
    r = m * (ybar - A_fft(haar_synthesis(theta, theta.shape[0] // 3), psf))
    return 0.5 * float(np.sum(r * r)) + lam * float(np.sum(np.abs(theta)))


def objective_haar(x, ybar, mask, psf, lam, levels=4, ll_free=False):
    """lam ||P x||_1 over all 3 L + 1 bands, or (ll_free=True) over the 3 L
    detail bands only (the coarse low-low band unpenalised)."""
    m = mask.astype(np.float64)
    r = m * (ybar - A_fft(x, psf))
    c = haar_analysis(x, levels)
    if ll_free:
        c = c[:-1]
    return 0.5 * float(np.sum(r * r)) + lam * float(np.sum(np.abs(c)))


# --------------------------------------------------------------------------
# ADMM iterations
# --------------------------------------------------------------------------
@dataclass
class State:
    """ADMM split and dual variables. TV: u2/d2 have shape (2, H, W) holding
    the (horizontal, vertical) components; Haar: (3 L + 1, H, W)."""
    u1: np.ndarray
    d1: np.ndarray
    u2: np.ndarray
    d2: np.ndarray
    x: np.ndarray
    k: int = 0
    theta: np.ndarray | None = None    # synthesis coefficients (FS-MD only)
    xi: np.ndarray | None = None       # TV-CG / FA-CG: the conjugate-gradient iterate of
                                       # (B C B^T - I) xi = B C r, one entry per unobserved
                                       # pixel, stored on the full grid (0 elsewhere)

    @staticmethod
    def zeros(H, W, reg="tv", levels=4):
        nb = 2 if reg in ("tv", "tv_aniso") else haar_nbands(levels)
        z = np.zeros((H, W))
        return State(z.copy(), z.copy(), np.zeros((nb, H, W)), np.zeros((nb, H, W)), z.copy(), 0)

    def copy(self):
        return State(self.u1.copy(), self.d1.copy(), self.u2.copy(), self.d2.copy(),
                     self.x.copy(), self.k, None if self.theta is None else self.theta.copy(),
                     None if self.xi is None else self.xi.copy())


def tvmd_step(st: State, ybar, mask, psf, lam, mu1, mu2, otf=None, denom=None, aniso=False) -> State:
    """One iteration of TV-MD: Algorithm 3 with line 7 replaced by eq. new_line.
    aniso=True: anisotropic TV, whose prox (lines 9-10) is the soft threshold
    of eq. soft applied to each difference component instead of vector-soft."""
    H, W = ybar.shape
    if otf is None:
        otf = psf_otf(psf, H, W)
    if denom is None:
        denom = tv_denominator_diag(psf, H, W, mu1, mu2)
    # Alg. 3, lines 3-5: zeta = u_k + d_k, split into zeta1 and (delta_h, delta_v)
    zeta1 = st.u1 + st.d1
    delta_h = st.u2[0] + st.d2[0]
    delta_v = st.u2[1] + st.d2[1]
    # line 6: z = K (mu1 A^T zeta1 + mu2 Dh^T delta_h + mu2 Dv^T delta_v), K of eq. fast_inversion
    rhs = mu1 * np.real(idft2(np.conj(otf) * dft2(zeta1))) \
        + mu2 * DhT(delta_h) + mu2 * DvT(delta_v)
    x = np.real(idft2(dft2(rhs) / denom))
    # line 7 -> eq. new_line: u1 = (M^T M + mu1 I)^{-1} (M^T y + mu1 (A z - d1))
    ax = np.real(idft2(otf * dft2(x)))
    u1 = mask_prox(ax - st.d1, ybar, mask, mu1)
    # line 8: d1 = d1 - (A z - u1)
    d1 = st.d1 - (ax - u1)
    # lines 9-11: per pixel vector-soft and dual update
    gh, gv = Dh(x), Dv(x)
    if aniso:
        uh, uv = soft(gh - st.d2[0], lam / mu2), soft(gv - st.d2[1], lam / mu2)
    else:
        uh, uv = vsoft(gh - st.d2[0], gv - st.d2[1], lam / mu2)
    d2 = np.stack([st.d2[0] - (gh - uh), st.d2[1] - (gv - uv)])
    return State(u1, d1, np.stack([uh, uv]), d2, x, st.k + 1)


def haar_band_spectra(H, W, levels=4):
    """|DFT|^2 of each band's filter: the bands of P applied to a unit
    impulse at (0, 0), transformed (P_b is a periodic convolution, so
    P_b^T P_b is the circulant with this diagonal). Shape (3 L + 1, H, W)."""
    e = np.zeros((H, W))
    e[0, 0] = 1.0
    return np.stack([np.abs(dft2(b)) ** 2 for b in haar_analysis(e, levels)])


def famd_step(st: State, ybar, mask, psf, lam, mu1, mu2, levels=4, otf=None, ll_free=False,
              mu_bands=None) -> State:
    """One iteration of FA-MD: Algorithm 2 with H1 = A, H2 = P, line 4 from
    eqs. invAnalysis/invAnalysisp1 and line 6 from eqs. prox_g_1_uBC and prox_g_2.
    ll_free=True leaves the last (low-low) band unpenalised: its prox is the
    identity (a threshold of zero). mu_bands (3 L + 1 values, optional): one
    penalty per band instead of mu2 for all, i.e. Algorithm 2 with J = 3 L + 2
    functions and the block-diagonal Upsilon of eq. diagonal_penalty; line 4 is
    then eq. quadratic_problem, (mu1 A^T A + sum_b mu_b P_b^T P_b)^{-1}
    (mu1 A^T zeta1 + sum_b mu_b P_b^T zeta_b), diagonal in the DFT domain since
    each P_b is a convolution, and band b is thresholded at lambda / mu_b."""
    H, W = ybar.shape
    if otf is None:
        otf = psf_otf(psf, H, W)
    if mu_bands is not None:
        mub = np.asarray(mu_bands, dtype=np.float64)
        gb = mub / mu1
        zeta1 = st.u1 + st.d1
        zeta2 = st.u2 + st.d2
        rhs = np.real(idft2(np.conj(otf) * dft2(zeta1))) + haar_synthesis(gb[:, None, None] * zeta2, levels)
        denom = np.abs(otf) ** 2 + np.tensordot(gb, haar_band_spectra(H, W, levels), axes=1)
        x = np.real(idft2(dft2(rhs) / denom))
        ax = np.real(idft2(otf * dft2(x)))
        u1 = mask_prox(ax - st.d1, ybar, mask, mu1)
        d1 = st.d1 - (ax - u1)
        c = haar_analysis(x, levels)
        u2 = soft(c - st.d2, (lam / mub)[:, None, None])
        if ll_free:
            u2[-1] = c[-1] - st.d2[-1]
        d2 = st.d2 - (c - u2)
        return State(u1, d1, u2, d2, x, st.k + 1)
    gam = mu2 / mu1
    # line 3
    zeta1 = st.u1 + st.d1
    zeta2 = st.u2 + st.d2
    # line 4 with P^T P = I: z = U* (|Lambda|^2 + gamma)^{-1} U (A^T zeta1 + gamma P^T zeta2)
    rhs = np.real(idft2(np.conj(otf) * dft2(zeta1))) + gam * haar_synthesis(zeta2, levels)
    x = np.real(idft2(dft2(rhs) / (np.abs(otf) ** 2 + gam)))
    # lines 6-7, j = 1: mask-decoupled prox and dual update
    ax = np.real(idft2(otf * dft2(x)))
    u1 = mask_prox(ax - st.d1, ybar, mask, mu1)
    d1 = st.d1 - (ax - u1)
    # lines 6-7, j = 2: soft threshold of the frame coefficients
    c = haar_analysis(x, levels)
    u2 = soft(c - st.d2, lam / mu2)
    if ll_free:
        u2[-1] = c[-1] - st.d2[-1]
    d2 = st.d2 - (c - u2)
    return State(u1, d1, u2, d2, x, st.k + 1)


def fsmd_step(st: State, ybar, mask, psf, lam, mu1, mu2, levels=4, otf=None) -> State:
    """One iteration of FS-MD (Sec. IV-B): Algorithm 2 on the synthesis
    formulation, the unknown being the frame coefficients theta with
    x = W theta, W = P^T, H1 = A W and H2 = I (eqs. H_1_synth, H_2_synth).
    Line 4 (eq. inverse_synth2) solves (W^T A^T A W + gamma I) theta = r,
    r = W^T A^T zeta1 + gamma zeta2, with the Sherman-Morrison-Woodbury form
    that W W^T = I allows (eq. inverse_synth):
        theta = (r - W^T A^T (A A^T + gamma I)^{-1} A W r) / gamma,
    (A A^T + gamma I)^{-1} diagonal in the DFT domain. Line 6: the mask prox
    for u1 and the soft threshold of eq. soft for u2 = prox(theta - d2)."""
    H, W = ybar.shape
    if otf is None:
        otf = psf_otf(psf, H, W)
    gam = mu2 / mu1
    zeta1 = st.u1 + st.d1
    zeta2 = st.u2 + st.d2
    r = haar_analysis(np.real(idft2(np.conj(otf) * dft2(zeta1))), levels) + gam * zeta2
    awr = dft2(haar_synthesis(r, levels)) * otf
    q = np.real(idft2(np.conj(otf) * awr / (np.abs(otf) ** 2 + gam)))
    theta = (r - haar_analysis(q, levels)) / gam
    x = haar_synthesis(theta, levels)
    ax = np.real(idft2(otf * dft2(x)))
    u1 = mask_prox(ax - st.d1, ybar, mask, mu1)
    d1 = st.d1 - (ax - u1)
    u2 = soft(theta - st.d2, lam / mu2)
    d2 = st.d2 - (theta - u2)
    return State(u1, d1, u2, d2, x, st.k + 1, theta)


def reeves_sorel_xstep(r, mask, psf, denom, xi_prev, cg_iters=1, otf=None):
    """x = C r - C B^T xi with xi ~ (B C B^T - I)^{-1} B C r (eqs. ReevesTV and
    reeves3, Sec. IV-B's eq. reeves): C is the circulant inverse whose DFT
    diagonal is 1 / denom; B holds the rows of A at the unobserved pixels
    (mask == 0), so B v = (A v) on those pixels and B^T w = A^T of w placed on
    them. The system for xi is solved by `cg_iters` conjugate-gradient
    iterations started from xi_prev (Sec. IV-B: one iteration, warm-started).
    B C B^T - I is negative definite; CG on it takes the same steps as on its
    negation. Returns (x, xi)."""
    H, W = r.shape
    if otf is None:
        otf = psf_otf(psf, H, W)
    unobs = mask == 0

    def C(v):
        return np.real(idft2(dft2(v) / denom))

    def B(v):
        return np.real(idft2(otf * dft2(v)))[unobs]

    def Bt(w):
        full = np.zeros((H, W))
        full[unobs] = w
        return np.real(idft2(np.conj(otf) * dft2(full)))

    def S(w):                      # (B C B^T - I) w
        return B(C(Bt(w))) - w

    Cr = C(r)
    b = B(Cr)
    xi = xi_prev[unobs].copy()
    res = b - S(xi)
    p = res.copy()
    rr = float(res @ res)
    for _ in range(cg_iters):
        if rr == 0.0:
            break
        Sp = S(p)
        alpha = rr / float(p @ Sp)
        xi = xi + alpha * p
        res = res - alpha * Sp
        rr_new = float(res @ res)
        p = res + (rr_new / rr) * p
        rr = rr_new
    x = Cr - C(Bt(xi))
    xi_full = np.zeros((H, W))
    xi_full[unobs] = xi
    return x, xi_full


def tvcg_step(st: State, ybar, mask, psf, lam, mu1, mu2, otf=None, denom=None, cg_iters=1) -> State:
    """One iteration of TV-CG (Sec. IV-D, "Using the Reeves-Sorel technique"):
    Algorithm 3 with H1 = M A (eq. H_1_analysis_sorel), g1(u) = 1/2 ||y - u||^2
    (eq. g_1), so that in line 6 A^T becomes A^T M^T and K is eq. ReevesTV,
    and in line 8 A becomes M A. u1 and d1 live on the observed pixels only
    (zero elsewhere in these full-grid arrays)."""
    H, W = ybar.shape
    if otf is None:
        otf = psf_otf(psf, H, W)
    gam = mu2 / mu1
    if denom is None:
        denom = tv_denominator_diag(psf, H, W, 1.0, gam)     # C^{-1} = A^T A + gamma D^T D
    obs = mask != 0
    xi_prev = st.xi if st.xi is not None else np.zeros((H, W))
    # lines 3-5
    zeta1 = np.where(obs, st.u1 + st.d1, 0.0)               # M^T zeta1
    delta_h = st.u2[0] + st.d2[0]
    delta_v = st.u2[1] + st.d2[1]
    # line 6: x = K (mu1 A^T M^T zeta1 + mu2 D^T delta), K = (1/mu1)(C - C B^T (B C B^T - I)^{-1} B C)
    r = np.real(idft2(np.conj(otf) * dft2(zeta1))) + gam * (DhT(delta_h) + DvT(delta_v))
    x, xi = reeves_sorel_xstep(r, mask, psf, denom, xi_prev, cg_iters, otf)
    # line 7 with g1 = 1/2 ||y - u||^2: u1 = (y + mu1 (M A x - d1)) / (1 + mu1)
    max_ = np.where(obs, np.real(idft2(otf * dft2(x))), 0.0)
    u1 = np.where(obs, (ybar + mu1 * (max_ - st.d1)) / (1.0 + mu1), 0.0)
    # line 8 with M A: d1 = d1 - (M A x - u1)
    d1 = np.where(obs, st.d1 - (max_ - u1), 0.0)
    # lines 9-11 unchanged
    gh, gv = Dh(x), Dv(x)
    uh, uv = vsoft(gh - st.d2[0], gv - st.d2[1], lam / mu2)
    d2 = np.stack([st.d2[0] - (gh - uh), st.d2[1] - (gv - uv)])
    return State(u1, d1, np.stack([uh, uv]), d2, x, st.k + 1, None, xi)


def facg_step(st: State, ybar, mask, psf, lam, mu1, mu2, levels=4, otf=None, cg_iters=1) -> State:
    """One iteration of FA-CG (Sec. IV-C, "Using the Reeves-Sorel technique"):
    Algorithm 2 with H1 = M A (eq. H_1_analysis_sorel), H2 = P, g1(u) =
    1/2 ||y - u||^2; line 4 is eq. invAnalysis_sorel applied as eq. reeves3,
    C = (gamma I + A^T A)^{-1}; line 6 the prox of g1 and eq. soft."""
    H, W = ybar.shape
    if otf is None:
        otf = psf_otf(psf, H, W)
    gam = mu2 / mu1
    obs = mask != 0
    xi_prev = st.xi if st.xi is not None else np.zeros((H, W))
    zeta1 = np.where(obs, st.u1 + st.d1, 0.0)
    zeta2 = st.u2 + st.d2
    r = np.real(idft2(np.conj(otf) * dft2(zeta1))) + gam * haar_synthesis(zeta2, levels)
    x, xi = reeves_sorel_xstep(r, mask, psf, np.abs(otf) ** 2 + gam, xi_prev, cg_iters, otf)
    max_ = np.where(obs, np.real(idft2(otf * dft2(x))), 0.0)
    u1 = np.where(obs, (ybar + mu1 * (max_ - st.d1)) / (1.0 + mu1), 0.0)
    d1 = np.where(obs, st.d1 - (max_ - u1), 0.0)
    c = haar_analysis(x, levels)
    u2 = soft(c - st.d2, lam / mu2)
    d2 = st.d2 - (c - u2)
    return State(u1, d1, u2, d2, x, st.k + 1, None, xi)


@dataclass
class SolveResult:
    x: np.ndarray
    state: State
    iters: int
    converged: bool
    objective: float
    rel_x: float
    rel_obj: float
    history: list = field(default_factory=list)


def solve(ybar, mask, psf, lam, mu1, mu2, reg="tv", iters=200, stop="iters", tol=0.0,
          levels=4, state0: State | None = None, record=False, mu_bands=None) -> SolveResult:
    """Run TV-MD or FA-MD from ``state0`` (default: u0 = d0 = 0) until ``iters``
    iterations or, for stop = 'rel_x' / 'rel_obj', until the relative change of
    x / of the objective between consecutive iterations is below ``tol``.
    reg: 'tv', 'tv_aniso' (anisotropic TV), 'haar', 'haar_ll_free' (the
    low-low band unpenalised), 'haar_synthesis' (FS-MD: the frame synthesis
    prior; its objective is evaluated on the coefficients theta), 'tv_cg',
    'haar_cg' (the Reeves-Sorel variants TV-CG and FA-CG)."""
    H, W = ybar.shape
    tv = reg in ("tv", "tv_aniso", "tv_cg")
    aniso, ll_free, fs = reg == "tv_aniso", reg == "haar_ll_free", reg == "haar_synthesis"
    cg = reg in ("tv_cg", "haar_cg")
    st = state0.copy() if state0 is not None else State.zeros(H, W, "tv" if tv else "haar", levels)
    otf = psf_otf(psf, H, W)
    if reg == "tv_cg":
        denom = tv_denominator_diag(psf, H, W, 1.0, mu2 / mu1)
    else:
        denom = tv_denominator_diag(psf, H, W, mu1, mu2) if tv else None
    if fs:
        obj_fn = lambda x: objective_synthesis(st.theta, ybar, mask, psf, lam)  # noqa: E731
    elif tv:
        obj_fn = lambda x: objective_tv(x, ybar, mask, psf, lam, aniso)  # noqa: E731
    else:
        obj_fn = lambda x: objective_haar(x, ybar, mask, psf, lam, levels, ll_free)  # noqa: E731
    hist = []
    f_prev = None
    rel_x = rel_obj = float("inf")
    converged = False
    n = 0
    for n in range(1, iters + 1):
        x_prev = st.x
        if reg == "tv_cg":
            st = tvcg_step(st, ybar, mask, psf, lam, mu1, mu2, otf, denom)
        elif reg == "haar_cg":
            st = facg_step(st, ybar, mask, psf, lam, mu1, mu2, levels, otf)
        elif tv:
            st = tvmd_step(st, ybar, mask, psf, lam, mu1, mu2, otf, denom, aniso)
        elif fs:
            st = fsmd_step(st, ybar, mask, psf, lam, mu1, mu2, levels, otf)
        else:
            st = famd_step(st, ybar, mask, psf, lam, mu1, mu2, levels, otf, ll_free, mu_bands)
        nx = float(np.linalg.norm(st.x))
        rel_x = float(np.linalg.norm(st.x - x_prev)) / nx if nx > 0 else float("inf")
        f = obj_fn(st.x) if (stop == "rel_obj" or record) else float("nan")
        if f_prev is not None and f == f:
            rel_obj = abs(f - f_prev) / abs(f) if f != 0 else float("inf")
        f_prev = f
        if record:
            hist.append((n, f, rel_x))
        # the rule compares consecutive iterates of this run: x_1 has no
        # predecessor (from a warm start it is the given x0 itself)
        if stop == "rel_x" and n > 1 and rel_x < tol:
            converged = True
            break
        if stop == "rel_obj" and n > 1 and rel_obj < tol:
            converged = True
            break
    return SolveResult(st.x, st, n, converged, obj_fn(st.x), rel_x, rel_obj, hist)


# --------------------------------------------------------------------------
# figures of merit (Sec. V uses ISNR and SNR without defining them)
# --------------------------------------------------------------------------
def isnr(x_true, ybar, x_hat, region):
    """10 log10(||x - ybar||^2 / ||x - x_hat||^2) over the boolean region."""
    r = region.astype(bool)
    num = np.sum((x_true[r] - ybar[r]) ** 2)
    den = np.sum((x_true[r] - x_hat[r]) ** 2)
    return 10.0 * math.log10(num / den)


def snr(x_true, x_hat):
    return 10.0 * math.log10(np.sum(x_true ** 2) / np.sum((x_true - x_hat) ** 2))
