"""Pins for the FP64 oracle: each check compares it with something other than
itself -- a definition written out as loops, a closed form, an invariant, a
dense linear-algebra solve, an independent convex solver, or a value printed
in the paper. A dropped term, wrong sign, wrong index or transposed operand in
any oracle function fails at least one of these."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_psf(g, ph, pw):
    k = g.uniform(0.0, 1.0, size=(ph, pw))
    k[0, -1] += 2.0          # make it clearly asymmetric
    return k / k.sum()


# ----------------------------------------------------------------------------
# A, A^T, M
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("H,W,ph,pw", [(5, 7, 3, 3), (8, 8, 5, 3), (16, 12, 7, 5), (9, 16, 9, 9)])
def test_convolution_matches_definition_loops(H, W, ph, pw):
    """Periodic convolution (Sec. IV-A: A with periodic BC on the full domain)
    written as explicit index loops equals the FFT-diagonalised A of eq.
    DFT_fact and the tap-sum A_direct; the adjoint equals the correlation."""
    g = S.rng(1)
    x = g.standard_normal((H, W))
    h = _rand_psf(g, ph, pw)
    lr, lc = ph // 2, pw // 2
    ref = np.zeros((H, W))
    reft = np.zeros((H, W))
    for r in range(H):
        for c in range(W):
            s = st = 0.0
            for a in range(-lr, lr + 1):
                for b in range(-lc, lc + 1):
                    s += h[a + lr, b + lc] * x[(r - a) % H, (c - b) % W]
                    st += h[a + lr, b + lc] * x[(r + a) % H, (c + b) % W]
            ref[r, c] = s
            reft[r, c] = st
    np.testing.assert_allclose(O.A_fft(x, h), ref, rtol=0, atol=1e-13)
    np.testing.assert_allclose(O.A_direct(x, h), ref, rtol=0, atol=1e-13)
    np.testing.assert_allclose(O.At_fft(x, h), reft, rtol=0, atol=1e-13)
    np.testing.assert_allclose(O.At_direct(x, h), reft, rtol=0, atol=1e-13)


def test_adjoint_identities():
    """<Ax, y> = <x, A^T y>, and the same for D^h, D^v and the Haar frame."""
    g = S.rng(2)
    H, W = 16, 24
    x = g.standard_normal((H, W))
    y = g.standard_normal((H, W))
    h = _rand_psf(g, 7, 5)
    for fwd, adj in ((lambda v: O.A_fft(v, h), lambda v: O.At_fft(v, h)),
                     (O.Dh, O.DhT), (O.Dv, O.DvT)):
        lhs = np.vdot(fwd(x), y)
        rhs = np.vdot(x, adj(y))
        assert abs(lhs - rhs) <= 1e-13 * max(1.0, abs(lhs))
    c = g.standard_normal((13, H, W))
    lhs = np.vdot(O.haar_analysis(x, 4), c)
    rhs = np.vdot(x, O.haar_synthesis(c, 4))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_periodic_model_equals_valid_convolution():
    """Sec. IV-A: on the valid region the periodic A x equals the
    non-periodic blur used to form observations (so the BC is irrelevant)."""
    g = S.rng(3)
    x = g.uniform(size=(40, 33))
    h = S.psf_motion(9.0, 30.0, 9)
    vm = S.valid_mask(40, 33, 9, 9).astype(bool)
    np.testing.assert_allclose(O.A_fft(x, h)[vm], S.conv_valid(x, h)[vm], rtol=0, atol=1e-13)


def test_paper_valid_region_sizes():
    """Sec. V: 256 x 256 image with 19 x 19 blurs gives a 238 x 238 observed
    region, m = 56644 and 8892 unknown boundary pixels."""
    with open(os.path.join(GOLDEN, "paper_sizes.json")) as f:
        gold = json.load(f)
    m = S.valid_mask(gold["H"], gold["W"], gold["psf_side"], gold["psf_side"])
    assert int(m.sum()) == gold["m"] == gold["observed_side"] ** 2
    assert m.size - int(m.sum()) == gold["unknown_boundary_pixels"]
    assert m.size == gold["n"]
    assert gold["psf_side"] == 2 * gold["l"] + 1
    # m = (sqrt(n) - 2 l)^2 (Sec. IV-A)
    assert (int(math.isqrt(gold["n"])) - 2 * gold["l"]) ** 2 == gold["m"]


def test_lowpass_dc_gain():
    """Sec. III-C, after the ADMM-TV convergence proposition: A 1 = beta 1
    with beta the DC gain of the filter."""
    g = S.rng(4)
    h = _rand_psf(g, 9, 9) * 0.7
    one = np.ones((20, 20))
    np.testing.assert_allclose(O.A_fft(one, h), 0.7 * one, atol=1e-14)
    np.testing.assert_allclose(abs(O.psf_otf(h, 20, 20)[0, 0]), 0.7, atol=1e-14)


# ----------------------------------------------------------------------------
# D, the TV denominator, Haar
# ----------------------------------------------------------------------------
def test_differences_and_spectrum_closed_form():
    """D 1 = 0 (Sec. III-C, proof of the ADMM-TV proposition); |Delta^h|^2 =
    4 sin^2(pi k_c / W) and |Delta^v|^2 = 4 sin^2(pi k_r / H) for forward
    periodic differences, so the denominator of eq. fast_inversion is known
    in closed form."""
    one = np.ones((6, 10))
    assert np.all(O.Dh(one) == 0) and np.all(O.Dv(one) == 0)
    H, W = 12, 10
    h = S.psf_box(3)
    mu1, mu2 = 0.7, 0.3
    kr = np.arange(H)[:, None]
    kc = np.arange(W)[None, :]
    lam = np.zeros((H, W), dtype=complex)
    for a in range(-1, 2):
        for b in range(-1, 2):
            lam += h[a + 1, b + 1] * np.exp(-2j * np.pi * (kr * a / H + kc * b / W))
    closed = mu1 * np.abs(lam) ** 2 + mu2 * 4 * np.sin(np.pi * kc / W) ** 2 \
        + mu2 * 4 * np.sin(np.pi * kr / H) ** 2
    np.testing.assert_allclose(O.tv_denominator_diag(h, H, W, mu1, mu2), closed, rtol=1e-13, atol=1e-14)


def _dense(op, H, W):
    n = H * W
    cols = []
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        cols.append(np.asarray(op(e.reshape(H, W))).reshape(-1))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("H,W", [(8, 8), (16, 16), (8, 12)])
def test_haar_parseval_dense(H, W):
    """Sec. III-B requires a Parseval frame, P^T P = I; 4 levels give 13 bands."""
    assert O.haar_nbands(4) == 13
    P = _dense(lambda v: O.haar_analysis(v, 4), H, W)
    assert P.shape == (13 * H * W, H * W)
    np.testing.assert_allclose(P.T @ P, np.eye(H * W), atol=1e-14)
    # the frame is redundant: P P^T is not the identity
    assert np.linalg.norm(P @ P.T - np.eye(13 * H * W)) > 1.0


def test_haar_bands_closed_form():
    """The last low-low band of the 4-level a-trous Haar is the mean of x over
    the 16 x 16 periodic window starting at the pixel; the level-0 detail
    bands are the 2 x 2 Haar differences. Written out as loops."""
    g = S.rng(5)
    H, W = 20, 18
    x = g.standard_normal((H, W))
    c = O.haar_analysis(x, 4)
    ll = np.zeros((H, W))
    b0 = np.zeros((H, W)); b1 = np.zeros((H, W)); b2 = np.zeros((H, W))
    for r in range(H):
        for q in range(W):
            ll[r, q] = sum(x[(r + i) % H, (q + j) % W] for i in range(16) for j in range(16)) / 256.0
            p00, p01 = x[r, q], x[r, (q + 1) % W]
            p10, p11 = x[(r + 1) % H, q], x[(r + 1) % H, (q + 1) % W]
            b0[r, q] = (p00 - p01 + p10 - p11) / 4.0     # rows low, columns high
            b1[r, q] = (p00 + p01 - p10 - p11) / 4.0     # rows high, columns low
            b2[r, q] = (p00 - p01 - p10 + p11) / 4.0     # rows high, columns high
    np.testing.assert_allclose(c[12], ll, atol=1e-13)
    np.testing.assert_allclose(c[0], b0, atol=1e-14)
    np.testing.assert_allclose(c[1], b1, atol=1e-14)
    np.testing.assert_allclose(c[2], b2, atol=1e-14)
    # level-1 uses taps {0, 2}
    r, q = 3, 4
    p = [[x[(r + 2 * i) % H, (q + 2 * j) % W] for j in range(2)] for i in range(2)]
    a1 = np.array([[sum(x[(r + 2 * i + ii) % H, (q + 2 * j + jj) % W] for ii in range(2) for jj in range(2)) / 4
                    for j in range(2)] for i in range(2)])
    del p
    assert abs(c[5][r, q] - (a1[0, 0] - a1[0, 1] - a1[1, 0] + a1[1, 1]) / 4.0) < 1e-14


# ----------------------------------------------------------------------------
# proximity operators: closed forms vs brute-force minimisation
# ----------------------------------------------------------------------------
def test_soft_is_l1_prox():
    """eq. soft: soft(v, t) = argmin_u t|u| + (u - v)^2 / 2, checked on a grid."""
    grid = np.linspace(-3, 3, 600001)
    for v in (-2.0, -0.3, 0.0, 0.2, 0.5, 1.7):
        t = 0.4
        u_star = grid[np.argmin(t * np.abs(grid) + 0.5 * (grid - v) ** 2)]
        assert abs(O.soft(np.array(v), t) - u_star) < 2e-5


def test_vsoft_is_l2_prox_with_zero_convention():
    """vector-soft (Sec. III-C) = argmin_u t||u|| + ||u - v||^2 / 2, incl. v = 0."""
    g1 = np.linspace(-1.5, 1.5, 1501)
    U, V = np.meshgrid(g1, g1, indexing="ij")
    t = 0.3
    for vh, vv in ((0.0, 0.0), (0.1, -0.1), (0.9, 0.4), (-1.0, 0.2), (0.25, 0.15)):
        f = t * np.sqrt(U ** 2 + V ** 2) + 0.5 * ((U - vh) ** 2 + (V - vv) ** 2)
        i = np.unravel_index(np.argmin(f), f.shape)
        uh, uv = O.vsoft(np.array(vh), np.array(vv), t)
        assert abs(uh - g1[i[0]]) < 3e-3 and abs(uv - g1[i[1]]) < 3e-3
    uh, uv = O.vsoft(np.zeros(3), np.zeros(3), 0.0)
    assert np.all(uh == 0) and np.all(uv == 0) and not np.any(np.isnan(uh))


def test_mask_prox_minimises():
    """eq. prox_g_1_uBC: u = argmin ||M u - y||^2 + mu1 ||u - v||^2 (per pixel)."""
    grid = np.linspace(-4, 4, 800001)
    mu1 = 0.35
    for m, y, v in ((1, 1.2, -0.4), (0, 1.2, -0.4), (1, -0.7, 2.0), (0, 0.0, 0.9)):
        f = m * (grid - y) ** 2 + mu1 * (grid - v) ** 2
        u_star = grid[np.argmin(f)]
        u = O.mask_prox(np.array(v), np.array(y * m), np.array(m, dtype=np.uint8), mu1)
        assert abs(u - u_star) < 2e-5


# ----------------------------------------------------------------------------
# the x-step against a dense solve (Algorithm 2 line 4, eq. quadratic_problem)
# ----------------------------------------------------------------------------
def _one_step_inputs(reg, H=8, W=8, seed=6):
    g = S.rng(seed)
    h = _rand_psf(g, 3, 5)
    nb = 2 if reg == "tv" else 13
    st = O.State(g.standard_normal((H, W)), g.standard_normal((H, W)),
                 g.standard_normal((nb, H, W)), g.standard_normal((nb, H, W)),
                 np.zeros((H, W)))
    ybar = g.standard_normal((H, W))
    mask = (g.uniform(size=(H, W)) > 0.3).astype(np.uint8)
    return g, h, st, ybar, mask


def test_tv_xstep_dense_solve():
    """x_{k+1} = (sum mu_j H_j^T H_j)^{-1} sum mu_j H_j^T zeta_j with dense
    A, D^h, D^v (eq. quadratic_problem) equals the oracle's Fourier solve."""
    H = W = 8
    g, h, st, ybar, mask = _one_step_inputs("tv")
    mu1, mu2, lam = 0.8, 0.05, 0.01
    A = _dense(lambda v: O.A_direct(v, h), H, W)
    Dh = _dense(O.Dh, H, W)
    Dv = _dense(O.Dv, H, W)
    Mat = mu1 * A.T @ A + mu2 * (Dh.T @ Dh + Dv.T @ Dv)
    z1 = (st.u1 + st.d1).ravel()
    dh = (st.u2[0] + st.d2[0]).ravel()
    dv = (st.u2[1] + st.d2[1]).ravel()
    x_dense = np.linalg.solve(Mat, mu1 * A.T @ z1 + mu2 * (Dh.T @ dh + Dv.T @ dv))
    nxt = O.tvmd_step(st, ybar, mask, h, lam, mu1, mu2)
    np.testing.assert_allclose(nxt.x.ravel(), x_dense, atol=1e-12)
    # the rest of the step, restated with dense operators
    a = A @ x_dense
    m = mask.ravel().astype(float)
    u1 = (m * ybar.ravel() + mu1 * (a - st.d1.ravel())) / (m + mu1)
    np.testing.assert_allclose(nxt.u1.ravel(), u1, atol=1e-12)
    np.testing.assert_allclose(nxt.d1.ravel(), st.d1.ravel() - a + u1, atol=1e-12)
    gh, gv = Dh @ x_dense, Dv @ x_dense
    sh, sv = gh - st.d2[0].ravel(), gv - st.d2[1].ravel()
    nrm = np.hypot(sh, sv)
    sc = np.maximum(nrm - lam / mu2, 0) / np.where(nrm > 0, nrm, 1)
    np.testing.assert_allclose(nxt.u2[0].ravel(), sc * sh, atol=1e-12)
    np.testing.assert_allclose(nxt.d2[1].ravel(), st.d2[1].ravel() - gv + sc * sv, atol=1e-12)


def test_haar_xstep_dense_solve():
    """FA-MD x-step (eq. invAnalysis) with dense A and P; P^T P = I is not
    assumed by the dense side."""
    H = W = 8
    g, h, st, ybar, mask = _one_step_inputs("haar")
    mu1, mu2, lam = 0.6, 0.09, 0.02
    A = _dense(lambda v: O.A_direct(v, h), H, W)
    P = _dense(lambda v: O.haar_analysis(v, 4), H, W)
    gam = mu2 / mu1
    Mat = A.T @ A + gam * P.T @ P
    x_dense = np.linalg.solve(Mat, A.T @ (st.u1 + st.d1).ravel() + gam * P.T @ (st.u2 + st.d2).ravel())
    nxt = O.famd_step(st, ybar, mask, h, lam, mu1, mu2, 4)
    np.testing.assert_allclose(nxt.x.ravel(), x_dense, atol=1e-12)
    c = P @ x_dense
    s = c - st.d2.ravel()
    u2 = np.sign(s) * np.maximum(np.abs(s) - lam / mu2, 0)
    np.testing.assert_allclose(nxt.u2.ravel(), u2, atol=1e-12)
    np.testing.assert_allclose(nxt.d2.ravel(), st.d2.ravel() - c + u2, atol=1e-12)


# ----------------------------------------------------------------------------
# whole-iteration pins
# ----------------------------------------------------------------------------
def _small_problem(H=16, W=16, seed=7, side=5, keep=0.8, bsnr=40.0):
    g = S.rng(seed)
    x = S.shapes_image(H, W, g, 6, rmax=5.0)
    h = S.psf_gaussian(side, 1.2)
    keepm = (g.uniform(size=(H, W)) < keep).astype(np.uint8)
    ybar, mask, _ = S.observe(x, h, keepm, bsnr, g)
    return x, h, ybar, mask


def test_tv_kkt_certificate_at_convergence():
    """At a fixed point of TV-MD the scaled duals certify optimality of eq.
    unconstrained_TV_uBC (from Algorithm 2 lines 4-7 with u = G z):
    -mu1 d1 = M^T (M A x - y),  mu1 A^T d1 + mu2 D^T d2 = 0,
    ||mu2 d2_i|| <= lambda with equality and alignment where D_i x != 0."""
    x, h, ybar, mask = _small_problem()
    lam, mu1, mu2 = 2e-3, 1.0, 2e-2
    r = O.solve(ybar, mask, h, lam, mu1, mu2, "tv", iters=20000, stop="rel_x", tol=1e-13)
    st = r.state
    ax = O.A_fft(st.x, h)
    m = mask.astype(float)
    np.testing.assert_allclose(-mu1 * st.d1, m * (ax - ybar), atol=1e-9)
    stat = mu1 * O.At_fft(st.d1, h) + mu2 * (O.DhT(st.d2[0]) + O.DvT(st.d2[1]))
    assert np.max(np.abs(stat)) < 1e-9
    pn = mu2 * np.hypot(st.d2[0], st.d2[1])
    assert np.max(pn) <= lam * (1 + 1e-9)
    gh, gv = O.Dh(st.x), O.Dv(st.x)
    gn = np.hypot(gh, gv)
    act = gn > 1e-6
    assert act.sum() > 10
    np.testing.assert_allclose(pn[act], lam, rtol=1e-6)
    # -mu2 d2_i points along D_i x
    np.testing.assert_allclose(-mu2 * st.d2[0][act], lam * gh[act] / gn[act], atol=1e-6 * lam + 1e-9)


def test_haar_kkt_certificate_at_convergence():
    """Same certificate for FA-MD (eq. unconstrained_analysis_uBC):
    -mu1 d1 = M^T(MAx - y), mu1 A^T d1 + mu2 P^T d2 = 0, |mu2 d2| <= lambda."""
    x, h, ybar, mask = _small_problem(seed=8)
    lam, mu1, mu2 = 1e-2, 1.0, 1e-1
    r = O.solve(ybar, mask, h, lam, mu1, mu2, "haar", iters=20000, stop="rel_x", tol=1e-13)
    assert r.converged
    st = r.state
    ax = O.A_fft(st.x, h)
    m = mask.astype(float)
    np.testing.assert_allclose(-mu1 * st.d1, m * (ax - ybar), atol=1e-9)
    stat = mu1 * O.At_fft(st.d1, h) + mu2 * O.haar_synthesis(st.d2, 4)
    assert np.max(np.abs(stat)) < 1e-9
    assert np.max(np.abs(mu2 * st.d2)) <= lam * (1 + 1e-9)
    c = O.haar_analysis(st.x, 4)
    act = np.abs(c) > 1e-7
    np.testing.assert_allclose(-mu2 * st.d2[act], lam * np.sign(c[act]), atol=1e-6 * lam)


def _pdhg_tv(A, Dh, Dv, m, ybar, lam, iters=200000):
    """Chambolle-Pock primal-dual hybrid gradient on
    min_x 1/2 sum_i m_i (A x - y)_i^2 + lam sum_i ||(Dh x, Dv x)_i||,
    with K = [A; Dh; Dv]; written independently of the ADMM oracle."""
    n = A.shape[1]
    K = np.vstack([A, Dh, Dv])
    L = np.linalg.norm(K, 2)
    tau = sig = 0.99 / L
    x = np.zeros(n); xb = x.copy()
    p = np.zeros(n); q = np.zeros((2, n))
    for _ in range(iters):
        # dual step for F1*(p): F1(v) = 1/2 sum m (v - y)^2
        v = p + sig * (A @ xb)
        p = np.where(m > 0, (v - sig * ybar) / (1.0 + sig), 0.0)
        # dual step for F2*: projection on ||q_i|| <= lam
        w = q + sig * np.stack([Dh @ xb, Dv @ xb])
        nrm = np.maximum(1.0, np.hypot(w[0], w[1]) / lam)
        q = w / nrm
        x_new = x - tau * (A.T @ p + Dh.T @ q[0] + Dv.T @ q[1])
        xb = 2 * x_new - x
        x = x_new
    return x


def test_tv_optimum_matches_independent_pdhg():
    """8 x 8 problem: the objective reached by TV-MD equals the one reached by
    an independent dense-matrix PDHG (Chambolle-Pock) solver."""
    H = W = 8
    g = S.rng(9)
    xt = S.shapes_image(H, W, g, 3, rmax=3.0)
    h = S.psf_gaussian(3, 0.8)
    keep = (g.uniform(size=(H, W)) < 0.9).astype(np.uint8)
    ybar, mask, _ = S.observe(xt, h, keep, 30.0, g)
    lam, mu1, mu2 = 5e-3, 1.0, 5e-2
    r = O.solve(ybar, mask, h, lam, mu1, mu2, "tv", iters=50000, stop="rel_x", tol=1e-14)
    A = _dense(lambda v: O.A_direct(v, h), H, W)
    Dh = _dense(O.Dh, H, W)
    Dv = _dense(O.Dv, H, W)
    xp = _pdhg_tv(A, Dh, Dv, mask.ravel().astype(float), ybar.ravel(), lam, iters=60000)
    f_pd = O.objective_tv(xp.reshape(H, W), ybar, mask, h, lam)
    assert abs(r.objective - f_pd) <= 1e-8 * abs(f_pd) + 1e-12


def test_periodic_unregularised_closed_form():
    """Special cases of Sec. IV-A: with M = I (periodic deconvolution) and
    lambda = 0 the minimiser is x = U* (Y / Lambda) for an invertible blur."""
    H, W = 16, 16
    g = S.rng(10)
    h = np.zeros((3, 3)); h[1, 1] = 0.8; h[1, 2] = 0.1; h[0, 1] = 0.1
    xt = g.uniform(size=(H, W))
    y = O.A_fft(xt, h)
    mask = np.ones((H, W), dtype=np.uint8)
    r = O.solve(y, mask, h, 0.0, 1.0, 0.1, "tv", iters=3000, stop="rel_x", tol=1e-15)
    closed = np.real(np.fft.ifft2(np.fft.fft2(y) / O.psf_otf(h, H, W)))
    np.testing.assert_allclose(r.x, closed, atol=1e-9)
    np.testing.assert_allclose(closed, xt, atol=1e-12)


def test_pure_inpainting_special_case():
    """A = I (a 1 x 1 unit kernel) turns the model into inpainting (Sec. IV-A):
    observed pixels with lambda -> 0 are reproduced; the TV-MD iterate
    matches the data on the mask."""
    H, W = 12, 12
    g = S.rng(11)
    xt = S.shapes_image(H, W, g, 4, rmax=4.0)
    h = np.ones((1, 1))
    mask = (g.uniform(size=(H, W)) < 0.7).astype(np.uint8)
    ybar = xt * mask
    r = O.solve(ybar, mask, h, 1e-9, 1.0, 1e-8, "tv", iters=4000, stop="rel_x", tol=1e-14)
    assert np.max(np.abs((r.x - xt)[mask.astype(bool)])) < 1e-6


def test_arbitrary_initialisation_converges_to_same_objective():
    """Theorem 1 (Eckstein-Bertsekas): ADMM converges from arbitrary u0, d0."""
    x, h, ybar, mask = _small_problem(seed=12)
    lam, mu1, mu2 = 2e-3, 1.0, 2e-2
    r0 = O.solve(ybar, mask, h, lam, mu1, mu2, "tv", iters=20000, stop="rel_x", tol=1e-13)
    g = S.rng(13)
    H, W = ybar.shape
    st = O.State(g.standard_normal((H, W)), g.standard_normal((H, W)),
                 g.standard_normal((2, H, W)), g.standard_normal((2, H, W)), np.zeros((H, W)))
    r1 = O.solve(ybar, mask, h, lam, mu1, mu2, "tv", iters=20000, stop="rel_x", tol=1e-13, state0=st)
    assert abs(r0.objective - r1.objective) <= 1e-7 * r0.objective
    np.testing.assert_allclose(r0.x, r1.x, atol=1e-6)


def test_objective_decreases_after_burn_in():
    """ADMM gives no per-step monotone decrease (Theorem 1 is a convergence
    result), but on these problems f(x_k) <= f(x_{k-20}) after 20 iterations."""
    p = S.config1_problem(0)
    r = O.solve(p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, "tv", iters=200, record=True)
    f = [h[1] for h in r.history]
    for k in range(40, len(f)):
        assert f[k] <= f[k - 20] * (1 + 1e-12)


# --------------------------------------------------------------------------
# variants: anisotropic TV (soft threshold per difference component) and the
# frame prior with the low-low band left unpenalised
# --------------------------------------------------------------------------
def _pdhg_tv_aniso(A, Dh, Dv, m, ybar, lam, iters=60000):
    """Chambolle-Pock on min_x 1/2 sum_i m_i (A x - y)_i^2 + lam sum_i (|Dh x|_i + |Dv x|_i):
    the dual step of the regulariser projects each component on [-lam, lam]."""
    n = A.shape[1]
    K = np.vstack([A, Dh, Dv])
    L = np.linalg.norm(K, 2)
    tau = sig = 0.99 / L
    x = np.zeros(n); xb = x.copy()
    p = np.zeros(n); q = np.zeros((2, n))
    for _ in range(iters):
        v = p + sig * (A @ xb)
        p = np.where(m > 0, (v - sig * ybar) / (1.0 + sig), 0.0)
        q = np.clip(q + sig * np.stack([Dh @ xb, Dv @ xb]), -lam, lam)
        x_new = x - tau * (A.T @ p + Dh.T @ q[0] + Dv.T @ q[1])
        xb = 2 * x_new - x
        x = x_new
    return x


def test_aniso_tv_kkt_certificate_at_convergence():
    """Anisotropic TV: -mu1 d1 = M^T(M A x - y), mu1 A^T d1 + mu2 D^T d2 = 0,
    |mu2 d2| <= lambda per component with -mu2 d2 = lambda sign(D x) where D x != 0
    (the subgradient of the l1 norm, eq. soft's optimality)."""
    x, h, ybar, mask = _small_problem()
    lam, mu1, mu2 = 2e-3, 1.0, 2e-2
    r = O.solve(ybar, mask, h, lam, mu1, mu2, "tv_aniso", iters=20000, stop="rel_x", tol=1e-13)
    assert r.converged
    st = r.state
    m = mask.astype(float)
    np.testing.assert_allclose(-mu1 * st.d1, m * (O.A_fft(st.x, h) - ybar), atol=1e-9)
    stat = mu1 * O.At_fft(st.d1, h) + mu2 * (O.DhT(st.d2[0]) + O.DvT(st.d2[1]))
    assert np.max(np.abs(stat)) < 1e-9
    assert np.max(np.abs(mu2 * st.d2)) <= lam * (1 + 1e-9)
    for comp, gfun in ((0, O.Dh), (1, O.Dv)):
        gx = gfun(st.x)
        act = np.abs(gx) > 1e-6
        assert act.sum() > 10
        np.testing.assert_allclose(-mu2 * st.d2[comp][act], lam * np.sign(gx[act]), atol=1e-6 * lam)
    # the isotropic solution of the same problem is a different point
    ri = O.solve(ybar, mask, h, lam, mu1, mu2, "tv", iters=20000, stop="rel_x", tol=1e-13)
    assert np.max(np.abs(ri.x - r.x)) > 1e-4


def test_aniso_tv_optimum_matches_independent_pdhg():
    H = W = 8
    g = S.rng(19)
    xt = S.shapes_image(H, W, g, 3, rmax=3.0)
    h = S.psf_gaussian(3, 0.8)
    keep = (g.uniform(size=(H, W)) < 0.9).astype(np.uint8)
    ybar, mask, _ = S.observe(xt, h, keep, 30.0, g)
    lam, mu1, mu2 = 5e-3, 1.0, 5e-2
    r = O.solve(ybar, mask, h, lam, mu1, mu2, "tv_aniso", iters=50000, stop="rel_x", tol=1e-14)
    A = _dense(lambda v: O.A_direct(v, h), H, W)
    xp = _pdhg_tv_aniso(A, _dense(O.Dh, H, W), _dense(O.Dv, H, W), mask.ravel().astype(float), ybar.ravel(),
                        lam)
    f_pd = O.objective_tv(xp.reshape(H, W), ybar, mask, h, lam, aniso=True)
    assert abs(r.objective - f_pd) <= 1e-8 * abs(f_pd) + 1e-12


def test_ll_free_frame_kkt_and_zero_low_low_dual():
    """Frame prior with the low-low band unpenalised: the low-low dual is zero
    after every iteration (its prox is the identity), and the certificate of
    the remaining bands holds: mu1 A^T d1 + mu2 P^T d2 = 0, |mu2 d2| <= lambda."""
    x, h, ybar, mask = _small_problem(seed=8)
    lam, mu1, mu2 = 1e-2, 1.0, 1e-1
    r = O.solve(ybar, mask, h, lam, mu1, mu2, "haar_ll_free", iters=20000, stop="rel_x", tol=1e-13)
    assert r.converged
    st = r.state
    assert np.max(np.abs(st.d2[-1])) < 1e-12
    m = mask.astype(float)
    np.testing.assert_allclose(-mu1 * st.d1, m * (O.A_fft(st.x, h) - ybar), atol=1e-9)
    stat = mu1 * O.At_fft(st.d1, h) + mu2 * O.haar_synthesis(st.d2, 4)
    assert np.max(np.abs(stat)) < 1e-9
    assert np.max(np.abs(mu2 * st.d2)) <= lam * (1 + 1e-9)
    c = O.haar_analysis(st.x, 4)[:-1]
    act = np.abs(c) > 1e-7
    np.testing.assert_allclose(-mu2 * st.d2[:-1][act], lam * np.sign(c[act]), atol=1e-6 * lam)


@pytest.mark.parametrize("reg", ["tv", "tv_aniso", "haar_ll_free", "haar"])
def test_strong_weight_limit(reg):
    """With a weight far above the data term, a regulariser that vanishes on
    constants (TV, anisotropic TV, details-only frame) leaves the best constant:
    A 1 = beta 1 gives x = sum of observed y / (beta * #observed); the full frame
    prior, which also penalises the low-low band, drives x to zero."""
    g = S.rng(21)
    H = W = 16
    x = S.shapes_image(H, W, g, 4, rmax=4.0)
    h = S.psf_gaussian(5, 1.0)
    keep = (g.uniform(size=(H, W)) < 0.8).astype(np.uint8)
    ybar, mask, _ = S.observe(x, h, keep, 40.0, g)
    cstar = ybar[mask > 0].sum() / (h.sum() * mask.sum())
    r = O.solve(ybar, mask, h, 10.0, 0.3, 3.0, reg, iters=3000)
    target = 0.0 if reg == "haar" else cstar
    assert np.max(np.abs(r.x - target)) < 1e-9


# --------------------------------------------------------------------------
# FS-MD: the frame synthesis formulation (x = W theta, W = P^T)
# --------------------------------------------------------------------------
def test_fs_theta_step_dense_solve():
    """The SMW theta-step equals a dense solve of (W^T A^T A W + gamma I) theta
    = W^T A^T zeta1 + gamma zeta2 with W the dense synthesis matrix (W W^T = I
    is not assumed by the dense side); x = W theta; then the mask prox and the
    soft threshold of theta - d2."""
    H = W = 8
    g, h, st, ybar, mask = _one_step_inputs("haar")
    mu1, mu2, lam = 0.6, 0.09, 0.02
    gam = mu2 / mu1
    A = _dense(lambda v: O.A_direct(v, h), H, W)
    Wm = _dense(lambda v: O.haar_analysis(v, 4), H, W).T          # synthesis = transpose of analysis
    Mat = Wm.T @ A.T @ A @ Wm + gam * np.eye(Wm.shape[1])
    rhs = Wm.T @ A.T @ (st.u1 + st.d1).ravel() + gam * (st.u2 + st.d2).ravel()
    th = np.linalg.solve(Mat, rhs)
    nxt = O.fsmd_step(st, ybar, mask, h, lam, mu1, mu2, 4)
    np.testing.assert_allclose(nxt.theta.ravel(), th, atol=1e-11)
    np.testing.assert_allclose(nxt.x.ravel(), Wm @ th, atol=1e-11)
    s = th - st.d2.ravel()
    u2 = np.sign(s) * np.maximum(np.abs(s) - lam / mu2, 0)
    np.testing.assert_allclose(nxt.u2.ravel(), u2, atol=1e-11)
    np.testing.assert_allclose(nxt.d2.ravel(), st.d2.ravel() - th + u2, atol=1e-11)
    ax = A @ (Wm @ th)
    m = mask.ravel().astype(float)
    u1 = (m * ybar.ravel() + mu1 * (ax - st.d1.ravel())) / (m + mu1)
    np.testing.assert_allclose(nxt.u1.ravel(), u1, atol=1e-11)


def test_fs_kkt_certificate_at_convergence():
    """Synthesis problem min 1/2 ||M(y - A W theta)||^2 + lam ||theta||_1 at a
    fixed point of FS-MD (H1 = A W, H2 = I): -mu1 d1 = M^T(M A W theta - y),
    mu1 W^T A^T d1 + mu2 d2 = 0, |mu2 d2| <= lam with -mu2 d2 = lam sign(theta)
    where theta != 0."""
    g = S.rng(11)
    x = S.shapes_image(8, 8, g, 3, rmax=3.0)
    h = S.psf_gaussian(3, 0.8)
    keepm = (g.uniform(size=(8, 8)) < 0.9).astype(np.uint8)
    ybar, mask, _ = S.observe(x, h, keepm, 40.0, g)
    lam, mu1, mu2 = 1e-2, 0.1, 0.03
    r = O.solve(ybar, mask, h, lam, mu1, mu2, "haar_synthesis", iters=30000, stop="rel_x", tol=1e-13)
    assert r.converged
    st = r.state
    m = mask.astype(float)
    np.testing.assert_allclose(-mu1 * st.d1, m * (O.A_fft(st.x, h) - ybar), atol=1e-9)
    stat = mu1 * O.haar_analysis(O.At_fft(st.d1, h), 4) + mu2 * st.d2
    assert np.max(np.abs(stat)) < 1e-9
    assert np.max(np.abs(mu2 * st.d2)) <= lam * (1 + 1e-9)
    act = np.abs(st.theta) > 1e-7
    assert act.sum() > 10
    np.testing.assert_allclose(-mu2 * st.d2[act], lam * np.sign(st.theta[act]), atol=1e-6 * lam)
    np.testing.assert_allclose(O.haar_synthesis(st.theta, 4), st.x, atol=1e-12)


def test_fs_optimum_matches_independent_fista():
    """8 x 8: the objective FS-MD reaches equals the one of FISTA (Beck and
    Teboulle's accelerated proximal gradient, a published method written here
    with dense matrices) on the same synthesis problem; and it differs from the
    analysis (FA) problem's optimum on this redundant frame."""
    H = W = 8
    g = S.rng(29)
    xt = S.shapes_image(H, W, g, 3, rmax=3.0)
    h = S.psf_gaussian(3, 0.8)
    keep = (g.uniform(size=(H, W)) < 0.9).astype(np.uint8)
    ybar, mask, _ = S.observe(xt, h, keep, 30.0, g)
    lam, mu1, mu2 = 5e-3, 0.1, 0.015
    r = O.solve(ybar, mask, h, lam, mu1, mu2, "haar_synthesis", iters=60000, stop="rel_x", tol=1e-14)
    A = _dense(lambda v: O.A_direct(v, h), H, W)
    Wm = _dense(lambda v: O.haar_analysis(v, 4), H, W).T
    K = mask.ravel().astype(float)[:, None] * (A @ Wm)
    yv = mask.ravel().astype(float) * ybar.ravel()
    Lc = np.linalg.norm(K, 2) ** 2
    th = np.zeros(K.shape[1]); z = th.copy(); tk = 1.0
    for _ in range(60000):
        gz = z - K.T @ (K @ z - yv) / Lc
        th_new = np.sign(gz) * np.maximum(np.abs(gz) - lam / Lc, 0)
        tk_new = 0.5 * (1 + np.sqrt(1 + 4 * tk * tk))
        z = th_new + (tk - 1) / tk_new * (th_new - th)
        th, tk = th_new, tk_new
    f_fista = 0.5 * float(np.sum((K @ th - yv) ** 2)) + lam * float(np.sum(np.abs(th)))
    assert abs(r.objective - f_fista) <= 1e-8 * abs(f_fista) + 1e-12
    ra = O.solve(ybar, mask, h, lam, mu1, mu2, "haar", iters=60000, stop="rel_x", tol=1e-14)
    assert np.max(np.abs(ra.x - r.x)) > 1e-4


def test_fs_strong_weight_gives_zero():
    g = S.rng(21)
    x = S.shapes_image(16, 16, g, 4, rmax=4.0)
    h = S.psf_gaussian(5, 1.0)
    ybar, mask, _ = S.observe(x, h, None, 40.0, g)
    r = O.solve(ybar, mask, h, 10.0, 0.3, 3.0, "haar_synthesis", iters=3000)
    assert np.max(np.abs(r.x)) < 1e-9 and np.max(np.abs(r.state.theta)) < 1e-9


# ----------------------------------------------------------------------------
# the oracle's own DFT (Sec. III-C, eq. DFT_fact)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("H,W", [(5, 7), (9, 3), (8, 12), (1, 6)])
def test_own_dft_closed_forms_and_library(H, W):
    """dft2 / idft2 against closed forms -- a unit impulse at (r0, c0) has the
    spectrum exp(-2 pi i (k_r r0 / H + k_c c0 / W)); a constant has all its
    energy at k = 0; the complex exponential of frequency (k0, l0) is n times
    the impulse there -- against an independent FFT library (numpy.fft), and
    the inverse and Parseval's identity on random data, including odd sides."""
    g = S.rng(40)
    kr = np.arange(H)[:, None]
    kc = np.arange(W)[None, :]
    r0, c0 = H // 2, W - 1
    e = np.zeros((H, W))
    e[r0, c0] = 1.0
    np.testing.assert_allclose(O.dft2(e), np.exp(-2j * np.pi * (kr * r0 / H + kc * c0 / W)), atol=1e-14)
    const = np.full((H, W), 2.5)
    expect = np.zeros((H, W), dtype=complex)
    expect[0, 0] = 2.5 * H * W
    np.testing.assert_allclose(O.dft2(const), expect, atol=1e-12)
    k0, l0 = (1 % H), (2 % W)
    rr = np.arange(H)[:, None]
    cc = np.arange(W)[None, :]
    wave = np.exp(2j * np.pi * (k0 * rr / H + l0 * cc / W))
    expect = np.zeros((H, W), dtype=complex)
    expect[k0, l0] = H * W
    np.testing.assert_allclose(O.dft2(wave), expect, atol=1e-12)
    x = g.standard_normal((H, W)) + 1j * g.standard_normal((H, W))
    X = O.dft2(x)
    np.testing.assert_allclose(X, np.fft.fft2(x), atol=1e-12)
    np.testing.assert_allclose(O.idft2(X), x, atol=1e-13)
    np.testing.assert_allclose(O.idft2(x), np.fft.ifft2(x), atol=1e-13)
    np.testing.assert_allclose(np.sum(np.abs(X) ** 2), H * W * np.sum(np.abs(x) ** 2), rtol=1e-12)


def test_psf_otf_odd_size_explicit_sum():
    """Lambda on an odd, non-square domain equals the DFT sum of the centred
    kernel written out tap by tap: sum_{a,b} h[a+l_r, b+l_c] exp(-2 pi i
    (k_r a / H + k_c b / W)) (reading 1: the kernel's centre at (0, 0))."""
    g = S.rng(41)
    H, W = 9, 11
    h = _rand_psf(g, 5, 3)
    lam = np.zeros((H, W), dtype=complex)
    for kr in range(H):
        for kc in range(W):
            acc = 0j
            for a in range(-2, 3):
                for b in range(-1, 2):
                    acc += h[a + 2, b + 1] * np.exp(-2j * np.pi * (kr * a / H + kc * b / W))
            lam[kr, kc] = acc
    np.testing.assert_allclose(O.psf_otf(h, H, W), lam, atol=1e-14)


# ----------------------------------------------------------------------------
# the objectives (eq. unconstrained_TV_uBC, eq. unconstrained_analysis_uBC) and
# the figure of merit ISNR (Sec. V)
# ----------------------------------------------------------------------------
def test_objective_tv_closed_forms():
    """Closed forms of eq. unconstrained_TV_uBC that a dropped 1/2, a missing
    mask in the data term, a wrong lambda factor or a wrong TV norm would fail:
      x = 0:                      f = 1/2 sum over observed pixels of y^2
      x = c (constant):           f = 1/2 sum_obs (y - beta c)^2, beta = sum(h)
                                  (A 1 = beta 1, and D 1 = 0)
      x[r, c] = c (column ramp):  forward periodic differences are 1, except
                                  1 - W at the wrap; TV = H (W - 1) + H (W - 1)
      x[r, c] = r + c:            isotropic TV is sqrt(2) on the (H-1)(W-1)
                                  interior pixels, sqrt((W-1)^2 + 1) on the last
                                  column, sqrt((H-1)^2 + 1) on the last row and
                                  sqrt((H-1)^2 + (W-1)^2) at the corner;
                                  anisotropic TV is 2 H (W - 1) + 2 W (H - 1)."""
    g = S.rng(42)
    H, W = 7, 10
    h = _rand_psf(g, 3, 5) * 0.8
    beta = h.sum()
    ybar = g.standard_normal((H, W))
    mask = (g.uniform(size=(H, W)) > 0.4).astype(np.uint8)
    obs = mask.astype(bool)
    lam = 0.37
    zero = np.zeros((H, W))
    np.testing.assert_allclose(O.objective_tv(zero, ybar, mask, h, lam), 0.5 * np.sum(ybar[obs] ** 2), rtol=1e-13)
    np.testing.assert_allclose(O.objective_tv(zero, ybar, mask, h, lam, aniso=True),
                               0.5 * np.sum(ybar[obs] ** 2), rtol=1e-13)
    c = 0.6
    np.testing.assert_allclose(O.objective_tv(np.full((H, W), c), ybar, mask, h, lam),
                               0.5 * np.sum((ybar[obs] - beta * c) ** 2), rtol=1e-12)
    rr, cc = np.meshgrid(np.arange(H, dtype=float), np.arange(W, dtype=float), indexing="ij")
    # with nothing observed only the regulariser remains
    none = np.zeros((H, W), dtype=np.uint8)
    np.testing.assert_allclose(O.objective_tv(cc, ybar, none, h, lam), lam * 2 * H * (W - 1), rtol=1e-13)
    iso = ((H - 1) * (W - 1) * math.sqrt(2.0) + (H - 1) * math.hypot(W - 1, 1) + (W - 1) * math.hypot(H - 1, 1)
           + math.hypot(H - 1, W - 1))
    np.testing.assert_allclose(O.objective_tv(rr + cc, ybar, none, h, lam), lam * iso, rtol=1e-13)
    np.testing.assert_allclose(O.objective_tv(rr + cc, ybar, none, h, lam, aniso=True),
                               lam * (2 * H * (W - 1) + 2 * W * (H - 1)), rtol=1e-13)


def test_objective_haar_closed_forms():
    """Closed forms of eq. unconstrained_analysis_uBC with the 13-band frame:
    for x = a (-1)^(r+c) + b on an even torus the level-0 high-high band is
    a (-1)^(r+c), every other detail band is zero and the final low-low band
    is b, so ||P x||_1 = n (|a| + |b|), and n |a| with the low-low band
    unpenalised; for x = a (-1)^c + b only the level-0 rows-low/columns-high
    band and the low-low band survive, with the same sums. The data term is
    checked at x = 0 and at a constant, where A x = beta x."""
    g = S.rng(43)
    H, W = 16, 16
    n = H * W
    h = _rand_psf(g, 5, 5) * 1.3
    beta = h.sum()
    ybar = g.standard_normal((H, W))
    mask = (g.uniform(size=(H, W)) > 0.3).astype(np.uint8)
    obs = mask.astype(bool)
    lam = 0.21
    none = np.zeros((H, W), dtype=np.uint8)
    rr, cc = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    a, b = -0.7, 0.45
    for x in (a * (-1.0) ** (rr + cc) + b, a * (-1.0) ** cc + b):
        np.testing.assert_allclose(O.objective_haar(x, ybar, none, h, lam), lam * n * (abs(a) + abs(b)), rtol=1e-12)
        np.testing.assert_allclose(O.objective_haar(x, ybar, none, h, lam, ll_free=True), lam * n * abs(a),
                                   rtol=1e-12)
    zero = np.zeros((H, W))
    np.testing.assert_allclose(O.objective_haar(zero, ybar, mask, h, lam), 0.5 * np.sum(ybar[obs] ** 2), rtol=1e-13)
    cst = np.full((H, W), b)
    np.testing.assert_allclose(O.objective_haar(cst, ybar, mask, h, lam),
                               0.5 * np.sum((ybar[obs] - beta * b) ** 2) + lam * n * abs(b), rtol=1e-12)
    np.testing.assert_allclose(O.objective_haar(cst, ybar, mask, h, lam, ll_free=True),
                               0.5 * np.sum((ybar[obs] - beta * b) ** 2), rtol=1e-12)


def _dense_conv_loops(h, H, W):
    """The matrix of periodic convolution, entry by entry from its definition
    (reading 1): row (r, c) has h[a + l_r, b + l_c] at column ((r-a) mod H, (c-b) mod W)."""
    ph, pw = h.shape
    lr, lc = ph // 2, pw // 2
    A = np.zeros((H * W, H * W))
    for r in range(H):
        for c in range(W):
            for a in range(-lr, lr + 1):
                for b in range(-lc, lc + 1):
                    A[r * W + c, ((r - a) % H) * W + (c - b) % W] += h[a + lr, b + lc]
    return A


def test_objectives_brute_force_on_random_inputs():
    """On random x, y, masks and asymmetric kernels: the data term from the
    convolution matrix built entry by entry, and the regularisers summed pixel
    by pixel (TV with forward periodic differences, reading 3; the frame
    coefficients from the bands' defining two-tap sums, reading 6)."""
    g = S.rng(44)
    H, W = 6, 8
    h = _rand_psf(g, 3, 5)
    A = _dense_conv_loops(h, H, W)
    x = g.standard_normal((H, W))
    ybar = g.standard_normal((H, W))
    mask = (g.uniform(size=(H, W)) > 0.35).astype(np.uint8)
    lam = 0.13
    ax = (A @ x.ravel()).reshape(H, W)
    data = 0.0
    for r in range(H):
        for c in range(W):
            if mask[r, c]:
                data += 0.5 * (ybar[r, c] - ax[r, c]) ** 2
    iso = aniso = 0.0
    for r in range(H):
        for c in range(W):
            gh = x[r, (c + 1) % W] - x[r, c]
            gv = x[(r + 1) % H, c] - x[r, c]
            iso += math.sqrt(gh * gh + gv * gv)
            aniso += abs(gh) + abs(gv)
    np.testing.assert_allclose(O.objective_tv(x, ybar, mask, h, lam), data + lam * iso, rtol=1e-12)
    np.testing.assert_allclose(O.objective_tv(x, ybar, mask, h, lam, aniso=True), data + lam * aniso, rtol=1e-12)
    # one-level frame (2 x 2 Haar at taps {0, 1}) on an 8 x 8 torus, by its sums
    H = W = 8
    A = _dense_conv_loops(h, H, W)
    x = g.standard_normal((H, W))
    ybar = g.standard_normal((H, W))
    mask = (g.uniform(size=(H, W)) > 0.35).astype(np.uint8)
    ax = (A @ x.ravel()).reshape(H, W)
    data = 0.5 * sum((ybar[r, c] - ax[r, c]) ** 2 for r in range(H) for c in range(W) if mask[r, c])
    l1 = l1_ll = 0.0
    for r in range(H):
        for c in range(W):
            p, q = x[r, c], x[r, (c + 1) % W]
            s, t = x[(r + 1) % H, c], x[(r + 1) % H, (c + 1) % W]
            lh = 0.25 * ((p - q) + (s - t))      # rows low, columns high
            hl = 0.25 * ((p + q) - (s + t))      # rows high, columns low
            hh = 0.25 * ((p - q) - (s - t))
            ll = 0.25 * (p + q + s + t)
            l1 += abs(lh) + abs(hl) + abs(hh) + abs(ll)
            l1_ll += abs(lh) + abs(hl) + abs(hh)
    np.testing.assert_allclose(O.objective_haar(x, ybar, mask, h, lam, levels=1), data + lam * l1, rtol=1e-12)
    np.testing.assert_allclose(O.objective_haar(x, ybar, mask, h, lam, levels=1, ll_free=True),
                               data + lam * l1_ll, rtol=1e-12)


def test_isnr_hand_computed():
    """ISNR = 10 log10(||x - ybar||^2 / ||x - x_hat||^2) over the region
    (reading 13), on a 3 x 3 case computed by hand: inside the region (the
    top-left 2 x 2) the observation errs by 1 and the estimate by 0.1, so the
    ratio is 100 and ISNR = 20 dB; pixels outside the region do not count."""
    x = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0], [7.0, 8.0, 9.0]])
    ybar = x.copy()
    ybar[:2, :2] -= 1.0
    ybar[2, 2] = 100.0            # outside the region: ignored
    xh = x.copy()
    xh[:2, :2] += 0.1
    xh[0, 2] = -50.0              # outside the region: ignored
    region = np.zeros((3, 3), dtype=bool)
    region[:2, :2] = True
    assert abs(O.isnr(x, ybar, xh, region) - 20.0) < 1e-12
    # halving the estimate's error adds 10 log10(4) dB
    xh2 = x.copy()
    xh2[:2, :2] += 0.05
    assert abs(O.isnr(x, ybar, xh2, region) - (20.0 + 10.0 * math.log10(4.0))) < 1e-12
    # SNR = 10 log10(||x||^2 / ||x - x_hat||^2) over the whole image
    assert abs(O.snr(x, x + 0.1 * np.sign(x)) - 10.0 * math.log10(np.sum(x ** 2) / (9 * 0.01))) < 1e-12


# ----------------------------------------------------------------------------
# the Reeves-Sorel variants TV-CG and FA-CG (Sec. IV-B/C/D, eqs. reeves,
# reeves3 and ReevesTV)
# ----------------------------------------------------------------------------
def _cg_inputs(H=8, W=8, seed=61, keep=0.6):
    g = S.rng(seed)
    h = _rand_psf(g, 3, 3)
    mask = (g.uniform(size=(H, W)) < keep).astype(np.uint8)
    return g, h, mask


@pytest.mark.parametrize("reg", ["tv", "haar"])
def test_reeves_sorel_inverse_dense(reg):
    """With the inner system solved exactly (CG run to convergence), the
    x-step equals the dense solve of (A^T M^T M A + gamma D^T D) x = r (TV,
    eq. ReevesTV) or (A^T M^T M A + gamma I) x = r (frame, eqs.
    invAnalysis_sorel and reeves3): the Sherman-Morrison-Woodbury identity of
    eq. reeves, checked against matrices built from the operators' definitions."""
    H = W = 8
    g, h, mask = _cg_inputs()
    gam = 0.07
    A = _dense_conv_loops(h, H, W)
    Mm = np.diag(mask.ravel().astype(float))
    if reg == "tv":
        Dh = _dense(O.Dh, H, W)
        Dv = _dense(O.Dv, H, W)
        Mat = A.T @ Mm @ A + gam * (Dh.T @ Dh + Dv.T @ Dv)
        denom = O.tv_denominator_diag(h, H, W, 1.0, gam)
    else:
        Mat = A.T @ Mm @ A + gam * np.eye(H * W)
        denom = np.abs(O.psf_otf(h, H, W)) ** 2 + gam
    r = g.standard_normal((H, W))
    x_dense = np.linalg.solve(Mat, r.ravel())
    x, xi = O.reeves_sorel_xstep(r, mask, h, denom, np.zeros((H, W)), cg_iters=400)
    np.testing.assert_allclose(x.ravel(), x_dense, atol=1e-10)
    assert np.all(xi[mask != 0] == 0)


def test_reeves_sorel_single_cg_step_is_exact_line_minimiser():
    """One CG iteration from a warm start xi0 on S xi = b (S = B C B^T - I,
    negative definite) is the exact minimiser of the quadratic
    1/2 xi^T (-S) xi + b^T xi along the residual direction: with dense B
    (rows of the convolution matrix at the unobserved pixels) and C, the new
    residual is orthogonal to the old one, and the error in the (-S) norm
    drops. Also: x = C r - C B^T xi for the returned xi."""
    H = W = 8
    g, h, mask = _cg_inputs(seed=62)
    gam = 0.11
    A = _dense_conv_loops(h, H, W)
    Dh = _dense(O.Dh, H, W)
    Dv = _dense(O.Dv, H, W)
    C = np.linalg.inv(A.T @ A + gam * (Dh.T @ Dh + Dv.T @ Dv))
    U = np.flatnonzero(mask.ravel() == 0)
    B = A[U]
    S_ = B @ C @ B.T - np.eye(len(U))
    r = g.standard_normal((H, W))
    b = B @ C @ r.ravel()
    xi0 = np.zeros((H, W))
    xi0.ravel()[U] = g.standard_normal(len(U))
    denom = O.tv_denominator_diag(h, H, W, 1.0, gam)
    x, xi = O.reeves_sorel_xstep(r, mask, h, denom, xi0, cg_iters=1)
    res0 = b - S_ @ xi0.ravel()[U]
    res1 = b - S_ @ xi.ravel()[U]
    assert abs(res0 @ res1) <= 1e-10 * (res0 @ res0)
    xs = np.linalg.solve(S_, b)
    e0, e1 = xi0.ravel()[U] - xs, xi.ravel()[U] - xs
    assert -(e1 @ S_ @ e1) < -(e0 @ S_ @ e0)
    np.testing.assert_allclose(x.ravel(), C @ r.ravel() - C @ B.T @ xi.ravel()[U], atol=1e-11)


def test_tvcg_equals_tvmd_when_everything_is_observed():
    """With M = I the set of unobserved pixels is empty: B has no rows, the
    x-step is the plain inverse, and TV-CG's iterates are TV-MD's (Sec. IV-D:
    the two methods differ only in how they treat M)."""
    g = S.rng(63)
    H, W = 16, 12
    h = S.psf_gaussian(5, 1.0)
    ybar = g.standard_normal((H, W))
    mask = np.ones((H, W), dtype=np.uint8)
    lam, mu1, mu2 = 0.02, 0.5, 0.2
    a = O.solve(ybar, mask, h, lam, mu1, mu2, "tv", iters=30)
    b = O.solve(ybar, mask, h, lam, mu1, mu2, "tv_cg", iters=30)
    np.testing.assert_allclose(b.x, a.x, atol=1e-11)
    c = O.solve(ybar, mask, h, lam, mu1, mu2, "haar", iters=20)
    d = O.solve(ybar, mask, h, lam, mu1, mu2, "haar_cg", iters=20)
    np.testing.assert_allclose(d.x, c.x, atol=1e-11)


@pytest.mark.parametrize("reg", ["tv", "haar"])
def test_cg_variants_reach_the_md_optimum(reg):
    """TV-CG / FA-CG and TV-MD / FA-MD minimise the same objective (eqs.
    unconstrained_TV_uBC and unconstrained_analysis_uBC): run to convergence
    on a 16 x 16 problem with the valid region and missing pixels, they reach
    the same objective value and the same x."""
    x, h, ybar, mask = _small_problem(seed=64)
    lam = 2e-3
    mu1, mu2 = 0.1, 10 * lam
    md = O.solve(ybar, mask, h, lam, mu1, mu2, reg, iters=6000, stop="rel_x", tol=1e-12)
    cg = O.solve(ybar, mask, h, lam, mu1, mu2, reg + "_cg", iters=6000, stop="rel_x", tol=1e-12)
    np.testing.assert_allclose(cg.objective, md.objective, rtol=1e-7)
    assert np.linalg.norm(cg.x - md.x) <= 1e-4 * np.linalg.norm(md.x)


def test_tvcg_kkt_certificate_at_convergence():
    """At a fixed point of TV-CG (u1 on the observed pixels only): -mu1 d1 =
    M A x - y on the observed pixels, mu1 A^T M^T d1 + mu2 D^T d2 = 0, and
    ||mu2 d2_i|| <= lambda."""
    x, h, ybar, mask = _small_problem(seed=65)
    lam = 2e-3
    mu1, mu2 = 0.1, 10 * lam
    r = O.solve(ybar, mask, h, lam, mu1, mu2, "tv_cg", iters=8000, stop="rel_x", tol=1e-13)
    st = r.state
    obs = mask != 0
    ax = O.A_direct(r.x, h)
    np.testing.assert_allclose(-mu1 * st.d1[obs], ax[obs] - ybar[obs], atol=1e-8)
    stat = mu1 * O.At_direct(np.where(obs, st.d1, 0.0), h) + mu2 * (O.DhT(st.d2[0]) + O.DvT(st.d2[1]))
    assert np.abs(stat).max() < 1e-8
    assert np.max(np.hypot(mu2 * st.d2[0], mu2 * st.d2[1])) <= lam * (1 + 1e-8)


# ----------------------------------------------------------------------------
# one penalty per band (Sec. II, eq. diagonal_penalty: a positive diagonal
# Upsilon, block-constant over each function g_j)
# ----------------------------------------------------------------------------
def _band_mu(levels=4, mu2=0.05):
    return mu2 * np.array([0.5, 2.0, 1.0] * levels + [0.25])[: 3 * levels + 1]


def test_band_spectra_closed_form_and_parseval():
    """|H_b|^2 of the a-trous Haar bands: with c_j = cos^2(pi k 2^j / N) and
    s_j = sin^2(pi k 2^j / N) per axis, level j's bands are prod_{i<j} c_i(r)
    c_i(c) times c_j(r) s_j(c), s_j(r) c_j(c), s_j(r) s_j(c) (rows low /
    columns high, rows high / columns low, both high), the last band
    prod_{i<L} c_i(r) c_i(c); they sum to 1 (P^T P = I)."""
    H, W, L = 16, 24, 3
    S_ = O.haar_band_spectra(H, W, L)
    kr = np.arange(H)[:, None] * np.ones((1, W))
    kc = np.ones((H, 1)) * np.arange(W)[None, :]
    cr = lambda j: np.cos(np.pi * kr * 2 ** j / H) ** 2
    sr = lambda j: np.sin(np.pi * kr * 2 ** j / H) ** 2
    cc = lambda j: np.cos(np.pi * kc * 2 ** j / W) ** 2
    sc = lambda j: np.sin(np.pi * kc * 2 ** j / W) ** 2
    chain = np.ones((H, W))
    for j in range(L):
        np.testing.assert_allclose(S_[3 * j], chain * cr(j) * sc(j), atol=1e-13)
        np.testing.assert_allclose(S_[3 * j + 1], chain * sr(j) * cc(j), atol=1e-13)
        np.testing.assert_allclose(S_[3 * j + 2], chain * sr(j) * sc(j), atol=1e-13)
        chain = chain * cr(j) * cc(j)
    np.testing.assert_allclose(S_[3 * L], chain, atol=1e-13)
    np.testing.assert_allclose(S_.sum(axis=0), 1.0, atol=1e-13)


def test_band_penalty_xstep_dense_solve():
    """eq. quadratic_problem with Upsilon = diag(mu1 I, mu_1 I, ..., mu_13 I)
    (one penalty per band) against a dense solve built from the dense band
    matrices; and the band thresholds lambda / mu_b."""
    H = W = 8
    g, h, st, ybar, mask = _one_step_inputs("haar")
    mu1, lam = 0.6, 0.02
    mub = _band_mu(4, 0.09)
    A = _dense(lambda v: O.A_direct(v, h), H, W)
    Pb = [_dense(lambda v, b=b: O.haar_analysis(v, 4)[b], H, W) for b in range(13)]
    Mat = mu1 * A.T @ A + sum(mub[b] * Pb[b].T @ Pb[b] for b in range(13))
    z2 = st.u2 + st.d2
    rhs = mu1 * A.T @ (st.u1 + st.d1).ravel() + sum(mub[b] * Pb[b].T @ z2[b].ravel() for b in range(13))
    x_dense = np.linalg.solve(Mat, rhs)
    nxt = O.famd_step(st, ybar, mask, h, lam, mu1, 0.09, 4, mu_bands=mub)
    np.testing.assert_allclose(nxt.x.ravel(), x_dense, atol=1e-11)
    c = np.stack([(Pb[b] @ x_dense).reshape(H, W) for b in range(13)])
    for b in range(13):
        s_ = c[b] - st.d2[b]
        np.testing.assert_allclose(nxt.u2[b], np.sign(s_) * np.maximum(np.abs(s_) - lam / mub[b], 0), atol=1e-11)
    # uniform band penalties give the scalar-penalty step exactly
    a = O.famd_step(st, ybar, mask, h, lam, mu1, 0.09, 4)
    b_ = O.famd_step(st, ybar, mask, h, lam, mu1, 0.09, 4, mu_bands=np.full(13, 0.09))
    np.testing.assert_allclose(b_.x, a.x, atol=1e-12)
    np.testing.assert_allclose(b_.d2, a.d2, atol=1e-12)


def test_band_penalties_reach_the_same_optimum():
    """Theorem 1 holds for any positive penalties: with one penalty per band
    the iteration converges to the same minimiser of eq.
    unconstrained_analysis_uBC as with a single mu2."""
    x, h, ybar, mask = _small_problem(seed=66)
    lam = 2e-3
    mu1, mu2 = 0.1, 10 * lam
    a = O.solve(ybar, mask, h, lam, mu1, mu2, "haar", iters=30000, stop="rel_x", tol=1e-13)
    b = O.solve(ybar, mask, h, lam, mu1, mu2, "haar", iters=30000, stop="rel_x", tol=1e-13,
                mu_bands=_band_mu(4, mu2))
    assert a.converged and b.converged
    np.testing.assert_allclose(b.objective, a.objective, rtol=1e-7)
    assert np.linalg.norm(b.x - a.x) <= 1e-4 * np.linalg.norm(a.x)
