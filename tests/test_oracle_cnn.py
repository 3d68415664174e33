"""Pins of the FP64 warm-start network oracle (oracle/cnn.py) against
definitions that do not come from the oracle itself: index loops, a library
cross-correlation, adjoint identities, finite differences, Adam's first steps
in closed form, and the ADMM fixed point (Theorem 1)."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.cnn as C
import synth as S


def _loops_conv(a, w, b):
    cin, H, W = a.shape
    out = np.zeros((w.shape[0], H, W))
    for o in range(w.shape[0]):
        for r in range(H):
            for c in range(W):
                s = b[o]
                for i in range(cin):
                    for p in (-1, 0, 1):
                        for q in (-1, 0, 1):
                            rr, cc = r + p, c + q
                            if 0 <= rr < H and 0 <= cc < W:
                                s += w[o, i, p + 1, q + 1] * a[i, rr, cc]
                out[o, r, c] = s
    return out


def test_conv_matches_index_loops():
    g = S.rng(1)
    a = g.standard_normal((2, 5, 4))
    w = g.standard_normal((3, 2, 3, 3))
    b = g.standard_normal(3)
    np.testing.assert_allclose(C.conv3x3(a, w, b), _loops_conv(a, w, b), rtol=0, atol=1e-13)


def test_conv_single_channel_is_library_correlation():
    scipy_signal = pytest.importorskip("scipy.signal")
    g = S.rng(2)
    a = g.standard_normal((1, 9, 7))
    w = g.standard_normal((1, 1, 3, 3))
    ref = scipy_signal.correlate2d(a[0], w[0, 0], mode="same", boundary="fill", fillvalue=0.0)
    np.testing.assert_allclose(C.conv3x3(a, w, np.zeros(1))[0], ref, rtol=0, atol=1e-13)


def test_grad_input_is_the_adjoint():
    g = S.rng(3)
    a = g.standard_normal((3, 6, 5))
    w = g.standard_normal((4, 3, 3, 3))
    gy = g.standard_normal((4, 6, 5))
    lhs = np.vdot(C.conv3x3(a, w, np.zeros(4)), gy)
    rhs = np.vdot(a, C.conv3x3_grad_input(gy, w))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_grad_weight_by_finite_differences():
    g = S.rng(4)
    a = g.standard_normal((2, 5, 6))
    w = g.standard_normal((3, 2, 3, 3))
    b = g.standard_normal(3)
    gy = g.standard_normal((3, 5, 6))
    gw, gb = C.conv3x3_grad_weight(gy, a)
    f = lambda w_, b_: float(np.vdot(gy, C.conv3x3(a, w_, b_)))
    h = 1e-6
    for idx in [(0, 0, 0, 0), (1, 1, 2, 1), (2, 0, 1, 2), (2, 1, 0, 0)]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        assert abs((f(wp, b) - f(wm, b)) / (2 * h) - gw[idx]) <= 1e-7 * (1 + abs(gw[idx]))
    for o in range(3):
        bp, bm = b.copy(), b.copy()
        bp[o] += h
        bm[o] -= h
        assert abs((f(w, bp) - f(w, bm)) / (2 * h) - gb[o]) <= 1e-7 * (1 + abs(gb[o]))


def test_network_gradients_by_finite_differences():
    """A 3-layer, width-4 network on two 6 x 5 images: every weight and bias
    gradient against central differences of the loss (FP64, rel 1e-6)."""
    g = S.rng(5)
    params = C.init_params(7, layers=3, width=4)
    for w, b in params:
        b[:] = g.standard_normal(b.shape) * 0.1
    inputs = [g.standard_normal((2, 6, 5)) for _ in range(2)]
    targets = [g.standard_normal((4, 6, 5)) for _ in range(2)]
    cw = np.array([1.0, 0.5, 2.0, 0.25])
    L, grads = C.batch_loss_and_grads(params, inputs, targets, cw)

    def loss(ps):
        return C.batch_loss_and_grads(ps, inputs, targets, cw)[0]

    h = 1e-6
    for k in range(len(params)):
        for j in range(2):
            flat = params[k][j].reshape(-1)
            for e in range(0, flat.size, max(1, flat.size // 7)):
                keep = flat[e]
                flat[e] = keep + h
                lp = loss(params)
                flat[e] = keep - h
                lm = loss(params)
                flat[e] = keep
                fd = (lp - lm) / (2 * h)
                an = grads[k][j].reshape(-1)[e]
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) * 10, (k, j, e, fd, an)


def test_relu_blocks_gradient():
    """A unit whose pre-activation is negative everywhere passes no gradient
    to the layers below it."""
    params = C.init_params(3, layers=2, width=1)
    params[0][0][:] = 0.0
    params[0][1][:] = -1.0            # z = -1 everywhere -> relu = 0
    a0 = S.rng(6).standard_normal((2, 4, 4))
    o, acts = C.forward(params, a0)
    gr = C.backward(params, acts, np.ones_like(o))
    assert np.all(gr[0][0] == 0.0) and np.all(gr[0][1] == 0.0)


def test_adam_first_two_steps_closed_form():
    """Step 1: m_hat = g, v_hat = g^2 -> theta -= lr g / (|g| + eps).
    Step 2 with gradients g1, g2 (scalar): m_hat = (0.9*0.1 g1 + 0.1 g2) / (1 - 0.81),
    v_hat = (0.999*0.001 g1^2 + 0.001 g2^2) / (1 - 0.999^2)."""
    p = [[np.array([[0.5, -0.25]]), np.array([1.0])]]
    opt = C.Adam(p, lr=0.01)
    g1 = [[np.array([[0.2, -3.0]]), np.array([1e-3])]]
    p = opt.step(p, g1)
    for theta0, g, theta in ((0.5, 0.2, p[0][0][0, 0]), (-0.25, -3.0, p[0][0][0, 1]), (1.0, 1e-3, p[0][1][0])):
        assert abs(theta - (theta0 - 0.01 * g / (abs(g) + 1e-8))) <= 1e-15
    g2 = [[np.array([[-0.1, 1.0]]), np.array([2e-3])]]
    before = p[0][0][0, 0]
    p = opt.step(p, g2)
    mh = (0.9 * 0.1 * 0.2 + 0.1 * -0.1) / (1 - 0.9 ** 2)
    vh = (0.999 * 0.001 * 0.04 + 0.001 * 0.01) / (1 - 0.999 ** 2)
    assert abs(p[0][0][0, 0] - (before - 0.01 * mh / (math.sqrt(vh) + 1e-8))) <= 1e-14


def test_network_input_zero_extends_the_observation():
    ybar = S.rng(8).standard_normal((5, 5))
    mask = np.zeros((5, 5), dtype=np.uint8)
    mask[1:4, 1:4] = 1
    a0 = C.network_input(ybar, mask)
    assert a0.shape == (2, 5, 5)
    assert np.all(a0[0][mask == 0] == 0.0) and np.all(a0[0][mask == 1] == ybar[mask == 1])
    assert np.all(a0[1] == mask)


@pytest.mark.parametrize("reg", ["tv", "haar"])
def test_warm_state_first_x_step_returns_x0(reg):
    g = S.rng(9)
    H, W = 24, 32
    psf = S.psf_gaussian(5, 1.0)
    x0 = g.uniform(size=(H, W))
    ybar, mask, _ = S.observe(g.uniform(size=(H, W)), psf, None, 40.0, g)
    nb = 2 if reg == "tv" else O.haar_nbands(4)
    d1 = g.standard_normal((H, W)) * 0.1
    d2 = g.standard_normal((nb, H, W)) * 0.05
    st = C.warm_state(x0, d1, d2, psf, reg)
    step = O.tvmd_step if reg == "tv" else O.famd_step
    s1 = step(st, ybar, mask, psf, 1e-3, 3e-2, 1e-2)
    np.testing.assert_allclose(s1.x, x0, rtol=0, atol=1e-12)
    # the dual update of that iteration starts from d0 (Algorithm 2, line 7)
    ax = O.A_fft(x0, psf)
    u1 = O.mask_prox(ax - d1, ybar, mask, 3e-2)
    np.testing.assert_allclose(s1.d1, d1 - (ax - u1), rtol=0, atol=1e-12)


def test_warm_start_at_the_fixed_point_stays_there():
    """Started from a nearly converged (x*, d*), TV-MD stays put: five more
    iterations move x by no more than five of the cold run's last steps (a
    start far from the fixed point moves it by orders of magnitude more)."""
    p = S.config1_problem(0)
    ref = O.solve(p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, "tv", iters=3000)
    st = C.warm_state(ref.x, ref.state.d1, ref.state.d2, p.psf, "tv")
    r = O.solve(p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, "tv", iters=5, state0=st)
    assert ref.rel_x < 1e-7
    assert np.linalg.norm(r.x - ref.x) <= 10 * 5 * ref.rel_x * np.linalg.norm(ref.x)
    # the same start without the duals is not a fixed point
    st0 = C.warm_state(ref.x, None, None, p.psf, "tv")
    r0 = O.solve(p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, "tv", iters=5, state0=st0)
    assert np.linalg.norm(r0.x - ref.x) >= 100 * np.linalg.norm(r.x - ref.x)
