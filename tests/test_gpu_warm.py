"""GPU parity of the warm start (admm_deconv_warm_start) against the FP64
oracle: Algorithm 2 started from u0 = H x0 - d0 with given (x0, d0), which
Theorem 1 allows, for TV-MD and FA-MD; the start serves one solve; a batch
mixing warm and cold problems gives the bits of solving each alone."""
import numpy as np
import pytest

import oracle as O
import oracle.cnn as C
import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ad():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.init()
    import paper_1210_2687_gb300 as mod
    return mod


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _start(H, W, reg, seed, ybar):
    """A plausible, non-trivial start: the observation smoothed, plus random
    duals of the size the fixed point has (|d2| <= lambda / mu2)."""
    g = S.rng(seed)
    x0 = np.where(ybar != 0, ybar, ybar[ybar != 0].mean()) + 0.02 * g.standard_normal((H, W))
    nb = 2 if reg == "tv" else O.haar_nbands(4)
    d1 = 0.05 * g.standard_normal((H, W))
    d2 = 0.05 * g.standard_normal((nb, H, W))
    return x0, d1, d2


def _flat_state(d1, d2, reg):
    """admm_deconv_get_state layout: d1, then d2 (TV: (h, v) per pixel)."""
    if reg == "tv":
        return np.concatenate([d1.ravel(), np.stack([d2[0], d2[1]], axis=-1).ravel()]).astype(np.float32)
    return np.concatenate([d1.ravel(), d2.ravel()]).astype(np.float32)


@pytest.mark.parametrize("reg,H,W,psf_fn,keep", [
    ("tv", 64, 64, lambda: S.psf_box(9), None),
    ("tv", 256, 128, lambda: S.psf_motion(11.0, 30.0, 11), 0.7),
    ("haar", 128, 128, lambda: S.psf_gaussian(7, 1.5), 0.8),
    ("haar", 64, 256, lambda: S.psf_box(5), None),
])
def test_warm_start_matches_oracle(ad, reg, H, W, psf_fn, keep):
    import torch
    psf = psf_fn()
    g = S.rng(31)
    x = S.textured_image(H, W, g)
    km = None if keep is None else (g.uniform(size=(H, W)) < keep).astype(np.uint8)
    ybar, mask, _ = S.observe(x, psf, km, 40.0, g)
    lam, mu1, mu2 = 1e-3, 3e-2, 1e-2
    x0, d1, d2 = _start(H, W, reg, 32, ybar)
    st = C.warm_state(x0, d1, d2, psf, reg)
    step = O.tvmd_step if reg == "tv" else O.famd_step
    y_d = torch.from_numpy(ybar.astype(np.float32)).cuda()
    m_d = torch.from_numpy(mask).cuda()
    x0_d = torch.from_numpy(x0.astype(np.float32)).cuda()
    dflat = torch.from_numpy(_flat_state(d1, d2, reg)).cuda()
    for k in range(1, 11):
        st = step(st, ybar, mask, psf, lam, mu1, mu2)
        if k in (1, 2, 10):
            plan = ad.Plan(H, W, psf, lam, mu1, mu2, reg, max_iters=k)
            plan.warm_start(x0_d, dflat)
            xo = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
            r = ad.solve(plan, y_d, m_d, xo)
            torch.cuda.synchronize()
            assert r.iters == k
            assert _rel(xo.cpu().numpy().astype(np.float64), st.x) <= 2e-5, (k, reg)
    n = H * W
    d = torch.empty(plan.state_size(), dtype=torch.float32, device="cuda")
    ad.admm_deconv_get_state(plan.handle, d.data_ptr())
    torch.cuda.synchronize()
    d = d.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(d[:n].reshape(H, W) - st.d1)) <= 2e-5 * np.abs(st.d1).max() + 1e-9


def test_warm_start_from_host_buffers_and_null_duals(ad):
    import torch
    p = S.config1_problem(0)
    x0 = np.ascontiguousarray(np.clip(p.ybar, 0, 1).astype(np.float32))
    st = C.warm_state(x0.astype(np.float64), None, None, p.psf, "tv")
    for _ in range(5):
        st = O.tvmd_step(st, p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2)
    plan = ad.Plan(64, 64, p.psf, p.lam, p.mu1, p.mu2, "tv", max_iters=5)
    plan.warm_start(x0, None)                       # host x0, zero duals
    xo = np.full((64, 64), np.nan, dtype=np.float32)
    r = ad.solve(plan, p.ybar.astype(np.float32), p.mask, xo)
    assert r.iters == 5
    assert _rel(xo.astype(np.float64), st.x) <= 2e-5


def test_warm_start_serves_one_solve(ad):
    import torch
    p = S.config1_problem(0)
    y = torch.from_numpy(p.ybar.astype(np.float32)).cuda()
    m = torch.from_numpy(p.mask).cuda()
    plan = ad.Plan(64, 64, p.psf, p.lam, p.mu1, p.mu2, "tv", max_iters=20)
    cold = torch.empty((64, 64), dtype=torch.float32, device="cuda")
    ad.solve(plan, y, m, cold)
    plan.warm_start(torch.ones((64, 64), dtype=torch.float32, device="cuda"), None)
    warm = torch.empty_like(cold)
    ad.solve(plan, y, m, warm)
    again = torch.empty_like(cold)
    ad.solve(plan, y, m, again)
    torch.cuda.synchronize()
    assert not torch.equal(warm, cold)
    assert torch.equal(again, cold)


def test_restart_from_own_solution_stops_at_once(ad):
    """Warm-started from a converged solve's (x, d), the rel-x rule is met
    within a few iterations of the first one where it is evaluated."""
    import torch
    p = S.config2_problem(3, "gauss", 40, size=256)
    lam = 1e-3                      # a weight at which rel-x < 1e-5 means close to the fixed point
    mu1, mu2 = S.default_mu(lam)
    y = torch.from_numpy(p.ybar.astype(np.float32)).cuda()
    m = torch.from_numpy(p.mask).cuda()
    plan = ad.Plan(256, 256, p.psf, lam, mu1, mu2, "tv", stop="rel_x", tol=1e-5, max_iters=5000,
                   check_every=1)
    x = torch.empty((256, 256), dtype=torch.float32, device="cuda")
    r = ad.solve(plan, y, m, x)
    assert r.converged == 1 and r.iters > 50
    d = torch.empty(plan.state_size(), dtype=torch.float32, device="cuda")
    ad.admm_deconv_get_state(plan.handle, d.data_ptr())
    plan.warm_start(x.clone(), d)
    x2 = torch.empty_like(x)
    r2 = ad.solve(plan, y, m, x2)
    torch.cuda.synchronize()
    assert r2.converged == 1 and r2.iters <= 5, r2.iters
    assert _rel(x2.cpu().numpy().astype(np.float64), x.cpu().numpy().astype(np.float64)) < 1e-4


def test_batch_mixing_warm_and_cold_problems(ad):
    import torch
    specs = [(64, 64, "tv", True), (64, 64, "tv", False), (128, 128, "haar", True), (128, 128, "haar", False),
             (128, 64, "tv", True)]
    plans, ys, ms, xs, starts = [], [], [], [], []
    for i, (H, W, reg, warm) in enumerate(specs):
        psf = S.psf_gaussian(5, 1.0)
        g = S.rng(50 + i)
        ybar, mask, _ = S.observe(S.textured_image(H, W, g), psf, None, 40.0, g)
        plans.append(ad.Plan(H, W, psf, 1e-3, 3e-2, 1e-2, reg, max_iters=12))
        ys.append(torch.from_numpy(ybar.astype(np.float32)).cuda())
        ms.append(torch.from_numpy(mask).cuda())
        xs.append(torch.empty((H, W), dtype=torch.float32, device="cuda"))
        if warm:
            x0, d1, d2 = _start(H, W, reg, 60 + i, ybar)
            starts.append((torch.from_numpy(x0.astype(np.float32)).cuda(),
                           torch.from_numpy(_flat_state(d1, d2, reg)).cuda()))
        else:
            starts.append(None)
    for pl, s0 in zip(plans, starts):
        if s0 is not None:
            pl.warm_start(*s0)
    ad.solve_batch(plans, ys, ms, xs)
    torch.cuda.synchronize()
    for i in range(len(specs)):
        if starts[i] is not None:
            plans[i].warm_start(*starts[i])
        xo = torch.empty_like(xs[i])
        ad.solve(plans[i], ys[i], ms[i], xo)
        torch.cuda.synchronize()
        assert torch.equal(xo, xs[i]), i
