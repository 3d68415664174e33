"""GPU parity of the Reeves-Sorel variants TV-CG and FA-CG (Sec. IV-C/IV-D,
"Using the Reeves-Sorel technique") against the FP64 oracle (tvcg_step,
facg_step): x after a few and after many iterations, the duals, the
relative-change stop rule, a batch mixing CG and MD problems, and the
degenerate case with every pixel observed (no inner system)."""
import numpy as np
import pytest

import oracle as O
import synth as S

pytestmark = pytest.mark.gpu

TOL_SHORT = 2e-5
TOL_X = 1e-4


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


def _problem(H, W, psf_fn, keep, seed, bsnr=40.0):
    g = S.rng(seed)
    x = S.textured_image(H, W, g)
    psf = psf_fn()
    keepm = None if keep is None else (g.uniform(size=(H, W)) < keep).astype(np.uint8)
    ybar, mask, _ = S.observe(x, psf, keepm, bsnr, g)
    return x, psf, ybar, mask


def _gpu(ad, reg, ybar, mask, psf, lam, mu1, mu2, iters, **kw):
    import torch
    H, W = ybar.shape
    plan = ad.Plan(H, W, psf, lam, mu1, mu2, reg, max_iters=iters, **kw)
    y = torch.from_numpy(ybar.astype(np.float32)).cuda()
    m = torch.from_numpy(mask).cuda()
    x = torch.empty((H, W), dtype=torch.float32, device="cuda")
    res = ad.solve(plan, y, m, x)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.float64), res, plan


CASES = [
    # reg, H, W, psf factory, keep, seed
    ("tv_cg", 64, 64, lambda: S.psf_box(9), None, 1),
    ("tv_cg", 128, 256, lambda: S.psf_motion(9.0, 30.0, 9), 0.6, 2),
    ("tv_cg", 512, 512, lambda: S.psf_gaussian(19, 3.0), 0.6, 3),
    ("tv_cg", 1024, 128, lambda: S.psf_box(13), None, 4),
    ("haar_cg", 64, 128, lambda: S.psf_gaussian(7, 1.5), 0.8, 5),
    ("haar_cg", 256, 256, lambda: S.psf_box(13), None, 6),
    ("haar_cg", 128, 1024, lambda: S.psf_motion(11.0, 120.0, 11), 0.7, 7),
]


@pytest.mark.parametrize("reg,H,W,psf_fn,keep,seed", CASES)
def test_iterates_and_duals_match_oracle(ad, reg, H, W, psf_fn, keep, seed):
    """x after 2, 3 and 10 iterations and the duals after 10: multi-tile,
    multi-strip domains, square and non-square, with and without missing
    pixels inside the valid region."""
    import torch
    _, psf, ybar, mask = _problem(H, W, psf_fn, keep, seed)
    lam = 3e-4
    mu1, mu2 = S.default_mu(lam)
    tv = reg == "tv_cg"
    st = O.State.zeros(H, W, "tv" if tv else "haar")
    for k in range(1, 11):
        st = (O.tvcg_step if tv else O.facg_step)(st, ybar, mask, psf, lam, mu1, mu2)
        if k in (2, 3, 10):
            x, res, plan = _gpu(ad, reg, ybar, mask, psf, lam, mu1, mu2, k)
            assert res.iters == k
            assert _rel(x, st.x) <= TOL_SHORT, (k, _rel(x, st.x))
    n = H * W
    d = torch.empty(plan.state_size(), dtype=torch.float32, device="cuda")
    ad.admm_deconv_get_state(plan.handle, d.data_ptr())
    d = d.cpu().numpy().astype(np.float64)
    d1 = d[:n].reshape(H, W)
    assert np.all(d1[mask == 0] == 0)
    assert np.max(np.abs(d1 - st.d1)) <= 2e-5 * np.abs(st.d1).max() + 1e-9
    if tv:
        d2 = d[n:].reshape(H, W, 2)
        for comp in (0, 1):
            assert np.max(np.abs(d2[..., comp] - st.d2[comp])) <= 2e-4 * (lam / mu2)
    else:
        d2 = d[n:].reshape(-1, H, W)
        assert np.max(np.abs(d2 - st.d2)) <= 2e-4 * (lam / mu2)
    plan.close()


@pytest.mark.parametrize("reg", ["tv_cg", "haar_cg"])
def test_long_run_and_objective_match_oracle(ad, reg):
    """200 iterations on a 128 x 128 deblur + inpainting problem: x within
    1e-4 relative, ISNR within 0.01 dB, objective within 1e-5 relative."""
    xt, psf, ybar, mask = _problem(128, 128, lambda: S.psf_gaussian(9, 2.0), 0.7, 21)
    lam = 1e-3
    mu1, mu2 = S.default_mu(lam)
    ref = O.solve(ybar, mask, psf, lam, mu1, mu2, reg, iters=200, record=True)
    x, res, plan = _gpu(ad, reg, ybar, mask, psf, lam, mu1, mu2, 200)
    assert res.iters == 200
    assert _rel(x, ref.x) <= TOL_X
    vm = S.valid_mask(128, 128, 9, 9)
    assert abs(O.isnr(xt, ybar, x, vm) - O.isnr(xt, ybar, ref.x, vm)) <= 0.01
    assert abs(res.objective - ref.objective) <= 1e-5 * ref.objective
    plan.close()


def test_rel_x_stop_matches_oracle(ad):
    """The relative-change rule (tol 1e-5, checked every iteration) stops
    TV-CG at the oracle's iteration up to rounding near the threshold."""
    _, psf, ybar, mask = _problem(128, 128, lambda: S.psf_box(7), 0.8, 22)
    lam = 1e-3
    mu1, mu2 = S.default_mu(lam)
    ref = O.solve(ybar, mask, psf, lam, mu1, mu2, "tv_cg", iters=4000, stop="rel_x", tol=1e-5)
    x, res, plan = _gpu(ad, "tv_cg", ybar, mask, psf, lam, mu1, mu2, 4000, stop="rel_x", tol=1e-5)
    assert ref.converged and res.converged == 1
    assert abs(res.iters - ref.iters) <= max(3, ref.iters // 100)
    assert _rel(x, ref.x) <= TOL_X
    plan.close()


def test_everything_observed_equals_md(ad):
    """With M = I (raw mask of ones) no pixel is unobserved: the inner system
    is empty, alpha is 0, and TV-CG's iterate is TV-MD's up to FP32 rounding."""
    g = S.rng(23)
    H = W = 128
    ybar = g.uniform(size=(H, W))
    mask = np.ones((H, W), dtype=np.uint8)
    psf = S.psf_gaussian(7, 1.5)
    lam = 1e-3
    mu1, mu2 = S.default_mu(lam)
    x_md, _, p1 = _gpu(ad, "tv", ybar, mask, psf, lam, mu1, mu2, 30, raw_mask=True)
    x_cg, _, p2 = _gpu(ad, "tv_cg", ybar, mask, psf, lam, mu1, mu2, 30, raw_mask=True)
    assert _rel(x_cg, x_md) <= 2e-6
    p1.close()
    p2.close()


def test_batch_mixing_cg_and_md_gives_solo_bits(ad):
    """A batch of TV-MD, TV-CG, FA-MD and FA-CG problems of two sizes gives
    each problem the bits of its solo solve."""
    import torch
    specs = [("tv", 128), ("tv_cg", 128), ("haar_cg", 128), ("tv_cg", 256), ("haar", 256), ("haar_cg", 256)]
    lam = 1e-3
    mu1, mu2 = S.default_mu(lam)
    plans, ys, ms, xs, solo = [], [], [], [], []
    for i, (reg, n) in enumerate(specs):
        _, psf, ybar, mask = _problem(n, n, lambda: S.psf_box(7), 0.8, 30 + i)
        x, _, p = _gpu(ad, reg, ybar, mask, psf, lam, mu1, mu2, 25)
        solo.append(x)
        plans.append(p)
        ys.append(torch.from_numpy(ybar.astype(np.float32)).cuda())
        ms.append(torch.from_numpy(mask).cuda())
        xs.append(torch.empty((n, n), dtype=torch.float32, device="cuda"))
    res = ad.solve_batch(plans, ys, ms, xs)
    torch.cuda.synchronize()
    for i in range(len(specs)):
        assert res[i].iters == 25
        assert np.array_equal(xs[i].cpu().numpy().astype(np.float64), solo[i]), specs[i]
    for p in plans:
        p.close()
