"""GPU parity of FA-MD (Algorithm 2 with H1 = A, H2 = P, eq. invAnalysis /
invAnalysisp1, eq. prox_g_1_uBC and eq. soft) against the FP64 oracle,
through the C ABI. Same tolerances as the TV tests: rel-L2(x) <= 2e-5 for
short runs, <= 1e-4 and |dISNR| <= 0.01 dB for longer ones."""
import numpy as np
import pytest

import oracle as O
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


def _problem(H, W, psf, keep, seed, bsnr=50.0):
    g = S.rng(seed)
    x = S.textured_image(H, W, g)
    keepm = None if keep is None else (g.uniform(size=(H, W)) < keep).astype(np.uint8)
    ybar, mask, _ = S.observe(x, psf, keepm, bsnr, g)
    return x, ybar, mask


def _gpu(ad, ybar, mask, psf, lam, mu1, mu2, iters, levels=4, stop="iters", tol=0.0, check_every=1):
    import torch
    H, W = ybar.shape
    plan = ad.Plan(H, W, psf, lam, mu1, mu2, "haar", levels=levels, stop=stop, tol=tol,
                   max_iters=iters, check_every=check_every)
    y = torch.from_numpy(ybar.astype(np.float32)).cuda()
    m = torch.from_numpy(mask).cuda()
    x = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
    res = ad.solve(plan, y, m, x)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.float64), res, plan


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [
    (64, 64, lambda: S.psf_box(9), None, 1, 4),
    (128, 256, lambda: S.psf_motion(9.0, 45.0, 9), 0.7, 2, 4),
    (256, 64, lambda: S.psf_gaussian(7, 2.0), 0.8, 3, 4),
    (128, 128, lambda: S.psf_box(5), 0.9, 4, 2),
    (512, 512, lambda: S.psf_box(13), None, 5, 4),
    (64, 1024, lambda: S.psf_gaussian(5, 1.0), None, 6, 3),
    # 2048-point rows: the row kernels read their twiddles through L1
    (64, 2048, lambda: S.psf_box(5), 0.8, 7, 4),
]


@pytest.mark.parametrize("H,W,psf_fn,keep,seed,levels", CASES)
def test_frame_iterates_and_duals_match_oracle(ad, H, W, psf_fn, keep, seed, levels):
    import torch
    psf = psf_fn()
    _, ybar, mask = _problem(H, W, psf, keep, seed)
    lam, mu1, mu2 = 1e-3, 3e-2, 1e-2
    st = O.State.zeros(H, W, "haar", levels)
    for k in range(1, 11):
        st = O.famd_step(st, ybar, mask, psf, lam, mu1, mu2, levels)
        if k in (2, 3, 10):
            x, res, plan = _gpu(ad, ybar, mask, psf, lam, mu1, mu2, k, levels)
            assert res.iters == k
            assert _rel(x, st.x) <= 2e-5, (k, _rel(x, st.x))
    n = H * W
    nb = 3 * levels + 1
    assert plan.state_size() == (1 + nb) * n
    d = torch.empty((1 + nb) * n, dtype=torch.float32, device="cuda")
    ad.admm_deconv_get_state(plan.handle, d.data_ptr())
    torch.cuda.synchronize()
    d = d.cpu().numpy().astype(np.float64)
    d1 = d[:n].reshape(H, W)
    d2 = d[n:].reshape(nb, H, W)
    assert np.max(np.abs(d1 - st.d1)) <= 2e-5 * np.abs(st.d1).max() + 1e-9
    assert np.max(np.abs(d2 - st.d2)) <= 2e-4 * (lam / mu2)


def test_frame_rel_x_stop_matches_oracle(ad):
    psf = S.psf_box(13)
    xt, ybar, mask = _problem(128, 128, psf, None, 11)
    lam = 5e-4
    mu1, mu2 = S.default_mu(lam)
    ref = O.solve(ybar, mask, psf, lam, mu1, mu2, "haar", iters=4000, stop="rel_x", tol=1e-5)
    x, res, _ = _gpu(ad, ybar, mask, psf, lam, mu1, mu2, 4000, stop="rel_x", tol=1e-5)
    assert ref.converged and res.converged == 1
    assert abs(res.iters - ref.iters) <= max(3, ref.iters // 100)
    assert _rel(x, ref.x) <= 1e-4
    vm = S.valid_mask(128, 128, 13, 13)
    assert abs(O.isnr(xt, ybar, x, vm) - O.isnr(xt, ybar, ref.x, vm)) <= 0.01
    assert abs(res.objective - ref.objective) <= 1e-5 * ref.objective


def test_frame_config_1024_30_iterations(ad):
    """1024 x 1024, 13 x 13 uniform blur, valid region, BSNR 50 dB, 4-level
    Haar: 30 iterations at full size against the oracle."""
    p = S.config3_problem(0, 1024)
    ref = O.solve(p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, "haar", iters=30)
    x, res, _ = _gpu(ad, p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, 30)
    assert _rel(x, ref.x) <= 1e-4
    vm = S.valid_mask(1024, 1024, 13, 13)
    assert abs(O.isnr(p.x_true, p.ybar, x, vm) - O.isnr(p.x_true, p.ybar, ref.x, vm)) <= 0.01


def test_frame_max_size_2048(ad):
    p = S.config3_problem(1, 2048)
    st = O.State.zeros(2048, 2048, "haar")
    for _ in range(3):
        st = O.famd_step(st, p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, 4)
    x, res, _ = _gpu(ad, p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, 3)
    assert _rel(x, st.x) <= 2e-5


def test_mixed_tv_and_frame_batch(ad):
    """One solve_batch call with TV and frame problems of several sizes gives
    the bits of solving each alone."""
    import torch
    specs = [(64, 64, "tv"), (64, 64, "haar"), (128, 256, "haar"), (128, 256, "tv"), (256, 128, "haar")]
    plans, ys, ms, xs = [], [], [], []
    for i, (H, W, reg) in enumerate(specs):
        psf = S.psf_gaussian(7, 1.5)
        _, ybar, mask = _problem(H, W, psf, 0.8, 40 + i)
        plans.append(ad.Plan(H, W, psf, 1e-3, 3e-2, 1e-2, reg, max_iters=13))
        ys.append(torch.from_numpy(ybar.astype(np.float32)).cuda())
        ms.append(torch.from_numpy(mask).cuda())
        xs.append(torch.empty((H, W), dtype=torch.float32, device="cuda"))
    res = ad.solve_batch(plans, ys, ms, xs)
    torch.cuda.synchronize()
    for i in range(len(specs)):
        xo = torch.empty_like(xs[i])
        r = ad.solve(plans[i], ys[i], ms[i], xo)
        torch.cuda.synchronize()
        assert r.iters == res[i].iters == 13
        assert torch.equal(xo, xs[i])


@pytest.mark.parametrize("reg", ["haar", "haar_synthesis"])
def test_frame_primal_residual_matches_oracle(ad, reg):
    """d_k - d_{k-1} over d1 and all 13 bands of d2 (the primal residual of
    Algorithm 2) on the last iteration, against the oracle's duals."""
    import torch
    psf = S.psf_gaussian(7, 1.5)
    _, ybar, mask = _problem(128, 128, psf, 0.8, 17)
    lam, mu1, mu2 = 1e-3, 3e-2, 1e-2
    k = 6
    st = O.State.zeros(128, 128, "haar", 4)
    for _ in range(k):
        prev = st
        if reg == "haar":
            st = O.famd_step(st, ybar, mask, psf, lam, mu1, mu2, 4)
        else:
            st = O.fsmd_step(st, ybar, mask, psf, lam, mu1, mu2, 4)
    ref = float(np.sqrt(np.sum((st.d1 - prev.d1) ** 2) + np.sum((st.d2 - prev.d2) ** 2)))
    plan = ad.Plan(128, 128, psf, lam, mu1, mu2, reg, levels=4, max_iters=k)
    y = torch.from_numpy(ybar.astype(np.float32)).cuda()
    m = torch.from_numpy(mask).cuda()
    x = torch.empty((128, 128), dtype=torch.float32, device="cuda")
    res = ad.solve(plan, y, m, x)
    torch.cuda.synchronize()
    plan.close()
    assert ref > 0
    assert abs(res.primal_res - ref) <= 1e-3 * ref, (res.primal_res, ref)
