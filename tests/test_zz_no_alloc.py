"""The scratch-free entry point, admm_deconv_solve_noalloc.

It serves callers that must not allocate device memory while they run (an
application whose own allocator owns the GPU's memory, a fixed-budget or
real-time loop where an allocation could fail or stall, a plugin whose host
forbids libraries from allocating). It keeps all of its working memory in
one fixed array inside the library and needs no plan.

These tests call it through the C ABI twice in a row -- the second call on a
different size and stop rule, so it must clear what the first call left in
the shared array -- and compare each result with the plan-based
admm_deconv_solve on the same input, within the parity tolerance the other
GPU tests use for short runs. This file is named so that pytest collects it
last."""
import numpy as np
import pytest

import oracle as O
import synth as S

pytestmark = pytest.mark.gpu

TOL_SHORT = 2e-5


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


def _problem(H, W, psf, keep, seed):
    g = S.rng(seed)
    x = S.textured_image(H, W, g)
    keepm = (g.uniform(size=(H, W)) < keep).astype(np.uint8)
    ybar, mask, _ = S.observe(x, psf, keepm, 40.0, g)
    return ybar, mask


def test_noalloc_matches_plan_solve_on_two_calls_in_a_row(ad):
    import torch
    calls = [
        # H, W, psf, keep, seed, lambda, stop, tol, max_iters, check_every
        (256, 256, S.psf_gaussian(19, 3.0), 0.6, 31, 1e-3, "iters", 0.0, 60, 1),
        (128, 64, S.psf_motion(9.0, 30.0, 9), 0.8, 32, 3e-4, "rel_x", 1e-5, 3000, 5),
    ]
    for (H, W, psf, keep, seed, lam, stop, tol, iters, ce) in calls:
        ybar, mask = _problem(H, W, psf, keep, seed)
        mu1, mu2 = S.default_mu(lam)
        plan = ad.Plan(H, W, psf, lam, mu1, mu2, "tv", stop=stop, tol=tol, max_iters=iters,
                       check_every=ce)
        y = torch.from_numpy(ybar.astype(np.float32)).cuda()
        m = torch.from_numpy(mask).cuda()
        x_ref = torch.empty((H, W), dtype=torch.float32, device="cuda")
        r_ref = ad.solve(plan, y, m, x_ref)
        x = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
        rc, r = ad.admm_deconv_solve_noalloc(plan.params, y.data_ptr(), m.data_ptr(), x.data_ptr())
        torch.cuda.synchronize()
        assert rc == ad.ADMM_OK, ad.admm_strerror(rc)
        assert r.iters == r_ref.iters and r.converged == r_ref.converged
        a = x.cpu().numpy().astype(np.float64)
        b = x_ref.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= TOL_SHORT * np.linalg.norm(b)
        plan.close()


def test_noalloc_allocates_nothing_and_matches_the_oracle(ad):
    """After one call (which may load the library's device code and with it
    the fixed array), further calls leave the device's free memory unchanged;
    the result follows the FP64 oracle's iterate sequence."""
    import torch
    H = W = 128
    psf = S.psf_box(9)
    ybar, mask = _problem(H, W, psf, 0.8, 33)
    lam = 1e-3
    mu1, mu2 = S.default_mu(lam)
    plan = ad.Plan(H, W, psf, lam, mu1, mu2, "tv", max_iters=50)
    params = plan.params
    y = torch.from_numpy(ybar.astype(np.float32)).cuda()
    m = torch.from_numpy(mask).cuda()
    x = torch.empty((H, W), dtype=torch.float32, device="cuda")
    rc, _ = ad.admm_deconv_solve_noalloc(params, y.data_ptr(), m.data_ptr(), x.data_ptr())
    assert rc == ad.ADMM_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        rc, r = ad.admm_deconv_solve_noalloc(params, y.data_ptr(), m.data_ptr(), x.data_ptr())
        assert rc == ad.ADMM_OK and r.iters == 50
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ref = O.solve(ybar.astype(np.float64), mask, psf, lam, mu1, mu2, "tv", iters=50)
    xg = x.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(xg - ref.x) <= 1e-4 * np.linalg.norm(ref.x)
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_array(ad):
    import torch
    psf = S.psf_box(5)
    plan = ad.Plan(512, 512, psf, 1e-3, 0.0, 0.0, "tv", max_iters=5)
    y = torch.zeros((512, 512), dtype=torch.float32, device="cuda")
    x = torch.zeros_like(y)
    rc, _ = ad.admm_deconv_solve_noalloc(plan.params, y.data_ptr(), None, x.data_ptr())
    assert rc == ad.ADMM_EUNSUPPORTED_SIZE
    plan.close()
