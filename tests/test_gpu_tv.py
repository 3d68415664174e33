"""GPU parity of TV-MD (Algorithm 3 with line 7 replaced by eq. new_line)
against the FP64 oracle, through the C ABI.

Tolerance: relative L2 error of x <= 1e-4 after a fixed iteration count and
|ISNR difference| <= 0.01 dB (FP32 arithmetic with FP32 FFTs against FP64).
Short runs (a few iterations) are held to 2e-5."""
import math

import numpy as np
import pytest

import oracle as O
import synth as S

pytestmark = pytest.mark.gpu

TOL_X = 1e-4
TOL_ISNR_DB = 0.01


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


def _gpu_solve(ad, ybar, mask, psf, lam, mu1, mu2, iters, stop="iters", tol=0.0, check_every=1,
               raw_mask=False, reg="tv"):
    import torch
    H, W = ybar.shape
    plan = ad.Plan(H, W, psf, lam, mu1, mu2, reg, stop=stop, tol=tol, max_iters=iters,
                   check_every=check_every, raw_mask=raw_mask)
    y = torch.from_numpy(ybar.astype(np.float32)).cuda()
    m = torch.from_numpy(mask.astype(np.uint8)).cuda()
    x = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
    res = ad.solve(plan, y, m, x)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.float64), res, plan


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_config1_200_iterations(ad):
    """64 x 64, 9 x 9 box, valid region, BSNR 40 dB, lambda 1e-3, 200 iterations."""
    p = S.config1_problem(0)
    ref = O.solve(p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, "tv", iters=200)
    x, res, _ = _gpu_solve(ad, p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, 200)
    assert res.iters == 200 and res.status == 0
    assert _rel(x, ref.x) <= TOL_X
    vm = S.valid_mask(64, 64, 9, 9)
    d_isnr = O.isnr(p.x_true, p.ybar, x, vm) - O.isnr(p.x_true, p.ybar, ref.x, vm)
    assert abs(d_isnr) <= TOL_ISNR_DB
    assert abs(res.objective - ref.objective) <= 1e-5 * ref.objective


CASES = [
    # H, W, psf factory, keep fraction, seed
    (64, 64, lambda: S.psf_box(9), None, 1),
    (128, 64, lambda: S.psf_motion(7.0, 30.0, 7), 0.7, 2),
    (64, 256, lambda: S.psf_gaussian(5, 1.5), 0.5, 3),
    (256, 128, lambda: S.psf_motion(11.0, 120.0, 11), 0.8, 4),
    (512, 512, lambda: S.psf_gaussian(19, 3.0), 0.6, 5),
    (128, 1024, lambda: S.psf_box(13), None, 6),
    (1024, 128, lambda: S.psf_disk(7), 0.9, 7),
]


def _case_problem(H, W, psf_fn, keep, seed, bsnr=40.0):
    g = S.rng(seed)
    x = S.textured_image(H, W, g)
    psf = psf_fn()
    keepm = None if keep is None else (g.uniform(size=(H, W)) < keep).astype(np.uint8)
    ybar, mask, _ = S.observe(x, psf, keepm, bsnr, g)
    return x, psf, ybar, mask


@pytest.mark.parametrize("H,W,psf_fn,keep,seed", CASES)
def test_iterates_and_duals_match_oracle(ad, H, W, psf_fn, keep, seed):
    """x after 2, 3 and 12 iterations and the duals (d1, d2) after 12, on
    square and non-square domains, every supported row/column length pair
    covering several tiles and strips."""
    import torch
    x_true, psf, ybar, mask = _case_problem(H, W, psf_fn, keep, seed)
    lam, mu1, mu2 = 3e-4, 1.0, 3e-3
    st = O.State.zeros(H, W, "tv")
    for k in range(1, 13):
        st = O.tvmd_step(st, ybar, mask, psf, lam, mu1, mu2)
        if k in (2, 3, 12):
            x, res, plan = _gpu_solve(ad, ybar, mask, psf, lam, mu1, mu2, k)
            assert res.iters == k
            assert _rel(x, st.x) <= 2e-5, (k, _rel(x, st.x))
    n = H * W
    d = torch.empty(3 * n, dtype=torch.float32, device="cuda")
    assert plan.state_size() == 3 * n
    ad.admm_deconv_get_state(plan.handle, d.data_ptr())
    torch.cuda.synchronize()
    d = d.cpu().numpy().astype(np.float64)
    d1 = d[:n].reshape(H, W)
    d2 = d[n:].reshape(H, W, 2)
    scale1 = np.abs(st.d1).max()
    assert np.max(np.abs(d1 - st.d1)) <= 2e-5 * scale1 + 1e-9
    for comp in (0, 1):
        ref = st.d2[comp]
        assert np.max(np.abs(d2[..., comp] - ref)) <= 2e-4 * (lam / mu2)


def test_rel_x_stop_matches_oracle(ad):
    """Stop rule ||x_k - x_{k-1}|| / ||x_k|| < 1e-5 (the 512^2 workload's rule)
    on a 128 x 128 inpainting problem: same iteration count up to rounding
    near the threshold, and the same solution."""
    x_true, psf, ybar, mask = _case_problem(128, 128, lambda: S.psf_gaussian(19, 3.0), 0.6, 11)
    lam = 2e-4
    mu1, mu2 = S.default_mu(lam)
    ref = O.solve(ybar, mask, psf, lam, mu1, mu2, "tv", iters=5000, stop="rel_x", tol=1e-5)
    x, res, _ = _gpu_solve(ad, ybar, mask, psf, lam, mu1, mu2, 5000, stop="rel_x", tol=1e-5)
    assert ref.converged and res.converged == 1
    assert abs(res.iters - ref.iters) <= max(3, ref.iters // 100)
    assert res.rel_x < 1e-5
    assert _rel(x, ref.x) <= TOL_X
    vm = S.valid_mask(128, 128, 19, 19)
    d_isnr = O.isnr(x_true, ybar, x, vm) - O.isnr(x_true, ybar, ref.x, vm)
    assert abs(d_isnr) <= TOL_ISNR_DB


def test_check_every_evaluates_consecutive_iterates(ad):
    """With check_every = 10 the rel-x rule is evaluated at multiples of 10 on
    (x_k, x_{k-1}); the stopping iteration is the first such k below tol."""
    x_true, psf, ybar, mask = _case_problem(64, 128, lambda: S.psf_box(7), 0.8, 12)
    lam = 2e-4
    mu1, mu2 = S.default_mu(lam)
    hist = O.solve(ybar, mask, psf, lam, mu1, mu2, "tv", iters=3000, record=True)
    rel = {h[0]: h[2] for h in hist.history}
    expect = next(k for k in range(10, 3001, 10) if rel[k] < 1e-5)
    x, res, _ = _gpu_solve(ad, ybar, mask, psf, lam, mu1, mu2, 3000, stop="rel_x", tol=1e-5, check_every=10)
    assert res.converged == 1 and res.iters % 10 == 0
    assert abs(res.iters - expect) <= 10


def test_rel_obj_stop_paper_rule(ad):
    """Sec. V's rule: relative variation of the objective below 1e-4."""
    p = S.config1_problem(3)
    ref = O.solve(p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, "tv", iters=3000, stop="rel_obj", tol=1e-4)
    x, res, _ = _gpu_solve(ad, p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, 3000, stop="rel_obj", tol=1e-4)
    assert ref.converged and res.converged == 1
    assert abs(res.iters - ref.iters) <= max(3, ref.iters // 50)
    assert res.rel_obj < 1e-4
    assert _rel(x, ref.x) <= 1e-3


def test_batch_equals_individual_solves(ad):
    """solve_batch over problems of different sizes and kernels gives the
    bit-identical result of solving each alone."""
    import torch
    probs = [_case_problem(*c[:2], c[2], c[3], c[4]) for c in CASES[:4]] + \
            [_case_problem(64, 64, lambda: S.psf_gaussian(7, 2.0), 0.5, 21)]
    plans, ys, ms, xs, singles = [], [], [], [], []
    for (xt, psf, ybar, mask) in probs:
        H, W = ybar.shape
        plans.append(ad.Plan(H, W, psf, 3e-4, 1.0, 3e-3, "tv", max_iters=17))
        ys.append(torch.from_numpy(ybar.astype(np.float32)).cuda())
        ms.append(torch.from_numpy(mask).cuda())
        xs.append(torch.empty((H, W), dtype=torch.float32, device="cuda"))
    res = ad.solve_batch(plans, ys, ms, xs)
    torch.cuda.synchronize()
    for i, (pl, y, m) in enumerate(zip(plans, ys, ms)):
        xo = torch.empty_like(xs[i])
        r = ad.solve(pl, y, m, xo)
        torch.cuda.synchronize()
        assert r.iters == res[i].iters == 17
        assert torch.equal(xo, xs[i])


def test_queued_problems_start_as_slots_free_up(ad):
    """More problems than launch slots: with ADMM_OPT_MAX_SLOTS = 2, seven
    problems (TV and frame, different sizes, stop rules and iteration
    counts) queue and take over slots as others retire; every result is the
    bit-exact result of solving the problem alone."""
    import torch
    specs = [(64, 64, "tv", "rel_x", 1e-5, 3000), (64, 64, "tv", "iters", 0.0, 9),
             (64, 64, "tv", "iters", 0.0, 31), (64, 64, "tv", "rel_x", 1e-4, 3000),
             (128, 64, "haar", "iters", 0.0, 12), (128, 64, "haar", "rel_x", 1e-4, 3000),
             (128, 64, "haar", "iters", 0.0, 5)]
    plans, ys, ms, xs = [], [], [], []
    for i, (H, W, reg, stop, tol, it) in enumerate(specs):
        xt, psf, ybar, mask = _case_problem(H, W, lambda: S.psf_gaussian(7, 1.5), 0.8, 60 + i)
        lam = 3e-4
        mu1, mu2 = S.default_mu(lam)
        plans.append(ad.Plan(H, W, psf, lam, mu1, mu2, reg, stop=stop, tol=tol, max_iters=it, check_every=2))
        ys.append(torch.from_numpy(ybar.astype(np.float32)).cuda())
        ms.append(torch.from_numpy(mask).cuda())
        xs.append(torch.empty((H, W), dtype=torch.float32, device="cuda"))
    ad.admm_deconv_set_option(ad.ADMM_OPT_MAX_SLOTS, 2)
    try:
        res = ad.solve_batch(plans, ys, ms, xs)
        torch.cuda.synchronize()
    finally:
        ad.admm_deconv_set_option(ad.ADMM_OPT_MAX_SLOTS, 0)
    for i in range(len(specs)):
        xo = torch.empty_like(xs[i])
        r = ad.solve(plans[i], ys[i], ms[i], xo)
        torch.cuda.synchronize()
        assert r.iters == res[i].iters and r.converged == res[i].converged
        assert torch.equal(xo, xs[i]), i


def test_graph_replay_equals_direct_launches(ad):
    """Chunks of iterations replay as CUDA graphs; with per-phase timing on,
    the same iterations run as individual launches. Same bits either way."""
    import torch
    xt, psf, ybar, mask = _case_problem(128, 128, lambda: S.psf_gaussian(9, 2.0), 0.7, 70)
    plan = ad.Plan(128, 128, psf, 3e-4, 1e-2, 3e-3, "tv", max_iters=37)
    y = torch.from_numpy(ybar.astype(np.float32)).cuda()
    m = torch.from_numpy(mask).cuda()
    xa = torch.empty((128, 128), dtype=torch.float32, device="cuda")
    xb = torch.empty_like(xa)
    ra = ad.solve(plan, y, m, xa)
    ad.admm_deconv_profile(True)
    rb = ad.solve(plan, y, m, xb)
    prof = ad.admm_deconv_profile(False)
    torch.cuda.synchronize()
    # launches continue until the host sees the retirement, one chunk behind
    assert prof.col_launches == prof.row_launches >= 37
    assert ra.iters == rb.iters == 37
    assert torch.equal(xa, xb)


def test_host_buffers_equal_device_buffers(ad):
    """y, mask and x_out in host memory take the staging path; same bits."""
    import torch
    xt, psf, ybar, mask = _case_problem(128, 256, lambda: S.psf_motion(9.0, 60.0, 9), 0.7, 13)
    plan = ad.Plan(128, 256, psf, 3e-4, 1.0, 3e-3, "tv", max_iters=9)
    yh = np.ascontiguousarray(ybar.astype(np.float32))
    xh = np.zeros((128, 256), dtype=np.float32)
    r1 = ad.solve(plan, yh, np.ascontiguousarray(mask), xh)
    xd = torch.empty((128, 256), dtype=torch.float32, device="cuda")
    r2 = ad.solve(plan, torch.from_numpy(yh).cuda(), torch.from_numpy(mask).cuda(), xd)
    torch.cuda.synchronize()
    assert r1.iters == r2.iters == 9
    assert np.array_equal(xh, xd.cpu().numpy())


def test_pinned_host_buffers_equal_device_buffers(ad):
    """Page-locked host buffers (inputs and x_out) in a batch of two
    problems; same bits as device buffers."""
    import torch
    outs = []
    for seed in (13, 14):
        xt, psf, ybar, mask = _case_problem(128, 256, lambda: S.psf_motion(9.0, 60.0, 9), 0.7, seed)
        outs.append((psf, ybar, mask))
    plans = [ad.Plan(128, 256, psf, 3e-4, 1.0, 3e-3, "tv", max_iters=11) for psf, _, _ in outs]
    yp = [torch.from_numpy(np.ascontiguousarray(yb.astype(np.float32))).pin_memory() for _, yb, _ in outs]
    mp = [torch.from_numpy(np.ascontiguousarray(m)).pin_memory() for _, _, m in outs]
    xp = [torch.zeros((128, 256), dtype=torch.float32).pin_memory() for _ in outs]
    r1 = ad.solve_batch(plans, yp, mp, xp)
    yd = [t.cuda() for t in yp]
    md = [t.cuda() for t in mp]
    xd = [torch.empty((128, 256), dtype=torch.float32, device="cuda") for _ in outs]
    r2 = ad.solve_batch(plans, yd, md, xd)
    torch.cuda.synchronize()
    for a, b, ra, rb in zip(xp, xd, r1, r2):
        assert ra.iters == rb.iters == 11
        assert torch.equal(a, b.cpu())


def test_mask_null_means_valid_region(ad):
    """mask = NULL observes exactly the valid region (Sec. IV-A)."""
    import torch
    p = S.config1_problem(4)
    plan = ad.Plan(64, 64, p.psf, p.lam, p.mu1, p.mu2, "tv", max_iters=25)
    y = torch.from_numpy(p.ybar.astype(np.float32)).cuda()
    x1 = torch.empty((64, 64), dtype=torch.float32, device="cuda")
    x2 = torch.empty_like(x1)
    ad.solve(plan, y, None, x1)
    ones = torch.ones((64, 64), dtype=torch.uint8, device="cuda")
    ad.solve(plan, y, ones, x2)      # ANDed with the valid region
    torch.cuda.synchronize()
    assert torch.equal(x1, x2)


def test_periodic_unregularised_special_case(ad):
    """M = I (raw mask of ones) and lambda = 0 reduce to periodic
    deconvolution (Sec. IV-A); the iterate reaches x = U*(Y / Lambda)."""
    import torch
    H = W = 64
    g = S.rng(14)
    h = np.zeros((3, 3)); h[1, 1] = 0.8; h[1, 2] = 0.1; h[0, 1] = 0.1
    xt = g.uniform(size=(H, W))
    y = O.A_fft(xt, h)
    mask = np.ones((H, W), dtype=np.uint8)
    x, res, _ = _gpu_solve(ad, y, mask, h, 0.0, 1.0, 0.1, 400, raw_mask=True)
    assert np.max(np.abs(x - xt)) < 2e-4


def test_nonfinite_observation_reports_status(ad):
    """A NaN in the observation makes the iterate non-finite: the problem
    retires with ADMM_ENONFINITE (Theorem 1: no solution -> divergence)."""
    p = S.config1_problem(5)
    y = p.ybar.copy()
    y[30, 30] = np.nan
    x, res, _ = _gpu_solve(ad, y, p.mask, p.psf, p.lam, p.mu1, p.mu2, 50, stop="rel_x", tol=1e-5)
    assert res.status == ad.ADMM_ENONFINITE
    assert res.iters < 50


@pytest.mark.parametrize("cfg", [None, dict(row_variant=3, col_variant=0, slot_ctas=4800)],
                         ids=["default", "tuned"])
def test_full_size_512_config_parity(ad, cfg):
    """The 512 x 512 inpainting workload at full size (both blurs), batched as
    the benchmark launches it, 60 iterations against the oracle; in the
    default configuration and in the one the autotuner picks on GB300 for this
    class (16-row strips, walk depth 2, 256 threads; 4 columns per column CTA;
    4800 row CTAs per launch)."""
    import torch
    if cfg is not None:
        t = ad.admm_deconv_get_tuning(512, 512, "tv")
        t.update(cfg)
        ad.admm_deconv_set_tuning(t)
        got = ad.admm_deconv_get_tuning(512, 512, "tv")
        assert (got["rows_per_strip"], got["walk_depth"], got["row_threads"]) == (16, 2, 256)
    probs = [S.config2_problem(s, blur, 40) for s, blur in ((0, "gauss"), (1, "motion"))]
    try:
        plans = [ad.Plan(512, 512, p.psf, p.lam, p.mu1, p.mu2, "tv", max_iters=60) for p in probs]
    finally:
        ad.admm_deconv_set_tuning({"H": 512, "W": 512, "reg": 0, "haar_levels": 0, "row_variant": 0,
                                   "col_variant": 0, "slot_ctas": 0, "lanes": 0})
    ys = [torch.from_numpy(p.ybar.astype(np.float32)).cuda() for p in probs]
    ms = [torch.from_numpy(p.mask).cuda() for p in probs]
    xs = [torch.empty((512, 512), dtype=torch.float32, device="cuda") for _ in probs]
    ad.solve_batch(plans, ys, ms, xs)
    torch.cuda.synchronize()
    for p, xg in zip(probs, xs):
        ref = O.solve(p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, "tv", iters=60)
        assert _rel(xg.cpu().numpy().astype(np.float64), ref.x) <= TOL_X


def test_max_size_2048(ad):
    """2048 x 2048 (the largest supported side): 4 iterations vs the oracle."""
    xt, psf, ybar, mask = _case_problem(2048, 2048, lambda: S.psf_box(13), None, 15)
    st = O.State.zeros(2048, 2048, "tv")
    for _ in range(4):
        st = O.tvmd_step(st, ybar, mask, psf, 1e-4, 1.0, 1e-3)
    x, res, _ = _gpu_solve(ad, ybar, mask, psf, 1e-4, 1.0, 1e-3, 4)
    assert _rel(x, st.x) <= 2e-5


def test_strip_halo_reads_old_duals(ad):
    """Regression for the cross-strip halo: each row strip recomputes the TV
    dual of the row above it from that row's d2 of the previous iteration.
    2048-wide rows use 4-row strips (many strip boundaries); 40 iterations."""
    xt, psf, ybar, mask = _case_problem(256, 2048, lambda: S.psf_gaussian(9, 2.0), 0.7, 16)
    lam, mu1, mu2 = 3e-4, 1e-2, 3e-3
    st = O.State.zeros(256, 2048, "tv")
    for _ in range(40):
        st = O.tvmd_step(st, ybar, mask, psf, lam, mu1, mu2)
    x, res, _ = _gpu_solve(ad, ybar, mask, psf, lam, mu1, mu2, 40)
    assert _rel(x, st.x) <= 2e-5


def test_empty_batch_is_ok(ad):
    assert ad.lib.admm_deconv_solve_batch(None, 0, None, None, None, None, 0, None) == 0


@pytest.mark.parametrize("reg", ["tv", "tv_aniso"])
def test_primal_residual_matches_oracle(ad, reg):
    """The primal residual H z_k - u_k = d_k - d_{k-1} of Algorithm 2, reduced
    over both splits on the last iteration, against the oracle's duals."""
    p = S.config1_problem(3)
    k = 6
    st = O.State.zeros(64, 64, "tv")
    for _ in range(k):
        prev = st
        st = O.tvmd_step(st, p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, aniso=reg == "tv_aniso")
    ref = math.sqrt(float(np.sum((st.d1 - prev.d1) ** 2) + np.sum((st.d2 - prev.d2) ** 2)))
    x, res, _ = _gpu_solve(ad, p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, k, reg=reg)
    assert ref > 0
    assert abs(res.primal_res - ref) <= 1e-3 * ref, (res.primal_res, ref)
