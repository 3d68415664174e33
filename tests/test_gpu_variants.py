"""GPU parity of the regulariser variants against the FP64 oracle, through
the C ABI: anisotropic TV (eq. soft per difference component in place of
vector-soft), the frame prior with the low-low band unpenalised (its prox is
the identity), and FS-MD, the frame synthesis formulation (x = W theta, the
duals on theta). Tolerances as for the other short runs (2e-5 relative L2 on
x after a few iterations, 1e-4 after 200)."""
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


def _problem(H, W, seed, psf, keep=0.7):
    g = S.rng(seed)
    x = S.textured_image(H, W, g)
    keepm = (g.uniform(size=(H, W)) < keep).astype(np.uint8)
    ybar, mask, _ = S.observe(x, psf, keepm, 40.0, g)
    return x, ybar, mask


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _gpu(ad, reg, ybar, mask, psf, lam, mu1, mu2, iters, levels=4):
    import torch
    H, W = ybar.shape
    plan = ad.Plan(H, W, psf, lam, mu1, mu2, reg, levels=levels, max_iters=iters)
    y = torch.from_numpy(ybar.astype(np.float32)).cuda()
    m = torch.from_numpy(mask).cuda()
    x = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
    res = ad.solve(plan, y, m, x)
    n = plan.state_size()
    d = torch.empty(n, dtype=torch.float32, device="cuda")
    ad.admm_deconv_get_state(plan.handle, d.data_ptr())
    torch.cuda.synchronize()
    plan.close()
    return x.cpu().numpy().astype(np.float64), d.cpu().numpy().astype(np.float64), res


@pytest.mark.parametrize("H,W", [(64, 64), (256, 128), (512, 512), (128, 1024)])
def test_aniso_tv_iterates_and_duals(ad, H, W):
    psf = S.psf_motion(9.0, 30.0, 9)
    _, ybar, mask = _problem(H, W, 200 + H + W, psf)
    lam, mu1, mu2, iters = 3e-4, 1e-2, 3e-3, 6
    st = O.State.zeros(H, W, "tv_aniso")
    for _ in range(iters):
        st = O.tvmd_step(st, ybar, mask, psf, lam, mu1, mu2, aniso=True)
    x, d, res = _gpu(ad, "tv_aniso", ybar, mask, psf, lam, mu1, mu2, iters)
    assert res.iters == iters and res.status == 0
    assert _rel(x, st.x) <= 2e-5
    n = H * W
    d2 = d[n:].reshape(H, W, 2)
    for comp in (0, 1):
        assert np.max(np.abs(d2[..., comp] - st.d2[comp])) <= 2e-4 * (lam / mu2)
    # the anisotropic prox differs from vector-soft on these inputs
    sti = O.State.zeros(H, W, "tv")
    for _ in range(iters):
        sti = O.tvmd_step(sti, ybar, mask, psf, lam, mu1, mu2)
    assert _rel(st.x, sti.x) > 1e-3


def test_aniso_tv_200_iterations_and_objective(ad):
    p = S.config1_problem(0)
    ref = O.solve(p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, "tv_aniso", iters=200)
    x, _, res = _gpu(ad, "tv_aniso", p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, 200)
    assert _rel(x, ref.x) <= 1e-4
    assert abs(res.objective - ref.objective) <= 1e-5 * ref.objective


@pytest.mark.parametrize("H,W,levels", [(128, 128, 4), (256, 512, 4), (1024, 256, 3)])
def test_ll_free_frame_iterates_and_duals(ad, H, W, levels):
    psf = S.psf_box(7)
    _, ybar, mask = _problem(H, W, 300 + H + W, psf, keep=0.8)
    lam, mu1, mu2, iters = 1e-4, 1e-2, 1e-3, 5
    st = O.State.zeros(H, W, "haar", levels)
    for _ in range(iters):
        st = O.famd_step(st, ybar, mask, psf, lam, mu1, mu2, levels=levels, ll_free=True)
    x, d, res = _gpu(ad, "haar_ll_free", ybar, mask, psf, lam, mu1, mu2, iters, levels=levels)
    assert res.iters == iters and res.status == 0
    assert _rel(x, st.x) <= 2e-5
    n = H * W
    nb = 3 * levels + 1
    d2 = d[n:].reshape(nb, H, W)
    assert np.max(np.abs(d2[-1])) <= 1e-6 * (lam / mu2)        # the low-low dual stays zero
    assert np.max(np.abs(d2[:-1] - st.d2[:-1])) <= 2e-4 * (lam / mu2)


def test_variants_and_paper_priors_in_one_batch(ad):
    """One solve_batch over all five regularisers of one size (five size
    classes), each matching its own oracle run."""
    import torch
    H = W = 128
    psf = S.psf_gaussian(9, 2.0)
    regs = ["tv", "tv_aniso", "haar", "haar_ll_free", "haar_synthesis"]
    probs = [_problem(H, W, 400 + i, psf) for i in range(len(regs))]
    lam, mu1, mu2, iters = 3e-4, 1e-2, 3e-3, 9
    plans = [ad.Plan(H, W, psf, lam, mu1, mu2, r, max_iters=iters) for r in regs]
    ys = [torch.from_numpy(p[1].astype(np.float32)).cuda() for p in probs]
    ms = [torch.from_numpy(p[2]).cuda() for p in probs]
    xs = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in probs]
    res = ad.solve_batch(plans, ys, ms, xs)
    torch.cuda.synchronize()
    for r, (_, ybar, mask), xg, rs in zip(regs, probs, xs, res):
        ref = O.solve(ybar, mask, psf, lam, mu1, mu2, r, iters=iters)
        assert rs.iters == iters
        assert _rel(xg.cpu().numpy().astype(np.float64), ref.x) <= 2e-5, r
    for p in plans:
        p.close()


def test_replayed_graphs_follow_the_regulariser(ad):
    """Isotropic and anisotropic TV classes of one shape and configuration have
    the same batch layout; the replayed iteration graphs (chunks of eight
    iterations, cached by layout) must still run each class's own kernel."""
    psf = S.psf_box(5)
    _, ybar, mask = _problem(64, 64, 500, psf)
    lam, mu1, mu2, iters = 3e-4, 1e-2, 3e-3, 40
    for reg in ("tv", "tv_aniso", "tv"):
        ref = O.solve(ybar, mask, psf, lam, mu1, mu2, reg, iters=iters)
        x, _, res = _gpu(ad, reg, ybar, mask, psf, lam, mu1, mu2, iters)
        assert res.iters == iters
        assert _rel(x, ref.x) <= 1e-4, reg


@pytest.mark.parametrize("H,W,levels", [(128, 128, 4), (256, 512, 4), (1024, 256, 3), (64, 64, 1)])
def test_fs_iterates_and_duals(ad, H, W, levels):
    psf = S.psf_gaussian(9, 2.0)
    _, ybar, mask = _problem(H, W, 600 + H + W + levels, psf, keep=0.8)
    lam, mu1, mu2, iters = 1e-4, 1e-2, 1e-3, 6
    st = O.State.zeros(H, W, "haar", levels)
    for _ in range(iters):
        st = O.fsmd_step(st, ybar, mask, psf, lam, mu1, mu2, levels=levels)
    x, d, res = _gpu(ad, "haar_synthesis", ybar, mask, psf, lam, mu1, mu2, iters, levels=levels)
    assert res.iters == iters and res.status == 0
    assert _rel(x, st.x) <= 2e-5
    n = H * W
    d1 = d[:n].reshape(H, W)
    d2 = d[n:].reshape(3 * levels + 1, H, W)
    assert np.max(np.abs(d1 - st.d1)) <= 2e-5 * np.abs(st.d1).max() + 1e-9
    assert np.max(np.abs(d2 - st.d2)) <= 2e-4 * (lam / mu2)
    # the synthesis problem's iterates differ from the analysis problem's
    sta = O.State.zeros(H, W, "haar", levels)
    for _ in range(iters):
        sta = O.famd_step(sta, ybar, mask, psf, lam, mu1, mu2, levels=levels)
    assert _rel(st.x, sta.x) > 1e-4


def test_fs_200_iterations_and_objective(ad):
    psf = S.psf_box(7)
    x_true, ybar, mask = _problem(128, 128, 700, psf, keep=0.8)
    lam, mu1, mu2 = 1e-3, 3e-2, 1e-2
    ref = O.solve(ybar, mask, psf, lam, mu1, mu2, "haar_synthesis", iters=200)
    x, _, res = _gpu(ad, "haar_synthesis", ybar, mask, psf, lam, mu1, mu2, 200)
    assert _rel(x, ref.x) <= 1e-4
    assert abs(res.objective - ref.objective) <= 1e-5 * ref.objective
    vm = S.valid_mask(128, 128, *psf.shape)
    assert abs(O.isnr(x_true, ybar, x, vm) - O.isnr(x_true, ybar, ref.x, vm)) <= 0.01


def test_fs_rejects_a_warm_start(ad):
    psf = S.psf_box(5)
    plan = ad.Plan(64, 64, psf, 1e-3, 0.0, 0.0, "haar_synthesis", max_iters=5)
    with pytest.raises(ad.AdmmError) as e:
        plan.warm_start()
    assert e.value.code == ad.ADMM_EINVAL
    plan.close()
