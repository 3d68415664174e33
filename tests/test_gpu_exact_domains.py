"""GPU parity on exact domains whose sides are not powers of two (Sec. IV-A:
the unknown domain only has to hold the image and the kernel support, so its
size is free). Sides m 2^k with m = 3 or 5 run the mixed-radix kernels on the
exact domain -- no padding -- and are compared with the FP64 oracle on the
same domain: TV (isotropic and anisotropic) and the frame priors, iterates,
duals, the relative-change stop, batches mixing exact and power-of-two
domains, restart from a saved state and a learned warm start."""
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
    assert plan.domain() == (H, W)           # exact: no padding
    y = torch.from_numpy(ybar.astype(np.float32)).cuda()
    m = torch.from_numpy(mask).cuda()
    x = torch.empty((H, W), dtype=torch.float32, device="cuda")
    res = ad.solve(plan, y, m, x)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.float64), res, plan


STEP = {"tv": O.tvmd_step, "tv_aniso": lambda *a: O.tvmd_step(*a, aniso=True), "haar": O.famd_step}

CASES = [
    # reg, H, W, psf factory, keep, seed
    ("tv", 384, 384, lambda: S.psf_gaussian(9, 2.0), 0.6, 1),
    ("tv", 384, 512, lambda: S.psf_motion(11.0, 30.0, 11), None, 2),
    ("tv", 320, 640, lambda: S.psf_box(7), 0.8, 3),
    ("tv", 768, 192, lambda: S.psf_box(13), None, 4),
    ("tv", 96, 1536, lambda: S.psf_gaussian(5, 1.0), 0.7, 5),
    ("tv_aniso", 192, 160, lambda: S.psf_box(5), 0.8, 6),
    ("haar", 384, 384, lambda: S.psf_box(9), None, 7),
    ("haar", 320, 256, lambda: S.psf_gaussian(7, 1.5), 0.7, 8),
]


@pytest.mark.parametrize("reg,H,W,psf_fn,keep,seed", CASES)
def test_iterates_and_duals_match_oracle(ad, reg, H, W, psf_fn, keep, seed):
    """x after 2, 3 and 10 iterations and the duals after 10 on exact
    domains with sides 3 2^k and 5 2^k (and mixed with powers of two)."""
    import torch
    _, psf, ybar, mask = _problem(H, W, psf_fn, keep, seed)
    lam = 3e-4
    mu1, mu2 = S.default_mu(lam)
    st = O.State.zeros(H, W, "haar" if reg == "haar" else "tv")
    for k in range(1, 11):
        st = STEP[reg](st, ybar, mask, psf, lam, mu1, mu2)
        if k in (2, 3, 10):
            x, res, plan = _gpu(ad, reg, ybar, mask, psf, lam, mu1, mu2, k)
            assert res.iters == k
            assert _rel(x, st.x) <= TOL_SHORT, (k, _rel(x, st.x))
    n = H * W
    d = torch.empty(plan.state_size(), dtype=torch.float32, device="cuda")
    ad.admm_deconv_get_state(plan.handle, d.data_ptr())
    d = d.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(d[:n].reshape(H, W) - st.d1)) <= 2e-5 * np.abs(st.d1).max() + 1e-9
    if reg == "haar":
        assert np.max(np.abs(d[n:].reshape(-1, H, W) - st.d2)) <= 2e-4 * (lam / mu2)
    else:
        d2 = d[n:].reshape(H, W, 2)
        for comp in (0, 1):
            assert np.max(np.abs(d2[..., comp] - st.d2[comp])) <= 2e-4 * (lam / mu2)
    plan.close()


@pytest.mark.parametrize("reg", ["tv", "haar"])
def test_rel_x_stop_and_isnr_match_oracle(ad, reg):
    """384 x 384 (the batched workload's side that is not a power of two) to
    rel-x < 1e-5 on the exact domain: stopping iteration, x and ISNR."""
    xt, psf, ybar, mask = _problem(384, 384, lambda: S.psf_gaussian(11, 2.0), 0.7, 11)
    lam = 3e-4 if reg == "tv" else 1e-3
    mu1, mu2 = S.default_mu(lam)
    ref = O.solve(ybar, mask, psf, lam, mu1, mu2, reg, iters=3000, stop="rel_x", tol=1e-5)
    x, res, plan = _gpu(ad, reg, ybar, mask, psf, lam, mu1, mu2, 3000, stop="rel_x", tol=1e-5)
    assert ref.converged and res.converged == 1
    assert abs(res.iters - ref.iters) <= max(3, ref.iters // 100)
    assert _rel(x, ref.x) <= TOL_X
    vm = S.valid_mask(384, 384, *psf.shape)
    assert abs(O.isnr(xt, ybar, x, vm) - O.isnr(xt, ybar, ref.x, vm)) <= 0.01
    plan.close()


def test_frame_variants_on_an_exact_domain(ad):
    """The unpenalised low-low band and the synthesis formulation run on the
    exact-domain kernels too."""
    _, psf, ybar, mask = _problem(192, 384, lambda: S.psf_box(5), None, 12)
    lam = 1e-3
    mu1, mu2 = S.default_mu(lam)
    for reg, step in (("haar_ll_free", lambda *a: O.famd_step(*a, ll_free=True)), ("haar_synthesis", O.fsmd_step)):
        st = O.State.zeros(192, 384, "haar")
        for _ in range(6):
            st = step(st, ybar, mask, psf, lam, mu1, mu2)
        x, res, plan = _gpu(ad, reg, ybar, mask, psf, lam, mu1, mu2, 6)
        assert _rel(x, st.x) <= TOL_SHORT, reg
        plan.close()


def test_batch_mixing_exact_and_power_of_two_domains_gives_solo_bits(ad):
    import torch
    specs = [("tv", 384), ("tv", 512), ("haar", 384), ("tv", 320), ("haar", 256), ("tv", 384)]
    lam = 1e-3
    mu1, mu2 = S.default_mu(lam)
    plans, ys, ms, xs, solo = [], [], [], [], []
    for i, (reg, n) in enumerate(specs):
        _, psf, ybar, mask = _problem(n, n, lambda: S.psf_box(7), 0.8, 40 + i)
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


@pytest.mark.parametrize("reg", ["tv", "haar"])
def test_restart_on_an_exact_domain_is_bit_identical(ad, reg):
    import torch
    H, W = 384, 320
    _, psf, ybar, mask = _problem(H, W, lambda: S.psf_gaussian(7, 1.5), 0.7, 13)
    lam = 1e-3
    mu1, mu2 = S.default_mu(lam)
    y = torch.from_numpy(ybar.astype(np.float32)).cuda()
    m = torch.from_numpy(mask).cuda()
    full = ad.Plan(H, W, psf, lam, mu1, mu2, reg, max_iters=40)
    x40 = torch.empty((H, W), dtype=torch.float32, device="cuda")
    ad.solve(full, y, m, x40)
    a = ad.Plan(H, W, psf, lam, mu1, mu2, reg, max_iters=20)
    xa = torch.empty_like(x40)
    ad.solve(a, y, m, xa)
    st = torch.empty(a.full_state_size(), dtype=torch.float32, device="cuda")
    a.get_full_state(st)
    b = ad.Plan(H, W, psf, lam, mu1, mu2, reg, max_iters=20)
    b.set_state(st)
    xb = torch.empty_like(x40)
    ad.solve(b, y, m, xb)
    torch.cuda.synchronize()
    assert torch.equal(xb, x40)
    for p in (full, a, b):
        p.close()


def test_warm_start_on_an_exact_domain_matches_oracle(ad):
    """admm_deconv_warm_start (u0 = H x0 - d0) on a 384 x 384 exact domain
    against the oracle's literal warm start (the first x-step from that u0)."""
    import torch
    import oracle.cnn as C
    H = W = 384
    _, psf, ybar, mask = _problem(H, W, lambda: S.psf_box(9), None, 14)
    lam = 1e-3
    mu1, mu2 = S.default_mu(lam)
    g = S.rng(15)
    x0 = np.where(mask != 0, ybar, ybar[mask != 0].mean()) + 0.02 * g.standard_normal((H, W))
    d1 = 0.05 * g.standard_normal((H, W))
    d2 = 0.05 * g.standard_normal((2, H, W))
    st = C.warm_state(x0, d1, d2, psf, "tv")
    for _ in range(8):
        st = O.tvmd_step(st, ybar, mask, psf, lam, mu1, mu2)
    plan = ad.Plan(H, W, psf, lam, mu1, mu2, "tv", max_iters=8)
    flat = np.concatenate([d1.ravel(), np.stack([d2[0], d2[1]], axis=-1).ravel()]).astype(np.float32)
    plan.warm_start(x0.astype(np.float32), flat)
    x = torch.empty((H, W), dtype=torch.float32, device="cuda")
    ad.solve(plan, torch.from_numpy(ybar.astype(np.float32)).cuda(), torch.from_numpy(mask).cuda(), x)
    assert _rel(x.cpu().numpy().astype(np.float64), st.x) <= TOL_SHORT
    plan.close()


def test_sizes_and_padding_policy(ad):
    """Exact sides need m 2^k (m = 1, 3, 5) and a multiple of 32; with
    ADMM_PAD_NEXT other sides go to the next such size (300 -> 320), and the
    Reeves-Sorel variants, which have no mixed-radix form, to the next power
    of two."""
    psf = S.psf_box(5)
    with pytest.raises(ad.AdmmError) as e:
        ad.Plan(300, 300, psf, 1e-3, max_iters=2)
    assert e.value.code == ad.ADMM_EUNSUPPORTED_SIZE
    p = ad.Plan(300, 200, psf, 1e-3, max_iters=2, pad=True)
    assert p.domain() == (320, 256)
    p.close()
    p = ad.Plan(384, 384, psf, 1e-3, max_iters=2)
    assert p.domain() == (384, 384)
    p.close()
    p = ad.Plan(384, 384, psf, 1e-3, reg="tv_cg", max_iters=2, pad=True)
    assert p.domain() == (512, 512)
    p.close()
    with pytest.raises(ad.AdmmError):
        ad.Plan(384, 384, psf, 1e-3, reg="tv_cg", max_iters=2)
