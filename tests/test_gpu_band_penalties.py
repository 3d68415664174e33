"""GPU parity of the frame prior with one penalty per band (Sec. II, eq.
diagonal_penalty: Algorithm 2 with a positive diagonal Upsilon that gives each
of the 3 L + 1 band functions its own mu_b) against the FP64 oracle
(famd_step(mu_bands=...)): the x-step denominator sum_b gamma_b |H_b|^2 built on
the device, the per-band thresholds lambda / mu_b and the weighted synthesis."""
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _band_mu(levels, mu2, seed):
    g = S.rng(seed)
    return (mu2 * np.exp(g.uniform(-1.5, 1.5, size=3 * levels + 1))).astype(np.float32)


@pytest.mark.parametrize("reg,H,W,levels,keep", [
    ("haar", 128, 128, 4, 0.7),
    ("haar", 256, 64, 2, None),
    ("haar_ll_free", 128, 256, 3, 0.8),
    ("haar", 384, 320, 4, 0.8),          # exact mixed-radix domain
])
def test_band_penalties_match_oracle(ad, reg, H, W, levels, keep):
    import torch
    g = S.rng(71)
    x = S.textured_image(H, W, g)
    psf = S.psf_gaussian(7, 1.5)
    km = None if keep is None else (g.uniform(size=(H, W)) < keep).astype(np.uint8)
    ybar, mask, _ = S.observe(x, psf, km, 40.0, g)
    lam = 1e-3
    mu1, mu2 = S.default_mu(lam)
    mub = _band_mu(levels, mu2, 72)
    st = O.State.zeros(H, W, "haar", levels)
    y = torch.from_numpy(ybar.astype(np.float32)).cuda()
    m = torch.from_numpy(mask).cuda()
    for k in range(1, 13):
        st = O.famd_step(st, ybar, mask, psf, lam, mu1, mu2, levels, ll_free=reg == "haar_ll_free",
                         mu_bands=mub.astype(np.float64))
        if k in (2, 12):
            plan = ad.Plan(H, W, psf, lam, mu1, mu2, reg, levels=levels, max_iters=k, band_mu=mub)
            xg = torch.empty((H, W), dtype=torch.float32, device="cuda")
            ad.solve(plan, y, m, xg)
            assert _rel(xg.cpu().numpy().astype(np.float64), st.x) <= TOL_SHORT, k
    d = torch.empty(plan.state_size(), dtype=torch.float32, device="cuda")
    ad.admm_deconv_get_state(plan.handle, d.data_ptr())
    d2 = d.cpu().numpy().astype(np.float64)[H * W:].reshape(-1, H, W)
    for b in range(3 * levels + 1):
        assert np.max(np.abs(d2[b] - st.d2[b])) <= 2e-4 * (lam / mub[b]) + 1e-7, b
    plan.close()


def test_uniform_band_penalties_give_the_scalar_bits(ad):
    """band_mu = mu2 for every band runs the same arithmetic as band_mu = NULL."""
    import torch
    H = W = 128
    g = S.rng(73)
    x = S.textured_image(H, W, g)
    psf = S.psf_box(9)
    ybar, mask, _ = S.observe(x, psf, None, 40.0, g)
    lam = 1e-3
    mu1, mu2 = S.default_mu(lam)
    y = torch.from_numpy(ybar.astype(np.float32)).cuda()
    m = torch.from_numpy(mask).cuda()
    out = []
    for bm in (None, np.full(13, np.float32(mu2))):
        plan = ad.Plan(H, W, psf, lam, mu1, mu2, "haar", max_iters=30, band_mu=bm)
        xg = torch.empty((H, W), dtype=torch.float32, device="cuda")
        ad.solve(plan, y, m, xg)
        out.append(xg.cpu().numpy())
        plan.close()
    assert _rel(out[1].astype(np.float64), out[0].astype(np.float64)) <= 1e-6
