"""Launch configurations and the autotuner, through the C ABI.

Every compiled configuration of the TV row phase (rows per strip, walk rows
in flight, threads per CTA) and of the column phase (columns per CTA) must
compute the same iteration: each is checked against the FP64 oracle after a
few iterations (tolerance 2e-5, as for the other short runs). The autotuner
must install the fastest trial, and plans of one size class made under two
configurations must still batch together correctly."""
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


def _problem(H, W, seed, keep=0.7):
    g = S.rng(seed)
    x = S.textured_image(H, W, g)
    psf = S.psf_gaussian(9, 2.0)
    keepm = (g.uniform(size=(H, W)) < keep).astype(np.uint8)
    ybar, mask, _ = S.observe(x, psf, keepm, 40.0, g)
    return psf, ybar, mask


def _set(ad, H, W, reg, rv, cv, st=0, levels=0, lanes=0):
    ad.admm_deconv_set_tuning({"H": H, "W": W, "reg": reg, "haar_levels": levels, "row_variant": rv,
                               "col_variant": cv, "slot_ctas": st, "lanes": lanes})


def _reset(ad, H, W, reg, levels=0):
    _set(ad, H, W, reg, 0, 0, 0, levels)


def _solve(ad, psf, ybar, mask, lam, mu1, mu2, iters, reg="tv"):
    import torch
    H, W = ybar.shape
    plan = ad.Plan(H, W, psf, lam, mu1, mu2, reg, max_iters=iters)
    y = torch.from_numpy(ybar.astype(np.float32)).cuda()
    m = torch.from_numpy(mask).cuda()
    x = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
    res = ad.solve(plan, y, m, x)
    torch.cuda.synchronize()
    plan.close()
    return x.cpu().numpy().astype(np.float64), res


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


SIZES = [(64, 64), (128, 128), (256, 256), (512, 512), (1024, 1024), (2048, 128), (128, 2048)]


@pytest.mark.parametrize("H,W", SIZES)
def test_every_tv_configuration_matches_oracle(ad, H, W):
    psf, ybar, mask = _problem(H, W, 40 + H // 64 + W)
    lam, mu1, mu2 = 3e-4, 1e-2, 3e-3
    iters = 5
    st = O.State.zeros(H, W, "tv")
    for _ in range(iters):
        st = O.tvmd_step(st, ybar, mask, psf, lam, mu1, mu2)
    nr, nc = ad.admm_deconv_variants(H, W, "tv")
    assert nr >= 2 and nc >= 2
    try:
        for rv in range(nr):
            for cv in range(nc):
                _set(ad, H, W, ad.ADMM_REG_TV, rv, cv)
                cfg = ad.admm_deconv_get_tuning(H, W, "tv")
                assert (cfg["row_variant"], cfg["col_variant"]) == (rv, cv)
                x, res = _solve(ad, psf, ybar, mask, lam, mu1, mu2, iters)
                assert res.iters == iters and res.status == 0
                assert _rel(x, st.x) <= 2e-5, (cfg, _rel(x, st.x))
    finally:
        _reset(ad, H, W, ad.ADMM_REG_TV)


@pytest.mark.parametrize("H,W", [(256, 256), (1024, 512), (2048, 256)])
def test_every_frame_column_configuration_matches_oracle(ad, H, W):
    psf, ybar, mask = _problem(H, W, 70 + H // 64 + W)
    lam, mu1, mu2 = 1e-4, 1e-2, 1e-3
    iters = 4
    st = O.State.zeros(H, W, "haar", levels=4)
    for _ in range(iters):
        st = O.famd_step(st, ybar, mask, psf, lam, mu1, mu2, levels=4)
    nr, nc = ad.admm_deconv_variants(H, W, "haar")
    assert nr == 1 and nc >= 2
    try:
        for cv in range(nc):
            _set(ad, H, W, ad.ADMM_REG_HAAR, 0, cv, levels=4)
            x, res = _solve(ad, psf, ybar, mask, lam, mu1, mu2, iters, reg="haar")
            assert res.iters == iters and res.status == 0
            assert _rel(x, st.x) <= 2e-5, (cv, _rel(x, st.x))
    finally:
        _reset(ad, H, W, ad.ADMM_REG_HAAR, 4)


def test_autotune_installs_the_fastest_trial(ad):
    import torch
    H = W = 128
    try:
        best, trials = ad.admm_deconv_autotune(H, W, "tv", problems=6, iters=16)
        nr, nc = ad.admm_deconv_variants(H, W, "tv")
        assert len(trials) == nr * nc * 3 + 2
        assert all(t["us_per_iter"] > 0 for t in trials)
        assert best["us_per_iter"] == min(t["us_per_iter"] for t in trials)
        cfg = ad.admm_deconv_get_tuning(H, W, "tv")
        for k in ("row_variant", "col_variant", "slot_ctas", "lanes", "rows_per_strip", "col_block", "col_min_ctas"):
            assert cfg[k] == best[k], k
        # a plan made now runs the tuned configuration and still matches the oracle
        psf, ybar, mask = _problem(H, W, 99)
        st = O.State.zeros(H, W, "tv")
        for _ in range(6):
            st = O.tvmd_step(st, ybar, mask, psf, 3e-4, 1e-2, 3e-3)
        x, res = _solve(ad, psf, ybar, mask, 3e-4, 1e-2, 3e-3, 6)
        assert _rel(x, st.x) <= 2e-5
    finally:
        _reset(ad, H, W, ad.ADMM_REG_TV)
    torch.cuda.synchronize()


def test_one_class_under_two_configurations_in_one_batch(ad):
    """Plans keep the configuration they were made with; a batch groups them
    by configuration as well as by shape."""
    import torch
    H = W = 256
    probs = [_problem(H, W, 120 + i) for i in range(4)]
    lam, mu1, mu2, iters = 3e-4, 1e-2, 3e-3, 7
    try:
        plans = []
        for i, (psf, _, _) in enumerate(probs):
            _set(ad, H, W, ad.ADMM_REG_TV, i % 2, i % 2)
            plans.append(ad.Plan(H, W, psf, lam, mu1, mu2, "tv", max_iters=iters))
    finally:
        _reset(ad, H, W, ad.ADMM_REG_TV)
    ys = [torch.from_numpy(p[1].astype(np.float32)).cuda() for p in probs]
    ms = [torch.from_numpy(p[2]).cuda() for p in probs]
    xs = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in probs]
    res = ad.solve_batch(plans, ys, ms, xs)
    torch.cuda.synchronize()
    for (psf, ybar, mask), xg, r in zip(probs, xs, res):
        st = O.State.zeros(H, W, "tv")
        for _ in range(iters):
            st = O.tvmd_step(st, ybar, mask, psf, lam, mu1, mu2)
        assert r.iters == iters
        assert _rel(xg.cpu().numpy().astype(np.float64), st.x) <= 2e-5
    for p in plans:
        p.close()


@pytest.mark.parametrize("lanes", [1, 3, 4])
def test_lane_counts_give_the_same_iterates(ad, lanes):
    """A class split into 1, 3 or 4 independent lanes (graph branches, each
    with its own slots and queue) computes every problem's iterates."""
    import torch
    H = W = 128
    probs = [_problem(H, W, 150 + i) for i in range(7)]
    lam, mu1, mu2, iters = 3e-4, 1e-2, 3e-3, 20     # > one chunk of 8: graph replays
    try:
        _set(ad, H, W, ad.ADMM_REG_TV, 0, 0, 0, lanes=lanes)
        assert ad.admm_deconv_get_tuning(H, W, "tv")["lanes"] == lanes
        plans = [ad.Plan(H, W, psf, lam, mu1, mu2, "tv", max_iters=iters) for psf, _, _ in probs]
    finally:
        _reset(ad, H, W, ad.ADMM_REG_TV)
    ys = [torch.from_numpy(p[1].astype(np.float32)).cuda() for p in probs]
    ms = [torch.from_numpy(p[2]).cuda() for p in probs]
    xs = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in probs]
    res = ad.solve_batch(plans, ys, ms, xs)
    torch.cuda.synchronize()
    for (psf, ybar, mask), xg, r in zip(probs, xs, res):
        st = O.State.zeros(H, W, "tv")
        for _ in range(iters):
            st = O.tvmd_step(st, ybar, mask, psf, lam, mu1, mu2)
        assert r.iters == iters
        assert _rel(xg.cpu().numpy().astype(np.float64), st.x) <= 2e-5
    for p in plans:
        p.close()
