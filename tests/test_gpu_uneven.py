"""Batched solves of uneven problems: sizes, kernels, masks and regularizers
mixed in one solve_batch call, every size class iterating in the same loop.
Each problem's iterate is a function of that problem alone (Algorithm 2 run
per problem), so a batch must give the bits of solving each problem alone;
padded domains (a side that is not a power of two, solved on the next power
of two with the padding unobserved, Sec. IV-A) are checked against the FP64
oracle on the same padded problem."""
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


def _plan(ad, p, stop="rel_x", tol=1e-5, max_iters=5000):
    H, W = p.ybar.shape
    return ad.Plan(H, W, p.psf, p.lam, p.mu1, p.mu2, p.reg, stop=stop, tol=tol, max_iters=max_iters,
                   check_every=1)


def _dev(p):
    import torch
    return (torch.from_numpy(p.ybar.astype(np.float32)).cuda(), torch.from_numpy(p.mask).cuda(),
            torch.full(p.ybar.shape, float("nan"), dtype=torch.float32, device="cuda"))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_uneven_batch_gives_the_bits_of_solo_solves(ad):
    import torch
    probs = S.config4_batch(5, 10, sizes=(128, 256, 384))
    assert len({(p.ybar.shape, p.reg) for p in probs}) >= 3
    plans = [_plan(ad, p) for p in probs]
    dev = [_dev(p) for p in probs]
    res = ad.solve_batch(plans, [d[0] for d in dev], [d[1] for d in dev], [d[2] for d in dev])
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        y, m, _ = dev[i]
        xo = torch.empty_like(dev[i][2])
        r = ad.solve(plans[i], y, m, xo)
        torch.cuda.synchronize()
        assert r.converged == res[i].converged, (i, p.meta)
        assert r.iters == res[i].iters
        assert torch.equal(xo, dev[i][2]), (i, p.meta)
        assert 0.0 <= res[i].t_start_ms < res[i].t_done_ms


def test_uneven_batch_with_one_slot_per_class_queues_problems(ad):
    """With one launch slot per size class, problems of a class run one after
    the other (each starts when the previous one retires) and the results do
    not change."""
    import torch
    probs = S.config4_batch(6, 9, sizes=(128, 256))
    plans = [_plan(ad, p, max_iters=1500) for p in probs]
    dev = [_dev(p) for p in probs]
    ref = ad.solve_batch(plans, [d[0] for d in dev], [d[1] for d in dev], [d[2] for d in dev])
    torch.cuda.synchronize()
    x_ref = [d[2].clone() for d in dev]
    ad.admm_deconv_set_option(ad.ADMM_OPT_MAX_SLOTS, 1)
    try:
        for d in dev:
            d[2].fill_(float("nan"))
        res = ad.solve_batch(plans, [d[0] for d in dev], [d[1] for d in dev], [d[2] for d in dev])
        torch.cuda.synchronize()
    finally:
        ad.admm_deconv_set_option(ad.ADMM_OPT_MAX_SLOTS, 0)
    classes = {}
    for i, p in enumerate(probs):
        assert res[i].iters == ref[i].iters
        assert torch.equal(dev[i][2], x_ref[i])
        classes.setdefault((p.ybar.shape, p.reg), []).append(i)
    for idx in classes.values():
        spans = sorted((res[i].t_start_ms, res[i].t_done_ms) for i in idx)
        for (s0, d0), (s1, d1) in zip(spans, spans[1:]):
            assert d0 <= s1 + 1e-3 and s1 < d1          # one problem at a time per class


@pytest.mark.parametrize("reg", ["tv", "haar"])
def test_padded_domain_matches_oracle(ad, reg):
    """A 384 x 384 image solved on the 512 x 512 domain (padding unobserved)
    against the oracle on the same padded problem; ISNR over the image's
    valid region."""
    import torch
    p = S.config4_problem(S.rng(21), size=384, reg=reg)
    assert p.ybar.shape == (512, 512) and p.meta["window"] == 384
    assert not p.mask[384:, :].any() and not p.mask[:, 384:].any()
    iters = 25
    ref = O.solve(p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, reg, iters=iters)
    plan = _plan(ad, p, stop="iters", tol=0.0, max_iters=iters)
    y, m, x = _dev(p)
    r = ad.solve(plan, y, m, x)
    torch.cuda.synchronize()
    assert r.iters == iters
    xg = x.cpu().numpy().astype(np.float64)
    assert _rel(xg, ref.x) <= 2e-5
    vm = np.zeros((512, 512), dtype=np.uint8)
    vm[:384, :384] = S.valid_mask(384, 384, *p.psf.shape)
    assert abs(O.isnr(p.x_true, p.ybar, xg, vm) - O.isnr(p.x_true, p.ybar, ref.x, vm)) <= 0.01
