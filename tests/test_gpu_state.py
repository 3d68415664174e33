"""GPU tests of the boundary's state, padding, learned-start and failure paths:

* exact checkpoint / restart (admm_deconv_get_full_state, admm_deconv_set_state):
  Algorithm 2 carries (u_k, d_k) from one iteration to the next, so a solve
  stopped after k iterations and restarted from its complete state must
  produce the bits of one uninterrupted solve;
* fft_pad_policy = ADMM_PAD_NEXT: an image whose sides are not supported
  transform sizes is solved on the next supported domain with the added rows
  and columns unobserved (more unknown boundary, Sec. IV-A); the oracle
  solves the same padded problem;
* admm_deconv_solve_batch(..., use_warmstart=1): the network loaded by
  admm_warmstart_load gives the start that admm_cnn_predict_start and
  admm_deconv_warm_start give by hand, bit for bit;
* ADMM_OPT_FAIL_ALLOC: every allocation a plan, a batch or a network makes
  can fail, the call returns ADMM_ENOMEM, frees what it took, and the next
  call works;
* ADMM_OPT_TEST_STALL: a bulk copy the TV row phase waits for is withheld,
  the bounded wait runs out, the problem retires with ADMM_ETIMEOUT, and the
  device stays usable (no fault, no hang).
"""
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _problem(H, W, psf, keep, seed, bsnr=40.0):
    g = S.rng(seed)
    x = S.textured_image(H, W, g)
    km = None if keep is None else (g.uniform(size=(H, W)) < keep).astype(np.uint8)
    ybar, mask, _ = S.observe(x, psf, km, bsnr, g)
    return x, ybar.astype(np.float32), mask


@pytest.mark.parametrize("reg,H,W,psf_fn,keep,lam", [
    ("tv", 128, 128, lambda: S.psf_gaussian(9, 2.0), 0.7, 1e-3),
    ("tv_aniso", 64, 256, lambda: S.psf_box(5), None, 3e-4),
    ("haar", 128, 64, lambda: S.psf_motion(9.0, 30.0, 9), 0.8, 1e-3),
    ("haar_ll_free", 64, 64, lambda: S.psf_box(7), None, 1e-3),
    ("haar_synthesis", 64, 128, lambda: S.psf_gaussian(5, 1.0), None, 1e-3),
    ("tv_cg", 128, 64, lambda: S.psf_gaussian(7, 1.5), 0.7, 1e-3),
    ("haar_cg", 64, 128, lambda: S.psf_box(9), 0.8, 1e-3),
])
def test_restart_from_full_state_is_bit_identical(ad, reg, H, W, psf_fn, keep, lam):
    """30 iterations, then get_full_state -> set_state on a second plan -> 30
    more, against 60 uninterrupted iterations: x and the duals bit-identical."""
    import torch
    psf = psf_fn()
    _, ybar, mask = _problem(H, W, psf, keep, 51)
    mu1, mu2 = S.default_mu(lam)
    y = torch.from_numpy(ybar).cuda()
    m = torch.from_numpy(mask).cuda()
    full = ad.Plan(H, W, psf, lam, mu1, mu2, reg, max_iters=60)
    x60 = torch.empty((H, W), dtype=torch.float32, device="cuda")
    r60 = ad.solve(full, y, m, x60)
    assert r60.iters == 60
    first = ad.Plan(H, W, psf, lam, mu1, mu2, reg, max_iters=30)
    x30 = torch.empty_like(x60)
    ad.solve(first, y, m, x30)
    st = torch.empty(first.full_state_size(), dtype=torch.float32, device="cuda")
    assert first.get_full_state(st) == 30
    second = ad.Plan(H, W, psf, lam, mu1, mu2, reg, max_iters=30)
    second.set_state(st.cpu().numpy())           # host copy: the call copies it in
    xr = torch.empty_like(x60)
    rr = ad.solve(second, y, m, xr)
    torch.cuda.synchronize()
    assert rr.iters == 30
    assert torch.equal(xr, x60), float((xr - x60).abs().max())
    d60 = torch.empty(full.state_size(), dtype=torch.float32, device="cuda")
    dr = torch.empty_like(d60)
    ad.admm_deconv_get_state(full.handle, d60.data_ptr())
    ad.admm_deconv_get_state(second.handle, dr.data_ptr())
    assert torch.equal(dr, d60)
    # the restored state serves one solve: the next solve starts cold again
    xc = torch.empty_like(x60)
    ad.solve(second, y, m, xc)
    assert torch.equal(xc, x30)
    for p in (full, first, second):
        p.close()


@pytest.mark.parametrize("reg", ["tv", "haar", "haar_synthesis", "haar_cg"])
def test_state_round_trip_before_any_iteration(ad, reg):
    """set_state on a fresh plan, then get_full_state and get_state before
    any solve: the same floats come back (the frame priors keep zeta2 and
    bits only once an iteration has run; before that the buffers hold the
    restored d2, and for FS-MD the restored zeta2, as given)."""
    import torch
    H, W = 64, 128                # the Reeves-Sorel variants take powers of two
    psf = S.psf_box(5)
    plan = ad.Plan(H, W, psf, 1e-3, 3e-3, 1e-2, reg, max_iters=5)
    g = np.random.default_rng(5)
    st = g.standard_normal(plan.full_state_size()).astype(np.float32)
    plan.set_state(st)
    out = torch.empty(plan.full_state_size(), dtype=torch.float32, device="cuda")
    plan.get_full_state(out)
    assert np.array_equal(out.cpu().numpy(), st)
    d = torch.empty(plan.state_size(), dtype=torch.float32, device="cuda")
    ad.admm_deconv_get_state(plan.handle, d.data_ptr())
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy(), st[:plan.state_size()])
    plan.close()


def test_restart_resumes_the_oracle_sequence(ad):
    """The restarted GPU run follows the FP64 oracle's 60-iteration sequence
    (TV, 128 x 128) to the tolerance of the fixed-iteration parity tests."""
    import torch
    H = W = 128
    psf = S.psf_box(9)
    xt, ybar, mask = _problem(H, W, psf, 0.8, 52)
    lam = 1e-3
    mu1, mu2 = S.default_mu(lam)
    ref = O.solve(ybar.astype(np.float64), mask, psf, lam, mu1, mu2, "tv", iters=60)
    y = torch.from_numpy(ybar).cuda()
    m = torch.from_numpy(mask).cuda()
    a = ad.Plan(H, W, psf, lam, mu1, mu2, "tv", max_iters=25)
    x = torch.empty((H, W), dtype=torch.float32, device="cuda")
    ad.solve(a, y, m, x)
    st = np.empty(a.full_state_size(), dtype=np.float32)
    a.get_full_state(st)
    b = ad.Plan(H, W, psf, lam, mu1, mu2, "tv", max_iters=35)
    b.set_state(st)
    ad.solve(b, y, m, x)
    assert _rel(x.cpu().numpy().astype(np.float64), ref.x) <= 1e-4
    a.close()
    b.close()


def _next_side(n):
    """The next side the library solves on exactly: m 2^k with m in {1, 3, 5},
    a multiple of 32, at least 64."""
    m = max(n, 64)
    while True:
        odd = m
        while odd % 2 == 0:
            odd //= 2
        if m % 32 == 0 and odd in (1, 3, 5):
            return m
        m += 1


@pytest.mark.parametrize("reg,H,W,psf_fn,keep", [
    ("tv", 200, 300, lambda: S.psf_gaussian(7, 1.5), 0.7),
    ("tv", 130, 700, lambda: S.psf_box(5), 0.8),
    ("haar", 96, 100, lambda: S.psf_box(5), None),
    ("tv", 384, 384, lambda: S.psf_motion(11.0, 60.0, 11), 0.8),
])
def test_padded_domain_matches_oracle(ad, reg, H, W, psf_fn, keep):
    """ADMM_PAD_NEXT: the plan's domain is the next supported size (200 ->
    256, 300 -> 320, 130 -> 160, 700 -> 768, 100 -> 128; 96 and 384 are
    solved as they are); the oracle solves the same problem on that domain (the image top-left, the
    rest never observed; the valid region is the image's own); x is returned
    on the caller's H x W window and matches the oracle there."""
    import torch
    psf = psf_fn()
    xt, ybar, mask = _problem(H, W, psf, keep, 53)
    lam = 1e-3
    mu1, mu2 = S.default_mu(lam)
    iters = 40
    plan = ad.Plan(H, W, psf, lam, mu1, mu2, reg, max_iters=iters, pad=True)
    Hd, Wd = plan.domain()
    assert (Hd, Wd) == (_next_side(H), _next_side(W))
    yb = np.zeros((Hd, Wd))
    mk = np.zeros((Hd, Wd), dtype=np.uint8)
    yb[:H, :W] = ybar
    mk[:H, :W] = mask
    ref = O.solve(yb, mk, psf, lam, mu1, mu2, reg, iters=iters)
    x = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
    res = ad.solve(plan, torch.from_numpy(ybar).cuda(), torch.from_numpy(mask).cuda(), x)
    assert res.iters == iters
    xg = x.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(xg))
    assert _rel(xg, ref.x[:H, :W]) <= 1e-4
    # host buffers give the same bits
    xh = np.empty((H, W), dtype=np.float32)
    ad.solve(plan, ybar, mask, xh)
    assert np.array_equal(xh, x.cpu().numpy())
    plan.close()


def test_padding_policy_exact_rejects_unsupported_sizes(ad):
    with pytest.raises(ad.AdmmError) as e:
        ad.Plan(200, 300, S.psf_box(5), 1e-3, max_iters=5)
    assert e.value.code == ad.ADMM_EUNSUPPORTED_SIZE
    p = ad.Plan(256, 256, S.psf_box(5), 1e-3, max_iters=5, pad=True)   # supported: no padding
    assert p.domain() == (256, 256)
    p.close()


def test_use_warmstart_equals_the_manual_learned_start(ad):
    """solve_batch(use_warmstart=1) with the committed weights gives the bits
    of admm_cnn_predict_start + admm_deconv_warm_start + a plain solve; a
    frame problem in the same batch starts cold; the start converges to the
    same stop rule."""
    import torch
    from paper_1210_2687_gb300 import warmstart as ws
    params, scales, _ = ws.load()
    H = W = 256
    lam = ws.LAM
    mu1, mu2 = S.default_mu(lam)
    probs = [ws.eval_problem(900 + i, H) for i in range(3)]
    ad.admm_warmstart_load(ws.WEIGHTS_BIN)
    try:
        plans = [ad.Plan(H, W, p[3], lam, mu1, mu2, "tv", stop="rel_x", tol=1e-5, max_iters=3000,
                         check_every=1) for p in probs]
        ys = [torch.from_numpy(p[1]).cuda() for p in probs]
        ms = [torch.from_numpy(p[2]).cuda() for p in probs]
        xs = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in probs]
        hp = ad.Plan(H, W, S.psf_box(5), lam, mu1, mu2, "haar", max_iters=20)
        xh = torch.empty((H, W), dtype=torch.float32, device="cuda")
        res = ad.solve_batch(plans + [hp], ys + [ys[0]], ms + [ms[0]], xs + [xh], use_warmstart=True)
        # by hand
        net = ad.Cnn(H * W)
        net.set_params(params)
        x0 = torch.empty((1, H, W), dtype=torch.float32, device="cuda")
        d0 = torch.empty((1, 3 * H * W), dtype=torch.float32, device="cuda")
        for i, p in enumerate(probs):
            yb = torch.from_numpy(np.where(p[2] != 0, p[1], 0).astype(np.float32)).cuda()[None]
            net.predict_start(yb, ms[i][None], scales, x0, d0)
            plans[i].warm_start(x0[0], d0[0])
            xm = torch.empty((H, W), dtype=torch.float32, device="cuda")
            rm = ad.solve(plans[i], ys[i], ms[i], xm)
            torch.cuda.synchronize()
            assert torch.equal(xm, xs[i])
            assert rm.iters == res[i].iters and res[i].converged == 1
        xc = torch.empty((H, W), dtype=torch.float32, device="cuda")
        ad.solve(hp, ys[0], ms[0], xc)
        assert torch.equal(xc, xh)
        net.close()
        for p in plans + [hp]:
            p.close()
    finally:
        ad.admm_warmstart_load(None)


def test_use_warmstart_groups_match_one_image_passes(ad):
    """18 problems of 128 x 256 take the learned start in two passes of the
    network (16 + 2 images, per-image pointer tables); after 25 iterations
    each x has the bits of a solve started from a one-image prediction and
    admm_deconv_warm_start."""
    import torch
    from paper_1210_2687_gb300 import warmstart as ws
    params, scales, _ = ws.load()
    H, W = 128, 256
    lam = ws.LAM
    mu1, mu2 = S.default_mu(lam)
    rng = np.random.default_rng(5)
    count = 18
    psfs = [S.psf_box(5), S.psf_gaussian(7, 1.2), S.psf_box(3)]
    probs = []
    for i in range(count):
        y = rng.uniform(0.0, 1.0, size=(H, W)).astype(np.float32)
        m = (rng.uniform(size=(H, W)) > 0.3).astype(np.uint8)
        probs.append((y, m, psfs[i % 3]))
    ad.admm_warmstart_load(ws.WEIGHTS_BIN)
    try:
        plans = [ad.Plan(H, W, p[2], lam, mu1, mu2, "tv", stop="iters", max_iters=25) for p in probs]
        ys = [torch.from_numpy(p[0]).cuda() for p in probs]
        ms = [torch.from_numpy(p[1]).cuda() for p in probs]
        xs = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in probs]
        res = ad.solve_batch(plans, ys, ms, xs, use_warmstart=True)
        assert all(r.iters == 25 for r in res)
        net = ad.Cnn(H * W)
        net.set_params(params)
        x0 = torch.empty((1, H, W), dtype=torch.float32, device="cuda")
        d0 = torch.empty((1, 3 * H * W), dtype=torch.float32, device="cuda")
        for i, pl in enumerate(plans):
            vm = S.valid_mask(H, W, *probs[i][2].shape).astype(bool) & (probs[i][1] != 0)
            yb = torch.from_numpy(np.where(vm, probs[i][0], 0).astype(np.float32)).cuda()[None]
            mk = torch.from_numpy(vm.astype(np.uint8)).cuda()[None]
            net.predict_start(yb, mk, scales, x0, d0)
            pl.warm_start(x0[0], d0[0])
            xm = torch.empty((H, W), dtype=torch.float32, device="cuda")
            ad.solve(pl, ys[i], ms[i], xm)
            torch.cuda.synchronize()
            assert torch.equal(xm, xs[i]), i
        net.close()
        for pl in plans:
            pl.close()
    finally:
        ad.admm_warmstart_load(None)


def test_bounded_wait_runs_out_and_the_device_stays_usable(ad):
    """The row phase's wait for its spectrum rows is bounded (about a second):
    with one copy withheld the problem retires after its first iteration with
    ADMM_ETIMEOUT (also the call's return code); the hook serves one solve,
    and the next solves give the bits of an undisturbed plan."""
    import torch
    H = W = 128
    psf = S.psf_box(7)
    _, ybar, mask = _problem(H, W, psf, 0.8, 54)
    lam = 1e-3
    mu1, mu2 = S.default_mu(lam)
    y = torch.from_numpy(ybar).cuda()
    m = torch.from_numpy(mask).cuda()
    plan = ad.Plan(H, W, psf, lam, mu1, mu2, "tv", max_iters=6)
    x = torch.empty((H, W), dtype=torch.float32, device="cuda")
    ad.admm_deconv_set_option(ad.ADMM_OPT_TEST_STALL, 1)
    res = ad.solve(plan, y, m, x)
    assert res.status == ad.ADMM_ETIMEOUT and res.iters == 1 and res.converged == 0
    res = ad.solve(plan, y, m, x)
    torch.cuda.synchronize()
    assert res.status == ad.ADMM_OK and res.iters == 6
    other = ad.Plan(H, W, psf, lam, mu1, mu2, "tv", max_iters=6)
    x2 = torch.empty_like(x)
    ad.solve(other, y, m, x2)
    assert torch.equal(x, x2)
    plan.close()
    other.close()


_FAULT_SCRIPT = r"""
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
torch.cuda.init()
import paper_1210_2687_gb300 as ad
import synth as S
psf = S.psf_box(5)
H = W = 128
ys = [torch.zeros((H, W), dtype=torch.float32, device="cuda") for _ in range(3)]
xs = [torch.empty_like(y) for y in ys]


def sweep():
    fails = 0
    for n in range(1, 200):
        plans, net, done = [], None, False
        ad.admm_deconv_set_option(ad.ADMM_OPT_FAIL_ALLOC, n)
        try:
            for _ in range(3):
                plans.append(ad.Plan(H, W, psf, 1e-3, max_iters=3))
            ad.solve_batch(plans[:1], ys[:1], None, xs[:1])     # the library's tables, first size
            ad.solve_batch(plans, ys, None, xs)                 # the tables grown
            net = ad.Cnn(64 * 64, training=True)
            done = True
        except ad.AdmmError as e:
            assert e.code == ad.ADMM_ENOMEM, (n, e.code)
            fails += 1
        finally:
            ad.admm_deconv_set_option(ad.ADMM_OPT_FAIL_ALLOC, 0)
            for p in plans:
                p.close()
            if net is not None:
                net.close()
        if done:
            return fails
    raise AssertionError("no pass succeeded")


first = sweep()      # also loads the device code and sizes the library's tables
assert first >= 20, first
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
second = sweep()     # the same failures again, on warm tables: nothing may leak
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
assert second >= 10, second
assert abs(free0 - free1) < (1 << 20), (free0, free1)
# with the injection spent, a solve works and gives a finite image
p = ad.Plan(H, W, psf, 1e-3, max_iters=3)
ad.solve(p, ys[0] + 0.5, None, xs[0])
assert torch.isfinite(xs[0]).all()
p.close()
print("fault-injection ok", first, second)
"""


def test_injected_allocation_failures_return_enomem_and_recover(ad):
    """Host-side fault injection (ADMM_OPT_FAIL_ALLOC) in a fresh process: the
    n-th allocation fails for n = 1, 2, ... through three plans, a batch's
    first solve (the library's tables), a larger batch (the tables grown) and
    a training network, until one pass succeeds. Every failing call returns
    ADMM_ENOMEM. A second sweep, once the device code is loaded and the
    tables sized, must leave the device's free memory where it was (nothing
    a failing call took is leaked); afterwards a solve works."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FAULT_SCRIPT, root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "fault-injection ok" in r.stdout
