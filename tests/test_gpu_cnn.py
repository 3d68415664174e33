"""GPU parity of the warm-start network (BF16 tensor-core convolutions, FP32
accumulate) against the FP64 oracle in oracle/cnn.py: forward output,
loss and every parameter gradient, within a tolerance set by BF16 rounding
(relative L2 error per tensor <= 3e-2 and cosine >= 0.999), the Adam update
and the layout of the predicted warm start."""
import numpy as np
import pytest

import oracle.cnn as C
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


def _flat(params):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params]).astype(np.float32)


def _unflat(vec, like):
    out, o = [], 0
    for w, b in like:
        nw, nb = w.size, b.size
        out.append([vec[o:o + nw].reshape(w.shape).astype(np.float64), vec[o + nw:o + nw + nb].astype(np.float64)])
        o += nw + nb
    return out


def _params(seed):
    g = S.rng(seed)
    ps = C.init_params(seed)
    ps[-1][0] *= 10.0                       # an output of order one, not near zero
    for w, b in ps:
        b[:] = 0.05 * g.standard_normal(b.shape)
    return ps


def _batch(seed, count, H, W):
    g = S.rng(seed)
    ybar = g.uniform(0.0, 1.0, size=(count, H, W))
    mask = (g.uniform(size=(count, H, W)) < 0.7).astype(np.uint8)
    ybar = np.where(mask > 0, ybar, 0.0)
    tgt = g.standard_normal((count, H, W, 4)) * 0.5
    return ybar, mask, tgt


def _close(a, b, rel=3e-2, cos=0.999):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    r = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
    c = float(a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))
    return r <= rel and c >= cos, (r, c)


def _dev(ad, ybar, mask, tgt=None):
    import torch
    y = torch.from_numpy(ybar.astype(np.float32)).cuda()
    m = torch.from_numpy(mask).cuda()
    t = None if tgt is None else torch.from_numpy(tgt.astype(np.float32)).cuda()
    return y, m, t


@pytest.mark.parametrize("count,H,W", [(2, 32, 48), (1, 64, 16), (1, 512, 512), (2, 128, 96)])
def test_forward_matches_oracle(ad, count, H, W):
    import torch
    ps = _params(3)
    ybar, mask, _ = _batch(4, count, H, W)
    net = ad.Cnn(count * H * W)
    net.set_params(_flat(ps))
    y, m, _ = _dev(ad, ybar, mask)
    out = torch.empty((count, H, W, 4), dtype=torch.float32, device="cuda")
    net.forward(y, m, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for i in range(count):
        ref, _ = C.forward(ps, C.network_input(ybar[i], mask[i]))
        for k in range(4):
            ok, info = _close(got[i, :, :, k], ref[k])
            assert ok, (i, k, info)


@pytest.mark.parametrize("count,H,W", [(2, 32, 32), (1, 128, 96)])
def test_gradients_match_oracle(ad, count, H, W):
    import torch
    ps = _params(5)
    ybar, mask, tgt = _batch(6, count, H, W)
    cw = np.array([1.0, 0.5, 2.0, 2.0])
    net = ad.Cnn(count * H * W, training=True)
    net.set_params(_flat(ps))
    y, m, t = _dev(ad, ybar, mask, tgt)
    grads = torch.empty(ad.Cnn.param_count(), dtype=torch.float32, device="cuda")
    loss = net.gradients(y, m, t, cw, grads)
    inputs = [C.network_input(ybar[i], mask[i]) for i in range(count)]
    targets = [np.moveaxis(tgt[i], -1, 0) for i in range(count)]
    L, gref = C.batch_loss_and_grads(ps, inputs, targets, cw)
    assert abs(loss - L) <= 2e-2 * L
    got = _unflat(grads.cpu().numpy(), ps)
    for layer in range(len(ps)):
        for j, name in ((0, "w"), (1, "b")):
            ok, info = _close(got[layer][j], gref[layer][j])
            assert ok, (layer, name, info)


def test_adam_step_applies_the_update_to_its_own_gradients(ad):
    import torch
    ps = _params(7)
    count, H, W = 1, 32, 32
    ybar, mask, tgt = _batch(8, count, H, W)
    cw = np.array([1.0, 1.0, 1.0, 1.0])
    net = ad.Cnn(count * H * W, training=True)
    p0 = _flat(ps)
    net.set_params(p0)
    y, m, t = _dev(ad, ybar, mask, tgt)
    grads = torch.empty(ad.Cnn.param_count(), dtype=torch.float32, device="cuda")
    net.gradients(y, m, t, cw, grads)
    g = grads.cpu().numpy().astype(np.float64)
    lr = 1e-3
    net.train_step(y, m, t, cw, lr)
    p1 = net.get_params().astype(np.float64)
    # the oracle's Adam (Kingma and Ba, Algorithm 1) on the same gradients
    like = _unflat(p0, ps)
    want = _flat(C.Adam(like, lr=lr).step(like, _unflat(g.astype(np.float32), ps))).astype(np.float64)
    sel = np.abs(g) > 1e-6 * np.abs(g).max()
    np.testing.assert_allclose(p1[sel], want[sel], rtol=0, atol=2e-6)


def test_predict_start_layout(ad):
    import torch
    ps = _params(9)
    count, H, W = 2, 16, 32
    ybar, mask, _ = _batch(10, count, H, W)
    net = ad.Cnn(count * H * W)
    net.set_params(_flat(ps))
    y, m, _ = _dev(ad, ybar, mask)
    out = torch.empty((count, H, W, 4), dtype=torch.float32, device="cuda")
    net.forward(y, m, out)
    n = H * W
    x0 = torch.empty((count, H, W), dtype=torch.float32, device="cuda")
    d0 = torch.empty((count, 3 * n), dtype=torch.float32, device="cuda")
    sc = (0.9, 0.2, 0.1, 0.0)
    net.predict_start(y, m, sc, x0, d0)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    x0 = x0.cpu().numpy()
    d0 = d0.cpu().numpy()
    np.testing.assert_allclose(x0, sc[0] * o[..., 0], rtol=1e-6, atol=1e-7)
    for i in range(count):
        np.testing.assert_allclose(d0[i, :n].reshape(H, W), sc[1] * o[i, ..., 1], rtol=1e-6, atol=1e-7)
        d2 = d0[i, n:].reshape(H, W, 2)
        np.testing.assert_allclose(d2[..., 0], sc[2] * o[i, ..., 2], rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(d2[..., 1], sc[2] * o[i, ..., 3], rtol=1e-6, atol=1e-7)


def test_training_lowers_the_loss(ad):
    """A hundred Adam steps on one small batch lower its loss fourfold."""
    import torch
    ps = C.init_params(11)
    count, H, W = 4, 32, 32
    ybar, mask, _ = _batch(12, count, H, W)
    # a learnable target: the observation, its mask and two constants
    tgt = np.stack([ybar, mask.astype(np.float64), np.full_like(ybar, 0.3), np.full_like(ybar, -0.2)], axis=-1)
    net = ad.Cnn(count * H * W, training=True)
    net.set_params(_flat(ps))
    y, m, t = _dev(ad, ybar, mask, tgt)
    cw = (1.0, 1.0, 1.0, 1.0)
    first = net.train_step(y, m, t, cw, 3e-3)
    for _ in range(98):
        net.train_step(y, m, t, cw, 3e-3, want_loss=False)
    last = net.train_step(y, m, t, cw, 3e-3)
    assert last < 0.25 * first, (first, last)
