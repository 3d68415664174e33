"""Plain FP64 CPU oracle for the learned warm start of the ADMM solver.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): only the
tests, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` use it; it
shares no code with the CUDA path.

The paper has no learned component; its Theorem 1 makes ADMM converge from
any (u0, d0), which is what allows a predicted starting point. The network
is a plain stack of 3 x 3 convolutions:

    input  a0 = [M^T y, mask]                       (2 channels, H x W)
    z_l   = conv3x3(a_{l-1}; w_l, b_l),  a_l = relu(z_l)   for l = 1 .. L-1
    output o  = conv3x3(a_{L-1}; w_L, b_L)           (4 channels, no activation)

conv3x3 is a cross-correlation with zero padding outside the image ("same"
size):   z[o, r, c] = b[o] + sum_i sum_{p,q in {-1,0,1}} w[o, i, p+1, q+1] a[i, r+p, c+q].

The four output channels, each multiplied by a fixed scale, are the starting
point (x0, d1, d2h, d2v). The warm state is u0 = H x0 - d0 (so the first
x-step of Algorithm 2 returns x0) and d0 = (d1, d2); see ``warm_state``.

Training: squared error against targets per channel (weights c_k), averaged
over pixels and images; gradients by the chain rule written out below; Adam
(Kingma and Ba, ICLR 2015, Algorithm 1) on the weights and biases.
"""
from __future__ import annotations

import math

import numpy as np

from . import State, A_fft, Dh, Dv, haar_analysis, haar_nbands


# --------------------------------------------------------------------------
# layers
# --------------------------------------------------------------------------
def conv3x3(a: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """a: (Cin, H, W); w: (Cout, Cin, 3, 3); b: (Cout,) -> (Cout, H, W)."""
    cin, H, W = a.shape
    ap = np.zeros((cin, H + 2, W + 2))
    ap[:, 1:H + 1, 1:W + 1] = a
    z = np.zeros((w.shape[0], H, W)) + b[:, None, None]
    for p in (-1, 0, 1):
        for q in (-1, 0, 1):
            # shifted[i, r, c] = a[i, r + p, c + q] (zero outside)
            shifted = ap[:, 1 + p:1 + p + H, 1 + q:1 + q + W]
            z += np.einsum("oi,irc->orc", w[:, :, p + 1, q + 1], shifted)
    return z


def conv3x3_grad_input(g: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Adjoint of conv3x3 in its input: g (Cout, H, W) -> (Cin, H, W),
    ga[i, r, c] = sum_o sum_{p,q} w[o, i, p+1, q+1] g[o, r-p, c-q] (zero outside)."""
    cout, H, W = g.shape
    gp = np.zeros((cout, H + 2, W + 2))
    gp[:, 1:H + 1, 1:W + 1] = g
    ga = np.zeros((w.shape[1], H, W))
    for p in (-1, 0, 1):
        for q in (-1, 0, 1):
            shifted = gp[:, 1 - p:1 - p + H, 1 - q:1 - q + W]     # g[o, r - p, c - q]
            ga += np.einsum("oi,orc->irc", w[:, :, p + 1, q + 1], shifted)
    return ga


def conv3x3_grad_weight(g: np.ndarray, a: np.ndarray):
    """Gradients of sum(g * conv3x3(a; w, b)) in w and b:
    gw[o, i, p+1, q+1] = sum_{r,c} g[o, r, c] a[i, r+p, c+q];  gb[o] = sum g[o]."""
    cin, H, W = a.shape
    ap = np.zeros((cin, H + 2, W + 2))
    ap[:, 1:H + 1, 1:W + 1] = a
    gw = np.zeros((g.shape[0], cin, 3, 3))
    for p in (-1, 0, 1):
        for q in (-1, 0, 1):
            shifted = ap[:, 1 + p:1 + p + H, 1 + q:1 + q + W]
            gw[:, :, p + 1, q + 1] = np.einsum("orc,irc->oi", g, shifted)
    return gw, g.sum(axis=(1, 2))


def relu(z):
    return np.maximum(z, 0.0)


# --------------------------------------------------------------------------
# network
# --------------------------------------------------------------------------
def network_input(ybar: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """[M^T y, mask]: the observation zero-extended to the full domain (zero
    wherever the mask is 0) and the mask itself."""
    m = mask.astype(np.float64)
    return np.stack([np.where(m > 0, ybar, 0.0), m])


def layer_shapes(layers: int = 8, width: int = 32, cin: int = 2, cout: int = 4):
    """(Cout, Cin) of each convolution."""
    shapes = [(width, cin)]
    shapes += [(width, width)] * (layers - 2)
    shapes += [(cout, width)]
    return shapes


def init_params(seed: int, layers: int = 8, width: int = 32, cin: int = 2, cout: int = 4):
    """He-normal weights (std sqrt(2 / (9 Cin))), zero biases; the last layer's
    weights scaled by 0.1 so the initial prediction is near zero."""
    g = np.random.Generator(np.random.PCG64(seed))
    params = []
    shapes = layer_shapes(layers, width, cin, cout)
    for li, (co, ci) in enumerate(shapes):
        std = math.sqrt(2.0 / (9.0 * ci))
        if li == len(shapes) - 1:
            std *= 0.1
        params.append([g.standard_normal((co, ci, 3, 3)) * std, np.zeros(co)])
    return params


def forward(params, a0: np.ndarray):
    """Returns (output, list of post-activation inputs of every layer)."""
    acts = [a0]
    a = a0
    for li, (w, b) in enumerate(params):
        z = conv3x3(a, w, b)
        if li + 1 < len(params):
            a = relu(z)
            acts.append(a)
        else:
            return z, acts
    raise AssertionError("empty network")


def loss_and_grad_output(o: np.ndarray, t: np.ndarray, c: np.ndarray):
    """L = sum_k c_k mean_{r,c} (o_k - t_k)^2 and dL/do."""
    n = o.shape[1] * o.shape[2]
    diff = o - t
    L = float(np.sum(c[:, None, None] * diff * diff) / n)
    return L, 2.0 * c[:, None, None] * diff / n


def backward(params, acts, go: np.ndarray):
    """Gradients of the loss in every (w, b), given dL/do of the output."""
    grads = [None] * len(params)
    g = go
    for li in range(len(params) - 1, -1, -1):
        w, _ = params[li]
        a_in = acts[li]
        grads[li] = list(conv3x3_grad_weight(g, a_in))
        if li > 0:
            # through conv (adjoint in the input) and the relu that made a_in
            g = conv3x3_grad_input(g, w) * (a_in > 0.0)
    return grads


def batch_loss_and_grads(params, inputs, targets, c):
    """Mean over images of the per-image loss, and its gradients."""
    tot = 0.0
    acc = None
    for a0, t in zip(inputs, targets):
        o, acts = forward(params, a0)
        L, go = loss_and_grad_output(o, t, c)
        gr = backward(params, acts, go)
        tot += L
        if acc is None:
            acc = [[gw.copy(), gb.copy()] for gw, gb in gr]
        else:
            for k in range(len(gr)):
                acc[k][0] += gr[k][0]
                acc[k][1] += gr[k][1]
    nb = len(inputs)
    return tot / nb, [[gw / nb, gb / nb] for gw, gb in acc]


class Adam:
    """Kingma and Ba (2015), Algorithm 1: biased moments m, v; bias-corrected
    step lr * m_hat / (sqrt(v_hat) + eps)."""

    def __init__(self, params, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.t = 0
        self.m = [[np.zeros_like(w), np.zeros_like(b)] for w, b in params]
        self.v = [[np.zeros_like(w), np.zeros_like(b)] for w, b in params]

    def step(self, params, grads):
        self.t += 1
        for k in range(len(params)):
            for j in range(2):
                g = grads[k][j]
                self.m[k][j] = self.b1 * self.m[k][j] + (1.0 - self.b1) * g
                self.v[k][j] = self.b2 * self.v[k][j] + (1.0 - self.b2) * g * g
                mh = self.m[k][j] / (1.0 - self.b1 ** self.t)
                vh = self.v[k][j] / (1.0 - self.b2 ** self.t)
                params[k][j] = params[k][j] - self.lr * mh / (np.sqrt(vh) + self.eps)
        return params


# --------------------------------------------------------------------------
# warm start of the ADMM (Theorem 1: any u0, d0)
# --------------------------------------------------------------------------
def warm_state(x0, d1, d2, psf, reg="tv", levels=4) -> State:
    """State whose first x-step returns x0 and whose duals are d0 = (d1, d2):
    u0 = H x0 - d0 with H = (A, D) for TV or (A, P) for the frame prior, so
    zeta0 = u0 + d0 = H x0 and line 4 of Algorithm 2 solves
    H^T H x = H^T H x0. ``d2`` has shape (2, H, W) (TV) or (3L+1, H, W); None
    means zero duals."""
    H, W = x0.shape
    d1 = np.zeros((H, W)) if d1 is None else np.asarray(d1, dtype=np.float64)
    if reg in ("tv", "tv_aniso"):
        hx2 = np.stack([Dh(x0), Dv(x0)])
    else:
        hx2 = haar_analysis(x0, levels)
    if d2 is None:
        d2 = np.zeros_like(hx2)
    d2 = np.asarray(d2, dtype=np.float64)
    assert d2.shape == hx2.shape
    u1 = A_fft(x0, psf) - d1
    return State(u1, d1.copy(), hx2 - d2, d2.copy(), np.asarray(x0, dtype=np.float64).copy(), 0)


__all__ = ["conv3x3", "conv3x3_grad_input", "conv3x3_grad_weight", "relu", "network_input",
           "layer_shapes", "init_params", "forward", "loss_and_grad_output", "backward",
           "batch_loss_and_grads", "Adam", "warm_state", "haar_nbands"]
