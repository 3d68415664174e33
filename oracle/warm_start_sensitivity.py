"""How close a warm start has to be for TV-MD to save iterations: iterations
to rel-x < 1e-5 from perturbed copies of the fixed point (x*, d*) of one
128 x 128 problem (piecewise-constant image, 9 x 9 box, valid region, BSNR
40 dB, lambda 1e-3, mu by synth.default_mu). The start is u0 = H x0 - d0,
d0 given (oracle.cnn.warm_state). Run as a script; uses the oracle only
(test infrastructure)."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle as O  # noqa: E402
import oracle.cnn as C  # noqa: E402
import synth as S  # noqa: E402


def main(size=128):
    g = S.rng(5)
    x = S.shapes_image(size, size, g, 20, rmax=size / 4)
    psf = S.psf_box(9)
    ybar, mask, _ = S.observe(x, psf, None, 40.0, g)
    lam = 1e-3
    mu1, mu2 = S.default_mu(lam)
    cold = O.solve(ybar, mask, psf, lam, mu1, mu2, "tv", iters=5000, stop="rel_x", tol=1e-5)
    ref = O.solve(ybar, mask, psf, lam, mu1, mu2, "tv", iters=20000, stop="rel_x", tol=1e-12)
    xs, d1s, d2s = ref.x, ref.state.d1, ref.state.d2
    print("cold start", cold.iters)
    rng = np.random.default_rng(0)

    def run(x0, d1, d2, label):
        st = C.warm_state(x0, d1, d2, psf, "tv")
        r = O.solve(ybar, mask, psf, lam, mu1, mu2, "tv", iters=5000, stop="rel_x", tol=1e-5, state0=st)
        err = np.linalg.norm(r.x - xs) / np.linalg.norm(xs)
        print(f"{label:42s} iterations {r.iters:5d}   |x - x*|/|x*| {err:.1e}")

    run(xs, None, None, "x*, zero duals")
    run(xs, d1s, d2s, "x*, d*")
    for eps in (0.3, 0.1, 0.03, 0.01):
        run(xs, d1s * (1 + eps * rng.standard_normal(d1s.shape)), d2s * (1 + eps * rng.standard_normal(d2s.shape)),
            f"x*, d* with {eps:g} relative noise")
    for eps in (0.1, 0.03, 0.01):
        run(xs + eps * np.std(xs) * rng.standard_normal(xs.shape), d1s, d2s, f"x* + {eps:g} std noise, d*")
    run(np.where(mask > 0, ybar, ybar[mask > 0].mean()), None, None, "observation, zero duals")


if __name__ == "__main__":
    main()
