"""Pick lambda per (blur, BSNR) for the 512 x 512 TV inpainting workload by
best oracle ISNR after 300 TV-MD iterations on one calibration image (seed
1000), as the paper tuned lambda per condition for the best ISNR (Sec. V).
Run as a script; prints the table stored in synth.CONFIG2_LAMBDA (with the
argument "batched": the table synth.CONFIG4_LAMBDA).
Test infrastructure: uses the oracle only."""
import sys
import os

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle as O  # noqa: E402
import synth as S  # noqa: E402


def main(size=256, iters=300):
    grid = [1e-5, 3e-5, 1e-4, 3e-4, 1e-3, 3e-3]
    for blur in ("gauss", "motion"):
        for bsnr in (40, 60):
            best = None
            for lam in grid:
                S.CONFIG2_LAMBDA[(blur, bsnr)] = lam
                p = S.config2_problem(1000, blur, bsnr, size=size)
                r = O.solve(p.ybar, p.mask, p.psf, p.lam, p.mu1, p.mu2, "tv", iters=iters)
                v = O.isnr(p.x_true, p.ybar, r.x, S.valid_mask(size, size, *p.psf.shape))
                print(blur, bsnr, lam, round(v, 3), flush=True)
                if best is None or v > best[1]:
                    best = (lam, v)
            print("BEST", blur, bsnr, best, flush=True)




def main_batched(size=256, iters=300):
    """lambda per (regularizer, blur family) for the batched uneven workload
    at BSNR 40 dB, on one calibration image per family (seed 1000)."""
    grid = [1e-5, 3e-5, 1e-4, 3e-4, 1e-3, 3e-3]
    kernels = {"box": S.psf_box(13), "gauss": S.psf_gaussian(17, 2.5), "motion": S.psf_motion(15.0, 30.0, 15)}
    for reg in ("tv", "haar"):
        for fam, psf in kernels.items():
            g = S.rng(1000)
            x = S.textured_image(size, size, g)
            keep = (g.uniform(0.0, 1.0, size=(size, size)) >= 0.25).astype("uint8")
            ybar, mask, _ = S.observe(x, psf, keep, 40.0, g, fast=True)
            best = None
            for lam in grid:
                mu1, mu2 = S.default_mu(lam)
                r = O.solve(ybar, mask, psf, lam, mu1, mu2, reg, iters=iters)
                v = O.isnr(x, ybar, r.x, S.valid_mask(size, size, *psf.shape))
                print(reg, fam, lam, round(v, 3), flush=True)
                if best is None or v > best[1]:
                    best = (lam, v)
            print("BEST", reg, fam, best, flush=True)


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "batched":
        main_batched(*(int(a) for a in sys.argv[2:]))
    else:
        main(*(int(a) for a in sys.argv[1:]))
