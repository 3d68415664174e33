"""Pick the regularisation weight lambda per condition by the best oracle ISNR
of the converged solution, as the paper tuned lambda per condition for the
best ISNR (Sec. V). One calibration image per condition (seed 1000), the
grid {1e-5, 3e-5, 1e-4, 3e-4, 1e-3, 3e-3}, penalties by synth.default_mu,
solved to rel-x < 1e-5 (at most 3000 iterations); a value whose run did not
converge within the cap is not a candidate (its ISNR is not the method's).

Conditions:
  inpainting TV workload   (blur, BSNR) in {Gaussian 19 sigma 3, motion 15 at 30}
                           x {40, 60} dB, 40 % of interior pixels missing
                           -> synth.CONFIG2_LAMBDA
  batched uneven workload  (regularizer, blur family) in {TV, Haar}
                           x {box 13, Gaussian 17 sigma 2.5, motion 15 at 30},
                           25 % missing, 40 dB -> synth.CONFIG4_LAMBDA

Run as a script (prints the tables). Test infrastructure: uses the oracle
only."""
import multiprocessing as mp
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle as O  # noqa: E402
import synth as S  # noqa: E402

GRID = [1e-5, 3e-5, 1e-4, 3e-4, 1e-3, 3e-3]


def _kernel(name):
    return {"gauss19": lambda: S.psf_gaussian(19, 3.0),
            "motion15": lambda: S.psf_motion(15.0, 30.0, 15),
            "box13": lambda: S.psf_box(13),
            "gauss17": lambda: S.psf_gaussian(17, 2.5)}[name]()


def _isnr(job):
    table, key, kname, bsnr, missing, reg, lam, size = job
    psf = _kernel(kname)
    g = S.rng(1000)
    x = S.textured_image(size, size, g)
    keep = (g.uniform(0.0, 1.0, size=(size, size)) >= missing).astype("uint8")
    ybar, mask, _ = S.observe(x, psf, keep, float(bsnr), g, fast=True)
    mu1, mu2 = S.default_mu(lam)
    r = O.solve(ybar, mask, psf, lam, mu1, mu2, reg, iters=3000, stop="rel_x", tol=1e-5)
    v = O.isnr(x, ybar, r.x, S.valid_mask(size, size, *psf.shape))
    return table, key, lam, v, r.iters, r.converged


def jobs(size):
    out = []
    for blur, kname in (("gauss", "gauss19"), ("motion", "motion15")):
        for bsnr in (40, 60):
            for lam in GRID:
                out.append(("CONFIG2_LAMBDA", (blur, bsnr), kname, bsnr, 0.4, "tv", lam, size))
    for reg in ("tv", "haar"):
        for fam, kname in (("box", "box13"), ("gauss", "gauss17"), ("motion", "motion15")):
            for lam in GRID:
                out.append(("CONFIG4_LAMBDA", (reg, fam), kname, 40, 0.25, reg, lam, size))
    return out


def main(size=128, procs=8):
    best = {}
    with mp.get_context("spawn").Pool(procs) as pool:
        for table, key, lam, v, it, conv in pool.imap_unordered(_isnr, jobs(size)):
            print(table, key, lam, round(v, 3), it, "converged" if conv else "not converged", flush=True)
            k = (table, key)
            if conv and (k not in best or v > best[k][1]):
                best[k] = (lam, v)
    for (table, key), (lam, v) in sorted(best.items()):
        print("BEST", table, key, lam, round(v, 3))


if __name__ == "__main__":
    main(*(int(a) for a in sys.argv[1:]))
