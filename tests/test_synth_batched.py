"""Host checks of the batched uneven workload's input generator: the FFT
valid-region convolution equals the direct tap sum, kernels follow the
stated law, and padded domains keep the padding unobserved."""
import numpy as np
import pytest

import synth as S


@pytest.mark.parametrize("psf", [S.psf_box(7), S.psf_gaussian(9, 2.0), S.psf_motion(11.0, 30.0, 11),
                                 S.psf_box(21)])
def test_fft_valid_convolution_equals_direct_sum(psf):
    x = S.rng(3).uniform(size=(45, 52))
    np.testing.assert_allclose(S.conv_valid_fft(x, psf), S.conv_valid(x, psf), rtol=0, atol=1e-13)


def test_fft_domain():
    assert [S.fft_domain(n) for n in (10, 64, 65, 128, 384, 512, 1000, 1024)] == \
        [64, 64, 128, 128, 512, 512, 1024, 1024]


def test_batched_law_and_padding():
    probs = S.config4_batch(0, 40)
    fams = set()
    for p in probs:
        n = p.meta["window"]
        N = S.fft_domain(n)
        assert n in S.CONFIG4_SIZES and p.ybar.shape == (N, N) == p.mask.shape
        ph, pw = p.psf.shape
        assert ph == pw and ph % 2 == 1 and 5 <= ph <= 25
        assert abs(p.psf.sum() - 1.0) < 1e-12 and (p.psf >= 0).all()
        assert 0.0 <= p.meta["missing"] <= 0.5
        assert p.reg in ("tv", "haar")
        fams.add(p.meta["family"])
        # observed pixels lie in the image's valid region; nothing on the padding
        vm = np.zeros((N, N), dtype=np.uint8)
        vm[:n, :n] = S.valid_mask(n, n, ph, pw)
        assert not (p.mask & (1 - vm)).any()
        assert (p.ybar[p.mask == 0] == 0).all()
        kept = p.mask.sum() / vm.sum()
        assert abs(kept - (1.0 - p.meta["missing"])) < 0.05
    assert fams == {"box", "gauss", "motion"}
    assert {p.meta["window"] for p in probs} == set(S.CONFIG4_SIZES)
