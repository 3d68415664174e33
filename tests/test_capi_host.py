"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every function include/admm_deconv.h declares, and rejects invalid
parameters before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def ad():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1210_2687_gb300 as mod
    return mod


def _declared_functions():
    txt = "".join(open(h).read() for h in HEADERS)
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"ADMM_API\s+[\w\s\*]+?\b(admm_\w+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("admm_deconv_plan", "admm_deconv_solve", "admm_deconv_solve_batch",
                     "admm_deconv_destroy", "admm_strerror", "admm_deconv_warm_start",
                     "admm_cnn_create", "admm_cnn_train_step", "admm_cnn_predict_start"):
        assert required in names


def test_library_exports_every_declared_symbol(ad):
    so = ctypes.CDLL(ad.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(so, name), name
    assert set(_declared_functions()) <= set(ad.EXPORTED)


def test_strerror_and_version(ad):
    assert ad.admm_strerror(0) == "ok"
    for code in (-1, -2, -3, -4, -5, -6):
        assert ad.admm_strerror(code) not in ("ok", "unknown status")
    assert ad.admm_strerror(-99) == "unknown status"
    assert "sm_103a" in ad.admm_deconv_version()


def test_struct_layout_matches_header(ad):
    # admm_params_t: 4 ints, pointer, 3 floats, 3 ints, double, 4 ints, pointer
    assert ctypes.sizeof(ad.admm_params_t) == 80
    assert ad.admm_params_t.tol.offset == 48
    assert ad.admm_params_t.fft_pad_policy.offset == 68
    assert ad.admm_params_t.band_mu.offset == 72
    assert ctypes.sizeof(ad.admm_result_t) == 64
    assert ad.admm_result_t.primal_res.offset == 56


@pytest.mark.parametrize("change,code", [
    (dict(H=100), -4), (dict(W=32), -4), (dict(H=4096), -4),
    (dict(psf=np.ones((4, 5)) / 20), -1),          # even side
    (dict(psf=np.zeros((3, 3))), -1),              # zero DC gain
    (dict(lam=-1.0), -1),
    (dict(reg=7), -1), (dict(stop=9), -1),
    (dict(max_iters=0), -1), (dict(check_every=0), -1),
    (dict(reg="haar", levels=5), -1), (dict(reg="haar_ll_free", levels=5), -1), (dict(reg=8), -1),
    (dict(reg="haar_cg", levels=5), -1),
    (dict(reg="haar_synthesis", levels=5), -1),
    (dict(psf=np.ones((65, 65)) / 65 ** 2), -1),   # larger than supported kernel side
    (dict(H=4096, pad=True), -4), (dict(W=2049, pad=True), -4),   # no supported size to pad to
    (dict(H=100, W=100, psf=np.ones((101, 3)) / 303, pad=True), -1),   # kernel taller than the image
    (dict(reg="tv", band_mu=np.ones(13)), -1),                 # per-band penalties: frame priors only
    (dict(reg="haar", band_mu=np.r_[np.ones(12), 0.0]), -1),   # a penalty that is not > 0
    (dict(reg="haar", band_mu=np.r_[np.ones(12), np.nan]), -1),
    (dict(reg="haar_synthesis", band_mu=np.ones(13)), -1),
    (dict(reg="haar_cg", band_mu=np.ones(13)), -1),
])
def test_plan_rejects_invalid_parameters_on_host(ad, change, code):
    kw = dict(H=64, W=64, psf=np.ones((3, 3)) / 9, lam=1e-3, reg="tv", levels=4, stop="iters",
              max_iters=10, check_every=1)
    kw.update(change)
    H, W, psf, lam = kw.pop("H"), kw.pop("W"), kw.pop("psf"), kw.pop("lam")
    with pytest.raises(ad.AdmmError) as e:
        ad.Plan(H, W, psf, lam, **kw)
    assert e.value.code == code


def test_null_arguments(ad):
    lib = ad.lib
    assert lib.admm_deconv_plan(None, None, None) == ad.ADMM_EINVAL
    assert lib.admm_deconv_solve_batch(None, 1, None, None, None, None, 0, None) == ad.ADMM_EINVAL
    assert lib.admm_deconv_solve_batch(None, 0, None, None, None, None, 0, None) == ad.ADMM_OK
    assert lib.admm_deconv_solve_batch(None, -1, None, None, None, None, 0, None) == ad.ADMM_EINVAL
    assert lib.admm_deconv_state_size(None) == -1
    assert lib.admm_deconv_full_state_size(None) == -1
    assert lib.admm_deconv_get_full_state(None, None, None, None) == ad.ADMM_EINVAL
    assert lib.admm_deconv_set_state(None, None, None) == ad.ADMM_EINVAL
    assert lib.admm_deconv_domain(None, None, None) == ad.ADMM_EINVAL
    # use_warmstart must be 0 or 1
    assert lib.admm_deconv_solve_batch(None, 1, None, None, None, None, 2, None) == ad.ADMM_EINVAL
    lib.admm_deconv_destroy(None)   # no-op


def test_pad_policy_must_be_known(ad):
    p = ad.admm_params_t()
    k = (ctypes.c_float * 9)(*([1.0 / 9] * 9))
    p.H = p.W = 64
    p.psf_h = p.psf_w = 3
    p.psf = ctypes.cast(k, ctypes.POINTER(ctypes.c_float))
    p.max_iters, p.check_every = 10, 1
    p.fft_pad_policy = 2
    h = ctypes.c_void_p()
    assert ad.lib.admm_deconv_plan(ctypes.byref(h), ctypes.byref(p), None) == ad.ADMM_EINVAL


def test_warmstart_file_loads_and_bad_files_are_rejected(ad, tmp_path):
    """admm_warmstart_load reads the committed weights (parsed on the host;
    the network is created on the device only when a solve uses it) and
    rejects a wrong magic, a wrong count, a truncated file, trailing bytes and
    non-finite parameters; use_warmstart without a loaded network is EINVAL."""
    from paper_1210_2687_gb300 import warmstart as ws
    assert os.path.exists(ws.WEIGHTS_BIN)
    ad.admm_warmstart_load(None)
    assert ad.lib.admm_deconv_solve_batch(None, 1, None, None, None, None, 1, None) == ad.ADMM_EINVAL
    ad.admm_warmstart_load(ws.WEIGHTS_BIN)
    good = open(ws.WEIGHTS_BIN, "rb").read()
    bad = {"magic": b"ADMMCNN2" + good[8:], "count": good[:16] + np.array([5], "<i8").tobytes() + good[24:],
           "short": good[:-4], "long": good + b"\0\0\0\0",
           "nan": good[:40] + np.array([np.nan], "<f4").tobytes() + good[44:]}
    for name, blob in bad.items():
        f = tmp_path / f"{name}.bin"
        f.write_bytes(blob)
        assert ad.lib.admm_warmstart_load(os.fsencode(str(f))) == ad.ADMM_EINVAL, name
    assert ad.lib.admm_warmstart_load(os.fsencode(str(tmp_path / "missing.bin"))) == ad.ADMM_EINVAL
    ad.admm_warmstart_load(None)


def test_set_option_validates(ad):
    assert ad.lib.admm_deconv_set_option(ad.ADMM_OPT_MAX_SLOTS, -1) == ad.ADMM_EINVAL
    assert ad.lib.admm_deconv_set_option(ad.ADMM_OPT_FAIL_ALLOC, -1) == ad.ADMM_EINVAL
    assert ad.lib.admm_deconv_set_option(ad.ADMM_OPT_FAIL_ALLOC, 0) == ad.ADMM_OK
    assert ad.lib.admm_deconv_set_option(ad.ADMM_OPT_TEST_STALL, 2) == ad.ADMM_EINVAL
    assert ad.lib.admm_deconv_set_option(ad.ADMM_OPT_TEST_STALL, 0) == ad.ADMM_OK
    assert ad.lib.admm_deconv_set_option(99, 1) == ad.ADMM_EINVAL
    assert ad.lib.admm_deconv_set_option(ad.ADMM_OPT_MAX_SLOTS, 0) == ad.ADMM_OK


def test_cnn_parameter_count_matches_the_oracle_network(ad):
    import oracle.cnn as C
    n = sum(co * ci * 9 + co for co, ci in C.layer_shapes())
    assert ad.Cnn.param_count() == n == 57252


def test_cnn_null_arguments(ad):
    lib = ad.lib
    assert lib.admm_cnn_create(None, 1, 0) == ad.ADMM_EINVAL
    assert lib.admm_cnn_set_params(None, None) == ad.ADMM_EINVAL
    assert lib.admm_cnn_forward(None, 1, 16, 16, None, None, None, None) == ad.ADMM_EINVAL
    assert lib.admm_deconv_warm_start(None, None, None, None) == ad.ADMM_EINVAL
    lib.admm_cnn_destroy(None)


def test_tuning_struct_layout(ad):
    # admm_tuning_t: 14 ints, double
    assert ctypes.sizeof(ad.admm_tuning_t) == 64
    assert ad.admm_tuning_t.us_per_iter.offset == 56


def test_every_size_has_compiled_configurations(ad):
    sides = (64, 128, 256, 512, 1024, 2048)
    for H in sides:
        for W in sides:
            nr, nc = ad.admm_deconv_variants(H, W, "tv")
            assert nr >= 2 and nc >= 2
            nr, nc = ad.admm_deconv_variants(H, W, "haar")
            assert nr == 1 and nc >= 2
    n_r, n_c = ctypes.c_int(), ctypes.c_int()
    assert ad.lib.admm_deconv_variants(384, 512, 0, ctypes.byref(n_r), ctypes.byref(n_c)) == ad.ADMM_EUNSUPPORTED_SIZE
    assert ad.lib.admm_deconv_variants(512, 512, 7, ctypes.byref(n_r), ctypes.byref(n_c)) == ad.ADMM_EINVAL
    assert ad.lib.admm_deconv_variants(512, 512, 0, None, None) == ad.ADMM_EINVAL


@pytest.mark.parametrize("change", [dict(row_variant=99), dict(col_variant=-1), dict(slot_ctas=-5), dict(lanes=5),
                                    dict(reg=1, row_variant=1), dict(reg=1, haar_levels=9)])
def test_set_tuning_rejects_out_of_range_on_host(ad, change):
    t = ad.admm_tuning_t(H=512, W=512, reg=0, haar_levels=0, row_variant=0, col_variant=0, slot_ctas=0)
    for k, v in change.items():
        setattr(t, k, v)
    assert ad.lib.admm_deconv_set_tuning(ctypes.byref(t)) == ad.ADMM_EINVAL
    t = ad.admm_tuning_t(H=500, W=512)
    assert ad.lib.admm_deconv_set_tuning(ctypes.byref(t)) == ad.ADMM_EUNSUPPORTED_SIZE
    assert ad.lib.admm_deconv_set_tuning(None) == ad.ADMM_EINVAL


def test_headers_compile_as_c99(tmp_path):
    """The boundary is plain C: both headers compile as C99 with warnings as
    errors (no C++ types or syntax leak into the ABI)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text('#include "admm_deconv.h"\n#include "admm_warmstart.h"\n'
                   "int main(void) { admm_params_t p; admm_result_t r; admm_tuning_t t; admm_profile_t f;\n"
                   "  (void)p; (void)r; (void)t; (void)f; return 0; }\n")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), "-c", str(src), "-o", str(tmp_path / "abi.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_launch_overlap_switch_on_host(ad):
    """The launch-chain switch is a host-side setting (no device needed):
    on by default, and it reads back what was set."""
    assert ad.admm_deconv_get_launch_overlap() is True
    try:
        ad.admm_deconv_set_launch_overlap(False)
        assert ad.admm_deconv_get_launch_overlap() is False
        assert ad.lib.admm_deconv_set_launch_overlap(7) == ad.ADMM_OK
        assert ad.lib.admm_deconv_get_launch_overlap() == 1
    finally:
        ad.admm_deconv_set_launch_overlap(True)
