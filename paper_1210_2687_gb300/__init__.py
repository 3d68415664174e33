"""Python binding of libadmm_deconv (mask-decoupled ADMM deconvolution on sm_103a).

Argument marshalling only: every step of the solve runs in the CUDA library
declared by include/admm_deconv.h. Importing this module loads the in-tree
``libadmm_deconv.so`` and raises if it is missing -- there is no CPU fallback.
Build it with ``python paper_1210_2687_gb300/build.py``.

The function names mirror the C ABI (admm_deconv_plan, admm_deconv_solve,
admm_deconv_solve_batch, admm_deconv_destroy, admm_strerror, ...); ``Plan``
and ``solve`` are conveniences on top that take numpy arrays or torch tensors
(host or CUDA) and pass their data pointers.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libadmm_deconv.so")

ADMM_OK = 0
ADMM_EINVAL = -1
ADMM_ENOMEM = -2
ADMM_ECUDA = -3
ADMM_EUNSUPPORTED_SIZE = -4
ADMM_ENONFINITE = -5
ADMM_ETIMEOUT = -6

ADMM_REG_TV = 0
ADMM_REG_HAAR = 1
ADMM_REG_TV_ANISO = 2
ADMM_REG_HAAR_LL_FREE = 3
ADMM_REG_HAAR_SYNTHESIS = 4
ADMM_REG_TV_CG = 5
ADMM_REG_HAAR_CG = 6
ADMM_PAD_EXACT = 0
ADMM_PAD_NEXT = 1
ADMM_STOP_ITERS = 0
ADMM_STOP_REL_X = 1
ADMM_STOP_REL_OBJ = 2

_REG = {"tv": ADMM_REG_TV, "haar": ADMM_REG_HAAR, "tv_aniso": ADMM_REG_TV_ANISO,
        "haar_ll_free": ADMM_REG_HAAR_LL_FREE, "haar_synthesis": ADMM_REG_HAAR_SYNTHESIS,
        "tv_cg": ADMM_REG_TV_CG, "haar_cg": ADMM_REG_HAAR_CG}
_STOP = {"iters": ADMM_STOP_ITERS, "rel_x": ADMM_STOP_REL_X, "rel_obj": ADMM_STOP_REL_OBJ}

EXPORTED = ("admm_deconv_plan", "admm_deconv_solve", "admm_deconv_solve_batch",
            "admm_deconv_state_size", "admm_deconv_get_state", "admm_deconv_destroy",
            "admm_strerror", "admm_deconv_version", "admm_deconv_profile",
            "admm_deconv_set_launch_overlap", "admm_deconv_get_launch_overlap",
            "admm_deconv_solve_noalloc", "admm_deconv_set_option", "admm_deconv_warm_start",
            "admm_deconv_variants", "admm_deconv_get_tuning", "admm_deconv_set_tuning", "admm_deconv_autotune",
            "admm_cnn_param_count", "admm_cnn_create", "admm_cnn_set_params", "admm_cnn_get_params",
            "admm_cnn_forward", "admm_cnn_gradients", "admm_cnn_train_step", "admm_cnn_predict_start",
            "admm_cnn_launches", "admm_cnn_destroy",
            "admm_deconv_domain", "admm_deconv_full_state_size", "admm_deconv_get_full_state",
            "admm_deconv_set_state", "admm_warmstart_load")

ADMM_OPT_MAX_SLOTS = 1
ADMM_OPT_FAIL_ALLOC = 2
ADMM_OPT_TEST_STALL = 3


class admm_params_t(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int),
                ("psf_h", ctypes.c_int), ("psf_w", ctypes.c_int),
                ("psf", ctypes.POINTER(ctypes.c_float)),
                ("lambda_", ctypes.c_float), ("mu1", ctypes.c_float), ("mu2", ctypes.c_float),
                ("reg", ctypes.c_int), ("haar_levels", ctypes.c_int),
                ("stop", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_iters", ctypes.c_int), ("check_every", ctypes.c_int),
                ("raw_mask", ctypes.c_int), ("fft_pad_policy", ctypes.c_int),
                ("band_mu", ctypes.POINTER(ctypes.c_float))]


class admm_result_t(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("status", ctypes.c_int), ("reserved", ctypes.c_int),
                ("objective", ctypes.c_double), ("rel_x", ctypes.c_double),
                ("rel_obj", ctypes.c_double), ("t_start_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double), ("primal_res", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class admm_profile_t(ctypes.Structure):
    _fields_ = [("col_ms", ctypes.c_double), ("row_ms", ctypes.c_double),
                ("col_launches", ctypes.c_longlong), ("row_launches", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class admm_tuning_t(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("reg", ctypes.c_int), ("haar_levels", ctypes.c_int),
                ("row_variant", ctypes.c_int), ("col_variant", ctypes.c_int), ("slot_ctas", ctypes.c_int),
                ("lanes", ctypes.c_int),
                ("rows_per_strip", ctypes.c_int), ("walk_depth", ctypes.c_int), ("row_threads", ctypes.c_int),
                ("col_block", ctypes.c_int), ("col_min_ctas", ctypes.c_int), ("col_persistent", ctypes.c_int),
                ("us_per_iter", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class AdmmError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        super().__init__(f"{what}: {admm_strerror(code)} ({code})")
        self.code = code


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing; build it with `python paper_1210_2687_gb300/build.py`")
    lib = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    lib.admm_deconv_plan.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(admm_params_t), vp]
    lib.admm_deconv_plan.restype = ctypes.c_int
    lib.admm_deconv_solve.argtypes = [vp, vp, vp, vp, ctypes.POINTER(admm_result_t), vp]
    lib.admm_deconv_solve.restype = ctypes.c_int
    lib.admm_deconv_solve_batch.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp),
                                            ctypes.POINTER(vp), ctypes.POINTER(vp),
                                            ctypes.POINTER(admm_result_t), ctypes.c_int, vp]
    lib.admm_deconv_solve_batch.restype = ctypes.c_int
    lib.admm_deconv_domain.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.admm_deconv_domain.restype = ctypes.c_int
    lib.admm_deconv_full_state_size.argtypes = [vp]
    lib.admm_deconv_full_state_size.restype = ctypes.c_longlong
    lib.admm_deconv_get_full_state.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int), vp]
    lib.admm_deconv_get_full_state.restype = ctypes.c_int
    lib.admm_deconv_set_state.argtypes = [vp, vp, vp]
    lib.admm_deconv_set_state.restype = ctypes.c_int
    lib.admm_warmstart_load.argtypes = [ctypes.c_char_p]
    lib.admm_warmstart_load.restype = ctypes.c_int
    lib.admm_deconv_state_size.argtypes = [vp]
    lib.admm_deconv_state_size.restype = ctypes.c_longlong
    lib.admm_deconv_get_state.argtypes = [vp, vp, vp]
    lib.admm_deconv_get_state.restype = ctypes.c_int
    lib.admm_deconv_warm_start.argtypes = [vp, vp, vp, vp]
    lib.admm_deconv_warm_start.restype = ctypes.c_int
    lib.admm_deconv_destroy.argtypes = [vp]
    lib.admm_deconv_destroy.restype = None
    lib.admm_strerror.argtypes = [ctypes.c_int]
    lib.admm_strerror.restype = ctypes.c_char_p
    lib.admm_deconv_version.argtypes = []
    lib.admm_deconv_version.restype = ctypes.c_char_p
    lib.admm_deconv_profile.argtypes = [ctypes.c_int, ctypes.POINTER(admm_profile_t)]
    lib.admm_deconv_profile.restype = ctypes.c_int
    lib.admm_deconv_set_launch_overlap.argtypes = [ctypes.c_int]
    lib.admm_deconv_set_launch_overlap.restype = ctypes.c_int
    lib.admm_deconv_get_launch_overlap.argtypes = []
    lib.admm_deconv_get_launch_overlap.restype = ctypes.c_int
    lib.admm_deconv_solve_noalloc.argtypes = [ctypes.POINTER(admm_params_t), vp, vp, vp,
                                              ctypes.POINTER(admm_result_t), vp]
    lib.admm_deconv_solve_noalloc.restype = ctypes.c_int
    lib.admm_deconv_set_option.argtypes = [ctypes.c_int, ctypes.c_longlong]
    lib.admm_deconv_set_option.restype = ctypes.c_int
    tp = ctypes.POINTER(admm_tuning_t)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.admm_deconv_variants.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ip]
    lib.admm_deconv_variants.restype = ctypes.c_int
    lib.admm_deconv_get_tuning.argtypes = [tp]
    lib.admm_deconv_get_tuning.restype = ctypes.c_int
    lib.admm_deconv_set_tuning.argtypes = [tp]
    lib.admm_deconv_set_tuning.restype = ctypes.c_int
    lib.admm_deconv_autotune.argtypes = [ctypes.c_int] * 6 + [tp, ctypes.c_int, ip, tp, vp]
    lib.admm_deconv_autotune.restype = ctypes.c_int
    ci, fp = ctypes.c_int, ctypes.c_float
    dp = ctypes.POINTER(ctypes.c_double)
    lib.admm_cnn_param_count.argtypes = []
    lib.admm_cnn_param_count.restype = ctypes.c_longlong
    lib.admm_cnn_launches.argtypes = []
    lib.admm_cnn_launches.restype = ctypes.c_longlong
    lib.admm_cnn_create.argtypes = [ctypes.POINTER(vp), ctypes.c_longlong, ci]
    lib.admm_cnn_create.restype = ci
    lib.admm_cnn_set_params.argtypes = [vp, vp]
    lib.admm_cnn_set_params.restype = ci
    lib.admm_cnn_get_params.argtypes = [vp, vp]
    lib.admm_cnn_get_params.restype = ci
    lib.admm_cnn_forward.argtypes = [vp, ci, ci, ci, vp, vp, vp, vp]
    lib.admm_cnn_forward.restype = ci
    lib.admm_cnn_gradients.argtypes = [vp, ci, ci, ci, vp, vp, vp, ctypes.POINTER(fp), vp, dp, vp]
    lib.admm_cnn_gradients.restype = ci
    lib.admm_cnn_train_step.argtypes = [vp, ci, ci, ci, vp, vp, vp, ctypes.POINTER(fp), fp, dp, vp]
    lib.admm_cnn_train_step.restype = ci
    lib.admm_cnn_predict_start.argtypes = [vp, ci, ci, ci, vp, vp, ctypes.POINTER(fp), vp, vp, vp]
    lib.admm_cnn_predict_start.restype = ci
    lib.admm_cnn_destroy.argtypes = [vp]
    lib.admm_cnn_destroy.restype = None
    return lib


lib = _load()


# ---- thin C-ABI mirrors ----------------------------------------------------
def admm_strerror(code: int) -> str:
    return lib.admm_strerror(int(code)).decode()


def admm_deconv_version() -> str:
    return lib.admm_deconv_version().decode()


def admm_deconv_plan(params: admm_params_t, stream=None) -> int:
    h = ctypes.c_void_p()
    rc = lib.admm_deconv_plan(ctypes.byref(h), ctypes.byref(params), _stream(stream))
    if rc != ADMM_OK:
        raise AdmmError(rc, "admm_deconv_plan")
    return h.value


def admm_deconv_solve(plan: int, y_ptr: int, mask_ptr: int | None, x_ptr: int, stream=None) -> admm_result_t:
    res = admm_result_t()
    rc = lib.admm_deconv_solve(ctypes.c_void_p(plan), ctypes.c_void_p(y_ptr), ctypes.c_void_p(mask_ptr or 0),
                               ctypes.c_void_p(x_ptr), ctypes.byref(res), _stream(stream))
    if rc not in (ADMM_OK, ADMM_ENONFINITE, ADMM_ETIMEOUT):   # per-problem statuses: in the result
        raise AdmmError(rc, "admm_deconv_solve")
    return res


def admm_deconv_solve_batch(plans: Sequence[int], y_ptrs, mask_ptrs, x_ptrs, use_warmstart=False, stream=None):
    n = len(plans)
    P = (ctypes.c_void_p * n)(*plans)
    Y = (ctypes.c_void_p * n)(*y_ptrs)
    M = (ctypes.c_void_p * n)(*[m or 0 for m in mask_ptrs]) if mask_ptrs is not None else None
    X = (ctypes.c_void_p * n)(*x_ptrs)
    R = (admm_result_t * n)()
    rc = lib.admm_deconv_solve_batch(P, n, Y, M, X, R, int(bool(use_warmstart)), _stream(stream))
    if rc not in (ADMM_OK, ADMM_ENONFINITE, ADMM_ETIMEOUT):   # per-problem statuses: in the results
        raise AdmmError(rc, "admm_deconv_solve_batch")
    return list(R)


def admm_deconv_state_size(plan: int) -> int:
    return int(lib.admm_deconv_state_size(ctypes.c_void_p(plan)))


def admm_deconv_get_state(plan: int, out_ptr: int, stream=None) -> None:
    rc = lib.admm_deconv_get_state(ctypes.c_void_p(plan), ctypes.c_void_p(out_ptr), _stream(stream))
    if rc != ADMM_OK:
        raise AdmmError(rc, "admm_deconv_get_state")


def admm_deconv_domain(plan: int) -> tuple[int, int]:
    h, w = ctypes.c_int(), ctypes.c_int()
    rc = lib.admm_deconv_domain(ctypes.c_void_p(plan), ctypes.byref(h), ctypes.byref(w))
    if rc != ADMM_OK:
        raise AdmmError(rc, "admm_deconv_domain")
    return h.value, w.value


def admm_deconv_full_state_size(plan: int) -> int:
    return int(lib.admm_deconv_full_state_size(ctypes.c_void_p(plan)))


def admm_deconv_get_full_state(plan: int, out_ptr: int, stream=None) -> int:
    """Copy the complete iteration state out; returns the iterations of the last solve."""
    it = ctypes.c_int()
    rc = lib.admm_deconv_get_full_state(ctypes.c_void_p(plan), ctypes.c_void_p(out_ptr), ctypes.byref(it),
                                        _stream(stream))
    if rc != ADMM_OK:
        raise AdmmError(rc, "admm_deconv_get_full_state")
    return it.value


def admm_deconv_set_state(plan: int, state_ptr: int, stream=None) -> None:
    rc = lib.admm_deconv_set_state(ctypes.c_void_p(plan), ctypes.c_void_p(state_ptr), _stream(stream))
    if rc != ADMM_OK:
        raise AdmmError(rc, "admm_deconv_set_state")


def admm_warmstart_load(path: str | None) -> None:
    """Load the learned warm-start network from a weights file (None unloads it)."""
    rc = lib.admm_warmstart_load(None if path is None else os.fsencode(path))
    if rc != ADMM_OK:
        raise AdmmError(rc, "admm_warmstart_load")


def admm_deconv_warm_start(plan: int, x0_ptr, d0_ptr, stream=None) -> None:
    rc = lib.admm_deconv_warm_start(ctypes.c_void_p(plan), ctypes.c_void_p(x0_ptr),
                                    ctypes.c_void_p(d0_ptr), _stream(stream))
    if rc != ADMM_OK:
        raise AdmmError(rc, "admm_deconv_warm_start")


def admm_deconv_set_launch_overlap(enable: bool) -> None:
    """Launch the batch engine's iteration kernels as a programmatic
    dependent chain (True, the default) or as plain stream-ordered launches."""
    lib.admm_deconv_set_launch_overlap(int(bool(enable)))


def admm_deconv_get_launch_overlap() -> bool:
    return bool(lib.admm_deconv_get_launch_overlap())


def admm_deconv_profile(enable: bool) -> admm_profile_t:
    """Read-and-reset the launch counters, then switch per-phase timing."""
    out = admm_profile_t()
    lib.admm_deconv_profile(int(bool(enable)), ctypes.byref(out))
    return out


def admm_deconv_solve_noalloc(params: admm_params_t, y_ptr: int, mask_ptr: int | None, x_ptr: int,
                              stream=None):
    """TV solve that allocates nothing (for callers that may not allocate
    device memory while running); device pointers only, H, W <= 256.
    Returns (status code, admm_result_t)."""
    res = admm_result_t()
    rc = lib.admm_deconv_solve_noalloc(ctypes.byref(params), ctypes.c_void_p(y_ptr),
                                       ctypes.c_void_p(mask_ptr or 0), ctypes.c_void_p(x_ptr),
                                       ctypes.byref(res), _stream(stream))
    return rc, res


def _f4(vals):
    arr = (ctypes.c_float * 4)(*[float(v) for v in vals])
    return arr


def _check(rc, what):
    if rc != ADMM_OK:
        raise AdmmError(rc, what)


class Cnn:
    """Owns one admm_cnn_t (the warm-start network). Images are passed as
    contiguous CUDA tensors of shape (count, H, W) (float32 ybar, uint8 mask);
    targets (count, H, W, 4) float32."""

    def __init__(self, max_pixels: int, training: bool = False):
        h = ctypes.c_void_p()
        _check(lib.admm_cnn_create(ctypes.byref(h), int(max_pixels), int(bool(training))), "admm_cnn_create")
        self.handle = h.value

    @staticmethod
    def param_count() -> int:
        return int(lib.admm_cnn_param_count())

    def set_params(self, params) -> None:
        _check(lib.admm_cnn_set_params(ctypes.c_void_p(self.handle), ctypes.c_void_p(_ptr(params, np.float32))),
               "admm_cnn_set_params")

    def get_params(self) -> np.ndarray:
        out = np.empty(self.param_count(), dtype=np.float32)
        _check(lib.admm_cnn_get_params(ctypes.c_void_p(self.handle), ctypes.c_void_p(out.ctypes.data)),
               "admm_cnn_get_params")
        return out

    def forward(self, ybar, mask, out, stream=None) -> None:
        n, H, W = ybar.shape
        _check(lib.admm_cnn_forward(ctypes.c_void_p(self.handle), n, H, W, ctypes.c_void_p(_ptr(ybar, np.float32)),
                                    ctypes.c_void_p(_ptr(mask, np.uint8)), ctypes.c_void_p(_ptr(out, np.float32)),
                                    _stream(stream)), "admm_cnn_forward")

    def gradients(self, ybar, mask, target, chan_w, grads, stream=None) -> float:
        n, H, W = ybar.shape
        loss = ctypes.c_double()
        _check(lib.admm_cnn_gradients(ctypes.c_void_p(self.handle), n, H, W, ctypes.c_void_p(_ptr(ybar, np.float32)),
                                      ctypes.c_void_p(_ptr(mask, np.uint8)), ctypes.c_void_p(_ptr(target, np.float32)),
                                      _f4(chan_w), ctypes.c_void_p(_ptr(grads, np.float32)), ctypes.byref(loss),
                                      _stream(stream)), "admm_cnn_gradients")
        return loss.value

    def train_step(self, ybar, mask, target, chan_w, lr, want_loss=True, stream=None):
        n, H, W = ybar.shape
        loss = ctypes.c_double()
        _check(lib.admm_cnn_train_step(ctypes.c_void_p(self.handle), n, H, W, ctypes.c_void_p(_ptr(ybar, np.float32)),
                                       ctypes.c_void_p(_ptr(mask, np.uint8)),
                                       ctypes.c_void_p(_ptr(target, np.float32)), _f4(chan_w), float(lr),
                                       ctypes.byref(loss) if want_loss else None, _stream(stream)),
               "admm_cnn_train_step")
        return loss.value if want_loss else None

    def predict_start(self, ybar, mask, scales, x0, d0, stream=None) -> None:
        n, H, W = ybar.shape
        _check(lib.admm_cnn_predict_start(ctypes.c_void_p(self.handle), n, H, W,
                                          ctypes.c_void_p(_ptr(ybar, np.float32)),
                                          ctypes.c_void_p(_ptr(mask, np.uint8)), _f4(scales),
                                          ctypes.c_void_p(_ptr(x0, np.float32)), ctypes.c_void_p(_ptr(d0, np.float32)),
                                          _stream(stream)), "admm_cnn_predict_start")

    def close(self):
        if getattr(self, "handle", None):
            lib.admm_cnn_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def admm_cnn_launches() -> int:
    return int(lib.admm_cnn_launches())


def admm_deconv_set_option(option: int, value: int) -> None:
    rc = lib.admm_deconv_set_option(int(option), int(value))
    if rc != ADMM_OK:
        raise AdmmError(rc, "admm_deconv_set_option")


def admm_deconv_variants(H: int, W: int, reg="tv") -> tuple[int, int]:
    """(TV row-phase configurations of W, column-phase configurations of H)."""
    nr, nc = ctypes.c_int(), ctypes.c_int()
    _check(lib.admm_deconv_variants(int(H), int(W), _REG.get(reg, reg), ctypes.byref(nr), ctypes.byref(nc)),
           "admm_deconv_variants")
    return nr.value, nc.value


def admm_deconv_get_tuning(H: int, W: int, reg="tv", levels: int = 4) -> dict:
    t = admm_tuning_t(H=int(H), W=int(W), reg=_REG.get(reg, reg), haar_levels=int(levels))
    _check(lib.admm_deconv_get_tuning(ctypes.byref(t)), "admm_deconv_get_tuning")
    return t.as_dict()


def admm_deconv_set_tuning(cfg: dict) -> None:
    t = admm_tuning_t(**{k: cfg[k] for k, _ in admm_tuning_t._fields_ if k in cfg})
    _check(lib.admm_deconv_set_tuning(ctypes.byref(t)), "admm_deconv_set_tuning")


def admm_deconv_autotune(H: int, W: int, reg="tv", levels: int = 4, problems: int = 0, iters: int = 0,
                         stream=None) -> tuple[dict, list[dict]]:
    """Time every compiled configuration of the class on the current device
    and install the fastest; returns (best, all trials)."""
    nr, nc = admm_deconv_variants(H, W, reg)
    cap = nr * nc * 3 + 2
    trials = (admm_tuning_t * cap)()
    n = ctypes.c_int()
    best = admm_tuning_t()
    _check(lib.admm_deconv_autotune(int(H), int(W), _REG.get(reg, reg), int(levels), int(problems), int(iters),
                                    trials, cap, ctypes.byref(n), ctypes.byref(best), _stream(stream)),
           "admm_deconv_autotune")
    return best.as_dict(), [trials[i].as_dict() for i in range(min(n.value, cap))]


def tuning_cache_key(H: int, W: int, reg="tv", levels: int = 4, device_name: str = "", problems: int = 0) -> str:
    r = _REG.get(reg, reg)
    key = f"{device_name}|{int(H)}x{int(W)}|{'tv' if r == ADMM_REG_TV else 'haar'}|{0 if r == ADMM_REG_TV else int(levels) or 4}"
    return key + (f"|p{int(problems)}" if problems > 0 else "")


def autotune_cached(H: int, W: int, reg="tv", levels: int = 4, path: str | None = None, device_name: str = "",
                    retune: bool = False, problems: int = 0, stream=None) -> dict:
    """Install the configuration of the class from the JSON tuning cache at
    `path` (keyed by device name, size, regulariser, levels and, when given,
    the number of problems solved together), or autotune it (with that many
    problems per trial; 0 = enough to fill the launches) and add it to the
    cache. Returns the installed configuration, with "source": "cache" or
    "autotune" and, after a tuning run, "trials"."""
    import json
    key = tuning_cache_key(H, W, reg, levels, device_name, problems)
    cache = {}
    if path and os.path.exists(path):
        with open(path) as f:
            cache = json.load(f)
    if not retune and key in cache:
        admm_deconv_set_tuning(cache[key])
        out = admm_deconv_get_tuning(H, W, reg, levels)
        out["us_per_iter"] = cache[key].get("us_per_iter", 0.0)
        out["source"] = "cache"
        return out
    best, trials = admm_deconv_autotune(H, W, reg, levels, problems=problems, stream=stream)
    if path:
        cache[key] = best
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return dict(best, source="autotune", trials=trials)


def admm_deconv_destroy(plan: int) -> None:
    lib.admm_deconv_destroy(ctypes.c_void_p(plan))


# ---- conveniences -----------------------------------------------------------
def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(a, dtype) -> int:
    """Data pointer of a contiguous numpy array or torch tensor of `dtype`."""
    if a is None:
        return 0
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags.c_contiguous:
            raise TypeError(f"expected a C-contiguous {np.dtype(dtype).name} array")
        return a.ctypes.data
    import torch
    tmap = {np.float32: torch.float32, np.uint8: torch.uint8}
    if not isinstance(a, torch.Tensor) or a.dtype != tmap[dtype] or not a.is_contiguous():
        raise TypeError(f"expected a contiguous {tmap[dtype]} tensor")
    return a.data_ptr()


class Plan:
    """Owns one admm_plan_t. psf: 2-D array with odd sides (host)."""

    def __init__(self, H, W, psf, lam, mu1=0.0, mu2=0.0, reg="tv", levels=4, stop="iters",
                 tol=0.0, max_iters=200, check_every=1, raw_mask=False, pad=False, band_mu=None, stream=None):
        k = np.ascontiguousarray(np.asarray(psf, dtype=np.float32))
        self._psf = k
        p = admm_params_t()
        p.H, p.W = int(H), int(W)
        p.psf_h, p.psf_w = k.shape
        p.psf = k.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        p.lambda_ = float(lam)
        p.mu1, p.mu2 = float(mu1), float(mu2)
        p.reg = _REG[reg] if isinstance(reg, str) else int(reg)
        p.haar_levels = int(levels)
        p.stop = _STOP[stop] if isinstance(stop, str) else int(stop)
        p.tol = float(tol)
        p.max_iters = int(max_iters)
        p.check_every = int(check_every)
        p.raw_mask = int(bool(raw_mask))
        p.fft_pad_policy = ADMM_PAD_NEXT if pad else ADMM_PAD_EXACT
        if band_mu is not None:
            self._band_mu = np.ascontiguousarray(np.asarray(band_mu, dtype=np.float32))
            p.band_mu = self._band_mu.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        self.params = p
        self.H, self.W = p.H, p.W
        self.handle = admm_deconv_plan(p, stream)

    def domain(self) -> tuple[int, int]:
        """The domain the plan solves on (H x W, or the padded size)."""
        return admm_deconv_domain(self.handle)

    def state_size(self) -> int:
        return admm_deconv_state_size(self.handle)

    def full_state_size(self) -> int:
        return admm_deconv_full_state_size(self.handle)

    def get_full_state(self, out, stream=None) -> int:
        """Copy the complete state (full_state_size float32) into `out`;
        returns the iterations of the last solve."""
        return admm_deconv_get_full_state(self.handle, _ptr(out, np.float32), stream)

    def set_state(self, state, stream=None) -> None:
        """Resume the next solve from a state of get_full_state."""
        admm_deconv_set_state(self.handle, _ptr(state, np.float32), stream)

    def warm_start(self, x0=None, d0=None, stream=None) -> None:
        """Start the next solve from x0 (H x W) and duals d0 (state_size
        floats, admm_deconv_get_state layout); None = zeros."""
        admm_deconv_warm_start(self.handle, _ptr(x0, np.float32), _ptr(d0, np.float32), stream)

    def close(self):
        if getattr(self, "handle", None):
            admm_deconv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(plan: Plan, y, mask, x_out, stream=None) -> admm_result_t:
    """Run one solve; y/x_out float32 and mask uint8 (or None), numpy or torch, host or CUDA."""
    return admm_deconv_solve(plan.handle, _ptr(y, np.float32), _ptr(mask, np.uint8), _ptr(x_out, np.float32),
                             stream)


def solve_batch(plans: Sequence[Plan], ys, masks, x_outs, use_warmstart=False, stream=None):
    return admm_deconv_solve_batch([p.handle for p in plans], [_ptr(y, np.float32) for y in ys],
                                   None if masks is None else [_ptr(m, np.uint8) for m in masks],
                                   [_ptr(x, np.float32) for x in x_outs], use_warmstart, stream)
