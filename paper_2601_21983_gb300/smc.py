"""Python binding of libsmc (include/smc.h): the same function names, argument
marshalling only.  Host arrays are numpy arrays; device arrays are torch CUDA
tensors (passed by data pointer).  Every call raises SMCError on a non-zero
status.  There is no fallback: if libsmc.so is missing the import of the
library fails loudly."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsmc.so")

ABI_VERSION = 1
LAYER_DENSE, LAYER_CONV, LAYER_MAXPOOL2 = 0, 1, 2
ACT_TANH, ACT_RELU, ACT_IDENTITY = 0, 1, 2
LIK_CATEGORICAL, LIK_GAUSSIAN = 0, 1
PREC_FP32, PREC_BF16 = 0, 1
RESAMPLE_SYSTEMATIC, RESAMPLE_MULTINOMIAL = 0, 1
SCHED = {"constant": 0, "fb": 1, "ctr": 2, "linear": 3, "automated": 4, "sda": 5, "constant_fresh": 6,
         "ctr_fresh": 7}
PROPOSAL_PLAIN, PROPOSAL_LEARNED, PROPOSAL_EXPLORE = 0, 1, 2
LEARNED_NUM_PARAMS = 706
STATUS = {0: "SMC_OK", 1: "SMC_EINVAL", 2: "SMC_ENOMEM", 3: "SMC_ECUDA", 4: "SMC_ESTATE",
          5: "SMC_ENUMERIC", 6: "SMC_ETIMEOUT", 7: "SMC_EUNSUPPORTED"}
N_FAMILIES = 10
FAMILIES = ["fwd_gemm", "head", "wgrad_gemm", "hidden_gemm", "leapfrog", "weights", "resample",
            "simt_net", "reduce", "fused_fwd_head"]


class SMCError(RuntimeError):
    def __init__(self, status, where, detail=""):
        super().__init__(f"{where}: {STATUS.get(status, status)} {detail}".strip())
        self.status = status


class smc_layer(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_in", C.c_int32), ("n_out", C.c_int32), ("ksize", C.c_int32)]


class smc_model(C.Structure):
    _fields_ = [("version", C.c_int32), ("n_layers", C.c_int32), ("layers", C.POINTER(smc_layer)),
                ("in_c", C.c_int32), ("in_h", C.c_int32), ("in_w", C.c_int32),
                ("activation", C.c_int32), ("likelihood", C.c_int32),
                ("prior_sigma", C.c_double), ("noise_sigma", C.c_double)]


class smc_data(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y_class", C.c_void_p), ("y_value", C.c_void_p),
                ("n", C.c_int64), ("on_device", C.c_int32)]


class smc_config(C.Structure):
    _fields_ = [("version", C.c_int32), ("n_particles", C.c_int32), ("seed", C.c_uint64),
                ("precision", C.c_int32), ("resampler", C.c_int32), ("scaled", C.c_int32),
                ("chunk_rows", C.c_int64), ("stream", C.c_void_p), ("timing", C.c_int32)]


class smc_schedule(C.Structure):
    _fields_ = [("kind", C.c_int32), ("C", C.c_int64), ("kappa", C.c_int64), ("K", C.c_int32),
                ("k_start", C.c_int32), ("beta0", C.c_double), ("beta_reinit", C.c_double),
                ("delta_s", C.c_double)]


class smc_step_params(C.Structure):
    _fields_ = [("h", C.c_double), ("S", C.c_int32), ("proposal", C.c_int32), ("groups", C.c_int32),
                ("pad_", C.c_int32), ("explore_sigma", C.c_double)]


class smc_step_stats(C.Structure):
    _fields_ = [("ess", C.c_double), ("mean_logpi", C.c_double), ("beta", C.c_double),
                ("rows", C.c_int64), ("k", C.c_int32), ("n_nonfinite", C.c_int32),
                ("grad_evals", C.c_int32), ("proposal_used", C.c_int32), ("h_used", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad_"}


class smc_anneal_info(C.Structure):
    _fields_ = [("appended", C.c_int32), ("k", C.c_int32), ("rows", C.c_int64),
                ("rows_full", C.c_int64), ("beta", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None

_SIGS = {
    "smc_init": (C.c_int, [C.POINTER(smc_model), C.POINTER(smc_data), C.POINTER(smc_config), C.POINTER(C.c_void_p)]),
    "smc_destroy": (None, [C.c_void_p]),
    "smc_status_string": (C.c_char_p, [C.c_int]),
    "smc_last_error": (C.c_char_p, [C.c_void_p]),
    "smc_num_params": (C.c_int64, [C.c_void_p]),
    "smc_set_schedule": (C.c_int, [C.c_void_p, C.POINTER(smc_schedule), C.POINTER(smc_step_stats)]),
    "smc_step": (C.c_int, [C.c_void_p, C.POINTER(smc_step_params), C.POINTER(smc_step_stats)]),
    "smc_anneal_next": (C.c_int, [C.c_void_p, C.POINTER(smc_anneal_info)]),
    "smc_resample": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    "smc_posterior_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p]),
    "smc_upload_rows": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "smc_upload_rows_async": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "smc_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "smc_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "smc_set_noise": (C.c_int, [C.c_void_p, C.c_void_p]),
    "smc_set_uniforms": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "smc_eval": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "smc_set_state_device": (C.c_int, [C.c_void_p, C.c_void_p]),
    "smc_eval_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "smc_get_weights": (C.c_int, [C.c_void_p, C.c_void_p]),
    "smc_get_permutation": (C.c_int, [C.c_void_p, C.c_void_p]),
    "smc_get_ancestors": (C.c_int, [C.c_void_p, C.c_void_p]),
    "smc_set_shard": (C.c_int, [C.c_void_p, C.c_int64]),
    "smc_draw_uniforms": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "smc_set_weights": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double]),
    "smc_sda_partials": (C.c_int, [C.c_void_p, C.c_void_p]),
    "smc_anneal_next_moments": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(smc_anneal_info)]),
    "smc_checkpoint": (C.c_int, [C.c_void_p, C.c_char_p]),
    "smc_restore": (C.c_int, [C.c_void_p, C.c_char_p]),
    "smc_get_counters": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.c_void_p, C.c_int32, C.c_void_p]),
    "smc_reset_counters": (C.c_int, [C.c_void_p]),
    "smc_learned_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "smc_learned_train": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.POINTER(C.c_double)]),
    "smc_learned_data": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.c_void_p, C.c_void_p]),
    "smc_learned_reset_data": (C.c_int, [C.c_void_p]),
    "smc_learned_load_data": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]),
    "smc_learned_last": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "smc_num_segments": (C.c_int32, [C.c_void_p]),
    "smc_k_learned_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                          C.POINTER(C.c_double), C.c_void_p]),
    "smc_k_normalise": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "smc_k_resample": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "smc_k_resample_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "smc_k_philox_normals": (C.c_int, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64, C.c_int64, C.c_void_p,
                                       C.c_void_p]),
    "smc_k_philox_u32": (C.c_int, [C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int64, C.c_void_p,
                                   C.c_void_p]),
    "smc_k_wait_probe": (C.c_int, [C.c_double, C.c_int32, C.c_void_p]),
    "smc_k_gemm_bf16": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                  C.c_int64, C.c_int64, C.c_int64, C.c_int32, C.c_void_p]),
}
EXPORTED = sorted(_SIGS)


def load():
    """Load libsmc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(a):
    """Pointer of a numpy array (host) or torch tensor (device); None -> NULL."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "host arrays must be C-contiguous"
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "device tensors must be contiguous"
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(type(a))


def _stream(s):
    if s is None:
        return None
    return s.cuda_stream if hasattr(s, "cuda_stream") else int(s)


def _check(status, where, ctx=None):
    if status != 0:
        detail = ""
        if ctx is not None:
            detail = (load().smc_last_error(ctx) or b"").decode()
        raise SMCError(status, where, detail)


# -------------------------------------------------------------- structs
def make_model(layers, in_shape, activation=ACT_TANH, likelihood=LIK_CATEGORICAL, prior_sigma=1.0,
               noise_sigma=1.0):
    """layers: list of ("dense", n_in, n_out) / ("conv", c_in, c_out, k) / ("pool2",)."""
    arr = (smc_layer * len(layers))()
    for i, l in enumerate(layers):
        if l[0] == "dense":
            arr[i] = smc_layer(LAYER_DENSE, l[1], l[2], 0)
        elif l[0] == "conv":
            arr[i] = smc_layer(LAYER_CONV, l[1], l[2], l[3])
        else:
            arr[i] = smc_layer(LAYER_MAXPOOL2, 0, 0, 0)
    shp = tuple(in_shape) + (1,) * (3 - len(in_shape))
    m = smc_model(ABI_VERSION, len(layers), arr, shp[0], shp[1], shp[2], activation, likelihood,
                  prior_sigma, noise_sigma)
    m._keep = arr
    return m


def make_config(J, seed, precision=PREC_FP32, resampler=RESAMPLE_SYSTEMATIC, scaled=1, chunk_rows=0,
                stream=None, timing=0):
    return smc_config(ABI_VERSION, J, seed, precision, resampler, scaled, chunk_rows, _stream(stream), timing)


def make_schedule(kind, C_, kappa, K, k_start=0, beta0=0.1, beta_reinit=0.1, delta_s=1.0):
    return smc_schedule(SCHED[kind] if isinstance(kind, str) else kind, C_, kappa, K, k_start, beta0,
                        beta_reinit, delta_s)


# ------------------------------------------------------------ functions
def smc_init(model, x, y_class=None, y_value=None, cfg=None):
    """x / y on the host (numpy) or the device (torch CUDA tensors)."""
    on_dev = not isinstance(x, np.ndarray)
    data = smc_data(_ptr(x), _ptr(y_class), _ptr(y_value), x.shape[0], 1 if on_dev else 0)
    ctx = C.c_void_p()
    _check(load().smc_init(C.byref(model), C.byref(data), C.byref(cfg), C.byref(ctx)), "smc_init")
    return ctx


def smc_destroy(ctx):
    load().smc_destroy(ctx)


def smc_num_params(ctx):
    return int(load().smc_num_params(ctx))


def smc_set_schedule(ctx, sched):
    st = smc_step_stats()
    _check(load().smc_set_schedule(ctx, C.byref(sched), C.byref(st)), "smc_set_schedule", ctx)
    return st.as_dict()


def smc_step(ctx, h, S, proposal=PROPOSAL_PLAIN, groups=0, explore_sigma=0.0):
    st = smc_step_stats()
    p = smc_step_params(h, S, proposal, groups, 0, explore_sigma)
    _check(load().smc_step(ctx, C.byref(p), C.byref(st)), "smc_step", ctx)
    return st.as_dict()


def smc_anneal_next(ctx):
    info = smc_anneal_info()
    _check(load().smc_anneal_next(ctx, C.byref(info)), "smc_anneal_next", ctx)
    return info.as_dict()


def smc_anneal_next_moments(ctx, moments):
    m = np.ascontiguousarray(moments, np.float64)
    assert m.shape == (4,)
    info = smc_anneal_info()
    _check(load().smc_anneal_next_moments(ctx, _ptr(m), C.byref(info)), "smc_anneal_next_moments", ctx)
    return info.as_dict()


def smc_set_shard(ctx, first_particle):
    _check(load().smc_set_shard(ctx, int(first_particle)), "smc_set_shard", ctx)


def smc_draw_uniforms(ctx, n):
    u = np.empty(int(n), np.float64)
    _check(load().smc_draw_uniforms(ctx, int(n), _ptr(u)), "smc_draw_uniforms", ctx)
    return u


def smc_set_weights(ctx, wn, ess):
    w = np.ascontiguousarray(wn, np.float64)
    _check(load().smc_set_weights(ctx, _ptr(w), float(ess)), "smc_set_weights", ctx)


def smc_sda_partials(ctx):
    out = np.empty(4, np.float64)
    _check(load().smc_sda_partials(ctx, _ptr(out)), "smc_sda_partials", ctx)
    return out


def smc_resample(ctx, force=False):
    did = C.c_int32(0)
    _check(load().smc_resample(ctx, 1 if force else 0, C.byref(did)), "smc_resample", ctx)
    return bool(did.value)


def smc_posterior_predict(ctx, x, out):
    on_dev = 0 if isinstance(x, np.ndarray) else 1
    _check(load().smc_posterior_predict(ctx, _ptr(x), x.shape[0], on_dev, _ptr(out)), "smc_posterior_predict", ctx)
    return out


def smc_upload_rows(ctx, row0, x, y_class=None, y_value=None):
    _check(load().smc_upload_rows(ctx, row0, x.shape[0], _ptr(x), _ptr(y_class), _ptr(y_value)),
           "smc_upload_rows", ctx)


def smc_upload_rows_async(ctx, row0, x, y_class=None, y_value=None):
    """Enqueue the rows' host-to-device copy and return at once; they take
    effect at the next smc_set_schedule / smc_anneal_next.  The caller keeps
    x / y alive (and unchanged) until then; pinned arrays copy asynchronously."""
    _check(load().smc_upload_rows_async(ctx, row0, x.shape[0], _ptr(x), _ptr(y_class), _ptr(y_value)),
           "smc_upload_rows_async", ctx)


def smc_get_state(ctx, J, D, theta=True):
    th = np.empty((J, D), np.float32) if theta else None
    lw = np.empty(J, np.float64)
    lp = np.empty(J, np.float64)
    _check(load().smc_get_state(ctx, _ptr(th), _ptr(lw), _ptr(lp)), "smc_get_state", ctx)
    return th, lw, lp


def smc_set_state(ctx, theta=None, logw=None, logpi=None):
    th = None if theta is None else np.ascontiguousarray(theta, np.float32)
    lw = None if logw is None else np.ascontiguousarray(logw, np.float64)
    lp = None if logpi is None else np.ascontiguousarray(logpi, np.float64)
    _check(load().smc_set_state(ctx, _ptr(th), _ptr(lw), _ptr(lp)), "smc_set_state", ctx)


def smc_set_noise(ctx, z):
    z = np.ascontiguousarray(z, np.float32)
    _check(load().smc_set_noise(ctx, _ptr(z)), "smc_set_noise", ctx)


def smc_set_uniforms(ctx, u):
    u = np.ascontiguousarray(np.atleast_1d(u), np.float64)
    _check(load().smc_set_uniforms(ctx, _ptr(u), len(u)), "smc_set_uniforms", ctx)


def smc_eval(ctx, J, D):
    lp = np.empty(J, np.float64)
    g = np.empty((J, D), np.float32)
    la = np.empty(J, np.float64)
    lb = np.empty(J, np.float64)
    _check(load().smc_eval(ctx, _ptr(lp), _ptr(g), _ptr(la), _ptr(lb)), "smc_eval", ctx)
    return lp, g, la, lb


def smc_set_state_device(ctx, theta):
    """Overwrite the particles from a contiguous float32 CUDA tensor [J, D]."""
    _check(load().smc_set_state_device(ctx, _ptr(theta)), "smc_set_state_device", ctx)


def smc_eval_device(ctx, logpi=None, grad=None):
    """Enqueue log pi [J] (float64) and grad log pi [J, D] (float32) of the
    current target into CUDA tensors (either may be None)."""
    _check(load().smc_eval_device(ctx, _ptr(logpi), _ptr(grad)), "smc_eval_device", ctx)


def smc_get_weights(ctx, J):
    w = np.empty(J, np.float64)
    _check(load().smc_get_weights(ctx, _ptr(w)), "smc_get_weights", ctx)
    return w


def smc_learned_params(ctx, set_params=None):
    got = np.empty(LEARNED_NUM_PARAMS, np.float32)
    sp = None if set_params is None else np.ascontiguousarray(set_params, np.float32)
    _check(load().smc_learned_params(ctx, _ptr(got), _ptr(sp)), "smc_learned_params", ctx)
    return got


def smc_learned_train(ctx, epochs, lr):
    loss = C.c_double(0.0)
    _check(load().smc_learned_train(ctx, epochs, lr, C.byref(loss)), "smc_learned_train", ctx)
    return loss.value


def smc_learned_data(ctx, cap=16384):
    n = C.c_int64(cap)
    F = np.empty((cap, 8), np.float32)
    T = np.empty((cap, 2), np.float32)
    _check(load().smc_learned_data(ctx, C.byref(n), _ptr(F), _ptr(T)), "smc_learned_data", ctx)
    k = min(cap, n.value)
    return F[:k].copy(), T[:k].copy()


def smc_learned_reset_data(ctx):
    _check(load().smc_learned_reset_data(ctx), "smc_learned_reset_data", ctx)


def smc_learned_load_data(ctx, F, T):
    F = np.ascontiguousarray(F, np.float32)
    T = np.ascontiguousarray(T, np.float32)
    _check(load().smc_learned_load_data(ctx, _ptr(F), _ptr(T), F.shape[0]), "smc_learned_load_data", ctx)


def smc_num_segments(ctx):
    return int(load().smc_num_segments(ctx))


def smc_learned_last(ctx, groups=1):
    ns = smc_num_segments(ctx)
    F = np.empty((ns, 8), np.float32)
    cand = np.empty((max(groups, 1), ns + 1), np.float32)
    sc = np.empty(max(groups, 1) + 1, np.float64)
    _check(load().smc_learned_last(ctx, _ptr(F), _ptr(cand), _ptr(sc)), "smc_learned_last", ctx)
    return F, cand, sc


def smc_k_learned_loss_grad(F, T, params, stream=None):
    F = np.ascontiguousarray(F, np.float32)
    T = np.ascontiguousarray(T, np.float32)
    P = np.ascontiguousarray(params, np.float32)
    g = np.empty(LEARNED_NUM_PARAMS, np.float32)
    loss = C.c_double(0.0)
    _check(load().smc_k_learned_loss_grad(_ptr(F), _ptr(T), F.shape[0], _ptr(P), _ptr(g), C.byref(loss),
                                          _stream(stream)), "smc_k_learned_loss_grad")
    return loss.value, g


def smc_get_permutation(ctx, N):
    p = np.empty(N, np.int32)
    _check(load().smc_get_permutation(ctx, _ptr(p)), "smc_get_permutation", ctx)
    return p


def smc_get_ancestors(ctx, J):
    a = np.empty(J, np.int32)
    _check(load().smc_get_ancestors(ctx, _ptr(a)), "smc_get_ancestors", ctx)
    return a


def smc_checkpoint(ctx, path):
    """Write the sampler's dynamic state to `path` (see include/smc.h)."""
    _check(load().smc_checkpoint(ctx, os.fsencode(path)), "smc_checkpoint", ctx)


def smc_restore(ctx, path):
    """Load a checkpoint into a context built with the same model, data, J, seed
    and precision."""
    _check(load().smc_restore(ctx, os.fsencode(path)), "smc_restore", ctx)


def smc_get_counters(ctx):
    n = C.c_int64(0)
    t = np.zeros(N_FAMILIES, np.float64)
    calls = np.zeros(N_FAMILIES, np.int64)
    _check(load().smc_get_counters(ctx, C.byref(n), _ptr(t), N_FAMILIES, _ptr(calls)), "smc_get_counters", ctx)
    return int(n.value), dict(zip(FAMILIES, t.tolist())), dict(zip(FAMILIES, calls.tolist()))


def smc_reset_counters(ctx):
    _check(load().smc_reset_counters(ctx), "smc_reset_counters", ctx)


def smc_k_normalise(logw_dev, wn_dev, ess_dev, stream=None):
    _check(load().smc_k_normalise(_ptr(logw_dev), logw_dev.numel(), _ptr(wn_dev), _ptr(ess_dev), _stream(stream)),
           "smc_k_normalise")


def smc_k_resample(wn_dev, kind, u, anc_dev, stream=None):
    u = np.ascontiguousarray(np.atleast_1d(u), np.float64)
    _check(load().smc_k_resample(_ptr(wn_dev), wn_dev.numel(), kind, _ptr(u), _ptr(anc_dev), _stream(stream)),
           "smc_k_resample")


def smc_k_resample_noalloc(wn_dev, kind, u, anc_dev, stream=None, J=None):
    u = np.ascontiguousarray(np.atleast_1d(u), np.float64)
    n = wn_dev.numel() if J is None else J
    st = load().smc_k_resample_noalloc(_ptr(wn_dev), n, kind, _ptr(u), _ptr(anc_dev), _stream(stream))
    if st != 0:
        raise SMCError(st, "smc_k_resample_noalloc", (load().smc_last_error(None) or b"").decode())


def smc_k_philox_normals(seed, stream_id, iteration, offset, out_dev, stream=None):
    _check(load().smc_k_philox_normals(seed, stream_id, iteration, offset, out_dev.numel(), _ptr(out_dev),
                                       _stream(stream)), "smc_k_philox_normals")


def smc_k_philox_u32(k0, k1, c2, c3, out_dev, stream=None):
    _check(load().smc_k_philox_u32(k0, k1, c2, c3, out_dev.shape[0], _ptr(out_dev), _stream(stream)),
           "smc_k_philox_u32")


def smc_k_gemm_bf16(A, B, Cout, accumulate=False, stream=None):
    """A [M][K], B [N][K] BF16 and Cout [M][N] FP32 device tensors with unit
    inner stride (row pitches may exceed the logical width)."""
    M, K = A.shape
    N = B.shape[0]
    assert A.stride(1) == 1 and B.stride(1) == 1 and Cout.stride(1) == 1
    _check(load().smc_k_gemm_bf16(A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), Cout.data_ptr(),
                                  Cout.stride(0), M, N, K, 1 if accumulate else 0, _stream(stream)),
           "smc_k_gemm_bf16")


def smc_k_wait_probe(limit_ms, arrive, stream=None):
    """Bounded device wait on an mbarrier (completed by the kernel only when
    `arrive`); raises SMCError(SMC_ETIMEOUT) when the wait gives up."""
    _check(load().smc_k_wait_probe(float(limit_ms), 1 if arrive else 0, _stream(stream)), "smc_k_wait_probe")
