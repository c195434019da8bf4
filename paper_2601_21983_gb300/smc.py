"""Python binding of libsmc (include/smc.h): the same function names, argument
marshalling only.  Host arrays are numpy arrays; device arrays are torch CUDA
tensors (passed by data pointer).  Every call raises SMCError on a non-zero
status.  There is no fallback: if libsmc.so is missing the import of the
library fails loudly.

The C calls take bare pointers and trust the caller for sizes, so the binding
checks every array before the call (dtype, host or device placement,
contiguity, element count against the context's J, D, rows, input width and
outputs, recorded by smc_init) and raises TypeError / ValueError instead of
letting the library read or write past a buffer."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsmc.so")

ABI_VERSION = 1
LAYER_DENSE, LAYER_CONV, LAYER_MAXPOOL2, LAYER_BNORM = 0, 1, 2, 3
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
N_FAMILIES = 12
FAMILIES = ["fwd_gemm", "head", "wgrad_gemm", "hidden_gemm", "leapfrog", "weights", "resample",
            "simt_net", "reduce", "fused_fwd_head", "adjoint_gemm", "hidden_wgrad_gemm"]


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
    "smc_k_gemm_bf16_batched": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_int64, C.c_void_p, C.c_int32,
                                          C.c_int64, C.c_int64, C.c_void_p, C.c_int64, C.c_int64, C.c_int64,
                                          C.c_int64, C.c_int64, C.c_int32, C.c_int32, C.c_void_p]),
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


def _numel(a):
    return int(a.size) if isinstance(a, np.ndarray) else int(a.numel())


def _arg(a, where, name, dtype, n=None, place=None, contiguous=True):
    """Pointer of argument `a` (None -> NULL) after checking it: a numpy array
    (host) or a torch tensor (host or CUDA) of dtype `dtype` (a numpy dtype,
    or "bfloat16"), C-contiguous unless told otherwise, with n elements (None:
    any), on place "host", "device" or either (None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if place == "device":
            raise TypeError(f"{where}: {name} must be a CUDA tensor, got a numpy array")
        if dtype == "bfloat16" or a.dtype != np.dtype(dtype):
            raise TypeError(f"{where}: {name} has dtype {a.dtype}, expected {np.dtype(dtype) if dtype != 'bfloat16' else dtype}")
        if contiguous and not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{where}: {name} must be C-contiguous")
        ptr = a.ctypes.data
    elif hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        import torch
        want = getattr(torch, dtype if isinstance(dtype, str) else np.dtype(dtype).name)
        if place == "device" and not a.is_cuda:
            raise TypeError(f"{where}: {name} must be a CUDA tensor")
        if place == "host" and a.is_cuda:
            raise TypeError(f"{where}: {name} must be in host memory")
        if a.dtype != want:
            raise TypeError(f"{where}: {name} has dtype {a.dtype}, expected {want}")
        if contiguous and not a.is_contiguous():
            raise ValueError(f"{where}: {name} must be contiguous")
        ptr = a.data_ptr()
    else:
        raise TypeError(f"{where}: {name} must be a numpy array or a torch tensor, got {type(a).__name__}")
    if n is not None and _numel(a) != n:
        raise ValueError(f"{where}: {name} has {_numel(a)} elements, expected {n}")
    return ptr


def _on_device(a):
    return not isinstance(a, np.ndarray) and bool(getattr(a, "is_cuda", False))


# Dimensions of every live context made by smc_init, keyed by its address:
# particles J, parameters D, training rows N, input width F, outputs C.
_CTX = {}


def _key(ctx):
    return ctx.value if isinstance(ctx, C.c_void_p) else ctx


def _dims(ctx, where):
    d = _CTX.get(_key(ctx))
    if d is None:
        raise ValueError(f"{where}: not a live context made by smc_init")
    return d


def _same(where, name, given, actual):
    if given is not None and int(given) != actual:
        raise ValueError(f"{where}: {name} = {given}, the context has {actual}")
    return actual


def _model_dims(model):
    """(input width, output width) of a model by the shape rules of its layers."""
    shp = (model.in_c, model.in_h, model.in_w)
    for i in range(model.n_layers):
        l = model.layers[i]
        if l.kind == LAYER_DENSE:
            shp = (l.n_out, 1, 1)
        elif l.kind == LAYER_CONV:
            shp = (l.n_out, shp[1] - l.ksize + 1, shp[2] - l.ksize + 1)
        elif l.kind == LAYER_MAXPOOL2:
            shp = (shp[0], shp[1] // 2, shp[2] // 2)
    return model.in_c * model.in_h * model.in_w, shp[0] * shp[1] * shp[2]


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
    """layers: list of ("dense", n_in, n_out) / ("conv", c_in, c_out, k) / ("pool2",) /
    ("bnorm", c)."""
    arr = (smc_layer * len(layers))()
    for i, l in enumerate(layers):
        if l[0] == "dense":
            arr[i] = smc_layer(LAYER_DENSE, l[1], l[2], 0)
        elif l[0] == "conv":
            arr[i] = smc_layer(LAYER_CONV, l[1], l[2], l[3])
        elif l[0] == "bnorm":
            arr[i] = smc_layer(LAYER_BNORM, l[1], l[1], 0)
        elif l[0] == "pool2":
            arr[i] = smc_layer(LAYER_MAXPOOL2, 0, 0, 0)
        else:
            raise ValueError(f"make_model: unknown layer {l!r}")
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
    """x [N][input] float32 and y (y_class int32 or y_value float32 [N]) both
    on the host (numpy) or both on the device (torch CUDA tensors)."""
    W = "smc_init"
    if cfg is None:
        raise ValueError(f"{W}: cfg is required (make_config)")
    F, Cout = _model_dims(model)
    on_dev = _on_device(x)
    place = "device" if on_dev else "host"
    if isinstance(x, np.ndarray) or hasattr(x, "data_ptr"):
        N = int(x.shape[0]) if len(x.shape) > 0 else 0
    else:
        raise TypeError(f"{W}: x must be a numpy array or a torch tensor")
    px = _arg(x, W, "x", np.float32, N * F, place)
    pyc = _arg(y_class, W, "y_class", np.int32, N, place)
    pyv = _arg(y_value, W, "y_value", np.float32, N, place)
    data = smc_data(px, pyc, pyv, N, 1 if on_dev else 0)
    ctx = C.c_void_p()
    _check(load().smc_init(C.byref(model), C.byref(data), C.byref(cfg), C.byref(ctx)), W)
    lib = load()
    _CTX[_key(ctx)] = {"J": int(cfg.n_particles), "D": int(lib.smc_num_params(ctx)), "N": N, "F": F, "C": Cout}
    return ctx


def smc_destroy(ctx):
    _CTX.pop(_key(ctx), None)
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
    pm = _arg(m, "smc_anneal_next_moments", "moments", np.float64, 4, "host")
    info = smc_anneal_info()
    _check(load().smc_anneal_next_moments(ctx, pm, C.byref(info)), "smc_anneal_next_moments", ctx)
    return info.as_dict()


def smc_set_shard(ctx, first_particle):
    _check(load().smc_set_shard(ctx, int(first_particle)), "smc_set_shard", ctx)


def smc_draw_uniforms(ctx, n):
    if int(n) < 0:
        raise ValueError(f"smc_draw_uniforms: n = {n}")
    u = np.empty(int(n), np.float64)
    _check(load().smc_draw_uniforms(ctx, int(n), _arg(u, "smc_draw_uniforms", "u", np.float64)),
           "smc_draw_uniforms", ctx)
    return u


def smc_set_weights(ctx, wn, ess):
    W = "smc_set_weights"
    w = np.ascontiguousarray(wn, np.float64)
    pw = _arg(w, W, "wn", np.float64, _dims(ctx, W)["J"], "host")
    _check(load().smc_set_weights(ctx, pw, float(ess)), W, ctx)


def smc_sda_partials(ctx):
    out = np.empty(4, np.float64)
    _check(load().smc_sda_partials(ctx, _arg(out, "smc_sda_partials", "out", np.float64)), "smc_sda_partials", ctx)
    return out


def smc_resample(ctx, force=False):
    did = C.c_int32(0)
    _check(load().smc_resample(ctx, 1 if force else 0, C.byref(did)), "smc_resample", ctx)
    return bool(did.value)


def smc_posterior_predict(ctx, x, out):
    """probs out [n][outputs] float32 of test rows x [n][input] float32; x and
    out both on the host or both on the device."""
    W = "smc_posterior_predict"
    d = _dims(ctx, W)
    on_dev = _on_device(x)
    place = "device" if on_dev else "host"
    n = int(x.shape[0])
    px = _arg(x, W, "x", np.float32, n * d["F"], place)
    po = _arg(out, W, "out", np.float32, n * d["C"], place)
    _check(load().smc_posterior_predict(ctx, px, n, 1 if on_dev else 0, po), W, ctx)
    return out


def _upload_args(ctx, W, row0, x, y_class, y_value):
    d = _dims(ctx, W)
    n = int(x.shape[0])
    if row0 < 0 or row0 + n > d["N"]:
        raise ValueError(f"{W}: rows [{row0}, {row0 + n}) outside the {d['N']} training rows")
    return (n, _arg(x, W, "x", np.float32, n * d["F"], "host"), _arg(y_class, W, "y_class", np.int32, n, "host"),
            _arg(y_value, W, "y_value", np.float32, n, "host"))


def smc_upload_rows(ctx, row0, x, y_class=None, y_value=None):
    """Replace training rows [row0, row0 + n) (annealed order) with host x
    [n][input] float32 and y [n]."""
    n, px, pyc, pyv = _upload_args(ctx, "smc_upload_rows", row0, x, y_class, y_value)
    _check(load().smc_upload_rows(ctx, row0, n, px, pyc, pyv), "smc_upload_rows", ctx)


def smc_upload_rows_async(ctx, row0, x, y_class=None, y_value=None):
    """Enqueue the rows' host-to-device copy and return at once; they take
    effect at the next smc_set_schedule / smc_anneal_next.  The caller keeps
    x / y alive (and unchanged) until then; pinned arrays copy asynchronously."""
    n, px, pyc, pyv = _upload_args(ctx, "smc_upload_rows_async", row0, x, y_class, y_value)
    _check(load().smc_upload_rows_async(ctx, row0, n, px, pyc, pyv), "smc_upload_rows_async", ctx)


def smc_get_state(ctx, J=None, D=None, theta=True):
    """Particles [J][D] float32 (None with theta=False), raw log-weights [J]
    and log pi [J]; J and D, if given, must be the context's."""
    W = "smc_get_state"
    d = _dims(ctx, W)
    J, D = _same(W, "J", J, d["J"]), _same(W, "D", D, d["D"])
    th = np.empty((J, D), np.float32) if theta else None
    lw = np.empty(J, np.float64)
    lp = np.empty(J, np.float64)
    _check(load().smc_get_state(ctx, _arg(th, W, "theta", np.float32), _arg(lw, W, "logw", np.float64),
                                _arg(lp, W, "logpi", np.float64)), W, ctx)
    return th, lw, lp


def smc_set_state(ctx, theta=None, logw=None, logpi=None):
    """Overwrite particles [J][D], log-weights [J] and / or log pi [J] (host;
    None leaves that part)."""
    W = "smc_set_state"
    d = _dims(ctx, W)
    th = None if theta is None else np.ascontiguousarray(theta, np.float32)
    lw = None if logw is None else np.ascontiguousarray(logw, np.float64)
    lp = None if logpi is None else np.ascontiguousarray(logpi, np.float64)
    args = (_arg(th, W, "theta", np.float32, d["J"] * d["D"], "host"),
            _arg(lw, W, "logw", np.float64, d["J"], "host"), _arg(lp, W, "logpi", np.float64, d["J"], "host"))
    _check(load().smc_set_state(ctx, *args), W, ctx)


def smc_set_noise(ctx, z):
    """Standard-normal momentum draws z [J][D] (host) for the next move."""
    W = "smc_set_noise"
    d = _dims(ctx, W)
    z = np.ascontiguousarray(z, np.float32)
    pz = _arg(z, W, "z", np.float32, d["J"] * d["D"], "host")
    _check(load().smc_set_noise(ctx, pz), W, ctx)


def smc_set_uniforms(ctx, u):
    u = np.ascontiguousarray(np.atleast_1d(u), np.float64)
    _check(load().smc_set_uniforms(ctx, _arg(u, "smc_set_uniforms", "u", np.float64, None, "host"), len(u)),
           "smc_set_uniforms", ctx)


def smc_eval(ctx, J=None, D=None):
    """log pi [J], log-likelihood gradient [J][D] and the two region sums [J]
    at the current particles; J and D, if given, must be the context's."""
    W = "smc_eval"
    d = _dims(ctx, W)
    J, D = _same(W, "J", J, d["J"]), _same(W, "D", D, d["D"])
    lp = np.empty(J, np.float64)
    g = np.empty((J, D), np.float32)
    la = np.empty(J, np.float64)
    lb = np.empty(J, np.float64)
    _check(load().smc_eval(ctx, _arg(lp, W, "logpi", np.float64), _arg(g, W, "grad", np.float32),
                           _arg(la, W, "la", np.float64), _arg(lb, W, "lb", np.float64)), W, ctx)
    return lp, g, la, lb


def smc_set_state_device(ctx, theta):
    """Overwrite the particles from a contiguous float32 CUDA tensor [J, D]."""
    W = "smc_set_state_device"
    d = _dims(ctx, W)
    pt = _arg(theta, W, "theta", np.float32, d["J"] * d["D"], "device")
    _check(load().smc_set_state_device(ctx, pt), W, ctx)


def smc_eval_device(ctx, logpi=None, grad=None):
    """Enqueue log pi [J] (float64) and grad log pi [J, D] (float32) of the
    current target into CUDA tensors (either may be None)."""
    W = "smc_eval_device"
    d = _dims(ctx, W)
    pl = _arg(logpi, W, "logpi", np.float64, d["J"], "device")
    pg = _arg(grad, W, "grad", np.float32, d["J"] * d["D"], "device")
    _check(load().smc_eval_device(ctx, pl, pg), W, ctx)


def smc_get_weights(ctx, J=None):
    W = "smc_get_weights"
    J = _same(W, "J", J, _dims(ctx, W)["J"])
    w = np.empty(J, np.float64)
    _check(load().smc_get_weights(ctx, _arg(w, W, "wn", np.float64)), W, ctx)
    return w


def smc_learned_params(ctx, set_params=None):
    W = "smc_learned_params"
    got = np.empty(LEARNED_NUM_PARAMS, np.float32)
    sp = None if set_params is None else np.ascontiguousarray(set_params, np.float32)
    _check(load().smc_learned_params(ctx, _arg(got, W, "get", np.float32),
                                     _arg(sp, W, "set", np.float32, LEARNED_NUM_PARAMS, "host")), W, ctx)
    return got


def smc_learned_train(ctx, epochs, lr):
    loss = C.c_double(0.0)
    _check(load().smc_learned_train(ctx, epochs, lr, C.byref(loss)), "smc_learned_train", ctx)
    return loss.value


def smc_learned_data(ctx, cap=16384):
    W = "smc_learned_data"
    n = C.c_int64(cap)
    F = np.empty((cap, 8), np.float32)
    T = np.empty((cap, 2), np.float32)
    _check(load().smc_learned_data(ctx, C.byref(n), _arg(F, W, "features", np.float32),
                                   _arg(T, W, "targets", np.float32)), W, ctx)
    k = min(cap, n.value)
    return F[:k].copy(), T[:k].copy()


def smc_learned_reset_data(ctx):
    _check(load().smc_learned_reset_data(ctx), "smc_learned_reset_data", ctx)


def smc_learned_load_data(ctx, F, T):
    W = "smc_learned_load_data"
    F = np.ascontiguousarray(F, np.float32)
    T = np.ascontiguousarray(T, np.float32)
    n = int(F.shape[0])
    pf = _arg(F, W, "features", np.float32, 8 * n, "host")
    pt = _arg(T, W, "targets", np.float32, 2 * n, "host")
    _check(load().smc_learned_load_data(ctx, pf, pt, n), W, ctx)


def smc_num_segments(ctx):
    return int(load().smc_num_segments(ctx))


def smc_learned_last(ctx, groups=1):
    W = "smc_learned_last"
    ns = smc_num_segments(ctx)
    F = np.empty((ns, 8), np.float32)
    cand = np.empty((max(groups, 1), ns + 1), np.float32)
    sc = np.empty(max(groups, 1) + 1, np.float64)
    _check(load().smc_learned_last(ctx, _arg(F, W, "features", np.float32), _arg(cand, W, "candidates", np.float32),
                                   _arg(sc, W, "scores", np.float64)), W, ctx)
    return F, cand, sc


def smc_k_learned_loss_grad(F, T, params, stream=None):
    W = "smc_k_learned_loss_grad"
    F = np.ascontiguousarray(F, np.float32)
    T = np.ascontiguousarray(T, np.float32)
    P = np.ascontiguousarray(params, np.float32)
    n = int(F.shape[0])
    g = np.empty(LEARNED_NUM_PARAMS, np.float32)
    loss = C.c_double(0.0)
    args = (_arg(F, W, "features", np.float32, 8 * n, "host"), _arg(T, W, "targets", np.float32, 2 * n, "host"), n,
            _arg(P, W, "params", np.float32, LEARNED_NUM_PARAMS, "host"), _arg(g, W, "grad", np.float32))
    _check(load().smc_k_learned_loss_grad(*args, C.byref(loss), _stream(stream)), W)
    return loss.value, g


def smc_get_permutation(ctx, N=None):
    W = "smc_get_permutation"
    N = _same(W, "N", N, _dims(ctx, W)["N"])
    p = np.empty(N, np.int32)
    _check(load().smc_get_permutation(ctx, _arg(p, W, "perm", np.int32)), W, ctx)
    return p


def smc_get_ancestors(ctx, J=None):
    W = "smc_get_ancestors"
    J = _same(W, "J", J, _dims(ctx, W)["J"])
    a = np.empty(J, np.int32)
    _check(load().smc_get_ancestors(ctx, _arg(a, W, "ancestors", np.int32)), W, ctx)
    return a


def smc_checkpoint(ctx, path):
    """Write the sampler's dynamic state to `path` (see include/smc.h)."""
    _check(load().smc_checkpoint(ctx, os.fsencode(path)), "smc_checkpoint", ctx)


def smc_restore(ctx, path):
    """Load a checkpoint into a context built with the same model, data, J, seed
    and precision."""
    _check(load().smc_restore(ctx, os.fsencode(path)), "smc_restore", ctx)


def smc_get_counters(ctx):
    W = "smc_get_counters"
    n = C.c_int64(0)
    t = np.zeros(N_FAMILIES, np.float64)
    calls = np.zeros(N_FAMILIES, np.int64)
    _check(load().smc_get_counters(ctx, C.byref(n), _arg(t, W, "ms", np.float64), N_FAMILIES,
                                   _arg(calls, W, "calls", np.int64)), W, ctx)
    return int(n.value), dict(zip(FAMILIES, t.tolist())), dict(zip(FAMILIES, calls.tolist()))


def smc_reset_counters(ctx):
    _check(load().smc_reset_counters(ctx), "smc_reset_counters", ctx)


def smc_k_normalise(logw_dev, wn_dev, ess_dev, stream=None):
    """wn [J] and ESS [1] (float64 CUDA tensors) of log-weights [J] (float64 CUDA)."""
    W = "smc_k_normalise"
    pl = _arg(logw_dev, W, "logw", np.float64, None, "device")
    J = _numel(logw_dev)
    pw = _arg(wn_dev, W, "wn", np.float64, J, "device")
    pe = _arg(ess_dev, W, "ess", np.float64, 1, "device")
    _check(load().smc_k_normalise(pl, J, pw, pe, _stream(stream)), W)


def _resample_args(W, wn_dev, kind, u, anc_dev, J):
    pw = _arg(wn_dev, W, "wn", np.float64, None, "device")
    J = _numel(wn_dev) if J is None else int(J)
    if J < 0 or J > _numel(wn_dev):
        raise ValueError(f"{W}: J = {J} for {_numel(wn_dev)} weights")
    u = np.ascontiguousarray(np.atleast_1d(u), np.float64)
    need = 1 if kind == RESAMPLE_SYSTEMATIC else J
    if len(u) < need:
        raise ValueError(f"{W}: {len(u)} uniforms, the resampler reads {need}")
    pu = _arg(u, W, "u", np.float64, None, "host")
    pa = _arg(anc_dev, W, "ancestors", np.int32, None, "device")
    if _numel(anc_dev) < J:
        raise ValueError(f"{W}: ancestors has {_numel(anc_dev)} elements, expected {J}")
    return pw, J, pu, pa, u


def smc_k_resample(wn_dev, kind, u, anc_dev, stream=None):
    """Ancestors [J] (int32 CUDA) from normalised weights [J] (float64 CUDA)
    and host uniforms (1 for systematic, J for multinomial)."""
    W = "smc_k_resample"
    pw, J, pu, pa, _keep = _resample_args(W, wn_dev, kind, u, anc_dev, None)
    _check(load().smc_k_resample(pw, J, kind, pu, pa, _stream(stream)), W)


def smc_k_resample_noalloc(wn_dev, kind, u, anc_dev, stream=None, J=None):
    W = "smc_k_resample_noalloc"
    pw, n, pu, pa, _keep = _resample_args(W, wn_dev, kind, u, anc_dev, J)
    st = load().smc_k_resample_noalloc(pw, n, kind, pu, pa, _stream(stream))
    if st != 0:
        raise SMCError(st, W, (load().smc_last_error(None) or b"").decode())


def smc_k_philox_normals(seed, stream_id, iteration, offset, out_dev, stream=None):
    W = "smc_k_philox_normals"
    po = _arg(out_dev, W, "out", np.float32, None, "device")
    _check(load().smc_k_philox_normals(seed, stream_id, iteration, offset, _numel(out_dev), po, _stream(stream)), W)


def smc_k_philox_u32(k0, k1, c2, c3, out_dev, stream=None):
    """Raw Philox4x32-10 blocks into out_dev [n][4] (int32 CUDA tensor, read as u32)."""
    W = "smc_k_philox_u32"
    if len(out_dev.shape) != 2 or out_dev.shape[1] != 4:
        raise ValueError(f"{W}: out must be [n][4], got {tuple(out_dev.shape)}")
    po = _arg(out_dev, W, "out", np.int32, None, "device")
    _check(load().smc_k_philox_u32(k0, k1, c2, c3, out_dev.shape[0], po, _stream(stream)), W)


def smc_k_gemm_bf16(A, B, Cout, accumulate=False, stream=None):
    """A [M][K], B [N][K] BF16 and Cout [M][N] FP32 device tensors with unit
    inner stride (row pitches may exceed the logical width)."""
    W = "smc_k_gemm_bf16"
    for t, name, dt in ((A, "A", "bfloat16"), (B, "B", "bfloat16"), (Cout, "Cout", np.float32)):
        _arg(t, W, name, dt, None, "device", contiguous=False)
        if len(t.shape) != 2 or t.stride(1) != 1:
            raise ValueError(f"{W}: {name} must be a 2-D tensor with unit inner stride")
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K or tuple(Cout.shape) != (M, N):
        raise ValueError(f"{W}: shapes A {tuple(A.shape)}, B {tuple(B.shape)}, Cout {tuple(Cout.shape)} do not match")
    _check(load().smc_k_gemm_bf16(A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), Cout.data_ptr(),
                                  Cout.stride(0), M, N, K, 1 if accumulate else 0, _stream(stream)), W)


def smc_k_gemm_bf16_batched(A, a_layout, B, b_layout, Cout, c_layout, M, N, K, batch, accumulate=False,
                            stream=None):
    """C_b[m][n] = sum_k A_b[m][k] B_b[n][k] for b < batch.  A, B: BF16 device
    tensors; Cout: FP32 device tensor.  a_layout = (mn_major, ld, bstride) in
    elements (element (m, k) of A_b at b bstride + (k ld + m if mn_major else
    m ld + k)); b_layout likewise for (n, k); c_layout = (ldc, c_bstride).  Every
    element the call may touch must lie inside its tensor."""
    W = "smc_k_gemm_bf16_batched"
    for t, name, dt in ((A, "A", "bfloat16"), (B, "B", "bfloat16"), (Cout, "Cout", np.float32)):
        _arg(t, W, name, dt, None, "device", contiguous=False)
        if not t.is_contiguous():
            raise ValueError(f"{W}: {name} must be contiguous")

    def last(layout, rows):
        mn, ld, bs = layout
        return (batch - 1) * bs + ((K - 1) * ld + rows - 1 if mn else (rows - 1) * ld + K - 1)
    if last(a_layout, M) >= A.numel() or last(b_layout, N) >= B.numel():
        raise ValueError(f"{W}: the layout reaches past an operand")
    ldc, cbs = c_layout
    if (batch - 1) * cbs + (M - 1) * ldc + N - 1 >= Cout.numel():
        raise ValueError(f"{W}: the layout reaches past Cout")
    _check(load().smc_k_gemm_bf16_batched(A.data_ptr(), int(a_layout[0]), a_layout[1], a_layout[2],
                                          B.data_ptr(), int(b_layout[0]), b_layout[1], b_layout[2],
                                          Cout.data_ptr(), ldc, cbs, M, N, K, batch, 1 if accumulate else 0,
                                          _stream(stream)), W)


def smc_k_wait_probe(limit_ms, arrive, stream=None):
    """Bounded device wait on an mbarrier (completed by the kernel only when
    `arrive`); raises SMCError(SMC_ETIMEOUT) when the wait gives up."""
    _check(load().smc_k_wait_probe(float(limit_ms), 1 if arrive else 0, _stream(stream)), "smc_k_wait_probe")
