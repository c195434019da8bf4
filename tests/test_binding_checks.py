"""CPU tests of the Python binding's argument checks (no GPU, no library call):
every array handed to the C ABI is checked for dtype, host / device
placement, contiguity and element count against the context's dimensions,
and a bad one raises TypeError / ValueError before any C function runs.  The
library is replaced by a recorder, so the tests also see that well-formed
arguments do reach the C call."""
import ctypes as C

import numpy as np
import pytest

from oracle import nn
from paper_2601_21983_gb300 import smc as S

torch = pytest.importorskip("torch")

DIMS = {"J": 4, "D": 10, "N": 50, "F": 16, "C": 3}


class _Recorder:
    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def call(*args):
            self.calls.append(name)
            return 0
        return call


@pytest.fixture
def lib(monkeypatch):
    rec = _Recorder()
    monkeypatch.setattr(S, "_lib", rec)
    monkeypatch.setitem(S._CTX, 4242, dict(DIMS))
    return rec


CTX = C.c_void_p(4242)
f32, f64, i32 = np.float32, np.float64, np.int32


BAD = {
    "theta rows": (lambda: S.smc_set_state(CTX, np.zeros((3, 10), f32)), ValueError),
    "logw length": (lambda: S.smc_set_state(CTX, logw=np.zeros(5)), ValueError),
    "get_state J": (lambda: S.smc_get_state(CTX, 5, 10), ValueError),
    "eval D": (lambda: S.smc_eval(CTX, 4, 11), ValueError),
    "weights J": (lambda: S.smc_get_weights(CTX, 3), ValueError),
    "ancestors J": (lambda: S.smc_get_ancestors(CTX, 8), ValueError),
    "permutation N": (lambda: S.smc_get_permutation(CTX, 49), ValueError),
    "noise size": (lambda: S.smc_set_noise(CTX, np.zeros((4, 9), f32)), ValueError),
    "set_weights J": (lambda: S.smc_set_weights(CTX, np.ones(3), 3.0), ValueError),
    "moments": (lambda: S.smc_anneal_next_moments(CTX, [1.0, 2.0, 3.0]), ValueError),
    "predict out size": (lambda: S.smc_posterior_predict(CTX, np.zeros((7, 16), f32), np.zeros((7, 2), f32)),
                         ValueError),
    "predict x width": (lambda: S.smc_posterior_predict(CTX, np.zeros((7, 15), f32), np.zeros((7, 3), f32)),
                        ValueError),
    "predict x dtype": (lambda: S.smc_posterior_predict(CTX, np.zeros((7, 16), f64), np.zeros((7, 3), f32)),
                        TypeError),
    "predict out not contiguous": (
        lambda: S.smc_posterior_predict(CTX, np.zeros((7, 16), f32), np.zeros((3, 7), f32).T), ValueError),
    "upload range": (lambda: S.smc_upload_rows(CTX, 45, np.zeros((10, 16), f32), np.zeros(10, i32)), ValueError),
    "upload label dtype": (lambda: S.smc_upload_rows(CTX, 0, np.zeros((10, 16), f32), np.zeros(10, np.int64)),
                           TypeError),
    "upload label count": (lambda: S.smc_upload_rows_async(CTX, 0, np.zeros((10, 16), f32), np.zeros(9, i32)),
                           ValueError),
    "device state from host": (lambda: S.smc_set_state_device(CTX, np.zeros((4, 10), f32)), TypeError),
    "device state from a CPU tensor": (lambda: S.smc_set_state_device(CTX, torch.zeros(4, 10)), TypeError),
    "device eval dtype": (lambda: S.smc_eval_device(CTX, torch.zeros(4, dtype=torch.float32)), TypeError),
    "learned params size": (lambda: S.smc_learned_params(CTX, np.zeros(10, f32)), ValueError),
    "learned data shapes": (lambda: S.smc_learned_load_data(CTX, np.zeros((5, 8), f32), np.zeros((4, 2), f32)),
                            ValueError),
    "unknown context": (lambda: S.smc_get_state(C.c_void_p(999), 4, 10), ValueError),
    "normalise on host": (lambda: S.smc_k_normalise(np.zeros(4), np.zeros(4), np.zeros(1)), TypeError),
    "resample on a CPU tensor": (
        lambda: S.smc_k_resample(torch.zeros(4, dtype=torch.float64), S.RESAMPLE_SYSTEMATIC, [0.5],
                                 torch.zeros(4, dtype=torch.int32)), TypeError),
    "gemm on CPU tensors": (
        lambda: S.smc_k_gemm_bf16(torch.zeros(4, 8, dtype=torch.bfloat16), torch.zeros(4, 8, dtype=torch.bfloat16),
                                  torch.zeros(4, 4)), TypeError),
    "not an array": (lambda: S.smc_set_noise(CTX, object()), TypeError),
}


@pytest.mark.parametrize("case", sorted(BAD))
def test_bad_arguments_raise_before_the_c_call(lib, case):
    fn, exc = BAD[case]
    with pytest.raises(exc):
        fn()
    assert lib.calls == [], f"{case}: reached {lib.calls}"


def test_well_formed_arguments_reach_the_c_call(lib):
    S.smc_set_state(CTX, np.zeros((4, 10)), np.zeros(4), np.zeros(4))   # float64 theta is converted
    S.smc_set_noise(CTX, np.zeros(40))                                    # any shape with J x D elements
    S.smc_get_state(CTX)
    S.smc_eval(CTX, 4, 10)
    S.smc_posterior_predict(CTX, np.zeros((7, 4, 4), f32), np.zeros((7, 3), f32))
    S.smc_upload_rows(CTX, 40, np.zeros((10, 16), f32), np.zeros(10, i32))
    S.smc_set_weights(CTX, np.full(4, 0.25), 4.0)
    assert lib.calls == ["smc_set_state", "smc_set_noise", "smc_get_state", "smc_eval", "smc_posterior_predict",
                         "smc_upload_rows", "smc_set_weights"]


def test_destroy_forgets_the_context(lib):
    S.smc_destroy(CTX)
    assert lib.calls == ["smc_destroy"]
    with pytest.raises(ValueError):
        S.smc_get_state(CTX)


def test_init_checks_data_against_the_model(lib):
    model = S.make_model([("dense", 16, 8), ("dense", 8, 3)], (16,), S.ACT_TANH)
    cfg = S.make_config(4, 1)
    with pytest.raises(TypeError):
        S.smc_init(model, np.zeros((20, 16), f64), y_class=np.zeros(20, i32), cfg=cfg)
    with pytest.raises(ValueError):
        S.smc_init(model, np.zeros((20, 15), f32), y_class=np.zeros(20, i32), cfg=cfg)
    with pytest.raises(ValueError):
        S.smc_init(model, np.zeros((20, 16), f32), y_class=np.zeros(19, i32), cfg=cfg)
    with pytest.raises(TypeError):
        S.smc_init(model, np.zeros((20, 16), f32), y_class=np.zeros(20, np.int64), cfg=cfg)
    with pytest.raises(ValueError):
        S.smc_init(model, np.zeros((20, 16), f32), y_class=np.zeros(20, i32))
    assert lib.calls == []


@pytest.mark.parametrize("layers,shape", [
    ([("dense", 784, 100), ("dense", 100, 10)], (784,)),
    ([("conv", 3, 16, 5), ("pool2",), ("conv", 16, 32, 5), ("pool2",), ("dense", 800, 10)], (3, 32, 32)),
    ([("conv", 1, 6, 5), ("pool2",), ("conv", 6, 16, 5), ("pool2",), ("dense", 400, 120), ("dense", 120, 84),
      ("dense", 84, 10)], (1, 32, 32)),
    ([("conv", 3, 4, 3), ("pool2",), ("conv", 4, 3, 3), ("dense", 12, 5)], (3, 10, 10)),
    ([("conv", 2, 3, 3), ("pool2",)], (2, 9, 7)),
    ([("conv", 1, 8, 3), ("bnorm", 8), ("pool2",), ("conv", 8, 16, 3), ("bnorm", 16), ("pool2",),
      ("dense", 400, 232), ("dense", 232, 10)], (1, 28, 28)),
])
def test_model_dims_follow_the_layer_shape_rules(layers, shape):
    """Input and output widths the binding derives from the C model struct
    equal those of the oracle's network description."""
    spec = nn.Spec(layers, shape, nn.TANH)
    model = S.make_model(layers, shape, S.ACT_TANH)
    assert S._model_dims(model) == (int(np.prod(shape)), spec.out_dim)
