"""CPU checks of the C ABI boundary: libsmc.so builds, loads without a GPU and
exports every function include/smc.h declares; the Python binding covers the
same names.  No compute call is made here."""
import os
import re
import subprocess

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "smc.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(smc_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_21983_gb300 import smc
    if not os.path.exists(smc.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return smc.load()


def test_header_declares_the_boundary_calls():
    names = _declared()
    for required in ["smc_init", "smc_set_schedule", "smc_step", "smc_anneal_next", "smc_resample",
                     "smc_posterior_predict", "smc_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2601_21983_gb300 import smc
    out = subprocess.run(["nm", "-D", "--defined-only", smc.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(smc_[a-z0-9_]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        assert hasattr(lib, n)


def test_binding_covers_declared_names():
    from paper_2601_21983_gb300 import smc
    assert sorted(smc.EXPORTED) == _declared()


def test_status_strings(lib):
    assert lib.smc_status_string(0) == b"ok"
    assert lib.smc_status_string(7) == b"unsupported"


def test_struct_sizes_match_header_layout():
    import ctypes as C
    from paper_2601_21983_gb300 import smc
    assert C.sizeof(smc.smc_layer) == 16
    assert C.sizeof(smc.smc_step_stats) == 56
    assert C.sizeof(smc.smc_step_params) == 32
    assert C.sizeof(smc.smc_schedule) == 56


def _header_constants():
    """NAME = value pairs of the header's enums and #defines (comments removed)."""
    txt = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    vals = {n: int(v) for n, v in re.findall(r"\b(SMC_[A-Z0-9_]+)\s*=\s*(\d+)", txt)}
    vals.update({n: int(v) for n, v in re.findall(r"#define\s+(SMC_[A-Z0-9_]+)\s+(\d+)", txt)})
    return vals


def test_binding_constants_match_the_header():
    """Every enum value the binding passes to the library (layer kinds,
    activations, likelihoods, precisions, resamplers, schedule kinds,
    proposals) equals the header's."""
    from paper_2601_21983_gb300 import smc
    h = _header_constants()
    pairs = {
        "LAYER_DENSE": "SMC_LAYER_DENSE", "LAYER_CONV": "SMC_LAYER_CONV", "LAYER_MAXPOOL2": "SMC_LAYER_MAXPOOL2",
        "LAYER_BNORM": "SMC_LAYER_BNORM", "ACT_TANH": "SMC_ACT_TANH", "ACT_RELU": "SMC_ACT_RELU",
        "ACT_IDENTITY": "SMC_ACT_IDENTITY", "LIK_CATEGORICAL": "SMC_LIK_CATEGORICAL",
        "LIK_GAUSSIAN": "SMC_LIK_GAUSSIAN", "PREC_FP32": "SMC_PREC_FP32", "PREC_BF16": "SMC_PREC_BF16",
        "RESAMPLE_SYSTEMATIC": "SMC_RESAMPLE_SYSTEMATIC", "RESAMPLE_MULTINOMIAL": "SMC_RESAMPLE_MULTINOMIAL",
        "PROPOSAL_PLAIN": "SMC_PROPOSAL_PLAIN", "PROPOSAL_LEARNED": "SMC_PROPOSAL_LEARNED",
        "PROPOSAL_EXPLORE": "SMC_PROPOSAL_EXPLORE", "LEARNED_NUM_PARAMS": "SMC_LEARNED_NUM_PARAMS",
    }
    for py, c in pairs.items():
        assert getattr(smc, py) == h[c], (py, c)
    sched = {"constant": "SMC_SCHED_CONSTANT", "fb": "SMC_SCHED_FB", "ctr": "SMC_SCHED_CTR",
             "linear": "SMC_SCHED_LINEAR", "automated": "SMC_SCHED_AUTOMATED", "sda": "SMC_SCHED_SDA",
             "constant_fresh": "SMC_SCHED_CONSTANT_FRESH", "ctr_fresh": "SMC_SCHED_CTR_FRESH"}
    for name, c in sched.items():
        assert smc.SCHED[name] == h[c], name
