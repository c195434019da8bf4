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
