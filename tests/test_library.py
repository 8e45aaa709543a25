"""The native library builds for sm_103a, loads without a GPU and exports every
entry point that include/tn.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2307_04890_gb300 as tn
from paper_2307_04890_gb300.build import INCLUDE, LIB, build_library


def declared_functions():
    text = open(os.path.join(INCLUDE, "tn.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tn_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    return build_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("tn_component_matrix", "tn_out_sizes", "tn_hash_proxy", "tn_hash_estimate",
                     "tn_status_string", "tn_plan_create", "tn_plan_apply", "tn_plan_apply_batch",
                     "tn_out_component_sizes_host"):
        assert required in names


def test_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True)
    exported = set(re.findall(r"\sT\s(tn_[a-z_0-9]+)", out.stdout))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(lib_path)
    for f in declared_functions():
        assert getattr(lib, f) is not None


def test_host_helpers_without_gpu(lib_path):
    assert tn.tn_row_words(0) == 0
    assert tn.tn_row_words(1) == 16
    assert tn.tn_row_words(1024) == 16
    assert tn.tn_row_words(1025) == 32
    assert tn.tn_row_words(100_000) == 1568
    assert tn.tn_status_string(tn.TN_ERANGE).startswith("TN_ERANGE")
    assert tn.tn_status_string(12345) == "unknown tn_status"


def test_binding_fails_loudly_without_library(tmp_path):
    import importlib
    import sys
    code = ("import paper_2307_04890_gb300 as tn\n"
            f"tn.load_library({str(tmp_path / 'missing.so')!r})\n")
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                         cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    assert res.returncode != 0 and "not found" in res.stderr


def test_server_needs_a_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tn.TnError) as exc:
        tn.Server()
    assert exc.value.status == tn.TN_ECUDA
