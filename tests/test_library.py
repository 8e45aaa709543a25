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
    # serving charge: matrix rows rounded up to 1,024, sizes, 256 B, 160 B per event of the largest batch
    assert tn.tn_server_job_bytes(3000, 1000) == 3072 * 48 * 8 + 3000 * 4 + 256 + 1000 * 160
    assert tn.tn_server_job_bytes(1024, 0) == 1024 * 16 * 8 + 1024 * 4 + 256


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


def test_growth_and_online_reject_bad_arguments_before_any_device_call(lib_path):
    """Host-side argument checks of the node-growth and online-state entry
    points return TN_EINVAL before touching a device (no GPU needed)."""
    lib = tn.load_library()
    vp = ctypes.c_void_p
    fake = vp(0x1000)  # never dereferenced: every call below fails its argument checks first
    assert lib.tn_grow_matrix(fake, 100, fake, 50, None) == tn.TN_EINVAL      # shrinking
    assert lib.tn_grow_matrix(None, 10, fake, 20, None) == tn.TN_EINVAL       # no old matrix
    assert lib.tn_grow_matrix(fake, 0, None, 20, None) == tn.TN_EINVAL        # no new matrix
    assert lib.tn_grow_matrix(fake, 10, fake, 1 << 30, None) == tn.TN_EINVAL  # too many nodes
    # in place is only allowed while the row stride stays (1000 -> 2000 nodes changes it)
    assert lib.tn_grow_matrix(fake, 1000, fake, 2000, None) == tn.TN_EINVAL
    # partially overlapping buffers
    assert lib.tn_grow_matrix(vp(0x100000), 1000, vp(0x100000 + 4096), 1000, None) == tn.TN_EINVAL
    h = vp()
    assert lib.tn_online_create(0, None, None, ctypes.byref(h)) == tn.TN_EINVAL
    assert lib.tn_online_create(1 << 30, None, None, ctypes.byref(h)) == tn.TN_EINVAL
    assert lib.tn_online_create(10, None, None, None) == tn.TN_EINVAL
    assert lib.tn_online_push(None, fake, fake, fake, 5, 0, None) == tn.TN_EINVAL
    assert lib.tn_online_flush(None, None) == tn.TN_EINVAL
    assert lib.tn_online_grow(None, 10, None) == tn.TN_EINVAL
    assert lib.tn_online_status(None, None) == tn.TN_EINVAL
    assert lib.tn_online_destroy(None, None) == tn.TN_EINVAL


def test_resident_option_checked_before_any_device_call(lib_path):
    """The resident-slab option is validated on the host: an unsupported width,
    or one combined with the column-slab options, returns TN_EINVAL, and online
    states do not take it."""
    lib = tn.load_library()
    vp = ctypes.c_void_p
    fake = vp(0x1000)  # never dereferenced
    assert tn.tn_resident_max_rows(3) == 0 and tn.tn_resident_max_rows(4) == 0 and tn.tn_resident_max_rows(0) == 0
    h = vp()
    for kw in (dict(resident_words=3), dict(resident_words=4), dict(resident_words=8), dict(resident_words=1, slab_words=16),
               dict(resident_words=2, smem_rows=64), dict(resident_words=1, wave_ctas=152)):
        opt = tn._plan_options(**kw)
        assert lib.tn_plan_create(fake, fake, fake, 10, 100, None, ctypes.byref(opt), None,
                                  ctypes.byref(h)) == tn.TN_EINVAL, kw
    opt = tn._plan_options(resident_words=1)
    assert lib.tn_online_create(100, ctypes.byref(opt), None, ctypes.byref(h)) == tn.TN_EINVAL
