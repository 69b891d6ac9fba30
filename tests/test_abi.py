"""The C-ABI library loads and exports every entry point include/*.h declares (no GPU).

Only calls that return before touching the device are exercised here.
"""
import ctypes
import glob
import os
import re

import pytest

import paper_1912_03565_gb300 as H
from paper_1912_03565_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return H.load()


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(hdr).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(hs_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "hs_solve" in names and "hs_plan" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    assert set(H.EXPORTED) <= set(declared_functions())


def test_status_strings(lib):
    for s in (0, 1, 2, -1, -2, -3, -4, -5, -6, -7):
        assert lib.hs_status_str(s).decode().startswith("HS_")


def test_argument_validation_before_device(lib):
    h = ctypes.c_void_p()
    assert lib.hs_plan(None, 4, 4, 4, 1.0, 1.0, 1.0, 4, 0, 0, 0, 1) == H.HS_ERR_INVALID_ARG
    assert lib.hs_plan(ctypes.byref(h), 0, 4, 4, 1.0, 1.0, 1.0, 4, 0, 0, 0, 1) == H.HS_ERR_INVALID_ARG
    assert lib.hs_plan(ctypes.byref(h), 4, 4, 4, 1.0, 1.0, 1.0, 5, 0, 0, 0, 1) == H.HS_ERR_INVALID_ARG
    assert lib.hs_plan(ctypes.byref(h), 4, 4, 4, 1.0, 1.0, 1.0, 6, 1, 0, 0, 1) == H.HS_ERR_INVALID_ARG
    assert lib.hs_plan(ctypes.byref(h), 4, 4, 4, 1.0, 1.0, -1.0, 4, 0, 0, 0, 1) == H.HS_ERR_INVALID_ARG
    assert lib.hs_plan(ctypes.byref(h), 4, 4, 5, 1.0, 1.0, 1.0, 6, 0, 0, 0, 1) == H.HS_ERR_INVALID_ARG
    assert lib.hs_plan(ctypes.byref(h), 4, 4, 4, 1.0, 1.0, 1.0, 4, 0, 3, 0, 1) == H.HS_ERR_UNSUPPORTED
    assert lib.hs_plan(ctypes.byref(h), 4, 4, 4, 1.0, 1.0, 1.0, 4, 0, 0, 0, 0) == H.HS_ERR_INVALID_ARG
    assert h.value is None
    assert lib.hs_destroy(None) == H.HS_OK
    assert lib.hs_solve(None, None, 0, 0, None, None, 1, None, None) == H.HS_ERR_INVALID_ARG
    assert lib.hs_set_coeff(None, None, None, None, 0) == H.HS_ERR_INVALID_ARG
    assert lib.hs_workspace_bytes(None) == 0


def test_binding_fails_loudly_without_library(tmp_path):
    with pytest.raises(RuntimeError):
        H._lib_backup = H._lib
        try:
            H._lib = None
            H.load(str(tmp_path / "missing.so"))
        finally:
            H._lib = H._lib_backup


def test_complex_plan_and_host_io_argument_validation(lib):
    """The complex plan, host-I/O and callback entry points reject bad arguments before
    touching the device."""
    h = ctypes.c_void_p()
    assert lib.hs_zplan(None, 4, 4, 4, 1.0, 1.0, 1.0, 4) == H.HS_ERR_INVALID_ARG
    assert lib.hs_zplan(ctypes.byref(h), 0, 4, 4, 1.0, 1.0, 1.0, 4) == H.HS_ERR_INVALID_ARG
    assert lib.hs_zplan(ctypes.byref(h), 4, 4, 4, 1.0, 1.0, 1.0, 5) == H.HS_ERR_INVALID_ARG
    assert lib.hs_zplan(ctypes.byref(h), 4, 4, 4, 1.0, 1.0, 1.3, 6) == H.HS_ERR_INVALID_ARG
    assert lib.hs_zplan(ctypes.byref(h), 4, 4, 4, 1.0, -1.0, 1.0, 4) == H.HS_ERR_INVALID_ARG
    assert h.value is None
    assert lib.hs_zplan_set_coeff(None, None) == H.HS_ERR_INVALID_ARG
    assert lib.hs_zplan_set_faces(None, 0, None, None, 0, None, None) == H.HS_ERR_INVALID_ARG
    assert lib.hs_zplan_set_sides(None, 0, 0) == H.HS_ERR_INVALID_ARG
    assert lib.hs_zsolve(None, None, None, None, None, None) == H.HS_ERR_INVALID_ARG
    assert lib.hs_zsolve_ex(None, None, None, None, None, None, None) == H.HS_ERR_INVALID_ARG
    assert lib.hs_zplan_set_stage_timing(None, 1) == H.HS_ERR_INVALID_ARG
    assert lib.hs_zplan_stage_times(None, None) == H.HS_ERR_INVALID_ARG
    assert lib.hs_zplan_workspace_bytes(None) == 0
    assert lib.hs_zplan_last_error(None).decode() == "no plan"
    lib.hs_zplan_destroy(None)
    assert lib.hs_set_host_io(None, 0) == H.HS_ERR_INVALID_ARG
    assert lib.hs_host_io_wait(None, None) == H.HS_ERR_INVALID_ARG
    assert lib.hs_set_coeff_fn(None, H.HS_COEFF_FN(lambda z, d, u: 0.0), None, 0) == \
        H.HS_ERR_INVALID_ARG


def test_autotune_cache_file_round_trip(lib, tmp_path):
    """The autotune cache's text format: a written file loads back to the same entries,
    and malformed or out-of-range content merges nothing (host only, no GPU)."""
    H.hs_autotune_cache_clear()
    assert H.hs_autotune_cache_count() == 0
    good = tmp_path / "tune.txt"
    good.write_text("# hs autotune cache v1\n"
                    "NVIDIA_GB300 152 255 255 255 6 0 1 1 1 1 5 0.046 0.055\n"
                    "NVIDIA_GB300 152 511 511 511 6 0 0 -1 6 6 -1 1.2 1.3\n"
                    "\n")
    H.hs_autotune_cache_load(str(good))
    assert H.hs_autotune_cache_count() == 2
    out = tmp_path / "out.txt"
    H.hs_autotune_cache_save(str(out))
    lines = [l.split() for l in out.read_text().splitlines() if not l.startswith("#")]
    assert sorted(l[:13] for l in lines) == sorted([
        "NVIDIA_GB300 152 255 255 255 6 0 1 1 1 1 5".split() + ["0.046"],
        "NVIDIA_GB300 152 511 511 511 6 0 0 -1 6 6 -1".split() + ["1.2"]])
    H.hs_autotune_cache_clear()
    H.hs_autotune_cache_load(str(out))
    assert H.hs_autotune_cache_count() == 2
    for bad_line in ("NVIDIA_GB300 152 255 255 255 6 0 1 1 9 1 5 0.1 0.1\n",    # variant 9
                     "NVIDIA_GB300 152 255 255 255 5 0 1 1 1 1 5 0.1 0.1\n",    # order 5
                     "NVIDIA_GB300 152 255 255 255 6 0 1 1 1 1 5 0.1\n",        # short
                     "NVIDIA_GB300 152 255 255 255 6 0 1 1 1 1 5 0.1 0.1 7\n"):  # extra field
        bad = tmp_path / "bad.txt"
        bad.write_text("NVIDIA_GB300 152 63 63 63 4 0 1 1 0 0 0 0.01 0.01\n" + bad_line)
        with pytest.raises(H.HsError) as e:
            H.hs_autotune_cache_load(str(bad))
        assert e.value.status == H.HS_ERR_INVALID_ARG
        assert H.hs_autotune_cache_count() == 2   # nothing merged, not even the good line
    with pytest.raises(H.HsError):
        H.hs_autotune_cache_load(str(tmp_path / "missing.txt"))
    H.hs_autotune_cache_clear()
    assert H.hs_autotune_cache_count() == 0


def test_check_finite_argument_validation(lib):
    """hs_check_finite refuses a NULL plan or count before touching the device."""
    cnt = ctypes.c_ulonglong()
    assert lib.hs_check_finite(None, None, 0, 0, None, ctypes.byref(cnt)) == H.HS_ERR_INVALID_ARG
    assert lib.hs_check_finite(None, None, 0, 0, None, None) == H.HS_ERR_INVALID_ARG


def test_static_residual_binding_checks_layout_on_cpu():
    """The allocation-free residual's binding rejects, before any library call,
    arrays the bare pointers cannot describe: wrong dtype, wrong size, strided."""
    torch = pytest.importorskip("torch")
    import numpy as np
    c4 = np.full(4, 25.0)
    good = torch.zeros((2, 2, 2), dtype=torch.float64)
    strided = torch.zeros((2, 2, 4), dtype=torch.float64)[:, :, ::2]
    assert strided.numel() == 8 and not strided.is_contiguous()
    cases = [(torch.zeros((2, 2, 2), dtype=torch.float32), good),
             (torch.zeros((2, 2, 3), dtype=torch.float64), good),
             (strided, good), (good, strided)]
    for F, u in cases:
        with pytest.raises(ValueError):
            H.hs_residual_static(2, 2, 2, 1.0, 1.0, 1.0, 4, H.HS_HELMHOLTZ, H.HS_CD_CORRECTED,
                                 c4, None, None, F, u)
