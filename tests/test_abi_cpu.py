"""The C ABI library builds, loads without a GPU and exports every entry
point declared in include/lgw.h.  No compute calls are made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2310_20103_gb300.build import build
    path = build()
    return ctypes.CDLL(path)


def _declared():
    src = open(os.path.join(ROOT, "include", "lgw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lgw_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["lgw_create", "lgw_destroy", "lgw_prepare_system", "lgw_release_system",
              "lgw_sigma_c", "lgw_sigma_c_batched", "lgw_lanczos_coeffs",
              "lgw_sigma_from_coeffs", "lgw_sigma_c_backward", "lgw_status_string",
              "lgw_last_error", "lgw_apply_casida"]:
        assert n in names, n


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    lib.lgw_status_string.restype = ctypes.c_char_p
    lib.lgw_status_string.argtypes = [ctypes.c_int]
    assert lib.lgw_status_string(0) == b"ok"
    assert lib.lgw_status_string(5).startswith(b"Casida")
    assert lib.lgw_status_string(99) == b"unknown status"


def test_null_arguments_are_rejected(lib):
    lib.lgw_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert lib.lgw_create(None, 0, None) == 1          # LGW_ERR_ARG
    lib.lgw_destroy.argtypes = [ctypes.c_void_p]
    assert lib.lgw_destroy(None) == 0
    lib.lgw_release_system.argtypes = [ctypes.c_void_p]
    assert lib.lgw_release_system(None) == 0


def test_binding_struct_layouts_match_header():
    from paper_2310_20103_gb300 import lgw as L
    # field counts follow the header's structs
    src = open(os.path.join(ROOT, "include", "lgw.h")).read()
    body = src[src.index("typedef struct {\n  double ms_total;"):src.index("} lgw_report;")]
    names = re.findall(r"\b(ms_\w+|gemm_flops|reorth_elems|min_theta|n_vectors|n_sub_batches|"
                       r"b_sub|k_min|k_max|n_second_pass|gpu_launches|gemm1_splits)\b", body)
    assert [f for f, _ in L.lgw_report._fields_] == names
    assert ctypes.sizeof(L.lgw_options) == 48
