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


def test_every_declared_symbol_has_a_binding_of_the_same_name():
    from paper_2310_20103_gb300 import lgw
    missing = [n for n in _declared() if not callable(getattr(lgw, n, None))]
    assert not missing, missing


def test_null_handle_is_rejected_by_the_backward_entry_points(lib):
    """A NULL handle gives LGW_ERR_ARG before anything touches the device."""
    P = ctypes.c_void_p
    for name in ("lgw_sigma_c_backward", "lgw_sigma_c_tda_backward"):
        fn = getattr(lib, name)
        fn.argtypes = [P] * 7
        fn.restype = ctypes.c_int
        assert fn(None, None, None, None, None, None, None) == 1, name
    fn = lib.lgw_sigma_c_poly_backward
    fn.argtypes = [P] * 8
    fn.restype = ctypes.c_int
    assert fn(None, None, None, None, None, None, None, None) == 1


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
    assert ctypes.sizeof(L.lgw_options) == 56


def test_binding_offsets_match_c_compiler(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    that a C compiler gives the header's struct, and the binding's enum
    values equal the header's."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_2310_20103_gb300 import lgw as L
    structs = {"lgw_system_desc": L.lgw_system_desc, "lgw_problem": L.lgw_problem,
               "lgw_poly": L.lgw_poly,
               "lgw_options": L.lgw_options, "lgw_report": L.lgw_report}
    enums = {"LGW_FP64": L.PRECISION["fp64"], "LGW_BF16": L.PRECISION["bf16"],
             "LGW_FP8": L.PRECISION["fp8"], "LGW_FP8_DEQ": L.PRECISION["fp8_deq"],
             "LGW_REORTH_NONE": L.REORTH["none"],
             "LGW_REORTH_CGS2": L.REORTH["cgs2"], "LGW_REORTH_CGS1K": L.REORTH["cgs1k"],
             "LGW_RA_AUTO": L.REORTH_ARITH["auto"], "LGW_RA_FP64": L.REORTH_ARITH["fp64"],
             "LGW_RA_SPLIT": L.REORTH_ARITH["split"], "LGW_RA_SPLIT32": L.REORTH_ARITH["split32"],
             "LGW_SYS_NO_FP64": L.SYS_NO_FP64, "LGW_SYS_NO_BF16": L.SYS_NO_BF16,
             "LGW_SYS_FP8": L.SYS_FP8}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "lgw.h"', "int main(void) {"]
    expect = []
    for name, cls in structs.items():
        lines.append(f'  printf("%zu\\n", sizeof({name}));')
        expect.append(ctypes.sizeof(cls))
        for f, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({name}, {f}));')
            expect.append(getattr(cls, f).offset)
    for name, v in enums.items():
        lines.append(f'  printf("%d\\n", (int){name});')
        expect.append(v)
    lines += ["  return 0;", "}"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "abi"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert got == expect
