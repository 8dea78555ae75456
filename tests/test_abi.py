"""CPU checks of the C ABI: the library loads, exports every symbol the headers declare, the ctypes structs match
the C layouts, and argument validation rejects bad sizes without touching a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1407_7506_gb300 as pk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("ppcg.h", "ppcg_steps.h")]


@pytest.fixture(scope="module")
def lib():
    from paper_1407_7506_gb300 import build
    build.build()
    return pk.lib()


def _declared():
    names = []
    for h in HEADERS:
        names += re.findall(r"^PPCG_API\s+[\w\s\*]+?\b(ppcg_\w+)\s*\(", open(h).read(), flags=re.M)
    return names


def test_exports_match_headers(lib):
    declared = _declared()
    assert len(declared) == 19
    assert sorted(declared) == sorted(pk.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", pk.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ppcg_\w+)", out))
    assert set(declared) <= exported
    assert exported <= set(declared)            # nothing else leaks out of the library


def test_struct_layouts_match_c(tmp_path):
    # every field offset and every struct size of the ctypes mirrors against the C compiler's
    structs = [pk.ppcg_operator, pk.ppcg_options, pk.ppcg_stats, pk.ppcg_batch_item]
    cnames = {"lam": "lambda"}                                  # a Python keyword in C
    lines, want = [], []
    for st in structs:
        lines.append(f'printf("%zu\\n", sizeof({st.__name__}));')
        want.append(ctypes.sizeof(st))
        for f, _ in st._fields_:
            lines.append(f'printf("%zu\\n", offsetof({st.__name__}, {cnames.get(f, f)}));')
            want.append(getattr(st, f).offset)
    src = tmp_path / "sz.c"
    src.write_text('#include "ppcg.h"\n#include <stdio.h>\n#include <stddef.h>\nint main(void){' + "".join(lines)
                   + " return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert got == want


def test_status_strings(lib):
    for s in range(9):
        assert pk.ppcg_status_string(s).startswith("PPCG_")
    assert "unknown" in pk.ppcg_status_string(99)


def _op(N, nx=None):
    nx = N if nx is None else nx
    return pk.ppcg_operator(nx, N, N, 1.0, None, (ctypes.c_double * 3)(0, 0, 0), 0)


def test_workspace_bytes_scales_with_size(lib):
    b1 = pk.ppcg_workspace_bytes(_op(16), 16 ** 3, 64, 1)
    b2 = pk.ppcg_workspace_bytes(_op(32), 32 ** 3, 256, 4)
    # seven n x k blocks dominate
    assert b1 > 7 * 4096 * 64 * 8
    assert b2 > 7 * 32768 * 256 * 8 and b2 < 2 * 7 * 32768 * 256 * 8 + (64 << 20)


@pytest.mark.parametrize("n,k,q,nbuf,expect", [
    (16 ** 3 + 1, 64, 1, 0, pk.PPCG_ERR_ARG),     # n != nx ny nz
    (16 ** 3, 0, 1, 0, pk.PPCG_ERR_ARG),          # k < 1
    (16 ** 3, 2049, 1, 0, pk.PPCG_ERR_ARG),       # k > n / 2
    (16 ** 3, 64, 0, 0, pk.PPCG_ERR_ARG),         # sbsize < 1
    (16 ** 3, 64, 17, 0, pk.PPCG_ERR_ARG),        # sbsize above the sub-block solver's limit
    (16 ** 3, 4, 5, 0, pk.PPCG_ERR_ARG),          # sbsize > k
    (16 ** 3, 64, 4, -1, pk.PPCG_ERR_ARG),        # nbuf < 0
])
def test_argument_validation(lib, n, k, q, nbuf, expect):
    opt = pk.ppcg_options()
    opt.nbuf = nbuf
    out = ctypes.c_size_t(0)
    st = lib.ppcg_workspace_bytes(ctypes.byref(_op(16)), n, k, q, ctypes.byref(opt), ctypes.byref(out))
    assert st == expect


@pytest.mark.parametrize("field,value", [("orth", 2), ("orth", -1), ("orth_skip_tol", -1e-3),
                                         ("orth_skip_tol", float("nan")), ("fp64_gemm", 2)])
def test_invalid_option_values(lib, field, value):
    opt = pk.ppcg_options()
    setattr(opt, field, value)
    out = ctypes.c_size_t(0)
    assert (lib.ppcg_workspace_bytes(ctypes.byref(_op(16)), 4096, 8, 2, ctypes.byref(opt), ctypes.byref(out))
            == pk.PPCG_ERR_ARG)


def test_unsupported_options_are_reported(lib):
    op = _op(16)
    op.dtype = 2                                        # no such dtype
    out = ctypes.c_size_t(0)
    assert lib.ppcg_workspace_bytes(ctypes.byref(op), 4096, 8, 2, None, ctypes.byref(out)) == pk.PPCG_ERR_UNSUPPORTED
    op = _op(16)
    op.theta[1] = 0.5                                   # a Bloch twist needs the complex dtype
    assert lib.ppcg_workspace_bytes(ctypes.byref(op), 4096, 8, 2, None, ctypes.byref(out)) == pk.PPCG_ERR_UNSUPPORTED
    opt = pk.ppcg_options()
    opt.precision = 3                                   # no such precision
    assert (lib.ppcg_workspace_bytes(ctypes.byref(_op(16)), 4096, 8, 2, ctypes.byref(opt), ctypes.byref(out))
            == pk.PPCG_ERR_UNSUPPORTED)
    opt.precision = 2                                   # the BF16 mixed form is provided
    assert (lib.ppcg_workspace_bytes(ctypes.byref(_op(16)), 4096, 8, 2, ctypes.byref(opt), ctypes.byref(out))
            == pk.PPCG_OK)


def test_null_handles_and_pointers(lib):
    assert lib.ppcg_destroy(None) == pk.PPCG_OK
    assert lib.ppcg_solve(None, None, 1e-8, None, None, None, None) == pk.PPCG_ERR_ARG
    assert lib.ppcg_create(None, 1, 1, 1, 1, None, None, None, 0, None) == pk.PPCG_ERR_ARG
    assert lib.ppcg_apply_operator(None, None, 0, None, 0, 1) == pk.PPCG_ERR_ARG


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    V = np.zeros(16 ** 3)
    op = _op(16)
    op.V = V.ctypes.data
    h = ctypes.c_void_p(0)
    st = lib.ppcg_create(ctypes.byref(op), 4096, 8, 2, 5, None, None, None, 0, ctypes.byref(h))
    assert st == pk.PPCG_ERR_CUDA and not h.value


def test_batched_and_autotune_validate_arguments(lib):
    assert lib.ppcg_solve_batched(None, 1, 0) == pk.PPCG_ERR_ARG
    items = (pk.ppcg_batch_item * 2)()
    assert lib.ppcg_solve_batched(items, 2, 0) == pk.PPCG_ERR_ARG       # NULL handles
    assert lib.ppcg_solve_batched(items, -1, 0) == pk.PPCG_ERR_ARG
    assert lib.ppcg_solve_batched(items, 0, 0) == pk.PPCG_OK
    best = ctypes.c_int32(0)
    assert lib.ppcg_autotune_sbsize(None, 4096, 8, 5, None, None, 1e-8, None, 0, None, ctypes.byref(best),
                                    None) == pk.PPCG_ERR_ARG


def test_complex_handles_size_the_real_form(lib):
    # a C128 problem is solved in its real form of order 2n with 2(k + nbuf) columns and sub-blocks of 2 sbsize
    real, cplx = _op(16), _op(16)
    cplx.dtype = 1
    cplx.theta[0] = 0.3
    a, b = ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert lib.ppcg_workspace_bytes(ctypes.byref(real), 4096, 8, 2, None, ctypes.byref(a)) == pk.PPCG_OK
    assert lib.ppcg_workspace_bytes(ctypes.byref(cplx), 4096, 8, 2, None, ctypes.byref(b)) == pk.PPCG_OK
    assert b.value > 2 * a.value
    assert lib.ppcg_workspace_bytes(ctypes.byref(cplx), 4096, 16, 9, None, ctypes.byref(a)) == pk.PPCG_ERR_ARG
    cplx.theta[2] = float("inf")
    assert lib.ppcg_workspace_bytes(ctypes.byref(cplx), 4096, 8, 2, None, ctypes.byref(a)) == pk.PPCG_ERR_ARG
