"""The C-ABI library builds, loads and exports every symbol declared in
include/hh.h; host-side argument checks answer without touching a GPU."""

import ctypes
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "hh.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hh_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2208_02320_gb300 import _build
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc") and not os.path.exists(_build.LIB):
        pytest.skip("nvcc not available")
    _build.build()
    from paper_2208_02320_gb300 import binding
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "hh_homogenize_hierarchical" in names and "hh_fit_inverse_n" in names
    for n in names:
        assert hasattr(lib, n), n
    from paper_2208_02320_gb300 import _build
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hh_[a-z0-9_]+)", out))
    assert set(names) <= exported


def test_binding_covers_every_symbol():
    from paper_2208_02320_gb300 import binding
    assert set(_declared()) == set(binding._SIGNATURES)


def test_host_side_calls(lib):
    from paper_2208_02320_gb300 import binding as B
    assert b"libhh" in lib.hh_version()
    for s in (0, 1, -1, -2, -3, -4, -5, -6, -7):
        assert lib.hh_status_string(s)
    o = B.Options()
    assert lib.hh_options_default(ctypes.byref(o)) == 0
    assert o.precision == B.HH_FP32 and o.tol == 1e-6 and o.max_iter == 20000 and o.use_graphs == 1
    assert lib.hh_options_default(None) == B.HH_ERR_ARG
    # argument checks that return before any device work
    ns = np.array([16, 32], dtype=np.int32)
    M = np.array([1.0, 2.0])
    mi, c = ctypes.c_double(), ctypes.c_double()
    assert lib.hh_fit_inverse_n(None, ns.ctypes.data_as(ctypes.c_void_p), M.ctypes.data_as(ctypes.c_void_p), 2,
                                ctypes.byref(mi), ctypes.byref(c)) == B.HH_ERR_ARG
    assert lib.hh_create(None, 0, None) == B.HH_ERR_ARG


def test_header_struct_layouts_match_binding():
    """Offsets of the option and result structs agree between the C header and
    the ctypes mirror (checked with the host C compiler)."""
    from paper_2208_02320_gb300 import binding as B
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "hh.h"
int main(void){
 printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(hh_options), offsetof(hh_options, workspace_bytes),
        offsetof(hh_options, check_every), offsetof(hh_options, wave_boxes), offsetof(hh_options, fused),
        sizeof(hh_result), offsetof(hh_result, status));
 return 0;}
'''
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run([cc, "-I" + os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert vals == [ctypes.sizeof(B.Options), B.Options.workspace_bytes.offset, B.Options.check_every.offset,
                    B.Options.wave_boxes.offset, B.Options.fused.offset, ctypes.sizeof(B.Result),
                    B.Result.status.offset]


def _declared_arity():
    """Parameter count of every function declared in include/hh.h."""
    txt = open(os.path.join(ROOT, "include", "hh.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(hh_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", txt):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_arity_matches_header():
    from paper_2208_02320_gb300 import binding as B
    ar = _declared_arity()
    assert set(ar) == set(B._SIGNATURES)
    for name, (_, args) in B._SIGNATURES.items():
        assert len(args) == ar[name], name


def test_null_arguments_fail_cleanly(lib):
    """Every entry point answers NULL pointers (a NULL context first) with
    HH_ERR_ARG and an error text, before any device work."""
    from paper_2208_02320_gb300 import binding as B
    skip = {"hh_version", "hh_status_string", "hh_last_error", "hh_cnn_num_params", "hh_destroy"}
    fill = {ctypes.c_void_p: None, ctypes.c_int: 1, ctypes.c_double: 1.0, ctypes.c_int64: 1,
            ctypes.c_uint64: 0, ctypes.c_char_p: None}
    for name, (_, argtypes) in B._SIGNATURES.items():
        if name in skip:
            continue
        args = [fill[t] for t in argtypes]
        assert getattr(lib, name)(*args) == B.HH_ERR_ARG, name
        assert lib.hh_last_error(None), name
    lib.hh_destroy(None)  # a no-op
