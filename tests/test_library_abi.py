"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/tsvd.h; host-side argument checks work without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2603_11953_gb300 as T
from paper_2603_11953_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tsvd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tsvd_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return T.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 9
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (tsvd_\w+)", out))
    for nm_ in names:
        assert nm_ in exported, nm_
        assert hasattr(lib, nm_)
    assert set(T.EXPORTED) == set(names)
    # internal kernels and helpers stay hidden
    assert all(s.startswith("tsvd_") for s in exported)


def test_status_strings(lib):
    for code in range(10):
        s = T.tsvd_status_string(code)
        assert s.startswith("TSVD_")
    assert T.tsvd_status_string(0) == "TSVD_OK"
    assert T.tsvd_status_string(77) == "TSVD_ERR_UNKNOWN"


def test_host_argument_checks_without_device(lib):
    # null handle / null pointers are rejected on the host before any CUDA call
    assert lib.tsvd_gram(None, None, 10, 2, 10, 0, 1, None, 2) == T.TSVD_ERR_ARG
    assert lib.tsvd_solve(None, None, 10, 2, 10, 0, 1, None, None, 2, None, 0, None) == T.TSVD_ERR_ARG
    assert lib.tsvd_destroy(None) == T.TSVD_ERR_ARG
    assert lib.tsvd_create(None, 0, None, None) == T.TSVD_ERR_ARG
    bad = T.tsvd_opts(slices=3)
    h = ctypes.c_void_p()
    assert lib.tsvd_create(ctypes.byref(h), 0, None, ctypes.byref(bad)) == T.TSVD_ERR_UNSUPPORTED


def test_struct_layouts_match_header():
    assert ctypes.sizeof(T.tsvd_info) == 24
    hdr = open(os.path.join(ROOT, "include", "tsvd.h")).read()
    body = hdr[hdr.index("typedef struct {\n    int slices"):]
    body = body[:body.index("} tsvd_opts;")]
    fields = re.findall(r"\b(?:int|double|long long)\s+(\w+);", body)
    assert fields == [f[0] for f in T.tsvd_opts._fields_]
