"""CPU-only checks of the C ABI: the library builds, loads, and exports every
entry point include/kmpar.h declares; argument errors are reported without a GPU;
the product package never touches the oracle."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "kmpar.h")).read()
    return sorted(set(re.findall(r"KMPAR_API\s+[\w\s\*]*?\b(kmpar_\w+)\s*\(", hdr)))


@pytest.fixture(scope="module")
def lib():
    from paper_1203_6402_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["kmpar_init", "kmpar_round", "kmpar_weight", "kmpar_recluster", "kmpar_lloyd", "kmpar_cost"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1203_6402_gb300 import kmpar
    assert sorted(kmpar.EXPORTED) == declared_symbols()
    for name in kmpar.EXPORTED:
        assert callable(getattr(kmpar, name))


def test_argument_errors_need_no_gpu(lib):
    from paper_1203_6402_gb300 import kmpar
    kmpar.load()
    h = ctypes.c_void_p()
    st = kmpar._lib.kmpar_init(ctypes.byref(h), 1, 0, 3, 2, 4.0, 2, 0, kmpar.KMPAR_FP32, None)
    assert st == kmpar.KMPAR_ERR_ARG and h.value is None
    assert b"n out of range" in kmpar._lib.kmpar_last_error(None)
    st = kmpar._lib.kmpar_init(ctypes.byref(h), 1, 10, 3, 2, 4.0, 2, 0, 99, None)
    assert st == kmpar.KMPAR_ERR_UNSUPPORTED
    st = kmpar._lib.kmpar_init(ctypes.byref(h), 1, 10, 3, 2, 1e6, 2, 0, kmpar.KMPAR_FP32, None)
    assert st == kmpar.KMPAR_ERR_UNSUPPORTED
    assert kmpar._lib.kmpar_status_string(kmpar.KMPAR_ERR_CAPACITY) == b"round drew more points than its capacity"
    with pytest.raises(kmpar.KmparError):
        kmpar.kmpar_init(1, 10, 0, 2, 4.0, 2, 0, kmpar.KMPAR_FP32)
    # setters refuse a missing context before touching the device
    assert kmpar._lib.kmpar_set_recluster(None, 8) == kmpar.KMPAR_ERR_ARG
    assert kmpar._lib.kmpar_set_sampling(None, kmpar.KMPAR_SAMPLE_EXACT) == kmpar.KMPAR_ERR_ARG
    # no context has allocated, so there is no pool to trim
    assert kmpar._lib.kmpar_release_cached_memory() == kmpar.KMPAR_OK


def test_missing_library_fails_loudly(tmp_path):
    from paper_1203_6402_gb300 import kmpar
    saved = kmpar._lib
    kmpar._lib = None
    try:
        with pytest.raises(FileNotFoundError):
            kmpar.load(str(tmp_path / "absent.so"))
    finally:
        kmpar._lib = saved


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1203_6402_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", src, re.M), f
                assert "kmpar_oracle" not in src and "liboracle" not in src, f


def header_constants():
    """KMPAR_* values from the header: enum members and #define'd integers."""
    hdr = open(os.path.join(ROOT, "include", "kmpar.h")).read()
    vals = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(KMPAR_[A-Z0-9_]+)\s*=\s*(\d+)", hdr)}
    vals.update({m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(KMPAR_[A-Z0-9_]+)\s+(\d+)\b", hdr)})
    return vals


def test_binding_constants_match_the_header():
    from paper_1203_6402_gb300 import kmpar
    consts = header_constants()
    assert len(consts) >= 15
    for name, value in consts.items():
        assert getattr(kmpar, name) == value, name
    assert kmpar.PRECISIONS == {"fp32": consts["KMPAR_FP32"], "bf16": consts["KMPAR_BF16"],
                                "bf16x3": consts["KMPAR_BF16X3"], "fp8": consts["KMPAR_FP8E4M3"]}
    assert kmpar.SAMPLINGS == {"bernoulli": consts["KMPAR_SAMPLE_BERNOULLI"],
                               "exact": consts["KMPAR_SAMPLE_EXACT"]}
