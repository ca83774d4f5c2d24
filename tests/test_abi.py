"""The C-ABI library builds, loads and exports every symbol include/shtg.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "shtg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(shtg_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_declared_symbols():
    from paper_2306_15511_gb300 import _native, build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(_native.SYMBOLS) <= set(names)


def test_version_and_error_string_without_gpu():
    from paper_2306_15511_gb300 import _native
    lib = _native.load()
    assert lib.shtg_version() >= 1
    # argument validation happens before any CUDA call
    h = ctypes.c_void_p()
    rc = lib.shtg_plan_create(7, 8, 0, 16, 1, 1, ctypes.byref(h))
    assert rc == -1
    assert b"geometry" in lib.shtg_last_error_string()


def test_oracle_builds():
    from oracle import _lib
    assert os.path.exists(_lib.build())


def test_chains_rejects_bad_arguments_without_gpu():
    """Argument checks of the chains entry point run before any CUDA call."""
    from paper_2306_15511_gb300 import _native
    lib = _native.load()
    rc = lib.shtg_cg_sample_chains(0, None, None, None, None, None, None)
    assert rc == -1
    assert b"chains" in lib.shtg_last_error_string()
    h = ctypes.c_void_p(1234)   # never dereferenced: the duplicate check comes first
    plans = (ctypes.c_void_p * 2)(h, h)
    probs = (_native.Problem * 2)()
    outs = (ctypes.c_void_p * 2)()
    rc = lib.shtg_cg_sample_chains(2, plans, probs, outs, None, None, None)
    assert rc == -1
    assert b"own plan" in lib.shtg_last_error_string()


def test_binding_constants_match_header():
    """Every #define the binding mirrors has the header's value, and the
    option struct keeps the header's field order."""
    from paper_2306_15511_gb300 import _native as N
    src = open(os.path.join(ROOT, "include", "shtg.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"#define\s+(SHTG_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", src)}
    pairs = {"FP64": "SHTG_FP64", "FP32": "SHTG_FP32", "TC32": "SHTG_TC32", "DF64": "SHTG_DF64",
             "ARITH_DEFAULT": "SHTG_ARITH_DEFAULT", "ARITH_FP64": "SHTG_ARITH_FP64",
             "ARITH_DF64": "SHTG_ARITH_DF64", "CG_FP64": "SHTG_CG_FP64", "CG_MIXED": "SHTG_CG_MIXED",
             "CG_MIXED_TC": "SHTG_CG_MIXED_TC", "HOST_INPUTS": "SHTG_HOST_INPUTS",
             "PROFILE": "SHTG_PROFILE", "NO_GRAPHS": "SHTG_NO_GRAPHS", "SPIN0": "SHTG_SPIN0",
             "SPIN2": "SHTG_SPIN2"}
    for py, c in pairs.items():
        assert getattr(N, py) == defs[c], (py, c)
    end = src.index("} shtg_cg_opts;")
    body = src[src.rindex("typedef struct {", 0, end):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(?:int|double)\s+(\w+)\s*;", body)
    assert fields == [f for f, _ in N.CGOpts._fields_]
