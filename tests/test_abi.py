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
    assert lib.shtg_version() == 3
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


def test_grouped_chains_rejects_options_without_gpu():
    """SHTG_GROUPED checks its options before it touches a plan or the GPU:
    the group count, the mode, the preconditioner, the flags it does not
    combine with, equal ncomp and the total number of realizations."""
    from paper_2306_15511_gb300 import _native as N
    lib = N.load()

    def call(ng, mode=N.CG_MIXED, precond=N.PRECOND_DIAG, flags=0, ncomp=(1,), nbatch=2):
        plans = (ctypes.c_void_p * ng)(*[ctypes.c_void_p(4096 * (g + 1)) for g in range(ng)])
        probs = (N.Problem * ng)()
        for g in range(ng):
            probs[g].ncomp = ncomp[g % len(ncomp)]
            probs[g].nbatch = nbatch
        outs = (ctypes.c_void_p * ng)()
        o = N.CGOpts()
        o.tol, o.maxiter, o.mode, o.precond, o.flags = 1e-6, 10, mode, precond, N.GROUPED | flags
        rc = lib.shtg_cg_sample_chains(ng, plans, probs, outs, ctypes.byref(o), None, None)
        return rc, lib.shtg_last_error_string()

    for kw, msg in (({"ng": 17}, b"1 to 16"), ({"ng": 2, "mode": N.CG_FP64}, b"mode"),
                    ({"ng": 2, "mode": N.CG_BLOCK}, b"mode"),
                    ({"ng": 2, "precond": N.PRECOND_LOWL}, b"SHTG_PRECOND"),
                    ({"ng": 2, "flags": N.SPLIT_RHS}, b"SPLIT_RHS"),
                    ({"ng": 2, "flags": N.PROFILE}, b"SPLIT_RHS or SHTG_PROFILE"),
                    ({"ng": 2, "ncomp": (1, 3)}, b"ncomp"),
                    ({"ng": 16, "nbatch": 4096}, b"65535")):
        rc, err = call(**kw)
        assert rc == -1, (kw, rc)
        assert msg in err, (kw, err)


def test_binding_constants_match_header():
    """Every #define the binding mirrors has the header's value, and the
    option struct keeps the header's field order."""
    from paper_2306_15511_gb300 import _native as N
    src = open(os.path.join(ROOT, "include", "shtg.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"#define\s+(SHTG_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", src)}
    pairs = {"FP64": "SHTG_FP64", "FP32": "SHTG_FP32", "TC32": "SHTG_TC32", "DF64": "SHTG_DF64",
             "ARITH_DEFAULT": "SHTG_ARITH_DEFAULT", "ARITH_FP64": "SHTG_ARITH_FP64",
             "ARITH_DF64": "SHTG_ARITH_DF64", "CG_FP64": "SHTG_CG_FP64", "CG_MIXED": "SHTG_CG_MIXED",
             "CG_MIXED_TC": "SHTG_CG_MIXED_TC", "CG_BLOCK": "SHTG_CG_BLOCK", "BLOCK_SOLVER": "SHTG_BLOCK_SOLVER", "HOST_INPUTS": "SHTG_HOST_INPUTS",
             "PROFILE": "SHTG_PROFILE", "NO_GRAPHS": "SHTG_NO_GRAPHS", "SPLIT_RHS": "SHTG_SPLIT_RHS",
             "GROUPED": "SHTG_GROUPED",
             "SPIN0": "SHTG_SPIN0",
             "SPIN2": "SHTG_SPIN2", "PRECOND_NONE": "SHTG_PRECOND_NONE",
             "PRECOND_DIAG": "SHTG_PRECOND_DIAG", "PRECOND_LOWL": "SHTG_PRECOND_LOWL",
             "PRECOND_AZIM": "SHTG_PRECOND_AZIM"}
    for py, c in pairs.items():
        assert getattr(N, py) == defs[c], (py, c)
    end = src.index("} shtg_cg_opts;")
    body = src[src.rindex("typedef struct {", 0, end):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(?:int|double)\s+(\w+)\s*;", body)
    assert fields == [f for f, _ in N.CGOpts._fields_]


def test_plan_create_limits_without_gpu():
    """Every documented limit of shtg_plan_create is checked before any CUDA
    call, so invalid plans fail with SHTG_ERR_ARG even without a GPU."""
    from paper_2306_15511_gb300 import _native as N
    lib = N.load()
    H, G = 0, 1   # SHTG_GEOM_HEALPIX, SHTG_GEOM_GAUSS
    bad = [
        (H, 8, 0, -1, 1),        # lmax < 0
        (H, 8, 0, 8193, 1),      # lmax > 8192
        (H, 8, 0, 16, 0),        # max_batch < 1
        (H, 8, 0, 16, 4097),     # max_batch > 4096
        (H, 0, 0, 0, 1),         # N_side < 1
        (H, 8193, 0, 16, 1),     # N_side > 8192
        (H, 8, 0, 33, 1),        # lmax > 4 N_side
        (G, 16, 0, 8, 1),        # nphi_gauss < 1
        (G, 16, 65537, 8, 1),    # nphi_gauss > 65536
        (G, 65537, 32, 8, 1),    # rings > 65536
        (5, 8, 0, 16, 1),        # unknown geometry
    ]
    for geom, n, nphi, lmax, mb in bad:
        h = ctypes.c_void_p(7)
        rc = lib.shtg_plan_create(geom, n, nphi, lmax, mb, N.SPIN0, ctypes.byref(h))
        assert rc == -1, (geom, n, nphi, lmax, mb, rc)
        assert h.value is None, "a failed create must clear *out"
        assert lib.shtg_last_error_string()
    assert lib.shtg_plan_create(H, 8, 0, 16, 1, N.SPIN0, None) == -1


def test_transform_and_solver_calls_reject_null_plans_without_gpu():
    from paper_2306_15511_gb300 import _native as N
    lib = N.load()
    buf = ctypes.c_void_p(16)   # never dereferenced: the plan check comes first
    for f in (lib.shtg_alm2map, lib.shtg_alm2map_adjoint, lib.shtg_alm2map_vjp):
        assert f(None, 0, N.FP64, buf, buf, 1, None) == -1
    assert lib.shtg_map2alm(None, 0, N.FP64, buf, buf, 1, 0, None) == -1
    pr, o, st = N.Problem(), N.CGOpts(), N.CGStats()
    assert lib.shtg_cg_sample(None, ctypes.byref(pr), buf, ctypes.byref(o), ctypes.byref(st),
                              None) == -1
    assert lib.shtg_apply_operator(None, ctypes.byref(pr), buf, buf, None) == -1
    nn = ctypes.c_int(0)
    assert lib.shtg_lowl_block(None, ctypes.byref(pr), 0, buf, buf, ctypes.byref(nn), None) == -1
    assert lib.shtg_precond_apply(None, ctypes.byref(pr), ctypes.byref(o), buf, buf, None) == -1
    info = N.PlanInfo()
    assert lib.shtg_plan_get_info(None, ctypes.byref(info)) == -1
    assert lib.shtg_plan_destroy(None) == N.SHTG_OK


def test_noalloc_rejects_invalid_sizes_without_gpu():
    from paper_2306_15511_gb300 import _native as N
    lib = N.load()
    f = lib.shtg_alm2map_adjoint_noalloc
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    buf = ctypes.c_void_p(16)
    for nside, lmax, a, b in [(0, 0, buf, buf), (8193, 16, buf, buf), (8, -1, buf, buf),
                              (8, 33, buf, buf), (8, 16, None, buf), (8, 16, buf, None),
                              (512, 1024, buf, buf)]:     # scratch above 16 MiB
        assert f(nside, lmax, a, b, None) == -1, (nside, lmax)
        assert b"noalloc" in lib.shtg_last_error_string()


def test_joint_acceptance_without_gpu():
    """The acceptance rule of the joint move (Eq. acceptance-rate) is host
    arithmetic in the library: min(1, exp of the log ratio), checked against
    the oracle's restatement."""
    from oracle import solver as osol
    from paper_2306_15511_gb300 import _native as N
    lib = N.load()
    out = ctypes.c_double(-1.0)
    for lpn, lpo, prn, pro in ((-10.0, -12.0, 0.0, 0.0), (-12.0, -10.0, 0.0, 0.0),
                               (-1e7 - 3.5, -1e7, 0.25, -0.5), (5.0, 5.0, -1.0, 0.0)):
        assert lib.shtg_joint_acceptance(lpn, lpo, prn, pro, ctypes.byref(out)) == 0
        assert out.value == osol.joint_acceptance(lpn, lpo, prn, pro)
    assert lib.shtg_joint_acceptance(float("nan"), 0.0, 0.0, 0.0, ctypes.byref(out)) == -5
    assert lib.shtg_joint_acceptance(0.0, 0.0, 0.0, 0.0, None) == -1
