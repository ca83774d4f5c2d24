"""The allocation-free transpose transform (for callers that cannot allocate
device memory and so cannot create a plan) against the plan-based
shtg_alm2map_adjoint, through the C ABI, on two calls in a row that reuse
the library's static scratch buffer.  Collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_adjoint_matches_plan_on_two_calls():
    from paper_2306_15511_gb300 import _native
    lib = _native.load()
    fn = lib.shtg_alm2map_adjoint_noalloc
    fn.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    torch.cuda.set_device(0)
    nside, lmax = 64, 150
    npix, nalm = 12 * nside * nside, (lmax + 1) * (lmax + 2) // 2
    h = C.c_void_p()
    assert lib.shtg_plan_create(0, nside, 0, lmax, 1, 1, C.byref(h)) == 0
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    try:
        rng = np.random.default_rng(21)
        for call in range(2):            # the second call reuses the scratch of the first
            m = torch.tensor(rng.normal(size=npix) * (1 + call), dtype=torch.float64, device="cuda")
            ref = torch.empty(nalm, dtype=torch.complex128, device="cuda")
            got = torch.full((nalm,), float("nan"), dtype=torch.complex128, device="cuda")
            assert lib.shtg_alm2map_adjoint(h, 0, 0, C.c_void_p(m.data_ptr()),
                                            C.c_void_p(ref.data_ptr()), 1, stream) == 0
            assert fn(nside, lmax, C.c_void_p(m.data_ptr()), C.c_void_p(got.data_ptr()), stream) == 0
            torch.cuda.synchronize()
            g, r = got.cpu().numpy(), ref.cpu().numpy()
            err = np.linalg.norm(g - r) / np.linalg.norm(r)
            assert err < 1e-10, (call, err)
        # sizes beyond the static buffer are refused with an error, not run
        big = torch.zeros(12 * 512 * 512, dtype=torch.float64, device="cuda")
        out = torch.zeros(1025 * 1026 // 2, dtype=torch.complex128, device="cuda")
        assert fn(512, 1024, C.c_void_p(big.data_ptr()), C.c_void_p(out.data_ptr()), stream) == -1
        assert b"static buffer" in lib.shtg_last_error_string()
    finally:
        lib.shtg_plan_destroy(h)
