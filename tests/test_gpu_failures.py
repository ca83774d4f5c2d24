"""Failure paths of the constrained-realization call, through the C ABI.

Every failure here is made on the host: a NaN planted in the data map, a
negative C_l, an iteration budget too small to converge, and an expired
tensor-core wait faked by the host's flag check (SHTG_FAKE_WAIT_EXPIRY), so
no device wait is ever forced to expire.  After each failure the same plan
must still give a correct result."""
import numpy as np
import pytest

from inputs import configs as C
from oracle import sht as osht
from oracle import solver as osol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cuda(x, dt):
    return torch.tensor(np.ascontiguousarray(x), dtype=dt, device="cuda")


def _setup(nside=16, lmax=32):
    from paper_2306_15511_gb300 import Plan
    p = C.masked_temperature(nside, lmax)
    g = osht.healpix(nside)
    ls = osht.ls_of(lmax)
    d = (osht.alm2map(g, lmax, p.signal_alm[0] * p.bl[ls]) + p.noise_map[0])[None, None]
    plan = Plan(nside=nside, lmax=lmax)
    args = [p.cl, p.bl, _cuda(p.ninv, torch.float64), _cuda(d, torch.float64),
            _cuda(p.w1[None], torch.complex128), _cuda(p.w2[None], torch.float64)]
    prob = osol.Problem(g, lmax, p.cl, p.bl, p.ninv)
    b = prob.rhs(d[0], p.w1, p.w2)
    return plan, args, prob, b


def _code(excinfo):
    return excinfo.value.code


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_nan_in_data_is_nonfinite(mode):
    from paper_2306_15511_gb300._native import ShtgError
    plan, args, prob, b = _setup()
    bad = args[3].clone()
    bad[0, 0, 17] = float("nan")
    with pytest.raises(ShtgError) as ei:
        plan.cg_sample(*args[:3], bad, *args[4:], tol=1e-6, mode=mode)
    assert _code(ei) == -5 and "non-finite" in str(ei.value)
    x, st = plan.cg_sample(*args, tol=1e-6, mode=mode)       # the plan is still usable
    assert st["converged"] == 1
    assert osol.true_residual(prob, x.cpu().numpy()[0], b) <= 1.05e-6


def test_negative_cl_is_not_spd():
    from paper_2306_15511_gb300._native import ShtgError
    plan, args, prob, b = _setup()
    cl = np.array(args[0], copy=True)
    cl[5] = -1.0
    with pytest.raises(ShtgError) as ei:
        plan.cg_sample(cl, *args[1:], tol=1e-6, mode="mixed")
    assert _code(ei) == -6 and "l = 5" in str(ei.value)
    x, st = plan.cg_sample(*args, tol=1e-6, mode="mixed")
    assert st["converged"] == 1


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_maxiter_is_not_converged_with_best_iterate(mode):
    """maxiter = 2: SHTG_ERR_NOT_CONVERGED; the output holds the last iterate
    and the stats are filled (the reported residual is the oracle's)."""
    from paper_2306_15511_gb300._native import ShtgError
    plan, args, prob, b = _setup()
    with pytest.raises(ShtgError) as ei:
        plan.cg_sample(*args, tol=1e-6, mode=mode, maxiter=2, check_every=1)
    assert _code(ei) == -3
    x, st = plan.cg_sample(*args, tol=1e-6, mode=mode, maxiter=2, check_every=1,
                           allow_not_converged=True)
    assert st["converged"] == 0 and st["iterations"] == 2
    xh = x.cpu().numpy()[0]
    assert np.all(np.isfinite(xh)) and np.linalg.norm(xh) > 0
    res = osol.true_residual(prob, xh, b)
    assert 1e-6 < res < 1.0
    assert abs(st["rel_residual"] - res) <= 1e-6 * res


def test_fake_wait_expiry_maps_to_timeout(monkeypatch):
    """An expired bounded wait (faked on the host) is SHTG_ERR_TIMEOUT from a
    tensor-core transform and from a tensor-core solve; the flag is cleared
    and the next call succeeds."""
    from paper_2306_15511_gb300._native import ShtgError
    plan, args, prob, b = _setup()
    a = torch.zeros(1, plan.nalm, dtype=torch.complex64, device="cuda")
    monkeypatch.setenv("SHTG_FAKE_WAIT_EXPIRY", "1")
    with pytest.raises(ShtgError) as ei:
        plan.alm2map(a, tensor_cores=True)
    assert _code(ei) == -4 and "bounded" in str(ei.value)
    with pytest.raises(ShtgError) as ei:
        plan.cg_sample(*args, tol=1e-6, mode="mixed_tc")
    assert _code(ei) == -4
    monkeypatch.delenv("SHTG_FAKE_WAIT_EXPIRY")
    plan.alm2map(a, tensor_cores=True)
    x, st = plan.cg_sample(*args, tol=1e-6, mode="mixed_tc")
    assert st["converged"] == 1
    assert osol.true_residual(prob, x.cpu().numpy()[0], b) <= 1.05e-6
