"""The joint (C_l, a) move of Sect. 2.2.2 on the GPU, through the C ABI,
against the FP64 oracle: the mean-field / fluctuation split of the
right-hand side (Eqs. mean-field-map and fluc-map) as one batch, the
fluctuation rescaling (C')^{1/2} C^{-1/2}, log pi(theta) of Eq.
(acceptance-rate) and one complete joint-move step."""
import numpy as np
import pytest

from inputs import configs as C
from oracle import sht as osht
from oracle import solver as osol
from tests._util import rand_alm, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cuda(x, dt):
    return torch.tensor(np.ascontiguousarray(x), dtype=dt, device="cuda")


def _data(p, g):
    L = p.lmax
    ls = osht.ls_of(L)
    if p.ncomp == 1:
        return (osht.alm2map(g, L, p.signal_alm[0] * p.bl[ls]) + p.noise_map[0])[None]
    T = osht.alm2map(g, L, p.signal_alm[0] * p.bl[ls])
    Q, U = osht.alm2map_spin2(g, L, p.signal_alm[1] * p.bl[ls], p.signal_alm[2] * p.bl[ls])
    return np.stack([T, Q, U]) + p.noise_map


def _teb(nb=2, nside=16, lmax=32):
    from paper_2306_15511_gb300 import Plan
    p = C.teb_realizations(nb, nside, lmax)
    g = osht.healpix(nside)
    ds = np.stack([_data(q, g) for q in p])
    w1 = np.stack([q.w1 for q in p])
    w2 = np.stack([q.w2 for q in p])
    plan = Plan(nside=nside, lmax=lmax, max_batch=2 * nb, spin2=True)
    prob = osol.Problem(g, lmax, p[0].cl, p[0].bl, p[0].ninv)
    return p, g, ds, w1, w2, plan, prob


def _perturbed(cl4):
    """A proposal's T+E+B spectra: every block stays positive definite."""
    tt, ee, bb, te = cl4
    return np.stack([1.1 * tt, 0.9 * ee, 1.2 * bb, 1.05 * te])


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_split_rhs_mean_field_and_fluctuation(mode):
    p, g, ds, w1, w2, plan, prob = _teb()
    args = (p[0].cl, p[0].bl, _cuda(p[0].ninv, torch.float64), _cuda(ds, torch.float64),
            _cuda(w1, torch.complex128), _cuda(w2, torch.float64))
    x, st = plan.cg_sample(*args, tol=1e-8, mode=mode, maxiter=4000, split=True)
    assert st["converged"] == 1 and tuple(x.shape[:2]) == (2, 2)
    xh = x.cpu().numpy()
    for k in range(2):
        bm, bf = prob.rhs_parts(ds[k], w1[k], w2[k])
        assert osol.true_residual(prob, xh[0, k], bm) <= 1.05e-8
        assert osol.true_residual(prob, xh[1, k], bf) <= 1.05e-8
        # a = a^ + f^ solves the full system (Eq. mapmakingeq)
        b = prob.rhs(ds[k], w1[k], w2[k])
        assert osol.true_residual(prob, xh[0, k] + xh[1, k], b) <= 2.1e-8


def test_split_rhs_host_inputs_match_device_inputs():
    p, g, ds, w1, w2, plan, prob = _teb(nb=1)
    dev = plan.cg_sample(p[0].cl, p[0].bl, _cuda(p[0].ninv, torch.float64), _cuda(ds, torch.float64),
                         _cuda(w1, torch.complex128), _cuda(w2, torch.float64), tol=1e-8, mode="fp64",
                         split=True)[0].cpu().numpy()
    host = plan.cg_sample(p[0].cl, p[0].bl, np.ascontiguousarray(p[0].ninv), np.ascontiguousarray(ds),
                          np.ascontiguousarray(w1), np.ascontiguousarray(w2), tol=1e-8, mode="fp64",
                          split=True)[0].numpy()
    assert np.array_equal(dev, host)


@pytest.mark.parametrize("ncomp", [1, 3])
def test_fluctuation_rescale_vs_oracle(ncomp):
    from paper_2306_15511_gb300 import Plan
    L = 40
    plan = Plan(nside=16, lmax=L, max_batch=2, spin2=True)
    rng = np.random.default_rng(31 + ncomp)
    tt = C.cl_damped(L)
    cl4 = np.stack([tt, 0.05 * tt, 5e-5 * tt, 0.3 * np.sqrt(0.05) * tt])
    co = tt if ncomp == 1 else cl4
    cn = 1.1 * tt if ncomp == 1 else _perturbed(cl4)
    f = rand_alm(L, rng, (2, ncomp))
    got = plan.fluctuation_rescale(co, cn, _cuda(f, torch.complex128)).cpu().numpy()
    for b in range(2):
        ref = osol.fluctuation_rescale(co, cn, f[b], L)
        assert rel_l2(got[b], ref) < 1e-14
    # the identity move changes nothing (active multipoles) and held ones are 0
    same = plan.fluctuation_rescale(co, co, _cuda(f, torch.complex128)).cpu().numpy()
    ls = osht.ls_of(L)
    assert rel_l2(same[..., ls >= 2], f[..., ls >= 2]) < 1e-14
    assert np.all(same[..., ls < 2] == 0)


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_joint_log_target_vs_oracle(precision):
    p, g, ds, w1, w2, plan, prob = _teb()
    L = p[0].lmax
    rng = np.random.default_rng(5)
    sc = np.sqrt(np.maximum(p[0].cl[0], 0.0))
    a = rand_alm(L, rng, (2, 3), sc)
    f = rand_alm(L, rng, (2, 3), sc)
    lp = plan.joint_log_target(p[0].cl, p[0].bl, _cuda(p[0].ninv, torch.float64), _cuda(ds, torch.float64),
                               _cuda(a, torch.complex128), _cuda(f, torch.complex128), precision=precision)
    for k in range(2):
        ref = osol.joint_log_target(prob, ds[k], a[k], f[k])
        assert abs(lp[k] - ref) <= 1e-11 * abs(ref), (k, lp[k], ref)


def test_joint_log_target_temperature_with_cl_scale():
    from paper_2306_15511_gb300 import Plan
    pt = C.masked_temperature(32, 64)
    g = osht.healpix(32)
    d = _data(pt, g)
    plan = Plan(nside=32, lmax=64, max_batch=2)
    rng = np.random.default_rng(8)
    a = rand_alm(64, rng, (2, 1), np.sqrt(pt.cl))
    f = rand_alm(64, rng, (2, 1), np.sqrt(pt.cl))
    dd = np.stack([d, d])
    lp = plan.joint_log_target(pt.cl, pt.bl, _cuda(pt.ninv, torch.float64), _cuda(dd, torch.float64),
                               _cuda(a, torch.complex128), _cuda(f, torch.complex128), cl_scale=[1.0, 1.3])
    for k, s_ in enumerate((1.0, 1.3)):
        prob = osol.Problem(g, 64, s_ * pt.cl, pt.bl, pt.ninv)
        ref = osol.joint_log_target(prob, d, a[k], f[k])
        assert abs(lp[k] - ref) <= 1e-11 * abs(ref)


def test_joint_move_step_vs_oracle():
    """One step of the joint sampler (Sect. 2.2.2): at theta^i the mean field
    and fluctuation (one split solve); the proposal theta' = perturbed
    spectra; its mean field (a solve with w1 = w2 = 0), the rescaled
    fluctuation, log pi at both points and the acceptance probability.  The
    oracle runs the same step with its own solves (to 1e-11): log pi agrees
    to 1e-9 relative and the acceptance probability to 1e-6."""
    from paper_2306_15511_gb300 import joint_acceptance
    p, g, ds, w1, w2, plan, prob = _teb(nb=1)
    L = p[0].lmax
    cl0, cl1 = p[0].cl, _perturbed(p[0].cl)
    dev = lambda x, dt: _cuda(x, dt)  # noqa: E731
    nv, dd = dev(p[0].ninv, torch.float64), dev(ds, torch.float64)
    x0, _ = plan.cg_sample(cl0, p[0].bl, nv, dd, dev(w1, torch.complex128), dev(w2, torch.float64),
                           tol=1e-11, mode="fp64", maxiter=4000, split=True)
    a0, f0 = x0[0].contiguous(), x0[1].contiguous()
    z1, z2 = torch.zeros_like(dev(w1, torch.complex128)), torch.zeros_like(dev(w2, torch.float64))
    a1, _ = plan.cg_sample(cl1, p[0].bl, nv, dd, z1, z2, tol=1e-11, mode="fp64", maxiter=4000)
    f1 = plan.fluctuation_rescale(cl0, cl1, f0)
    lp0 = plan.joint_log_target(cl0, p[0].bl, nv, dd, a0, f0)[0]
    lp1 = plan.joint_log_target(cl1, p[0].bl, nv, dd, a1.contiguous(), f1)[0]
    acc = joint_acceptance(lp1, lp0)
    # the oracle's own step
    prob1 = osol.Problem(g, L, cl1, p[0].bl, p[0].ninv)
    bm0, bf0 = prob.rhs_parts(ds[0], w1[0], w2[0])
    oa0 = osol.pcg(prob, bm0, 1e-11, 4000)[0]
    of0 = osol.pcg(prob, bf0, 1e-11, 4000)[0]
    bm1, _ = prob1.rhs_parts(ds[0], w1[0], w2[0])
    oa1 = osol.pcg(prob1, bm1, 1e-11, 4000)[0]
    of1 = osol.fluctuation_rescale(cl0, cl1, of0, L)
    olp0 = osol.joint_log_target(prob, ds[0], oa0, of0)
    olp1 = osol.joint_log_target(prob1, ds[0], oa1, of1)
    oacc = osol.joint_acceptance(olp1, olp0)
    print(f"joint move: log pi {lp0:.6f} -> {lp1:.6f} (oracle {olp0:.6f} -> {olp1:.6f}), "
          f"acceptance {acc:.6f} (oracle {oacc:.6f})")
    assert abs(lp0 - olp0) <= 1e-9 * abs(olp0)
    assert abs(lp1 - olp1) <= 1e-9 * abs(olp1)
    assert abs(acc - oacc) <= 1e-6
