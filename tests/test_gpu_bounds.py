"""Spectral bounds (Sec. II-C: the expansion needs bounds that contain the
spectrum of Hp) through the C ABI.

The bounds a solve uses are a Lanczos estimate certified by three logistic
steps X <- 4 X (I - X) (Chebyshev T_8 of the rescaled Hp): whatever the
estimate, the certified interval must contain every eigenvalue and lie inside
the Gershgorin interval.  The test hook fe_k_narrow_bounds shrinks the estimate
until it cuts into the spectrum; the certificate must widen it back, and the
answer must meet the oracle tolerances:
||D - D_ref||_F / sqrt(N_e) <= 1e-6, |E_band - E_ref| / N_e <= 1e-7,
|tr D - N_e| <= 1e-9, ||D^2 - D||_F <= 1e-8 (zero temperature)."""
import math

import numpy as np
import pytest

import hp_synth
import oracle
from gpu_util import need_gpu, torch

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]

TOL_EPS1, TOL_E, TOL_TR, TOL_IDEM = 1e-6, 1e-7, 1e-9, 1e-8


def _problems():
    return [dict(p=hp_synth.gapped(700, 400, (-3.0, -0.01), (0.01, 1.0), 801), kT=0.0),
            dict(p=hp_synth.gapped(1300, 1000, (-2.0, -0.05), (0.05, 2.0), 802), kT=0.0),
            dict(p=hp_synth.gapped(257, 64, (-3.0, -0.01), (0.01, 1.0), 803), kT=0.0),
            dict(p=hp_synth.smeared(600, 510.0, 0.02, -2.0, 1.0, 804), kT=0.02)]


def _check(it, D, r, gersh):
    import paper_2301_04642_gb300 as fe
    p, kT = it["p"], it["kT"]
    assert r["status"] == fe.FE_OK
    if kT > 0:
        ref = oracle.density(p.H, p.ne, kT)
        Dref, Eref = ref["D"], ref["e_band"]
    else:
        f = (np.arange(p.n) < int(p.ne)).astype(float)
        Dref = oracle.density_from_eig(p.Q, f)
        Eref = float(np.sum(f * p.lam))
        assert np.linalg.norm(oracle.matmul(D, D) - D) <= TOL_IDEM
    assert np.linalg.norm(D - Dref) / math.sqrt(p.ne) <= TOL_EPS1
    assert abs(r["e_band"] - Eref) / p.ne <= TOL_E
    assert abs(np.trace(D) - p.ne) <= TOL_TR
    # the bounds used contain the spectrum and lie within Gershgorin
    assert r["eps_min"] <= p.lam[0] and p.lam[-1] <= r["eps_max"]
    assert gersh[0] <= r["eps_min"] and r["eps_max"] <= gersh[1]


def _gersh(c, p):
    lo, hi, _, _ = c.gershgorin(torch.from_numpy(p.H).cuda())
    return lo, hi


def _solve(c, it):
    D = np.zeros_like(it["p"].H)
    r = c.solve(it["p"].H, it["p"].ne, kT=it["kT"], tol=it["p"].tol, D=D)
    return D, r


def test_certified_bounds_are_tight():
    """Without the hook: the certified interval contains the spectrum and is far
    inside Gershgorin (at most ~1.3x the spectral width for these sizes)."""
    need_gpu()
    import paper_2301_04642_gb300 as fe
    with fe.Context(device=0) as c:
        for it in _problems():
            p = it["p"]
            D, r = _solve(c, it)
            g = _gersh(c, p)
            _check(it, D, r, g)
            width = p.lam[-1] - p.lam[0]
            assert r["eps_max"] - r["eps_min"] <= 1.6 * width
            assert r["eps_max"] - r["eps_min"] < 0.5 * (g[1] - g[0])


@pytest.mark.parametrize("factor", [0.25, 0.6, 0.9])
def test_too_tight_estimate_is_widened(factor):
    need_gpu()
    import paper_2301_04642_gb300 as fe
    with fe.Context(device=0) as c:
        c.narrow_bounds(factor)
        for it in _problems():
            D, r = _solve(c, it)
            _check(it, D, r, _gersh(c, it["p"]))


def test_too_tight_estimate_batch_and_serve():
    need_gpu()
    import paper_2301_04642_gb300 as fe
    items = _problems()
    with fe.Context(device=0) as c:
        c.narrow_bounds(0.4)
        g = [_gersh(c, it["p"]) for it in items]
        outs = [np.zeros_like(it["p"].H) for it in items]
        _, rs = c.solve_batch([dict(H=it["p"].H, ne=it["p"].ne, kT=it["kT"], tol=it["p"].tol, D=D)
                               for it, D in zip(items, outs)])
        for it, D, r, gg in zip(items, outs, rs, g):
            _check(it, D, r, gg)
        outs = [np.zeros_like(it["p"].H) for it in items]
        tickets = [c.submit(it["p"].H, it["p"].ne, kT=it["kT"], tol=it["p"].tol, D=D)
                   for it, D in zip(items, outs)]
        for it, D, t, gg in zip(items, outs, tickets, g):
            _check(it, D, c.wait(t, timeout_s=300), gg)


def test_fp64_precision_certified():
    """The FP64-only schedule certifies with the FP64 product kernel."""
    need_gpu()
    import paper_2301_04642_gb300 as fe
    it = _problems()[2]
    p = it["p"]
    with fe.Context(device=0) as c:
        c.narrow_bounds(0.5)
        D = np.zeros_like(p.H)
        r = c.solve(p.H, p.ne, tol=p.tol, D=D, precision="fp64")
        _check(it, D, r, _gersh(c, p))


def test_narrow_bounds_rejects_bad_factor():
    need_gpu()
    import paper_2301_04642_gb300 as fe
    with fe.Context(device=0) as c:
        for bad in (0.0, -1.0, 1.5, float("nan")):
            with pytest.raises(fe.FeError) as ei:
                c.narrow_bounds(bad)
            assert ei.value.status == fe.FE_EINVAL
