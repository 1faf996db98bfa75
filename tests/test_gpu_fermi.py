"""Finite-temperature expansion through the C ABI against the oracle's exact
Fermi-Dirac density matrix (Sec. II-A).

Tolerances: ||D - D_ref||_F / sqrt(N_e) <= 1e-6, |E_band - E_ref| / N_e <= 1e-7,
|tr D - N_e| <= 1e-9.  D_ref = Q f Q^T from the oracle's own eigensolver at
small n, from the known construction of Hp otherwise (sampled entries and
random probes at the full size)."""
import math

import numpy as np
import pytest

import hp_synth
import oracle
from gpu_util import ctx, torch

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]

TOL_EPS1, TOL_E, TOL_TR = 1e-6, 1e-7, 1e-9


@pytest.mark.parametrize("n,ne,kT,seed", [(300, 255.0, 0.02, 7), (517, 440.5, 0.01, 8),
                                          (1000, 850.0, 0.003, 9), (1500, 1275.0, 0.001, 10)])
def test_fermi_matches_oracle(n, ne, kT, seed):
    p = hp_synth.smeared(n, ne, kT, -2.0, 1.0, seed)
    D = np.zeros_like(p.H)
    r = ctx().solve(p.H, ne, kT=kT, D=D)
    ref = oracle.density(p.H, ne, kT)            # own eigensolver + bisection for mu
    eps1 = np.linalg.norm(D - ref["D"]) / math.sqrt(ne)
    e_err = abs(r["e_band"] - ref["e_band"]) / ne
    print(n, kT, r["iters"], eps1, e_err, r["mu"], ref["mu"])
    assert r["status"] == 0
    assert eps1 <= TOL_EPS1 and e_err <= TOL_E
    assert abs(np.trace(D) - ne) <= TOL_TR
    assert abs(r["trace"] - ne) <= TOL_TR
    assert abs(r["mu"] - ref["mu"]) <= 1e-2 * kT    # chemical potential reported
    # the spectrum of f(Hp) lies in [0, 1]; the split-FP16 rounding of the last
    # stages moves saturated eigenvalues by ~1e-6 (1.3e-6 at kT = 1 mHa)
    ev = np.linalg.eigvalsh(D)
    assert ev.min() > -5e-6 and ev.max() < 1 + 5e-6


def test_fermi_high_temperature_and_device_pointers():
    p = hp_synth.smeared(256, 100.25, 0.5, -2.0, 1.0, 12)
    Hd = torch.from_numpy(p.H).cuda()
    Dd = torch.empty_like(Hd)
    r = ctx().solve(Hd, p.ne, kT=0.5, D=Dd)
    ref = oracle.density(p.H, p.ne, 0.5)
    assert np.linalg.norm(Dd.cpu().numpy() - ref["D"]) / math.sqrt(p.ne) <= TOL_EPS1
    assert abs(r["trace"] - p.ne) <= TOL_TR


def test_fermi_rejects_zero_temperature():
    import paper_2301_04642_gb300 as fe
    p = hp_synth.gapped(64, 32, (-3.0, -0.01), (0.01, 1.0), 3)
    with pytest.raises(fe.FeError) as ei:
        ctx().solve(p.H, 32, kT=0.0, method=fe.FE_METHOD_FERMI)
    assert ei.value.status == fe.FE_EINVAL


def test_fermi_config_n16384():
    """The full finite-temperature workload: n=16384, semicircle [-2, 1] Ha,
    N_e=14000, kT=0.003 Ha.  Checked by the exact trace, the band energy
    against sum f_i lambda_i, sampled entries of Q f Q^T, and ||D - D_ref||_F
    estimated with random probes (E ||(D - D_ref) v||^2 = ||D - D_ref||_F^2)."""
    p = hp_synth.workload_n16384_ft(device="cuda")
    lam = p.lam
    f, mu = oracle.occupations(lam, p.ne, p.kT)
    H = p.H
    D = torch.empty_like(H)
    r = ctx().solve(H, p.ne, kT=p.kT, D=D)
    assert r["status"] == 0
    assert abs(r["trace"] - p.ne) <= TOL_TR
    e_ref = float(np.sum(f * lam))
    assert abs(r["e_band"] - e_ref) / p.ne <= TOL_E
    Q = p.Q.cpu().numpy()
    Dh = D.cpu().numpy()
    rng = np.random.default_rng(5)
    rows, cols = rng.integers(0, p.n, 2000), rng.integers(0, p.n, 2000)
    want = oracle.density_entries(Q, f, rows, cols)
    assert np.abs(Dh[rows, cols] - want).max() <= 1e-6
    V = rng.standard_normal((p.n, 4))
    err = Dh @ V - Q @ (f[:, None] * (Q.T @ V))
    eps1 = math.sqrt(np.sum(err ** 2) / 4) / math.sqrt(p.ne)
    print(r, eps1, abs(r["mu"] - mu))
    assert eps1 <= TOL_EPS1


@pytest.mark.parametrize("n,kT,seed", [(9397, 0.00119, 3134), (13707, 0.0062, 3116)])
def test_fermi_serving_sizes(n, kT, seed):
    """Finite-T requests of the serving mix (semicircle on [-2, 1] Ha,
    N_e = 0.85 n, Q from Householder reflectors), checked on this GPU in FP64
    with 16 Gaussian probes against D_ref = Q diag(f) Q^T of the constructed
    spectrum (f from bisection for mu)."""
    ne = float(round(0.85 * n))
    p = hp_synth.smeared_reflected(n, ne, kT, -2.0, 1.0, seed, device="cuda")
    D = torch.empty_like(p.H)
    r = ctx().solve(p.H, ne, kT=kT, tol=p.tol, D=D)
    assert r["status"] == 0
    assert abs(r["trace"] - ne) <= TOL_TR
    lam = np.asarray(p.lam)
    lo, hi = lam.min() - 1.0, lam.max() + 1.0
    for _ in range(200):
        mu = 0.5 * (lo + hi)
        f = 0.5 * (1.0 - np.tanh((lam - mu) / (2.0 * kT)))
        lo, hi = (lo, mu) if f.sum() > ne else (mu, hi)
    assert abs(r["e_band"] - float(np.dot(f, lam))) / ne <= TOL_E
    fd = torch.from_numpy(f).cuda()
    g = torch.Generator(device="cuda").manual_seed(9)
    V = torch.randn(n, 16, dtype=torch.float64, device="cuda", generator=g)
    err = D @ V - p.Q.mul(fd[:, None] * p.Q.tmul(V))
    eps1 = float(torch.sqrt((err ** 2).sum() / 16)) / math.sqrt(ne)
    print(n, kT, r["iters"], r["iters_by_phase"], eps1)
    assert eps1 <= TOL_EPS1


@pytest.mark.parametrize("kT", [0.001, 0.006])
def test_fermi_nearly_diagonal_hp_matches_oracle(kT):
    """Hp = Q diag(lambda) Q^T with Q from 8 Householder reflectors (diagonal
    plus a rank-16 perturbation, eigenvectors mostly localised): the case in
    which the expansion's diagonal form keeps each near-mu eigenvalue's
    diagonal entry in FP64.  Against the oracle's own eigensolver and
    Fermi-Dirac occupations at n = 1200."""
    n, ne = 1200, 1020.0
    p = hp_synth.smeared_reflected(n, ne, kT, -2.0, 1.0, 91)
    H = np.asarray(p.H.cpu().numpy() if hasattr(p.H, "cpu") else p.H, dtype=np.float64)
    D = np.zeros_like(H)
    r = ctx().solve(H, ne, kT=kT, D=D)
    ref = oracle.density(H, ne, kT)
    eps1 = np.linalg.norm(D - ref["D"]) / math.sqrt(ne)
    print(kT, r["iters"], eps1)
    assert r["status"] == 0
    assert eps1 <= TOL_EPS1 and abs(r["e_band"] - ref["e_band"]) / ne <= TOL_E
    assert abs(np.trace(D) - ne) <= TOL_TR
