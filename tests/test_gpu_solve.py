"""End-to-end solves through the C ABI against the FP64 oracle.

Tolerances (zero temperature): ||D - D_ref||_F / sqrt(N_e) <= 1e-6,
|E_band - E_ref| / N_e <= 1e-7 Ha, |tr D - N_e| <= 1e-9, ||D^2 - D||_F <= 1e-8.
D_ref is the oracle's projector: from its own eigensolver for small n, else
Q f(lambda) Q^T from the known construction of Hp."""
import math

import numpy as np
import pytest

import hp_synth
import oracle
from gpu_util import ctx, torch

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]

TOL_EPS1, TOL_E, TOL_TR, TOL_IDEM = 1e-6, 1e-7, 1e-9, 1e-8


def check_zero_t(p, D, res, use_eig=False, idem=True):
    ne = p.ne
    if use_eig:
        r = oracle.density(p.H, ne)
        Dref, Eref = r["D"], r["e_band"]
    else:
        f = (np.arange(p.n) < int(ne)).astype(float)
        Dref = oracle.density_from_eig(p.Q, f)
        Eref = float(np.sum(f * p.lam))
    eps1 = np.linalg.norm(D - Dref) / math.sqrt(max(ne, 1))
    out = dict(eps1=eps1, e_err=abs(res["e_band"] - Eref) / max(ne, 1),
               tr_err=abs(np.trace(D) - ne))
    if idem:
        D2 = oracle.matmul(D, D)
        out["idem"] = np.linalg.norm(D2 - D)
    return out


def run(p, precision, **kw):
    D = np.zeros_like(p.H)
    res = ctx().solve(p.H, p.ne, tol=p.tol, D=D, precision=precision, **kw)
    return D, res


def test_n256_fp64_config():
    p = hp_synth.workload_n256()
    D, res = run(p, "fp64")
    m = check_zero_t(p, D, res, use_eig=True)
    assert res["status"] == 0
    assert m["eps1"] <= TOL_EPS1 and m["e_err"] <= TOL_E
    assert m["tr_err"] <= TOL_TR and m["idem"] <= TOL_IDEM
    assert 20 <= res["iters"] <= 100
    assert abs(res["trace"] - np.trace(D)) < 1e-9


@pytest.mark.parametrize("n,ne", [(300, 250), (1000, 850), (1250, 1000)])
def test_mixed_medium(n, ne):
    p = hp_synth.gapped(n, ne, (-3.0, -0.01), (0.01, 1.0), 4000 + n)
    D, res = run(p, "mixed")
    m = check_zero_t(p, D, res)
    print(n, res, m)
    assert res["status"] == 0
    assert m["eps1"] <= TOL_EPS1 and m["e_err"] <= TOL_E
    assert m["tr_err"] <= TOL_TR and m["idem"] <= TOL_IDEM


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_paper_matrix_n1000(precision):
    """The paper's own synthetic Hamiltonian (Sec. IV) at N_e = 0.9 n: a
    continuous band whose gap at N_e is 1.4e-3 Ha at n = 1000 (against 3.7 Ha
    of spectrum), far narrower than the gapped workloads'.  D_ref from the
    oracle's own eigensolver.  Measured: mixed eps1 6.2e-7 (44 + 2 products),
    FP64 5.5e-14."""
    p = hp_synth.paper_matrix(1000)
    D, res = run(p, precision)
    m = check_zero_t(p, D, res, use_eig=True)
    print(precision, res["iters_by_phase"], m)
    assert res["status"] == 0
    assert m["eps1"] <= TOL_EPS1 and m["e_err"] <= TOL_E
    assert m["tr_err"] <= TOL_TR and m["idem"] <= TOL_IDEM


@pytest.mark.parametrize("n,ne", [(300, 250), (1000, 850), (2000, 1500)])
def test_try_fp16_reports_its_error(n, ne):
    """Single FP16 products while RelTr >= 5e-4 (Sec. III-A's switch point),
    then split products, then the FP64-accurate polish.  The polish restores
    the trace and idempotency, but not the subspace: an FP16 product error
    E at step k turns the occupied subspace by about |E_ij| / (x_i - x_j)
    between states on either side of the gap, SP2 keeps whatever subspace it
    is given, and the early steps, where the gap is still narrow in x, are
    the worst.  So this schedule misses ||D - D_ref||_F / sqrt(N_e) <= 1e-6 on
    gapped inputs (measured ~3e-4 at n = 300); the bound checked here is the
    one it meets."""
    p = hp_synth.gapped(n, ne, (-3.0, -0.01), (0.01, 1.0), 4100 + n)
    D, res = run(p, "try_fp16")
    m = check_zero_t(p, D, res)
    print(n, res, m)
    assert res["status"] == 0
    assert res["iters_by_phase"][0] > 0 and res["iters_by_phase"][1] > 0
    assert m["eps1"] <= 2e-3
    assert m["tr_err"] <= TOL_TR and m["idem"] <= TOL_IDEM


def test_fp32_schedule_reports_its_error():
    p = hp_synth.gapped(600, 500, (-3.0, -0.01), (0.01, 1.0), 77)
    D, res = run(p, "fp32")
    m = check_zero_t(p, D, res, idem=False)
    print(res, m)
    assert res["status"] == 0
    assert m["eps1"] <= 1e-5          # FP32-class: no FP64 polish


def test_device_pointers_and_ld():
    p = hp_synth.gapped(500, 400, (-3.0, -0.01), (0.01, 1.0), 11)
    ld = 512
    Hd = torch.zeros((p.n, ld), dtype=torch.float64, device="cuda")
    Hd[:, :p.n] = torch.from_numpy(p.H).cuda()
    Dd = torch.full((p.n, ld), 5.0, dtype=torch.float64, device="cuda")
    res = ctx().solve(Hd[:, :p.n], p.ne, D=Dd[:, :p.n], precision="mixed")
    Dh = Dd.cpu().numpy()
    assert np.all(Dh[:, p.n:] == 5.0)
    m = check_zero_t(p, Dh[:, :p.n].copy(), res)
    assert m["eps1"] <= TOL_EPS1 and m["idem"] <= TOL_IDEM


def test_degenerate_occupations():
    p = hp_synth.gapped(200, 200, (-3.0, -0.01), (0.01, 1.0), 12)
    D, res = run(p, "mixed")
    assert np.abs(D - np.eye(200)).max() < 1e-10
    p = hp_synth.gapped(200, 0, (-3.0, -0.01), (0.01, 1.0), 12)
    D, res = run(p, "mixed")
    assert np.abs(D).max() < 1e-10


def test_permutation_and_shift_covariance():
    p = hp_synth.gapped(400, 300, (-3.0, -0.01), (0.01, 1.0), 31)
    D, _ = run(p, "mixed")
    perm = np.random.default_rng(0).permutation(400)
    Hp = p.H[np.ix_(perm, perm)]
    D2 = np.zeros_like(Hp)
    ctx().solve(Hp, p.ne, D=D2, precision="mixed")
    assert np.linalg.norm(D2 - D[np.ix_(perm, perm)]) / math.sqrt(300) < 2 * TOL_EPS1
    D3 = np.zeros_like(Hp)
    ctx().solve(p.H + 0.7 * np.eye(400), p.ne, D=D3, precision="mixed")
    assert np.linalg.norm(D3 - D) / math.sqrt(300) < 2 * TOL_EPS1


def test_invalid_inputs():
    import paper_2301_04642_gb300 as fe
    p = hp_synth.gapped(64, 32, (-3.0, -0.01), (0.01, 1.0), 3)
    H = p.H.copy(); H[5, 5] = np.inf
    with pytest.raises(fe.FeError) as ei:
        ctx().solve(H, 32)
    assert ei.value.status == fe.FE_EINVAL
    with pytest.raises(fe.FeError) as ei:
        ctx().solve(p.H, 32.5)                # non-integral N_e at kT = 0
    assert ei.value.status == fe.FE_EINVAL
    with pytest.raises(fe.FeError) as ei:
        ctx().solve(p.H, 65)
    assert ei.value.status == fe.FE_EINVAL


def test_iteration_cap_reports_notconv():
    import paper_2301_04642_gb300 as fe
    p = hp_synth.gapped(256, 128, (-3.0, -0.01), (0.01, 1.0), 8)
    with fe.Context(max_iters=3) as c:
        r = c.solve(p.H, p.ne, check=False)
    assert r["status"] == fe.FE_ENOTCONV


def test_config_n4096_mixed():
    p = hp_synth.workload_n4096()
    D, res = run(p, "mixed")
    f = (np.arange(p.n) < 3500).astype(float)
    Dref = oracle.density_from_eig(p.Q, f)
    eps1 = np.linalg.norm(D - Dref) / math.sqrt(3500)
    e_err = abs(res["e_band"] - np.sum(f * p.lam)) / 3500
    tr_err = abs(np.trace(D) - 3500)
    # idempotency through 4 random probes: E||(D^2 - D) v||^2 = ||D^2 - D||_F^2
    rng = np.random.default_rng(1)
    V = rng.standard_normal((p.n, 4))
    DV = D @ V
    idem = math.sqrt(np.sum((D @ DV - DV) ** 2) / 4)
    print(res, eps1, e_err, tr_err, idem)
    assert res["status"] == 0
    assert eps1 <= TOL_EPS1 and e_err <= TOL_E and tr_err <= TOL_TR and idem <= TOL_IDEM


def test_config_n16384_mixed():
    """The zero-temperature schedule at n = 16384 (gap 0.02 Ha in a spectrum
    4 Ha wide: a slowly converging eigenvalue next to the gap).
    Checked by the exact trace, the band energy, sampled entries of the
    constructed projector, and ||D - D_ref||_F and ||D^2 - D||_F estimated with
    random probes (E ||A v||^2 = ||A||_F^2 for v ~ N(0, I))."""
    n, ne = 16384, 13926
    p = hp_synth.gapped(n, ne, (-3.0, -0.01), (0.01, 1.0), 1004, device="cuda")
    D = torch.empty_like(p.H)
    r = ctx().solve(p.H, ne, tol=p.tol, D=D)
    assert r["status"] == 0
    f = (np.arange(n) < ne).astype(float)
    assert abs(r["trace"] - ne) <= TOL_TR
    assert abs(r["e_band"] - float(np.sum(f * p.lam))) / ne <= TOL_E
    Q = p.Q.cpu().numpy()
    Dh = D.cpu().numpy()
    assert abs(np.trace(Dh) - ne) <= TOL_TR
    rng = np.random.default_rng(6)
    rows, cols = rng.integers(0, n, 2000), rng.integers(0, n, 2000)
    want = oracle.density_entries(Q, f, rows, cols)
    assert np.abs(Dh[rows, cols] - want).max() <= 1e-6
    V = rng.standard_normal((n, 4))
    DV = Dh @ V
    err = DV - Q @ (f[:, None] * (Q.T @ V))
    eps1 = math.sqrt(np.sum(err ** 2) / 4) / math.sqrt(ne)
    idem = math.sqrt(np.sum((Dh @ DV - DV) ** 2) / 4)
    print(r, eps1, idem)
    assert eps1 <= TOL_EPS1 and idem <= TOL_IDEM


def test_pinned_host_output_matches_staged():
    """A page-locked host D is written by the output kernel directly; the
    result is the one the staged copy of a pageable D receives, bit for bit."""
    p = hp_synth.gapped(700, 500, (-3.0, -0.01), (0.01, 1.0), 4700)
    Dpin = torch.empty(p.n, p.n, dtype=torch.float64).pin_memory()
    Dpin.fill_(np.nan)
    r1 = ctx().solve(p.H, p.ne, tol=p.tol, D=Dpin.numpy())
    D2 = np.zeros_like(p.H)
    r2 = ctx().solve(p.H, p.ne, tol=p.tol, D=D2)
    assert r1["status"] == 0 and r2["status"] == 0
    assert np.array_equal(Dpin.numpy(), D2)
    m = check_zero_t(p, D2, r2)
    assert m["eps1"] <= TOL_EPS1 and m["tr_err"] <= TOL_TR and m["idem"] <= TOL_IDEM
    # a row stride wider than n: only the n x n block is written
    big = torch.full((p.n, p.n + 5), -7.0, dtype=torch.float64).pin_memory()
    Hw = np.zeros((p.n, p.n + 5))
    Hw[:, :p.n] = p.H
    r3 = ctx().solve(Hw[:, :p.n], p.ne, tol=p.tol, D=big.numpy()[:, :p.n])
    assert r3["status"] == 0
    assert np.array_equal(big.numpy()[:, :p.n], D2)
    assert np.all(big.numpy()[:, p.n:] == -7.0)


@pytest.mark.parametrize("kind,precision", [("degenerate", "mixed"), ("gap1e-5", "mixed"), ("gap1e-5", "fp64")])
def test_unresolvable_gap_reports_notconv_or_meets_tolerances(kind, precision):
    """A Fermi level that the products can hardly resolve: a two-fold
    degenerate HOMO split by N_e (D is not unique, Sec. II-A needs a gap), or
    a gap of 1e-5 Ha in a 4 Ha spectrum.  A solve that reports success must
    meet the trace, idempotency and band-energy tolerances (the polish
    reports FE_ENOTCONV when it cannot reach them).  The subspace itself is
    set by the early products: split-FP16 rounding (2^-22) over an x-gap of
    2.5e-6 turns it by ~1e-5, which the mixed schedule cannot see from traces
    (measured eps1 1.3e-5 at gap 1e-5); the FP64 schedule meets eps1 too."""
    import paper_2301_04642_gb300 as fe
    n, ne = 400, 300
    lam = hp_synth.gapped_spectrum(n, ne, (-3.0, -0.01), (0.01, 1.0), 77)
    if kind == "degenerate":
        lam[ne] = lam[ne - 1]
    else:
        lam[ne] = lam[ne - 1] + 1e-5
    lam = np.sort(lam)
    Q = hp_synth.haar_q(n, 78)
    H = hp_synth.assemble(Q, lam)
    D = np.zeros_like(H)
    r = ctx().solve(H, ne, D=D, check=False, precision=precision)
    print(kind, precision, r["status"], r["iters_by_phase"])
    if r["status"] == fe.FE_ENOTCONV:
        return
    assert r["status"] == 0
    p = hp_synth.Problem(kind, H, Q, lam, float(ne), 0.0, 5e-8, 77)
    m = check_zero_t(p, D, r)
    print(m)
    assert m["e_err"] <= TOL_E and m["tr_err"] <= TOL_TR and m["idem"] <= TOL_IDEM
    if kind == "degenerate" or precision == "fp64":
        assert m["eps1"] <= TOL_EPS1
    else:
        assert m["eps1"] <= 1e-4


@pytest.mark.parametrize("n,gap,seed", [(10278, 0.0565, 3110), (16040, 0.0550, 3115)])
def test_polish_ends_at_large_n(n, gap, seed):
    """Gapped problems of the serving mix (N_e = 0.85 n, Q from Householder
    reflectors).  At these sizes t1 - t2 after the polishing pairs is a few
    ulp(N_e) below zero from the rounding of the two FP64 sums: the stopping
    test must accept it (these ended with FE_ENOTCONV while D met every
    tolerance).  Checked with probes on this GPU in FP64 against
    D_ref = Q diag(f) Q^T of the constructed spectrum."""
    ne = int(round(0.85 * n))
    p = hp_synth.gapped_reflected(n, ne, (-3.0, -gap / 2), (gap / 2, 1.0), seed, device="cuda")
    D = torch.empty_like(p.H)
    r = ctx().solve(p.H, ne, tol=p.tol, D=D)
    assert r["status"] == 0
    assert r["iters_by_phase"][2] <= 4                   # two polishing pairs at most
    f = torch.from_numpy((np.arange(n) < ne).astype(float)).cuda()
    assert abs(r["trace"] - ne) <= TOL_TR
    assert abs(r["e_band"] - float(np.sum((np.arange(n) < ne) * p.lam))) / ne <= TOL_E
    g = torch.Generator(device="cuda").manual_seed(5)
    V = torch.randn(n, 4, dtype=torch.float64, device="cuda", generator=g)
    DV = D @ V
    err = DV - p.Q.mul(f[:, None] * p.Q.tmul(V))
    eps1 = float(torch.sqrt((err ** 2).sum() / 4)) / math.sqrt(ne)
    idem = float(torch.sqrt(((D @ DV - DV) ** 2).sum() / 4))
    print(r["iters_by_phase"], eps1, idem)
    assert eps1 <= TOL_EPS1 and idem <= TOL_IDEM
