"""Pins for the CPU oracle against closed forms, invariants, brute force and
independent library routines (no GPU).

Every oracle function is exercised by at least one check here that a dropped
term, a wrong sign/index or a transposed operand would break."""
import json
import math
import os

import numpy as np
import pytest

import hp_synth
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def sym_random(n, seed):
    G = hp_synth.normal(seed, n * n).reshape(n, n)
    return 0.5 * (G + G.T)


# ---------------------------------------------------------------- generator

def test_splitmix64_reference_vector():
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.startswith("0x")]
    got = [int(x) for x in hp_synth.splitmix64(0, 3)]
    assert got == want


def test_generator_is_exact_similarity():
    p = hp_synth.gapped(64, 50, (-2, -0.05), (0.05, 0.6), 7)
    assert np.abs(p.Q.T @ p.Q - np.eye(64)).max() < 1e-13
    assert np.abs(p.H @ p.Q - p.Q * p.lam[None, :]).max() < 1e-12
    assert p.lam[49] == -0.05 and p.lam[50] == 0.05      # pinned gap edges


def test_semicircle_moments():
    lam = hp_synth.semicircle_spectrum(200000, -1.0, 1.0, 3)
    # semicircle on [-1, 1]: mean 0, variance 1/4
    assert abs(lam.mean()) < 5e-3 and abs(lam.var() - 0.25) < 5e-3
    assert lam.min() >= -1 and lam.max() <= 1


def test_paper_matrix_entries():
    """The paper's synthetic Hamiltonian (Sec. IV), read as symmetric with the
    smaller index inside the sine: entries written out by hand."""
    p = hp_synth.paper_matrix(40)
    H = p.H
    assert H.shape == (40, 40) and p.ne == 36.0 and p.Q is None and p.n == 40
    assert np.array_equal(H, H.T)
    assert H[0, 0] == math.sin(1.0)
    assert H[7, 7] == math.sin(8.0)
    assert abs(H[2, 5] - math.exp(-1.5) * math.sin(3.0)) < 1e-16
    assert abs(H[5, 2] - math.exp(-1.5) * math.sin(3.0)) < 1e-16
    assert abs(H[0, 39] - math.exp(-19.5) * math.sin(1.0)) < 1e-22
    assert hp_synth.paper_matrix(100, 0.85).ne == 85.0


# ---------------------------------------------------------------- eigensolvers

@pytest.mark.parametrize("solver", [oracle.eigh_ql, oracle.eigh_jacobi])
def test_eigh_2x2_closed_form(solver):
    a, b, c = 0.3, -1.7, 2.2
    w, Q = solver(np.array([[a, b], [b, c]]))
    m, r = 0.5 * (a + c), math.hypot(0.5 * (a - c), b)
    assert np.allclose(w, [m - r, m + r], atol=1e-14)
    # eigenvector of lambda: (b, lambda - a) normalised
    for k in range(2):
        v = np.array([b, w[k] - a]); v /= np.linalg.norm(v)
        assert abs(abs(v @ Q[:, k]) - 1) < 1e-13


@pytest.mark.parametrize("solver", [oracle.eigh_ql, oracle.eigh_jacobi])
def test_eigh_diagonal(solver):
    d = np.array([3.0, -1.0, 0.5, 2.0, -4.0])
    w, Q = solver(np.diag(d))
    assert np.array_equal(w, np.sort(d))
    assert np.allclose(np.abs(Q), np.abs(Q).round())     # a permutation


def test_eigh_brute_force_small():
    # n <= 4: eigenvalues are the roots of det(H - x I); check the oracle's
    # eigenvalues make the determinant vanish and the count below each
    # midpoint (Sylvester inertia of H - x I by elimination) is right.
    for n in (3, 4):
        H = sym_random(n, 11 + n)
        w, _ = oracle.eigh_ql(H)
        scale = np.abs(H).sum()
        for x in w:
            assert abs(np.linalg.det(H - x * np.eye(n))) < 1e-12 * scale ** n
        for k in range(n - 1):
            x = 0.5 * (w[k] + w[k + 1])
            A = H - x * np.eye(n)
            neg = 0
            for i in range(n):                     # plain LDL^T pivots
                piv = A[i, i]
                neg += piv < 0
                A[i + 1:, i + 1:] -= np.outer(A[i + 1:, i], A[i, i + 1:]) / piv
            assert neg == k + 1


def test_eigh_ql_vs_jacobi_vs_lapack():
    H = sym_random(120, 5)
    wq, Qq = oracle.eigh_ql(H)
    wj, Qj = oracle.eigh_jacobi(H)
    wl = np.linalg.eigvalsh(H)                       # independent library routine
    assert np.abs(wq - wj).max() < 1e-12 * np.abs(wl).max()
    assert np.abs(wq - wl).max() < 1e-12 * np.abs(wl).max()
    assert np.abs(H @ Qq - Qq * wq).max() < 1e-12 * np.abs(wl).max()
    assert np.abs(Qq.T @ Qq - np.eye(120)).max() < 1e-13


def test_eigh_ql_constructed():
    p = hp_synth.gapped(300, 250, (-2, -0.05), (0.05, 0.6), 1001)
    w, Q = oracle.eigh_ql(p.H)
    assert np.abs(w - p.lam).max() < 1e-13
    assert np.abs(p.H @ Q - Q * w).max() < 1e-13


# ---------------------------------------------------------------- occupations / D

def test_occupations_step_and_fd_diagonal():
    w = np.array([-1.0, -0.5, 0.0, 0.4, 1.0])
    f, mu = oracle.occupations(w, 3, 0.0)
    assert list(f) == [1, 1, 1, 0, 0] and mu == 0.2
    kT = 0.05
    f, mu = oracle.occupations(w, 2.5, kT)
    assert abs(f.sum() - 2.5) < 1e-12
    want = 1.0 / (1.0 + np.exp((w - mu) / kT))
    assert np.abs(f - want).max() < 1e-15


def test_fermi_overflow_safe_and_symmetric():
    assert oracle.fermi(1e4, 0.0, 1e-3) == 0.0
    assert oracle.fermi(-1e4, 0.0, 1e-3) == 1.0
    for x in (0.3, 1.7, 12.0):
        assert abs(oracle.fermi(x, 0, 1) + oracle.fermi(-x, 0, 1) - 1) < 1e-15


def test_fd_low_temperature_limit_is_step():
    p = hp_synth.gapped(80, 60, (-2, -0.05), (0.05, 0.6), 9)
    r0 = oracle.density(p.H, 60, 0.0)
    r1 = oracle.density(p.H, 60, 1e-4)               # kT << gap/2
    assert np.abs(r0["D"] - r1["D"]).max() < 1e-12


def test_zero_t_density_invariants():
    p = hp_synth.gapped(200, 160, (-2, -0.05), (0.05, 0.6), 17)
    r = oracle.density(p.H, 160)
    D = r["D"]
    assert np.abs(D @ D - D).max() < 1e-13                 # idempotent
    assert abs(np.trace(D) - 160) < 1e-11                  # tr D = N_e
    assert np.abs(p.H @ D - D @ p.H).max() < 1e-12         # commutes with H
    Dc = oracle.density_from_eig(p.Q, (p.lam < 0).astype(float))
    assert np.abs(D - Dc).max() < 1e-12                    # construction
    assert abs(r["e_band"] - p.lam[:160].sum()) < 1e-12
    assert abs(r["e_band"] - np.sum(p.H * D)) < 1e-11      # tr(H D)


def test_finite_t_density_invariants():
    p = hp_synth.smeared(150, 120.5, 0.02, -2.0, 1.0, 23)
    r = oracle.density(p.H, 120.5, 0.02)
    D = r["D"]
    assert abs(np.trace(D) - 120.5) < 1e-10
    assert np.abs(p.H @ D - D @ p.H).max() < 1e-12
    ev = np.linalg.eigvalsh(D)
    assert ev.min() > -1e-13 and ev.max() < 1 + 1e-13
    want = 1.0 / (1.0 + np.exp((p.lam - r["mu"]) / 0.02))
    Dc = oracle.density_from_eig(p.Q, want)
    assert np.abs(D - Dc).max() < 1e-12


def test_density_entries_match_full():
    p = hp_synth.gapped(40, 30, (-2, -0.05), (0.05, 0.6), 5)
    f = (p.lam < 0).astype(float)
    D = oracle.density_from_eig(p.Q, f)
    rows, cols = [0, 3, 39, 17], [0, 20, 1, 17]
    assert np.abs(oracle.density_entries(p.Q, f, rows, cols) - D[rows, cols]).max() < 1e-15


# ---------------------------------------------------------------- Gershgorin, matmul

def test_gershgorin():
    H = np.array([[2.0, -1.0, 0.5], [-1.0, 0.0, 0.25], [0.5, 0.25, -3.0]])
    lo, hi = oracle.gershgorin(H)
    assert lo == min(2 - 1.5, 0 - 1.25, -3 - 0.75) and hi == max(2 + 1.5, 1.25, -3 + 0.75)
    p = hp_synth.gapped(100, 80, (-2, -0.05), (0.05, 0.6), 3)
    lo, hi = oracle.gershgorin(p.H)
    assert lo <= p.lam[0] and hi >= p.lam[-1]


def test_matmul_vs_library():
    A, B = sym_random(70, 1), sym_random(70, 2)
    B[3, 5] += 1.0                                    # non-symmetric B catches a transpose
    assert np.abs(oracle.matmul(A, B) - A @ B).max() < 1e-12


# ---------------------------------------------------------------- SP2

def test_sp2_reaches_projector_config_n256():
    p = hp_synth.workload_n256()
    X, it, br = oracle.sp2(p.H, p.ne, tol=p.tol)
    Dref = oracle.density_from_eig(p.Q, (np.arange(256) < 200).astype(float))
    assert it > 0
    # The RelTr stop leaves a small idempotency residual; the paper reports
    # eps1 of order 1e-10 for FP64 (Sec. IV).  More products remove it.
    assert np.linalg.norm(X - Dref) / math.sqrt(200) < 1e-9
    assert abs(np.trace(X) - 200) < 1e-8
    X2, it2, _ = oracle.sp2(p.H, p.ne, tol=0.0, max_iter=it + 4)
    assert np.linalg.norm(X2 - Dref) / math.sqrt(200) < 1e-12
    band = json.load(open(os.path.join(GOLDEN, "paper_sanity_bands.json")))
    # the paper reports ~50 products at RelTr 5e-8 (Sec. IV); same order here
    assert 0.5 * band["sp2_fp64_iterations_approx"] <= it <= 2 * band["sp2_fp64_iterations_approx"]
    assert set(np.unique(br)) == {0, 1}


def test_sp2_branch_rule_moves_trace_toward_ne():
    p = hp_synth.gapped(96, 70, (-2, -0.05), (0.05, 0.6), 41)
    X0, _, _ = oracle.sp2(p.H, p.ne, max_iter=0)
    for k in range(6):
        X, _, br = oracle.sp2(p.H, p.ne, tol=1e-300, max_iter=k + 1)
        t1, t2 = np.trace(X0), np.sum(X0 * X0)
        # the rule picks the candidate whose trace is nearer N_e
        assert br[k] == (abs(t2 - 70) <= abs(2 * t1 - t2 - 70))
        X0 = X


def test_sp2_degenerate_counts():
    p = hp_synth.gapped(50, 50, (-2, -0.05), (0.05, 0.6), 2)     # every state occupied
    X, it, _ = oracle.sp2(p.H, 50, tol=1e-12)
    assert np.abs(X - np.eye(50)).max() < 1e-10
    p = hp_synth.gapped(50, 0, (-2, -0.05), (0.05, 0.6), 2)      # no electrons
    X, it, _ = oracle.sp2(p.H, 0.0, tol=1e-12, max_iter=80)
    assert np.abs(X).max() < 1e-10


# ---------------------------------------------------------------- accelerated SP2 (A-Z-RFOE reading)

def test_sp2_accel_first_step_on_diagonal_by_hand():
    """H = diag(-1, -0.6, 0.2, 1), N_e = 2: Gershgorin bounds [-1, 1], X0 =
    diag(1, 0.8, 0.4, 0); HOMO -0.6 and LUMO 0.2 give a = 0.4, b = 0.8.
    The gap (a, b) lies above the middle (a + b = 1.2 > 1): the X^2 branch
    (the trace rule agrees: t1 = 2.2, t2 = 1.8, |t2 - 2| = 0.2 <
    |2 t1 - t2 - 2| = 0.6), folded at s = a/2 = 0.2 (b - a = 0.4, no cap):
    p(x) = ((x - 0.2)/0.8)^2, so X1 = diag(1, 9/16, 1/16, 1/16) (p(0) = p(a):
    the unoccupied interval is folded onto itself)."""
    H = np.diag([-1.0, -0.6, 0.2, 1.0])
    X, it, br = oracle.sp2_accel(H, 2.0, -0.6, 0.2, max_iter=1)
    assert it == -1 and list(br) == [1]
    assert np.allclose(X, np.diag([1.0, 9 / 16, 1 / 16, 1 / 16]), rtol=0, atol=1e-15)


def test_sp2_accel_without_gap_information_is_sp2():
    """Bounds that do not bracket a gap leave the shift at 0: every step is
    the SP2 step, bit for bit."""
    p = hp_synth.gapped(80, 60, (-2, -0.05), (0.05, 0.6), 11)
    X0, it0, br0 = oracle.sp2(p.H, p.ne, tol=1e-12)
    X1, it1, br1 = oracle.sp2_accel(p.H, p.ne, 0.3, 0.3, tol=1e-12)
    assert it1 == it0 and np.array_equal(br1, br0) and np.array_equal(X1, X0)


@pytest.mark.parametrize("make", [lambda: hp_synth.paper_matrix(400),
                                  lambda: hp_synth.gapped(300, 250, (-3.0, -0.01), (0.01, 1.0), 7)])
def test_sp2_accel_reaches_projector_in_fewer_products(make):
    """With the exact HOMO/LUMO the folded recursion reaches the same
    projector as SP2 in about 40% fewer products (the paper reports about
    30 against 50, Sec. IV); with estimates inside the gap but 40% short of
    each edge it still converges, in between.  Estimates outside the gap
    (five gaps too wide) are not what the folds need: the recursion either
    still lands on the projector or reports the estimates as inconsistent
    (-2), never a wrong projector."""
    p = make()
    ne = int(p.ne)
    w = np.linalg.eigvalsh(p.H)          # the library routine only supplies the estimates
    h, l = w[ne - 1], w[ne]
    D = oracle.density(p.H, p.ne)["D"]
    _, it0, _ = oracle.sp2(p.H, p.ne, tol=1e-12)
    X, it, _ = oracle.sp2_accel(p.H, p.ne, h, l, tol=1e-12)
    assert it > 0 and np.abs(X - D).max() < 1e-9
    assert it <= 0.7 * it0
    g = l - h
    Xi, iti, _ = oracle.sp2_accel(p.H, p.ne, h + 0.4 * g, l - 0.4 * g, tol=1e-12)
    assert iti > 0 and np.abs(Xi - D).max() < 1e-9
    assert it <= iti <= it0
    Xl, itl, _ = oracle.sp2_accel(p.H, p.ne, h - 5 * g, l + 5 * g, tol=1e-12)
    assert itl == -2 or (itl > 0 and np.abs(Xl - D).max() < 1e-9)


@pytest.mark.parametrize("shift", [-1, 1, 2])
def test_sp2_accel_flags_misplaced_estimates(shift):
    """Estimates that put the gap between the wrong pair of states (`shift`
    states up or down) cannot give the projector onto the N_e lowest states:
    the trace bounds N_e b <= tr X <= N_e + (n - N_e) a (or the spread bound
    on tr(X - X^2)) fail by a whole state, and the oracle returns -2 within
    about as many products as SP2 takes."""
    p = hp_synth.gapped(200, 150, (-3.0, -0.02), (0.02, 1.0), 21)
    ne = 150
    lam = p.lam
    h, l = lam[ne - 1 + shift], lam[ne + shift]
    _, it0, _ = oracle.sp2(p.H, p.ne, tol=1e-12)
    _, it, _ = oracle.sp2_accel(p.H, p.ne, h + 0.1 * (l - h), l - 0.1 * (l - h), tol=1e-12, max_iter=200)
    assert it == -2
    assert oracle.sp2_accel_status(it) == "inconsistent"


def test_sp2_accel_branch_follows_the_bounds_and_caps_the_fold():
    """Two steps by hand.  H = diag(-1, -0.9, -0.8, 0.9, 1), N_e = 3,
    bounds [-1, 1]: X0 = diag(1, 0.95, 0.9, 0.05, 0); HOMO -0.8, LUMO -0.79
    give a = 0.895, b = 0.9 (gap 0.005 < 1e-2).  a + b > 1: X^2, whose fold
    s = a/2 = 0.4475 is capped at 1/4: p(x) = ((x - 1/4)/(3/4))^2 gives
    X1 = diag(1, 196/225, 169/225, 16/225, 1/9) (the fold puts 0 above
    0.05), a1 = p(a) = 0.7396, b1 = p(b) = 0.75111.  Again a1 + b1 > 1, now
    with b1 - a1 = 0.0115 >= 1e-2: X^2 folded at the uncapped s = a1/2."""
    H = np.diag([-1.0, -0.9, -0.8, 0.9, 1.0])
    X, it, br = oracle.sp2_accel(H, 3.0, -0.8, -0.79, max_iter=1)
    x1 = np.array([225.0, 196.0, 169.0, 16.0, 25.0]) / 225.0
    assert it == -1 and list(br) == [1]
    assert np.allclose(np.diag(X), x1, rtol=0, atol=1e-15)
    a1 = (0.895 - 0.25) ** 2 / 0.5625
    s2 = a1 / 2
    X2, it2, br2 = oracle.sp2_accel(H, 3.0, -0.8, -0.79, max_iter=2)
    assert list(br2) == [1, 1]
    assert np.allclose(np.diag(X2), ((x1 - s2) / (1 - s2)) ** 2, rtol=0, atol=1e-14)


def test_sp2_accel_estimates_inside_the_gap_are_never_flagged():
    """Random gapped problems (n, N_e, gap, spectral scaling) with HOMO/LUMO
    estimates drawn anywhere inside the true gap: every one converges to the
    projector; the consistency test never fires on valid estimates."""
    rng = np.random.default_rng(5)
    for t in range(12):
        n = int(rng.integers(40, 160))
        ne = int(rng.integers(1, n))
        gap = 10 ** rng.uniform(-3, -0.7)
        p = hp_synth.gapped(n, ne, (-3.0, -gap / 2), (gap / 2, 1.0), 600 + t)
        h, l = p.lam[ne - 1], p.lam[ne]
        u = np.sort(rng.uniform(0.0, 1.0, 2))
        hh, ll = h + u[0] * (l - h), h + max(u[1], u[0] + 1e-3) * (l - h)
        X, it, _ = oracle.sp2_accel(p.H, p.ne, hh, ll, tol=1e-12)
        f = (np.arange(n) < ne).astype(float)
        assert it > 0, (t, n, ne, gap, u)
        assert np.abs(X - oracle.density_from_eig(p.Q, f)).max() < 1e-8


# ---------------------------------------------------------------- products either side

def test_gemm_against_library_and_closed_forms():
    """op(A) op(B) against numpy on rectangular and transposed operands, and
    two closed forms of the subspace-iteration products: for Psi with
    orthonormal columns Psi^T Psi = I, and with H Psi = Psi diag(lam) the
    projection Psi^T (H Psi) = diag(lam); rotating by D = I returns Psi."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((37, 21))
    B = rng.standard_normal((21, 13))
    assert np.allclose(oracle.gemm(A, B), A @ B, rtol=0, atol=1e-12)
    assert np.allclose(oracle.gemm(A, A, ta=True), A.T @ A, rtol=0, atol=1e-12)
    assert np.allclose(oracle.gemm(B, B, tb=True), B @ B.T, rtol=0, atol=1e-12)
    assert np.allclose(oracle.gemm(B, A, ta=True, tb=True), (A @ B).T, rtol=0, atol=1e-12)
    Psi = hp_synth.haar_q(60, 4)[:, :17]
    assert np.abs(oracle.gemm(Psi, Psi, ta=True) - np.eye(17)).max() < 1e-14
    lam = np.linspace(-2.0, 1.0, 17)
    assert np.abs(oracle.gemm(Psi, Psi * lam[None, :], ta=True) - np.diag(lam)).max() < 1e-14
    assert np.array_equal(oracle.gemm(Psi, np.eye(17)), Psi)
    # by hand: [[1, 2], [3, 4]]^T [[5], [6]] = [[23], [34]]
    assert np.array_equal(oracle.gemm(np.array([[1.0, 2.0], [3.0, 4.0]]), np.array([[5.0], [6.0]]), ta=True),
                          np.array([[23.0], [34.0]]))


# ---------------------------------------------------------------- truncated SP2 at finite T

def _apply_branches(x, branches):
    """The SP2 maps of Eq. (1) applied in the given order to scalars."""
    x = np.array(x, dtype=float)
    for b in branches:
        x = x * x if b else 2.0 * x - x * x
    return x


def test_trfoe_first_steps_by_hand():
    """H = diag(-1, -0.5, 0.5, 1), N_e = 2, bounds [-1, 1] (w = 2):
    x0 = (1, 0.75, 0.25, 0).  At step 0 the slope is 1/w = 0.5, so beta = 1
    (beta/4 = 0.25) stops at once with mu = 0.  With beta = 4 (beta/4 = 1):
    t1 = 2, t2 = 1.625 is a tie (0.375 either way) and goes to X^2: x1 =
    (1, 0.5625, 0.0625, 0), midpoint u0 = sqrt(1/2), slope 2 u0 / 2 =
    0.7071 < 1; then t1 = 1.625, t2 = 1.3203125 pick 2X - X^2 (|t2 - 2| =
    0.68 > |2 t1 - t2 - 2| = 0.0703): u1 = 1 - sqrt(1/2), u0 = sqrt(u1),
    slope (2 - 2 u1) (2 u0) / 2 = 0.7654 < 1; and so on."""
    lam = np.array([-1.0, -0.5, 0.5, 1.0])
    g, m, br, mu = oracle.trfoe(lam, 2.0, 1.0, -1.0, 1.0)
    assert m == 0 and mu == 0.0 and np.array_equal(g, [1.0, 0.75, 0.25, 0.0])
    g2, m2, br2, _ = oracle.trfoe(lam, 2.0, 0.25, -1.0, 1.0, max_iter=2)
    assert m2 == -1 and list(br2[:2]) == [1, 0]  # cap reached before the slope
    assert np.allclose(g2, [1.0, 0.80859375, 0.12109375, 0.0], rtol=0, atol=1e-15)


def test_trfoe_stop_rule_against_finite_differences():
    """The stop rule compares |dG_m/de| at the midpoint G_m = 1/2 with
    beta/4.  Here G_k is evaluated by applying the recorded branches to
    energies on a grid, its midpoint found by bisection and its slope by a
    central difference (no use of the closed-form inverses): the slope after
    m - 1 steps is below beta/4 and after m steps at or above it, and the
    reported mu is the midpoint of G_m."""
    p = hp_synth.smeared(300, 240.0, 0.004, -2.0, 1.0, 51)
    lo, hi = oracle.gershgorin(p.H)
    w = hi - lo
    beta = 1.0 / p.kT
    g, m, br, mu = oracle.trfoe(p.lam, p.ne, p.kT, lo, hi)
    assert m > 5

    def G(eps, k):
        return _apply_branches((hi - np.asarray(eps)) / w, br[:k])

    def midpoint_and_slope(k):
        a, b = lo, hi                        # G_k falls from 1 at lo to 0 at hi
        for _ in range(200):
            c = 0.5 * (a + b)
            if G(c, k) > 0.5:
                a = c
            else:
                b = c
        c = 0.5 * (a + b)
        h = 1e-7 * w
        return c, abs(G(c + h, k) - G(c - h, k)) / (2 * h)

    c_prev, s_prev = midpoint_and_slope(m - 1)
    c_m, s_m = midpoint_and_slope(m)
    assert s_prev < beta / 4 <= s_m * (1 + 1e-6)
    assert abs(c_m - mu) <= 1e-9 * w
    assert np.allclose(g, G(p.lam, m), rtol=0, atol=1e-14)


def test_trfoe_matrix_recursion_equals_scalar_on_eigenvalues():
    """The recursion is polynomial in H, so the matrix form (traces of the
    matrix deciding each branch, plain numpy products) equals
    Q diag(G_m(x(lambda))) Q^T with the oracle's branches."""
    p = hp_synth.smeared(120, 100.0, 0.01, -2.0, 1.0, 52)
    lo, hi = oracle.gershgorin(p.H)
    g, m, br, mu = oracle.trfoe(p.lam, p.ne, p.kT, lo, hi)
    X = (hi * np.eye(p.n) - p.H) / (hi - lo)
    for k in range(m):
        t1, t2 = np.trace(X), np.sum(X * X)
        sq = abs(t2 - p.ne) <= abs(2 * t1 - t2 - p.ne)
        assert sq == bool(br[k])
        X2 = X @ X
        X = X2 if sq else 2 * X - X2
    assert np.abs(X - oracle.density_from_eig(p.Q, g)).max() < 1e-11


def test_trfoe_low_temperature_limit_is_the_projector():
    """kT -> 0 on a gapped spectrum: G_m must become the step function, so
    the truncated expansion equals the zero-temperature projector."""
    p = hp_synth.gapped(150, 100, (-2.0, -0.1), (0.1, 1.0), 53)
    lo, hi = oracle.gershgorin(p.H)
    g, m, _, mu = oracle.trfoe(p.lam, p.ne, 1e-9, lo, hi)
    assert m > 0
    f = (np.arange(150) < 100).astype(float)
    assert np.abs(g - f).max() < 1e-12
    assert p.lam[99] < mu < p.lam[100]


def test_trfoe_distance_to_fermi_dirac_is_the_papers_magnitude():
    """Sanity band from Sec. IV: on the paper's own matrix at 500 K with
    N_e = 0.85 n, the truncated expansion takes a few tens of steps and sits
    at a relative distance of order 1e-3 .. 1e-2 from Fermi-Dirac (the paper
    quotes ~30 steps and eps1 ~ 1e-3; it is a smeared step, not FD)."""
    p = hp_synth.paper_matrix(600, frac=0.85)
    w, _ = oracle.eigh_ql(p.H)
    lo, hi = oracle.gershgorin(p.H)
    kT = 1.5834e-3
    g, m, _, mu = oracle.trfoe(w, p.ne, kT, lo, hi)
    f, mu_fd = oracle.occupations(w, p.ne, kT)
    eps1 = np.linalg.norm(g - f) / np.sqrt(p.ne)
    assert 20 <= m <= 60
    assert 1e-4 <= eps1 <= 1e-1
    assert abs(mu - mu_fd) < 0.05


# ---------------------------------------------------------------- finite-T recursion

def test_fermi_recursion_scalar_identity_on_diagonal():
    lam = np.linspace(-1, 1, 9)
    mu, kT, m = 0.1, 0.05, 12
    D = oracle.fermi_recursion(np.diag(lam), mu, kT, m)
    # z0 = a (lam - mu), then m times z -> 2 z / (1 + z^2)
    z = (1.0 / kT) / 2 ** (m + 1) * (lam - mu)
    for _ in range(m):
        z = 2 * z / (1 + z * z)
    assert np.abs(np.diag(D) - 0.5 * (1 - z)).max() < 1e-15
    assert np.abs(D - np.diag(np.diag(D))).max() == 0
    # identity 2 tanh a / (1 + tanh^2 a) = tanh 2a makes z_m ~ tanh(beta (lam - mu) / 2)
    assert np.abs(z - np.tanh((lam - mu) / (2 * kT))).max() < 1e-5


def test_fermi_recursion_matches_fd():
    p = hp_synth.smeared(160, 130.0, 0.01, -2.0, 1.0, 29)
    r = oracle.density(p.H, 130.0, 0.01)
    lo, hi = oracle.gershgorin(p.H)
    W = max(abs(lo - r["mu"]), abs(hi - r["mu"]))
    m = math.ceil(math.log2((W / 0.01) / (2 * 1e-3)))       # t0 <= 1e-3
    D = oracle.fermi_recursion(p.H, r["mu"], 0.01, m)
    assert np.linalg.norm(D - r["D"]) / math.sqrt(130) < 1e-6


# ---------------------------------------------------------------- metrics

def test_metrics():
    p = hp_synth.gapped(60, 45, (-2, -0.05), (0.05, 0.6), 8)
    Dref = oracle.density(p.H, 45)["D"]
    m = oracle.metrics(Dref, Dref, p.H)
    assert m["err_fro"] == 0 and abs(m["ref_fro"] - math.sqrt(45)) < 1e-12
    assert abs(m["e_band"] - p.lam[:45].sum()) < 1e-11 and m["idem_fro"] < 1e-13
    E = np.zeros((60, 60)); E[2, 7] = E[7, 2] = 1e-3
    m = oracle.metrics(Dref + E, Dref, p.H)
    assert abs(m["err_fro"] - math.sqrt(2) * 1e-3) < 1e-15
    assert abs(m["e_band"] - m["e_ref"] - 2e-3 * p.H[2, 7]) < 1e-14
