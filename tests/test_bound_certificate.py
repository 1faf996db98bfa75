"""The arithmetic of the spectral-bound certificate (Sec. II-C asks for bounds
that contain the spectrum; the library certifies a Lanczos estimate [lo, hi]).

With X0 = (hi I - Hp)/(hi - lo) and three logistic steps X <- 4 X (I - X):
  (1) X_3 = (I - T_8(A))/2 with A = (2 Hp - (hi + lo) I)/(hi - lo) and T_8 the
      Chebyshev polynomial of degree 8 (checked against numpy's Chebyshev
      series evaluated on the eigenvalues);
  (2) every eigenvalue a of A obeys |a| <= cosh(arccosh(1 + 2 ||X_3||_F) / 8),
      for any estimate, too narrow or not;
  (3) when [lo, hi] contains the spectrum the widening factor is at most
      cosh(arccosh(1 + 2 sqrt(n)) / 8).
Plain FP64 numpy on small seeded matrices; no GPU."""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev

import hp_synth


def _logistic3(H, lo, hi):
    n = H.shape[0]
    X = (hi * np.eye(n) - H) / (hi - lo)
    for _ in range(3):
        X = 4.0 * X @ (np.eye(n) - X)
    return X


def _amax(X3):
    f = np.linalg.norm(X3)
    return math.cosh(math.acosh(1.0 + 2.0 * f) / 8.0)


@pytest.mark.parametrize("factor", [1.0, 1.1, 0.9, 0.5, 0.25])
@pytest.mark.parametrize("seed", [11, 12])
def test_certificate_contains_spectrum(factor, seed):
    n = 48
    lam = hp_synth.gapped_spectrum(n, 20, (-3.0, -0.2), (0.3, 1.0), seed)
    H = hp_synth.assemble(hp_synth.haar_q(n, seed), lam)
    mid, half = 0.5 * (lam[0] + lam[-1]), 0.5 * (lam[-1] - lam[0]) * factor
    lo, hi = mid - half, mid + half
    X3 = _logistic3(H, lo, hi)
    a = (2.0 * lam - hi - lo) / (hi - lo)
    # (1) X_3 = (I - T_8(A)) / 2 on the eigenvalues
    t8 = chebyshev.chebval(a, [0] * 8 + [1])
    ev = np.linalg.eigvalsh(0.5 * (X3 + X3.T))
    np.testing.assert_allclose(np.sort(ev), np.sort(0.5 * (1.0 - t8)), rtol=1e-9,
                               atol=1e-9 * max(1.0, np.abs(t8).max()))
    # (2) the certified half-width covers every eigenvalue
    amax = _amax(X3)
    assert np.abs(a).max() <= amax * (1.0 + 1e-12)
    # (3) an estimate that contains the spectrum is widened by a bounded factor
    if factor >= 1.0:
        assert amax <= math.cosh(math.acosh(1.0 + 2.0 * math.sqrt(n)) / 8.0)


def test_certificate_is_tight_for_a_single_outlier():
    """One eigenvalue far outside the estimate dominates ||X_3||_F, and the
    certified half-width lands just above it."""
    n = 32
    lam = np.linspace(-1.0, 1.0, n)
    lam[-1] = 1.7
    H = hp_synth.assemble(hp_synth.haar_q(n, 5), lam)
    X3 = _logistic3(H, -1.0, 1.0)
    amax = _amax(X3)
    assert 1.7 <= amax <= 1.8
