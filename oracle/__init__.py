"""Plain FP64 CPU oracle for D = f(Hp) (arXiv 2301.04642).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline leg may import this package.  It shares no code
with the GPU library and the GPU library never calls it.

Each wrapper forwards to ``oracle.c``; see that file's header for the paper
passage each routine follows:

* ``eigh_ql`` / ``eigh_jacobi``  -- own eigensolvers (Sec. II-A needs H's
  eigenpairs to define D).
* ``occupations``               -- step (kT = 0) or Fermi-Dirac occupations,
  mu by bisection (Sec. II-A).
* ``density`` / ``density_from_eig`` / ``density_entries`` -- D = Q f Q^T.
* ``sp2``                       -- CPU SP2, Sec. II-B1 Eq. (1), with the trace
  rule of Sec. III-B and the RelTr stop of Sec. III-A.
* ``sp2_accel``                 -- accelerated SP2 (A-Z-RFOE, Sec. II-B2): the
  SP2 polynomials shifted and scaled with HOMO/LUMO bounds.
* ``fermi_recursion``           -- finite-T recursive expansion (Sec. II-B3,
  doubling reading).
* ``trfoe``                     -- the truncated SP2 expansion of Sec. II-B3,
  Eq. (2) as printed (T-RFOE), on the eigenvalues.
* ``metrics``                   -- eps1, eps2 ingredients (Sec. III-C).
* ``gemm``                      -- the plain products either side of the
  expansion in subspace iteration (Sec. III-A).

Every function here is pinned by a test in ``tests/test_oracle.py`` against
closed forms, invariants, brute force on tiny inputs or a library routine.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        d, i = ctypes.c_double, ctypes.c_int
        sig = {
            "oracle_matmul": (None, [i, _D, _D, _D]),
            "oracle_gemm": (None, [i, i, i, _D, i, i, _D, i, i, _D, i]),
            "oracle_gershgorin": (None, [i, _D, _D, _D]),
            "oracle_eigh_ql": (i, [i, _D, _D, _D]),
            "oracle_eigh_jacobi": (i, [i, _D, _D, _D, i]),
            "oracle_fermi": (d, [d, d, d]),
            "oracle_occupations": (d, [i, _D, d, d, _D]),
            "oracle_density_from_eig": (None, [i, _D, _D, _D]),
            "oracle_density_entry": (d, [i, _D, _D, i, i]),
            "oracle_density": (i, [i, _D, d, d, i, _D, _D, _D, _D]),
            "oracle_sp2": (i, [i, _D, d, d, i, _D, _I]),
            "oracle_sp2_accel": (i, [i, _D, d, d, d, d, i, _D, _I]),
            "oracle_fermi_recursion": (i, [i, _D, d, d, i, _D]),
            "oracle_trfoe": (i, [i, _D, d, d, d, d, i, _D, _I, _D]),
            "oracle_metrics": (None, [i, _D, _D, _D, _D]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_D)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def matmul(A, B):
    A, B = _c64(A), _c64(B)
    n = A.shape[0]
    C = np.empty((n, n))
    lib().oracle_matmul(n, _p(A), _p(B), _p(C))
    return C


def gemm(A, B, ta=False, tb=False):
    """op(A) op(B) in plain FP64 loops (op = transpose when ta / tb)."""
    A, B = _c64(A), _c64(B)
    m, k = (A.shape[1], A.shape[0]) if ta else A.shape
    n = B.shape[0] if tb else B.shape[1]
    assert (B.shape[1] if tb else B.shape[0]) == k
    C = np.empty((m, n))
    lib().oracle_gemm(m, n, k, _p(A), A.shape[1], int(ta), _p(B), B.shape[1], int(tb), _p(C), n)
    return C


def gershgorin(H):
    H = _c64(H)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    lib().oracle_gershgorin(H.shape[0], _p(H), ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def eigh_ql(H):
    H = _c64(H)
    n = H.shape[0]
    w, Q = np.empty(n), np.empty((n, n))
    st = lib().oracle_eigh_ql(n, _p(H), _p(w), _p(Q))
    if st != 0:
        raise RuntimeError("QL did not converge")
    return w, Q


def eigh_jacobi(H, max_sweeps=100):
    H = _c64(H)
    n = H.shape[0]
    w, Q = np.empty(n), np.empty((n, n))
    st = lib().oracle_eigh_jacobi(n, _p(H), _p(w), _p(Q), max_sweeps)
    if st != 0:
        raise RuntimeError("Jacobi did not converge")
    return w, Q


def fermi(lam, mu, kT):
    return lib().oracle_fermi(float(lam), float(mu), float(kT))


def occupations(w, ne, kT):
    """w ascending -> (f, mu)."""
    w = _c64(w)
    f = np.empty_like(w)
    mu = lib().oracle_occupations(w.shape[0], _p(w), float(ne), float(kT), _p(f))
    return f, mu


def density_from_eig(Q, f):
    Q, f = _c64(Q), _c64(f)
    n = Q.shape[0]
    D = np.empty((n, n))
    lib().oracle_density_from_eig(n, _p(Q), _p(f), _p(D))
    return D


def density_entries(Q, f, rows, cols):
    """D_ij = sum_k Q_ik f_k Q_jk for the sampled (i, j) pairs."""
    Q, f = _c64(Q), _c64(f)
    n = Q.shape[0]
    L = lib()
    return np.array([L.oracle_density_entry(n, _p(Q), _p(f), int(i), int(j))
                     for i, j in zip(rows, cols)])


def density(H, ne, kT=0.0, jacobi=False):
    """Oracle D_ref from its own eigendecomposition.

    Returns dict(D, w, f, mu, e_band, n_occ)."""
    H = _c64(H)
    n = H.shape[0]
    D, w, f, out = np.empty((n, n)), np.empty(n), np.empty(n), np.empty(3)
    st = lib().oracle_density(n, _p(H), float(ne), float(kT), int(jacobi),
                              _p(D), _p(w), _p(f), _p(out))
    if st != 0:
        raise RuntimeError("oracle eigensolver did not converge")
    return dict(D=D, w=w, f=f, mu=out[0], e_band=out[1], n_occ=out[2])


def sp2(H, ne, tol=5e-8, max_iter=200):
    """CPU SP2 -> (X, iterations, branches) ; iterations = -1 if not converged."""
    H = _c64(H)
    n = H.shape[0]
    X = np.empty((n, n))
    br = np.zeros(max_iter, dtype=np.int32)
    it = lib().oracle_sp2(n, _p(H), float(ne), float(tol), int(max_iter), _p(X),
                          br.ctypes.data_as(_I))
    return X, it, br[: max(it, 0) if it >= 0 else max_iter].copy()


def sp2_accel(H, ne, homo, lumo, tol=5e-8, max_iter=200):
    """Accelerated SP2 (A-Z-RFOE reading) with HOMO/LUMO estimates ->
    (X, iterations, branches); iterations = -1 if not converged."""
    H = _c64(H)
    n = H.shape[0]
    X = np.empty((n, n))
    br = np.zeros(max_iter, dtype=np.int32)
    it = lib().oracle_sp2_accel(n, _p(H), float(ne), float(homo), float(lumo), float(tol), int(max_iter),
                                _p(X), br.ctypes.data_as(_I))
    return X, it, br[: max(it, 0) if it >= 0 else max_iter].copy()


def sp2_accel_status(it):
    """Meaning of sp2_accel's iteration count: 'ok', 'cap' (-1) or
    'inconsistent' (-2: the HOMO/LUMO estimates do not lie inside the gap)."""
    return "ok" if it >= 0 else ("cap" if it == -1 else "inconsistent")


def trfoe(lam, ne, kT, emin, emax, max_iter=200):
    """Truncated SP2 at finite temperature (Sec. II-B3, Eq. (2)) on the
    eigenvalues lam of H with spectral bounds [emin, emax]:
    -> (g, m, branches, mu) with g = G_m((emax - lam)/(emax - emin)) the
    occupations (D = Q diag(g) Q^T), m the steps (-1: max_iter reached),
    branches[k] = 1 for X^2, and mu the energy where G_m crosses 1/2."""
    lam = _c64(lam)
    n = lam.shape[0]
    g = np.empty(n)
    br = np.zeros(max_iter + 1, dtype=np.int32)
    mu = ctypes.c_double()
    m = lib().oracle_trfoe(n, _p(lam), float(ne), 1.0 / float(kT), float(emin), float(emax), int(max_iter),
                           _p(g), br.ctypes.data_as(_I), ctypes.byref(mu))
    return g, m, br[: (m if m >= 0 else max_iter)].copy(), mu.value


def fermi_recursion(H, mu, kT, m):
    H = _c64(H)
    n = H.shape[0]
    D = np.empty((n, n))
    st = lib().oracle_fermi_recursion(n, _p(H), float(mu), float(kT), int(m), _p(D))
    if st != 0:
        raise RuntimeError("Cholesky failed in the finite-T recursion")
    return D


def metrics(D, Dref, H):
    """-> dict(err_fro, ref_fro, e_band, e_ref, trace, idem_fro)."""
    D, Dref, H = _c64(D), _c64(Dref), _c64(H)
    out = np.empty(6)
    lib().oracle_metrics(D.shape[0], _p(D), _p(Dref), _p(H), _p(out))
    keys = ("err_fro", "ref_fro", "e_band", "e_ref", "trace", "idem_fro")
    return dict(zip(keys, out.tolist()))
