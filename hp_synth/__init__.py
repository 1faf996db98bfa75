"""Seeded synthetic projected Hamiltonians Hp = Q diag(lambda) Q^T.

This module is the only code that both the oracle side (tests, CPU baseline)
and the GPU side (tests, benchmark) use.  It holds no arithmetic of the
density-matrix method: only a portable random stream, the spectrum recipes of
the benchmark workloads and the orthogonal similarity that builds Hp.

Random stream: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) -> 53-bit uniforms in (0, 1) -> Box-Muller
normals.  Everything is integer arithmetic on uint64 followed by IEEE double
operations, so the same seed gives the same bits on x86_64 and aarch64.

Q is the orthogonal factor of the QR factorisation of an n x n matrix of N(0,1)
draws, with column signs fixed so that diag(R) > 0 (this makes Q unique and
Haar-distributed).  Because Q and lambda are known, D_ref = Q f(lambda) Q^T is
an exact reference for any n.
"""
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, count):
    """`count` consecutive SplitMix64 outputs for a stream starting at `seed`."""
    with np.errstate(over="ignore"):
        state = np.uint64(seed) + _GOLDEN * np.arange(1, count + 1, dtype=np.uint64)
        z = state
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, count):
    """Uniform doubles in the open interval (0, 1): (top 53 bits + 0.5) / 2^53."""
    z = splitmix64(seed, count)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed, count):
    """Standard normals by Box-Muller from pairs of the uniform stream."""
    m = (count + 1) // 2
    u = uniform(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * math.pi * u2
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(t)
    out[1::2] = r * np.sin(t)
    return out[:count]


def haar_q(n, seed, device=None):
    """Orthogonal Q from QR of a seeded N(0,1) n x n matrix, diag(R) > 0.

    device=None -> numpy on the host; otherwise a torch device string (the QR
    then runs in FP64 with torch on that device; the Gaussian matrix is the
    same host stream)."""
    G = normal(seed, n * n).reshape(n, n)
    if device is None:
        Q, R = np.linalg.qr(G)
        s = np.sign(np.diag(R))
        s[s == 0] = 1.0
        return Q * s[None, :]
    import torch
    Gt = torch.from_numpy(G).to(device)
    Q, R = torch.linalg.qr(Gt)
    s = torch.sign(torch.diagonal(R))
    s[s == 0] = 1.0
    return Q * s[None, :]


def gapped_spectrum(n, ne, occ, emp, seed):
    """ne occupied eigenvalues uniform in occ=(a, b), n-ne empty uniform in
    emp=(c, d); the gap edges are pinned (max occupied = b, min empty = c) so
    the HOMO-LUMO gap is exactly c - b.  Returned ascending."""
    u = uniform(seed ^ 0x5DEECE66D, n)
    a, b = occ
    c, d = emp
    lo = a + (b - a) * u[:ne]
    hi = c + (d - c) * u[ne:]
    if ne > 0:
        lo[np.argmax(lo)] = b
    if n - ne > 0:
        hi[np.argmin(hi)] = c
    return np.sort(np.concatenate([lo, hi]))


def semicircle_spectrum(n, a, b, seed):
    """n draws from the Wigner semicircle density on [a, b], ascending.
    x = sqrt(u) cos(2 pi v) has the semicircle density on [-1, 1]."""
    u = uniform(seed ^ 0x5DEECE66D, 2 * n)
    x = np.sqrt(u[0::2]) * np.cos(2.0 * math.pi * u[1::2])
    return np.sort(0.5 * (a + b) + 0.5 * (b - a) * x)


def assemble(Q, lam):
    """Hp = Q diag(lam) Q^T, symmetrised, FP64 (numpy or torch, matching Q)."""
    if isinstance(Q, np.ndarray):
        H = (Q * lam[None, :]) @ Q.T
        return 0.5 * (H + H.T)
    import torch
    lt = torch.as_tensor(lam, dtype=Q.dtype, device=Q.device)
    H = (Q * lt[None, :]) @ Q.T
    return 0.5 * (H + H.T)


class Problem:
    """One synthetic solve: Hp with its exact eigendecomposition (Q, lam), or
    Q = lam = None for a matrix given by a formula."""

    def __init__(self, name, H, Q, lam, ne, kT, tol, seed):
        self.name, self.H, self.Q, self.lam = name, H, Q, lam
        self.n = H.shape[0]
        self.ne, self.kT, self.tol, self.seed = ne, kT, tol, seed

    def __repr__(self):
        return "Problem(%s, n=%d, ne=%g, kT=%g)" % (self.name, self.n, self.ne, self.kT)


def gapped(n, ne, occ, emp, seed, tol=5e-8, device=None, name="gapped"):
    lam = gapped_spectrum(n, ne, occ, emp, seed)
    Q = haar_q(n, seed, device)
    return Problem(name, assemble(Q, lam), Q, lam, float(ne), 0.0, tol, seed)


def smeared(n, ne, kT, a, b, seed, tol=5e-8, device=None, name="smeared"):
    lam = semicircle_spectrum(n, a, b, seed)
    Q = haar_q(n, seed, device)
    return Problem(name, assemble(Q, lam), Q, lam, float(ne), kT, tol, seed)


class ReflectedQ:
    """Q = H_0 H_1 ... H_{k-1}, H_j = I - 2 v_j v_j^T with unit v_j: an
    orthogonal factor applied in O(k n^2) (used where a QR of an n x n
    Gaussian would cost minutes: the serving workload reaches n = 32768).
    V holds the k vectors as rows (torch tensor on the device, or numpy)."""

    def __init__(self, V):
        self.V = V

    def _refl(self, X, j):
        v = self.V[j]
        return X - 2.0 * v[:, None] * (v[None, :] @ X)

    def mul(self, X):
        """Q X."""
        for j in range(self.V.shape[0] - 1, -1, -1):
            X = self._refl(X, j)
        return X

    def tmul(self, X):
        """Q^T X."""
        for j in range(self.V.shape[0]):
            X = self._refl(X, j)
        return X


def reflected_q(n, seed, k=8, device=None):
    V = normal(seed, k * n).reshape(k, n)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    if device is not None:
        import torch
        V = torch.from_numpy(V).to(device)
    return ReflectedQ(V)


def assemble_reflected(Q, lam):
    """Hp = Q diag(lam) Q^T for a ReflectedQ: starting from diag(lam), each
    reflector acts on both sides, H <- H - 2 v w^T - 2 w v^T + 4 (v^T w) v v^T
    with w = H v (exact similarity, symmetric by construction)."""
    V = Q.V
    if isinstance(V, np.ndarray):
        H = np.diag(np.asarray(lam, dtype=np.float64))
        for j in range(V.shape[0] - 1, -1, -1):
            v = V[j]
            w = H @ v
            a = float(v @ w)
            H -= 2.0 * np.outer(v, w) + 2.0 * np.outer(w, v) - 4.0 * a * np.outer(v, v)
        return H
    import torch
    H = torch.diag(torch.as_tensor(lam, dtype=torch.float64, device=V.device))
    for j in range(V.shape[0] - 1, -1, -1):
        v = V[j]
        w = H @ v
        a = float(v @ w)
        H.addr_(v, w, alpha=-2.0).addr_(w, v, alpha=-2.0).addr_(v, v, alpha=4.0 * a)
    return H


def gapped_reflected(n, ne, occ, emp, seed, tol=5e-8, device=None, name="gapped_reflected"):
    """The gapped recipe with Q from 8 Householder reflectors instead of a QR."""
    lam = gapped_spectrum(n, ne, occ, emp, seed)
    Q = reflected_q(n, seed, device=device)
    return Problem(name, assemble_reflected(Q, lam), Q, lam, float(ne), 0.0, tol, seed)


def smeared_reflected(n, ne, kT, a, b, seed, tol=5e-8, device=None, name="smeared_reflected"):
    """The semicircle recipe with Q from 8 Householder reflectors."""
    lam = semicircle_spectrum(n, a, b, seed)
    Q = reflected_q(n, seed, device=device)
    return Problem(name, assemble_reflected(Q, lam), Q, lam, float(ne), kT, tol, seed)


def serve_requests(count, rate, nmin, nmax, seed=3000):
    """The serving workload's request stream: for request k, n log-uniform in
    [nmin, nmax], 70% gapped (gap uniform in [0.01, 0.1] Ha at 0) and 30%
    finite temperature (kT uniform in [0.001, 0.01] Ha, semicircle spectrum
    on [-2, 1] Ha), N_e = round(0.85 n), and Poisson arrival gaps of mean
    1/rate.  Returns a list of dicts (n, ne, kT, gap, seed, dt)."""
    u = uniform(seed, 4 * count)
    dts = -np.log(1.0 - uniform(seed + 1, count)) / rate
    out = []
    for k in range(count):
        n = int(round(math.exp(math.log(nmin) + u[4 * k] * (math.log(nmax) - math.log(nmin)))))
        n = max(64, n)
        finite = u[4 * k + 1] >= 0.7
        out.append(dict(n=n, ne=int(round(0.85 * n)), kT=(0.001 + 0.009 * u[4 * k + 2]) if finite else 0.0,
                        gap=0.0 if finite else 0.01 + 0.09 * u[4 * k + 2], seed=seed + 100 + k, dt=float(dts[k])))
    return out


# --- the benchmark workloads (sizes, spectra, seeds) --------------------------

def workload_n256(device=None):
    """n=256, 200 occupied in [-2, -0.05] Ha, 56 empty in [0.05, 0.6] Ha."""
    return gapped(256, 200, (-2.0, -0.05), (0.05, 0.6), 1001, tol=1e-10,
                  device=device, name="gapped_n256_fp64")


def workload_n4096(device=None):
    """n=4096, N_e=3500, occupied [-3, -0.01], empty [0.01, 1.0] Ha."""
    return gapped(4096, 3500, (-3.0, -0.01), (0.01, 1.0), 1002,
                  device=device, name="gapped_n4096")


def workload_n16384_ft(device=None):
    """n=16384 semicircle on [-2, 1] Ha, N_e=14000, kT=0.003 Ha."""
    return smeared(16384, 14000, 0.003, -2.0, 1.0, 1003, device=device,
                   name="fermi_n16384_kT0.003")


def ragged_batch_sizes(count=64, lo=512, hi=6144, seed=2000):
    """n_i = round(exp(U[ln lo, ln hi])) with matrix i drawing from seed+i."""
    out = []
    for i in range(count):
        u = uniform(seed + i, 2)
        out.append(int(round(math.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * u[0]))))
    return out


def ragged_member(i, seed=2000, device=None, lo=512, hi=6144):
    """Batch member i: log-uniform n, N_e = round(0.85 n), gap U[0.01, 0.1]
    centred at 0, occupied down to -3, empty up to 1."""
    u = uniform(seed + i, 2)
    n = int(round(math.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * u[0])))
    gap = 0.01 + 0.09 * u[1]
    ne = int(round(0.85 * n))
    return gapped(n, ne, (-3.0, -gap / 2), (gap / 2, 1.0), seed + i, device=device,
                  name="ragged_%d" % i)


def paper_matrix(n, frac=0.9, tol=5e-8, device=None):
    """The synthetic Hamiltonian of the paper's scaling runs (Sec. IV):
    H_ij = exp(-0.5 |i - j|) sin(i + 1) as printed is not symmetric; the reading
    used here takes the smaller index, H_ij = H_ji = exp(-0.5 |i - j|)
    sin(min(i, j) + 1), 0-based indices, radians.  N_e = round(frac n) (0.9 at
    zero temperature).  Its spectrum is a continuous band in [-1.87, 1.87]:
    the gap at N_e = 0.9 n is about 1.4 / n."""
    ne = float(int(round(frac * n)))
    if device is None:
        i = np.arange(n, dtype=np.float64)
        H = np.exp(-0.5 * np.abs(i[:, None] - i[None, :])) * np.sin(np.minimum(i[:, None], i[None, :]) + 1.0)
    else:
        import torch
        i = torch.arange(n, dtype=torch.float64, device=device)
        H = torch.exp(-0.5 * (i[:, None] - i[None, :]).abs()) * torch.sin(torch.minimum(i[:, None], i[None, :]) + 1.0)
    return Problem("paper_matrix_n%d" % n, H, None, None, ne, 0.0, tol, 0)
