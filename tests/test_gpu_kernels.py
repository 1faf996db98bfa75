"""Single hot-path kernels through the C ABI against the CPU oracle."""
import math

import numpy as np
import pytest

import hp_synth
import oracle
from gpu_util import ctx, torch

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]


@pytest.mark.parametrize("n", [1, 37, 256, 1000])
def test_gershgorin_matches_oracle(n):
    p = hp_synth.gapped(n, n // 2, (-2, -0.05), (0.05, 0.6), 100 + n)
    H = torch.from_numpy(p.H).cuda()
    lo, hi, tr, bad = ctx().gershgorin(H)
    olo, ohi = oracle.gershgorin(p.H)
    scale = np.abs(p.H).sum(1).max()
    assert abs(lo - olo) <= 1e-13 * scale and abs(hi - ohi) <= 1e-13 * scale
    assert abs(tr - np.trace(p.H)) <= 1e-13 * scale * n
    assert bad == 0.0


def test_gershgorin_flags_nonfinite():
    p = hp_synth.gapped(64, 32, (-2, -0.05), (0.05, 0.6), 5)
    H = p.H.copy()
    H[3, 7] = np.nan
    lo, hi, tr, bad = ctx().gershgorin(torch.from_numpy(H).cuda())
    assert bad == 1.0


def sym_f32(n, seed, scale=1.0):
    G = hp_synth.normal(seed, n * n).reshape(n, n)
    return (scale * 0.5 * (G + G.T) / math.sqrt(n)).astype(np.float32)


@pytest.mark.parametrize("n", [16, 128, 200, 256, 300, 640, 1000, 2065])
@pytest.mark.parametrize("nslices", [2, 1])
def test_sym_square_matches_oracle(n, nslices):
    Y = sym_f32(n, 7 + n)
    Yd = torch.from_numpy(Y).cuda()
    C = torch.empty_like(Yd)
    ctx().sym_square(Yd, C, nslices=nslices, bound=float(np.abs(Y).max()))
    Ch = C.cpu().numpy().astype(np.float64)
    ref = oracle.matmul(Y.astype(np.float64), Y.astype(np.float64))
    absprod = oracle.matmul(np.abs(Y).astype(np.float64), np.abs(Y).astype(np.float64))
    # operand rounding: split FP16 keeps 22 bits (2^-21 on a product), one FP16
    # slice 11 bits (2^-10).  The tensor core adds each MMA into its FP32
    # accumulator with a one-sided rounding; the kernel keeps an accumulator
    # for one 64-wide K chunk (4 full-size additions, cross terms first) and
    # sums the chunks in registers with round-to-nearest.
    nchunks = math.ceil(n / 64)
    rel = (2.0 ** -21 if nslices == 2 else 2.0 ** -10) + 4 * 2.0 ** -23 + nchunks * 2.0 ** -24
    assert np.all(np.abs(Ch - ref) <= rel * absprod + 1e-30)
    assert np.array_equal(Ch, Ch.T)             # mirrored: exactly symmetric


def test_sym_square_leading_dimension_and_scale():
    n, ld = 300, 320
    Y = sym_f32(n, 3, scale=1e-3)
    Yp = np.zeros((n, ld), np.float32); Yp[:, :n] = Y
    Yd = torch.from_numpy(Yp).cuda()
    C = torch.full((n, ld), 7.0, device="cuda", dtype=torch.float32)
    ctx().sym_square(Yd[:, :n], C[:, :n], nslices=2, bound=float(np.abs(Y).max()))
    Ch = C.cpu().numpy()
    ref = Y.astype(np.float64) @ Y.astype(np.float64)
    absprod = np.abs(Y).astype(np.float64) @ np.abs(Y).astype(np.float64)
    rel = 2.0 ** -21 + 4 * 2.0 ** -23 + math.ceil(n / 64) * 2.0 ** -24
    assert np.all(np.abs(Ch[:, :n] - ref) <= rel * absprod)
    assert np.all(Ch[:, n:] == 7.0)             # padding untouched


def _sym_from_spectrum(n, lam, seed):
    Q = hp_synth.haar_q(n, seed)
    return hp_synth.assemble(Q, lam)


@pytest.mark.parametrize("n,ld,kind", [(100, 100, "proj"), (300, 304, "proj"), (1000, 1000, "proj"),
                                       (1290, 1296, "proj"), (517, 520, "wide"), (64, 64, "wide")])
def test_digit_square_is_fp64_accurate(n, ld, kind):
    """The FP64-accurate tensor-core product against the oracle's FP64 matmul:
    a near-projector (the polishing input: eigenvalues 0/1 off by ~1e-6) and a
    symmetric matrix with spectrum spread over [-1.9, 1.9]."""
    g = np.random.default_rng(n)
    if kind == "proj":
        lam = (np.arange(n) < int(0.8 * n)).astype(float) + 1e-6 * g.standard_normal(n)
    else:
        lam = g.uniform(-1.9, 1.9, n)
    X = _sym_from_spectrum(n, lam, 3000 + n)
    Xd = torch.zeros((n, ld), dtype=torch.float64, device="cuda")
    Xd[:, :n] = torch.from_numpy(X).cuda()
    Pd = torch.full((n, ld), float("nan"), dtype=torch.float64, device="cuda")
    ctx().digit_square(Xd[:, :n], Pd[:, :n])
    P = Pd[:, :n].cpu().numpy()
    ref = oracle.matmul(X, X)
    err = np.abs(P - ref).max()
    print(n, kind, err, np.linalg.norm(P - ref))
    assert np.array_equal(P, P.T)                    # mirrored: exactly symmetric
    # the reference's own FP64 rounding bound gamma_n |X||X| (u = 2^-53), plus
    # the kernel's final conversion to FP64 and its dropped digit levels
    absx = np.abs(X)
    bound = 2 * n * 2.0 ** -53 * oracle.matmul(absx, absx) + 2.0 ** -52
    assert np.all(np.abs(P - ref) <= bound)
