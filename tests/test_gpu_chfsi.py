"""The products either side of the expansion in Chebyshev-filtered subspace
iteration (Sec. III-A) through the C ABI (fe_project, fe_rotate), against
the oracle's plain FP64 products.

Bound (split FP16 operands, FP32 chunk sums, FP64 sum of the K parts):
|C_ij - C_ref_ij| <= (2^-21 + 4 2^-23 + c 2^-24) sum_k |A_ik| |B_kj| with c
the 64-wide K chunks summed in FP32 (the chunks of one K part: at most 128
for the projection, all ceil(n / 64) for the rotation), plus an absolute
2^-36 max|A| max|B| K: a low slice below 2^-14 (the FP16 normal range, for
entries under 2^-25 of the operand's largest) keeps fewer bits."""
import math

import numpy as np
import pytest

import hp_synth
import oracle
from gpu_util import ctx, torch

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]


def rel_bound(chunks):
    return 2.0 ** -21 + 4 * 2.0 ** -23 + chunks * 2.0 ** -24


def floor_abs(A, B, K):
    return 2.0 ** -36 * float(np.abs(A).max()) * float(np.abs(B).max()) * K


def rand(rows, cols, seed, scale=1.0):
    return scale * hp_synth.normal(seed, rows * cols).reshape(rows, cols)


@pytest.mark.parametrize("m,n,ld", [(1000, 1000, 1000), (20000, 300, 300), (9001, 517, 520), (70000, 200, 200)])
def test_project_matches_oracle(m, n, ld):
    Psi = rand(m, n, 11 + n) / math.sqrt(m)
    HPsi = rand(m, n, 12 + n, 3.0) / math.sqrt(m)
    P = np.zeros((m, ld))
    Y = np.zeros((m, ld))
    P[:, :n], Y[:, :n] = Psi, HPsi
    Pd, Yd = torch.from_numpy(P).cuda(), torch.from_numpy(Y).cuda()
    Hd = torch.full((n, n + 3), 7.0, dtype=torch.float64, device="cuda")
    ctx().project(Pd[:, :n], Yd[:, :n], Hd[:, :n])
    Hp = Hd.cpu().numpy()
    assert np.all(Hp[:, n:] == 7.0)                       # padding untouched
    Hp = Hp[:, :n]
    ref = oracle.gemm(Psi, HPsi, ta=True)
    absref = oracle.gemm(np.abs(Psi), np.abs(HPsi), ta=True)
    up = np.triu(np.ones((n, n), dtype=bool))
    err = np.abs(Hp - ref)
    print(m, n, "max rel to |A||B|", (err / absref)[up].max())
    assert np.all(err[up] <= rel_bound(min(128, math.ceil(m / 64))) * absref[up] + floor_abs(Psi, HPsi, m))
    assert np.array_equal(Hp, Hp.T)                     # upper triangle mirrored


def test_project_of_an_invariant_subspace_is_diagonal():
    """Psi with orthonormal columns and H Psi = Psi diag(lam): the exact
    projection is diag(lam)."""
    m, n = 4096, 300
    Q = hp_synth.haar_q(m, 21, device="cuda")[:, :n].contiguous()
    lam = torch.linspace(-2.0, 1.0, n, dtype=torch.float64, device="cuda")
    HPsi = Q * lam[None, :]
    Hp = torch.empty(n, n, dtype=torch.float64, device="cuda")
    ctx().project(Q, HPsi, Hp)
    absref = oracle.gemm(np.abs(Q.cpu().numpy()), np.abs(HPsi.cpu().numpy()), ta=True)
    err = np.abs(Hp.cpu().numpy() - np.diag(lam.cpu().numpy()))
    assert np.all(err <= rel_bound(64) * absref + floor_abs(Q.cpu().numpy(), HPsi.cpu().numpy(), m))


@pytest.mark.parametrize("m,n,ld", [(1000, 1000, 1000), (20000, 300, 304), (9001, 517, 517)])
def test_rotate_matches_oracle(m, n, ld):
    Psi = rand(m, n, 31 + n)
    P = np.zeros((m, ld))
    P[:, :n] = Psi
    p = hp_synth.gapped(n, int(0.8 * n), (-3.0, -0.01), (0.01, 1.0), 32 + n)
    D = oracle.density_from_eig(p.Q, (np.arange(n) < int(0.8 * n)).astype(float))
    Pd, Dd = torch.from_numpy(P).cuda(), torch.from_numpy(D).cuda()
    Od = torch.full((m, ld), 5.0, dtype=torch.float64, device="cuda")
    ctx().rotate(Pd[:, :n], Dd, Od[:, :n])
    Out = Od.cpu().numpy()
    assert np.all(Out[:, n:] == 5.0)
    Out = Out[:, :n]
    ref = oracle.gemm(Psi, D)
    absref = oracle.gemm(np.abs(Psi), np.abs(D))
    err = np.abs(Out - ref)
    print(m, n, "max rel to |A||B|", (err / absref).max())
    assert np.all(err <= rel_bound(math.ceil(n / 64)) * absref + floor_abs(Psi, D, n))


def test_rotate_by_identity_and_invalid_arguments():
    import paper_2301_04642_gb300 as fe
    m, n = 3000, 250
    Psi = torch.from_numpy(rand(m, n, 41)).cuda()
    I = torch.eye(n, dtype=torch.float64, device="cuda")
    Out = torch.empty_like(Psi)
    ctx().rotate(Psi, I, Out)
    # D = I: every entry is one product with 1 (a hi and a lo term added in the
    # tensor core's FP32 accumulator), within the same bound with |D| = I
    err = (Out - Psi).abs()
    print("max rel", float((err / Psi.abs().clamp_min(1e-300)).max()))
    assert torch.all(err <= rel_bound(math.ceil(n / 64)) * Psi.abs() + floor_abs(Psi.cpu().numpy(), 1.0, n)).item()
    L = fe.load()
    for args in [(0, n, n), (m, 0, n), (m, n, n - 1)]:
        rc = L.fe_rotate(ctx().h, Psi.data_ptr(), args[0], args[1], args[2], I.data_ptr(), n, Out.data_ptr(), n)
        assert rc == fe.FE_EINVAL
    rc = L.fe_project(ctx().h, None, Psi.data_ptr(), m, n, n, Out.data_ptr(), n)
    assert rc == fe.FE_EINVAL
