"""A ragged batch at the sizes of the batch workload (n log-spread over
[512, 6144], N_e = round(0.85 n), gap in [0.01, 0.1] Ha at 0) in one
fe_solve_batch, every member compared with its own constructed reference
D_ref = Q f Q^T (Q, lambda from the generator): the exact trace, the band
energy, 600 sampled entries of D_ref (oracle.density_entries) and
||D - D_ref||_F, ||D^2 - D||_F by four Gaussian probes
(E ||A v||^2 = ||A||_F^2).  Tolerances as for a single solve."""
import math

import numpy as np
import pytest

import hp_synth
import oracle
from gpu_util import ctx, torch

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]

SIZES = [512, 700, 1000, 1500, 2200, 3000, 4200, 6144]


def test_ragged_batch_members_match_their_references():
    rng = np.random.default_rng(31)
    probs = []
    for k, n in enumerate(SIZES):
        gap = 0.01 + 0.09 * rng.uniform()
        ne = int(round(0.85 * n))
        probs.append(hp_synth.gapped(n, ne, (-3.0, -gap / 2), (gap / 2, 1.0), 9100 + k, device="cuda"))
    items = [dict(H=p.H, ne=p.ne, D=torch.empty_like(p.H)) for p in probs]
    rc, res = ctx().solve_batch(items)
    assert rc == 0
    for p, it, r in zip(probs, items, res):
        n, ne = p.n, int(p.ne)
        f = (np.arange(n) < ne).astype(float)
        Q = p.Q.cpu().numpy()
        D = it["D"].cpu().numpy()
        rows, cols = rng.integers(0, n, 600), rng.integers(0, n, 600)
        ent = np.abs(D[rows, cols] - oracle.density_entries(Q, f, rows, cols)).max()
        V = rng.standard_normal((n, 4))
        DV = D @ V
        eps1 = math.sqrt(np.sum((DV - Q @ (f[:, None] * (Q.T @ V))) ** 2) / 4) / math.sqrt(ne)
        idem = math.sqrt(np.sum((D @ DV - DV) ** 2) / 4)
        e_err = abs(r["e_band"] - float(np.sum(f * p.lam))) / ne
        print(n, r["iters_by_phase"], ent, eps1, idem, e_err)
        assert r["status"] == 0
        assert abs(np.trace(D) - ne) <= 1e-9 and abs(r["trace"] - ne) <= 1e-9
        assert ent <= 1e-6 and eps1 <= 1e-6 and idem <= 1e-8 and e_err <= 1e-7
