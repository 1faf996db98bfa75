"""Continuous batching (fe_submit / fe_poll) through the C ABI.

Each request's answer must equal the same problem solved alone with fe_solve
within the stated tolerances (the tensor-core work of one launch is split over
the SMs by the total work of every problem in it, so the rounding of a
problem's sums depends on its company), and meet the oracle tolerances:
||D - D_ref||_F / sqrt(N_e) <= 1e-6, |E_band - E_ref| / N_e <= 1e-7,
|tr D - N_e| <= 1e-9."""
import math
import time

import numpy as np
import pytest

import hp_synth
import oracle
from gpu_util import need_gpu, torch

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]

TOL_EPS1, TOL_E, TOL_TR = 1e-6, 1e-7, 1e-9


def _mix():
    """Zero- and finite-temperature requests of several sizes."""
    return [
        dict(p=hp_synth.gapped(300, 250, (-3.0, -0.01), (0.01, 1.0), 501), kT=0.0),
        dict(p=hp_synth.smeared(300, 255.0, 0.02, -2.0, 1.0, 502), kT=0.02),
        dict(p=hp_synth.gapped(1000, 850, (-3.0, -0.01), (0.01, 1.0), 503), kT=0.0),
        dict(p=hp_synth.gapped(640, 500, (-2.0, -0.05), (0.05, 2.0), 504), kT=0.0),
        dict(p=hp_synth.smeared(517, 440.5, 0.01, -2.0, 1.0, 505), kT=0.01),
        dict(p=hp_synth.gapped(128, 64, (-3.0, -0.01), (0.01, 1.0), 506), kT=0.0),
    ]


def _check_oracle(it, D, res):
    p, kT = it["p"], it["kT"]
    if kT > 0:
        ref = oracle.density(p.H, p.ne, kT)
        Dref, Eref = ref["D"], ref["e_band"]
    else:
        f = (np.arange(p.n) < int(p.ne)).astype(float)
        Dref = oracle.density_from_eig(p.Q, f)
        Eref = float(np.sum(f * p.lam))
    assert np.linalg.norm(D - Dref) / math.sqrt(p.ne) <= TOL_EPS1
    assert abs(res["e_band"] - Eref) / p.ne <= TOL_E
    assert abs(np.trace(D) - p.ne) <= TOL_TR


def _serve_and_compare(c, items, stagger_s):
    import paper_2301_04642_gb300 as fe
    solo = []
    for it in items:
        D = np.zeros_like(it["p"].H)
        r = c.solve(it["p"].H, it["p"].ne, kT=it["kT"], tol=it["p"].tol, D=D)
        solo.append((D, r))
    tickets, outs = [], []
    for k, it in enumerate(items):
        D = np.zeros_like(it["p"].H)
        H = it["p"].H.copy()
        tickets.append(c.submit(H, it["p"].ne, kT=it["kT"], tol=it["p"].tol, D=D))
        H[:] = np.nan                       # Hp is copied at submit: reuse must not matter
        outs.append(D)
        if k % 2 == 1:
            time.sleep(stagger_s)           # staggered arrival: later ones join a running batch
    results = [c.wait(t, timeout_s=300) for t in tickets]
    for it, D, r, (Ds, rs) in zip(items, outs, results, solo):
        print(it["p"].n, it["kT"], r["status"], r["iters"], rs["iters"], r["ms"])
        assert r["status"] == fe.FE_OK
        ne = it["p"].ne
        assert np.linalg.norm(D - Ds) / math.sqrt(ne) <= TOL_EPS1   # the same alone and in the mix
        assert abs(r["e_band"] - rs["e_band"]) / ne <= TOL_E
        assert abs(r["trace"] - rs["trace"]) <= 2 * TOL_TR
        _check_oracle(it, D, r)
        assert r["ms"] > 0
    with pytest.raises(fe.FeError) as ei:   # a collected ticket is gone
        c.poll(tickets[0])
    assert ei.value.status == fe.FE_EINVAL


def test_serve_matches_solo_and_oracle():
    need_gpu()
    import paper_2301_04642_gb300 as fe
    with fe.Context(device=0) as c:
        _serve_and_compare(c, _mix(), stagger_s=0.002)


def test_serve_under_tight_budget_queues():
    """A budget with room for about two n = 1000 problems: the rest wait in
    the queue and start as slots free up."""
    need_gpu()
    import paper_2301_04642_gb300 as fe
    items = [dict(p=hp_synth.gapped(1000, 850 - 10 * k, (-3.0, -0.01), (0.01, 1.0), 600 + k), kT=0.0)
             for k in range(5)]
    with fe.Context(device=0, hbm_budget_bytes=100 << 20) as c:
        _serve_and_compare(c, items, stagger_s=0.0)


def test_serve_device_pointers_and_errors():
    need_gpu()
    import paper_2301_04642_gb300 as fe
    p = hp_synth.gapped(400, 300, (-3.0, -0.01), (0.01, 1.0), 701)
    with fe.Context(device=0, hbm_budget_bytes=64 << 20) as c:
        Hd = torch.from_numpy(p.H).cuda()
        Dd = torch.zeros_like(Hd)
        t = c.submit(Hd, p.ne, tol=p.tol, D=Dd)
        r = c.wait(t)
        assert r["status"] == fe.FE_OK
        _check_oracle(dict(p=p, kT=0.0), Dd.cpu().numpy(), r)
        big = hp_synth.gapped(2048, 1000, (-3.0, -0.01), (0.01, 1.0), 702)
        with pytest.raises(fe.FeError) as ei:      # larger than the whole budget
            c.submit(big.H, big.ne)
        assert ei.value.status == fe.FE_ENOMEM
        with pytest.raises(fe.FeError) as ei:      # invalid request: rejected at submit
            c.submit(p.H, p.n + 1)
        assert ei.value.status == fe.FE_EINVAL
        with pytest.raises(fe.FeError) as ei:
            c.poll(123456789)
        assert ei.value.status == fe.FE_EINVAL
