"""Failure detection without a GPU fault: every device wait is bounded, and
an expired wait ends the run with FE_ETIMEOUT while the context stays usable.

The test makes one wait run out on purpose, by the library's own hook
(fe_k_set_wait): the second CTA of every tile that the Stream-K schedule of
the tensor-core kernel splits between two CTAs waits on a word that nothing
writes, with a 1 ms limit.  The kernel records the error, waits (bounded) for
its own copies and products in flight, frees its tensor memory and returns;
the control kernel ends the problem.  Then the hook is disarmed and the same
context solves the same problem to the oracle's tolerances."""
import math

import numpy as np
import pytest

import hp_synth
import oracle
from gpu_util import need_gpu, torch

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]


def test_expired_partner_wait_reports_timeout_and_context_recovers():
    need_gpu()
    import paper_2301_04642_gb300 as fe
    # n = 3000: 24 row panels, 156 tiles of 128 x 256 over 152 CTAs, so the
    # Stream-K ranges split tiles between neighbouring CTAs
    n, ne = 3000, 2500
    p = hp_synth.gapped(n, ne, (-3.0, -0.01), (0.01, 1.0), 8800, device="cuda")
    H = p.H
    D = torch.empty_like(H)
    with fe.Context(device=0) as c:
        c.set_tile_width(n, 256)
        c.set_wait(limit_ms=1.0, fail_partner=True)
        r = c.solve(H, ne, D=D, check=False)
        print(r)
        assert r["status"] == fe.FE_ETIMEOUT
        assert "timed out" in c.last_error()
        c.set_wait(limit_ms=2000.0, fail_partner=False)
        r2 = c.solve(H, ne, D=D)
        assert r2["status"] == 0
    f = (np.arange(n) < ne).astype(float)
    Dh = D.cpu().numpy()
    Q = p.Q.cpu().numpy()
    eps1 = np.linalg.norm(Dh - oracle.density_from_eig(Q, f)) / math.sqrt(ne)
    e_err = abs(r2["e_band"] - float(np.sum(f * p.lam))) / ne
    idem = np.linalg.norm(oracle.matmul(Dh, Dh) - Dh)
    print(r2, eps1, e_err, idem)
    assert eps1 <= 1e-6 and e_err <= 1e-7 and abs(np.trace(Dh) - ne) <= 1e-9 and idem <= 1e-8


def test_wait_hook_rejects_bad_limits():
    need_gpu()
    import paper_2301_04642_gb300 as fe
    with fe.Context(device=0) as c:
        for bad in (0.0, -1.0, 1e9):
            with pytest.raises(fe.FeError) as ei:
                c.set_wait(limit_ms=bad)
            assert ei.value.status == fe.FE_EINVAL
