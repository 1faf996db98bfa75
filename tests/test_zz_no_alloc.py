"""The allocation-free Gershgorin entry point (fe_k_gershgorin_noalloc)
against the context-based fe_k_gershgorin, both through the C ABI.

Collected last on purpose: it must give the same answer in a fresh process
(its first call sets up the per-device scratch) and after every other test
has used the device.  Two calls in a row check that the shared scratch is
cleared between calls.  min/max bounds are exact (same per-row sums, order-
free min/max); tr H may differ by rounding order only."""
import numpy as np
import pytest

import hp_synth
from gpu_util import ctx, torch

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]


def _check(got, ref, n):
    assert got[0] == ref[0] and got[1] == ref[1] and got[3] == ref[3]
    assert abs(got[2] - ref[2]) <= 1e-13 * max(1.0, np.abs(ref[2])) * n


@pytest.mark.parametrize("n,ld", [(1000, 1000), (777, 800), (32768 // 4 + 3, 32768 // 4 + 8)])
def test_noalloc_matches_context_path_twice(n, ld):
    import paper_2301_04642_gb300 as fe
    p = hp_synth.gapped(n, n // 2, (-3.0, -0.01), (0.01, 1.0), 900 + n, device="cuda")
    H = torch.zeros((n, ld), dtype=torch.float64, device="cuda")
    H[:, :n] = p.H if torch.is_tensor(p.H) else torch.from_numpy(p.H).cuda()
    Hv = H[:, :n]
    ref = ctx().gershgorin(Hv)
    for _ in range(2):
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        fe.gershgorin_noalloc(Hv, out)
        torch.cuda.synchronize()
        _check(out.cpu().tolist(), ref, n)


def test_noalloc_fills_the_whole_scratch_and_matches_oracle():
    """n = 32768 (4096 blocks, the last row at the end of the fixed array)
    with ld > n, and a small case, against the oracle's Gershgorin bounds
    (the same row sums in another order: equal to rounding)."""
    import oracle
    import paper_2301_04642_gb300 as fe
    for n, ld in [(32768, 32776), (301, 301)]:
        p = hp_synth.paper_matrix(n, device="cuda")
        H = torch.zeros((n, ld), dtype=torch.float64, device="cuda")
        H[:, :n] = p.H
        del p
        Hv = H[:, :n]
        lo, hi = oracle.gershgorin(Hv.cpu().numpy())
        tr = float(torch.trace(Hv).item())
        for _ in range(2):
            out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
            fe.gershgorin_noalloc(Hv, out)
            torch.cuda.synchronize()
            got = out.cpu().tolist()
            scale = max(abs(lo), abs(hi))
            assert abs(got[0] - lo) <= 1e-12 * scale and abs(got[1] - hi) <= 1e-12 * scale
            assert abs(got[2] - tr) <= 1e-12 * n and got[3] == 0.0
        del H, Hv


def test_noalloc_binding_checks_its_arguments():
    import paper_2301_04642_gb300 as fe
    H = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    for bad_h, bad_o in [(H.float(), out), (H[:, :4], out), (H.t(), out), (H, out[:3]), (H, out.float()),
                         (H.cpu(), out)]:
        with pytest.raises(ValueError):
            fe.gershgorin_noalloc(bad_h, bad_o)


def test_noalloc_flags_nonfinite_then_recovers():
    import paper_2301_04642_gb300 as fe
    p = hp_synth.gapped(300, 150, (-3.0, -0.01), (0.01, 1.0), 31)
    Hd = torch.from_numpy(p.H).cuda()
    ref = ctx().gershgorin(Hd)
    bad = Hd.clone()
    bad[7, 11] = float("inf")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    fe.gershgorin_noalloc(bad, out)
    torch.cuda.synchronize()
    assert out[3].item() == 1.0
    fe.gershgorin_noalloc(Hd, out)          # the flag does not leak into the next call
    torch.cuda.synchronize()
    _check(out.cpu().tolist(), ref, 300)


def test_noalloc_rejects_oversize():
    """n above the fixed scratch (32768 rows) is refused on the host, before
    anything is queued, so small buffers suffice here."""
    import paper_2301_04642_gb300 as fe
    L = fe.load()
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = L.fe_k_gershgorin_noalloc(buf.data_ptr(), 32769, 32769, out.data_ptr(), None)
    assert rc == fe.FE_EINVAL
    assert b"32768" in L.fe_last_error_string(None)
