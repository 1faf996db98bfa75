"""Tensor-core tile shapes (128 x 256 and 128 x 128) and the tile-shape
autotuner through the C ABI, against the CPU oracle.

The symmetric product of Sec. III-B runs over upper-triangle tiles of either
width; a problem takes the width the context's table gives for its number of
128-row panels, and one launch may mix widths.  Every result must meet the
same tolerances whatever the width."""
import math

import numpy as np
import pytest

import hp_synth
import oracle
from gpu_util import need_gpu, torch

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]

TOL_EPS1, TOL_E, TOL_TR, TOL_IDEM = 1e-6, 1e-7, 1e-9, 1e-8


def new_ctx(**kw):
    need_gpu()
    import paper_2301_04642_gb300 as fe
    return fe.Context(device=0, **kw)


@pytest.fixture(scope="module")
def cx():
    c = new_ctx()
    yield c
    c.close()


def sym_f32(n, seed):
    G = hp_synth.normal(seed, n * n).reshape(n, n)
    return (0.5 * (G + G.T) / math.sqrt(n)).astype(np.float32)


@pytest.mark.parametrize("n", [16, 128, 200, 300, 1000, 2065])
@pytest.mark.parametrize("nslices", [2, 1])
def test_sym_square_narrow_tiles(cx, n, nslices):
    prec = "fp32" if nslices == 2 else "try_fp16"
    cx.set_tile_width(n, 128, prec)
    try:
        assert cx.tile_width(n, prec) == 128
        Y = sym_f32(n, 70 + n)
        Yd = torch.from_numpy(Y).cuda()
        C = torch.empty_like(Yd)
        cx.sym_square(Yd, C, nslices=nslices, bound=float(np.abs(Y).max()))
        Ch = C.cpu().numpy().astype(np.float64)
    finally:
        cx.set_tile_width(n, 0, prec)
    ref = oracle.matmul(Y.astype(np.float64), Y.astype(np.float64))
    absprod = oracle.matmul(np.abs(Y).astype(np.float64), np.abs(Y).astype(np.float64))
    # the same error bound as with 128 x 256 tiles: operand rounding (22 or 11
    # bits), four one-sided additions per 64-wide chunk, chunk sums rounded
    nchunks = math.ceil(n / 64)
    rel = (2.0 ** -21 if nslices == 2 else 2.0 ** -10) + 4 * 2.0 ** -23 + nchunks * 2.0 ** -24
    assert np.all(np.abs(Ch - ref) <= rel * absprod + 1e-30)
    assert np.array_equal(Ch, Ch.T)


def check_zero_t(p, D, res):
    f = (np.arange(p.n) < int(p.ne)).astype(float)
    Dref = oracle.density_from_eig(p.Q, f)
    Eref = float(np.sum(f * p.lam))
    assert res["status"] == 0
    assert np.linalg.norm(D - Dref) / math.sqrt(p.ne) <= TOL_EPS1
    assert abs(res["e_band"] - Eref) / p.ne <= TOL_E
    assert abs(np.trace(D) - p.ne) <= TOL_TR
    assert np.linalg.norm(oracle.matmul(D, D) - D) <= TOL_IDEM


@pytest.mark.parametrize("n,ne", [(300, 250), (1000, 850), (1250, 1000)])
@pytest.mark.parametrize("precision", ["mixed", "fp32"])
def test_zero_t_solve_narrow_tiles(cx, n, ne, precision):
    p = hp_synth.gapped(n, ne, (-3.0, -0.01), (0.01, 1.0), 4000 + n)
    cx.set_tile_width(n, 128, precision)
    try:
        D = np.zeros_like(p.H)
        res = cx.solve(p.H, p.ne, D=D, precision=precision)
    finally:
        cx.set_tile_width(n, 0, precision)
    if precision == "mixed":
        check_zero_t(p, D, res)
    else:
        # split-FP16 products only: D and the band energy within the FP64
        # tolerances, the trace matched, idempotency at the 22-bit level of
        # the products (the split phase stops once ||X^2 - X||_F <= 2^-20
        # sqrt(N_e); its last product at most doubles one side's deviations)
        assert res["status"] == 0
        f = (np.arange(n) < ne).astype(float)
        Dref = oracle.density_from_eig(p.Q, f)
        assert np.linalg.norm(D - Dref) / math.sqrt(ne) <= TOL_EPS1
        assert abs(res["e_band"] - float(np.sum(f * p.lam))) / ne <= TOL_E
        assert abs(np.trace(D) - p.ne) <= 1e-6 * p.ne
        assert np.linalg.norm(oracle.matmul(D, D) - D) <= 4.0 * 2.0 ** -20 * math.sqrt(ne)


def test_fermi_solve_narrow_tiles(cx):
    n, ne, kT = 517, 440.5, 0.01
    p = hp_synth.smeared(n, ne, kT, -2.0, 1.0, 8)
    cx.set_tile_width(n, 128, "mixed")
    try:
        D = np.zeros_like(p.H)
        r = cx.solve(p.H, ne, kT=kT, D=D)
    finally:
        cx.set_tile_width(n, 0, "mixed")
    ref = oracle.density(p.H, ne, kT)
    assert r["status"] == 0
    assert np.linalg.norm(D - ref["D"]) / math.sqrt(ne) <= TOL_EPS1
    assert abs(r["e_band"] - ref["e_band"]) / ne <= TOL_E
    assert abs(np.trace(D) - ne) <= TOL_TR


def test_batch_mixes_tile_widths(cx):
    """One launch per step over problems of both widths (narrow: 300 and 1250;
    wide: 700 and 2000); each result meets the tolerances and agrees with the
    same problem solved alone."""
    sizes = [(300, 250), (700, 600), (1250, 1000), (2000, 1700)]
    narrow = {300, 1250}
    ps = [hp_synth.gapped(n, ne, (-3.0, -0.01), (0.01, 1.0), 5200 + n) for n, ne in sizes]
    for p in ps:
        cx.set_tile_width(p.n, 128 if p.n in narrow else 256, "mixed")
    try:
        assert [cx.tile_width(p.n) for p in ps] == [128, 256, 128, 256]
        Ds = [np.zeros_like(p.H) for p in ps]
        _, rs = cx.solve_batch([dict(H=p.H, ne=p.ne, D=D) for p, D in zip(ps, Ds)])
        alone = []
        for p in ps[:2]:
            D1 = np.zeros_like(p.H)
            alone.append((D1, cx.solve(p.H, p.ne, D=D1)))
    finally:
        for p in ps:
            cx.set_tile_width(p.n, 0, "mixed")
    for p, D, r in zip(ps, Ds, rs):
        check_zero_t(p, D, r)
    # the rounding of a problem's sums depends on its company (the split of
    # the launch's work over the SMs): equal within the stated tolerances
    for (D1, r1), p, D, r in zip(alone, ps, Ds, rs):
        assert np.linalg.norm(D1 - D) / math.sqrt(p.ne) <= TOL_EPS1
        assert abs(r1["e_band"] - r["e_band"]) / p.ne <= TOL_E


def test_autotune_fills_table_and_file(tmp_path):
    path = tmp_path / "tiles.txt"
    with new_ctx(autotune_path=str(path)) as c:
        ents = c.autotune([300, 520, 1100], precision="mixed", reps=1)
        assert [e["n"] for e in ents] == [300, 520, 1100]
        for e in ents:
            assert e["bn"] in (128, 256)
            assert e["ms_256"] > 0 and e["ms_128"] > 0
            assert e["bn"] == (128 if e["ms_128"] < e["ms_256"] else 256)
            assert c.tile_width(e["n"]) == e["bn"]
        chosen = {e["n"]: e["bn"] for e in ents}
        # a size with no entry of its own takes the nearest panel count's
        assert c.tile_width(1000) == chosen[1100]
        # other policies are untouched
        assert c.tile_width(300, "fp32") == 256
    text = path.read_text().splitlines()
    assert text[0] == "fe-autotune 1" and len(text) == 4
    with new_ctx(autotune_path=str(path)) as c2:
        for n, bn in chosen.items():
            assert c2.tile_width(n) == bn
        # a solve with the loaded table meets the tolerances
        p = hp_synth.gapped(520, 440, (-3.0, -0.01), (0.01, 1.0), 5900)
        D = np.zeros_like(p.H)
        check_zero_t(p, D, c2.solve(p.H, p.ne, D=D))


def test_autotune_batch_keeps_a_faster_table():
    sizes = [(300, 250), (520, 440), (700, 600), (1250, 1000)]
    ps = [hp_synth.gapped(n, ne, (-3.0, -0.01), (0.01, 1.0), 6100 + n) for n, ne in sizes]
    with new_ctx() as c:
        items = [dict(H=p.H, ne=p.ne) for p in ps]
        trials = c.autotune_batch(items, reps=1)
        assert 2 <= len(trials) <= len(sizes) + 1 and all(t > 0 for t in trials)
        widths = [c.tile_width(p.n) for p in ps]
        k = sum(w == 128 for w in widths)
        # the smallest k sizes are narrow; every kept step was faster, the
        # first rejected one (if any) was not
        assert widths == [128] * k + [256] * (len(ps) - k)
        for i in range(1, k + 1):
            assert trials[i] < trials[i - 1]
        if k + 1 < len(trials):
            assert trials[k + 1] >= 0.995 * trials[k]
        Ds = [np.zeros_like(p.H) for p in ps]
        _, rs = c.solve_batch([dict(H=p.H, ne=p.ne, D=D) for p, D in zip(ps, Ds)])
        for p, D, r in zip(ps, Ds, rs):
            check_zero_t(p, D, r)


def test_autotune_file_errors(tmp_path):
    import paper_2301_04642_gb300 as fe
    bad = tmp_path / "bad.txt"
    bad.write_text("fe-autotune 1\n4 0 192 1.0 1.0\n")
    with pytest.raises(fe.FeError):
        new_ctx(autotune_path=str(bad))
    bad.write_text("something else\n")
    with pytest.raises(fe.FeError):
        new_ctx(autotune_path=str(bad))
    with new_ctx() as c:
        with pytest.raises(fe.FeError):
            c.autotune([300], precision="fp64")
        with pytest.raises(fe.FeError):
            c.autotune([1])
        with pytest.raises(fe.FeError):
            c.set_tile_width(300, 192)
