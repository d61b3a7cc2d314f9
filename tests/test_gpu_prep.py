"""Image-quality pre-processing (Sect. 3.2) through the C ABI, against the
FP32 oracle on identical inputs: master sky (NaN-aware, masked median),
nearest-in-time sky subtraction, sigma-clip bad pixel map and the
neighbour-median bad pixel correction -- all selections or exact
arithmetic, so compared bit for bit."""
import numpy as np
import pytest

import oracle
from paper_1510_04331_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_1510_04331_gb300 import graphic
    return graphic


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _same(a, b):
    return np.array_equal(np.isnan(a), np.isnan(b)) and np.array_equal(a[~np.isnan(a)], b[~np.isnan(b)])


@pytest.mark.parametrize("T", [1, 2, 7, 30])
def test_sky_median_against_oracle(g, T):
    rng = np.random.default_rng(40 + T)
    n = 64
    c = rng.normal(200.0, 10.0, (T, n, n)).astype(np.float32)
    c[rng.random((T, n, n)) < 0.02] = np.nan
    c[:, 5, 9] = np.nan                                   # no value left
    c[:, 11, 11] = 3.0                                    # ties
    mx, my = rng.uniform(10, 50, T), rng.uniform(10, 50, T)
    got = g.context().graphic_sky_median(_dev(c), mx, my, 6.5).cpu().numpy()
    assert _same(got, oracle.sky_median(c, mx, my, 6.5))
    got2 = g.context().graphic_sky_median(_dev(c)).cpu().numpy()
    assert _same(got2, oracle.sky_median(c))


def test_sky_median_long_stack(g):
    rng = np.random.default_rng(9)
    T, n = 300, 128
    c = rng.normal(50.0, 3.0, (T, n, n)).astype(np.float32)
    c[rng.random((T, n, n)) < 0.01] = np.nan
    mx, my = rng.uniform(30, 90, T), rng.uniform(30, 90, T)
    got = g.context().graphic_sky_median(_dev(c), mx, my, 12.0).cpu().numpy()
    assert _same(got, oracle.sky_median(c, mx, my, 12.0))


def test_sky_subtract_against_oracle(g):
    rng = np.random.default_rng(10)
    T, n = 11, 64
    c = rng.normal(0, 1, (T, n, n)).astype(np.float32)
    skies = rng.normal(0, 1, (4, n, n)).astype(np.float32)
    ft = np.sort(rng.uniform(0, 10, T))
    st = np.array([0.5, 3.0, 3.0 + 1e-9, 9.0])
    got = g.context().graphic_sky_subtract(_dev(c), _dev(skies), ft, st).cpu().numpy()
    assert np.array_equal(got, oracle.sky_subtract(c, skies, ft, st))


def test_bad_pixel_map_against_oracle(g):
    rng = np.random.default_rng(11)
    n = 128
    ref = rng.normal(1000.0, 20.0, (n, n)).astype(np.float32)
    idx = rng.choice(n * n, 60, replace=False)
    ref.ravel()[idx[:30]] = 5000.0
    ref.ravel()[idx[30:]] = -2000.0
    for C in (3.0, 5.0):
        got = g.context().graphic_bad_pixel_map(_dev(ref), C).cpu().numpy().astype(bool)
        assert np.array_equal(got, oracle.bad_pixel_map(ref, C))
    assert g.context().graphic_bad_pixel_map(_dev(ref), 5.0).cpu().numpy().sum() == 60


def test_bad_pixel_fix_against_oracle(g):
    rng = np.random.default_rng(12)
    T, n = 5, 64
    c = synth.random_frames(T, n, seed=13, smooth=True) * 100.0
    c += rng.normal(0, 1, c.shape).astype(np.float32)
    bad = rng.random((n, n)) < 0.01
    bad[20:24, 30:33] = True                              # a clump
    bad[0, :5] = True                                     # at the border
    c[1, 40, 41] = np.nan
    c[2, 7, 50] = np.inf
    c[3, 10:16, 10:16] = np.nan                           # a 6 x 6 hole in one frame
    want, st = oracle.bad_pixel_fix(c, bad)
    assert st == 0
    x = _dev(c)
    g.context().graphic_bad_pixel_fix(x, _dev(bad.astype(np.uint8)))
    got = x.cpu().numpy()
    assert np.array_equal(got, want)
    assert np.isfinite(got).all()


def test_bad_pixel_fix_without_map_and_hopeless_frame(g):
    c = np.full((2, 64, 64), 7.5, np.float32)
    c[0, 30:33, 30:33] = np.nan
    x = _dev(c)
    g.context().graphic_bad_pixel_fix(x)
    assert np.array_equal(x.cpu().numpy(), np.full((2, 64, 64), 7.5, np.float32))
    c[1] = np.nan
    with pytest.raises(g.GraphicError, match="NONFINITE"):
        g.context().graphic_bad_pixel_fix(_dev(c))


def test_prepared_cube_reduces(g):
    """Sky subtraction and bad pixel correction make a cube with NaN and hot
    pixels acceptable to the reduction (which refuses non-finite input)."""
    d = synth.make_cube(16, 64, seed=14, parang=np.linspace(0, 40, 16), edges=synth.default_edges(64))
    raw = d.cube + 50.0
    raw[3, 5, 5] = np.nan
    raw[:, 40, 40] = 1e6
    x = _dev(raw)
    sky = torch.full((1, 64, 64), 50.0, device="cuda")
    ctx = g.context()
    x = ctx.graphic_sky_subtract(x, sky, np.arange(16.0), [0.0])
    with pytest.raises(g.GraphicError):
        ctx.graphic_reduce(x, d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges)
    m = ctx.graphic_bad_pixel_map(x[0].contiguous(), 8.0)
    ctx.graphic_bad_pixel_fix(x, m)
    out = ctx.graphic_reduce(x, d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges).cpu().numpy()
    assert np.isfinite(out).all()
