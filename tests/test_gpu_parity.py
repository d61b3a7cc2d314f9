"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Floating-point steps (shift, rotation, whole reduction): max |gpu - oracle|
<= 1e-5 of the peak |value| of the step's input, element by element.
Selection steps (median PSF subtraction, collapse) on identical FP32 inputs:
bit-exact against the oracle's FP32 median arithmetic.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1510_04331_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def g():
    from paper_1510_04331_gb300 import graphic
    return graphic


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to("cuda:0")


def rel_err(gpu, ref, peak):
    return float(np.abs(gpu.cpu().numpy().astype(np.float64) - ref).max()) / peak


# --------------------------------------------------------------------------
# shift
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,T", [(64, 5), (128, 7), (256, 3), (512, 2), (1024, 1)])
def test_shift_matches_oracle(g, n, T):
    rng = np.random.default_rng(n + T)
    f = synth.random_frames(T, n, seed=n).astype(np.float32)
    dx = rng.uniform(-3, 3, T)
    dy = rng.uniform(-3, 3, T)
    dx[0], dy[0] = n / 2, -n / 2 + 0.3          # extreme shifts
    out = g.graphic_shift(dev(f), dx, dy)
    ref = oracle.shift(f.astype(np.float64), dx, dy)
    assert rel_err(out, ref, np.abs(f).max()) <= TOL


def test_shift_small_workload_with_star(g):
    d = synth.small_cube(seed=0)
    out = g.graphic_shift(dev(d.cube), d.dx, d.dy)
    ref = oracle.shift(d.cube.astype(np.float64), d.dx, d.dy)
    assert rel_err(out, ref, np.abs(d.cube).max()) <= TOL


def test_integer_shift_is_roll_and_zero_shift_is_exact(g):
    n = 128
    f = synth.random_frames(3, n, seed=1)
    out = g.graphic_shift(dev(f), [5, 0, -7], [-3, 0, 64]).cpu().numpy()
    ref = np.zeros_like(f)
    for t, (dx, dy) in enumerate([(5, -3), (0, 0), (-7, 64)]):
        src = f[t]
        for i in range(n):
            si = i - dy
            if 0 <= si < n:
                lo, hi = max(0, dx), min(n, n + dx)
                ref[t, i, lo:hi] = src[si, lo - dx:hi - dx]
    assert np.abs(out - ref).max() <= TOL * np.abs(f).max()
    assert np.array_equal(out[1], f[1])          # zero shift: exact copy


def test_shift_in_place_and_empty(g):
    f = synth.random_frames(4, 64, seed=2)
    t = dev(f)
    ref = g.graphic_shift(t, [0.3] * 4, [-0.2] * 4).cpu().numpy()
    g.graphic_shift(t, [0.3] * 4, [-0.2] * 4, out=t)
    assert np.array_equal(t.cpu().numpy(), ref)
    e = torch.empty((0, 64, 64), device="cuda:0")
    g.graphic_shift(e, [], [])


# --------------------------------------------------------------------------
# rotation
# --------------------------------------------------------------------------

ANGLES = [0.0, 11.3, -11.3, 44.99, 45.0, -45.0, 89.5, 90.0, 135.0, 180.0, -170.25, 270.0, 300.7, 359.9, -80.3]


@pytest.mark.parametrize("n", [64, 128, 256])
def test_rotate_matches_oracle(g, n):
    T = len(ANGLES)
    f = synth.random_frames(T, n, seed=n + 1)
    out = g.graphic_rotate(dev(f), ANGLES)
    ref = oracle.rotate(f.astype(np.float64), ANGLES)
    assert rel_err(out, ref, np.abs(f).max()) <= TOL


@pytest.mark.parametrize("n", [512, 1024])
def test_rotate_matches_oracle_large(g, n):
    th = [37.7, -101.2, 100.4, 171.9, -178.0]     # quarter turns q = 0, 3, 1, 2, 2
    f = synth.random_frames(len(th), n, seed=n + 2)
    out = g.graphic_rotate(dev(f), th)
    ref = oracle.rotate(f.astype(np.float64), th)
    assert rel_err(out, ref, np.abs(f).max()) <= TOL


@pytest.mark.parametrize("n", [64, 512])
def test_rotate_quarter_turns_exact(g, n):
    f = synth.random_frames(5, n, seed=3)
    th = [0.0, 90.0, 180.0, 270.0, -90.0]
    out = g.graphic_rotate(dev(f), th).cpu().numpy()
    ref = oracle.rotate(f.astype(np.float64), th).astype(np.float32)
    assert np.array_equal(out, ref)


def test_rotate_round_trip_paper_case(g):
    n = 128
    f = synth.random_frames(2, n, seed=4, smooth=True)
    t = g.graphic_rotate(dev(f), [11.3, 11.3])
    back = g.graphic_rotate(t, [-11.3, -11.3]).cpu().numpy()
    assert np.abs(back - f).max() <= 2e-5 * np.abs(f).max()


# --------------------------------------------------------------------------
# median PSF subtraction and collapse: bit-exact on identical FP32 inputs
# --------------------------------------------------------------------------

def _adi_case(T, n, seed, ties=False):
    rng = np.random.default_rng(seed)
    c = (rng.standard_normal((T, n, n)) * 50 + 100).astype(np.float32)
    pa = np.sort(rng.uniform(-40, 40, T))
    if ties and T > 3:
        pa[1] = pa[0]
        pa[T // 2] = pa[T // 2 - 1]
        c[:, 5, 5] = 3.0               # constant pixel: ties in value
    perm = rng.permutation(T)          # angles need not be sorted in time
    return c[perm].copy(), pa[perm].copy()


@pytest.mark.parametrize("T", [1, 2, 3, 31, 32, 33, 100, 257])
def test_adi_subtract_bit_exact(g, T):
    n = 64
    c, pa = _adi_case(T, n, seed=T, ties=True)
    edges = [0.0, 3.0, 6.0, 12.0, 24.0, 40.0]
    out = g.graphic_adi_subtract(dev(c), pa, 4.0, 1.5, edges).cpu().numpy()
    ref = oracle.adi_subtract(c, pa, 4.0, 1.5, edges)
    assert np.array_equal(out, ref)


def test_adi_subtract_small_workload_bit_exact(g):
    d = synth.small_cube(seed=0)
    out = g.graphic_adi_subtract(dev(d.cube), d.parang, d.fwhm, d.n_fwhm, d.edges).cpu().numpy()
    ref = oracle.adi_subtract(d.cube, d.parang, d.fwhm, d.n_fwhm, d.edges)
    assert np.array_equal(out, ref)


def test_adi_subtract_max_frames_bit_exact_sampled(g):
    T, n = 2048, 64
    c, pa = _adi_case(T, n, seed=7)
    edges = [2.0, 10.0, 20.0, 46.0]
    out = g.graphic_adi_subtract(dev(c), pa, 4.0, 1.5, edges).cpu().numpy()
    pix = np.random.default_rng(0).choice(n * n, 24, replace=False)
    ref = oracle.adi_subtract(c, pa, 4.0, 1.5, edges, pixels=pix)
    got = out.reshape(T, n * n)[:, pix].T
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("T", [1, 2, 3, 32, 33, 1000, 2048, 2049, 4097])
def test_collapse_bit_exact(g, T):
    n = 64
    rng = np.random.default_rng(T)
    c = (rng.standard_normal((T, n, n)) * 10).astype(np.float32)
    c[:, 0, :8] = 1.0                  # all-equal pixels
    c[:, 1, 0] = -0.0
    c[: T // 2, 1, 0] = 0.0            # signed zeros
    out = g.graphic_collapse_median(dev(c)).cpu().numpy()
    assert np.array_equal(out, np.median(c, axis=0).astype(np.float32))
    pix = np.arange(0, n * n, 97)
    assert np.array_equal(out.ravel()[pix], oracle.collapse_median(c, pixels=pix))


@pytest.mark.parametrize("T", [40, 500])
def test_adi_subtract_unsampled_spread_bit_exact(g, T):
    """Median PSF pixels whose spread an even 32-frame sample (in angle
    order) does not show: a constant sample around varying frames, heavy
    outliers, half the sample far below the rest."""
    n = 64
    rng = np.random.default_rng(200 + T)
    c = (rng.standard_normal((T, n, n)) * 50 + 100).astype(np.float32)   # angle order
    pa = np.sort(rng.uniform(-40, 40, T))
    sampled = (np.arange(32) * T) // 32
    rest = np.setdiff1d(np.arange(T), sampled)
    c[sampled, 10, :] = 7.0
    out_i = rng.choice(T, T // 10, replace=False)
    c[out_i, 11, :] = np.where(rng.random((out_i.size, 1)) < 0.5, -1e30, 1e30).astype(np.float32)
    c[sampled[::2], 12, :] = -1e4
    c[rest, 13, :] = np.float32(3.0)
    perm = rng.permutation(T)
    c, pa = c[perm].copy(), pa[perm].copy()
    edges = [2.0, 9.0, 16.0, 30.0]
    out = g.graphic_adi_subtract(dev(c), pa, 4.0, 1.5, edges).cpu().numpy()
    pix = np.concatenate([np.arange(10 * n, 14 * n), rng.choice(n * n, 64, replace=False)])
    ref = oracle.adi_subtract(c, pa, 4.0, 1.5, edges, pixels=pix)
    assert np.array_equal(out.reshape(T, n * n)[:, pix].T, ref)


@pytest.mark.parametrize("T", [32, 33, 64, 65, 500, 2000])
def test_collapse_outliers_and_unsampled_spread_bit_exact(g, T):
    """Pixels whose spread an even 32-frame sample of the cube does not show:
    heavy outliers, a constant sample around varying frames, a median
    outside the sample's range, a median equal to the sample's extreme."""
    n = 64
    rng = np.random.default_rng(100 + T)
    c = (rng.standard_normal((T, n, n)) * 10).astype(np.float32)
    sampled = (np.arange(32) * T) // 32
    rest = np.setdiff1d(np.arange(T), sampled)
    out_i = rng.choice(T, T // 10, replace=False)
    c[out_i, 0, 0] = np.where(rng.random(out_i.size) < 0.5, -1e30, 1e30).astype(np.float32)
    c[:, 0, 1] = 5.0
    c[rest, 0, 1] = rng.standard_normal(rest.size).astype(np.float32)
    c[sampled, 0, 2] = 0.0
    c[rest, 0, 2] = np.arange(1, rest.size + 1, dtype=np.float32)
    c[:, 0, 3] = np.float32(2.0)
    c[sampled[: 16], 0, 3] = np.float32(-7.0)
    c[rest, 0, 3] = rng.uniform(-7, 30, rest.size).astype(np.float32)
    c[:, 0, 4] = np.float32(-7.0)
    k = min(rest.size, T // 2 + 2)
    c[rest[:k], 0, 4] = rng.uniform(0, 1, k).astype(np.float32)
    out = g.graphic_collapse_median(dev(c)).cpu().numpy()
    assert np.array_equal(out, np.median(c, axis=0).astype(np.float32))


# --------------------------------------------------------------------------
# whole reduction
# --------------------------------------------------------------------------

def test_reduce_small_workload_matches_fp64_oracle(g):
    d = synth.small_cube(seed=0)
    out = g.graphic_reduce(dev(d.cube), d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges)
    ref = oracle.reduce(d.cube.astype(np.float64), d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges)
    assert rel_err(out, ref, np.abs(d.cube).max()) <= TOL


def test_reduce_host_equals_device_path(g):
    d = synth.small_cube(seed=1)
    a = g.graphic_reduce(dev(d.cube), d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges).cpu().numpy()
    b = g.graphic_reduce_host(d.cube, d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges)
    assert np.array_equal(a, b)


def test_reduce_host_pieces_equal_device_path(g):
    """300 frames of 512 x 512 (300 MB): the host-buffer path copies and
    shifts the cube in two pieces; the result is the device path's, bit for
    bit."""
    d = synth.make_cube(300, 512, seed=5, parang=synth.altaz_parang(300), edges=synth.default_edges(512))
    a = g.graphic_reduce(dev(d.cube), d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges).cpu().numpy()
    b = g.graphic_reduce_host(d.cube, d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges)
    assert np.array_equal(a, b)


@pytest.fixture(scope="module")
def survey():
    return synth.survey_cube(seed=1)


def test_survey_scale_stages_sampled(g, survey):
    """2000 frames of 512 x 512 (padded to 1024), stage by stage through the
    same calls graphic_reduce makes, checked on sampled frames / pixels."""
    d = survey
    T, n = d.cube.shape[0], d.cube.shape[1]
    cube = dev(d.cube)
    sh = g.graphic_shift(cube, d.dx, d.dy)
    fr = [0, 999, T - 1]
    ref = oracle.shift(d.cube[fr].astype(np.float64), d.dx[fr], d.dy[fr])
    assert rel_err(sh[fr], ref, np.abs(d.cube).max()) <= TOL

    res = g.graphic_adi_subtract(sh, d.parang, d.fwhm, d.n_fwhm, d.edges)
    sh_np = sh.cpu().numpy()
    pix = np.array([0, n * n // 2 + n // 2 + 5, (n // 2 + 7) * n + n // 2 - 3, (n // 2 - 60) * n + n // 2 + 41,
                    (n // 2 + 150) * n + 20, n * n - 1])
    ref = oracle.adi_subtract(sh_np, d.parang, d.fwhm, d.n_fwhm, d.edges, pixels=pix)
    got = res.cpu().numpy().reshape(T, n * n)[:, pix].T
    assert np.array_equal(got, ref)
    del sh_np

    rot = g.graphic_rotate(res, -d.parang)
    res_np = res.cpu().numpy()
    ref = oracle.rotate(res_np[fr].astype(np.float64), -d.parang[fr])
    assert rel_err(rot[fr], ref, np.abs(res_np).max()) <= TOL

    img = g.graphic_collapse_median(rot).cpu().numpy()
    rot_np = rot.cpu().numpy()
    sp = np.arange(0, n * n, 4099)
    assert np.array_equal(img.ravel()[sp], oracle.collapse_median(rot_np, pixels=sp))

    # the composite call runs the same kernels in the same order: bit-identical
    full = g.graphic_reduce(cube, d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges).cpu().numpy()
    assert np.array_equal(full, img)
    # the injected companions come back near their injected positions
    c = n // 2
    r, pa0, _ = d.companions[0]
    i0 = int(round(c + r * math.sin(math.radians(pa0))))
    j0 = int(round(c + r * math.cos(math.radians(pa0))))
    win = full[i0 - 3:i0 + 4, j0 - 3:j0 + 4]
    assert win.max() > 20.0


# --------------------------------------------------------------------------
# errors
# --------------------------------------------------------------------------

def test_errors(g):
    f = dev(synth.random_frames(2, 64, seed=0))
    with pytest.raises(g.GraphicError) as e:
        g.graphic_shift(f, [40.0, 0], [0, 0])
    assert e.value.code == -1
    with pytest.raises(g.GraphicError) as e:
        g.graphic_shift(dev(synth.random_frames(1, 96, seed=0)), [0.0], [0.0])
    assert e.value.code == -2
    bad = synth.random_frames(2, 64, seed=0)
    bad[1, 3, 4] = np.nan
    with pytest.raises(g.GraphicError) as e:
        g.graphic_shift(dev(bad), [0.1, 0.1], [0, 0])
    assert e.value.code == -5
    with pytest.raises(g.GraphicError) as e:
        g.graphic_rotate(dev(bad), [10.0, 10.0])
    assert e.value.code == -5
    with pytest.raises(g.GraphicError) as e:
        g.graphic_adi_subtract(f, [0, 1], 4.0, 1.5, [5.0, 2.0])
    assert e.value.code == -1
    with pytest.raises(g.GraphicError) as e:
        g.graphic_adi_subtract(dev(bad), [0, 10], 4.0, 1.5, [0.0, 50.0])
    assert e.value.code == -5
    big = torch.zeros((2049, 64, 64), device="cuda:0")
    with pytest.raises(g.GraphicError) as e:
        g.graphic_adi_subtract(big, np.zeros(2049), 4.0, 1.5, [0.0, 50.0])
    assert e.value.code == -2
    # the context stays usable after errors
    out = g.graphic_shift(f, [0.5, 0.5], [0.0, 0.0])
    assert torch.isfinite(out).all()


@pytest.mark.parametrize("T,levels", [(300, 3), (700, 7), (1500, 50), (2048, 2)])
def test_adi_subtract_ties_bit_exact(g, T, levels):
    """Quantised values: many keys equal to the band's boundary keys, which
    the band path has to split by frame order; results must stay exact."""
    n = 64
    rng = np.random.default_rng(T + levels)
    c = rng.integers(0, levels, (T, n, n)).astype(np.float32) * 0.5 - 1.0
    pa = np.linspace(-60, 60, T) + rng.uniform(-0.01, 0.01, T)
    edges = [1.0, 6.0, 14.0, 30.0, 46.0]
    out = g.graphic_adi_subtract(dev(c), pa, 4.0, 1.5, edges).cpu().numpy()
    pix = np.random.default_rng(1).choice(n * n, 40, replace=False)
    pix = np.concatenate([pix, [n * n // 2 + n // 2 + 3, (n // 2 + 20) * n + n // 2]])
    ref = oracle.adi_subtract(c, pa, 4.0, 1.5, edges, pixels=pix)
    assert np.array_equal(out.reshape(T, n * n)[:, pix].T, ref)


def test_adi_subtract_thin_annuli_bit_exact(g):
    """Annuli one pixel wide: a group of 4 neighbouring pixels spans up to
    four annuli (the band kernel stages two gates and reads the others)."""
    T, n = 120, 64
    c, pa = _adi_case(T, n, seed=3)
    edges = [6.0, 7.0, 8.0, 9.0, 10.0, 11.0, 12.0, 30.0]
    out = g.graphic_adi_subtract(dev(c), pa, 4.0, 1.5, edges).cpu().numpy()
    ref = oracle.adi_subtract(c, pa, 4.0, 1.5, edges)
    assert np.array_equal(out, ref)
