"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these re-types the oracle's formulas: every expected value comes
from a different route (a library routine, a closed form, an exact index
map, an invariant, a geometric identity), chosen so that a dropped term,
a flipped sign, a wrong index or a transposed operand in the oracle fails
at least one test.  CPU only.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1510_04331_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_cases.json")))


# --------------------------------------------------------------------------
# FFT (Sect. 3.3.1 definitions)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("M", [1, 2, 4, 8, 16, 32, 64])
def test_fft_matches_bruteforce_dft(M):
    rng = np.random.default_rng(M)
    x = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    X = oracle.fft(x)
    D = oracle.dft(x)
    assert np.abs(X - D).max() <= 1e-13 * max(1.0, np.abs(D).max())
    # library routine (numpy) as an independent second route
    assert np.abs(X - np.fft.fft(x)).max() <= 1e-13 * max(1.0, np.abs(D).max())
    assert np.abs(oracle.fft(x, inverse=True) - np.fft.ifft(x)).max() <= 1e-14 * max(1.0, np.abs(x).max())


@pytest.mark.parametrize("M", [128, 1024])
def test_fft_roundtrip_and_parseval(M):
    rng = np.random.default_rng(7)
    x = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    X = oracle.fft(x)
    assert abs(np.sum(np.abs(X) ** 2) / M - np.sum(np.abs(x) ** 2)) <= 1e-11 * np.sum(np.abs(x) ** 2)
    assert np.abs(oracle.fft(X, inverse=True) - x).max() <= 1e-13
    # a single tone lands in exactly one bin, at +k for exp(+i 2 pi k n / M)
    k = 5
    tone = np.exp(2j * np.pi * k * np.arange(M) / M)
    T = oracle.fft(tone)
    assert abs(T[k] - M) < 1e-9 and np.abs(np.delete(T, k)).max() < 1e-9


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fft(np.ones(12))


# --------------------------------------------------------------------------
# Shift (Sect. 3.3.1)
# --------------------------------------------------------------------------

def _roll_zero(f, dx, dy):
    """out[i][j] = in[i - dy][j - dx], zero where the source is outside."""
    N = f.shape[-1]
    out = np.zeros_like(f)
    for i in range(N):
        for j in range(N):
            si, sj = i - dy, j - dx
            if 0 <= si < N and 0 <= sj < N:
                out[..., i, j] = f[..., si, sj]
    return out


@pytest.mark.parametrize("dx,dy", [(1, 0), (0, 1), (2, -3), (-4, 4), (8, 8), (-8, -8), (0, 0)])
def test_integer_shift_is_zero_filled_roll(dx, dy):
    f = synth.random_frames(1, 16, seed=3).astype(np.float64)
    out = oracle.shift(f, [dx], [dy])
    assert np.abs(out - _roll_zero(f, dx, dy)).max() <= 1e-13
    assert oracle.last_max_imag() <= 1e-13


def _dirichlet_line(M, p0, d):
    """Closed form of a unit impulse at p0 shifted by d on a periodic line of
    length M with the Nyquist bin weighted by cos(pi d): the Dirichlet kernel
    sin((K + 1/2) u) / sin(u / 2), K = M/2 - 1, u = 2 pi (n - p0 - d) / M,
    plus cos(pi d) (-1)^(n - p0), all over M."""
    n = np.arange(M)
    u = 2.0 * np.pi * (n - p0 - d) / M
    K = M // 2 - 1
    with np.errstate(invalid="ignore", divide="ignore"):
        core = np.sin((K + 0.5) * u) / np.sin(u / 2.0)
    core = np.where(np.abs(np.sin(u / 2.0)) < 1e-300, 2 * K + 1.0, core)
    return (core + np.cos(np.pi * d) * (-1.0) ** (n - p0)) / M


def test_gibbs_single_pixel_matches_dirichlet_closed_form():
    case = GOLD["gibbs_single_pixel_shift"]
    dx, dy = case["dx"], case["dy"]
    N = 32
    M = 2 * N
    i0, j0 = 13, 17
    f = np.zeros((1, N, N))
    f[0, i0, j0] = 1.0
    out = oracle.shift(f, [dx], [dy])[0]
    kx = _dirichlet_line(M, j0 + N // 2, dx)[N // 2:N // 2 + N]
    ky = _dirichlet_line(M, i0 + N // 2, dy)[N // 2:N // 2 + N]
    assert np.abs(out - np.outer(ky, kx)).max() <= 1e-14
    # ringing present (the Gibbs pattern of the figure): negative lobes
    assert out.min() < -0.01


def test_shift_of_sampled_gaussian_is_analytic_gaussian():
    N = 64
    c = N / 2
    s = 2.5
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    g = lambda x0, y0: np.exp(-((xx - x0) ** 2 + (yy - y0) ** 2) / (2 * s * s))
    out = oracle.shift(g(c, c)[None], [1.37], [-2.61])[0]
    assert np.abs(out - g(c + 1.37, c - 2.61)).max() <= 1e-10


def test_shift_round_trip_paper_case():
    case = GOLD["shift_round_trip"]
    N = 64
    f = synth.random_frames(2, N, seed=5, smooth=True, dtype=np.float64)
    there = oracle.shift(f, [case["dx"]] * 2, [case["dy"]] * 2)
    back = oracle.shift(there, [-case["dx"]] * 2, [-case["dy"]] * 2)
    assert np.abs(back - f).max() <= 1e-9 * np.abs(f).max()


def test_shift_separable_equals_2d():
    f = synth.random_frames(1, 32, seed=9).astype(np.float64)
    both = oracle.shift(f, [0.37], [-1.21])
    x_then_y = oracle.shift(oracle.shift(f, [0.37], [0.0]), [0.0], [-1.21])
    assert np.abs(both - x_then_y).max() <= 1e-12


def test_shift_flux_conserved_on_padded_frame():
    f = synth.random_frames(1, 32, seed=11)[0].astype(np.float64)
    out = oracle.shift_padded(f, 0.41, -0.77)
    assert abs(out.sum() - f.sum()) <= 1e-11 * np.abs(f).sum()


@pytest.mark.parametrize("d", [0.0, 0.25, 0.5, 0.9, 3.3, -2.5])
def test_shift_line_parseval_with_nyquist_term(d):
    M = 64
    x = np.random.default_rng(1).standard_normal(M)
    y = oracle.shift_line(x, d)
    nyq = np.sum(x * (-1.0) ** np.arange(M))
    expect = np.sum(x * x) - math.sin(math.pi * d) ** 2 * nyq * nyq / M
    assert abs(np.sum(y * y) - expect) <= 1e-11 * np.sum(x * x)
    assert oracle.last_max_imag() <= 1e-12


def test_shift_sign_moves_content_positive():
    N = 64
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    f = np.exp(-((xx - 20.0) ** 2 + (yy - 30.0) ** 2) / (2 * 3.0 ** 2))[None]
    out = oracle.shift(f, [0.25], [-0.5])[0]
    # the centroid moves by (+0.25, -0.5): content moves by +d
    assert abs((out * xx).sum() / out.sum() - 20.25) < 1e-9
    assert abs((out * yy).sum() / out.sum() - 29.5) < 1e-9


# --------------------------------------------------------------------------
# Rotation (Sect. 3.4)
# --------------------------------------------------------------------------

def _rot90_map(f, q):
    """Exact rotation by 90 q degrees about (N/2, N/2), counter-clockwise,
    built from the geometry: output pixel (x, y) takes input R(-90q)(x, y)."""
    N = f.shape[-1]
    c = N // 2
    out = np.zeros_like(f)
    ang = -q * math.pi / 2
    ca, sa = round(math.cos(ang)), round(math.sin(ang))
    for i in range(N):
        for j in range(N):
            x, y = j - c, i - c
            xs, ys = ca * x - sa * y, sa * x + ca * y
            si, sj = ys + c, xs + c
            if 0 <= si < N and 0 <= sj < N:
                out[..., i, j] = f[..., si, sj]
    return out


@pytest.mark.parametrize("theta,q", [(90.0, 1), (180.0, 2), (270.0, 3), (-90.0, 3), (360.0, 0), (450.0, 1)])
def test_rotation_multiple_of_90_is_exact_index_map(theta, q):
    f = synth.random_frames(1, 16, seed=2).astype(np.float64)
    out = oracle.rotate(f, [theta])
    assert np.array_equal(out, _rot90_map(f, q))


@pytest.mark.parametrize("theta,q", [(90.0, 1), (-90.0, 3)])
def test_raw_three_shear_at_90_equals_index_map(theta, q):
    f = synth.random_frames(1, 16, seed=4).astype(np.float64)
    out = oracle.rotate(f, [theta], reduce90=False)
    assert np.abs(out - _rot90_map(f, q)).max() <= 1e-12


@pytest.mark.parametrize("theta", [11.3, -37.0, 44.9, 1.0])
def test_shear_matrix_identity(theta):
    t = math.radians(theta)
    Sx = np.array([[1.0, -math.tan(t / 2)], [0.0, 1.0]])
    Sy = np.array([[1.0, 0.0], [math.sin(t), 1.0]])
    R = np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]])
    assert np.abs(Sx @ Sy @ Sx - R).max() <= 1e-15


@pytest.mark.parametrize("theta", [11.3, -30.0, 44.0, 123.4, -161.0])
def test_rotated_elliptical_gaussian_is_analytic(theta):
    N = 64
    c = N / 2
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    sa, sb, phi0, x0, y0 = 3.0, 2.2, math.radians(20.0), 6.0, -4.0

    def g(rot_deg):
        r = math.radians(rot_deg)
        # centre and orientation of the content after a CCW rotation by rot_deg
        cx = c + x0 * math.cos(r) - y0 * math.sin(r)
        cy = c + x0 * math.sin(r) + y0 * math.cos(r)
        p = phi0 + r
        u = (xx - cx) * math.cos(p) + (yy - cy) * math.sin(p)
        v = -(xx - cx) * math.sin(p) + (yy - cy) * math.cos(p)
        return np.exp(-(u * u / (2 * sa * sa) + v * v / (2 * sb * sb)))

    out = oracle.rotate(g(0.0)[None], [theta])[0]
    assert np.abs(out - g(theta)).max() <= 1e-9
    assert oracle.last_max_imag() <= 1e-12


def test_rotation_round_trip_paper_case():
    th = GOLD["rotation_round_trip"]["theta_deg"]
    f = synth.random_frames(2, 64, seed=8, smooth=True, dtype=np.float64)
    back = oracle.rotate(oracle.rotate(f, [th, th]), [-th, -th])
    assert np.abs(back - f).max() <= 1e-9 * np.abs(f).max()


def test_rotation_composes_and_conserves_flux():
    f = synth.random_frames(1, 64, seed=12, smooth=True, dtype=np.float64)
    a = oracle.rotate(oracle.rotate(f, [17.0]), [21.0])
    b = oracle.rotate(f, [38.0])
    assert np.abs(a - b).max() <= 1e-8 * np.abs(f).max()
    assert abs(b.sum() - f.sum()) <= 1e-9 * np.abs(f).sum()


def test_rotation_moves_point_counter_clockwise():
    N = 64
    c = N // 2
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    f = np.exp(-((xx - (c + 10)) ** 2 + (yy - c) ** 2) / (2 * 2.0 ** 2))[None]
    out = oracle.rotate(f, [30.0])[0]
    i, j = np.unravel_index(np.argmax(out), out.shape)
    # (10, 0) rotated by +30 deg -> (8.66, 5.0): row c + 5, col c + 9 (nearest)
    assert (i, j) == (c + 5, c + 9)


# --------------------------------------------------------------------------
# Gate and medians (Sect. 3.3)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("r", [4.0, 8.0, 16.0, 100.0])
def test_alpha_min_is_chord_of_n_fwhm(r):
    fwhm, n = 4.0, 1.5
    a = oracle.alpha_min_deg(fwhm, n, r)
    # two points at radius r, alpha_min apart, are n * FWHM apart (chord)
    chord = 2.0 * r * math.sin(math.radians(a) / 2.0)
    if n * fwhm < 2.0 * r:
        assert abs(chord - n * fwhm) <= 1e-12 * n * fwhm
    else:
        assert a == 180.0


def test_gate_invariants():
    rng = np.random.default_rng(3)
    pa = np.sort(rng.uniform(-30, 30, 40))
    amin = 7.5
    masks = [oracle.gate_mask(pa, i, amin) for i in range(40)]
    for i in range(40):
        m = masks[i]
        assert not m[i]
        if m.any():
            # exactly the frames rotated by more than alpha_min, both sides
            d = np.abs(pa - pa[i])
            assert np.array_equal(m, d > amin)
            for k in np.nonzero(m)[0]:
                assert masks[k][i]  # symmetric
    # a larger alpha_min gives a subset
    for i in range(40):
        m2 = oracle.gate_mask(pa, i, amin * 2)
        if m2.any() and masks[i].any():
            assert not np.any(m2 & ~masks[i])


def test_gate_empty_set_falls_back_to_farthest_frames():
    pa = np.array([0.0, 1.0, 2.0, 3.0, 4.0])
    m = oracle.gate_mask(pa, 2, 10.0)     # nothing is 10 deg away
    assert m.tolist() == [True, False, False, False, True]   # tie: both ends
    m = oracle.gate_mask(pa, 1, 10.0)
    assert m.tolist() == [False, False, False, False, True]


@pytest.mark.parametrize("T", [1, 2, 3, 4, 7, 32, 33])
def test_collapse_median_f32_matches_numpy_bit_exact(T):
    rng = np.random.default_rng(T)
    c = (rng.standard_normal((T, 8, 8)) * 100).astype(np.float32)
    c[:, 0, 0] = 5.0  # ties
    ours = oracle.collapse_median(c)
    assert ours.dtype == np.float32
    assert np.array_equal(ours, np.median(c, axis=0).astype(np.float32))


def test_adi_subtract_small_alpha_min_is_median_of_others():
    # with fwhm -> 0 the gate keeps every frame with a different angle
    T, N = 9, 8
    rng = np.random.default_rng(4)
    c = rng.standard_normal((T, N, N)).astype(np.float32)
    pa = np.linspace(0, 40, T)
    edges = [0.5, 100.0]          # every pixel but the centre one (rho = 0)
    res = oracle.adi_subtract(c, pa, 1e-9, 1.0, edges)
    for t in range(T):
        others = np.delete(c, t, axis=0)
        expect = (c[t] - np.median(others, axis=0)).astype(np.float32)
        expect[N // 2, N // 2] = 0.0
        assert np.array_equal(res[t], expect)


def test_adi_subtract_masks_pixels_outside_annuli_and_uses_farthest_when_empty():
    T, N = 5, 16
    rng = np.random.default_rng(6)
    c = rng.standard_normal((T, N, N))
    pa = np.array([0.0, 1.0, 2.0, 3.0, 4.0])
    edges = [2.0, 5.0]
    res = oracle.adi_subtract(c, pa, 4.0, 1.5, edges)   # alpha_min > 4 deg -> fallback
    for i in range(N):
        for j in range(N):
            rho2 = (i - N // 2) ** 2 + (j - N // 2) ** 2
            if not (4.0 <= rho2 < 25.0):
                assert np.all(res[:, i, j] == 0.0)
            else:
                assert res[0, i, j] == c[0, i, j] - c[4, i, j]
                assert res[2, i, j] == c[2, i, j] - 0.5 * (c[0, i, j] + c[4, i, j])


# --------------------------------------------------------------------------
# Whole reduction
# --------------------------------------------------------------------------

def test_reduce_recovers_companion_at_injected_position():
    # noise-free small workload: the companion must come back at its
    # injected (r, PA0) once the frames are recentred, PSF-subtracted and
    # derotated by -parang (centroid within 0.5 px, as the registration
    # accuracy the paper quotes in Sect. 3.1)
    d = synth.make_cube(32, 128, 0, parang=np.linspace(0.0, 40.0, 32), peak=1e4, noise=False)
    out = oracle.reduce(d.cube, d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges)
    c = 128 // 2
    for (r, pa0, con) in d.companions:
        x = c + r * math.cos(math.radians(pa0))
        y = c + r * math.sin(math.radians(pa0))
        i0, j0 = int(round(y)), int(round(x))
        win = np.clip(out[i0 - 2:i0 + 3, j0 - 2:j0 + 3], 0, None)
        ii, jj = np.mgrid[i0 - 2:i0 + 3, j0 - 2:j0 + 3]
        assert abs((win * ii).sum() / win.sum() - y) <= 0.5
        assert abs((win * jj).sum() / win.sum() - x) <= 0.5
        assert out[i0, j0] > 0.3 * 1e4 * con


def test_reduce_of_static_cube_is_zero():
    T, N = 6, 16
    f = synth.random_frames(1, N, seed=1).astype(np.float64)
    c = np.repeat(f, T, axis=0)
    out = oracle.reduce(c, np.zeros(T), np.zeros(T), np.linspace(0, 50, T), 4.0, 1.0, [0.0, 12.0])
    assert np.abs(out).max() <= 1e-12


# --------------------------------------------------------------------------
# Time gate (maximum time separation t_max of the reference frames, Sect. 3.3)
# --------------------------------------------------------------------------

def _cube_1px(T, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((T, 4, 4))


def test_time_gate_infinite_t_max_equals_no_time_gate():
    T = 23
    c = _cube_1px(T, 3)
    pa = np.linspace(-30.0, 50.0, T)
    times = np.arange(T) * 37.0
    a = oracle.adi_subtract(c, pa, 1.0, 1.0, [0.0, 3.0])
    b = oracle.adi_subtract(c, pa, 1.0, 1.0, [0.0, 3.0], times=times, t_max=np.inf)
    assert np.array_equal(a, b)


def test_time_gate_nearest_neighbours_closed_form():
    # times = frame index, t_max = 1.5 and a vanishing alpha_min: the
    # reference set of frame i is {i - 1, i + 1} (strict ">" removes frame i
    # itself), so the residual is f_i minus the mean of its neighbours, and
    # at the ends f_0 - f_1, f_{T-1} - f_{T-2}
    T = 17
    c = _cube_1px(T, 4)
    pa = np.arange(T) * 2.0
    res = oracle.adi_subtract(c, pa, 1e-9, 1e-9, [0.0, 3.0], times=np.arange(T, dtype=float), t_max=1.5)
    ref = np.empty_like(c)
    ref[1:-1] = c[1:-1] - 0.5 * (c[:-2] + c[2:])
    ref[0] = c[0] - c[1]
    ref[-1] = c[-1] - c[-2]
    assert np.abs(res - ref).max() <= 1e-15


def test_time_gate_empty_set_falls_back_to_farthest_frames_in_the_window():
    # alpha_min = 180 deg (argument clamped): no frame qualifies, so the
    # reference set is the frame(s) farthest in angle within |t_k - t_i| < 2.5,
    # i.e. frames i - 2 and i + 2 (exact distances on an integer angle grid)
    T = 15
    c = _cube_1px(T, 5)
    pa = np.arange(T) * 1.0
    res = oracle.adi_subtract(c, pa, 1e6, 1.0, [0.0, 3.0], times=np.arange(T, dtype=float), t_max=2.5)
    ref = np.empty_like(c)
    for i in range(T):
        nb = [k for k in (i - 2, i + 2) if 0 <= k < T]
        if len(nb) == 1:                     # ends: window i..i+2 or i-2..i
            ref[i] = c[i] - c[nb[0]]
        else:
            ref[i] = c[i] - 0.5 * (c[nb[0]] + c[nb[1]])
    assert np.abs(res - ref).max() <= 1e-15


def test_time_gate_shrinks_the_reference_set():
    T = 40
    pa = np.sort(np.random.default_rng(6).uniform(-60, 60, T))
    times = np.cumsum(np.random.default_rng(7).uniform(0.5, 2.0, T))
    amin = 5.0
    for i in range(T):
        full = oracle.gate_mask(pa, i, amin)
        for tm in (3.0, 10.0, 1e9):
            sub = oracle.gate_mask(pa, i, amin, times=times, t_max=tm)
            inside = np.abs(times - times[i]) < tm
            if (full & inside).any():
                assert np.array_equal(sub, full & inside)
            else:   # fallback: farthest in angle among the frames in time
                d = np.where(inside, np.abs(pa - pa[i]), -1.0)
                assert np.array_equal(sub, d == d.max())


# --------------------------------------------------------------------------
# Image-quality pre-processing (Sect. 3.2): master sky, bad pixels
# --------------------------------------------------------------------------

def test_sky_median_equals_numpy_nanmedian_with_mask():
    rng = np.random.default_rng(11)
    T, N = 9, 20
    c = rng.normal(100.0, 5.0, (T, N, N)).astype(np.float32)
    c[2, 3, 4] = np.nan
    c[:, 7, 7] = np.nan                                  # no value left: NaN
    mx, my, r = rng.uniform(5, 15, T), rng.uniform(5, 15, T), 3.0
    ref = c.copy()
    yy, xx = np.mgrid[0:N, 0:N]
    for t in range(T):
        ref[t][(xx - mx[t]) ** 2 + (yy - my[t]) ** 2 < r * r] = np.nan
    with np.errstate(all="ignore"):
        import warnings
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")
            want = np.nanmedian(ref, axis=0).astype(np.float32)
    got = oracle.sky_median(c, mx, my, r)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.array_equal(got[ok], want[ok])


def test_sky_median_of_identical_frames_is_the_frame():
    f = np.random.default_rng(12).normal(0, 1, (1, 16, 16)).astype(np.float32)
    assert np.array_equal(oracle.sky_median(np.repeat(f, 6, axis=0)), f[0])


def test_sky_subtract_uses_the_closest_sky_in_time():
    rng = np.random.default_rng(13)
    T, N = 7, 8
    c = rng.normal(0, 1, (T, N, N)).astype(np.float32)
    skies = rng.normal(0, 1, (3, N, N)).astype(np.float32)
    ft = np.array([0.0, 1.0, 2.0, 3.0, 4.0, 5.0, 6.0])
    st = np.array([0.5, 3.0, 5.5])
    # frame 0 -> sky 0 (0.5), 1 -> tie 0.5 vs 2.0: sky 0, 2 -> sky 1, 3 -> 1, 4 -> 1 (1.0 vs 1.5), 5 -> 2, 6 -> 2
    j = [0, 0, 1, 1, 1, 2, 2]
    want = np.stack([c[t] - skies[j[t]] for t in range(T)])
    assert np.array_equal(oracle.sky_subtract(c, skies, ft, st), want)


def test_bad_pixel_map_flags_planted_outliers():
    rng = np.random.default_rng(14)
    N = 32
    ref = rng.normal(10.0, 1.0, (N, N)).astype(np.float32)
    hot = [(3, 4), (20, 7), (31, 31)]
    for (i, j) in hot:
        ref[i, j] = 500.0
    ref[10, 10] = -400.0
    m = oracle.bad_pixel_map(ref, 5.0)
    med = np.median(ref)
    sig = ref.astype(np.float64).std()
    assert np.array_equal(m, np.abs(ref.astype(np.float64) - float(med)) > 5.0 * sig)
    assert m.sum() == 4 and m[10, 10] and all(m[i, j] for (i, j) in hot)


def test_bad_pixel_fix_single_pixel_and_clump():
    N = 9
    f = (np.arange(N * N, dtype=np.float32).reshape(1, N, N) * 1.5) ** 1.1
    bad = np.zeros((N, N), bool)
    bad[1, 1] = True                                      # isolated: median of its 8 neighbours
    bad[4:7, 4:7] = True                                  # 3 x 3 clump: border first, centre next
    got, st = oracle.bad_pixel_fix(f, bad)
    assert st == 0
    g = f[0].copy()
    nb = [g[i, j] for i in range(0, 3) for j in range(0, 3) if (i, j) != (1, 1)]
    assert got[0, 1, 1] == np.median(np.array(nb, np.float32))
    # the clump, pass by pass, written out here independently
    h = g.copy()
    h[1, 1] = np.nan
    h[4:7, 4:7] = np.nan
    while np.isnan(h).any():
        prev = h.copy()
        for i in range(N):
            for j in range(N):
                if not np.isnan(prev[i, j]):
                    continue
                vals = [prev[a, b] for a in range(max(0, i - 1), min(N, i + 2))
                        for b in range(max(0, j - 1), min(N, j + 2)) if (a, b) != (i, j) and not np.isnan(prev[a, b])]
                if vals:
                    h[i, j] = np.median(np.array(vals, np.float32))
    assert np.array_equal(got[0], h)


def test_bad_pixel_fix_constant_frame_and_hopeless_frame():
    f = np.full((2, 6, 6), 3.25, np.float32)
    f[0, 0, 0] = np.inf
    f[0, 2:5, 2:5] = np.nan
    f[1] = np.nan
    got, st = oracle.bad_pixel_fix(f)
    assert np.array_equal(got[0], np.full((6, 6), 3.25, np.float32))
    assert st == 1                                        # frame 1 has no finite pixel


# --------------------------------------------------------------------------
# Registration (Sect. 3.1): centroid patch search, Moffat fit
# --------------------------------------------------------------------------

def _moffat_image(N, I0, x0, y0, al, be, bg):
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    u = 1.0 + ((xx - x0) ** 2 + (yy - y0) ** 2) / al ** 2
    return (I0 * (be - 1.0) / (math.pi * al * al) * u ** (-be) + bg).astype(np.float32)


def test_moffat_fit_recovers_noise_free_parameters():
    truth = (5e4, 31.3, 29.7, 3.1, 2.7, 12.0)
    img = _moffat_image(64, *truth)
    ok, cx, cy, sz = oracle.centroid(img, 12.0 + 0.05 * img.max(), 16, 4, 400)
    assert ok
    p, it = oracle.moffat_fit(img, cx, cy, max(1.0, math.sqrt(sz / math.pi)), 12)
    assert abs(p[1] - 31.3) < 1e-5 and abs(p[2] - 29.7) < 1e-5
    assert abs(p[3] / 3.1 - 1) < 1e-5 and abs(p[4] / 2.7 - 1) < 1e-5 and abs(p[0] / 5e4 - 1) < 1e-5
    assert abs(p[5] - 12.0) < 1e-3


def test_moffat_fwhm_is_the_width_at_half_maximum():
    # independent route: bisection for the radius where the profile halves
    for al, be in ((3.1, 2.7), (1.2, 1.5), (6.0, 8.0)):
        lo, hi = 0.0, 100.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if (1.0 + mid * mid / (al * al)) ** (-be) > 0.5:
                lo = mid
            else:
                hi = mid
        assert abs(oracle.moffat_fwhm(al, be) - 2.0 * lo) < 1e-12


def test_moffat_fit_follows_integer_translations():
    a = _moffat_image(64, 3e4, 30.4, 33.2, 2.5, 3.0, 5.0)
    b = np.roll(np.roll(a, 3, axis=1), -2, axis=0)        # content moves by (+3, -2); far from the edges
    pa, _ = oracle.moffat_fit(a, 30.0, 33.0, 2.0, 10)
    pb, _ = oracle.moffat_fit(b, 33.0, 31.0, 2.0, 10)
    assert abs(pb[1] - pa[1] - 3.0) < 1e-6 and abs(pb[2] - pa[2] + 2.0) < 1e-6


def test_centroid_of_a_symmetric_patch_and_its_flags():
    f = np.zeros((32, 32), np.float32)
    f[10, 20] = 9.0
    f[9, 20] = f[11, 20] = f[10, 19] = f[10, 21] = 4.0        # plus-shaped patch centred on (x, y) = (20, 10)
    ok, cx, cy, sz = oracle.centroid(f, 1.0, 5, 3, 10)
    assert ok and cx == 20.0 and cy == 10.0 and sz == 5
    assert not oracle.centroid(f, 10.0, 5, 3, 10)[0]          # seed below the threshold
    assert not oracle.centroid(f, 1.0, 5, 6, 10)[0]           # patch too small
    assert not oracle.centroid(f, 1.0, 5, 1, 4)[0]            # patch too large
    assert not oracle.centroid(f, 1.0, 0, 1, 10)[0]           # patch reaches the box edge


# --------------------------------------------------------------------------
# Photometric-accuracy and binning experiments (Sect. 4.2, 4.3)
# --------------------------------------------------------------------------

def test_bin_median_is_numpy_median_per_group():
    """Groups of B consecutive frames with a ragged last group; B = 1 is the
    identity and B >= T the median collapse."""
    rng = np.random.default_rng(60)
    c = rng.standard_normal((23, 12, 12)).astype(np.float32)
    c[3, 2, 2] = c[4, 2, 2]                                        # a tie
    for B in (1, 2, 5, 10, 23, 40):
        got = oracle.bin_median(c, B)
        want = np.stack([np.median(c[g:g + B], axis=0) for g in range(0, 23, B)]).astype(np.float32)
        assert got.shape == (-(-23 // B), 12, 12)
        assert np.array_equal(got, want), B
    assert np.array_equal(oracle.bin_median(c, 1), c)
    assert np.array_equal(oracle.bin_median(c, 23)[0], oracle.collapse_median(c))


def test_inject_total_flux_peak_and_position():
    """The Moffat companion carries its total flux (the tail outside a
    square window of half-size H is below (1 + H^2/alpha^2)^(1-beta)), its
    peak is flux (beta - 1) / (pi alpha^2) at an integer position, and its
    centre of light is the requested position at radius r, angle pa0 +
    parang counter-clockwise from +x."""
    N, H = 256, 120
    al, be, F = 3.0, 2.5, 5000.0
    z = np.zeros((1, N, N), np.float32)
    a = oracle.inject(z, [0.0], [128.0], [128.0], [0.0], [0.0], [F], [al], [be], H)
    tail = (1.0 + H * H / (al * al)) ** (1.0 - be)
    assert abs(float(a.astype(np.float64).sum()) - F) <= F * (tail + 1e-5)
    assert a[0, 128, 128] == np.float32(F * (be - 1.0) / (math.pi * al * al))
    # 30 deg of parallactic angle + 60 deg of position angle = straight up (+y, higher rows)
    b = oracle.inject(z, [30.0], [128.0], [128.0], [40.0], [60.0], [F], [al], [be], 60)
    assert np.unravel_index(np.argmax(b[0]), (N, N)) == (168, 128)
    # a sub-pixel position: the centre of light follows it
    th = math.radians(17.0 + 25.0)
    xp, yp = 128.0 + 33.3 * math.cos(th), 128.0 + 33.3 * math.sin(th)
    c = oracle.inject(z, [17.0], [128.0], [128.0], [33.3], [25.0], [F], [al], [be], 100).astype(np.float64)[0]
    yy, xx = np.mgrid[0:N, 0:N]
    assert abs((c * xx).sum() / c.sum() - xp) < 2e-3 and abs((c * yy).sum() / c.sum() - yp) < 2e-3


def test_inject_adds_in_fp64_then_rounds_and_clips_at_the_edges():
    rng = np.random.default_rng(61)
    base = rng.normal(100.0, 5.0, (3, 64, 64)).astype(np.float32)
    kw = dict(parang=[0.0, 10.0, 20.0], xc=[32.0, 31.5, 2.0], yc=[32.0, 30.0, 61.0], r=[5.0, 20.0],
              pa0=[0.0, 200.0], flux=[800.0, 50.0], alpha=[2.0, 2.5, 3.0], beta=[2.0, 3.0, 4.0], half=12)
    only = oracle.inject(np.zeros_like(base), **kw).astype(np.float64)
    both = oracle.inject(base, **kw).astype(np.float64)
    # one rounding of the FP64 sum: within an ulp of base + (the FP32-rounded injection)
    ulp = np.spacing(np.abs(base + only).astype(np.float32)).astype(np.float64)
    assert (np.abs(both - (base.astype(np.float64) + only)) <= ulp + np.spacing(only.astype(np.float32))).all()
    assert np.array_equal(both[only == 0.0], base.astype(np.float64)[only == 0.0])
    # frame 2's star sits 2 px from the left edge and 3 from the top: windows clip, nothing wraps
    assert only[2, :, 40:].sum() == 0.0 and np.isfinite(only).all()


def test_aperture_counts_lattice_points_and_sums():
    """A constant image gives the number of pixel centres in the disc (brute
    force); a ramp symmetric about an integer centre gives count x value."""
    N = 64
    ones = np.ones((N, N), np.float32)
    yy, xx = np.mgrid[0:N, 0:N]
    for (x, y, r) in [(32.0, 32.0, 5.0), (10.3, 40.7, 7.5), (0.0, 0.0, 3.0), (31.5, 31.5, 0.0)]:
        want = float(((xx - x) ** 2 + (yy - y) ** 2 <= r * r).sum())
        assert oracle.aperture(ones, [x], [y], r)[0] == want
    ramp = (xx + 2 * yy).astype(np.float32)
    cnt = float(((xx - 20) ** 2 + (yy - 30) ** 2 <= 36).sum())
    assert oracle.aperture(ramp, [20.0], [30.0], 6.0)[0] == cnt * (20 + 60)


def test_centroid_patch_is_the_8_connected_component():
    """The centroid's patch against scipy.ndimage.label (8-connectivity) on
    the box around the brightest pixel: same size, same flux-weighted
    centre, and the box-edge / size rules applied to that component."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(62)
    checked = 0
    for trial in range(40):
        N = 48
        f = rng.normal(0.0, 1.0, (N, N)).astype(np.float32)
        # a few blobs of random shape, one clearly brightest
        for _ in range(4):
            y, x = rng.integers(4, N - 4, 2)
            f[y - 2:y + 3, x - 2:x + 3] += rng.uniform(2.0, 6.0) * (rng.random((5, 5)) > 0.3)
        f[rng.integers(8, N - 8), rng.integers(8, N - 8)] += 20.0
        thresh, R = 1.5, int(rng.integers(3, 12))
        ok, cx, cy, sz = oracle.centroid(f, thresh, R, 1, 10 ** 6)
        r0, c0 = np.unravel_index(int(np.argmax(f)), f.shape)
        rlo, rhi, clo, chi = max(r0 - R, 0), min(r0 + R, N - 1), max(c0 - R, 0), min(c0 + R, N - 1)
        box = f[rlo:rhi + 1, clo:chi + 1].astype(np.float64)
        lab, _ = ndimage.label(box > thresh, structure=np.ones((3, 3), int))
        comp = lab == lab[r0 - rlo, c0 - clo]
        assert sz == int(comp.sum())
        H, W = comp.shape
        touches = ((comp[0].any() and rlo > 0) or (comp[-1].any() and rhi < N - 1) or
                   (comp[:, 0].any() and clo > 0) or (comp[:, -1].any() and chi < N - 1))
        assert ok == (not touches)
        if ok:
            yy, xx = np.mgrid[rlo:rhi + 1, clo:chi + 1]
            w = box * comp
            assert abs(cx - (w * xx).sum() / w.sum()) < 1e-9 and abs(cy - (w * yy).sum() / w.sum()) < 1e-9
            checked += 1
    assert checked >= 10


def test_moffat_fit_is_a_stationary_point_on_noisy_data():
    """On a noisy star the fitted parameters zero the gradient of the
    squared error, computed here by central differences of a numpy model
    (independent of the oracle's analytic Jacobian): a wrong derivative
    would stop the iteration at a point where this gradient is not zero."""
    rng = np.random.default_rng(63)
    N, w = 64, 10
    img = _moffat_image(N, 4e4, 31.3, 30.6, 3.2, 2.8, 20.0)
    img = (img + rng.normal(0.0, 5.0, img.shape)).astype(np.float32)
    ok, cx, cy, sz = oracle.centroid(img, 200.0, 16, 4, 400)
    assert ok
    p, it = oracle.moffat_fit(img, cx, cy, max(1.0, math.sqrt(sz / math.pi)), w)
    assert it < 200
    rc, cc = int(math.floor(cy + 0.5)), int(math.floor(cx + 0.5))
    yy, xx = np.mgrid[rc - w:rc + w + 1, cc - w:cc + w + 1].astype(np.float64)
    v = img[rc - w:rc + w + 1, cc - w:cc + w + 1].astype(np.float64)

    def cost(q):
        I0, x0, y0, al, be, bg = q
        m = I0 * (be - 1) / (math.pi * al * al) * (1 + ((xx - x0) ** 2 + (yy - y0) ** 2) / (al * al)) ** (-be) + bg
        return float(((m - v) ** 2).sum())

    c0 = cost(p)
    for k in range(6):
        h = 1e-5 * max(1.0, abs(p[k]))
        qp, qm = p.copy(), p.copy()
        qp[k] += h
        qm[k] -= h
        g = (cost(qp) - cost(qm)) / (2 * h)
        curv = (cost(qp) - 2 * c0 + cost(qm)) / (h * h)
        # the gradient is zero to the step the curvature allows: |g| / curv << h-scale
        assert abs(g) <= 1e-6 * c0 / max(1.0, abs(p[k])) + 1e-3 * abs(curv) * h, (k, g, curv)
    assert abs(p[1] - 31.3) < 0.1 and abs(p[2] - 30.6) < 0.1


# --------------------------------------------------------------------------
# Exact boundaries of the strict inequalities and tie rules (readings R19,
# R23, R24, R26): values placed exactly on the boundary, all exactly
# representable, so "<" against "<=" (or ">" against ">=") decides.
# --------------------------------------------------------------------------

def test_time_gate_boundary_is_strict():
    """|t_k - t_i| < t_max: a frame exactly t_max away is outside the set."""
    T = 9
    pa = np.linspace(0.0, 80.0, T)                  # every other frame passes the angle gate
    times = np.arange(T, dtype=np.float64)          # integer hours: differences exact
    m = oracle.gate_mask(pa, 4, 0.5, times=times, t_max=2.0)
    assert not m[2] and not m[6]                     # exactly 2 h away: excluded
    assert m[3] and m[5] and not m[4]                # 1 h away: included; the frame itself: not
    assert m.sum() == 2


def test_sky_subtract_tie_takes_the_earlier_sky():
    """A frame exactly halfway between two master skies takes the first."""
    cube = np.zeros((1, 8, 8), np.float32)
    skies = np.stack([np.full((8, 8), 1.0, np.float32), np.full((8, 8), 2.0, np.float32)])
    out = oracle.sky_subtract(cube, skies, [1.5], [1.0, 2.0])
    assert np.all(out == -1.0)
    out = oracle.sky_subtract(cube, skies[::-1].copy(), [1.5], [2.0, 1.0])   # the first listed sky wins
    assert np.all(out == -2.0)


def test_bad_pixel_map_boundary_is_strict():
    """|v - median| > C sigma: values of +-1 have median 0 and sigma 1
    exactly, so at C = 1 no pixel is flagged and at C slightly below 1 all."""
    ref = np.where((np.arange(16).reshape(4, 4) % 2) == 0, -1.0, 1.0).astype(np.float32)
    assert not oracle.bad_pixel_map(ref, 1.0).any()
    assert oracle.bad_pixel_map(ref, 0.999).all()


def test_centroid_threshold_is_strict():
    """Pixels equal to the threshold are below it: a seed equal to it is not
    found, and a neighbour equal to it stays out of the patch."""
    f = np.zeros((32, 32), np.float32)
    f[10, 10] = 8.0
    f[10, 11] = 4.0
    f[11, 10] = 5.0
    ok, cx, cy, sz = oracle.centroid(f, 4.0, 5, 1, 10)
    assert ok and sz == 2 and cx == 10.0 and cy == (10 * 8.0 + 11 * 5.0) / 13.0
    assert not oracle.centroid(f, 8.0, 5, 1, 10)[0]


def test_gate_boundary_is_strict():
    """|alpha_k - alpha_i| > alpha_min: a frame exactly alpha_min away (the
    differences below are exact) is outside the reference set (R11)."""
    amin = oracle.alpha_min_deg(4.0, 1.5, 20.0)
    pa = np.array([0.0, amin, 2.0 * amin])
    assert list(oracle.gate_mask(pa, 0, amin)) == [False, False, True]
    assert list(oracle.gate_mask(pa, 2, amin)) == [True, False, False]


def test_sky_median_mask_excludes_only_the_inside():
    """The star mask drops values strictly inside mask_r (R22): a pixel
    exactly mask_r from the centre stays in the master sky's median."""
    T, N = 3, 16
    c = np.zeros((T, N, N), np.float32)
    c[:, 5, 8] = [10.0, 20.0, 30.0]                  # pixel (x=8, y=5)
    c[:, 5, 6] = [10.0, 20.0, 30.0]                  # pixel (x=6, y=5)
    mx, my = np.array([5.0, 100.0, 100.0]), np.array([5.0, 100.0, 100.0])
    sky = oracle.sky_median(c, mx, my, 3.0)
    assert sky[5, 8] == 20.0                         # distance exactly 3: kept in every frame
    assert sky[5, 6] == 25.0                         # distance 1 in frame 0: masked there
