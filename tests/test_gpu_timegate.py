"""Median PSF subtraction with the paper's maximum time separation of the
reference frames (graphic_adi_subtract_ex, graphic_reduce_ex): bit-exact
against the FP32 oracle on identical inputs (medians are selections), equal
to the plain call when t_max is infinite, the empty-set fallback within the
time window, and the argument checks."""
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


@pytest.fixture(scope="module")
def cube():
    T, n = 48, 64
    d = synth.make_cube(T, n, seed=31, parang=synth.altaz_parang(T), edges=synth.default_edges(n))
    return d


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("t_max", [0.5, 1.5, 4.5, 12.0, 100.0])
def test_time_gate_bit_exact_against_oracle(g, cube, t_max):
    """times = frame index (monotone with the alt-az angles); t_max from one
    frame (every set empty: the window fallback) to the whole sequence."""
    d = cube
    T = d.cube.shape[0]
    times = np.arange(T, dtype=np.float64)
    got = g.graphic_adi_subtract(_dev(d.cube), d.parang, d.fwhm, d.n_fwhm, d.edges, times=times,
                                 t_max=t_max).cpu().numpy()
    ref = oracle.adi_subtract(d.cube, d.parang, d.fwhm, d.n_fwhm, d.edges, times=times, t_max=t_max)
    assert np.array_equal(got, ref)


def test_time_gate_descending_times_and_uneven_steps(g, cube):
    d = cube
    T = d.cube.shape[0]
    times = -np.cumsum(np.random.default_rng(3).uniform(0.2, 3.0, T))   # decreasing along the angles
    got = g.graphic_adi_subtract(_dev(d.cube), d.parang, d.fwhm, d.n_fwhm, d.edges, times=times,
                                 t_max=9.0).cpu().numpy()
    ref = oracle.adi_subtract(d.cube, d.parang, d.fwhm, d.n_fwhm, d.edges, times=times, t_max=9.0)
    assert np.array_equal(got, ref)


def test_infinite_t_max_equals_plain_call(g, cube):
    """The plain call runs the band path, the time-gated one the general
    path: the same medians, so the same bits."""
    d = cube
    x = _dev(d.cube)
    a = g.graphic_adi_subtract(x, d.parang, d.fwhm, d.n_fwhm, d.edges).cpu().numpy()
    b = g.graphic_adi_subtract(x, d.parang, d.fwhm, d.n_fwhm, d.edges, times=np.arange(d.cube.shape[0]),
                               t_max=np.inf).cpu().numpy()
    assert np.array_equal(a, b)


def test_time_gated_reduce_matches_fp64_oracle(g, cube):
    d = cube
    times = np.arange(d.cube.shape[0], dtype=np.float64)
    out = g.graphic_reduce(_dev(d.cube), d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges, times=times,
                           t_max=6.0).cpu().numpy()
    ref = oracle.reduce(d.cube.astype(np.float64), d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges, times=times,
                        t_max=6.0)
    assert np.abs(out - ref).max() <= 1e-5 * np.abs(d.cube).max()


def test_long_sequence_sampled_pixels(g):
    """600 frames of 128 x 128 (several 32-query chunks per lane), sampled
    pixels against the oracle."""
    T, n = 600, 128
    pa = synth.altaz_parang(T)
    x = synth.random_frames(T, n, seed=8)
    edges = synth.default_edges(n)
    times = np.linspace(0.0, 3.0, T)
    got = g.graphic_adi_subtract(_dev(x), pa, 4.0, 1.5, edges, times=times, t_max=0.35).cpu().numpy()
    pix = np.random.default_rng(9).choice(n * n, 300, replace=False)
    ref = oracle.adi_subtract(x, pa, 4.0, 1.5, edges, pixels=pix, times=times, t_max=0.35)
    assert np.array_equal(got.reshape(T, -1)[:, pix].T, ref)


def test_time_gate_argument_checks(g, cube):
    d = cube
    T = d.cube.shape[0]
    x = _dev(d.cube)
    bumpy = np.arange(T, dtype=np.float64)
    bumpy[T // 2] = -5.0                       # not monotone along the angles
    with pytest.raises(g.GraphicError, match="UNSUPPORTED"):
        g.graphic_adi_subtract(x, d.parang, d.fwhm, d.n_fwhm, d.edges, times=bumpy, t_max=3.0)
    with pytest.raises(g.GraphicError, match="INVALID_ARG"):
        g.graphic_adi_subtract(x, d.parang, d.fwhm, d.n_fwhm, d.edges, times=np.arange(T), t_max=0.0)
