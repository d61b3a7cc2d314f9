"""Seeded synthetic ADI cubes shaped like the paper's workloads.

Holds none of the reduction's arithmetic (no Fourier shift, shear, gate or
median): frames are built from analytic Gaussians and from pupil-plane
optics (|FFT(pupil * exp(i phi))|^2), then noise is added.  Both the CUDA
path and the oracle take their inputs from here.

Recipe (stated once, used by every workload):

* Star: Gaussian core, FWHM ``fwhm`` px, peak ``peak`` e-, centred on pixel
  (N/2, N/2) plus a per-frame offset delta ~ U(-off, off) px per axis.  The
  recentring shift handed to the reduction is ``dx, dy = -delta``.
* Quasi-static speckles: |FFT_{2N}(pupil * (exp(i phi_t) - <exp(i phi_t)>))|^2
  with a pupil disc of diameter N/2 px in a 2N grid (lambda/D = 4 px) and
  phi_t a Gaussian random phase screen with an f^(-11/3) power spectrum,
  0.3 rad rms.  phi_t evolves as AR(1), phi_t = rho phi_{t-1} +
  sqrt(1 - rho^2) eps_t; screens are drawn at anchor frames every
  ``anchor`` frames (rho^anchor per anchor step) and the halo intensity is
  interpolated linearly in between.  The halo is scaled so that its
  time-averaged maximum is ``halo_frac`` of the core peak.  The halo is
  not jittered with the star offset.
* Parallactic angles: linear in time (small workloads) or from the alt-az
  formula alpha = atan2(cos(lat) sin h, cos(dec) sin(lat) - sin(dec)
  cos(lat) cos h) with h linear in time.
* Fake companions: the core Gaussian times a contrast, at radius r and
  position angle PA0 + alpha_t on the detector (x = col - N/2, y = row -
  N/2, angle counter-clockwise from +x), plus the star offset.
* Noise: Poisson(image + sky) - sky + N(0, read^2); for cubes above ``4e7``
  pixels the Poisson draw is replaced by its Gaussian limit (sky = 50 e-
  keeps every mean >= 50).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class ADICube:
    cube: np.ndarray          # float32 [T][N][N]
    parang: np.ndarray        # float64 [T], degrees
    dx: np.ndarray            # float64 [T], recentring shift (content moves by +dx)
    dy: np.ndarray            # float64 [T]
    fwhm: float
    n_fwhm: float
    edges: np.ndarray         # float64 annulus edges, px
    peak: float
    companions: list = field(default_factory=list)   # (r px, PA0 deg, contrast)
    name: str = ""


def default_edges(N: int) -> np.ndarray:
    """Annulus edges 4, 8, 16, ... N/2 px plus one edge past the frame corner."""
    e = [4.0]
    while e[-1] * 2 <= N / 2:
        e.append(e[-1] * 2)
    e.append(float(math.ceil(N * math.sqrt(2.0) / 2.0) + 1))
    return np.array(e, np.float64)


def altaz_parang(T: int, dec_deg: float = -30.0, lat_deg: float = -24.6, h0_h: float = -1.5,
                 h1_h: float = 1.5) -> np.ndarray:
    """Parallactic angles (deg) for hour angles linear in [h0, h1] hours."""
    h = np.radians(np.linspace(h0_h, h1_h, T) * 15.0)
    d, p = math.radians(dec_deg), math.radians(lat_deg)
    return np.degrees(np.arctan2(math.cos(p) * np.sin(h), math.cos(d) * math.sin(p) - math.sin(d) * math.cos(p) * np.cos(h)))


def _screen(rng, G: int, rms: float, pupil: np.ndarray) -> np.ndarray:
    fx = np.fft.fftfreq(G)
    f = np.hypot(fx[None, :], fx[:, None])
    f[0, 0] = np.inf
    amp = f ** (-11.0 / 6.0)
    w = rng.standard_normal((G, G)) + 1j * rng.standard_normal((G, G))
    phi = np.real(np.fft.ifft2(w * amp))
    phi -= phi[pupil].mean()
    phi *= rms / phi[pupil].std()
    return phi


def _gauss_add(frame: np.ndarray, x0: float, y0: float, sigma: float, amp: float, half: int):
    """Add amp * exp(-r^2 / 2 sigma^2) centred at (x0, y0) (pixel coords) on a window."""
    N = frame.shape[0]
    ci, cj = int(round(y0)), int(round(x0))
    i0, i1 = max(0, ci - half), min(N, ci + half + 1)
    j0, j1 = max(0, cj - half), min(N, cj + half + 1)
    if i0 >= i1 or j0 >= j1:
        return
    yy = np.arange(i0, i1, dtype=np.float64)[:, None] - y0
    xx = np.arange(j0, j1, dtype=np.float64)[None, :] - x0
    frame[i0:i1, j0:j1] += (amp * np.exp(-(xx * xx + yy * yy) / (2.0 * sigma * sigma))).astype(frame.dtype)


def make_cube(T: int, N: int, seed: int, *, parang=None, fwhm: float = 4.0, n_fwhm: float = 1.5,
              peak: float = 1e4, halo_frac: float = 1e-2, rho: float = 1.0, anchor: int = 25,
              companions=None, off: float = 0.5, sky: float = 50.0, read: float = 5.0,
              edges=None, noise: bool = True, name: str = "") -> ADICube:
    rng = np.random.default_rng(seed)
    if parang is None:
        parang = np.linspace(0.0, 40.0, T)
    parang = np.asarray(parang, np.float64)
    G = 2 * N
    yy, xx = np.mgrid[0:G, 0:G]
    pupil = np.hypot(xx - G / 2 + 0.5, yy - G / 2 + 0.5) < (N / 4)

    # speckle halo at anchor frames (AR(1) screens), centred crop N x N
    n_anchor = 1 if rho >= 1.0 else max(2, (T + anchor - 1) // anchor + 1)
    step = anchor if n_anchor > 1 else max(T, 1)
    halos = []
    phi = _screen(rng, G, 0.3, pupil)
    for a in range(n_anchor):
        if a > 0:
            r = rho ** step
            phi = r * phi + math.sqrt(max(0.0, 1.0 - r * r)) * _screen(rng, G, 0.3, pupil)
        e = np.where(pupil, np.exp(1j * phi), 0)
        e[pupil] -= e[pupil].mean()
        h = np.abs(np.fft.fftshift(np.fft.fft2(e))) ** 2
        halos.append(h[N // 2:N // 2 + N, N // 2:N // 2 + N].astype(np.float32))
    hmax = float(np.mean([h.max() for h in halos]))
    scale = halo_frac * peak / hmax
    halos = [h * np.float32(scale) for h in halos]

    if companions is None:
        companions = [(20.0, float(rng.uniform(0, 360)), 1e-3), (40.0, float(rng.uniform(0, 360)), 1e-3)]
    sigma = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    delta = rng.uniform(-off, off, size=(T, 2))
    c = N / 2.0
    half = int(math.ceil(5 * sigma)) + 2
    cube = np.empty((T, N, N), np.float32)
    for t in range(T):
        if n_anchor > 1:
            u = t / step
            a0 = min(int(u), n_anchor - 2)
            w = u - a0
            fr = (1.0 - w) * halos[a0] + w * halos[a0 + 1]
        else:
            fr = halos[0].copy()
        x0, y0 = c + delta[t, 0], c + delta[t, 1]
        _gauss_add(fr, x0, y0, sigma, peak, half)
        for (r, pa0, con) in companions:
            ang = math.radians(pa0 + parang[t])
            _gauss_add(fr, x0 + r * math.cos(ang), y0 + r * math.sin(ang), sigma, peak * con, half)
        cube[t] = fr
    if noise:
        if cube.size <= 4e7:
            lam = np.clip(cube.astype(np.float64) + sky, 0, None)
            cube[...] = (rng.poisson(lam) - sky + rng.normal(0.0, read, cube.shape)).astype(np.float32)
        else:
            for t in range(T):
                lam = np.clip(cube[t] + np.float32(sky), 0, None)
                cube[t] += np.sqrt(lam + np.float32(read * read)) * rng.standard_normal((N, N), dtype=np.float32)
    if edges is None:
        edges = default_edges(N)
    return ADICube(cube=cube, parang=parang, dx=-delta[:, 0].copy(), dy=-delta[:, 1].copy(), fwhm=fwhm,
                   n_fwhm=n_fwhm, edges=np.asarray(edges, np.float64), peak=peak,
                   companions=list(companions), name=name)


def small_cube(seed: int = 0, T: int = 32, N: int = 128) -> ADICube:
    """32 frames of 128 x 128: Gaussian core FWHM 4 px, static speckles from a
    64-px pupil, angles linear over 0-40 deg, 2 companions at 20 and 40 px
    with contrast 1e-3, offsets U(-0.5, 0.5) px, Poisson + 5 e- read noise."""
    return make_cube(T, N, seed, parang=np.linspace(0.0, 40.0, T), peak=1e4, rho=1.0,
                     name=f"{T}x{N}x{N} linear 0-40 deg")


def survey_cube(seed: int = 1, T: int = 2000, N: int = 512) -> ADICube:
    """2000 frames of 512 x 512 padded to 1024: alt-az angles (dec -30, lat
    -24.6, h in [-1.5 h, +1.5 h]), AR(1) speckles with rho = 0.99 per frame,
    5 companions at 10-100 px with contrast 1e-3 to 1e-5, peak 1e5 e-."""
    rng = np.random.default_rng(1000 + seed)
    radii = [10.0, 30.0, 50.0, 75.0, 100.0]
    cons = np.logspace(-3, -5, 5)
    comps = [(r, float(rng.uniform(0, 360)), float(k)) for r, k in zip(radii, cons)]
    return make_cube(T, N, seed, parang=altaz_parang(T), peak=1e5, rho=0.99, companions=comps,
                     name=f"{T}x{N}x{N} alt-az")


def random_frames(T: int, N: int, seed: int, smooth: bool = False, dtype=np.float32) -> np.ndarray:
    """Plain seeded test frames ([T][N][N], float32 by default): white noise, or a smooth
    field: four axis-aligned elliptical Gaussians, widths 3 to max(3, N/32)
    px (content at the Nyquist frequency below 1e-18 of the peak), centres
    within N/10 of the frame centre, so the content stays more than seven
    widths inside the frame under shifts of a few pixels and any rotation."""
    rng = np.random.default_rng(seed)
    if not smooth:
        return rng.standard_normal((T, N, N)).astype(dtype)
    out = np.zeros((T, N, N), dtype)
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    c = N / 2.0
    smax = max(3.0, N / 32.0)
    for t in range(T):
        for _ in range(4):
            r = rng.uniform(0, N / 10)
            a = rng.uniform(0, 2 * np.pi)
            x0, y0 = c + r * np.cos(a), c + r * np.sin(a)
            sx, sy = rng.uniform(3.0, smax), rng.uniform(3.0, smax)
            out[t] += (rng.uniform(0.5, 2.0) * np.exp(-((xx - x0) ** 2 / (2 * sx * sx) + (yy - y0) ** 2 / (2 * sy * sy)))).astype(dtype)
    return out


def uneven_spec(seed: int = 3, n_cubes: int = 48, sides=(64, 128, 256, 512, 1024), t_range=(16, 400),
                max_shift: float = 2.0):
    """Shapes and per-frame parameters of an uneven batch: sides drawn from
    ``sides``, frame counts uniform in ``t_range``, shifts U(-2, 2) px,
    rotations U(0, 360) deg.  Returns a list of (n, T, dx, dy, theta)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_cubes):
        n = int(rng.choice(sides))
        T = int(rng.integers(t_range[0], t_range[1] + 1))
        out.append((n, T, rng.uniform(-max_shift, max_shift, T), rng.uniform(-max_shift, max_shift, T),
                    rng.uniform(0.0, 360.0, T)))
    return out


def uneven_batch(seed: int = 3, n_cubes: int = 48, sides=(64, 128, 256, 512, 1024), t_range=(16, 400),
                 max_shift: float = 2.0):
    """An uneven batch with its frames: white noise plus a Gaussian star at
    the centre (content does not matter to the geometry, the sizes do).
    Returns a list of (cube float32 [T][n][n], dx, dy, theta)."""
    rng = np.random.default_rng(seed + 7919)
    out = []
    for (n, T, dx, dy, th) in uneven_spec(seed, n_cubes, sides, t_range, max_shift):
        cube = rng.standard_normal((T, n, n), dtype=np.float32)
        yy, xx = np.mgrid[0:n, 0:n]
        cube += (100.0 * np.exp(-((xx - n / 2) ** 2 + (yy - n / 2) ** 2) / (2 * 1.7 ** 2))).astype(np.float32)
        out.append((cube, dx, dy, th))
    return out


@dataclass
class StarFrames:
    cube: np.ndarray          # float32 [T][N][N], sky-subtracted raw frames
    x: np.ndarray             # float64 [T], true star centre (column), NaN where the star is lost
    y: np.ndarray             # float64 [T], true star centre (row)
    fwhm: float               # FWHM of the core Gaussian, px
    peak: float


def star_frames(T: int, N: int, seed: int, *, fwhm: float = 4.0, peak: float = 1e4, jitter: float = 20.0,
                halo=((2.0, 0.08), (4.5, 0.012)), sky: float = 50.0, read: float = 5.0, lost: float = 0.0,
                second: float = 0.0) -> StarFrames:
    """Raw frames for registration: a star at (N/2, N/2) + delta, delta ~
    U(-jitter, jitter) px per axis (dithering and tip-tilt jitter), whose
    profile is a Gaussian core of FWHM ``fwhm`` and peak ``peak`` plus halo
    Gaussians of ``halo`` = (width factor, relative peak) pairs (a wing
    heavier than the core, as an AO-corrected PSF), sky-subtracted with
    noise N(0, read^2 + image + sky) (the Gaussian limit of the Poisson
    draw).  A fraction ``lost`` of the frames has the star at 1 % of its peak
    (AO loss: no patch above a threshold set for good frames).  ``second`` >
    0 adds a fainter star of that relative peak at a fixed offset (the
    brightest pixel stays on the target)."""
    rng = np.random.default_rng(seed)
    sig = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    cube = np.zeros((T, N, N), np.float32)
    xs = N / 2.0 + rng.uniform(-jitter, jitter, T)
    ys = N / 2.0 + rng.uniform(-jitter, jitter, T)
    is_lost = rng.random(T) < lost
    half = int(math.ceil(8.0 * sig * max([1.0] + [h[0] for h in halo])))
    for t in range(T):
        amp = peak * (0.01 if is_lost[t] else 1.0)
        frame = np.zeros((N, N), np.float64)
        _gauss_add(frame, xs[t], ys[t], sig, amp, half)
        for (k, rel) in halo:
            _gauss_add(frame, xs[t], ys[t], k * sig, amp * rel, half)
        if second > 0:
            _gauss_add(frame, xs[t] + 0.3 * N / 2, ys[t] - 0.2 * N / 2, sig, amp * second, half)
        var = read * read + sky + np.maximum(frame, 0.0)
        cube[t] = (frame + np.sqrt(var) * rng.standard_normal((N, N))).astype(np.float32)
    x = np.where(is_lost, np.nan, xs)
    y = np.where(is_lost, np.nan, ys)
    return StarFrames(cube=cube, x=x, y=y, fwhm=fwhm, peak=peak)
