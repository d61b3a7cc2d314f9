"""FP64 CPU oracle for the GRAPHIC ADI hot path (arXiv:1510.04331).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.  The
arithmetic lives in ``graphic_oracle.c`` (plain C, hand-written radix-2 FFT,
FP64 throughout, OpenMP over frames / pixels); this module only compiles it
with gcc and marshals numpy arrays through ctypes.

Functions and the passages they follow:

* ``fft`` / ``dft`` -- Sect. 3.3.1, definition of the Fourier transform.
* ``shift`` -- Sect. 3.3.1, shift theorem with the separable 2-D phasor on a
  zero-padded (2x) frame.
* ``rotate`` -- Sect. 3.4, rotation as three shears, each a 1-D Fourier shift
  per line on the 2x padded frame.
* ``alpha_min_deg`` / ``gate_mask`` / ``adi_subtract`` -- Sect. 3.3, the
  reference-frame condition on field rotation and the per-frame median PSF
  built without combination coefficients.
* ``collapse_median`` -- Sect. 3.4, merge of the derotated frames (a median).
* ``reduce`` -- the four steps chained (Sect. 3, items 3 and 4 of the
  reduction procedure).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphic_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_f = ctypes.POINTER(ctypes.c_float)
_ll = ctypes.POINTER(ctypes.c_longlong)
_u8 = ctypes.POINTER(ctypes.c_ubyte)


def build(force: bool = False) -> str:
    """Compile ``graphic_oracle.c`` into ``liboracle.so`` next to it (gcc)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.oracle_fft.argtypes = [_d, ctypes.c_int, ctypes.c_int]
            lib.oracle_dft.argtypes = [_d, _d, ctypes.c_int, ctypes.c_int]
            lib.oracle_shift_line.argtypes = [_d, _d, ctypes.c_int, ctypes.c_double]
            lib.oracle_shift.argtypes = [_d, _d, ctypes.c_longlong, ctypes.c_int, _d, _d]
            lib.oracle_shift_padded.argtypes = [_d, _d, ctypes.c_int, ctypes.c_double, ctypes.c_double]
            lib.oracle_rotate.argtypes = [_d, _d, ctypes.c_longlong, ctypes.c_int, _d, ctypes.c_int]
            lib.oracle_alpha_min_deg.argtypes = [ctypes.c_double] * 3
            lib.oracle_alpha_min_deg.restype = ctypes.c_double
            lib.oracle_gate_mask.argtypes = [_d, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_double, _u8]
            lib.oracle_gate_mask_t.argtypes = [_d, _d, ctypes.c_double, ctypes.c_longlong, ctypes.c_longlong,
                                               ctypes.c_double, _u8]
            lib.oracle_annulus_of.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _d, ctypes.c_int]
            lib.oracle_adi_subtract_pixels.argtypes = [
                _d, ctypes.c_longlong, ctypes.c_int, _d, ctypes.c_double, ctypes.c_double, _d, ctypes.c_int,
                _ll, ctypes.c_longlong, _d]
            lib.oracle_adi_subtract_pixels_f32.argtypes = [
                _f, ctypes.c_longlong, ctypes.c_int, _d, ctypes.c_double, ctypes.c_double, _d, ctypes.c_int,
                _ll, ctypes.c_longlong, _f]
            lib.oracle_collapse_median_pixels.argtypes = [_d, ctypes.c_longlong, ctypes.c_int, _ll,
                                                          ctypes.c_longlong, _d]
            lib.oracle_collapse_median_pixels_f32.argtypes = [_f, ctypes.c_longlong, ctypes.c_int, _ll,
                                                              ctypes.c_longlong, _f]
            lib.oracle_reduce.argtypes = [_d, _d, ctypes.c_longlong, ctypes.c_int, _d, _d, _d, ctypes.c_double,
                                          ctypes.c_double, _d, ctypes.c_int, _d]
            lib.oracle_adi_subtract_pixels_t.argtypes = [
                _d, ctypes.c_longlong, ctypes.c_int, _d, _d, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                _d, ctypes.c_int, _ll, ctypes.c_longlong, _d]
            lib.oracle_adi_subtract_pixels_f32_t.argtypes = [
                _f, ctypes.c_longlong, ctypes.c_int, _d, _d, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                _d, ctypes.c_int, _ll, ctypes.c_longlong, _f]
            lib.oracle_reduce_t.argtypes = [_d, _d, ctypes.c_longlong, ctypes.c_int, _d, _d, _d, _d,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_double, _d, ctypes.c_int, _d]
            lib.oracle_sky_median_f32.argtypes = [_f, ctypes.c_longlong, ctypes.c_int, _d, _d, ctypes.c_double, _f]
            lib.oracle_sky_subtract_f32.argtypes = [_f, _f, ctypes.c_longlong, ctypes.c_int, _f, ctypes.c_int, _d,
                                                    _d]
            lib.oracle_bad_pixel_map_f32.argtypes = [_f, ctypes.c_int, ctypes.c_double, _u8]
            lib.oracle_bad_pixel_fix_f32.argtypes = [_f, ctypes.c_longlong, ctypes.c_int, _u8]
            lib.oracle_centroid_frame_f32.argtypes = [_f, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                                      ctypes.c_int, _d, _d, ctypes.POINTER(ctypes.c_int)]
            lib.oracle_moffat_fit_f32.argtypes = [_f, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_double, ctypes.c_int, _d]
            lib.oracle_moffat_fwhm.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.oracle_moffat_fwhm.restype = ctypes.c_double
            lib.oracle_bin_median_f32.argtypes = [_f, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _f]
            lib.oracle_inject_f32.argtypes = [_f, ctypes.c_longlong, ctypes.c_int, _d, _d, _d, ctypes.c_int, _d, _d,
                                              _d, _d, _d, ctypes.c_int]
            lib.oracle_aperture_f32.argtypes = [_f, ctypes.c_int, ctypes.c_int, _d, _d, ctypes.c_double, _d]
            lib.oracle_last_max_imag.restype = ctypes.c_double
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a, typ):
    return a.ctypes.data_as(typ)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return _load().oracle_num_threads()


def last_max_imag() -> float:
    """Largest |imag part| discarded by the last shift / rotate call."""
    return _load().oracle_last_max_imag()


def fft(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Radix-2 FFT of a complex vector (power-of-two length)."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.complex128)).copy()
    buf = a.view(np.float64)
    if _load().oracle_fft(_p(buf, _d), a.size, int(inverse)) != 0:
        raise ValueError("length must be a power of two")
    return a


def dft(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Brute-force DFT (any length)."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
    out = np.empty_like(a)
    _load().oracle_dft(_p(a.view(np.float64), _d), _p(out.view(np.float64), _d), a.size, int(inverse))
    return out


def shift_line(x: np.ndarray, d: float) -> np.ndarray:
    """Periodic Fourier shift of one real line by d (content moves by +d)."""
    a = _c64(x)
    out = np.empty_like(a)
    if _load().oracle_shift_line(_p(a, _d), _p(out, _d), a.size, float(d)) != 0:
        raise ValueError("length must be a power of two")
    return out


def shift(cube: np.ndarray, dx, dy) -> np.ndarray:
    """Shift every frame of a [T][N][N] cube by (dx[t], dy[t]) pixels."""
    c = _c64(cube)
    T, N, _ = c.shape
    dx = _c64(np.broadcast_to(dx, (T,)))
    dy = _c64(np.broadcast_to(dy, (T,)))
    out = np.empty_like(c)
    if _load().oracle_shift(_p(c, _d), _p(out, _d), T, N, _p(dx, _d), _p(dy, _d)) != 0:
        raise ValueError("bad shape")
    return out


def shift_padded(frame: np.ndarray, dx: float, dy: float) -> np.ndarray:
    """Shift of one N x N frame without the final crop (M x M output)."""
    f = _c64(frame)
    N = f.shape[0]
    out = np.empty((2 * N, 2 * N), np.float64)
    _load().oracle_shift_padded(_p(f, _d), _p(out, _d), N, float(dx), float(dy))
    return out


def rotate(cube: np.ndarray, theta_deg, reduce90: bool = True) -> np.ndarray:
    """Rotate every frame of a [T][N][N] cube by theta_deg[t] (CCW)."""
    c = _c64(cube)
    T, N, _ = c.shape
    th = _c64(np.broadcast_to(theta_deg, (T,)))
    out = np.empty_like(c)
    if _load().oracle_rotate(_p(c, _d), _p(out, _d), T, N, _p(th, _d), int(reduce90)) != 0:
        raise ValueError("bad shape")
    return out


def alpha_min_deg(fwhm: float, n_fwhm: float, r: float) -> float:
    return _load().oracle_alpha_min_deg(float(fwhm), float(n_fwhm), float(r))


def _times(times, T):
    """Time stamps as a contiguous float64 array of T (None: no time gate)."""
    if times is None:
        return None
    t = _c64(times)
    if t.size != T:
        raise ValueError("times must have one entry per frame")
    return t


def gate_mask(parang, i: int, amin_deg: float, times=None, t_max=None) -> np.ndarray:
    """Reference set of frame i (Sect. 3.3); with ``times`` also |t_k - t_i| < t_max."""
    pa = _c64(parang)
    mask = np.zeros(pa.size, np.uint8)
    tt = _times(times, pa.size)
    _load().oracle_gate_mask_t(_p(pa, _d), None if tt is None else _p(tt, _d),
                               float(t_max) if tt is not None else 0.0, pa.size, int(i), float(amin_deg),
                               _p(mask, _u8))
    return mask.astype(bool)


def annulus_of(i: int, j: int, N: int, edges) -> int:
    e = _c64(edges)
    return _load().oracle_annulus_of(int(i), int(j), int(N), _p(e, _d), e.size)


def adi_subtract(cube: np.ndarray, parang, fwhm: float, n_fwhm: float, edges, pixels=None, times=None,
                 t_max=None) -> np.ndarray:
    """Angle-gated median PSF subtraction.

    FP64 for float64 cubes, FP32 median arithmetic for float32 cubes.  With
    ``pixels`` (flat indices) returns an array [n_pix][T]; without, the full
    residual cube [T][N][N].  ``times`` / ``t_max``: the paper's maximum time
    separation of reference frames (None: no time condition).
    """
    f32 = np.asarray(cube).dtype == np.float32
    c = np.ascontiguousarray(cube, dtype=np.float32 if f32 else np.float64)
    T, N, _ = c.shape
    pa = _c64(parang)
    e = _c64(edges)
    full = pixels is None
    pix = np.arange(N * N, dtype=np.int64) if full else np.ascontiguousarray(pixels, dtype=np.int64)
    out = np.empty((pix.size, T), np.float32 if f32 else np.float64)
    lib = _load()
    tt = _times(times, T)
    tp = None if tt is None else _p(tt, _d)
    tm = float(t_max) if tt is not None else 0.0
    if f32:
        rc = lib.oracle_adi_subtract_pixels_f32_t(_p(c, _f), T, N, _p(pa, _d), tp, tm, float(fwhm), float(n_fwhm),
                                                  _p(e, _d), e.size, _p(pix, _ll), pix.size, _p(out, _f))
    else:
        rc = lib.oracle_adi_subtract_pixels_t(_p(c, _d), T, N, _p(pa, _d), tp, tm, float(fwhm), float(n_fwhm),
                                              _p(e, _d), e.size, _p(pix, _ll), pix.size, _p(out, _d))
    if rc != 0:
        raise ValueError("bad arguments")
    if full:
        return np.ascontiguousarray(out.T.reshape(T, N, N))
    return out


def collapse_median(cube: np.ndarray, pixels=None) -> np.ndarray:
    """Per-pixel median over the frames (FP64, or FP32 for float32 input)."""
    f32 = np.asarray(cube).dtype == np.float32
    c = np.ascontiguousarray(cube, dtype=np.float32 if f32 else np.float64)
    T, N, _ = c.shape
    full = pixels is None
    pix = np.arange(N * N, dtype=np.int64) if full else np.ascontiguousarray(pixels, dtype=np.int64)
    out = np.empty(pix.size, np.float32 if f32 else np.float64)
    lib = _load()
    if f32:
        lib.oracle_collapse_median_pixels_f32(_p(c, _f), T, N, _p(pix, _ll), pix.size, _p(out, _f))
    else:
        lib.oracle_collapse_median_pixels(_p(c, _d), T, N, _p(pix, _ll), pix.size, _p(out, _d))
    return out.reshape(N, N) if full else out


def reduce(cube: np.ndarray, dx, dy, parang, fwhm: float, n_fwhm: float, edges, times=None,
           t_max=None) -> np.ndarray:
    """Shift, median PSF subtraction (optionally time-gated), derotation by
    -parang, median collapse."""
    c = _c64(cube)
    T, N, _ = c.shape
    work = np.empty_like(c)
    out = np.empty((N, N), np.float64)
    dx = _c64(np.broadcast_to(dx, (T,)))
    dy = _c64(np.broadcast_to(dy, (T,)))
    pa = _c64(parang)
    e = _c64(edges)
    tt = _times(times, T)
    rc = _load().oracle_reduce_t(_p(c, _d), _p(work, _d), T, N, _p(dx, _d), _p(dy, _d), _p(pa, _d),
                                 None if tt is None else _p(tt, _d), float(t_max) if tt is not None else 0.0,
                                 float(fwhm), float(n_fwhm), _p(e, _d), e.size, _p(out, _d))
    if rc != 0:
        raise ValueError("bad arguments")
    return out


# --------------------------------------------------------------------------
# Image-quality pre-processing (Sect. 3.2), FP32 data
# --------------------------------------------------------------------------

def _f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def sky_median(cube, mask_x=None, mask_y=None, mask_r=0.0) -> np.ndarray:
    """Master sky: per-pixel median over the frames of the finite values
    outside each frame's star mask (NaN where none is left)."""
    c = _f32(cube)
    T, N, _ = c.shape
    sky = np.empty((N, N), np.float32)
    mx = None if mask_x is None else _c64(np.broadcast_to(mask_x, (T,)))
    my = None if mask_y is None else _c64(np.broadcast_to(mask_y, (T,)))
    rc = _load().oracle_sky_median_f32(_p(c, _f), T, N, None if mx is None else _p(mx, _d),
                                       None if my is None else _p(my, _d), float(mask_r), _p(sky, _f))
    if rc != 0:
        raise ValueError("bad arguments")
    return sky


def sky_subtract(cube, skies, frame_times, sky_times) -> np.ndarray:
    """Each frame minus the master sky closest in time (earlier on a tie)."""
    c = _f32(cube)
    T, N, _ = c.shape
    sk = _f32(skies)
    ft = _c64(frame_times)
    st = _c64(sky_times)
    out = np.empty_like(c)
    rc = _load().oracle_sky_subtract_f32(_p(c, _f), _p(out, _f), T, N, _p(sk, _f), sk.shape[0], _p(ft, _d),
                                         _p(st, _d))
    if rc != 0:
        raise ValueError("bad arguments")
    return out


def bad_pixel_map(ref, C: float) -> np.ndarray:
    """Pixels of ref farther than C sigma from its median (bool map)."""
    r = _f32(ref)
    N = r.shape[0]
    m = np.zeros((N, N), np.uint8)
    _load().oracle_bad_pixel_map_f32(_p(r, _f), N, float(C), _p(m, _u8))
    return m.astype(bool)


def bad_pixel_fix(cube, bad_map=None):
    """Flagged and non-finite pixels replaced by the median of their finite
    8-neighbours, pass by pass until none is left.  Returns (cube, status)."""
    c = np.array(cube, dtype=np.float32, copy=True, order="C")
    T, N, _ = c.shape
    m = None if bad_map is None else np.ascontiguousarray(bad_map, dtype=np.uint8)
    st = _load().oracle_bad_pixel_fix_f32(_p(c, _f), T, N, None if m is None else _p(m, _u8))
    return c, st


# --------------------------------------------------------------------------
# Registration (Sect. 3.1): centroid patch search, Moffat fit
# --------------------------------------------------------------------------

def centroid(frame, thresh: float, R: int, min_size: int, max_size: int):
    """(found, cx, cy, patch size) of one frame."""
    f = _f32(frame)
    N = f.shape[0]
    cx, cy, sz = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    found = _load().oracle_centroid_frame_f32(_p(f, _f), N, float(thresh), int(R), int(min_size), int(max_size),
                                              ctypes.byref(cx), ctypes.byref(cy), ctypes.byref(sz))
    return bool(found), cx.value, cy.value, sz.value


def moffat_fit(frame, cx: float, cy: float, alpha0: float, w: int):
    """Levenberg-Marquardt Moffat fit: (p = [I0, x0, y0, alpha, beta, Bg], iterations)."""
    f = _f32(frame)
    N = f.shape[0]
    p = np.zeros(6)
    it = _load().oracle_moffat_fit_f32(_p(f, _f), N, float(cx), float(cy), float(alpha0), int(w), _p(p, _d))
    return p, it


def moffat_fwhm(alpha: float, beta: float) -> float:
    return _load().oracle_moffat_fwhm(float(alpha), float(beta))


def register(cube, thresh: float, R: int, min_size: int, max_size: int, w: int):
    """Per frame: centroid, then the Moffat fit started there with alpha0 =
    max(1, sqrt(patch size / pi)).  Returns arrays found, x0, y0, fwhm
    (NaN where no centroid was found)."""
    c = _f32(cube)
    T = c.shape[0]
    found = np.zeros(T, bool)
    x0 = np.full(T, np.nan)
    y0 = np.full(T, np.nan)
    fw = np.full(T, np.nan)
    for t in range(T):
        ok, cx, cy, sz = centroid(c[t], thresh, R, min_size, max_size)
        if not ok:
            continue
        p, _ = moffat_fit(c[t], cx, cy, max(1.0, math.sqrt(sz / math.pi)), w)
        found[t] = True
        x0[t], y0[t], fw[t] = p[1], p[2], moffat_fwhm(p[3], p[4])
    return found, x0, y0, fw


# --------------------------------------------------------------------------
# Photometric-accuracy and binning experiments (Sect. 4.2, 4.3)
# --------------------------------------------------------------------------

def bin_median(cube, B: int) -> np.ndarray:
    """Per-pixel median of each group of B consecutive frames (the last group
    may be shorter): ceil(T / B) frames."""
    c = _f32(cube)
    T, N = c.shape[0], c.shape[1]
    out = np.empty(((T + B - 1) // B, N, N), np.float32)
    if _load().oracle_bin_median_f32(_p(c, _f), T, N, int(B), _p(out, _f)) != 0:
        raise ValueError("bad arguments")
    return out


def inject(cube, parang, xc, yc, r, pa0, flux, alpha, beta, half: int) -> np.ndarray:
    """A copy of cube with Moffat companions (radius r_j, position angle
    pa0_j + parang_t, total flux flux_j, per-frame alpha, beta) added around
    the per-frame centres (xc, yc) on windows of half-size `half`."""
    c = _f32(cube).copy()
    T, N = c.shape[0], c.shape[1]
    pa, x, y = (_c64(np.broadcast_to(np.asarray(v, np.float64), (T,))) for v in (parang, xc, yc))
    al, be = (_c64(np.broadcast_to(np.asarray(v, np.float64), (T,))) for v in (alpha, beta))
    r, pa0, flux = (_c64(np.atleast_1d(v)) for v in (r, pa0, flux))
    if _load().oracle_inject_f32(_p(c, _f), T, N, _p(pa, _d), _p(x, _d), _p(y, _d), len(r), _p(r, _d), _p(pa0, _d),
                                 _p(flux, _d), _p(al, _d), _p(be, _d), int(half)) != 0:
        raise ValueError("bad arguments")
    return c


def aperture(img, x, y, radius: float) -> np.ndarray:
    """FP64 sums of img over the pixels within `radius` of each (x, y)."""
    f = _f32(img)
    x, y = _c64(np.atleast_1d(x)), _c64(np.atleast_1d(y))
    out = np.zeros(len(x))
    if _load().oracle_aperture_f32(_p(f, _f), f.shape[0], len(x), _p(x, _d), _p(y, _d), float(radius),
                                   _p(out, _d)) != 0:
        raise ValueError("bad arguments")
    return out

