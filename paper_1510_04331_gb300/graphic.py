"""Python binding of the C ABI in ``include/graphic.h`` (ctypes).

Argument marshalling only: every step runs in the CUDA library
``libgraphic.so``.  There is no CPU fallback; if the library is missing or
fails to load, every call raises :class:`GraphicError`.

Cubes are torch CUDA float32 tensors of shape (T, n, n) (C-contiguous);
per-frame parameters are anything numpy turns into float64 arrays.  Calls run
on the current torch CUDA stream of the cube's device and return when the
device work is done.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgraphic.so")

GRAPHIC_OK = 0
ERRORS = {
    -1: "GRAPHIC_ERR_INVALID_ARG",
    -2: "GRAPHIC_ERR_UNSUPPORTED",
    -3: "GRAPHIC_ERR_OOM",
    -4: "GRAPHIC_ERR_CUDA",
    -5: "GRAPHIC_ERR_NONFINITE",
    -6: "GRAPHIC_ERR_TIMEOUT",
    -7: "GRAPHIC_ERR_INTERNAL",
}
KERNELS = ["shift_x", "shift_y", "adi_general", "rot_pass1", "rot_pass2", "rot_pass3", "collapse_median",
           "batch_persistent", "register_argmax", "register_fit", "bin_median", "adi_band_prep", "adi_band_sweep"]
BATCH_PER_CUBE = 0
BATCH_PERSISTENT = 1
BATCH_GROUPED = 2
BATCH_AUTO = 3
PREC_FP32 = 0
PREC_BF16X3 = 1
PREC_FP16X3 = 2
PASS_SHIFT = 1
PASS_ROTATE = 2
SCHEDULE_KEYS = ["chunk_mb", "variant_1024", "batch_budget_mb", "batch_ctas_per_sm", "group_budget_mb",
                 "group_streams", "batch_mode"]


class BatchItem(ctypes.Structure):
    """graphic_batch_item of include/graphic.h."""
    _fields_ = [("in_", ctypes.c_void_p), ("out", ctypes.c_void_p), ("n_frames", ctypes.c_int64),
                ("n", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("dx", ctypes.POINTER(ctypes.c_double)), ("dy", ctypes.POINTER(ctypes.c_double)),
                ("theta_deg", ctypes.POINTER(ctypes.c_double))]
MAX_FRAMES_MEDIAN = 2048


class Cube(ctypes.Structure):
    """graphic_cube of include/graphic.h: a device cube with a frame stride."""
    _fields_ = [("data", ctypes.c_void_p), ("n_frames", ctypes.c_int64), ("n", ctypes.c_int32),
                ("reserved_", ctypes.c_int32), ("frame_stride", ctypes.c_int64)]


class ServerConfig(ctypes.Structure):
    """graphic_server_config of include/graphic_serve.h."""
    _fields_ = [("device", ctypes.c_int32), ("max_active", ctypes.c_int32), ("batch_mode", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("max_device_bytes", ctypes.c_int64),
                ("staging_bytes", ctypes.c_int64)]


class Request(ctypes.Structure):
    """graphic_request of include/graphic_serve.h."""
    _fields_ = [("host_in", ctypes.c_void_p), ("host_out", ctypes.c_void_p), ("n_frames", ctypes.c_int64),
                ("n", ctypes.c_int32), ("n_edges", ctypes.c_int32),
                ("dx", ctypes.POINTER(ctypes.c_double)), ("dy", ctypes.POINTER(ctypes.c_double)),
                ("parang", ctypes.POINTER(ctypes.c_double)), ("edges", ctypes.POINTER(ctypes.c_double)),
                ("fwhm", ctypes.c_double), ("n_fwhm", ctypes.c_double)]


class RequestInfo(ctypes.Structure):
    """graphic_request_info of include/graphic_serve.h."""
    _fields_ = [("status", ctypes.c_int32), ("reserved", ctypes.c_int32), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


SERVER_STATS = ["submitted", "admitted", "completed", "failed", "iterations", "batch_launches", "batch_items",
                "max_batch_items", "max_resident", "device_bytes_cap", "device_bytes_peak"]


class ServerStats(ctypes.Structure):
    """graphic_server_stats of include/graphic_serve.h."""
    _fields_ = [(k, ctypes.c_int64) for k in SERVER_STATS]


class GraphicError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32

# name -> argtypes, following include/graphic.h
_SIGS = {
    "graphic_create": [ctypes.POINTER(_P), ctypes.c_int],
    "graphic_destroy": [_P],
    "graphic_release": [_P],
    "graphic_set_stream": [_P, _P],
    "graphic_last_error": [],
    "graphic_version": [],
    "graphic_shift": [_P, _P, _P, _I64, _I32, _D, _D],
    "graphic_rotate": [_P, _P, _P, _I64, _I32, _D],
    "graphic_adi_subtract": [_P, _P, _P, _I64, _I32, _D, ctypes.c_double, ctypes.c_double, _D, _I32],
    "graphic_collapse_median": [_P, _P, _I64, _I32, _P],
    "graphic_reduce": [_P, _P, _P, _I64, _I32, _D, _D, _D, ctypes.c_double, ctypes.c_double, _D, _I32, _P],
    "graphic_adi_subtract_ex": [_P, _P, _P, _I64, _I32, _D, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                _D, _I32],
    "graphic_reduce_ex": [_P, _P, _P, _I64, _I32, _D, _D, _D, _D, ctypes.c_double, ctypes.c_double,
                          ctypes.c_double, _D, _I32, _P],
    "graphic_sky_median": [_P, _P, _I64, _I32, _D, _D, ctypes.c_double, _P],
    "graphic_sky_subtract": [_P, _P, _P, _I64, _I32, _P, _I32, _D, _D],
    "graphic_bad_pixel_map": [_P, _P, _I32, ctypes.c_double, _P],
    "graphic_bad_pixel_fix": [_P, _P, _I64, _I32, _P],
    "graphic_register": [_P, _P, _I64, _I32, ctypes.c_double, _I32, _I32, _I32, _I32, _P, _P],
    "graphic_bin_median": [_P, _P, _P, _I64, _I32, _I32],
    "graphic_bin_mean": [_D, _I64, _I32, _D],
    "graphic_inject": [_P, _P, _I64, _I32, _D, _D, _D, _I32, _D, _D, _D, _D, _D, _I32],
    "graphic_aperture": [_P, _P, _I32, _I32, _D, _D, ctypes.c_double, _D],
    "graphic_reduce_host": [_P, _P, _I64, _I32, _D, _D, _D, ctypes.c_double, ctypes.c_double, _D, _I32, _P],
    "graphic_profile": [_P, ctypes.c_int],
    "graphic_profile_read": [_P, _D, ctypes.POINTER(_I64), _I32],
    "graphic_kernel_name": [_I32],
    "graphic_rotate_noalloc": [_P, _P, _I64, _I32, _D, _P],
    "graphic_workspace_bytes": [_P, ctypes.POINTER(_I64)],
    "graphic_set_precision": [_P, _I32],
    "graphic_get_precision": [_P, ctypes.POINTER(_I32)],
    "graphic_server_create": [ctypes.POINTER(_P), ctypes.POINTER(ServerConfig)],
    "graphic_server_submit": [_P, ctypes.POINTER(Request), ctypes.POINTER(_I64)],
    "graphic_server_wait": [_P, _I64, ctypes.c_double, ctypes.POINTER(RequestInfo)],
    "graphic_server_clock": [_P],
    "graphic_server_stats_read": [_P, ctypes.POINTER(ServerStats)],
    "graphic_server_destroy": [_P],
    "graphic_batch_geom": [_P, _P, _I32, _I32],
    "graphic_autotune": [_P, _P, _I32, ctypes.c_char_p, _D],
    "graphic_get_schedule": [_P, ctypes.POINTER(_I32), _I32],
    "graphic_set_schedule": [_P, ctypes.POINTER(_I32), _I32],
    "graphic_shift_cube": [_P, ctypes.POINTER(Cube), ctypes.POINTER(Cube), _D, _D],
    "graphic_rotate_cube": [_P, ctypes.POINTER(Cube), ctypes.POINTER(Cube), _D],
    "graphic_adi_subtract_cube": [_P, ctypes.POINTER(Cube), ctypes.POINTER(Cube), _D, ctypes.c_double,
                                  ctypes.c_double, _D, _I32],
    "graphic_collapse_median_cube": [_P, ctypes.POINTER(Cube), _P],
    "graphic_reduce_cube": [_P, ctypes.POINTER(Cube), ctypes.POINTER(Cube), _D, _D, _D, ctypes.c_double,
                            ctypes.c_double, _D, _I32, _P],
}


def lib():
    """Load ``libgraphic.so`` (raises GraphicError when it is absent)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise GraphicError(-4, f"CUDA library not built ({LIB_PATH}); run paper_1510_04331_gb300.build.build()")
            try:
                L = ctypes.CDLL(LIB_PATH)
            except OSError as e:  # pragma: no cover
                raise GraphicError(-4, f"cannot load {LIB_PATH}: {e}")
            for name, args in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            L.graphic_last_error.restype = ctypes.c_char_p
            L.graphic_kernel_name.restype = ctypes.c_char_p
            L.graphic_server_clock.restype = ctypes.c_double
            _lib = L
    return _lib


def _check(rc: int):
    if rc != GRAPHIC_OK:
        raise GraphicError(rc, lib().graphic_last_error().decode())


def _f64(x, T):
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(x, np.float64), (T,)))
    return a, a.ctypes.data_as(_D)


def _cube(t, name="cube"):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.dim() == 3
            and t.is_contiguous() and t.shape[1] == t.shape[2]):
        raise GraphicError(-1, f"{name} must be a contiguous CUDA float32 tensor of shape (T, n, n)")
    return t


def _strided(t, name="cube"):
    """graphic_cube of a CUDA float32 tensor (T, n, n) whose rows and columns
    are dense and whose frames are frame_stride = t.stride(0) floats apart."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.dim() == 3
            and t.shape[1] == t.shape[2] and t.stride(2) == 1 and t.stride(1) == t.shape[2]):
        raise GraphicError(-1, f"{name} must be a CUDA float32 (T, n, n) tensor with dense frames")
    return Cube(t.data_ptr(), t.shape[0], t.shape[1], 0, t.stride(0))


class Context:
    """A library context bound to one CUDA device (owns its workspaces)."""

    def __init__(self, device: int = 0):
        h = _P()
        _check(lib().graphic_create(ctypes.byref(h), int(device)))
        self.h = h
        self.device = int(device)

    def close(self):
        if getattr(self, "h", None):
            lib().graphic_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        import torch
        s = torch.cuda.current_stream(self.device).cuda_stream
        _check(lib().graphic_set_stream(self.h, _P(s)))

    def graphic_shift(self, cube, dx, dy, out=None):
        import torch
        cube = _cube(cube)
        T, n = cube.shape[0], cube.shape[1]
        out = torch.empty_like(cube) if out is None else _cube(out, "out")
        dxa, pdx = _f64(dx, T)
        dya, pdy = _f64(dy, T)
        self._stream()
        _check(lib().graphic_shift(self.h, _P(cube.data_ptr()), _P(out.data_ptr()), T, n, pdx, pdy))
        return out

    # --- strided cubes (graphic_cube): views whose frames are not adjacent ---
    def graphic_shift_cube(self, cube, dx, dy, out):
        ci, co = _strided(cube), _strided(out, "out")
        T = cube.shape[0]
        dxa, pdx = _f64(dx, T)
        dya, pdy = _f64(dy, T)
        self._stream()
        _check(lib().graphic_shift_cube(self.h, ctypes.byref(ci), ctypes.byref(co), pdx, pdy))
        return out

    def graphic_rotate_cube(self, cube, theta_deg, out):
        ci, co = _strided(cube), _strided(out, "out")
        tha, pth = _f64(theta_deg, cube.shape[0])
        self._stream()
        _check(lib().graphic_rotate_cube(self.h, ctypes.byref(ci), ctypes.byref(co), pth))
        return out

    def graphic_adi_subtract_cube(self, cube, parang, fwhm, n_fwhm, edges, out):
        ci, co = _strided(cube), _strided(out, "out")
        paa, ppa = _f64(parang, cube.shape[0])
        e = np.ascontiguousarray(edges, np.float64)
        self._stream()
        _check(lib().graphic_adi_subtract_cube(self.h, ctypes.byref(ci), ctypes.byref(co), ppa, float(fwhm),
                                               float(n_fwhm), e.ctypes.data_as(_D), e.size))
        return out

    def graphic_collapse_median_cube(self, cube, out=None):
        import torch
        ci = _strided(cube)
        n = cube.shape[1]
        out = torch.empty((n, n), dtype=torch.float32, device=cube.device) if out is None else out
        self._stream()
        _check(lib().graphic_collapse_median_cube(self.h, ctypes.byref(ci), _P(out.data_ptr())))
        return out

    def graphic_reduce_cube(self, cube, dx, dy, parang, fwhm, n_fwhm, edges, work, out=None):
        import torch
        ci, cw = _strided(cube), _strided(work, "work")
        T, n = cube.shape[0], cube.shape[1]
        out = torch.empty((n, n), dtype=torch.float32, device=cube.device) if out is None else out
        dxa, pdx = _f64(dx, T)
        dya, pdy = _f64(dy, T)
        paa, ppa = _f64(parang, T)
        e = np.ascontiguousarray(edges, np.float64)
        self._stream()
        _check(lib().graphic_reduce_cube(self.h, ctypes.byref(ci), ctypes.byref(cw), pdx, pdy, ppa, float(fwhm),
                                         float(n_fwhm), e.ctypes.data_as(_D), e.size, _P(out.data_ptr())))
        return out

    def graphic_rotate(self, cube, theta_deg, out=None):
        import torch
        cube = _cube(cube)
        T, n = cube.shape[0], cube.shape[1]
        out = torch.empty_like(cube) if out is None else _cube(out, "out")
        tha, pth = _f64(theta_deg, T)
        self._stream()
        _check(lib().graphic_rotate(self.h, _P(cube.data_ptr()), _P(out.data_ptr()), T, n, pth))
        return out

    def graphic_adi_subtract(self, cube, parang, fwhm, n_fwhm, edges, out=None, times=None, t_max=None):
        """Median PSF subtraction; ``times`` / ``t_max`` add the maximum time
        separation of the reference frames (graphic_adi_subtract_ex)."""
        import torch
        cube = _cube(cube)
        T, n = cube.shape[0], cube.shape[1]
        out = torch.empty_like(cube) if out is None else _cube(out, "out")
        paa, ppa = _f64(parang, T)
        ta, pta = (None, None) if times is None else _f64(times, T)
        ea = np.ascontiguousarray(np.asarray(edges, np.float64).ravel())
        self._stream()
        _check(lib().graphic_adi_subtract_ex(self.h, _P(cube.data_ptr()), _P(out.data_ptr()), T, n, ppa, pta,
                                             float(t_max) if times is not None else 0.0, float(fwhm),
                                             float(n_fwhm), ea.ctypes.data_as(_D), ea.size))
        return out

    def graphic_collapse_median(self, cube, out=None):
        import torch
        cube = _cube(cube)
        T, n = cube.shape[0], cube.shape[1]
        out = torch.empty((n, n), dtype=torch.float32, device=cube.device) if out is None else out
        self._stream()
        _check(lib().graphic_collapse_median(self.h, _P(cube.data_ptr()), T, n, _P(out.data_ptr())))
        return out

    def graphic_reduce(self, cube, dx, dy, parang, fwhm, n_fwhm, edges, work=None, out=None, times=None,
                       t_max=None):
        """Full reduction; ``times`` / ``t_max`` as in graphic_adi_subtract."""
        import torch
        cube = _cube(cube)
        T, n = cube.shape[0], cube.shape[1]
        work = torch.empty_like(cube) if work is None else _cube(work, "work")
        out = torch.empty((n, n), dtype=torch.float32, device=cube.device) if out is None else out
        dxa, pdx = _f64(dx, T)
        dya, pdy = _f64(dy, T)
        paa, ppa = _f64(parang, T)
        ta, pta = (None, None) if times is None else _f64(times, T)
        ea = np.ascontiguousarray(np.asarray(edges, np.float64).ravel())
        self._stream()
        _check(lib().graphic_reduce_ex(self.h, _P(cube.data_ptr()), _P(work.data_ptr()), T, n, pdx, pdy, ppa, pta,
                                       float(t_max) if times is not None else 0.0, float(fwhm), float(n_fwhm),
                                       ea.ctypes.data_as(_D), ea.size, _P(out.data_ptr())))
        return out

    def graphic_reduce_host(self, cube_host, dx, dy, parang, fwhm, n_fwhm, edges, out_host=None):
        """Host buffers in, host result out (the library copies both ways).
        ``cube_host`` is a float32 numpy array or a (pinned) CPU torch tensor."""
        if hasattr(cube_host, "data_ptr"):
            T, n = int(cube_host.shape[0]), int(cube_host.shape[1])
            ptr = cube_host.data_ptr()
        else:
            cube_host = np.ascontiguousarray(cube_host, dtype=np.float32)
            T, n = cube_host.shape[0], cube_host.shape[1]
            ptr = cube_host.ctypes.data
        if out_host is None:
            out_host = np.empty((n, n), np.float32)
        optr = out_host.data_ptr() if hasattr(out_host, "data_ptr") else out_host.ctypes.data
        dxa, pdx = _f64(dx, T)
        dya, pdy = _f64(dy, T)
        paa, ppa = _f64(parang, T)
        ea = np.ascontiguousarray(np.asarray(edges, np.float64).ravel())
        self._stream()
        _check(lib().graphic_reduce_host(self.h, _P(ptr), T, n, pdx, pdy, ppa, float(fwhm), float(n_fwhm),
                                         ea.ctypes.data_as(_D), ea.size, _P(optr)))
        return out_host

    def _batch(self, cubes, outs, dx, dy, theta, passes=None):
        keep = []
        arr = (BatchItem * len(cubes))()
        for i, (c, o) in enumerate(zip(cubes, outs)):
            c = _cube(c)
            o = _cube(o, "out")
            T, n = c.shape[0], c.shape[1]
            a = [(None, None) if v is None else _f64(v, T) for v in (dx[i], dy[i], theta[i])]
            keep.append(a)
            arr[i] = BatchItem(c.data_ptr(), o.data_ptr(), T, n, 0 if passes is None else int(passes[i]),
                               a[0][1], a[1][1], a[2][1])
        return arr, keep

    def graphic_batch_geom(self, cubes, dx, dy, theta, outs=None, mode=BATCH_AUTO, passes=None):
        """Shift then rotate every frame of every cube (cubes of different n
        and frame counts); ``passes[i]`` (PASS_SHIFT / PASS_ROTATE mask, 0 =
        both) limits cube i to one step, whose unused parameters may be None.
        mode: BATCH_PER_CUBE, BATCH_PERSISTENT (one persistent launch),
        BATCH_GROUPED (per-size launches in one graph) or BATCH_AUTO (the
        schedule's mode)."""
        import torch
        outs = [torch.empty_like(c) for c in cubes] if outs is None else outs
        arr, keep = self._batch(cubes, outs, dx, dy, theta, passes)
        self._stream()
        _check(lib().graphic_batch_geom(self.h, ctypes.cast(arr, _P), len(cubes), int(mode)))
        return outs

    def graphic_autotune(self, cubes, dx, dy, theta, outs=None, cache_path=None):
        """Time the schedule candidates on this batch; returns (schedule dict,
        best per-cube ms, best persistent ms, best grouped ms)."""
        import torch
        outs = [torch.empty_like(c) for c in cubes] if outs is None else outs
        arr, keep = self._batch(cubes, outs, dx, dy, theta)
        best = (ctypes.c_double * 3)()
        self._stream()
        _check(lib().graphic_autotune(self.h, ctypes.cast(arr, _P), len(cubes),
                                      cache_path.encode() if cache_path else None, best))
        return self.schedule(), best[0], best[1], best[2]

    def schedule(self):
        k = len(SCHEDULE_KEYS)
        v = (_I32 * k)()
        _check(lib().graphic_get_schedule(self.h, v, k))
        return dict(zip(SCHEDULE_KEYS, list(v)))

    def set_schedule(self, **kw):
        cur = self.schedule()
        unknown = set(kw) - set(SCHEDULE_KEYS)
        if unknown:
            raise ValueError(f"unknown schedule keys {sorted(unknown)}")
        cur.update(kw)
        k = len(SCHEDULE_KEYS)
        v = (_I32 * k)(*[int(cur[key]) for key in SCHEDULE_KEYS])
        _check(lib().graphic_set_schedule(self.h, v, k))

    # --- image-quality pre-processing (Sect. 3.2) ---------------------------
    def graphic_sky_median(self, cube, mask_x=None, mask_y=None, mask_r=0.0, out=None):
        """Master sky: per-pixel median of the finite values outside each
        frame's star mask (NaN where none is left); returns an n x n tensor."""
        import torch
        cube = _cube(cube)
        T, n = cube.shape[0], cube.shape[1]
        out = torch.empty((n, n), dtype=torch.float32, device=cube.device) if out is None else out
        mxa, pmx = (None, None) if mask_x is None else _f64(mask_x, T)
        mya, pmy = (None, None) if mask_y is None else _f64(mask_y, T)
        self._stream()
        _check(lib().graphic_sky_median(self.h, _P(cube.data_ptr()), T, n, pmx, pmy, float(mask_r),
                                        _P(out.data_ptr())))
        return out

    def graphic_sky_subtract(self, cube, skies, frame_times, sky_times, out=None):
        """Each frame minus the master sky closest in time."""
        import torch
        cube = _cube(cube)
        skies = _cube(skies, "skies")
        T, n = cube.shape[0], cube.shape[1]
        out = torch.empty_like(cube) if out is None else _cube(out, "out")
        fta, pft = _f64(frame_times, T)
        sta, pst = _f64(sky_times, skies.shape[0])
        self._stream()
        _check(lib().graphic_sky_subtract(self.h, _P(cube.data_ptr()), _P(out.data_ptr()), T, n,
                                          _P(skies.data_ptr()), skies.shape[0], pft, pst))
        return out

    def graphic_bad_pixel_map(self, ref, C):
        """uint8 n x n map of the pixels of ref farther than C sigma from its median."""
        import torch
        if not (isinstance(ref, torch.Tensor) and ref.is_cuda and ref.dtype == torch.float32 and ref.dim() == 2
                and ref.is_contiguous() and ref.shape[0] == ref.shape[1]):
            raise GraphicError(-1, "ref must be a contiguous CUDA float32 n x n tensor")
        n = ref.shape[0]
        out = torch.empty((n, n), dtype=torch.uint8, device=ref.device)
        self._stream()
        _check(lib().graphic_bad_pixel_map(self.h, _P(ref.data_ptr()), n, float(C), _P(out.data_ptr())))
        return out

    def graphic_bad_pixel_fix(self, cube, bad_map=None):
        """In place: flagged and non-finite pixels replaced by the median of
        their finite 8-neighbours, pass by pass."""
        cube = _cube(cube)
        T, n = cube.shape[0], cube.shape[1]
        self._stream()
        _check(lib().graphic_bad_pixel_fix(self.h, _P(cube.data_ptr()), T, n,
                                           None if bad_map is None else _P(bad_map.data_ptr())))
        return cube

    def graphic_register(self, cube, thresh, R, min_size, max_size, w, out=None, iters=None):
        """Per frame: centroid of the thresholded patch around the brightest
        pixel, then a Moffat fit (Levenberg-Marquardt) started there.  Returns
        a (T, 8) float64 CUDA tensor: found, x0, y0, FWHM, I0, alpha, beta, Bg
        (iters, if given, a (T,) int32 CUDA tensor, receives the iterations)."""
        import torch
        cube = _cube(cube)
        T, n = cube.shape[0], cube.shape[1]
        if out is None:
            out = torch.empty((T, 8), dtype=torch.float64, device=cube.device)
        self._stream()
        _check(lib().graphic_register(self.h, _P(cube.data_ptr()), T, n, float(thresh), int(R), int(min_size),
                                      int(max_size), int(w), _P(out.data_ptr()),
                                      None if iters is None else _P(iters.data_ptr())))
        return out

    def graphic_bin_median(self, cube, B, out=None):
        """Median of every B consecutive frames (the last group may be
        shorter): a (ceil(T / B), n, n) CUDA tensor."""
        import torch
        cube = _cube(cube)
        T, n = cube.shape[0], cube.shape[1]
        if out is None:
            out = torch.empty(((T + int(B) - 1) // max(1, int(B)), n, n), dtype=torch.float32, device=cube.device)
        self._stream()
        _check(lib().graphic_bin_median(self.h, _P(cube.data_ptr()), _P(out.data_ptr()), T, n, int(B)))
        return out

    def graphic_inject(self, cube, parang, xc, yc, r, pa0, flux, alpha, beta, half):
        """In place: Moffat companions (radius r, position angle pa0 + parang,
        total flux) around the per-frame centres (xc, yc)."""
        cube = _cube(cube)
        T, n = cube.shape[0], cube.shape[1]
        pa, pa_p = _f64(parang, T)
        x, x_p = _f64(xc, T)
        y, y_p = _f64(yc, T)
        al, al_p = _f64(alpha, T)
        be, be_p = _f64(beta, T)
        rr = np.ascontiguousarray(np.atleast_1d(np.asarray(r, np.float64)))
        k = len(rr)
        p0, p0_p = _f64(pa0, k)
        fl, fl_p = _f64(flux, k)
        self._stream()
        _check(lib().graphic_inject(self.h, _P(cube.data_ptr()), T, n, pa_p, x_p, y_p, k, rr.ctypes.data_as(_D), p0_p,
                                    fl_p, al_p, be_p, int(half)))
        return cube

    def graphic_aperture(self, img, x, y, radius):
        """FP64 sums of the n x n CUDA image over the discs of `radius` around (x, y)."""
        import torch
        if not (isinstance(img, torch.Tensor) and img.is_cuda and img.dtype == torch.float32 and img.dim() == 2
                and img.is_contiguous() and img.shape[0] == img.shape[1]):
            raise GraphicError(-1, "img must be a contiguous CUDA float32 n x n tensor")
        xs = np.ascontiguousarray(np.atleast_1d(np.asarray(x, np.float64)))
        ys, ys_p = _f64(y, len(xs))
        out = np.zeros(len(xs))
        self._stream()
        _check(lib().graphic_aperture(self.h, _P(img.data_ptr()), img.shape[0], len(xs), xs.ctypes.data_as(_D), ys_p,
                                      float(radius), out.ctypes.data_as(_D)))
        return out

    def set_precision(self, precision: int):
        """PREC_FP32 (default), PREC_BF16X3 or PREC_FP16X3: arithmetic of the
        line passes for frames of n = 1024 (tensor-core DFT stages)."""
        _check(lib().graphic_set_precision(self.h, int(precision)))

    def precision(self) -> int:
        v = _I32()
        _check(lib().graphic_get_precision(self.h, ctypes.byref(v)))
        return v.value

    def profile(self, enable: bool):
        _check(lib().graphic_profile(self.h, int(bool(enable))))

    def profile_read(self):
        n = len(KERNELS)
        ms = (ctypes.c_double * n)()
        cnt = (_I64 * n)()
        _check(lib().graphic_profile_read(self.h, ms, cnt, n))
        return {KERNELS[k]: (ms[k], cnt[k]) for k in range(n)}

    def workspace_bytes(self) -> int:
        b = _I64()
        _check(lib().graphic_workspace_bytes(self.h, ctypes.byref(b)))
        return b.value

    def release(self):
        _check(lib().graphic_release(self.h))


_ctx = {}


class Server:
    """Serving loop (include/graphic_serve.h): full reductions of host cubes
    submitted by any thread, admitted by device memory and batched across
    requests on the GPU.  ``submit`` returns a request id; ``wait`` returns
    (result n x n float32 array, info dict with status and server-clock
    times).  The host cube must stay alive and unchanged until its request
    is waited for (pinned memory makes its copy asynchronous)."""

    def __init__(self, device=0, max_active=0, batch_mode=BATCH_GROUPED, max_device_bytes=0, staging_bytes=0):
        cfg = ServerConfig(int(device), int(max_active), int(batch_mode), 0, int(max_device_bytes),
                           int(staging_bytes))
        h = _P()
        _check(lib().graphic_server_create(ctypes.byref(h), ctypes.byref(cfg)))
        self.h = h
        self._keep = {}
        self._klock = threading.Lock()

    def submit(self, cube_host, dx, dy, parang, fwhm, n_fwhm, edges, out_host=None):
        if hasattr(cube_host, "data_ptr"):
            if cube_host.is_cuda or not cube_host.is_contiguous() or str(cube_host.dtype) != "torch.float32":
                raise GraphicError(-1, "cube must be a contiguous float32 host tensor")
            T, n = int(cube_host.shape[0]), int(cube_host.shape[1])
            ptr = cube_host.data_ptr()
        else:
            cube_host = np.ascontiguousarray(cube_host, dtype=np.float32)
            T, n = cube_host.shape[0], cube_host.shape[1]
            ptr = cube_host.ctypes.data
        if len(cube_host.shape) != 3 or cube_host.shape[1] != cube_host.shape[2]:
            raise GraphicError(-1, "cube must have shape (T, n, n)")
        if out_host is None:
            out_host = np.empty((n, n), np.float32)
        if tuple(out_host.shape) != (n, n):
            raise GraphicError(-1, "out must have shape (n, n)")
        optr = out_host.data_ptr() if hasattr(out_host, "data_ptr") else out_host.ctypes.data
        dxa, pdx = _f64(dx, T)
        dya, pdy = _f64(dy, T)
        paa, ppa = _f64(parang, T)
        ea = np.ascontiguousarray(np.asarray(edges, np.float64).ravel())
        rq = Request(ptr, optr, T, n, ea.size, pdx, pdy, ppa, ea.ctypes.data_as(_D), float(fwhm), float(n_fwhm))
        rid = _I64()
        _check(lib().graphic_server_submit(self.h, ctypes.byref(rq), ctypes.byref(rid)))
        with self._klock:
            self._keep[rid.value] = (cube_host, out_host)
        return rid.value

    def wait(self, rid, timeout=None):
        info = RequestInfo()
        _check(lib().graphic_server_wait(self.h, int(rid), -1.0 if timeout is None else float(timeout),
                                         ctypes.byref(info)))
        with self._klock:
            _, out = self._keep.pop(int(rid))
        d = {"status": info.status, "t_submit": info.t_submit, "t_admit": info.t_admit, "t_done": info.t_done}
        if info.status != GRAPHIC_OK:
            d["error"] = f"{ERRORS.get(info.status, info.status)}: {lib().graphic_last_error().decode()}"
        return out, d

    def clock(self):
        return lib().graphic_server_clock(self.h)

    def stats(self):
        st = ServerStats()
        _check(lib().graphic_server_stats_read(self.h, ctypes.byref(st)))
        return {k: getattr(st, k) for k in SERVER_STATS}

    def close(self):
        if getattr(self, "h", None):
            lib().graphic_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def context(device=None) -> Context:
    """Default per-device context."""
    import torch
    d = torch.cuda.current_device() if device is None else int(device)
    if d not in _ctx:
        _ctx[d] = Context(d)
    return _ctx[d]


def graphic_shift(cube, dx, dy, out=None):
    return context(cube.device.index).graphic_shift(cube, dx, dy, out)


def graphic_rotate(cube, theta_deg, out=None):
    return context(cube.device.index).graphic_rotate(cube, theta_deg, out)


def graphic_adi_subtract(cube, parang, fwhm, n_fwhm, edges, out=None, times=None, t_max=None):
    return context(cube.device.index).graphic_adi_subtract(cube, parang, fwhm, n_fwhm, edges, out, times, t_max)


def graphic_collapse_median(cube, out=None):
    return context(cube.device.index).graphic_collapse_median(cube, out)


def graphic_reduce(cube, dx, dy, parang, fwhm, n_fwhm, edges, work=None, out=None, times=None, t_max=None):
    return context(cube.device.index).graphic_reduce(cube, dx, dy, parang, fwhm, n_fwhm, edges, work, out, times,
                                                     t_max)


def graphic_rotate_noalloc(cube, theta_deg, out):
    """Rotation through the entry point that allocates no device memory
    (its working memory is a fixed static array in the library).  ``out``
    must be given: this path creates nothing on the device itself."""
    import torch
    cube = _cube(cube)
    out = _cube(out, "out")
    T, n = cube.shape[0], cube.shape[1]
    tha, pth = _f64(theta_deg, T)
    s = torch.cuda.current_stream(cube.device).cuda_stream
    with torch.cuda.device(cube.device):
        _check(lib().graphic_rotate_noalloc(_P(cube.data_ptr()), _P(out.data_ptr()), T, n, pth, _P(s)))
    return out


def graphic_reduce_host(cube_host, dx, dy, parang, fwhm, n_fwhm, edges, device=0, out_host=None):
    return context(device).graphic_reduce_host(cube_host, dx, dy, parang, fwhm, n_fwhm, edges, out_host)


def graphic_register(cube, thresh, R, min_size, max_size, w, out=None, iters=None):
    return context().graphic_register(cube, thresh, R, min_size, max_size, w, out, iters)


def graphic_bin_median(cube, B, out=None):
    return context().graphic_bin_median(cube, B, out)


def bin_mean(values, B):
    """Mean of every B consecutive values (the angle or time of a median bin)."""
    v = np.ascontiguousarray(np.asarray(values, np.float64))
    out = np.zeros((len(v) + int(B) - 1) // max(1, int(B)))
    _check(lib().graphic_bin_mean(v.ctypes.data_as(_D), len(v), int(B), out.ctypes.data_as(_D)))
    return out


def graphic_inject(cube, parang, xc, yc, r, pa0, flux, alpha, beta, half):
    return context().graphic_inject(cube, parang, xc, yc, r, pa0, flux, alpha, beta, half)


def graphic_aperture(img, x, y, radius):
    return context().graphic_aperture(img, x, y, radius)

