"""graphic_rotate_noalloc: the rotation entry point that allocates no device
memory, for callers that cannot call cudaMalloc (its working memory is a
fixed 16 MiB static array inside the library).  Checked through the C ABI
against graphic_rotate on two calls in a row, which also shows that the
second call does not depend on what the first left in the shared scratch.

Collected last on purpose (file name), so that a run stopping at the first
failure has run every other test before this one.
"""
import ctypes

import numpy as np
import pytest

from paper_1510_04331_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def _noalloc(lib, x, theta, out):
    th = np.ascontiguousarray(theta, dtype=np.float64)
    s = torch.cuda.current_stream().cuda_stream
    return lib.graphic_rotate_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      x.shape[0], x.shape[1], th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      ctypes.c_void_p(s))


def test_rotate_noalloc_matches_rotate_on_two_calls():
    from paper_1510_04331_gb300 import graphic
    lib = graphic.lib()
    rng = np.random.default_rng(5)
    # call 1: n = 256, 40 frames (two chunks of the static scratch)
    a = torch.from_numpy(synth.random_frames(40, 256, seed=11)).cuda()
    th_a = rng.uniform(-180, 180, 40)
    th_a[:4] = [0.0, 90.0, 45.0, -11.3]
    # call 2: n = 64, 600 frames (the plan array holds 512: a ragged second chunk)
    b = torch.from_numpy(synth.random_frames(600, 64, seed=12)).cuda()
    th_b = rng.uniform(-180, 180, 600)
    ref_a = graphic.graphic_rotate(a, th_a).cpu().numpy()
    ref_b = graphic.graphic_rotate(b, th_b).cpu().numpy()

    out_a = torch.full_like(a, float("nan"))
    out_b = torch.full_like(b, float("nan"))
    assert _noalloc(lib, a, th_a, out_a) == 0, lib.graphic_last_error()
    assert _noalloc(lib, b, th_b, out_b) == 0, lib.graphic_last_error()
    torch.cuda.synchronize()
    got_a, got_b = out_a.cpu().numpy(), out_b.cpu().numpy()
    assert np.abs(got_a - ref_a).max() <= TOL * np.abs(a.cpu().numpy()).max()
    assert np.abs(got_b - ref_b).max() <= TOL * np.abs(b.cpu().numpy()).max()

    # sizes beyond what it supports are refused with a message, not computed
    c = torch.zeros((2, 96, 96), device="cuda")
    assert _noalloc(lib, c, [1.0, 2.0], c) == -2
    assert b"n must be" in lib.graphic_last_error()
