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


def test_rotate_noalloc_matches_fp64_oracle_at_512_and_1024():
    """Against the FP64 oracle's three-shear rotation (Sect. 3.4) on the two
    largest sides, with ragged last chunks of the static scratch: 9 frames of
    512 x 512 (chunks of 8 + 1, the radix-32 warp kernel) and then 5 frames of
    1024 x 1024 (chunks of 2 + 2 + 1), two calls in a row."""
    import oracle
    from paper_1510_04331_gb300 import graphic
    lib = graphic.lib()
    rng = np.random.default_rng(77)
    cases = []
    for T, n, seed in ((9, 512, 21), (5, 1024, 22)):
        f = synth.random_frames(T, n, seed=seed) + 40.0 * synth.random_frames(T, n, seed=seed + 1, smooth=True)
        th = rng.uniform(-180, 180, T)
        th[:4] = [-170.0, -80.0, 11.3, 135.0]              # all four quarter turns
        cases.append((f.astype(np.float32), th))
    outs = []
    for f, th in cases:
        x = torch.from_numpy(f).cuda()
        out = torch.full_like(x, float("nan"))
        assert _noalloc(lib, x, th, out) == 0, lib.graphic_last_error()
        outs.append(out)
    torch.cuda.synchronize()
    for (f, th), out in zip(cases, outs):
        ref = oracle.rotate(f.astype(np.float64), th)
        err = np.abs(out.cpu().numpy().astype(np.float64) - ref).max()
        assert err <= TOL * np.abs(f).max(), (f.shape, err / np.abs(f).max())
