"""Strided cubes (graphic_cube, frame_stride > n*n): every step and the
whole reduction through the *_cube calls equal the dense calls bit for bit
(the same kernels, only the frame addresses differ), the reduction equals the
FP64 oracle within 1e-5 of the input peak, and the floats between frames are
neither read nor written."""
import numpy as np
import pytest

import oracle
from paper_1510_04331_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PAD_IN, PAD_WORK = 64, 36     # extra floats after every frame (multiples of 4)
SENTINEL = 12345.0


@pytest.fixture(scope="module")
def g():
    from paper_1510_04331_gb300 import graphic
    return graphic


def strided(x, pad):
    """A (T, n, n) view with frame stride n*n + pad into a larger buffer whose
    gaps hold SENTINEL; returns (view, buffer)."""
    T, n, _ = x.shape
    buf = torch.full((T, n * n + pad), SENTINEL, dtype=torch.float32, device="cuda")
    v = buf[:, :n * n].view(T, n, n)
    v.copy_(x)
    return v, buf


def gaps_untouched(buf, n):
    return bool((buf[:, n * n:] == SENTINEL).all().item())


def test_strided_steps_equal_dense_calls(g):
    d = synth.small_cube(seed=0)
    T, n = d.cube.shape[0], d.cube.shape[1]
    x = torch.from_numpy(d.cube).cuda()
    ctx = g.Context(0)
    xi, bi = strided(x, PAD_IN)
    xo, bo = strided(torch.zeros_like(x), PAD_WORK)
    ctx.graphic_shift_cube(xi, d.dx, d.dy, xo)
    assert torch.equal(xo, ctx.graphic_shift(x, d.dx, d.dy))
    ctx.graphic_rotate_cube(xi, -d.parang, xo)
    assert torch.equal(xo, ctx.graphic_rotate(x, -d.parang))
    ctx.graphic_adi_subtract_cube(xi, d.parang, d.fwhm, d.n_fwhm, d.edges, xo)
    assert torch.equal(xo, ctx.graphic_adi_subtract(x, d.parang, d.fwhm, d.n_fwhm, d.edges))
    assert torch.equal(ctx.graphic_collapse_median_cube(xi), ctx.graphic_collapse_median(x))
    # in place on a strided cube
    xw, bw = strided(x, PAD_WORK)
    ctx.graphic_shift_cube(xw, d.dx, d.dy, xw)
    assert torch.equal(xw, ctx.graphic_shift(x, d.dx, d.dy))
    assert torch.equal(xi, x)
    for b in (bi, bo, bw):
        assert gaps_untouched(b, n)
    ctx.close()


@pytest.mark.parametrize("n,T", [(128, 40), (512, 24)])
def test_strided_reduce_matches_dense_and_fp64_oracle(g, n, T):
    d = synth.make_cube(T, n, seed=5, parang=synth.altaz_parang(T), edges=synth.default_edges(n))
    x = torch.from_numpy(d.cube).cuda()
    ctx = g.Context(0)
    xi, bi = strided(x, PAD_IN)
    xw, bw = strided(torch.zeros_like(x), PAD_WORK)
    img = ctx.graphic_reduce_cube(xi, d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges, xw)
    dense = ctx.graphic_reduce(x, d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges)
    assert torch.equal(img, dense)
    ref = oracle.reduce(d.cube.astype(np.float64), d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges)
    assert np.abs(img.cpu().numpy().astype(np.float64) - ref).max() <= 1e-5 * np.abs(d.cube).max()
    assert torch.equal(xi, x) and gaps_untouched(bi, n) and gaps_untouched(bw, n)
    ctx.close()


def test_strided_rejects_bad_strides(g):
    ctx = g.Context(0)
    buf = torch.zeros((3, 64 * 64 + 2), device="cuda")
    v = buf[:, :64 * 64].view(3, 64, 64)     # stride not a multiple of 4
    with pytest.raises(g.GraphicError):
        ctx.graphic_shift_cube(v, [0.0] * 3, [0.0] * 3, v)
    ctx.close()
