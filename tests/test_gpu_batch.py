"""Uneven batches (cubes of different sizes and frame counts): the persistent
single-launch executor and the per-cube mode both equal graphic_shift then
graphic_rotate cube by cube (bit-identical: the same line arithmetic), and
the autotuner's schedule round-trips through its cache file."""
import json
import os

import numpy as np
import pytest

from paper_1510_04331_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_1510_04331_gb300 import graphic
    return graphic


@pytest.fixture(scope="module")
def batch():
    return synth.uneven_batch(seed=3, n_cubes=14, sides=(64, 128, 256, 512, 1024), t_range=(1, 9))


def _reference(g, batch, variant_1024=0):
    """graphic_shift then graphic_rotate cube by cube.  variant_1024 = 0: the
    generic radix-16 kernel for 1024-point lines, the one the persistent
    executor runs, so that the comparison can be bit-exact."""
    ctx = g.Context(0)
    ctx.set_schedule(variant_1024=variant_1024)
    out = []
    for cube, dx, dy, th in batch:
        c = torch.from_numpy(cube).cuda()
        out.append(ctx.graphic_rotate(ctx.graphic_shift(c, dx, dy), th).cpu().numpy())
    ctx.close()
    return out


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_modes_equal_per_call_passes(g, batch, mode):
    ctx = g.Context(0)
    ctx.set_schedule(variant_1024=0)
    ref = _reference(g, batch)
    cubes = [torch.from_numpy(c).cuda() for c, _, _, _ in batch]
    for rep in range(2):   # the second persistent call replays the recorded graph
        outs = ctx.graphic_batch_geom(cubes, [b[1] for b in batch], [b[2] for b in batch], [b[3] for b in batch],
                                      mode=mode)
        for o, r in zip(outs, ref):
            assert np.array_equal(o.cpu().numpy(), r)
    ctx.close()


def test_batch_persistent_matches_default_kernels_within_tolerance(g, batch):
    """Against the default schedule (radix-32 warp kernel for 1024-point
    lines): equal within 1e-5 of each cube's peak."""
    ref = _reference(g, batch, variant_1024=1)
    cubes = [torch.from_numpy(c).cuda() for c, _, _, _ in batch]
    outs = g.context().graphic_batch_geom(cubes, [b[1] for b in batch], [b[2] for b in batch],
                                          [b[3] for b in batch], mode=1)
    for o, r, b in zip(outs, ref, batch):
        assert np.abs(o.cpu().numpy() - r).max() <= 1e-5 * np.abs(b[0]).max()


def test_batch_persistent_small_waves_and_in_place(g, batch):
    """Waves far smaller than the batch (the scratch ring alternates many
    times) and in-place cubes."""
    ctx = g.Context(0)
    ctx.set_schedule(batch_budget_mb=9, batch_ctas_per_sm=1)
    ref = _reference(g, batch)
    cubes = [torch.from_numpy(c).cuda() for c, _, _, _ in batch]
    ctx.graphic_batch_geom(cubes, [b[1] for b in batch], [b[2] for b in batch], [b[3] for b in batch],
                           outs=cubes, mode=1)
    for o, r in zip(cubes, ref):
        assert np.array_equal(o.cpu().numpy(), r)
    ctx.close()


def test_autotune_writes_and_reloads_schedule(g, batch, tmp_path):
    path = str(tmp_path / "tune.json")
    ctx = g.Context(0)
    cubes = [torch.from_numpy(c).cuda() for c, _, _, _ in batch[:6]]
    sched, t_pc, t_ps = ctx.graphic_autotune(cubes, [b[1] for b in batch[:6]], [b[2] for b in batch[:6]],
                                             [b[3] for b in batch[:6]], cache_path=path)
    assert t_pc > 0 and t_ps > 0
    assert json.load(open(path)) == sched
    ctx.close()
    os.environ["GRAPHIC_TUNE_CACHE"] = path
    try:
        ctx2 = g.Context(0)
        assert ctx2.schedule() == sched
        ctx2.close()
    finally:
        del os.environ["GRAPHIC_TUNE_CACHE"]
