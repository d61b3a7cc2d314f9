"""Uneven batches (cubes of different sizes and frame counts): the persistent
single-launch executor, the grouped executor and the per-cube mode all equal
graphic_shift then graphic_rotate cube by cube (bit-identical: the same line
arithmetic), one-step items (shift only, rotation only) equal the one-step
calls, and the autotuner's schedule round-trips through its cache file."""
import json
import os

import numpy as np
import pytest

from paper_1510_04331_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PER_CUBE, PERSISTENT, GROUPED = 0, 1, 2


@pytest.fixture(scope="module")
def g():
    from paper_1510_04331_gb300 import graphic
    return graphic


@pytest.fixture(scope="module")
def batch():
    return synth.uneven_batch(seed=3, n_cubes=14, sides=(64, 128, 256, 512, 1024), t_range=(1, 9))


def _args(batch):
    return [b[1] for b in batch], [b[2] for b in batch], [b[3] for b in batch]


def _reference(g, batch, variant_1024=0, passes=None):
    """graphic_shift then graphic_rotate cube by cube (or the one step that
    passes[i] names).  variant_1024 = 0: the generic radix-16 kernel for
    1024-point lines, the one the persistent executor runs, so that the
    comparison can be bit-exact."""
    ctx = g.Context(0)
    ctx.set_schedule(variant_1024=variant_1024)
    out = []
    for i, (cube, dx, dy, th) in enumerate(batch):
        ps = 3 if passes is None or passes[i] == 0 else passes[i]
        c = torch.from_numpy(cube).cuda()
        if ps & 1:
            c = ctx.graphic_shift(c, dx, dy)
        if ps & 2:
            c = ctx.graphic_rotate(c, th)
        out.append(c.cpu().numpy())
    ctx.close()
    return out


@pytest.mark.parametrize("mode", [PER_CUBE, PERSISTENT, GROUPED])
def test_batch_modes_equal_per_call_passes(g, batch, mode):
    ctx = g.Context(0)
    ctx.set_schedule(variant_1024=0)
    ref = _reference(g, batch)
    cubes = [torch.from_numpy(c).cuda() for c, _, _, _ in batch]
    for rep in range(2):   # the second call replays the recorded graph
        outs = ctx.graphic_batch_geom(cubes, *_args(batch), mode=mode)
        for o, r in zip(outs, ref):
            assert np.array_equal(o.cpu().numpy(), r)
    ctx.close()


@pytest.mark.parametrize("mode", [PERSISTENT, GROUPED])
def test_batch_matches_default_kernels_within_tolerance(g, batch, mode):
    """Against the default schedule (radix-32 warp kernel for 1024-point
    lines): equal within 1e-5 of each cube's peak; the grouped executor runs
    the same kernels and stays bit-exact."""
    ref = _reference(g, batch, variant_1024=1)
    cubes = [torch.from_numpy(c).cuda() for c, _, _, _ in batch]
    ctx = g.Context(0)
    outs = ctx.graphic_batch_geom(cubes, *_args(batch), mode=mode)
    for o, r, b in zip(outs, ref, batch):
        if mode == GROUPED:
            assert np.array_equal(o.cpu().numpy(), r)
        else:
            assert np.abs(o.cpu().numpy() - r).max() <= 1e-5 * np.abs(b[0]).max()
    ctx.close()


@pytest.mark.parametrize("mode", [PER_CUBE, PERSISTENT, GROUPED])
def test_batch_one_step_items(g, batch, mode):
    """Shift-only, rotation-only and two-step items mixed in one batch (the
    serving loop's stages); a rotation-only item's unused shifts may be None
    and a shift-only item's angles too."""
    passes = [(1, 2, 0)[i % 3] for i in range(len(batch))]
    ref = _reference(g, batch, passes=passes)
    ctx = g.Context(0)
    ctx.set_schedule(variant_1024=0)
    cubes = [torch.from_numpy(c).cuda() for c, _, _, _ in batch]
    dx, dy, th = _args(batch)
    dx = [None if p == 2 else v for p, v in zip(passes, dx)]
    dy = [None if p == 2 else v for p, v in zip(passes, dy)]
    th = [None if p == 1 else v for p, v in zip(passes, th)]
    outs = ctx.graphic_batch_geom(cubes, dx, dy, th, mode=mode, passes=passes)
    for o, r in zip(outs, ref):
        assert np.array_equal(o.cpu().numpy(), r)
    ctx.close()


@pytest.mark.parametrize("mode,sched", [(PERSISTENT, dict(batch_budget_mb=9, batch_ctas_per_sm=1)),
                                        (GROUPED, dict(group_budget_mb=5, group_streams=3))])
def test_batch_small_waves_and_in_place(g, batch, mode, sched):
    """Waves far smaller than the batch (the scratch ring cycles many times)
    and in-place cubes."""
    ctx = g.Context(0)
    ctx.set_schedule(variant_1024=0, **sched)
    ref = _reference(g, batch)
    cubes = [torch.from_numpy(c).cuda() for c, _, _, _ in batch]
    ctx.graphic_batch_geom(cubes, *_args(batch), outs=cubes, mode=mode)
    for o, r in zip(cubes, ref):
        assert np.array_equal(o.cpu().numpy(), r)
    ctx.close()


def test_grouped_graph_follows_new_pointers(g, batch):
    """Same layout, other cubes: the recorded graph is replayed with the new
    frame tables (the plan is rewritten every call)."""
    ctx = g.Context(0)
    ctx.set_schedule(variant_1024=0)
    sub = batch[:5]
    ref = _reference(g, sub)
    a = [torch.from_numpy(c).cuda() for c, _, _, _ in sub]
    b = [x.clone() for x in a]
    ctx.graphic_batch_geom(a, *_args(sub), mode=GROUPED)
    outs = ctx.graphic_batch_geom(b, *_args(sub), mode=GROUPED)
    for o, r in zip(outs, ref):
        assert np.array_equal(o.cpu().numpy(), r)
    ctx.close()


def test_autotune_writes_and_reloads_schedule(g, batch, tmp_path):
    path = str(tmp_path / "tune.json")
    ctx = g.Context(0)
    sub = batch[:6]
    cubes = [torch.from_numpy(c).cuda() for c, _, _, _ in sub]
    sched, t_pc, t_ps, t_gr = ctx.graphic_autotune(cubes, *_args(sub), cache_path=path)
    assert t_pc > 0 and t_ps > 0 and t_gr > 0
    assert sched["batch_mode"] == (GROUPED if t_gr <= t_ps else PERSISTENT)
    assert json.load(open(path)) == sched
    ctx.close()
    os.environ["GRAPHIC_TUNE_CACHE"] = path
    try:
        ctx2 = g.Context(0)
        assert ctx2.schedule() == sched
        ctx2.close()
    finally:
        del os.environ["GRAPHIC_TUNE_CACHE"]


def test_batch_rejects_bad_passes_and_modes(g, batch):
    ctx = g.Context(0)
    cubes = [torch.from_numpy(batch[0][0]).cuda()]
    with pytest.raises(g.GraphicError):
        ctx.graphic_batch_geom(cubes, *_args(batch[:1]), passes=[4])
    with pytest.raises(g.GraphicError):
        ctx.graphic_batch_geom(cubes, *_args(batch[:1]), mode=7)
    with pytest.raises(g.GraphicError):
        ctx.set_schedule(group_streams=9)
    ctx.close()


# --------------------------------------------------------------------------
# Every executor and schedule against the FP64 oracle (shift, Sect. 3.3.1,
# then the three-shear rotation, Sect. 3.4), not only against the library's
# own per-call passes.
# --------------------------------------------------------------------------

def _oracle_batch():
    """Cubes of every supported side, one of 40 frames, with the angles of
    each cube spread over the four quarter turns (theta = 90 q + theta',
    q = 0..3) where its frame count allows, and all four present at every
    side taken together with the other cubes of that side."""
    rng = np.random.default_rng(2024)
    spec = [(64, 40), (128, 6), (256, 4), (512, 3), (1024, 2), (1024, 2), (512, 2), (64, 5)]
    out = []
    for k, (n, T) in enumerate(spec):
        cube = synth.random_frames(T, n, seed=100 + k)
        cube += synth.random_frames(T, n, seed=200 + k, smooth=True) * 50.0
        dx = rng.uniform(-2, 2, T)
        dy = rng.uniform(-2, 2, T)
        q = (np.arange(T) + 2 * (k % 2)) % 4              # quarter turns cycling 0..3
        th = 90.0 * q + rng.uniform(-44.9, 44.9, T)
        out.append((cube.astype(np.float32), dx, dy, th))
    return out


@pytest.fixture(scope="module")
def oracle_batch():
    import oracle
    b = _oracle_batch()
    ref = [oracle.rotate(oracle.shift(c.astype(np.float64), dx, dy), th) for c, dx, dy, th in b]
    return b, ref


def test_oracle_batch_covers_sizes_and_quarter_turns():
    b = _oracle_batch()
    sides = {c.shape[1] for c, _, _, _ in b}
    assert sides == {64, 128, 256, 512, 1024}
    assert max(c.shape[0] for c, _, _, _ in b) >= 32
    for n in sides:
        qs = set()
        for c, _, _, th in b:
            if c.shape[1] == n:
                qs |= {int(np.floor(t / 90.0 + 0.5)) % 4 for t in th}
        assert qs == {0, 1, 2, 3}, (n, qs)


@pytest.mark.parametrize("variant_1024", [0, 1])
@pytest.mark.parametrize("mode", [PER_CUBE, PERSISTENT, GROUPED])
def test_batch_executors_match_fp64_oracle(g, oracle_batch, mode, variant_1024):
    """Each executor (per-cube, persistent single launch, grouped graph) under
    both 1024-point line kernels (generic radix-16, radix-32 warp kernel)
    equals oracle.shift then oracle.rotate within 1e-5 of each cube's input
    peak, element by element, on two calls in a row (the second replays the
    recorded graph)."""
    b, ref = oracle_batch
    ctx = g.Context(0)
    ctx.set_schedule(variant_1024=variant_1024)
    cubes = [torch.from_numpy(c).cuda() for c, _, _, _ in b]
    for rep in range(2):
        outs = ctx.graphic_batch_geom(cubes, *_args(b), mode=mode)
        for o, r, (c, _, _, _) in zip(outs, ref, b):
            err = np.abs(o.cpu().numpy().astype(np.float64) - r).max()
            assert err <= 1e-5 * np.abs(c).max(), (c.shape, err / np.abs(c).max())
    ctx.close()


@pytest.mark.parametrize("variant_1024", [0, 1])
def test_per_call_1024_kernels_match_fp64_oracle(g, oracle_batch, variant_1024):
    """graphic_shift and graphic_rotate on 1024 x 1024 frames, each step
    against its own oracle step, with either 1024-point line kernel."""
    import oracle
    b, _ = oracle_batch
    ctx = g.Context(0)
    ctx.set_schedule(variant_1024=variant_1024)
    for c, dx, dy, th in b:
        if c.shape[1] not in (512, 1024):
            continue
        s = ctx.graphic_shift(torch.from_numpy(c).cuda(), dx, dy)
        ref_s = oracle.shift(c.astype(np.float64), dx, dy)
        assert np.abs(s.cpu().numpy() - ref_s).max() <= 1e-5 * np.abs(c).max()
        s32 = s.cpu().numpy()
        r = ctx.graphic_rotate(s, th)
        ref_r = oracle.rotate(s32.astype(np.float64), th)
        assert np.abs(r.cpu().numpy() - ref_r).max() <= 1e-5 * np.abs(s32).max()
    ctx.close()
