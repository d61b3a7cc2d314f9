"""Serving loop (include/graphic_serve.h): each request's result is the same
alone and in a mix of concurrent requests of different sizes -- bit-identical
to graphic_reduce, since the batched stages run the same per-frame
arithmetic -- and matches the FP64 oracle within 1e-5 of the cube's peak;
admission respects the device budget; a bad request fails alone."""
import threading

import numpy as np
import pytest

import oracle
from paper_1510_04331_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def g():
    from paper_1510_04331_gb300 import graphic
    return graphic


@pytest.fixture(scope="module")
def mix():
    """Ten requests: sides 64-512, 9-40 frames, alt-az angles resampled to
    each frame count, shifts within half a pixel."""
    shapes = [(64, 9), (128, 24), (256, 16), (64, 40), (512, 12), (128, 11), (256, 30), (64, 17), (128, 33),
              (512, 10)]
    out = []
    for i, (n, T) in enumerate(shapes):
        d = synth.make_cube(T, n, seed=100 + i, parang=synth.altaz_parang(T), edges=synth.default_edges(n))
        out.append(d)
    return out


@pytest.fixture(scope="module")
def reference(g, mix):
    ctx = g.Context(0)
    ref = [ctx.graphic_reduce_host(d.cube, d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges) for d in mix]
    ctx.close()
    return ref


def _submit(srv, d):
    return srv.submit(d.cube, d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges)


def test_serve_alone_equals_reduce(g, mix, reference):
    with g.Server(0) as srv:
        for d, r in zip(mix, reference):
            out, info = srv.wait(_submit(srv, d))
            assert info["status"] == 0, info
            assert np.array_equal(out, r)
            assert info["t_submit"] <= info["t_admit"] <= info["t_done"]


@pytest.mark.parametrize("mode", [1, 2])
def test_serve_mix_equals_alone(g, mix, reference, mode):
    """All requests submitted at once, so that their stages share batches;
    the persistent batch mode runs the generic kernel on 1024-point lines:
    within tolerance there, bit-identical with the grouped mode."""
    with g.Server(0, batch_mode=mode) as srv:
        ids = [_submit(srv, d) for d in mix]
        res = [srv.wait(i) for i in ids]
        st = srv.stats()
    for (out, info), r, d in zip(res, reference, mix):
        assert info["status"] == 0, info
        if mode == 2:
            assert np.array_equal(out, r)
        else:
            assert np.abs(out - r).max() <= TOL * np.abs(d.cube).max()
    assert st["completed"] == len(mix) and st["failed"] == 0
    # batching across requests happened: more request stages than batch calls
    assert st["batch_items"] > st["batch_launches"]
    assert st["max_batch_items"] >= 2


def test_serve_matches_fp64_oracle(g, mix):
    d = mix[0]
    with g.Server(0) as srv:
        ids = [_submit(srv, x) for x in mix[:4]]
        out, info = [srv.wait(i) for i in ids][0]
    ref = oracle.reduce(d.cube.astype(np.float64), d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges)
    assert np.abs(out - ref).max() <= TOL * np.abs(d.cube).max()


def test_serve_admission_under_a_small_budget(g, mix, reference):
    """A budget that holds the largest request but not two of them: requests
    wait for memory, all complete, and the arena never exceeds its size; a
    request that can never fit fails alone with GRAPHIC_ERR_OOM."""
    big = max(d.cube.nbytes for d in mix)
    budget = big + (4 << 20)
    huge = synth.make_cube(40, 512, seed=7, parang=synth.altaz_parang(40), edges=synth.default_edges(512),
                           noise=False)
    with g.Server(0, max_device_bytes=budget) as srv:
        ids = [_submit(srv, d) for d in mix]
        bad = _submit(srv, huge)
        res = [srv.wait(i) for i in ids]
        _, binfo = srv.wait(bad)
        st = srv.stats()
    for (out, info), r in zip(res, reference):
        assert info["status"] == 0, info
        assert np.array_equal(out, r)
    assert binfo["status"] == -3
    assert st["device_bytes_peak"] <= st["device_bytes_cap"] <= budget
    assert st["failed"] == 1


def test_serve_nonfinite_request_fails_alone(g, mix, reference):
    bad = synth.make_cube(12, 128, seed=9, parang=synth.altaz_parang(12), edges=synth.default_edges(128))
    bad.cube[3, 60, 61] = np.nan
    with g.Server(0) as srv:
        ids = [_submit(srv, d) for d in mix[:5]]
        bid = _submit(srv, bad)
        res = [srv.wait(i) for i in ids]
        _, binfo = srv.wait(bid)
    assert binfo["status"] == -5
    for (out, info), r in zip(res, reference[:5]):
        assert info["status"] == 0
        assert np.array_equal(out, r)


def test_serve_concurrent_clients(g, mix, reference):
    """Four client threads submit and wait on their own requests."""
    results = {}

    def client(k, srv):
        for i in range(k, len(mix), 4):
            out, info = srv.wait(_submit(srv, mix[i]))
            results[i] = (out, info)

    with g.Server(0, max_active=3) as srv:
        th = [threading.Thread(target=client, args=(k, srv)) for k in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        st = srv.stats()
    assert sorted(results) == list(range(len(mix)))
    for i, r in enumerate(reference):
        assert results[i][1]["status"] == 0
        assert np.array_equal(results[i][0], r)
    assert st["max_resident"] <= 3


def test_serve_rejects_bad_requests(g, mix):
    d = mix[0]
    with g.Server(0) as srv:
        with pytest.raises(g.GraphicError):
            srv.submit(d.cube, d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, [8.0, 4.0])   # edges must increase
        with pytest.raises(g.GraphicError):
            srv.submit(d.cube[:, :, :60].copy(), d.dx, d.dy, d.parang, d.fwhm, d.n_fwhm, d.edges)
        with pytest.raises(g.GraphicError):
            srv.wait(12345)
