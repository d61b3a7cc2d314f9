"""The C-ABI library builds, loads without a GPU and exports every function
declared in include/*.h; the host-side argument checks answer before any
device work; the binding's ctypes structures have the C layout.  CPU only
(no compute call needs a GPU here)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def declared_functions():
    names = set()
    for h in HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(graphic_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1510_04331_gb300 import build
    build.build()
    from paper_1510_04331_gb300 import graphic
    return graphic.lib()


def test_header_declares_the_path():
    names = declared_functions()
    for required in ["graphic_shift", "graphic_rotate", "graphic_adi_subtract", "graphic_collapse_median",
                     "graphic_reduce", "graphic_reduce_host", "graphic_create", "graphic_destroy",
                     "graphic_shift_cube", "graphic_rotate_cube", "graphic_adi_subtract_cube",
                     "graphic_collapse_median_cube", "graphic_reduce_cube"]:
        assert required in names


def test_strided_cube_calls_check_their_descriptions_without_gpu(lib):
    """graphic_cube arguments: null descriptions and bad frame strides (below
    n*n, or not a multiple of 4 floats) are refused on the host."""
    from paper_1510_04331_gb300 import graphic
    import ctypes as ct
    ctx = ct.c_void_p(1)   # never dereferenced: the description checks come first
    good = graphic.Cube(256, 3, 64, 0, 64 * 64 + 16)
    for stride in (64 * 64 - 4, 64 * 64 + 2):
        bad = graphic.Cube(256, 3, 64, 0, stride)
        assert lib.graphic_shift_cube(ctx, ct.byref(bad), ct.byref(good), None, None) == -1
        assert b"frame_stride" in lib.graphic_last_error()
        assert lib.graphic_collapse_median_cube(ctx, ct.byref(bad), ct.c_void_p(256)) == -1
    other = graphic.Cube(256, 4, 64, 0, 0)
    assert lib.graphic_rotate_cube(ctx, ct.byref(good), ct.byref(other), None) == -1
    assert b"differ" in lib.graphic_last_error()
    assert lib.graphic_reduce_cube(ctx, None, ct.byref(good), None, None, None, 4.0, 1.5, None, 2, None) == -1


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_checks_without_gpu(lib):
    from paper_1510_04331_gb300 import graphic
    assert lib.graphic_version() >= 10000
    # null context is rejected before any CUDA call
    rc = lib.graphic_shift(None, None, None, 1, 64, None, None)
    assert rc == -1
    assert b"ctx" in lib.graphic_last_error()
    assert lib.graphic_kernel_name(0) == b"shift_x"
    assert lib.graphic_kernel_name(99) is None
    assert graphic.KERNELS == [lib.graphic_kernel_name(k).decode() for k in range(len(graphic.KERNELS))]


def test_new_calls_reject_a_null_context_without_gpu(lib):
    """Every call added for the later rows checks its arguments on the host
    before any CUDA call (these run without a GPU)."""
    calls = [
        lambda: lib.graphic_register(None, None, 1, 64, 1.0, 8, 3, 400, 6, None, None),
        lambda: lib.graphic_bin_median(None, None, None, 10, 64, 5),
        lambda: lib.graphic_inject(None, None, 1, 64, None, None, None, 1, None, None, None, None, None, 5),
        lambda: lib.graphic_aperture(None, None, 64, 1, None, None, 3.0, None),
        lambda: lib.graphic_sky_median(None, None, 1, 64, None, None, 0.0, None),
        lambda: lib.graphic_bad_pixel_map(None, None, 64, 5.0, None),
        lambda: lib.graphic_bad_pixel_fix(None, None, 1, 64, None),
    ]
    for call in calls:
        assert call() == -1
        assert b"ctx" in lib.graphic_last_error()


def test_bin_mean_host_helper(lib):
    """Group means of the bin angles / times (host code of the C ABI)."""
    import numpy as np
    from paper_1510_04331_gb300 import graphic
    v = np.random.default_rng(1).uniform(-80, 80, 103)
    for B in (1, 10, 50, 103, 200):
        want = np.array([v[g:g + B].mean() for g in range(0, 103, B)])
        assert np.allclose(graphic.bin_mean(v, B), want, rtol=0, atol=1e-12)
    assert np.array_equal(graphic.bin_mean(v, 1), v)
    with pytest.raises(graphic.GraphicError):
        graphic.bin_mean(v, 0)


def test_server_host_side_checks_without_gpu(lib):
    assert lib.graphic_server_create(None, None) == -1
    assert lib.graphic_server_submit(None, None, None) == -1
    assert lib.graphic_server_wait(None, 1, 0.0, None) == -1
    assert lib.graphic_server_stats_read(None, None) == -1
    assert lib.graphic_server_destroy(None) == 0
    assert lib.graphic_server_clock(None) == 0.0


def test_binding_structures_match_the_c_layout(tmp_path):
    """sizeof and field offsets of every struct the binding mirrors, from a
    C program compiled against the headers."""
    from paper_1510_04331_gb300 import graphic
    structs = {"graphic_batch_item": graphic.BatchItem, "graphic_server_config": graphic.ServerConfig,
               "graphic_request": graphic.Request, "graphic_request_info": graphic.RequestInfo,
               "graphic_server_stats": graphic.ServerStats, "graphic_cube": graphic.Cube}
    c_names = {"in_": "in"}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "graphic_serve.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {c_names.get(f, f)}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)


def test_binding_rejects_host_tensors_for_the_new_calls():
    """The Python binding refuses tensors that are not contiguous CUDA
    float32 cubes / images before reaching the library (no GPU needed)."""
    torch = pytest.importorskip("torch")
    from paper_1510_04331_gb300 import graphic
    ctx = graphic.Context.__new__(graphic.Context)   # no device context: the checks come first
    cube = torch.zeros((2, 64, 64))
    for call in (lambda: graphic.Context.graphic_register(ctx, cube, 1.0, 8, 3, 400, 6),
                 lambda: graphic.Context.graphic_bin_median(ctx, cube, 2),
                 lambda: graphic.Context.graphic_inject(ctx, cube, [0, 0], [32, 32], [32, 32], [5.0], [0.0], [1.0],
                                                        [2.0, 2.0], [3.0, 3.0], 4),
                 lambda: graphic.Context.graphic_aperture(ctx, cube[0], [1.0], [1.0], 2.0)):
        with pytest.raises(graphic.GraphicError):
            call()
