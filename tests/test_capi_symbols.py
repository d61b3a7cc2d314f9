"""The C-ABI library builds, loads without a GPU and exports every function
declared in include/graphic.h; the host-side argument checks answer before
any device work.  CPU only (no compute call needs a GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "graphic.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(graphic_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1510_04331_gb300 import build
    build.build()
    from paper_1510_04331_gb300 import graphic
    return graphic.lib()


def test_header_declares_the_path():
    names = declared_functions()
    for required in ["graphic_shift", "graphic_rotate", "graphic_adi_subtract", "graphic_collapse_median",
                     "graphic_reduce", "graphic_reduce_host", "graphic_create", "graphic_destroy"]:
        assert required in names


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
