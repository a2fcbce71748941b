"""CPU-side checks of the C ABI: the header is valid C, the library loads and
exports every declared entry point, the ctypes mirrors match the C layouts,
and host-side argument checking works without a GPU."""
import ctypes as C
import os
import subprocess
import tempfile

import pytest

from paper_2412_12734_gb300 import _lib as L
from paper_2412_12734_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def test_every_declared_symbol_is_exported(lib):
    names = L.declared_symbols()
    assert {"gb_render_forward", "gb_render_backward", "gb_context_create"} <= set(names)
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_header_is_c_and_layouts_match():
    """Compiles a C program against include/gbill.h and compares sizeof /
    offsetof with the ctypes mirrors used by the Python binding."""
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "gbill.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(gb_camera), sizeof(gb_scene), sizeof(gb_grads),
         sizeof(gb_options), sizeof(gb_stats), offsetof(gb_scene, sigma));
  printf("%zu %zu %zu %zu\n", offsetof(gb_camera, world_to_cam), offsetof(gb_camera, scene),
         offsetof(gb_options, background), offsetof(gb_options, batch_depth_fwd));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(src, "w").write(prog)
        subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                               src, "-o", exe])
        lines = subprocess.check_output([exe], text=True).split("\n")
    a = [int(x) for x in lines[0].split()]
    b = [int(x) for x in lines[1].split()]
    assert a == [C.sizeof(L.gb_camera), C.sizeof(L.gb_scene), C.sizeof(L.gb_grads),
                 C.sizeof(L.gb_options), C.sizeof(L.gb_stats), L.gb_scene.sigma.offset]
    assert b == [L.gb_camera.world_to_cam.offset, L.gb_camera.scene.offset, L.gb_options.background.offset,
                 L.gb_options.batch_depth_fwd.offset]


def test_status_strings_and_null_arguments(lib):
    for code, name in L.STATUS.items():
        assert lib.gb_status_string(code).decode() == name
    assert lib.gb_context_create(0, None) == 1  # GB_ERR_INVALID_ARG
    assert lib.gb_context_destroy(None) == 0
    assert lib.gb_saved_destroy(None) == 0
    assert lib.gb_last_error(None).decode() == "null context"
    assert lib.gb_render_forward(None, None, None, 0, None, 0, None, None, None, None, None) == 1


def test_every_entry_point_rejects_null_handles(lib):
    """Every call that takes a context or a saved state returns
    GB_ERR_INVALID_ARG for a null one, before any CUDA call: all arguments
    null or zero."""
    import ctypes as C
    skip = {"gb_context_create", "gb_context_destroy", "gb_saved_destroy", "gb_last_error", "gb_status_string",
            "gb_kernel_launches"}
    names = [n for n in L.signatures() if n not in skip]
    assert len(names) >= 15
    for n in names:
        f = getattr(lib, n)
        args = [0 if t in (C.c_int, C.c_int32, C.c_int64, C.c_long, C.c_uint32) else None for t in f.argtypes]
        assert f(*args) == 1, n


def test_context_on_missing_device_reports_cuda_error(lib):
    """Device index far beyond any machine's count: GB_ERR_CUDA, no crash."""
    h = C.c_void_p()
    assert lib.gb_context_create(4096, C.byref(h)) == 3
    assert not h.value
