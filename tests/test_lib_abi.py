"""CPU-side checks of the CUDA library: it builds for sm_103a, loads, exports
every function include/mtssph.h declares, and rejects bad arguments before
touching the GPU.  No compute call runs here."""
import ctypes as C
import re

import pytest

from paper_2309_04010_gb300 import mtssph as M


def test_library_builds_and_exports_every_header_symbol():
    L = M.lib()
    names = M.header_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(L, n)]
    assert missing == []
    assert L.mts_version() >= 100


def test_binding_covers_every_header_function():
    src = open(M.__file__).read()
    for name in M.header_functions():
        assert re.search(rf'"{name}"', src), name


def test_null_arguments_are_rejected_without_gpu_work():
    L = M.lib()
    assert L.mts_body_create(None, None, None) == M.ERR_INVALID_ARG
    assert b"NULL" in L.mts_last_error()
    assert L.mts_advance_slow_step(None, None, None) == M.ERR_INVALID_ARG
    assert L.mts_read_field(None, 0, None, 0) == M.ERR_INVALID_ARG
    assert L.mts_set_damping(None, 1.0) == M.ERR_INVALID_ARG
    assert L.mts_ctx_create(0, None, None, None) == M.ERR_INVALID_ARG


def test_allocator_hook_is_validated():
    L = M.lib()
    bad = M.Allocator()          # NULL function pointers
    out = C.c_void_p()
    st = L.mts_ctx_create(0, None, C.byref(bad), C.byref(out))
    assert st in (M.ERR_INVALID_ARG, M.ERR_CUDA)   # no device here -> CUDA error first


def test_struct_layouts_match_header():
    assert C.sizeof(M.StepParams) == 5 * 8 + 8 + 4 * 4
    assert C.sizeof(M.StepReport) == 8 + 4 + 4 + 4 * 8 + 6 * 8 + 8 + 8 + 8
    assert C.sizeof(M.BodyDesc) == 4 + 4 + 8 + 8 + 8 + 8 + 4 + 4 + 3 * 8
