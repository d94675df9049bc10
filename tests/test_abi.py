"""The C ABI library builds, loads, and exports every function include/shmemg.h
declares (no GPU needed: nothing is called that touches a device)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "shmemg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(shmemg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2607_08006_gb300.builder import build

    return build()


def test_exports_every_declared_function(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (shmemg_[a-z0-9_]+)", out))
    decl = declared_functions()
    assert len(decl) > 60
    missing = [f for f in decl if f not in exported]
    assert not missing, missing


def test_library_loads_and_reports_errors_without_a_device(libpath):
    import ctypes as C

    import paper_2607_08006_gb300 as sg

    L = sg.lib()
    assert L.shmemg_strerror(sg.ERR_NOT_SYMMETRIC).decode().startswith("pointer")
    out = C.c_uint64(0)
    assert L.shmemg_required_heap_bytes(4, 1 << 20, C.byref(out)) == 0
    assert out.value == sg.RESERVED_BYTES + 4 * (1 << 20)
    assert L.shmemg_required_heap_bytes(4, 1000, C.byref(out)) == sg.ERR_INVALID_ARG   # H not a multiple of 256
    v = C.c_int(7)
    assert L.shmemg_initialized(C.byref(v)) == 0 and v.value == 0
    assert L.shmemg_malloc(64, C.byref(C.c_void_p())) == sg.ERR_NOT_INITIALIZED
    assert L.shmemg_putmem(None, None, 8, 0, 0, None) == sg.ERR_NOT_INITIALIZED


def test_record_layouts_agree():
    """The 64-byte op and request records: generator, binding and header agree."""
    import numpy as np

    import paper_2607_08006_gb300 as sg
    import workloads as W

    assert W.OP_DTYPE.itemsize == 64 and W.REQ_DTYPE.itemsize == 64
    assert W.REQ_DTYPE == sg.REQ_DTYPE
    import ctypes as C

    assert C.sizeof(sg.Req) == 64 and C.sizeof(sg.Completion) == 40 and C.sizeof(sg.CollDesc) == 48
    hdr = open(os.path.join(ROOT, "include", "shmemg.h")).read()
    for name in ("kind", "dtype", "sub", "team", "pe", "issuer", "dst", "src", "n", "operand", "cond", "aux"):
        assert name in W.OP_DTYPE.names and re.search(r"\b%s;" % name, hdr)
    assert np.dtype(W.OP_DTYPE).fields["aux"][1] == 56


def test_halo_stride_pads_the_side_columns(libpath):
    """Host-only: the halo buffer holds the north and south rows (nx floats each) and the
    west and east columns (ny floats each) padded to a multiple of 4, so each of the four
    parts, and the second buffer of the pair, starts on a 16-byte boundary."""
    import paper_2607_08006_gb300 as sg

    for nx, ny in ((4, 1), (8, 5), (1024, 1024), (2208, 9), (384, 37), (40, 7)):
        hs = sg.halo_stride(nx, ny)
        ny4 = (ny + 3) // 4 * 4
        assert hs == 2 * nx + 2 * ny4
        for part in (0, nx, 2 * nx, 2 * nx + ny4, hs):
            assert part % 4 == 0
        assert 2 * nx + ny4 + ny <= hs   # the east column fits inside the buffer
