"""The C ABI without a GPU: the library loads, exports every declared entry
point, and validates plans (no compute calls)."""
import ctypes
import os

import pytest

from paper_1705_08266_gb300 import build as B
from paper_1705_08266_gb300 import dwt2d as D


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(B.LIB):
        B.build()
    return D.lib()


def test_exports_every_header_function(L):
    names = D.header_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n


def _plan(L, h, w, lv, wav, sch, dt, bnd=0):
    p = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    st = L.dwt2d_plan(ctypes.byref(p), h, w, lv, wav, sch, bnd, dt, ctypes.byref(ws))
    return st, p, ws.value


@pytest.mark.parametrize("args,status", [
    ((0, 8, 1, 0, 1, 0), -1), ((8, 0, 1, 0, 1, 0), -1), ((8, 8, 0, 0, 1, 0), -1),
    ((8, 8, 17, 0, 1, 0), -1), ((70000, 8, 1, 0, 1, 0), -1),
    ((8, 8, 1, 0, 1, 1), -2),   # CDF 9/7 with int32 storage
    ((8, 8, 1, 1, 1, 0), -2),   # LeGall 5/3 with float storage
    ((8, 8, 1, 0, 9, 0), -1),   # unknown scheme
    ((8, 8, 1, 0, 1, 0), 0), ((1, 1, 16, 1, 0, 1), 0), ((7, 9, 3, 0, 5, 0), 0),
])
def test_plan_validation(L, args, status):
    h, w, lv, wav, sch, dt = args
    st, p, ws = _plan(L, h, w, lv, wav, sch, dt)
    assert st == status
    if st == 0:
        assert ws >= 256
        L.dwt2d_plan_destroy(p)


def test_boundary_other_than_symmetric_is_unsupported(L):
    st, _, _ = _plan(L, 8, 8, 1, 0, 1, 0, bnd=1)
    assert st == -2


def test_plan_info_groups(L):
    st, p, ws = _plan(L, 8192, 8192, 5, 0, 2, 0)
    assert st == 0
    n, ng = ctypes.c_int32(), ctypes.c_int32()
    fused = (ctypes.c_int32 * 16)()
    assert L.dwt2d_plan_info(p, ctypes.byref(n), fused, ctypes.byref(ng)) == 0
    assert sum(fused[i] for i in range(ng.value)) == 5
    assert all(1 <= fused[i] <= 3 for i in range(ng.value))
    L.dwt2d_plan_destroy(p)
    # multipass: one launch per lifting step per level
    st, p, ws2 = _plan(L, 8192, 8192, 5, 0, 3, 0)
    assert L.dwt2d_plan_info(p, ctypes.byref(n), None, ctypes.byref(ng)) == 0
    assert n.value == 8 * 5
    assert ws2 > 2 * 8192 * 8192 * 4  # two full-size ping-pong buffers
    L.dwt2d_plan_destroy(p)
    st, p, _ = _plan(L, 8192, 8192, 5, 0, 4, 0)
    assert L.dwt2d_plan_info(p, ctypes.byref(n), None, ctypes.byref(ng)) == 0
    assert n.value == 4 * 5
    L.dwt2d_plan_destroy(p)


def test_bad_pointers_rejected_without_gpu(L):
    st, p, ws = _plan(L, 8, 8, 1, 0, 1, 0)
    vp = ctypes.c_void_p
    # null pointers
    assert L.dwt2d_forward(p, None, 32, vp(16), 32, vp(32), 1.0, None) == -1
    # misaligned pointer / pitch
    assert L.dwt2d_forward(p, vp(8), 32, vp(16), 32, vp(32), 1.0, None) == -3
    assert L.dwt2d_forward(p, vp(16), 36, vp(48), 32, vp(64), 1.0, None) == -3
    # pitch shorter than a row
    assert L.dwt2d_forward(p, vp(16), 16, vp(48), 32, vp(64), 1.0, None) == -1
    # in place
    assert L.dwt2d_forward(p, vp(16), 32, vp(16), 32, vp(64), 1.0, None) == -1
    L.dwt2d_plan_destroy(p)


def test_status_strings(L):
    for s in (0, -1, -2, -3, -4, -5, -6):
        assert L.dwt2d_status_string(s)
