"""The C ABI without a GPU: the library loads, exports every declared entry
point, and validates plans (no compute calls)."""
import ctypes
import os

import pytest
import torch

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
    for s in (0, -1, -2, -3, -4, -5, -6, -7):
        assert L.dwt2d_status_string(s)


def _item(h, w, lv, wav=0, dt=0, inv=0, src=1 << 20, dst=2 << 20, sp=None, dp=None):
    es = 2 if dt in (2, 3) else 4
    pitch = (w * es + 15) // 16 * 16
    return D.BatchItem(h, w, lv, wav, dt, inv, src, sp if sp is not None else pitch, dst,
                       dp if dp is not None else pitch)


def _batch(L, items, scheme=2, tuning=None):
    arr = (D.BatchItem * max(1, len(items)))(*items)
    b = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    t = ctypes.byref(tuning) if tuning is not None else None
    st = L.dwt2d_batch_create(ctypes.byref(b), arr, len(items), scheme, t, ctypes.byref(ws))
    return st, b, ws.value


def test_batch_planning_launch_list(L):
    """Phases x (direction, storage, fusion depth) buckets; placeholder pointers
    (nothing is touched before upload)."""
    items = [_item(64, 64, 3), _item(100, 37, 1), _item(64, 64, 2, wav=1, dt=1),
             _item(64, 64, 3, inv=1), _item(64, 48, 2, dt=2)]
    st, b, ws = _batch(L, items)
    assert st == 0 and ws > 256
    n, w = ctypes.c_int32(), ctypes.c_int64()
    assert L.dwt2d_batch_info(b, ctypes.byref(n), ctypes.byref(w)) == 0
    # phase 0: fwd f32 nl1 (the 1-level item), fwd f32 nl2, fwd i32 nl2, fwd f16 nl2,
    #          inv f32 nl1 (the 3-level inverse runs its 1-level coarse group first)
    # phase 1: fwd f32 nl1 (the 3-level item), inv f32 nl2
    assert n.value == 7
    assert w.value >= len(items)
    L.dwt2d_batch_destroy(b)


@pytest.mark.parametrize("case,status", [
    ("multipass_scheme", -2), ("fuse3", -2), ("same_buffer", -1), ("bad_pitch", -3),
    ("bad_levels", -1), ("int_cdf", -2), ("empty", 0), ("cols4", 0), ("cols3", -1),
    ("cols4_persistent", 0)])
def test_batch_validation(L, case, status):
    items = [_item(64, 64, 2)]
    scheme, tun = 2, None
    if case == "multipass_scheme":
        scheme = 3
    elif case == "fuse3":
        tun = D.Tuning(0, 3, 0, 0)
    elif case == "same_buffer":
        items = [_item(64, 64, 2, dst=1 << 20)]
    elif case == "bad_pitch":
        items = [_item(64, 64, 2, sp=264)]
    elif case == "bad_levels":
        items = [_item(64, 64, 0)]
    elif case == "int_cdf":
        items = [_item(64, 64, 2, wav=0, dt=1)]
    elif case == "empty":
        items = []
    elif case.startswith("cols"):
        tun = D.Tuning(cols_per_lane=int(case[4]), persistent=int(case.endswith("persistent")))
    st, b, ws = _batch(L, items, scheme, tun)
    assert st == status
    if st == 0:
        L.dwt2d_batch_destroy(b)


@pytest.mark.parametrize("opts,status", [
    ({}, 0), ({"fuse_first": 3, "fuse_max": 3}, 0), ({"fwd_cols_per_lane": 4}, 0),
    ({"programmatic_launch": -1, "host_pipeline": -1, "inv_seg_interleave": -1}, 0),
    ({"fwd_warps_per_sm_large": -1, "host_bands": 64}, 0),
    ({"fuse_first": 4}, -1), ({"fuse_max": -2}, -1), ({"fwd_cols_per_lane": 3}, -1),
    ({"programmatic_launch": 2}, -1), ({"host_bands": 65}, -1), ({"min_segment": -1}, -1),
])
def test_plan_options_validation(L, opts, status):
    """dwt2d_plan_ex checks every launch option's range; defaults are all zeros."""
    p = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    o = D.plan_options(**opts)
    st = L.dwt2d_plan_ex(ctypes.byref(p), 512, 512, 5, 0, 2, 0, 0, ctypes.byref(o), ctypes.byref(ws))
    assert st == status
    if st == 0:
        L.dwt2d_plan_destroy(p)


def test_plan_options_change_the_launch_decomposition_only(L):
    """fuse_max = 1 gives one launch per level; the workspace grows with the LL it keeps."""
    for fm, groups in ((1, [1, 1, 1, 1, 1]), (2, [2, 2, 1]), (3, [2, 3])):
        p = ctypes.c_void_p()
        ws = ctypes.c_size_t()
        o = D.plan_options(fuse_max=fm)
        assert L.dwt2d_plan_ex(ctypes.byref(p), 1024, 1024, 5, 0, 2, 0, 0, ctypes.byref(o),
                               ctypes.byref(ws)) == 0
        n, ng = ctypes.c_int32(), ctypes.c_int32()
        fused = (ctypes.c_int32 * 16)()
        assert L.dwt2d_plan_info(p, ctypes.byref(n), fused, ctypes.byref(ng)) == 0
        assert [fused[i] for i in range(ng.value)] == groups
        L.dwt2d_plan_destroy(p)


def test_plan_launch_info_reports_the_chosen_shapes(L):
    """The forward's first launch of a large float image runs 4 quadruple
    columns per lane, the small later ones 2; LeGall 5/3 keeps 2; forcing the
    columns is honoured; the multipass schemes have no streaming launches."""
    p = D.Plan(8192, 8192, 5, "cdf97", "nonsep_reduced")
    shapes = p.launch_info()
    assert [f for f, _q, _w in shapes] == [2, 2, 1]
    assert shapes[0][1] == 4 and shapes[1][1] == 2 and shapes[2][1] == 2
    assert all(w > 0 for _f, _q, w in shapes)
    assert [f for f, _q, _w in p.launch_info(inverse=True)] == [1, 2, 2]
    assert D.Plan(8192, 8192, 5, "legall53", "nonsep").launch_info()[0][1] == 2
    assert D.Plan(8192, 8192, 5, "cdf97", "nonsep_reduced",
                  options={"fwd_cols_per_lane": 2}).launch_info()[0][1] == 2
    assert D.Plan(512, 512, 2, "cdf97", "nonsep_reduced",
                  options={"fwd_cols_per_lane": 4}).launch_info()[0][1] == 4
    with pytest.raises(D.DwtError):
        D.Plan(512, 512, 2, "cdf97", "nonsep_multipass").launch_info()


@pytest.mark.parametrize("h,w,lv,wav,dt", [(1080, 1920, 5, "cdf97", torch.float32),
                                           (77, 3001, 2, "legall53", torch.int32),
                                           (4096, 512, 6, "cdf97", torch.float16)])
def test_workspace_bytes_helper_matches_plan(h, w, lv, wav, dt):
    assert D.workspace_bytes(h, w, lv, wav, "nonsep_reduced", dt) == \
        D.Plan(h, w, lv, wav, "nonsep_reduced", dt).workspace_bytes
