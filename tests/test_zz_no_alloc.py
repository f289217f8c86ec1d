"""dwt2d_forward_noalloc: the forward transform without a caller-supplied workspace.

This entry point is for callers that are not allowed to allocate device
memory (a plugin whose host owns every byte of device memory, or a path where
an allocation is not acceptable).  Its scratch is a fixed array inside the
library.  The test calls it through the C ABI twice in a row, on two
different images, and checks each result against dwt2d_forward (which uses a
caller-allocated workspace): the second call must not be disturbed by what
the first one left in the shared array.  It also checks that a plan needing
more scratch than the array holds is refused before any GPU work.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1705_08266_gb300 import dwt2d as D
from tests.parity_util import device_image, make_input

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 8 << 20  # DWT2D_NOALLOC_SCRATCH_BYTES in include/dwt2d.h


def _entry():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    f = D.lib().dwt2d_forward_noalloc
    vp = ctypes.c_void_p
    f.argtypes = [vp, vp, ctypes.c_int64, vp, ctypes.c_int64, ctypes.c_float, vp]
    f.restype = ctypes.c_int
    return f


def _status(stream):
    g = D.lib().dwt2d_noalloc_status
    g.argtypes = [ctypes.c_void_p]
    g.restype = ctypes.c_int
    return g(ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("wavelet,scheme", [("cdf97", "nonsep_reduced"), ("legall53", "nonsep"),
                                            ("cdf97", "separable")])
def test_noalloc_matches_forward_on_two_calls(wavelet, scheme):
    f = _entry()
    h, w, levels = 1000, 1211, 5
    plan = D.Plan(h, w, levels, wavelet, scheme)
    assert len(plan.info()[1]) >= 2  # more than one launch: the scratch is really used
    assert plan.workspace_bytes <= SCRATCH_BYTES
    stream = torch.cuda.current_stream()
    for seed in (101, 202):
        x = make_input(wavelet, h, w, seed)
        xd = device_image(x)
        ref = plan.forward(xd).cpu().numpy()
        out = D.empty_image(h, w, xd.dtype)
        es = xd.element_size()
        st = f(plan._h, ctypes.c_void_p(xd.data_ptr()), xd.stride(0) * es,
               ctypes.c_void_p(out.data_ptr()), out.stride(0) * es, 1.0,
               ctypes.c_void_p(stream.cuda_stream))
        assert st == 0
        assert _status(stream) == 0  # no kernel recorded an error in the shared array
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # the same kernels on the same input: the same bits, for 9/7 as for 5/3
        assert np.array_equal(got, ref), seed


def test_noalloc_refuses_plans_larger_than_its_scratch():
    f = _entry()
    plan = D.Plan(16384, 16384, 6, "cdf97", "nonsep_reduced")
    assert plan.workspace_bytes > SCRATCH_BYTES
    src = D.empty_image(16, 16)  # never touched: the call must fail before any GPU work
    st = f(plan._h, ctypes.c_void_p(src.data_ptr()), 16 * 4 * 1024, ctypes.c_void_p(src.data_ptr() + 4096),
           16 * 4 * 1024, 1.0, None)
    assert st == -1


def test_noalloc_refuses_bad_arguments_before_any_gpu_work():
    f = _entry()
    plan = D.Plan(64, 64, 2, "cdf97", "nonsep_reduced")
    x = D.empty_image(64, 64)
    stream = torch.cuda.current_stream()
    sp = x.stride(0) * x.element_size()
    # source and destination are the same buffer: refused like dwt2d_forward refuses it
    st = f(plan._h, ctypes.c_void_p(x.data_ptr()), sp, ctypes.c_void_p(x.data_ptr()), sp, 1.0,
           ctypes.c_void_p(stream.cuda_stream))
    assert st == -1
    # a misaligned destination
    st = f(plan._h, ctypes.c_void_p(x.data_ptr()), sp, ctypes.c_void_p(x.data_ptr() + 4), sp, 1.0,
           ctypes.c_void_p(stream.cuda_stream))
    assert st == -3
    assert _status(stream) == 0
