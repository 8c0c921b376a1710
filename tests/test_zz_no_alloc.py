"""ffcz_check_static: FP64 certification with no plan and no device allocation.

This entry point exists for callers that cannot allocate device memory at the
moment they need a check -- hosts whose memory manager owns the whole device
pool, allocator-free callback pipelines, validation steps that must not fail
for lack of memory mid-run.  Its scratch is a fixed device array in the
library.  Here it is called through the C ABI and compared with the
plan-based ffcz_check on the same inputs, on two calls in a row (the second
call finds the first call's leftovers in the shared array), on shapes from the
smallest to the 2^22-point limit; repeated calls must leave the device's free
memory unchanged.
"""
import ctypes

import numpy as np
import pytest

from oracle import ffcz_oracle as O
from paper_2601_01596_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the two paths run the same FP64 kernels on the same tables


def _bounds(e0):
    v = O.f_violation(O.dft(e0.astype(np.float64)))
    s = float(np.max(np.abs(e0.astype(np.float64))))
    return [(s, 1.001 * v, 1), (s, 0.999 * v, 0), (0.9999 * s, 2.0 * v, 0)]


@pytest.mark.parametrize("shape,seed", [((64, 64, 128), 1), ((256, 512), 2), ((128, 128, 256), 3),
                                        ((8, 8, 16), 4), ((1024, 2048), 5), ((16, 1024, 256), 6),
                                        ((32, 16, 32), 7)])
def test_static_check_matches_plan_check_two_calls(shape, seed):
    import torch
    import paper_2601_01596_b300 as ffcz
    L = ffcz.lib()
    e0 = W.bimodal_error(shape, seed, E=1.0, dtype=np.float32)
    t = torch.from_numpy(e0.copy()).cuda()
    plan = ffcz.Plan([shape])
    dims = (ctypes.c_int64 * len(shape))(*shape)
    for E, D, want in _bounds(e0):
        ref = plan.check(t.reshape(-1), [E], [D])[0]
        assert ref["certified"] == want
        for call in range(2):
            st = ffcz.Stats()
            status = L.ffcz_check_static(ctypes.c_void_p(t.data_ptr()), len(shape), dims, E, D,
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                         ctypes.byref(st))
            assert status == (ffcz.OK if want else ffcz.ERR_CERT_FAILED), (call, status)
            assert st.certified == ref["certified"]
            assert abs(st.f_margin64 - ref["f_margin64"]) <= TOL, call
            assert abs(st.s_margin64 - ref["s_margin64"]) <= TOL, call
            assert abs(st.s_ratio - ref["s_ratio"]) <= TOL, call


def test_static_check_rejects_fields_over_the_limit():
    import torch
    import paper_2601_01596_b300 as ffcz
    L = ffcz.lib()
    t = torch.zeros(16, device="cuda")
    big = (256, 256, 128)                       # 2^23 points > FFCZ_STATIC_MAX_POINTS
    assert np.prod(big) > ffcz.STATIC_MAX_POINTS
    dims = (ctypes.c_int64 * 3)(*big)
    st = ffcz.Stats()
    s = L.ffcz_check_static(ctypes.c_void_p(t.data_ptr()), 3, dims, 1.0, 1.0, None, ctypes.byref(st))
    assert s == ffcz.ERR_INVALID
    assert b"static scratch limit" in L.ffcz_last_error()


def test_static_check_allocates_no_device_memory():
    """After a first call (the set-up), further calls on new shapes leave the
    device's free memory exactly as it was."""
    import torch
    import paper_2601_01596_b300 as ffcz
    fields = [torch.from_numpy(W.bimodal_error(sh, 9, E=1.0, dtype=np.float32)).cuda()
              for sh in ((16, 32, 64), (512, 1024), (8, 1024, 512))]
    torch.cuda.synchronize()
    ffcz.check_static(fields[0], 1.0, 1e9)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for t in fields * 3:
        s, st = ffcz.check_static(t, 1.0, 1e9)
        assert s == ffcz.OK and st["certified"] == 1
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
