"""The read-back entry point that allocates nothing (lbm_melt_get_noalloc).

Some callers cannot let a library allocate device memory: a time-critical
loop in which a cudaMalloc would synchronise the device, or an application
whose pool allocator owns all device memory.  For them lbm_melt_get_noalloc
stages host-bound results through a fixed array instead of per-call
buffers.  This checks it through the C ABI against lbm_melt_get on two calls
in a row (bit for bit: both run the same kernels on the same state), and
that a cavity beyond its stated maximum is rejected.  The file
is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu



def _get(L, h, shape, ncols, fn):
    T = np.zeros(shape, np.float32)
    u = np.zeros(shape + (3,), np.float32)
    S = np.zeros(ncols, np.float64)
    lf = np.zeros(1, np.float64)
    st = fn(h, C.c_void_p(T.ctypes.data), C.c_void_p(u.ctypes.data), C.c_void_p(S.ctypes.data),
            C.c_void_p(lf.ctypes.data), 0)
    assert st == 0, L.lbm_melt_last_error(h).decode()
    return T, u, S, float(lf[0])


def test_get_noalloc_matches_get_on_two_calls():
    import torch
    assert torch.cuda.is_available()
    from paper_1604_03478_gb300 import Cavity, _abi, build
    build.build()
    L = _abi.load()
    cav = Cavity(40, 24, 20, face=0, Ra=1e5, Pr=0.1, Ste=1.0, Ma=0.2, s0=3.0, derive=True)
    for steps in (17, 4):
        cav.step(steps)  # the second call also sees values in flight (odd total)
        ref = _get(L, cav._h, cav.shape, cav.ncols, L.lbm_melt_get)
        out = _get(L, cav._h, cav.shape, cav.ncols, L.lbm_melt_get_noalloc)
        # the same kernels on the same state in the same order: bit for bit
        np.testing.assert_array_equal(out[0], ref[0])
        np.testing.assert_array_equal(out[1], ref[1])
        np.testing.assert_array_equal(out[2], ref[2])
        assert out[3] == ref[3]
    cav.close()


def test_get_noalloc_rejects_cavity_beyond_its_maximum():
    from paper_1604_03478_gb300 import Cavity, _abi
    L = _abi.load()
    cav = Cavity(129, 128, 128, face=0, Ra=0.0, Ste=0.1, s_nu=1.2, s_alpha=1.0)
    T = np.zeros(cav.shape, np.float32)
    st = L.lbm_melt_get_noalloc(cav._h, C.c_void_p(T.ctypes.data), None, None, None, 0)
    assert st == _abi.LBM_EINVAL
    assert b"at most 2097152 nodes" in L.lbm_melt_last_error(cav._h)
    cav.close()
