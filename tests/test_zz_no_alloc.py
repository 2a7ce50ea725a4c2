"""The allocation-free dot-product SpMV entry point.

amg_bsr_spmv_dot_noalloc serves callers that cannot let the library
allocate device memory inside a call (an allocation may fail or wait for the
whole device where the caller runs on a fixed memory budget, or the caller's
device memory belongs to another allocator).  It keeps its scratch in a
static device array instead.  This test calls it through the C ABI and
checks it against amg_bsr_spmv_dot on two calls in a row (the second call
finds the previous call's partial sums still in the shared array).  The
file sorts last so that a run stopping at the first failure has run every
other test before it.
"""
import ctypes

import numpy as np
import pytest

import q1elasticity as q

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_spmv_dot_matches_allocating_entry_point():
    import paper_2202_09056_gb300 as amg
    lib = amg.load()
    fn = lib.amg_bsr_spmv_dot_noalloc
    fn.argtypes = [ctypes.c_void_p] * 5
    fn.restype = ctypes.c_int
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(11)
    for shape in ((9, 7, 8), (12, 12, 12)):
        p = q.make_problem(shape, traction=(0, 0, -1), inclusion_frac=0.2)
        rp, cl = torch.from_numpy(p.row_ptr).to(dev), torch.from_numpy(p.col).to(dev)
        val = torch.from_numpy(p.val).to(dev)
        A = amg.make_bsr(rp, cl, val)
        stream = torch.cuda.current_stream().cuda_stream
        for call in range(2):
            x = torch.from_numpy(rng.standard_normal(p.ndof)).to(dev)
            y_ref, d_ref = amg.bsr_spmv_dot(rp, cl, val, x)
            y = torch.full_like(x, np.nan)
            d = ctypes.c_double(np.nan)
            st = fn(ctypes.byref(A), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                    ctypes.byref(d), ctypes.c_void_p(stream))
            assert st == 0, lib.amg_last_error()
            assert torch.allclose(y, y_ref, rtol=1e-12, atol=0.0), call
            assert abs(d.value - d_ref) <= 1e-12 * abs(d_ref), (call, d.value, d_ref)
