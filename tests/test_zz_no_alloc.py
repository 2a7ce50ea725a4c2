"""The allocation-free dot-product SpMV entry point.

amg_bsr_spmv_dot_noalloc serves callers that cannot let the library
allocate device memory inside a call (an allocation may fail or wait for the
whole device where the caller runs on a fixed memory budget, or the caller's
device memory belongs to another allocator).  It keeps its scratch in a
static device array instead.  This test calls it through the C ABI and
checks it against amg_bsr_spmv_dot on two calls in a row (the second call
finds the previous call's partial sums still in the shared array): both use
the same grid, kernel and fixed-order reduction, so y and the dot product
must agree bit for bit.  It also checks that the calls allocate nothing:
neither PyTorch's caching allocator nor the CUDA runtime's default
stream-ordered pool (what amg_bsr_spmv_dot allocates from) sees any use.
The file sorts last so that a run stopping at the first failure has run
every other test before it.
"""
import ctypes
import gc

import numpy as np
import pytest

import q1elasticity as q

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

POOL_USED_MEM_CURRENT, POOL_USED_MEM_HIGH = 7, 8  # cudaMemPoolAttr values


def _pool_watch():
    """(reset, used) on the current device's default memory pool: reset()
    clears the high watermark of memory in use; used() returns (in use now,
    high watermark since the reset)."""
    rt = ctypes.CDLL("libcudart.so.13")
    dev = ctypes.c_int(0)
    assert rt.cudaGetDevice(ctypes.byref(dev)) == 0
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0

    def get(attr):
        v = ctypes.c_uint64(0)
        assert rt.cudaMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset():
        zero = ctypes.c_uint64(0)
        assert rt.cudaMemPoolSetAttribute(pool, POOL_USED_MEM_HIGH, ctypes.byref(zero)) == 0

    return reset, lambda: (get(POOL_USED_MEM_CURRENT), get(POOL_USED_MEM_HIGH))


def test_noalloc_spmv_dot_matches_allocating_entry_point():
    import paper_2202_09056_gb300 as amg
    lib = amg.load()
    fn = lib.amg_bsr_spmv_dot_noalloc
    fn.argtypes = [ctypes.c_void_p] * 5
    fn.restype = ctypes.c_int
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(11)
    reset, used = _pool_watch()
    for shape in ((9, 7, 8), (12, 12, 12)):
        p = q.make_problem(shape, traction=(0, 0, -1), inclusion_frac=0.2)
        rp, cl = torch.from_numpy(p.row_ptr).to(dev), torch.from_numpy(p.col).to(dev)
        val = torch.from_numpy(p.val).to(dev)
        A = amg.make_bsr(rp, cl, val)
        stream = torch.cuda.current_stream().cuda_stream
        xs = [torch.from_numpy(rng.standard_normal(p.ndof)).to(dev) for _ in range(2)]
        refs = [amg.bsr_spmv_dot(rp, cl, val, x) for x in xs]
        ys = [torch.full_like(x, np.nan) for x in xs]
        ds = [ctypes.c_double(np.nan) for _ in xs]
        # no garbage collection inside the measured window: an earlier
        # tensor freed there would lower torch's count for reasons of its own
        gc.collect()
        gc.disable()
        try:
            torch.cuda.synchronize()
            torch_before = torch.cuda.memory_allocated()
            torch.cuda.reset_peak_memory_stats()
            reset()
            pool_before, _ = used()
            for call in range(2):
                st = fn(ctypes.byref(A), ctypes.c_void_p(xs[call].data_ptr()),
                        ctypes.c_void_p(ys[call].data_ptr()), ctypes.byref(ds[call]),
                        ctypes.c_void_p(stream))
                assert st == 0, lib.amg_last_error()
            torch.cuda.synchronize()
            pool_now, pool_high = used()
            torch_now, torch_high = torch.cuda.memory_allocated(), torch.cuda.max_memory_allocated()
        finally:
            gc.enable()
        # an allocation during the calls would lift the watermark above the
        # memory in use before them
        assert pool_now == pool_before and pool_high <= pool_before, (pool_before, pool_high)
        assert torch_now == torch_before
        assert torch_high == torch_before
        for call in range(2):
            y_ref, d_ref = refs[call]
            assert torch.equal(ys[call], y_ref), call
            assert ds[call].value == d_ref, (call, ds[call].value, d_ref)
