// Allocation-free variant of amg_bsr_spmv_dot.
//
// amg_bsr_spmv_dot reduces the dot product x . (A x) through per-CTA partial
// sums that it keeps in device memory it allocates and frees around the
// launch.  Some callers cannot allow that: a device allocation may fail or
// wait for the whole device, which a caller that runs between fixed-budget
// phases of a larger application, or one whose device memory is entirely
// owned by another allocator, cannot accept.  This variant keeps its scratch
// in a file-scope device array instead.  The caller still passes x, y and the
// result pointer; the call makes no cudaMalloc, cudaFree or allocating
// library call.
//
// The array is part of the library image: every GPU that loads the library
// holds it (AMG_NOALLOC_SCRATCH_DOUBLES doubles, 32 KiB) until the process
// exits.  All calls share it and it keeps the contents of the last call, so
// two calls whose work overlaps on the GPU (different streams, or different
// host threads) race on it; calls on one stream are ordered and safe.
#include <cuda.h>

#include <mutex>

#include "amg_internal.cuh"

namespace amg {

// Partial sums of one launch (one per CTA) followed by the final sum.
static __device__ __align__(256) double g_spmv_dot_scratch[AMG_NOALLOC_SCRATCH_DOUBLES];

// The calling thread's current CUDA context (driver entry point fetched once
// through the runtime, so the library needs no link to the driver library).
static int current_context(void **out)
{
    using CtxGetCurrent = CUresult (*)(CUcontext *);
    static CtxGetCurrent fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrent>(p);
    });
    if (!fn) {
        set_error("cuCtxGetCurrent is not available");
        return AMG_ERR_CUDA;
    }
    CUcontext c = nullptr;
    if (fn(&c) != CUDA_SUCCESS) {
        set_error("cuCtxGetCurrent failed");
        return AMG_ERR_CUDA;
    }
    *out = (void *)c;
    return AMG_OK;
}

// Device address of the array, looked up once per device and context with
// that device current.  In host code the array's name is only a host-side
// stand-in, so the kernels must be given this address, never the name.  The
// address belongs to the context that loaded the module: a context made
// after the device was reset loads it again, possibly elsewhere, so the
// lookup is keyed by the context as well as the device.
static int scratch_address(double **out)
{
    struct Entry {
        int dev;
        void *ctx;
        double *addr;
    };
    constexpr int kEntries = 16;
    static Entry table[kEntries];
    static int used = 0, next = 0;
    static std::mutex mu;
    int dev = 0;
    AMG_TRY_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    void *ctx = nullptr;
    AMG_TRY(current_context(&ctx));
    if (ctx)
        for (int i = 0; i < used; ++i)
            if (table[i].dev == dev && table[i].ctx == ctx) {
                *out = table[i].addr;
                return AMG_OK;
            }
    void *p = nullptr;
    AMG_TRY_CUDA(cudaGetSymbolAddress(&p, g_spmv_dot_scratch));  // makes the context current
    AMG_TRY(current_context(&ctx));
    Entry e{dev, ctx, static_cast<double *>(p)};
    if (used < kEntries) table[used++] = e;
    else {
        table[next] = e;  // more devices or contexts than entries: replace the oldest
        next = (next + 1) % kEntries;
    }
    *out = e.addr;
    return AMG_OK;
}

}  // namespace amg

using namespace amg;

extern "C" int amg_bsr_spmv_dot_noalloc(const amg_bsr *A, const double *x, double *y,
                                        double *dot_out, void *stream)
{
    clear_error();
    AMG_TRY(check_bsr(A, 1));  // the same checks as amg_bsr_spmv_dot
    if (!x || !y || !dot_out) {
        set_error("amg_bsr_spmv_dot_noalloc: null argument");
        return AMG_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (A->nbrows == 0) {
        *dot_out = 0.0;
        return AMG_OK;
    }
    Geom g;
    AMG_TRY(query_geom(&g));
    // the SpMV launch uses one partial sum per CTA; its grid is the same as
    // amg_bsr_spmv_dot's, so both give the same bits
    const int grid = spmv_grid(A->nbrows, g);
    if (grid + 1 > AMG_NOALLOC_SCRATCH_DOUBLES) {
        set_error("amg_bsr_spmv_dot_noalloc: the launch needs %d partial sums, the static "
                  "scratch holds %d",
                  grid + 1, AMG_NOALLOC_SCRATCH_DOUBLES);
        return AMG_ERR_LIMIT;
    }
    double *scratch = nullptr;
    AMG_TRY(scratch_address(&scratch));
    SpmvArgs<double> a{};
    a.row_ptr = A->row_ptr;
    a.col = A->col;
    a.val = A->val;
    a.nbr = A->nbrows;
    a.x = x;
    a.y = y;
    a.partials = scratch;
    int used = 0;
    AMG_TRY((launch_spmv<double, double>(A->bs_r, A->bs_c, SPMV_PLAIN, DOT_XY, a, g, s, &used)));
    double *total = scratch + (AMG_NOALLOC_SCRATCH_DOUBLES - 1);
    AMG_TRY(launch_reduce_sum(scratch, used, total, s));
    AMG_TRY_CUDA(cudaMemcpyAsync(dot_out, total, sizeof(double), cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    return AMG_OK;
}
