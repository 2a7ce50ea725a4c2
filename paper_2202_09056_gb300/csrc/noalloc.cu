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
#include <mutex>

#include "amg_internal.cuh"

namespace amg {

// Partial sums of one launch (one per CTA) followed by the final sum.
static __device__ __align__(256) double g_spmv_dot_scratch[AMG_NOALLOC_SCRATCH_DOUBLES];

// Device address of the array, looked up once per device with that device
// current.  In host code the array's name is only a host-side stand-in, so
// the kernels must be given this address, never the name.
static int scratch_address(double **out)
{
    static std::mutex mu;
    static double *addr[64] = {nullptr};
    int dev = 0;
    AMG_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("device ordinal %d out of range", dev);
        return AMG_ERR_LIMIT;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        AMG_TRY_CUDA(cudaGetSymbolAddress(&p, g_spmv_dot_scratch));
        addr[dev] = static_cast<double *>(p);
    }
    *out = addr[dev];
    return AMG_OK;
}

}  // namespace amg

using namespace amg;

extern "C" int amg_bsr_spmv_dot_noalloc(const amg_bsr *A, const double *x, double *y,
                                        double *dot_out, void *stream)
{
    clear_error();
    if (!A || !x || !y || !dot_out || A->nbrows < 0 || A->nbrows != A->nbcols ||
        A->bs_r != A->bs_c || A->nnzb < 0 || !A->row_ptr || (A->nnzb > 0 && (!A->col || !A->val))) {
        set_error("amg_bsr_spmv_dot_noalloc: bad argument");
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
