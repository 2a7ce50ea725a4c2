// Block CSR sparse matrix-vector products for sm_103a: the memory-bound
// primitive of the paper's Sec. 2 (block values are loaded and used at once),
// with the fused epilogues of the V-cycle (Alg. 2): residual, smoothing,
// prolongation-correction and restriction, and the fused CG dot products.
//
// Design: one warp per block row, flat stream over the row's values.  The
// values of a block row are contiguous (nnz_row * BR * BC elements, blocks
// row-major), so lane k of the warp reads element k, k+32, ... of that segment:
// every warp-wide load is fully coalesced whatever the block shape, and the
// 72-byte 3x3 FP64 blocks need no padding.  Element k belongs to block k/BB,
// block row (k%BB)/BC and block column k%BC; the lane multiplies it with the
// gathered x entry (L2-resident) and accumulates into one of BR partial sums,
// which a butterfly shuffle reduces at the end of the row.  Values are read
// with the streaming (evict-first) hint; x with the read-only path.
//
// All reductions (row sums, fused dots) run in a fixed order for a fixed
// launch geometry, so results are bitwise reproducible run to run.
#include "amg_internal.cuh"

namespace amg {

__device__ __forceinline__ double ldv(const double *p) { return __ldcs(p); }
__device__ __forceinline__ float ldv(const float *p) { return __ldcs(p); }
__device__ __forceinline__ float ldv(const __nv_bfloat16 *p)
{
    unsigned short bits = __ldcs(reinterpret_cast<const unsigned short *>(p));
    return __uint_as_float(((unsigned int)bits) << 16);
}

template <class T> __device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    return v;
}

// Sum a per-thread double over the CTA in a fixed order; thread 0 gets it.
template <int NT> __device__ __forceinline__ double cta_sum(double v)
{
    __shared__ double red[NT / 32];
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NT / 32; ++k) s += red[k];
    }
    return s;
}

constexpr int SPMV_THREADS = 256;

template <int BR, int BC, class VT, class TV, int MODE, int DOT>
__global__ void __launch_bounds__(SPMV_THREADS) bsr_spmv_kernel(SpmvArgs<TV> a)
{
    using Acc = TV;
    constexpr int BB = BR * BC;
    if (a.stop && *a.stop) return;
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * (unsigned)blockDim.x) >> 5);
    const VT *__restrict__ val = static_cast<const VT *>(a.val);
    const int *__restrict__ col = a.col;
    const TV *__restrict__ x = a.x;
    double dot = 0.0;

    for (int row = warp; row < a.nbr; row += nwarps) {
        const int s = __ldg(a.row_ptr + row), e = __ldg(a.row_ptr + row + 1);
        const int nv = (e - s) * BB;
        const VT *vb = val + (int64_t)s * BB;
        const int *cb = col + s;
        Acc acc[BR];
#pragma unroll
        for (int r = 0; r < BR; ++r) acc[r] = Acc(0);
#pragma unroll 4
        for (int k = lane; k < nv; k += 32) {
            const int blk = k / BB;
            const int el = k - blk * BB;
            const int r = el / BC;
            const int c = el - r * BC;
            const Acc v = (Acc)ldv(vb + k);
            const Acc xv = (Acc)__ldg(x + (int64_t)__ldg(cb + blk) * BC + c);
#pragma unroll
            for (int rr = 0; rr < BR; ++rr)
                if (r == rr) acc[rr] = fma(v, xv, acc[rr]);
        }
#pragma unroll
        for (int rr = 0; rr < BR; ++rr) acc[rr] = warp_sum(acc[rr]);
        if (lane < BR) {
            Acc ax = acc[0];
#pragma unroll
            for (int rr = 1; rr < BR; ++rr)
                if (lane == rr) ax = acc[rr];
            const int64_t i = (int64_t)row * BR + lane;
            Acc out;
            if (MODE == SPMV_PLAIN) {
                out = ax;
            } else if (MODE == SPMV_RESID) {
                out = a.f[i] - ax;
            } else if (MODE == SPMV_SMOOTH) {
                out = x[i] + a.M[i] * (a.f[i] - ax);
            } else if (MODE == SPMV_AXPY) {
                out = a.u[i] + ax;
            } else {  // SPMV_RESTRICT
                out = ax;
            }
            a.y[i] = out;
            if (MODE == SPMV_RESTRICT && a.y2) a.y2[i] = a.M ? a.M[i] * out : Acc(0);
            if (DOT == DOT_XY) dot += (double)x[i] * (double)out;
            if (DOT == DOT_FY) dot += (double)a.f[i] * (double)out;
            if (DOT == DOT_YY) dot += (double)out * (double)out;
        }
    }
    if (DOT != DOT_NONE) {
        const double t = cta_sum<SPMV_THREADS>(dot);
        if (threadIdx.x == 0) a.partials[blockIdx.x] = t;
    }
}

template <int BR, int BC, class VT, class TV, int DOT>
static int csr_go(const SpmvArgs<TV> &a, int grid, cudaStream_t s)
{
    bsr_spmv_kernel<BR, BC, VT, TV, SPMV_PLAIN, DOT><<<grid, SPMV_THREADS, 0, s>>>(a);
    ::amg::count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    return AMG_OK;
}

// The CSR kernels serve the stateless primitives: y = A x, optionally with
// the fused x . y of a square matrix.
template <int BR, int BC, class VT, class TV>
static int launch_mode(int mode, int dot, const SpmvArgs<TV> &a, int grid, cudaStream_t s)
{
    if (mode != SPMV_PLAIN) {
        set_error("the CSR kernel only computes y = A x");
        return AMG_ERR_ARG;
    }
    if (dot == DOT_NONE) return csr_go<BR, BC, VT, TV, DOT_NONE>(a, grid, s);
    if constexpr (BR == BC)
        if (dot == DOT_XY) return csr_go<BR, BC, VT, TV, DOT_XY>(a, grid, s);
    set_error("unsupported dot mode %d", dot);
    return AMG_ERR_ARG;
}

int spmv_grid(int nbr, const Geom &g)
{
    const int rows_per_cta = SPMV_THREADS / 32;
    int grid = (nbr + rows_per_cta - 1) / rows_per_cta;
    if (grid > g.max_ctas) grid = g.max_ctas;
    if (grid < 1) grid = 1;
    return grid;
}

template <class VT, class TV>
int launch_spmv(int br, int bc, int mode, int dot, const SpmvArgs<TV> &a, const Geom &g,
                cudaStream_t s, int *grid_out)
{
    const int grid = spmv_grid(a.nbr, g);
    if (grid_out) *grid_out = grid;
    if (a.nbr == 0) {
        if (dot != DOT_NONE) AMG_TRY_CUDA(cudaMemsetAsync(a.partials, 0, sizeof(double), s));
        return AMG_OK;
    }
    if (br == 3 && bc == 3) return launch_mode<3, 3, VT, TV>(mode, dot, a, grid, s);
    if (br == 6 && bc == 6) return launch_mode<6, 6, VT, TV>(mode, dot, a, grid, s);
    if (br == 3 && bc == 6) return launch_mode<3, 6, VT, TV>(mode, dot, a, grid, s);
    if (br == 6 && bc == 3) return launch_mode<6, 3, VT, TV>(mode, dot, a, grid, s);
    set_error("unsupported block shape %dx%d", br, bc);
    return AMG_ERR_ARG;
}

template int launch_spmv<double, double>(int, int, int, int, const SpmvArgs<double> &,
                                         const Geom &, cudaStream_t, int *);


// ---------------------------------------------------------------- reductions
constexpr int RED_THREADS = 256;

__global__ void __launch_bounds__(RED_THREADS) reduce_sum_kernel(const double *p, int n,
                                                                  double *out)
{
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += RED_THREADS) v += p[i];
    const double t = cta_sum<RED_THREADS>(v);
    if (threadIdx.x == 0) *out = t;
}

int launch_reduce_sum(const double *partials, int n, double *out, cudaStream_t s)
{
    reduce_sum_kernel<<<1, RED_THREADS, 0, s>>>(partials, n, out); ::amg::count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    return AMG_OK;
}

// ---------------------------------------------------------------- coarse GEMV
// y = Ainv x with the dense inverse of the coarsest matrix (row-major, FP64),
// one warp per row; the input/output vectors may be FP32 in the reduced
// precision forms, the product is always accumulated in FP64.
template <class TV>
__global__ void __launch_bounds__(256) coarse_gemv_kernel(const double *__restrict__ Ainv, int n,
                                                          const TV *__restrict__ x,
                                                          TV *__restrict__ y)
{
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * (unsigned)blockDim.x) >> 5);
    for (int row = warp; row < n; row += nwarps) {
        const double *ar = Ainv + (int64_t)row * n;
        // eight independent partial sums per lane keep eight loads in flight
        // (one chain would wait on every load); summed in a fixed order
        double p[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) p[q] = 0.0;
        int j = lane;
        for (; j + 7 * 32 < n; j += 8 * 32) {
#pragma unroll
            for (int q = 0; q < 8; ++q) p[q] = fma(__ldg(ar + j + q * 32), (double)x[j + q * 32], p[q]);
        }
#pragma unroll
        for (int q = 0; q < 7; ++q)  // at most seven strides remain
            if (j + q * 32 < n) p[q] = fma(__ldg(ar + j + q * 32), (double)x[j + q * 32], p[q]);
        double acc = ((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7]));
        acc = warp_sum(acc);
        if (lane == 0) y[row] = (TV)acc;
    }
}

template <class TV>
int launch_coarse_gemv(const double *Ainv, int n, const TV *x, TV *y, const Geom &g,
                       cudaStream_t s)
{
    if (n == 0) return AMG_OK;
    int grid = (n + 7) / 8;
    if (grid > g.max_ctas) grid = g.max_ctas;
    coarse_gemv_kernel<TV><<<grid, 256, 0, s>>>(Ainv, n, x, y); ::amg::count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    return AMG_OK;
}
template int launch_coarse_gemv<double>(const double *, int, const double *, double *,
                                        const Geom &, cudaStream_t);
template int launch_coarse_gemv<float>(const double *, int, const float *, float *,
                                       const Geom &, cudaStream_t);

}  // namespace amg
