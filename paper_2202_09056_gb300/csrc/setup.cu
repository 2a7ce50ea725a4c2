// Setup kernels of Alg. 1 (Sec. 2) in block arithmetic: strength of
// connection on block norms, tentative prolongation from the rigid-body modes
// (per-aggregate modified Gram-Schmidt QR, the step Sec. 2 says needs scalar
// arithmetic, done here inside block-shaped kernels), the Gershgorin
// estimate for the damped-Jacobi prolongation smoother, the smoothed
// prolongation P = (I - omega D^-1 A) P_tent, R = P^T, the block Galerkin
// product A_c = R (A P) (Sec. 3: the expensive step kept in block form),
// the SPAI0 smoother, and the dense coarsest-level factorisation.
//
// Patterns are symbolic (structurally present products kept, zeros
// included) and column-sorted; every floating-point sum runs in a fixed
// order.  The strength norms are computed without fused multiply-adds so
// that the aggregation sees the same bits on every run and platform.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <climits>

#include "amg_internal.cuh"

namespace amg {

constexpr int T1D = 256;
static inline int nblk(int64_t n, int t = T1D) { return (int)((n + t - 1) / t); }

// ---------------------------------------------------------------- scan
constexpr int SCAN_T = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_T * SCAN_ITEMS;

__global__ void __launch_bounds__(SCAN_T) scan_tile_kernel(const int *__restrict__ in,
                                                           int *__restrict__ out, int n,
                                                           long long *__restrict__ tile_sum)
{
    __shared__ long long sh[SCAN_T];
    const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    long long v[SCAN_ITEMS], s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        s += v[i];
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < SCAN_T; off <<= 1) {
        long long t = (threadIdx.x >= (unsigned)off) ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    long long run = sh[threadIdx.x] - s;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < n) out[base + i] = (int)run;  // tile-local, fixed below
        run += v[i];
    }
    if (threadIdx.x == SCAN_T - 1) tile_sum[blockIdx.x] = sh[SCAN_T - 1];
}

__global__ void scan_add_kernel(int *out, int n, const int *__restrict__ tile_off)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_off[i / SCAN_TILE];
}

// out[0..n] = exclusive prefix sum of in[0..n-1]; out[n] = total.  The tile
// totals are combined on the host in 64-bit so that an int32 overflow is
// reported instead of wrapping.
int exclusive_scan_i32(const int *in, int *out, int n, int *total_host, DevArena &tmp,
                       cudaStream_t s)
{
    if (n == 0) {
        AMG_TRY_CUDA(cudaMemsetAsync(out, 0, sizeof(int), s));
        if (total_host) *total_host = 0;
        return AMG_OK;
    }
    const int ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    long long *tsum = nullptr;
    int *toff = nullptr;
    AMG_TRY(tmp.alloc_n(&tsum, ntiles));
    AMG_TRY(tmp.alloc_n(&toff, ntiles));
    scan_tile_kernel<<<ntiles, SCAN_T, 0, s>>>(in, out, n, tsum); ::amg::count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    std::vector<long long> h(ntiles);
    AMG_TRY_CUDA(cudaMemcpyAsync(h.data(), tsum, sizeof(long long) * ntiles,
                                 cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    std::vector<int> off(ntiles);
    long long run = 0;
    for (int t = 0; t < ntiles; ++t) {
        off[t] = (int)run;
        run += h[t];
        if (run > 2147483647LL) {
            set_error("prefix sum exceeds int32 (%lld)", run);
            return AMG_ERR_LIMIT;
        }
    }
    AMG_TRY_CUDA(cudaMemcpyAsync(toff, off.data(), sizeof(int) * ntiles,
                                 cudaMemcpyHostToDevice, s));
    scan_add_kernel<<<nblk(n), T1D, 0, s>>>(out, n, toff); ::amg::count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    const int total = (int)run;
    AMG_TRY_CUDA(cudaMemcpyAsync(out + n, &total, sizeof(int), cudaMemcpyHostToDevice, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));  // `off` and `total` are host stack memory
    tmp.release(tsum);
    tmp.release(toff);
    if (total_host) *total_host = total;
    return AMG_OK;
}

// ---------------------------------------------------------------- strength
// ||A_IJ||_F^2 with squares summed in row-major order, no FMA contraction.
__device__ __forceinline__ double block_norm2(const double *blk, int bb)
{
    double s = 0.0;
    for (int e = 0; e < bb; ++e) s = __dadd_rn(s, __dmul_rn(blk[e], blk[e]));
    return s;
}

__global__ void diag_norm_kernel(const int *__restrict__ rp, const int *__restrict__ col,
                                 const double *__restrict__ val, int nbr, int b,
                                 double *__restrict__ dn)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nbr) return;
    double v = 0.0;
    for (int p = rp[I]; p < rp[I + 1]; ++p)
        if (col[p] == I) v = __dsqrt_rn(block_norm2(val + (int64_t)p * b * b, b * b));
    dn[I] = v;
}

// J != I is strong iff ||A_IJ||^2 > (eps^2 ||A_II||) ||A_JJ||.  One warp per
// block row, the lanes over its blocks (each test is independent).
__global__ void strength_kernel(const int *__restrict__ rp, const int *__restrict__ col,
                                const double *__restrict__ val, int nbr, int b, double e2,
                                const double *__restrict__ dn, uint8_t *__restrict__ strong)
{
    const int I = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (I >= nbr) return;
    const double dI = dn[I];
    for (int p = rp[I] + lane; p < rp[I + 1]; p += 32) {
        const int J = col[p];
        uint8_t st = 0;
        if (J != I) {
            const double n2 = block_norm2(val + (int64_t)p * b * b, b * b);
            double thr = __dmul_rn(e2, dI);
            thr = __dmul_rn(thr, dn[J]);
            st = n2 > thr ? 1 : 0;
        }
        strong[p] = st;
    }
}

int compute_strength(const BsrD &A, double eps, uint8_t *strong, cudaStream_t s)
{
    if (A.nbr == 0) return AMG_OK;
    double *dn = nullptr;
    DevArena tmp;
    tmp.stream = s;
    AMG_TRY(tmp.alloc_n(&dn, (size_t)A.nbr));
    diag_norm_kernel<<<nblk(A.nbr), T1D, 0, s>>>(A.row_ptr, A.col, A.val, A.nbr, A.br, dn); ::amg::count_launch(1);
    const double e2 = eps * eps;
    strength_kernel<<<nblk((int64_t)A.nbr * 32), T1D, 0, s>>>(A.row_ptr, A.col, A.val, A.nbr, A.br,
                                                              e2, dn, strong);
    ::amg::count_launch(1);
    const cudaError_t e = cudaGetLastError();
    tmp.release_all();
    if (e != cudaSuccess) {
        set_error("strength kernels: %s", cudaGetErrorString(e));
        return AMG_ERR_CUDA;
    }
    return AMG_OK;
}

// ---------------------------------------------------------------- strong graph to the host
// The host's greedy aggregation reads, per node, its strong neighbours in
// column order.  Only those go to the host: per row the strong columns
// (row order kept), as CSR (srp, scol), instead of the whole pattern and a
// flag per block.
__global__ void strong_count_kernel(const int *__restrict__ rp, const uint8_t *__restrict__ strong,
                                    int nbr, int *__restrict__ cnt)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nbr) return;
    int c = 0;
    for (int p = rp[I]; p < rp[I + 1]; ++p) c += strong[p] ? 1 : 0;
    cnt[I] = c;
}

__global__ void strong_fill_kernel(const int *__restrict__ rp, const int *__restrict__ col,
                                   const uint8_t *__restrict__ strong, int nbr,
                                   const int *__restrict__ srp, int *__restrict__ scol)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nbr) return;
    int q = srp[I];
    for (int p = rp[I]; p < rp[I + 1]; ++p)
        if (strong[p]) scol[q++] = col[p];
}

int strong_graph_to_host(const BsrD &A, const uint8_t *strong, DevArena &tmp, cudaStream_t s,
                         HostStrongGraph *out)
{
    const int nbr = A.nbr;
    out->nn = nbr;
    out->srp.reset(new int[(size_t)nbr + 1]);
    int *cnt = nullptr, *srp = nullptr, *scol = nullptr;
    AMG_TRY(tmp.alloc_n(&cnt, (size_t)std::max(nbr, 1)));
    AMG_TRY(tmp.alloc_n(&srp, (size_t)nbr + 1));
    if (nbr > 0) {
        strong_count_kernel<<<nblk(nbr), T1D, 0, s>>>(A.row_ptr, strong, nbr, cnt);
        ::amg::count_launch(1);
    }
    int total = 0;
    AMG_TRY(exclusive_scan_i32(cnt, srp, nbr, &total, tmp, s));
    AMG_TRY(tmp.alloc_n(&scol, (size_t)std::max(total, 1)));
    if (nbr > 0 && total > 0) {
        strong_fill_kernel<<<nblk(nbr), T1D, 0, s>>>(A.row_ptr, A.col, strong, nbr, srp, scol);
        ::amg::count_launch(1);
    }
    AMG_TRY_CUDA(cudaGetLastError());
    out->scol.reset(new int[(size_t)std::max(total, 1)]);
    AMG_TRY_CUDA(cudaMemcpyAsync(out->srp.get(), srp, sizeof(int) * ((size_t)nbr + 1),
                                 cudaMemcpyDeviceToHost, s));
    if (total > 0)
        AMG_TRY_CUDA(cudaMemcpyAsync(out->scol.get(), scol, sizeof(int) * (size_t)total,
                                     cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    tmp.release(cnt);
    tmp.release(srp);
    tmp.release(scol);
    return AMG_OK;
}

// ---------------------------------------------------------------- tentative P
template <class T> __device__ __forceinline__ T wsum(T v)
{
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    return v;
}

// One warp per aggregate.  The member rows of B (ascending node order, b rows
// per node) are stacked into Qs (row-major, NS columns: NS rigid-body modes or
// 3 translations) and orthonormalised by
// modified Gram-Schmidt with one re-orthogonalisation pass; a column whose
// norm drops to <= 1e-10 of its original norm is dropped (zero Q column and
// zero R row).  Every lane owns rows lane, lane+32, ... of the stack, so only
// the reductions cross lanes.
template <int NS>
__global__ void tentative_kernel(int nagg, int b, const int *__restrict__ agg_ptr,
                                 const int *__restrict__ members, const double *__restrict__ B,
                                 double *__restrict__ Qs, double *__restrict__ ptent,
                                 double *__restrict__ Bc)
{
    const int lane = threadIdx.x & 31;
    const int a = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (a >= nagg) return;
    const int m0 = agg_ptr[a], m = (agg_ptr[a + 1] - m0) * b;
    double *Q = Qs + (int64_t)m0 * b * NS;
    for (int i = lane; i < m; i += 32) {
        const int node = members[m0 + i / b], r = i % b;
#pragma unroll
        for (int k = 0; k < NS; ++k) Q[i * NS + k] = B[((int64_t)node * b + r) * NS + k];
    }
    double R[NS][NS];
#pragma unroll
    for (int j = 0; j < NS; ++j)
#pragma unroll
        for (int k = 0; k < NS; ++k) R[j][k] = 0.0;
    bool dropped[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) dropped[k] = false;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        double s = 0.0;
        for (int i = lane; i < m; i += 32) s += Q[i * NS + k] * Q[i * NS + k];
        const double pre = sqrt(wsum(s));
        for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
            for (int j = 0; j < k; ++j) {
                if (dropped[j]) continue;
                double t = 0.0;
                for (int i = lane; i < m; i += 32) t += Q[i * NS + j] * Q[i * NS + k];
                const double d = wsum(t);
                R[j][k] += d;
                for (int i = lane; i < m; i += 32) Q[i * NS + k] -= d * Q[i * NS + j];
            }
        }
        s = 0.0;
        for (int i = lane; i < m; i += 32) s += Q[i * NS + k] * Q[i * NS + k];
        const double post = sqrt(wsum(s));
        if (post <= 1e-10 * pre) {
            dropped[k] = true;
            for (int i = lane; i < m; i += 32) Q[i * NS + k] = 0.0;
#pragma unroll
            for (int j = 0; j < NS; ++j) R[k][j] = 0.0;
        } else {
            for (int i = lane; i < m; i += 32) Q[i * NS + k] /= post;
            R[k][k] = post;
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NS; ++k)
#pragma unroll
            for (int j = 0; j < NS; ++j) Bc[(int64_t)a * NS * NS + k * NS + j] = R[k][j];
    }
    for (int i = lane; i < m; i += 32) {
        const int node = members[m0 + i / b], r = i % b;
#pragma unroll
        for (int k = 0; k < NS; ++k) ptent[((int64_t)node * b + r) * NS + k] = Q[i * NS + k];
    }
}

// ---------------------------------------------------------------- Jacobi diagonal, rho
// d_i = a_ii; g_i = sum_j |a_ij| / |a_ii| over scalar row i (blocks ascending,
// then columns); rho = max g_i (atomic max on the bits of a non-negative
// double, order independent).  This is the damped-Jacobi prolongation
// smoother's data on the unfiltered matrix.
__global__ void jacobi_rho_kernel(const int *__restrict__ rp, const int *__restrict__ col,
                                  const double *__restrict__ val, int nbr, int b,
                                  double *__restrict__ d, unsigned long long *__restrict__ rho_bits)
{
    // one thread per scalar row (b per block row)
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nbr * b) return;
    const int I = (int)(i / b), r = (int)(i % b);
    const int bb = b * b;
    double dia = 0.0, s = 0.0;
    for (int p = rp[I]; p < rp[I + 1]; ++p)
        for (int c = 0; c < b; ++c) {
            const double v = val[(int64_t)p * bb + r * b + c];
            if (col[p] == I && c == r) dia = v;
            s = __dadd_rn(s, fabs(v));
        }
    d[i] = dia;
    if (dia != 0.0) {
        const double g = __ddiv_rn(s, fabs(dia));
        atomicMax(rho_bits, (unsigned long long)__double_as_longlong(g));
    }
}

// ---------------------------------------------------------------- small sorted sets
template <int CAP> struct SortedSet {
    int n = 0;
    int v[CAP];
    __device__ __forceinline__ bool insert(int x)
    {
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (v[mid] < x) lo = mid + 1;
            else hi = mid;
        }
        if (lo < n && v[lo] == x) return true;
        if (n == CAP) return false;
        for (int t = n; t > lo; --t) v[t] = v[t - 1];
        v[lo] = x;
        ++n;
        return true;
    }
};

constexpr int SYM_CAP = 128;  // per-thread sorted set of the first symbolic pass

__device__ __forceinline__ int find_sorted(const int *a, int lo, int hi, int x)
{
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Symbolic C = X Y, routing: a row whose candidate products (the sum of the
// lengths of the Y rows it touches) are many goes straight to the bitmap
// pass: more than 4 SYM_CAP candidates, or more than SYM_CAP when C has at
// most 4096 columns (the bitmap is then at most 512 bytes).  The per-thread
// sorted set costs a binary search per candidate and a shift per new column,
// in local memory, which dominated the symbolic products on the coarse levels.
__global__ void sym_route_kernel(const int *__restrict__ xrp, const int *__restrict__ xcol,
                                 const int *__restrict__ yrp, int nrows, int ncols,
                                 uint8_t *__restrict__ islong, int *__restrict__ longrows,
                                 int *__restrict__ nlong)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows) return;
    int64_t cand = 0;
    for (int p = xrp[i]; p < xrp[i + 1]; ++p) {
        const int k = xcol[p];
        cand += yrp[k + 1] - yrp[k];
    }
    const bool lng = cand > 4 * SYM_CAP || (cand > SYM_CAP && ncols <= 4096);
    islong[i] = lng ? 1 : 0;
    if (lng) longrows[atomicAdd(nlong, 1)] = i;
}

// Symbolic C = X Y, first pass for the other rows: one thread per row keeps
// the row's distinct columns in a sorted local set.  Count mode writes the
// row length, or marks the row long and appends it to `longrows` when it has
// more than SYM_CAP distinct columns; write mode fills the short rows.
template <bool WRITE>
__global__ void sym_small_kernel(const int *__restrict__ xrp, const int *__restrict__ xcol,
                                 const int *__restrict__ yrp, const int *__restrict__ ycol,
                                 int nrows, int *__restrict__ cnt, const int *__restrict__ crp,
                                 int *__restrict__ ccol, uint8_t *__restrict__ islong,
                                 int *__restrict__ longrows, int *__restrict__ nlong)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows) return;
    if (islong[i]) return;
    SortedSet<SYM_CAP> S;
    for (int p = xrp[i]; p < xrp[i + 1]; ++p) {
        const int k = xcol[p];
        for (int q = yrp[k]; q < yrp[k + 1]; ++q)
            if (!S.insert(ycol[q])) {
                if (!WRITE) {
                    islong[i] = 1;
                    longrows[atomicAdd(nlong, 1)] = i;
                }
                return;
            }
    }
    if (!WRITE) cnt[i] = S.n;
    else
        for (int t = 0; t < S.n; ++t) ccol[crp[i] + t] = S.v[t];
}

// Symbolic C = X Y, second pass for the long rows: one CTA per row marks the
// row's columns in a shared-memory bitmap over the column range; counting is
// a popcount, and the fill walks the bitmap in order, so the columns come
// out sorted without a sort.
constexpr int SYM_T = 256;
template <bool WRITE>
__global__ void __launch_bounds__(SYM_T) sym_bitmap_kernel(
    const int *__restrict__ xrp, const int *__restrict__ xcol, const int *__restrict__ yrp,
    const int *__restrict__ ycol, int ncols, const int *__restrict__ rows, int nlist,
    int *__restrict__ cnt, const int *__restrict__ crp, int *__restrict__ ccol)
{
    extern __shared__ unsigned bits[];
    __shared__ int scan[SYM_T];
    const int nwords = (ncols + 31) >> 5;
    const int chunk = (nwords + SYM_T - 1) / SYM_T;
    for (int li = blockIdx.x; li < nlist; li += gridDim.x) {
        const int i = rows[li];
        for (int w = threadIdx.x; w < nwords; w += SYM_T) bits[w] = 0u;
        __syncthreads();
        for (int p = xrp[i] + threadIdx.x; p < xrp[i + 1]; p += SYM_T) {
            const int k = xcol[p];
            for (int q = yrp[k]; q < yrp[k + 1]; ++q) {
                const int c = ycol[q];
                atomicOr(&bits[c >> 5], 1u << (c & 31));
            }
        }
        __syncthreads();
        const int w0 = threadIdx.x * chunk, w1 = min(w0 + chunk, nwords);
        int mine = 0;
        for (int w = w0; w < w1; ++w) mine += __popc(bits[w]);
        scan[threadIdx.x] = mine;
        __syncthreads();
        for (int off = 1; off < SYM_T; off <<= 1) {  // inclusive scan of the chunk counts
            const int t = (threadIdx.x >= (unsigned)off) ? scan[threadIdx.x - off] : 0;
            __syncthreads();
            scan[threadIdx.x] += t;
            __syncthreads();
        }
        if (!WRITE) {
            if (threadIdx.x == SYM_T - 1) cnt[i] = scan[SYM_T - 1];
        } else {
            int o = crp[i] + scan[threadIdx.x] - mine;
            for (int w = w0; w < w1; ++w) {
                unsigned m = bits[w];
                while (m) {
                    const int b = __ffs(m) - 1;
                    ccol[o++] = (w << 5) + b;
                    m &= m - 1;
                }
            }
        }
        __syncthreads();
    }
}

// Row pattern of C = X Y (sorted columns, symbolic: every structurally
// present product creates an entry).  Allocates C's row pointers and columns
// in `keep`.
static int spgemm_symbolic(const int *xrp, const int *xcol, int nrows, const int *yrp,
                           const int *ycol, int ncols, DevArena &keep, DevArena &tmp,
                           cudaStream_t s, int **crp_out, int **ccol_out, int *nnz_out)
{
    int *cnt = nullptr, *ovf = nullptr, *novf = nullptr, *crp = nullptr, *ccol = nullptr;
    uint8_t *islong = nullptr;
    AMG_TRY(tmp.alloc_n(&cnt, (size_t)nrows + 1));
    AMG_TRY(tmp.alloc_n(&ovf, (size_t)std::max(nrows, 1)));
    AMG_TRY(tmp.alloc_n(&islong, (size_t)std::max(nrows, 1)));
    AMG_TRY(tmp.alloc_n(&novf, 1));
    AMG_TRY(keep.alloc_n(&crp, (size_t)nrows + 1));
    AMG_TRY_CUDA(cudaMemsetAsync(novf, 0, sizeof(int), s));
    if (nrows > 0) {
        sym_route_kernel<<<nblk(nrows), T1D, 0, s>>>(xrp, xcol, yrp, nrows, ncols, islong, ovf,
                                                     novf);
        sym_small_kernel<false><<<nblk(nrows), T1D, 0, s>>>(xrp, xcol, yrp, ycol, nrows, cnt,
                                                            nullptr, nullptr, islong, ovf, novf);
        ::amg::count_launch(2);
        AMG_TRY_CUDA(cudaGetLastError());
    }
    int nlong = 0;
    AMG_TRY_CUDA(cudaMemcpyAsync(&nlong, novf, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    const size_t smem = sizeof(unsigned) * (size_t)((ncols + 31) / 32);
    if (nlong > 0) {
        if (smem > 200 * 1024) {
            set_error("sparse product with %d block columns exceeds the bitmap limit", ncols);
            return AMG_ERR_LIMIT;
        }
        if (smem > 48 * 1024) {
            AMG_TRY_CUDA(cudaFuncSetAttribute(sym_bitmap_kernel<false>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            AMG_TRY_CUDA(cudaFuncSetAttribute(sym_bitmap_kernel<true>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        }
        sym_bitmap_kernel<false><<<std::min(nlong, 8192), SYM_T, smem, s>>>(
            xrp, xcol, yrp, ycol, ncols, ovf, nlong, cnt, nullptr, nullptr);
        ::amg::count_launch(1);
        AMG_TRY_CUDA(cudaGetLastError());
    }
    int total = 0;
    AMG_TRY(exclusive_scan_i32(cnt, crp, nrows, &total, tmp, s));
    AMG_TRY(keep.alloc_n(&ccol, (size_t)std::max(total, 1)));
    if (nrows > 0) {
        sym_small_kernel<true><<<nblk(nrows), T1D, 0, s>>>(xrp, xcol, yrp, ycol, nrows, cnt, crp,
                                                           ccol, islong, nullptr, nullptr);
        ::amg::count_launch(1);
        AMG_TRY_CUDA(cudaGetLastError());
    }
    if (nlong > 0) {
        sym_bitmap_kernel<true><<<std::min(nlong, 8192), SYM_T, smem, s>>>(
            xrp, xcol, yrp, ycol, ncols, ovf, nlong, cnt, crp, ccol);
        ::amg::count_launch(1);
        AMG_TRY_CUDA(cudaGetLastError());
    }
    tmp.release(cnt);
    tmp.release(ovf);
    tmp.release(islong);
    tmp.release(novf);
    *crp_out = crp;
    *ccol_out = ccol;
    *nnz_out = total;
    return AMG_OK;
}

__global__ void block_rows_kernel(const int *__restrict__ rp, int nbr, int *__restrict__ brow)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nbr) return;
    for (int p = rp[I]; p < rp[I + 1]; ++p) brow[p] = I;
}

// P block (I, a) = [a == agg(I)] Pt_I - diag(omega / d) sum_{J: agg(J) = a}
// A_IJ Pt_J, sums over J ascending then the inner index.
template <int B, int NS>
__global__ void p_values_kernel(const int *__restrict__ rp, const int *__restrict__ col,
                                const double *__restrict__ val, const uint8_t *__restrict__ strong,
                                const int *__restrict__ agg, const double *__restrict__ ptent,
                                const double *__restrict__ d, double omega,
                                const int *__restrict__ pbrow, const int *__restrict__ pcol,
                                int64_t nnzp, double *__restrict__ pval)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nnzp) return;
    const int I = pbrow[k], a = pcol[k];
    double acc[B][NS];
#pragma unroll
    for (int r = 0; r < B; ++r)
#pragma unroll
        for (int q = 0; q < NS; ++q) acc[r][q] = 0.0;
    for (int p = rp[I]; p < rp[I + 1]; ++p) {
        const int J = col[p];
        if (agg[J] != a) continue;
        const double *blk = val + (int64_t)p * B * B;
        const double *pt = ptent + (int64_t)J * B * NS;
#pragma unroll
        for (int r = 0; r < B; ++r)
#pragma unroll
            for (int c = 0; c < B; ++c) {
                const double af = blk[r * B + c];
#pragma unroll
                for (int q = 0; q < NS; ++q) acc[r][q] += af * pt[c * NS + q];
            }
    }
    const bool own = agg[I] == a;
#pragma unroll
    for (int r = 0; r < B; ++r) {
        const double dr = d[(int64_t)I * B + r];
        const double sc = (dr != 0.0) ? omega / dr : 0.0;
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const double pt = own ? ptent[((int64_t)I * B + r) * NS + q] : 0.0;
            pval[k * B * NS + r * NS + q] = pt - sc * acc[r][q];
        }
    }
}

// The same values with one CTA per block row I: the slot of agg(J) among the
// columns of P's row I is found once per block of A's row (in shared
// memory), then the threads take the (P block, r, q) entries of the row and
// walk the staged slots; every entry sees the same FMA sequence as above
// (blocks of A's row ascending, then c), so the bits are the same.
constexpr int PV_CT = 128;
template <int B, int NS>
__global__ void __launch_bounds__(PV_CT) p_values_cta_kernel(
    const int *__restrict__ rp, const int *__restrict__ col, const double *__restrict__ val,
    const int *__restrict__ agg, const double *__restrict__ ptent, const double *__restrict__ d,
    double omega, const int *__restrict__ prp, const int *__restrict__ pcol,
    double *__restrict__ pval)
{
    extern __shared__ int slot[];  // [longest row of A]
    const int I = blockIdx.x, tid = threadIdx.x;
    const int a0 = rp[I], na = rp[I + 1] - a0;
    const int p0 = prp[I], np = prp[I + 1] - p0;
    for (int t = tid; t < na; t += PV_CT) {
        const int g = agg[col[a0 + t]];
        const int pos = g >= 0 ? find_sorted(pcol, p0, p0 + np, g) : p0 + np;
        slot[t] = (pos < p0 + np && pcol[pos] == g) ? pos - p0 : -1;
    }
    __syncthreads();
    const int gI = agg[I];
    for (int task = tid; task < np * B * NS; task += PV_CT) {
        const int sl = task / (B * NS), e = task % (B * NS), r = e / NS, q = e % NS;
        double acc = 0.0;
        for (int t = 0; t < na; ++t) {
            if (slot[t] != sl) continue;
            const double *blk = val + (int64_t)(a0 + t) * B * B + r * B;
            const double *pt = ptent + (int64_t)col[a0 + t] * B * NS + q;
#pragma unroll
            for (int c = 0; c < B; ++c) acc += blk[c] * pt[c * NS];
        }
        const double dr = d[(int64_t)I * B + r];
        const double sc = (dr != 0.0) ? omega / dr : 0.0;
        const double own = (gI == pcol[p0 + sl]) ? ptent[((int64_t)I * B + r) * NS + q] : 0.0;
        pval[(int64_t)(p0 + sl) * B * NS + e] = own - sc * acc;
    }
}

// The same per-row product for rows of at most 32 blocks (the finest level,
// 27 on a hex mesh): the row's A blocks and the tentative blocks of its
// columns are staged in shared memory, and the first warp sorts the row's
// entries by output block (each lane one entry: its rank among the entries
// of the same output block by __match_any_sync, the blocks' offsets by a warp
// scan of their counts), so each output entry runs over the entries of its
// own block only, in ascending order.  In p_values_cta_kernel every task
// scanned the whole row, and the FMAs of the tasks of a warp (two or three
// output blocks) were issued once per entry of any of them: the FP64 pipe
// spent several times the products' work.  The same terms in the same order
// as there (the same bits).  One CTA of PV_ST threads per block row.
constexpr int PV_ST = 64;
template <int B, int NS>
__global__ void __launch_bounds__(PV_ST) p_values_staged_kernel(
    const int *__restrict__ rp, const int *__restrict__ col, const double *__restrict__ val,
    const int *__restrict__ agg, const double *__restrict__ ptent, const double *__restrict__ d,
    double omega, const int *__restrict__ prp, const int *__restrict__ pcol,
    double *__restrict__ pval)
{
    __shared__ double sa[32 * B * B], sp[32 * B * NS];
    __shared__ int list[32], first[33];
    const int I = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
    const int a0 = rp[I], na = rp[I + 1] - a0;  // <= 32 (checked on the host)
    const int p0 = prp[I], np = prp[I + 1] - p0;  // <= na
    for (int e = tid; e < na * B * B; e += PV_ST) sa[e] = val[(int64_t)a0 * B * B + e];
    for (int e = tid; e < na * B * NS; e += PV_ST) {
        const int t = e / (B * NS);
        sp[e] = ptent[(int64_t)col[a0 + t] * B * NS + e % (B * NS)];
    }
    if (tid < 32) {
        int sl = -1;
        if (lane < na) {
            const int g = agg[col[a0 + lane]];
            const int pos = g >= 0 ? find_sorted(pcol, p0, p0 + np, g) : p0 + np;
            sl = (pos < p0 + np && pcol[pos] == g) ? pos - p0 : -1;
        }
        const unsigned same = __match_any_sync(0xffffffffu, sl);
        const int rank = __popc(same & ((1u << lane) - 1u));
        // entries per output block (lane s counts block s), then offsets
        int cnt = 0;
        for (int t = 0; t < na; ++t) cnt += (__shfl_sync(0xffffffffu, sl, t) == lane) ? 1 : 0;
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        first[lane + 1] = incl;
        if (lane == 0) first[0] = 0;
        __syncwarp();
        if (sl >= 0) list[first[sl] + rank] = lane;
    }
    __syncthreads();
    const int gI = agg[I];
    for (int task = tid; task < np * B * NS; task += PV_ST) {
        const int sl = task / (B * NS), e = task % (B * NS), r = e / NS, q = e % NS;
        double acc = 0.0;
        for (int j = first[sl]; j < first[sl + 1]; ++j) {
            const int t = list[j];
            const double *blk = sa + t * B * B + r * B;
            const double *pt = sp + t * B * NS + q;
#pragma unroll
            for (int c = 0; c < B; ++c) acc += blk[c] * pt[c * NS];
        }
        const double dr = d[(int64_t)I * B + r];
        const double sc = (dr != 0.0) ? omega / dr : 0.0;
        const double own = (gI == pcol[p0 + sl]) ? ptent[((int64_t)I * B + r) * NS + q] : 0.0;
        pval[(int64_t)(p0 + sl) * B * NS + e] = own - sc * acc;
    }
}

// ---------------------------------------------------------------- transpose
__global__ void col_count_kernel(const int *__restrict__ col, int64_t nnz, int *__restrict__ cnt)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < nnz) atomicAdd(cnt + col[k], 1);
}

__global__ void transpose_scatter_kernel(const int *__restrict__ brow, const int *__restrict__ col,
                                         int64_t nnz, const int *__restrict__ trp,
                                         int *__restrict__ fill, int *__restrict__ tcol,
                                         int *__restrict__ tsrc)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nnz) return;
    const int c = col[k];
    const int pos = trp[c] + atomicAdd(fill + c, 1);
    tcol[pos] = brow[k];
    tsrc[pos] = (int)k;
}

// Sort each transposed row by column (the scatter order is arbitrary): the
// result does not depend on the order of the atomics.
constexpr int RSORT_MAX = 32;        // rows up to this length: insertion sort per thread
constexpr int RSORT_CTA_MAX = 4096;  // longer rows up to this: rank sort per CTA

__global__ void row_sort_kernel(const int *__restrict__ trp, int nrows, int *__restrict__ tcol,
                                int *__restrict__ tsrc)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    const int lo = trp[r], hi = trp[r + 1];
    if (hi - lo > RSORT_MAX && hi - lo <= RSORT_CTA_MAX) return;  // row_rank_sort_kernel
    for (int i = lo + 1; i < hi; ++i) {
        const int c = tcol[i], s = tsrc[i];
        int j = i - 1;
        while (j >= lo && tcol[j] > c) {
            tcol[j + 1] = tcol[j];
            tsrc[j + 1] = tsrc[j];
            --j;
        }
        tcol[j + 1] = c;
        tsrc[j + 1] = s;
    }
}

// Long rows: one CTA per row, keys staged in shared memory, every entry's
// rank = the number of smaller keys (the keys of a row are distinct).
__global__ void __launch_bounds__(256) row_rank_sort_kernel(const int *__restrict__ trp, int nrows,
                                                            int *__restrict__ tcol,
                                                            int *__restrict__ tsrc)
{
    __shared__ int kc[RSORT_CTA_MAX], ks[RSORT_CTA_MAX];
    for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int lo = trp[r], n = trp[r + 1] - lo;
        if (n <= RSORT_MAX || n > RSORT_CTA_MAX) continue;  // block-uniform
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            kc[i] = tcol[lo + i];
            ks[i] = tsrc[lo + i];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int c = kc[i];
            int rank = 0;
            for (int j = 0; j < n; ++j) rank += kc[j] < c;
            tcol[lo + rank] = c;
            tsrc[lo + rank] = ks[i];
        }
        __syncthreads();
    }
}

// R block q = (P block src)^T : (BR x BC) -> (BC x BR)
__global__ void transpose_values_kernel(const int *__restrict__ tsrc, int64_t nnz, int br, int bc,
                                        const double *__restrict__ pval, double *__restrict__ rval)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nnz) return;
    const double *src = pval + (int64_t)tsrc[q] * br * bc;
    double *dst = rval + q * br * bc;
    for (int r = 0; r < br; ++r)
        for (int c = 0; c < bc; ++c) dst[c * br + r] = src[r * bc + c];
}

static int transpose_bsr(const BsrD &P, const int *pbrow, DevArena &keep, DevArena &tmp,
                         cudaStream_t s, BsrD *R)
{
    R->nbr = P.nbc;
    R->nbc = P.nbr;
    R->br = P.bc;
    R->bc = P.br;
    R->nnzb = P.nnzb;
    int *cnt = nullptr, *fill = nullptr, *tsrc = nullptr;
    AMG_TRY(tmp.alloc_n(&cnt, (size_t)R->nbr + 1));
    AMG_TRY(tmp.alloc_n(&fill, (size_t)R->nbr + 1));
    AMG_TRY(tmp.alloc_n(&tsrc, (size_t)std::max<int64_t>(P.nnzb, 1)));
    AMG_TRY(keep.alloc_n(&R->row_ptr, (size_t)R->nbr + 1));
    AMG_TRY(keep.alloc_n(&R->col, (size_t)std::max<int64_t>(P.nnzb, 1)));
    AMG_TRY(keep.alloc_n(&R->val, (size_t)std::max<int64_t>(P.nnzb, 1) * P.br * P.bc));
    AMG_TRY_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (R->nbr + 1), s));
    AMG_TRY_CUDA(cudaMemsetAsync(fill, 0, sizeof(int) * (R->nbr + 1), s));
    if (P.nnzb > 0) {
        col_count_kernel<<<nblk(P.nnzb), T1D, 0, s>>>(P.col, P.nnzb, cnt); ::amg::count_launch(1);
        AMG_TRY_CUDA(cudaGetLastError());
    }
    int total = 0;
    AMG_TRY(exclusive_scan_i32(cnt, R->row_ptr, R->nbr, &total, tmp, s));
    if (P.nnzb > 0) {
        transpose_scatter_kernel<<<nblk(P.nnzb), T1D, 0, s>>>(pbrow, P.col, P.nnzb, R->row_ptr,
                                                               fill, R->col, tsrc); ::amg::count_launch(1);
        row_sort_kernel<<<nblk(R->nbr), T1D, 0, s>>>(R->row_ptr, R->nbr, R->col, tsrc); ::amg::count_launch(1);
        row_rank_sort_kernel<<<std::max(1, std::min(R->nbr, 8192)), 256, 0, s>>>(R->row_ptr, R->nbr, R->col, tsrc); ::amg::count_launch(1);
        transpose_values_kernel<<<nblk(P.nnzb), T1D, 0, s>>>(tsrc, P.nnzb, P.br, P.bc, P.val,
                                                              R->val); ::amg::count_launch(1);
        AMG_TRY_CUDA(cudaGetLastError());
    }
    tmp.release(cnt);
    tmp.release(fill);
    tmp.release(tsrc);
    return AMG_OK;
}

// ---------------------------------------------------------------- SpGEMM
// C block (i, j) = sum over X row i (ascending) of X_ik Y_kj; blocks XR x XC
// and XC x YC, the inner sums over k ascending then the inner index.
template <int XR, int XC, int YC>
__global__ void spgemm_values_kernel(const int *__restrict__ xrp, const int *__restrict__ xcol,
                                     const double *__restrict__ xval, const int *__restrict__ yrp,
                                     const int *__restrict__ ycol, const double *__restrict__ yval,
                                     const int *__restrict__ cbrow, const int *__restrict__ ccol,
                                     int64_t nnzc, int upper, double *__restrict__ cval)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nnzc) return;
    const int i = cbrow[q], j = ccol[q];
    if (upper && j < i) {  // filled from block (j, i) by mirror_lower_kernel
#pragma unroll
        for (int e = 0; e < XR * YC; ++e) cval[q * XR * YC + e] = 0.0;
        return;
    }
    double acc[XR][YC];
#pragma unroll
    for (int r = 0; r < XR; ++r)
#pragma unroll
        for (int c = 0; c < YC; ++c) acc[r][c] = 0.0;
    for (int p = xrp[i]; p < xrp[i + 1]; ++p) {
        const int k = xcol[p];
        const int lo = yrp[k], hi = yrp[k + 1];
        const int t = find_sorted(ycol, lo, hi, j);
        if (t >= hi || ycol[t] != j) continue;
        const double *xb = xval + (int64_t)p * XR * XC;
        const double *yb = yval + (int64_t)t * XC * YC;
#pragma unroll
        for (int r = 0; r < XR; ++r)
#pragma unroll
            for (int m = 0; m < XC; ++m) {
                const double xv = xb[r * XC + m];
#pragma unroll
                for (int c = 0; c < YC; ++c) acc[r][c] += xv * yb[m * YC + c];
            }
    }
#pragma unroll
    for (int r = 0; r < XR; ++r)
#pragma unroll
        for (int c = 0; c < YC; ++c) cval[q * XR * YC + r * YC + c] = acc[r][c];
}

// C = X Y by rows (Gustavson), L lanes per output row.  The row's columns
// (from the symbolic pass) and its block accumulators sit in shared memory;
// X row i is walked in ascending order, and for each X_ik the lanes take the
// entries of Y row k (distinct columns, so no two lanes touch the same
// accumulator) and add X_ik Y_kj into the block of column j, found by a
// binary search in the shared column list.  Every accumulator entry sees
// the same FMA sequence as in spgemm_values_kernel (k ascending, then the
// inner index), so both kernels give the same bits; this one does no search
// in Y's rows and no work for the (k, j) pairs that do not exist.
template <int XR, int XC, int YC, int L>
__global__ void __launch_bounds__(128) spgemm_rows_kernel(
    const int *__restrict__ xrp, const int *__restrict__ xcol, const double *__restrict__ xval,
    const int *__restrict__ yrp, const int *__restrict__ ycol, const double *__restrict__ yval,
    const int *__restrict__ crp, const int *__restrict__ ccol, int nrows, int cmax, int upper,
    double *__restrict__ cval)
{
    constexpr int CB = XR * YC;
    extern __shared__ double sm[];
    const int GROUPS = blockDim.x / L;
    const int g = threadIdx.x / L, lane = threadIdx.x % L;
    const unsigned mask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << ((threadIdx.x & 31) / L * L));
    double *acc = sm + (size_t)g * cmax * CB;
    int *cols = reinterpret_cast<int *>(sm + (size_t)GROUPS * cmax * CB) + (size_t)g * cmax;
    for (int i = blockIdx.x * GROUPS + g; i < nrows; i += gridDim.x * GROUPS) {
        // upper: only the blocks on and above the diagonal, columns >= i (the
        // row's tail) are kept; cmax is then the longest such tail
        const int r0 = crp[i], r1 = crp[i + 1];
        const int c0 = upper ? find_sorted(ccol, r0, r1, i) : r0, len = r1 - c0;
        for (int t = lane; t < len; t += L) cols[t] = ccol[c0 + t];
        for (int t = lane; t < len * CB; t += L) acc[t] = 0.0;
        __syncwarp(mask);
        for (int p = xrp[i]; p < xrp[i + 1]; ++p) {
            const int k = xcol[p];
            double xb[XR * XC];
#pragma unroll
            for (int e = 0; e < XR * XC; ++e) xb[e] = xval[(int64_t)p * XR * XC + e];
            const int hi = yrp[k + 1];
            const int lo = upper ? find_sorted(ycol, yrp[k], hi, i) : yrp[k];
            for (int t = lo + lane; t < hi; t += L) {
                const int j = ycol[t];
                const int pos = find_sorted(cols, 0, len, j);
                if (pos >= len || cols[pos] != j) continue;  // cannot happen: C holds every product
                const double *yb = yval + (int64_t)t * XC * YC;
                double *a = acc + (size_t)pos * CB;
#pragma unroll
                for (int r = 0; r < XR; ++r)
#pragma unroll
                    for (int c = 0; c < YC; ++c) {
                        double v = a[r * YC + c];
#pragma unroll
                        for (int m = 0; m < XC; ++m) v += xb[r * XC + m] * yb[m * YC + c];
                        a[r * YC + c] = v;
                    }
            }
            __syncwarp(mask);
        }
        for (int t = lane; t < len * CB; t += L) cval[(int64_t)c0 * CB + t] = acc[t];
        if (upper)  // lower blocks: zero here, mirror_lower_kernel fills them
            for (int t = lane; t < (c0 - r0) * CB; t += L) cval[(int64_t)r0 * CB + t] = 0.0;
        __syncwarp(mask);
    }
}

// C = X Y for few, long rows (the coarse levels): gridDim.y CTAs per output
// row, each holding a contiguous share of the row's output blocks as
// accumulators in shared memory and taking from Y row k only the entries
// whose columns fall in its share (with fewer than four rows per SM one CTA a
// row left most SMs idle: 161 rows of the 80^3 level-2 R (A P) took 5.2 ms).
// For each X_ik, k ascending, the threads first locate those columns of Y
// row k in the share, then take its (block, entry) pairs, so every
// accumulator entry sees the same FMA sequence as in the kernels above (k
// ascending, then the inner index) and gets the same bits, whatever the
// split.
constexpr int SPG_CT = 256;
template <int XR, int XC, int YC>
__global__ void __launch_bounds__(SPG_CT) spgemm_cta_kernel(
    const int *__restrict__ xrp, const int *__restrict__ xcol, const double *__restrict__ xval,
    const int *__restrict__ yrp, const int *__restrict__ ycol, const double *__restrict__ yval,
    const int *__restrict__ crp, const int *__restrict__ ccol, int cmax, int ymax, int upper,
    double *__restrict__ cval)
{
    constexpr int CB = XR * YC, XB = XR * XC, YB = XC * YC;
    extern __shared__ double sm[];
    double *acc = sm;                                     // [cmax * CB] (cmax: a share's bound)
    double *xb = sm + (size_t)cmax * CB;                  // [XB]
    int *cols = reinterpret_cast<int *>(xb + XB);         // [cmax]
    int *ypos = cols + cmax;                              // [ymax]
    const int i = blockIdx.x, tid = threadIdx.x, nsh = gridDim.y, sh = blockIdx.y;
    const int r0 = crp[i], r1 = crp[i + 1];
    const int c0 = upper ? find_sorted(ccol, r0, r1, i) : r0, full = r1 - c0;
    if (upper && sh == 0)  // lower blocks: zero here, mirror_lower_kernel fills them
        for (int t = tid; t < (c0 - r0) * CB; t += SPG_CT) cval[(int64_t)r0 * CB + t] = 0.0;
    const int q0 = (int)((int64_t)full * sh / nsh), q1 = (int)((int64_t)full * (sh + 1) / nsh);
    const int len = q1 - q0;  // <= cmax; the same for the whole CTA
    if (len <= 0) return;
    const int cfirst = ccol[c0 + q0], clast = ccol[c0 + q1 - 1];
    for (int t = tid; t < len; t += SPG_CT) cols[t] = ccol[c0 + q0 + t];
    for (int t = tid; t < len * CB; t += SPG_CT) acc[t] = 0.0;
    __syncthreads();
    for (int p = xrp[i]; p < xrp[i + 1]; ++p) {
        const int k = xcol[p];
        // Y row k's entries in the share's column range (the whole row, or
        // its tail from column i, when one CTA holds the row)
        int lo = yrp[k], hi = yrp[k + 1];
        if (nsh > 1 || upper) lo = find_sorted(ycol, lo, hi, cfirst);
        if (nsh > 1) hi = find_sorted(ycol, lo, hi, clast + 1);
        const int ny = hi - lo;  // <= ymax; the same for the whole CTA
        if (ny == 0) continue;
        if (tid < XB) xb[tid] = xval[(int64_t)p * XB + tid];
        for (int t = tid; t < ny; t += SPG_CT) {
            const int j = ycol[lo + t];
            const int pos = find_sorted(cols, 0, len, j);
            ypos[t] = (pos < len && cols[pos] == j) ? pos : -1;  // -1 cannot happen
        }
        __syncthreads();
        for (int task = tid; task < ny * CB; task += SPG_CT) {
            const int t = task / CB, e = task % CB;
            const int pos = ypos[t];
            if (pos < 0) continue;
            const int r = e / YC, c = e % YC;
            const double *yb = yval + (int64_t)(lo + t) * YB;
            double v = acc[(size_t)pos * CB + e];
#pragma unroll
            for (int m = 0; m < XC; ++m) v += xb[r * XC + m] * yb[m * YC + c];
            acc[(size_t)pos * CB + e] = v;
        }
        __syncthreads();
    }
    for (int t = tid; t < len * CB; t += SPG_CT) cval[(int64_t)(c0 + q0) * CB + t] = acc[t];
}

// shares per row: one CTA a row with four or more rows per SM, else enough
// shares for about four CTAs per SM (at most 16); more when a share's
// accumulators would not fit in 200 KB of shared memory (rows longer than
// that otherwise go to the per-block kernel)
template <int XR, int XC, int YC>
static int spgemm_cta(const BsrD &X, const BsrD &Y, BsrD *C, int cmax, int ymax, int upper,
                      cudaStream_t s, bool *done)
{
    constexpr int CB = XR * YC, XB = XR * XC;
    *done = false;
    if (X.nbr == 0) {
        *done = true;
        return AMG_OK;
    }
    Geom g;
    AMG_TRY(query_geom(&g));
    int nsh = 1;
    if (X.nbr < 4 * g.num_sms) nsh = std::min(16, (4 * g.num_sms + X.nbr - 1) / X.nbr);
    nsh = std::max(1, std::min(nsh, std::max(cmax, 1)));
    size_t smem = 0;
    int cm = 0;
    for (;;) {
        cm = (cmax + nsh - 1) / nsh;
        smem = (size_t)cm * CB * sizeof(double) + XB * sizeof(double) +
               (size_t)(cm + ymax) * sizeof(int);
        if (smem <= 200 * 1024) break;
        if (nsh >= 64 || nsh >= cmax) return AMG_OK;  // the per-block kernel
        nsh *= 2;
    }
    auto kern = spgemm_cta_kernel<XR, XC, YC>;
    if (smem > 48 * 1024)
        AMG_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
    kern<<<dim3(X.nbr, nsh), SPG_CT, smem, s>>>(X.row_ptr, X.col, X.val, Y.row_ptr, Y.col, Y.val,
                                                C->row_ptr, C->col, cm, ymax, upper, C->val);
    ::amg::count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    *done = true;
    return AMG_OK;
}

// longest tail (columns >= row) of a row: the upper part of a symmetric product
__global__ void row_max_upper_kernel(const int *__restrict__ rp, const int *__restrict__ col, int n,
                                     int *__restrict__ mx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicMax(mx, rp[i + 1] - find_sorted(col, rp[i], rp[i + 1], i));
}

__global__ void row_max_kernel(const int *__restrict__ rp, int n, int *__restrict__ mx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicMax(mx, rp[i + 1] - rp[i]);
}

template <int XR, int XC, int YC>
static int spgemm_rows(const BsrD &X, const BsrD &Y, BsrD *C, int cmax, int lanes, int upper,
                       cudaStream_t s, bool *done)
{
    constexpr int CB = XR * YC;
    *done = false;
    const size_t per = (size_t)cmax * (CB * sizeof(double) + sizeof(int));
    auto go = [&](auto kern, int L) -> int {
        const int groups = (int)std::min<size_t>(128 / L, (200 * 1024) / std::max<size_t>(per, 1));
        if (groups < 1) return AMG_OK;  // rows too long for shared memory: the per-block kernel
        const size_t smem = per * groups;
        if (smem > 48 * 1024)
            AMG_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
        const int grid = std::max(1, std::min((X.nbr + groups - 1) / groups, 1 << 20));
        kern<<<grid, groups * L, smem, s>>>(X.row_ptr, X.col, X.val, Y.row_ptr, Y.col, Y.val, C->row_ptr,
                                     C->col, X.nbr, cmax, upper, C->val);
        ::amg::count_launch(1);
        AMG_TRY_CUDA(cudaGetLastError());
        *done = true;
        return AMG_OK;
    };
    if (lanes <= 8) return go(spgemm_rows_kernel<XR, XC, YC, 8>, 8);
    if (lanes <= 16) return go(spgemm_rows_kernel<XR, XC, YC, 16>, 16);
    return go(spgemm_rows_kernel<XR, XC, YC, 32>, 32);
}

// Lower blocks of a product known to be symmetric: C_ij = C_ji^T, one warp
// per block row, the lanes over its lower blocks.
template <int BS>
__global__ void mirror_lower_kernel(const int *__restrict__ crp, const int *__restrict__ ccol,
                                    int nrows, double *__restrict__ cval)
{
    const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= nrows) return;
    for (int q = crp[i] + lane; q < crp[i + 1]; q += 32) {
        const int j = ccol[q];
        if (j >= i) break;  // columns ascend: the rest of this lane's blocks are upper
        const int lo = crp[j], hi = crp[j + 1];
        const int t = find_sorted(ccol, lo, hi, i);
        if (t >= hi || ccol[t] != i) continue;  // cannot happen for a symmetric pattern
        const double *src = cval + (int64_t)t * BS * BS;
        double *dst = cval + (int64_t)q * BS * BS;
#pragma unroll
        for (int r = 0; r < BS; ++r)
#pragma unroll
            for (int c = 0; c < BS; ++c) dst[r * BS + c] = src[c * BS + r];
    }
}

// C = X Y.  symmetric: C is known to be symmetric (the Galerkin product
// R (A P) with R = P^T and A symmetric): only the blocks on and above the
// diagonal are computed, the others are their transposes.
static int spgemm(const BsrD &X, const BsrD &Y, DevArena &keep, DevArena &tmp, cudaStream_t s,
                  BsrD *C, bool symmetric = false)
{
    C->nbr = X.nbr;
    C->nbc = Y.nbc;
    C->br = X.br;
    C->bc = Y.bc;
    int total = 0;
    AMG_TRY(spgemm_symbolic(X.row_ptr, X.col, X.nbr, Y.row_ptr, Y.col, Y.nbc, keep, tmp, s,
                            &C->row_ptr, &C->col, &total));
    C->nnzb = total;
    AMG_TRY(keep.alloc_n(&C->val, (size_t)std::max(total, 1) * C->br * C->bc));
    if (total == 0) return AMG_OK;
    const int xr = X.br, xc = X.bc, yc = Y.bc;
    if (!((xr == 3 && xc == 3 && yc == 6) || (xr == 6 && xc == 6 && yc == 6) ||
          (xr == 6 && xc == 3 && yc == 6) || (xr == 3 && xc == 3 && yc == 3) ||
          (xr == 1 && xc == 1 && yc == 1))) {
        set_error("unsupported block product %dx%d * %dx%d", xr, xc, X.bc, yc);
        return AMG_ERR_ARG;
    }
    // rows of C in shared memory, lanes per row ~ the mean length of Y's rows;
    // only when there are rows enough to fill the GPU (on the 80^3 hierarchy
    // the row kernel took 12 / 30 / 18 ms for the three products with 22k+
    // rows against 20 / 36 / 28 ms, and lost on the ones with 1694 and 141)
    const int upper = (symmetric && xr == yc && X.nbr == Y.nbc) ? 1 : 0;
    bool done = false;
    const double xlen = X.nbr ? (double)X.nnzb / X.nbr : 0.0;
    if (X.nbr < 16384 || (xlen >= 32.0 && xr > 1)) {
        // few rows, or long X rows (the restrictions and the coarse A P):
        // one CTA per output row (the shared-memory row must fit)
        int *mx = nullptr, hm[2] = {0, 0};
        AMG_TRY(tmp.alloc_n(&mx, 2));
        AMG_TRY_CUDA(cudaMemsetAsync(mx, 0, 2 * sizeof(int), s));
        if (upper)
            row_max_upper_kernel<<<nblk(X.nbr), T1D, 0, s>>>(C->row_ptr, C->col, X.nbr, mx);
        else
            row_max_kernel<<<nblk(X.nbr), T1D, 0, s>>>(C->row_ptr, X.nbr, mx);
        if (Y.nbr > 0) row_max_kernel<<<nblk(Y.nbr), T1D, 0, s>>>(Y.row_ptr, Y.nbr, mx + 1);
        ::amg::count_launch(Y.nbr > 0 ? 2 : 1);
        AMG_TRY_CUDA(cudaMemcpyAsync(hm, mx, sizeof(hm), cudaMemcpyDeviceToHost, s));
        AMG_TRY_CUDA(cudaStreamSynchronize(s));
        tmp.release(mx);
        if (xr == 1) AMG_TRY((spgemm_cta<1, 1, 1>(X, Y, C, hm[0], hm[1], upper, s, &done)));
        else if (xr == 3 && yc == 3) AMG_TRY((spgemm_cta<3, 3, 3>(X, Y, C, hm[0], hm[1], upper, s, &done)));
        else if (xr == 3) AMG_TRY((spgemm_cta<3, 3, 6>(X, Y, C, hm[0], hm[1], upper, s, &done)));
        else if (xc == 6) AMG_TRY((spgemm_cta<6, 6, 6>(X, Y, C, hm[0], hm[1], upper, s, &done)));
        else AMG_TRY((spgemm_cta<6, 3, 6>(X, Y, C, hm[0], hm[1], upper, s, &done)));
        if (done) goto mirror;
        if (X.nbr < 16384) goto per_block;
    }
    {
    int *mx = nullptr, cmax = 0;
    AMG_TRY(tmp.alloc_n(&mx, 1));
    AMG_TRY_CUDA(cudaMemsetAsync(mx, 0, sizeof(int), s));
    if (upper)
        row_max_upper_kernel<<<nblk(X.nbr), T1D, 0, s>>>(C->row_ptr, C->col, X.nbr, mx);
    else
        row_max_kernel<<<nblk(X.nbr), T1D, 0, s>>>(C->row_ptr, X.nbr, mx);
    ::amg::count_launch(1);
    AMG_TRY_CUDA(cudaMemcpyAsync(&cmax, mx, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    tmp.release(mx);
    // an upper product uses about half of each Y row
    const double ylen = (Y.nbr ? (double)Y.nnzb / Y.nbr : 0.0) * (upper ? 0.5 : 1.0);
    const int lanes = ylen <= 8.0 ? 8 : (ylen <= 16.0 ? 16 : 32);
    if (xr == 1) AMG_TRY((spgemm_rows<1, 1, 1>(X, Y, C, cmax, lanes, upper, s, &done)));
    else if (xr == 3 && yc == 3) AMG_TRY((spgemm_rows<3, 3, 3>(X, Y, C, cmax, lanes, upper, s, &done)));
    else if (xr == 3) AMG_TRY((spgemm_rows<3, 3, 6>(X, Y, C, cmax, lanes, upper, s, &done)));
    else if (xc == 6) AMG_TRY((spgemm_rows<6, 6, 6>(X, Y, C, cmax, lanes, upper, s, &done)));
    else AMG_TRY((spgemm_rows<6, 3, 6>(X, Y, C, cmax, lanes, upper, s, &done)));
    if (done) goto mirror;
    }
per_block:
    {
    int *cbrow = nullptr;
    AMG_TRY(tmp.alloc_n(&cbrow, (size_t)std::max(total, 1)));
    if (X.nbr > 0) {
        block_rows_kernel<<<nblk(X.nbr), T1D, 0, s>>>(C->row_ptr, X.nbr, cbrow);
        ::amg::count_launch(1);
    }
    AMG_TRY_CUDA(cudaGetLastError());
    const int g = nblk(total, 128);
#define AMG_SPGEMM_VALS(XR_, XC_, YC_)                                                       \
    spgemm_values_kernel<XR_, XC_, YC_><<<g, 128, 0, s>>>(X.row_ptr, X.col, X.val, Y.row_ptr, \
                                                          Y.col, Y.val, cbrow, C->col, total, \
                                                          upper, C->val)
    if (xr == 1) AMG_SPGEMM_VALS(1, 1, 1);
    else if (xr == 3 && yc == 3) AMG_SPGEMM_VALS(3, 3, 3);
    else if (xr == 3) AMG_SPGEMM_VALS(3, 3, 6);
    else if (xc == 6) AMG_SPGEMM_VALS(6, 6, 6);
    else AMG_SPGEMM_VALS(6, 3, 6);
    ::amg::count_launch(1);
#undef AMG_SPGEMM_VALS
    AMG_TRY_CUDA(cudaGetLastError());
    tmp.release(cbrow);
    }
mirror:
    if (upper) {
        const int mg = nblk((int64_t)X.nbr * 32);
        if (yc == 1)
            mirror_lower_kernel<1><<<mg, T1D, 0, s>>>(C->row_ptr, C->col, X.nbr, C->val);
        else if (yc == 3)
            mirror_lower_kernel<3><<<mg, T1D, 0, s>>>(C->row_ptr, C->col, X.nbr, C->val);
        else
            mirror_lower_kernel<6><<<mg, T1D, 0, s>>>(C->row_ptr, C->col, X.nbr, C->val);
        ::amg::count_launch(1);
        AMG_TRY_CUDA(cudaGetLastError());
    }
    return AMG_OK;
}

// Galerkin operator A_c = R (A P) (Alg. 1), block SpGEMM twice.
int galerkin(const BsrD &A, const BsrD &P, const BsrD &R, DevArena &keep, DevArena &tmp,
             cudaStream_t s, BsrD *Ac)
{
    BsrD AP;
    DevArena apmem;
    apmem.stream = s;
    int st = spgemm(A, P, apmem, tmp, s, &AP);
    if (st >= 0) st = spgemm(R, AP, keep, tmp, s, Ac, true);
    apmem.release_all();
    return st;
}

// The same Galerkin product in scalar arithmetic (the scalar setup of the
// Sec. 4 comparison): A, P and R unblocked to scalar CSR (every entry of
// their blocks, explicit zeros kept, so the scalar product has the unblocked
// block product's pattern), then the two SpGEMMs with 1x1 blocks.
int galerkin_scalar(const BsrD &A, const BsrD &P, const BsrD &R, DevArena &keep, DevArena &tmp,
                    cudaStream_t s, BsrD *Ac)
{
    BsrD uA, uP, uR;
    DevArena um;
    um.stream = s;
    int st = unblock_bsr(A, um, s, &uA);
    if (st >= 0) st = unblock_bsr(P, um, s, &uP);
    if (st >= 0) st = unblock_bsr(R, um, s, &uR);
    if (st >= 0) st = galerkin(uA, uP, uR, keep, tmp, s, Ac);
    cudaStreamSynchronize(s);
    um.release_all();
    return st;
}

// ---------------------------------------------------------------- transfer operators
int build_transfer(const BsrD &A, const double *B, int ns, const uint8_t *strong,
                   const int *agg_h, int nagg, double relax, DevArena &keep, DevArena &tmp,
                   cudaStream_t s, LevelBuild *out)
{
    const int nn = A.nbr, b = A.br;
    // aggregate membership lists (ascending node order) from the host aggregation
    std::vector<int> aptr(nagg + 1, 0), mem;
    for (int I = 0; I < nn; ++I)
        if (agg_h[I] >= 0) aptr[agg_h[I] + 1]++;
    for (int a = 0; a < nagg; ++a) aptr[a + 1] += aptr[a];
    mem.resize(std::max(aptr[nagg], 1));
    {
        std::vector<int> fill(aptr.begin(), aptr.end() - 1);
        for (int I = 0; I < nn; ++I)
            if (agg_h[I] >= 0) mem[fill[agg_h[I]]++] = I;
    }
    int *d_aptr = nullptr, *d_mem = nullptr;
    double *Qs = nullptr, *ptent = nullptr, *d = nullptr;
    unsigned long long *rho_bits = nullptr;
    AMG_TRY(tmp.alloc_n(&d_aptr, nagg + 1));
    AMG_TRY(tmp.alloc_n(&d_mem, mem.size()));
    AMG_TRY(keep.alloc_n(&out->agg, std::max(nn, 1)));
    AMG_TRY(tmp.alloc_n(&Qs, (size_t)std::max(aptr[nagg], 1) * b * ns));
    AMG_TRY(tmp.alloc_n(&ptent, (size_t)std::max(nn, 1) * b * ns));
    AMG_TRY(tmp.alloc_n(&d, (size_t)std::max(nn, 1) * b));
    AMG_TRY(tmp.alloc_n(&rho_bits, 1));
    AMG_TRY(keep.alloc_n(&out->Bc, (size_t)std::max(nagg, 1) * ns * ns));
    AMG_TRY_CUDA(cudaMemcpyAsync(d_aptr, aptr.data(), sizeof(int) * (nagg + 1),
                                 cudaMemcpyHostToDevice, s));
    AMG_TRY_CUDA(cudaMemcpyAsync(d_mem, mem.data(), sizeof(int) * mem.size(),
                                 cudaMemcpyHostToDevice, s));
    AMG_TRY_CUDA(cudaMemcpyAsync(out->agg, agg_h, sizeof(int) * nn, cudaMemcpyHostToDevice, s));
    AMG_TRY_CUDA(cudaMemsetAsync(ptent, 0, sizeof(double) * (size_t)nn * b * ns, s));
    AMG_TRY_CUDA(cudaMemsetAsync(rho_bits, 0, sizeof(unsigned long long), s));
    out->nagg = nagg;
    if (nagg > 0) {
        if (ns == 6)
            tentative_kernel<6><<<nblk((int64_t)nagg * 32), T1D, 0, s>>>(nagg, b, d_aptr, d_mem, B,
                                                                          Qs, ptent, out->Bc);
        else
            tentative_kernel<3><<<nblk((int64_t)nagg * 32), T1D, 0, s>>>(nagg, b, d_aptr, d_mem, B,
                                                                          Qs, ptent, out->Bc);
        ::amg::count_launch(1);
        AMG_TRY_CUDA(cudaGetLastError());
    }
    jacobi_rho_kernel<<<nblk((int64_t)nn * b), T1D, 0, s>>>(A.row_ptr, A.col, A.val, nn, b, d,
                                                            rho_bits);
    ::amg::count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    unsigned long long rb = 0;
    AMG_TRY_CUDA(cudaMemcpyAsync(&rb, rho_bits, sizeof(rb), cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));  // host vectors above go out of scope after this
    double rho;
    std::memcpy(&rho, &rb, sizeof rho);
    out->rho = rho;
    out->omega = (rho > 0.0) ? relax * (4.0 / 3.0) / rho : 0.0;

    // P pattern: the symbolic product of A's pattern with the tentative
    // prolongation's (one column, agg(J), per aggregated node J)
    BsrD &P = out->P;
    P.nbr = nn;
    P.nbc = nagg;
    P.br = b;
    P.bc = ns;
    std::vector<int> trp(nn + 1, 0), tcl;
    for (int J = 0; J < nn; ++J) {
        trp[J + 1] = trp[J] + (agg_h[J] >= 0 ? 1 : 0);
        if (agg_h[J] >= 0) tcl.push_back(agg_h[J]);
    }
    tcl.resize(std::max<size_t>(tcl.size(), 1));
    int *d_trp = nullptr, *d_tcl = nullptr;
    AMG_TRY(tmp.alloc_n(&d_trp, (size_t)nn + 1));
    AMG_TRY(tmp.alloc_n(&d_tcl, tcl.size()));
    AMG_TRY_CUDA(cudaMemcpyAsync(d_trp, trp.data(), sizeof(int) * (nn + 1), cudaMemcpyHostToDevice, s));
    AMG_TRY_CUDA(cudaMemcpyAsync(d_tcl, tcl.data(), sizeof(int) * tcl.size(), cudaMemcpyHostToDevice, s));
    int nnzp = 0;
    AMG_TRY(spgemm_symbolic(A.row_ptr, A.col, nn, d_trp, d_tcl, nagg, keep, tmp, s, &P.row_ptr,
                            &P.col, &nnzp));  // synchronises: trp/tcl may go out of scope
    P.nnzb = nnzp;
    int *pbrow = nullptr;
    AMG_TRY(keep.alloc_n(&P.val, (size_t)std::max(nnzp, 1) * b * ns));
    AMG_TRY(tmp.alloc_n(&pbrow, (size_t)std::max(nnzp, 1)));
    block_rows_kernel<<<nblk(nn), T1D, 0, s>>>(P.row_ptr, nn, pbrow); ::amg::count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    int amax = 0;  // longest row of A: the per-row kernel's staged slots
    if (nnzp > 0) {
        int *mx = nullptr;
        AMG_TRY(tmp.alloc_n(&mx, 1));
        AMG_TRY_CUDA(cudaMemsetAsync(mx, 0, sizeof(int), s));
        row_max_kernel<<<nblk(nn), T1D, 0, s>>>(A.row_ptr, nn, mx);
        ::amg::count_launch(1);
        AMG_TRY_CUDA(cudaMemcpyAsync(&amax, mx, sizeof(int), cudaMemcpyDeviceToHost, s));
        AMG_TRY_CUDA(cudaStreamSynchronize(s));
        tmp.release(mx);
    }
    if (nnzp > 0 && amax <= 32 && b == 3 && (ns == 6 || ns == 3)) {
        if (ns == 6)
            p_values_staged_kernel<3, 6><<<nn, PV_ST, 0, s>>>(
                A.row_ptr, A.col, A.val, out->agg, ptent, d, out->omega, P.row_ptr, P.col, P.val);
        else
            p_values_staged_kernel<3, 3><<<nn, PV_ST, 0, s>>>(
                A.row_ptr, A.col, A.val, out->agg, ptent, d, out->omega, P.row_ptr, P.col, P.val);
        ::amg::count_launch(1);
        AMG_TRY_CUDA(cudaGetLastError());
    } else if (nnzp > 0 && amax <= 12 * 1024) {
#define AMG_PVALS(B_, NS_)                                                                   \
    p_values_cta_kernel<B_, NS_><<<nn, PV_CT, sizeof(int) * amax, s>>>(                       \
        A.row_ptr, A.col, A.val, out->agg, ptent, d, out->omega, P.row_ptr, P.col, P.val)
        if (b == 3 && ns == 6) AMG_PVALS(3, 6);
        else if (b == 6 && ns == 6) AMG_PVALS(6, 6);
        else if (b == 3 && ns == 3) AMG_PVALS(3, 3);
        else {
            set_error("unsupported node block size %d with %d near-nullspace vectors", b, ns);
            return AMG_ERR_ARG;
        }
#undef AMG_PVALS
        ::amg::count_launch(1);
        AMG_TRY_CUDA(cudaGetLastError());
    } else if (nnzp > 0) {
#define AMG_PVALS(B_, NS_)                                                                   \
    p_values_kernel<B_, NS_><<<nblk(nnzp, 128), 128, 0, s>>>(A.row_ptr, A.col, A.val, strong,  \
                                                            out->agg, ptent, d, out->omega,    \
                                                            pbrow, P.col, nnzp, P.val)
        if (b == 3 && ns == 6) AMG_PVALS(3, 6);
        else if (b == 6 && ns == 6) AMG_PVALS(6, 6);
        else if (b == 3 && ns == 3) AMG_PVALS(3, 3);
        else {
            set_error("unsupported node block size %d with %d near-nullspace vectors", b, ns);
            return AMG_ERR_ARG;
        }
#undef AMG_PVALS
        ::amg::count_launch(1);
        AMG_TRY_CUDA(cudaGetLastError());
    }
    AMG_TRY(transpose_bsr(P, pbrow, keep, tmp, s, &out->R));
    tmp.release(d_aptr);
    tmp.release(d_mem);
    tmp.release(Qs);
    tmp.release(ptent);
    tmp.release(d);
    tmp.release(rho_bits);
    tmp.release(d_trp);
    tmp.release(d_tcl);
    tmp.release(pbrow);
    return AMG_OK;
}

// ---------------------------------------------------------------- SPAI0
// m_i = scale * a_ii / sum_j a_ij^2 over scalar row i (0 for an empty row).
__global__ void spai0_kernel(const int *__restrict__ rp, const int *__restrict__ col,
                             const double *__restrict__ val, int nbr, int b, double scale,
                             double *__restrict__ M)
{
    // one thread per scalar row (b per block row)
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nbr * b) return;
    const int I = (int)(i / b), r = (int)(i % b);
    const int bb = b * b;
    double dia = 0.0, s = 0.0;
    for (int p = rp[I]; p < rp[I + 1]; ++p)
        for (int c = 0; c < b; ++c) {
            const double v = val[(int64_t)p * bb + r * b + c];
            if (col[p] == I && c == r) dia = v;
            s += v * v;
        }
    const double m = (s != 0.0) ? dia / s : 0.0;
    M[i] = scale * m;
}

int spai0_diag(const BsrD &A, double scale, double *M, cudaStream_t s)
{
    if (A.nbr == 0) return AMG_OK;
    spai0_kernel<<<nblk((int64_t)A.nbr * A.br), T1D, 0, s>>>(A.row_ptr, A.col, A.val, A.nbr, A.br,
                                                             scale, M);
    ::amg::count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    return AMG_OK;
}

// ---------------------------------------------------------------- coarsest level
__global__ void densify_kernel(const int *__restrict__ brow, const int *__restrict__ col,
                               const double *__restrict__ val, int64_t nnzb, int b, int n,
                               double *__restrict__ D)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nnzb) return;
    const int I = brow[k], J = col[k];
    for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c)
            D[(int64_t)(I * b + r) * n + (J * b + c)] = val[k * b * b + r * b + c];
}

__global__ void zero_rows_kernel(const double *__restrict__ D, int n, uint8_t *__restrict__ z)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint8_t zr = 1;
    for (int j = 0; j < n; ++j)
        if (D[(int64_t)i * n + j] != 0.0) zr = 0;
    z[i] = zr;
}

// Blocked right-looking Cholesky in panels of CHOL_NB columns: the panel's
// diagonal block factored by one CTA, which also forms the inverse of that
// factor, the rows below it by a product with that inverse, then the trailing
// lower triangle updated by a tiled rank-CHOL_NB product.  A zero row (a
// dropped near-nullspace column) gets a unit pivot; a pivot <= 0 elsewhere
// records its column in *err.  Every step but the diagonal factor is a
// product spread over many CTAs: the FP64 rate of one SM is small, so a
// substitution chain per thread on a few SMs would dominate.
constexpr int CHOL_NB = 32;
constexpr int CHOL_TILE = 16;
constexpr int CHOL_W = CHOL_NB * CHOL_NB;  // doubles per diagonal-block inverse

// One CTA of 256 threads: the nb x nb diagonal block of panel c0 factored in
// shared memory (per column: scale of the column below the pivot, update of
// the trailing lower triangle), and W = L11^-1 formed alongside by the same
// row operations applied to the identity (row j scaled by the reciprocal
// pivot, then subtracted L[i][j] times from every row i > j).  Two barriers a
// column: thread 0 alone updates the next diagonal entry and at once takes
// its pivot (one reciprocal square root: d = s rsqrt(s), 1/d = rsqrt(s)),
// while the other threads update the rest, so the serial pivot overlaps the
// update.  L11 goes back to D; W goes to Wd as CHOL_NB x CHOL_NB, zero above
// the diagonal and past nb.
__device__ __forceinline__ void chol_pivot(double *diag, double *rp, int col, bool zero_row,
                                           int *err)
{
    double sj = *diag;
    if (zero_row) sj = 1.0;
    if (!(sj > 0.0)) {
        atomicExch(err, col + 1);
        sj = 1.0;
    }
    const double r = rsqrt(sj);
    *diag = sj * r;
    *rp = r;
}

__global__ void __launch_bounds__(256) chol_diag_kernel(double *__restrict__ D, int n, int c0,
                                                        int nb, const uint8_t *__restrict__ zrow,
                                                        int *__restrict__ err,
                                                        double *__restrict__ Wd)
{
    __shared__ double blk[CHOL_NB][CHOL_NB + 1], w[CHOL_NB][CHOL_NB + 1];
    __shared__ double rpiv[CHOL_NB];
    for (int t = threadIdx.x; t < CHOL_W; t += blockDim.x) {
        const int r = t / CHOL_NB, c = t % CHOL_NB;
        blk[r][c] = (r < nb && c <= r) ? D[(int64_t)(c0 + r) * n + c0 + c] : 0.0;
        w[r][c] = (r == c && r < nb) ? 1.0 : 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) chol_pivot(&blk[0][0], &rpiv[0], c0, zrow[c0] != 0, err);
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        const double r = rpiv[j];
        const int m = nb - j - 1;
        for (int t = threadIdx.x; t < m + j + 1; t += blockDim.x) {
            if (t < m) blk[j + 1 + t][j] *= r;  // column j of L
            else w[j][t - m] *= r;              // row j of W, columns <= j
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (m > 0) {  // the next diagonal entry, then its pivot
                blk[j + 1][j + 1] -= blk[j + 1][j] * blk[j + 1][j];
                chol_pivot(&blk[j + 1][j + 1], &rpiv[j + 1], c0 + j + 1, zrow[c0 + j + 1] != 0,
                           err);
            }
        } else {
            for (int t = threadIdx.x - 1; t < m * m + m * (j + 1); t += blockDim.x - 1) {
                if (t < m * m) {
                    const int i = j + 1 + t / m, k = j + 1 + t % m;
                    if (k <= i && !(i == j + 1 && k == j + 1)) blk[i][k] -= blk[i][j] * blk[k][j];
                } else {
                    const int u = t - m * m, i = j + 1 + u / (j + 1), k = u % (j + 1);
                    w[i][k] -= blk[i][j] * w[j][k];
                }
            }
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < CHOL_W; t += blockDim.x) {
        const int r = t / CHOL_NB, c = t % CHOL_NB;
        if (r < nb && c <= r) D[(int64_t)(c0 + r) * n + c0 + c] = blk[r][c];
        Wd[t] = w[r][c];
    }
}

// rows i >= c0 + nb of panel c0: L21 = A21 L11^-T = A21 W^T, 8 rows x CHOL_NB
// columns per CTA (the rows staged in shared memory, then overwritten; W's
// zero entries make every output a full CHOL_NB-term sum)
__global__ void __launch_bounds__(256) chol_trsm_kernel(double *__restrict__ D, int n, int c0,
                                                        int nb, const double *__restrict__ Wd)
{
    __shared__ double a[8][CHOL_NB + 1], w[CHOL_NB][CHOL_NB + 1];
    for (int e = threadIdx.x; e < CHOL_W; e += blockDim.x) w[e / CHOL_NB][e % CHOL_NB] = Wd[e];
    const int r = threadIdx.x / CHOL_NB, t = threadIdx.x % CHOL_NB;
    const int i = c0 + nb + blockIdx.x * 8 + r;
    a[r][t] = (i < n && t < nb) ? D[(int64_t)i * n + c0 + t] : 0.0;
    __syncthreads();
    if (i >= n || t >= nb) return;
    double v = 0.0;
#pragma unroll
    for (int q = 0; q < CHOL_NB; ++q) v = fma(a[r][q], w[t][q], v);
    D[(int64_t)i * n + c0 + t] = v;
}

// trailing update D[i][k] -= sum_t L21[i][t] L21[k][t], c1 <= k <= i < n,
// one CHOL_TILE x CHOL_TILE tile per CTA (tiles above the diagonal skipped)
__global__ void __launch_bounds__(CHOL_TILE * CHOL_TILE) chol_syrk_kernel(double *__restrict__ D,
                                                                         int n, int c0, int nb)
{
    const int c1 = c0 + nb;
    const int ti = blockIdx.y, tk = blockIdx.x;
    if (tk > ti) return;
    __shared__ double li[CHOL_TILE][CHOL_NB + 1], lk[CHOL_TILE][CHOL_NB + 1];
    const int i0 = c1 + ti * CHOL_TILE, k0 = c1 + tk * CHOL_TILE;
    for (int t = threadIdx.y * CHOL_TILE + threadIdx.x; t < CHOL_TILE * nb; t += CHOL_TILE * CHOL_TILE) {
        const int r = t / nb, c = t % nb;
        li[r][c] = i0 + r < n ? D[(int64_t)(i0 + r) * n + c0 + c] : 0.0;
        lk[r][c] = k0 + r < n ? D[(int64_t)(k0 + r) * n + c0 + c] : 0.0;
    }
    __syncthreads();
    const int i = i0 + threadIdx.y, k = k0 + threadIdx.x;
    if (i >= n || k > i) return;
    double v = 0.0;
    for (int t = 0; t < nb; ++t) v += li[threadIdx.y][t] * lk[threadIdx.x][t];
    D[(int64_t)i * n + k] -= v;
}

// Explicit inverse from the Cholesky factor: X = A^-1 solves L L^T X = I,
// blockwise over CHOL_NB-row blocks of L: forward, Y = L^-1 I (lower
// triangular), then backward, X = L^-T Y.  X is symmetric, so only its lower
// triangle (row >= column) is formed and then mirrored; every lower entry
// depends only on lower entries.  Zero rows (unit pivot, zero row of L off
// the diagonal) start from a zero right-hand side and end as zero rows and
// columns of X.

// The block's rows r0 .. r0 + nb - 1 of X, columns c < ncols: forward
// Y_b = W X_b, backward X_b = W^T Y_b, with W the inverse of the block's
// diagonal factor.  CHOL_NB rows x 8 columns per CTA (the strip staged in
// shared memory, then overwritten).
template <bool BWD>
__global__ void __launch_bounds__(256) inv_panel_kernel(const double *__restrict__ Wd,
                                                        double *__restrict__ X, int n, int r0,
                                                        int nb, int ncols)
{
    __shared__ double w[CHOL_NB][CHOL_NB + 1], xs[CHOL_NB][9];
    for (int e = threadIdx.x; e < CHOL_W; e += blockDim.x) w[e / CHOL_NB][e % CHOL_NB] = Wd[e];
    const int t = threadIdx.x / 8, cc = threadIdx.x % 8, c = blockIdx.x * 8 + cc;
    xs[t][cc] = (t < nb && c < ncols) ? X[(int64_t)(r0 + t) * n + c] : 0.0;
    __syncthreads();
    if (t >= nb || c >= ncols) return;
    double v = 0.0;
#pragma unroll
    for (int q = 0; q < CHOL_NB; ++q) v = fma(BWD ? w[q][t] : w[t][q], xs[q][cc], v);
    X[(int64_t)(r0 + t) * n + c] = v;
}

// C -= A B on X's rows [i0, i1) and columns [0, j1), the inner index over the
// block's nb rows r0 .. r0 + nb - 1: forward A(i, t) = L[i][r0 + t], backward
// A(i, t) = L[r0 + t][i] with only j <= i written; B(t, j) = X[r0 + t][j].
// TILE x TILE output tiles, (TILE / 16)^2 per thread.
template <bool BWD, int TILE>
__global__ void __launch_bounds__(256) inv_update_kernel(const double *__restrict__ D,
                                                         double *__restrict__ X, int n, int r0,
                                                         int nb, int i0, int i1, int j1)
{
    constexpr int TM = TILE / 16;
    const int ti0 = i0 + blockIdx.y * TILE, tj0 = blockIdx.x * TILE;
    if (ti0 >= i1 || tj0 >= j1) return;
    if (BWD && tj0 > ti0 + TILE - 1) return;  // tile wholly above the diagonal
    __shared__ double As[CHOL_NB][TILE + 1], Bs[CHOL_NB][TILE + 1];
    for (int e = threadIdx.x; e < nb * TILE; e += blockDim.x) {
        int t, ii;
        if (BWD) {
            t = e / TILE;
            ii = e % TILE;  // row r0 + t of L, consecutive columns
        } else {
            ii = e / nb;
            t = e % nb;     // row i of L, consecutive columns r0 + t
        }
        const int i = ti0 + ii;
        As[t][ii] = i < i1 ? (BWD ? D[(int64_t)(r0 + t) * n + i] : D[(int64_t)i * n + r0 + t])
                           : 0.0;
        const int tb = e / TILE, jj = e % TILE, j = tj0 + jj;
        Bs[tb][jj] = j < j1 ? X[(int64_t)(r0 + tb) * n + j] : 0.0;
    }
    __syncthreads();
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    double acc[TM][TM];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) acc[a][b] = 0.0;
    for (int t = 0; t < nb; ++t) {
        double av[TM], bv[TM];
#pragma unroll
        for (int a = 0; a < TM; ++a) av[a] = As[t][ty * TM + a];
#pragma unroll
        for (int b = 0; b < TM; ++b) bv[b] = Bs[t][tx * TM + b];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int b = 0; b < TM; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < TM; ++a) {
        const int i = ti0 + ty * TM + a;
        if (i >= i1) continue;
#pragma unroll
        for (int b = 0; b < TM; ++b) {
            const int j = tj0 + tx * TM + b;
            if (j < j1 && (!BWD || j <= i)) X[(int64_t)i * n + j] -= acc[a][b];
        }
    }
}

// one inverse update over rows [i0, i1) x columns [0, j1) in 32 x 32 tiles:
// with an SM's FP64 rate the limit, small CTAs (32k FMAs each) spread evenly
// over the SMs, where 64 x 64 tiles left a few SMs with one CTA more than the
// rest; four FMAs per four shared loads stay ahead of the FP64 pipe
template <bool BWD>
static void launch_inv_update(const double *D, double *X, int n, int r0, int nb, int i0, int i1,
                              int j1, cudaStream_t s)
{
    const dim3 g((j1 + 31) / 32, (i1 - i0 + 31) / 32);
    inv_update_kernel<BWD, 32><<<g, 256, 0, s>>>(D, X, n, r0, nb, i0, i1, j1);
    ::amg::count_launch(1);
}

__global__ void unit_diag_kernel(double *__restrict__ X, int n, const uint8_t *__restrict__ zrow)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) X[(int64_t)i * n + i] = zrow[i] ? 0.0 : 1.0;
}

// upper triangle = transpose of the lower one, 32 x 32 tiles through shared memory
__global__ void mirror_upper_kernel(double *__restrict__ X, int n)
{
    const int bi = blockIdx.y, bj = blockIdx.x;  // destination tile (bi, bj), bj >= bi
    if (bj < bi) return;
    __shared__ double t[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8 threads
    for (int r = ty; r < 32; r += 8) {  // source tile (bj, bi): rows of the lower triangle
        const int i = bj * 32 + r, j = bi * 32 + tx;
        t[r][tx] = (i < n && j < n) ? X[(int64_t)i * n + j] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int i = bi * 32 + r, j = bj * 32 + tx;
        if (i < n && j < n && j > i) X[(int64_t)i * n + j] = t[tx][r];
    }
}

constexpr int COARSE_MAX = 20000;

int coarse_inverse(const BsrD &A, DevArena &keep, DevArena &tmp, cudaStream_t s,
                   double **Ainv_out)
{
    const int n = A.nbr * A.br;
    if (n > COARSE_MAX) {
        set_error("coarsest system has %d unknowns (limit %d)", n, COARSE_MAX);
        return AMG_ERR_LIMIT;
    }
    const int nblk_rows = (n + CHOL_NB - 1) / CHOL_NB;
    double *D = nullptr, *X = nullptr, *Wd = nullptr;
    uint8_t *z = nullptr;
    int *brow = nullptr, *err = nullptr;
    AMG_TRY(tmp.alloc_n(&D, (size_t)n * n));
    AMG_TRY(keep.alloc_n(&X, (size_t)n * n));
    AMG_TRY(tmp.alloc_n(&Wd, (size_t)std::max(nblk_rows, 1) * CHOL_W));
    AMG_TRY(tmp.alloc_n(&z, n));
    AMG_TRY(tmp.alloc_n(&brow, (size_t)std::max<int64_t>(A.nnzb, 1)));
    AMG_TRY(tmp.alloc_n(&err, 1));
    AMG_TRY_CUDA(cudaMemsetAsync(D, 0, sizeof(double) * (size_t)n * n, s));
    AMG_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    block_rows_kernel<<<nblk(A.nbr), T1D, 0, s>>>(A.row_ptr, A.nbr, brow); ::amg::count_launch(1);
    if (A.nnzb > 0) {
        densify_kernel<<<nblk(A.nnzb), T1D, 0, s>>>(brow, A.col, A.val, A.nnzb, A.br, n, D); ::amg::count_launch(1); }
    zero_rows_kernel<<<nblk(n), T1D, 0, s>>>(D, n, z); ::amg::count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    for (int b = 0; b < nblk_rows; ++b) {
        const int c0 = b * CHOL_NB, nb = std::min(CHOL_NB, n - c0), rest = n - c0 - nb;
        double *W = Wd + (size_t)b * CHOL_W;
        chol_diag_kernel<<<1, 256, 0, s>>>(D, n, c0, nb, z, err, W);
        ::amg::count_launch(1);
        if (rest > 0) {
            chol_trsm_kernel<<<(rest + 7) / 8, 256, 0, s>>>(D, n, c0, nb, W);
            const int nt = (rest + CHOL_TILE - 1) / CHOL_TILE;
            chol_syrk_kernel<<<dim3(nt, nt), dim3(CHOL_TILE, CHOL_TILE), 0, s>>>(D, n, c0, nb);
            ::amg::count_launch(2);
        }
    }
    AMG_TRY_CUDA(cudaGetLastError());
    int herr = 0;
    AMG_TRY_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        set_error("coarsest matrix is not positive definite (pivot %d)", herr - 1);
        return AMG_ERR_COARSE;
    }
    AMG_TRY_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * (size_t)n * n, s));
    if (n > 0) {
        unit_diag_kernel<<<nblk(n), T1D, 0, s>>>(X, n, z);
        ::amg::count_launch(1);
    }
    for (int b = 0; b < nblk_rows; ++b) {  // forward: L Y = I, columns < r1
        const int r0 = b * CHOL_NB, nb = std::min(CHOL_NB, n - r0), r1 = r0 + nb;
        inv_panel_kernel<false><<<(r1 + 7) / 8, 256, 0, s>>>(Wd + (size_t)b * CHOL_W, X, n, r0,
                                                              nb, r1);
        ::amg::count_launch(1);
        if (r1 < n) launch_inv_update<false>(D, X, n, r0, nb, r1, n, r1, s);
    }
    for (int b = nblk_rows - 1; b >= 0; --b) {  // backward: L^T X = Y, lower triangle
        const int r0 = b * CHOL_NB, nb = std::min(CHOL_NB, n - r0), r1 = r0 + nb;
        inv_panel_kernel<true><<<(r1 + 7) / 8, 256, 0, s>>>(Wd + (size_t)b * CHOL_W, X, n, r0,
                                                             nb, r1);
        ::amg::count_launch(1);
        if (r0 > 0) launch_inv_update<true>(D, X, n, r0, nb, 0, r0, r0, s);
    }
    if (n > 0) {
        const int nt = (n + 31) / 32;
        mirror_upper_kernel<<<dim3(nt, nt), dim3(32, 8), 0, s>>>(X, n);
        ::amg::count_launch(1);
    }
    AMG_TRY_CUDA(cudaGetLastError());
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    tmp.release(Wd);
    tmp.release(D);
    tmp.release(z);
    tmp.release(brow);
    tmp.release(err);
    *Ainv_out = X;
    return AMG_OK;
}


// ---------------------------------------------------------------- scalar storage
// Scalar CSR of a BSR matrix: block row I becomes rows I br .. I br + br - 1,
// each holding the row's blocks' entries in block order (columns J bc + c,
// ascending); explicit zeros inside blocks are kept.
__global__ void unblock_rows_kernel(const int *__restrict__ rp, int nbr, int br, int bc,
                                    int *__restrict__ srp)
{
    const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (row > (int64_t)nbr * br) return;
    if (row == (int64_t)nbr * br) {
        srp[row] = rp[nbr] * br * bc;
        return;
    }
    const int I = (int)(row / br), r = (int)(row % br);
    srp[row] = rp[I] * br * bc + r * (rp[I + 1] - rp[I]) * bc;
}

__global__ void unblock_vals_kernel(const int *__restrict__ rp, const int *__restrict__ brow,
                                    const int *__restrict__ col, const double *__restrict__ val,
                                    int64_t nnzb, int br, int bc, const int *__restrict__ srp,
                                    int *__restrict__ scol, double *__restrict__ sval)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nnzb * br) return;
    const int64_t k = t / br;
    const int r = (int)(t % br);
    const int I = brow[k];
    const int64_t dst = srp[(int64_t)I * br + r] + (k - rp[I]) * bc;
    for (int c = 0; c < bc; ++c) {
        scol[dst + c] = col[k] * bc + c;
        sval[dst + c] = val[k * br * bc + r * bc + c];
    }
}

int unblock_bsr(const BsrD &B, DevArena &mem, cudaStream_t s, BsrD *out)
{
    const int64_t nnz = B.nnzb * B.br * B.bc;
    const int64_t nrows = (int64_t)B.nbr * B.br;
    if (nnz > INT32_MAX || nrows >= INT32_MAX || (int64_t)B.nbc * B.bc >= INT32_MAX) {
        set_error("scalar storage: %lld entries exceed 32-bit indices", (long long)nnz);
        return AMG_ERR_LIMIT;
    }
    BsrD U;
    U.nbr = (int)nrows;
    U.nbc = B.nbc * B.bc;
    U.br = U.bc = 1;
    U.nnzb = nnz;
    AMG_TRY(mem.alloc_n(&U.row_ptr, (size_t)nrows + 1));
    AMG_TRY(mem.alloc_n(&U.col, (size_t)std::max<int64_t>(nnz, 1)));
    AMG_TRY(mem.alloc_n(&U.val, (size_t)std::max<int64_t>(nnz, 1)));
    unblock_rows_kernel<<<nblk(nrows + 1), T1D, 0, s>>>(B.row_ptr, B.nbr, B.br, B.bc, U.row_ptr);
    ::amg::count_launch(1);
    if (B.nnzb > 0) {
        int *brow = nullptr;
        AMG_TRY(mem.alloc_n(&brow, (size_t)B.nnzb));
        block_rows_kernel<<<nblk(B.nbr), T1D, 0, s>>>(B.row_ptr, B.nbr, brow);
        unblock_vals_kernel<<<nblk(B.nnzb * B.br), T1D, 0, s>>>(B.row_ptr, brow, B.col, B.val,
                                                                 B.nnzb, B.br, B.bc, U.row_ptr,
                                                                 U.col, U.val);
        ::amg::count_launch(2);
        AMG_TRY_CUDA(cudaGetLastError());
        AMG_TRY_CUDA(cudaStreamSynchronize(s));
        mem.release(brow);
    }
    AMG_TRY_CUDA(cudaGetLastError());
    *out = U;
    return AMG_OK;
}


// ---------------------------------------------------------------- scalar setup
// The hierarchy built in scalar arithmetic, as the paper's scalar solvers do
// (Sec. 3: "NS Scalar", and "NS Hybrid1", which converts the scalar
// hierarchy into blocks afterwards, Listing 1): every matrix is scalar CSR
// (1x1 blocks) and a level's nodes are groups of b consecutive scalar rows
// (b = 3 on the finest level, the near-nullspace size below).  Strength and
// aggregation see the node graph condensed from the scalar pattern
// (point-wise aggregation with block size b, Sec. 4); the tentative
// prolongation, its smoothing, the Galerkin product and SPAI0 run on scalar
// rows.  The arithmetic of every value is the block setup's, entry by entry.

__global__ void node_membership_kernel(int nn, int b, int *__restrict__ xrp, int *__restrict__ xcol)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= nn) xrp[i] = i * b;
    if (i < nn * b) xcol[i] = i;
}

__global__ void col_div_kernel(const int *__restrict__ col, int64_t nnz, int bc, int *__restrict__ out)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < nnz) out[k] = col[k] / bc;
}

// Block pattern of a scalar CSR matrix S in br x bc blocks (Sec. 2's block
// CSR): block (I, J) is present iff a scalar of rows I br .. I br + br - 1
// lies in columns J bc .. J bc + bc - 1.  The symbolic product of the row
// membership (block row I -> its br scalar rows) with S's pattern read in
// block columns: sorted, each block once.
static int condense_pattern(const BsrD &S, int br, int bc, DevArena &keep, DevArena &tmp,
                            cudaStream_t s, BsrD *out)
{
    const int nbr = S.nbr / br, nbc = S.nbc / bc;
    int *xrp = nullptr, *xcol = nullptr, *ycol = nullptr;
    AMG_TRY(tmp.alloc_n(&xrp, (size_t)nbr + 1));
    AMG_TRY(tmp.alloc_n(&xcol, (size_t)std::max(S.nbr, 1)));
    AMG_TRY(tmp.alloc_n(&ycol, (size_t)std::max<int64_t>(S.nnzb, 1)));
    node_membership_kernel<<<nblk((int64_t)nbr * br + 1), T1D, 0, s>>>(nbr, br, xrp, xcol);
    ::amg::count_launch(1);
    if (S.nnzb > 0) {
        col_div_kernel<<<nblk(S.nnzb), T1D, 0, s>>>(S.col, S.nnzb, bc, ycol);
        ::amg::count_launch(1);
    }
    AMG_TRY_CUDA(cudaGetLastError());
    int total = 0;
    AMG_TRY(spgemm_symbolic(xrp, xcol, nbr, S.row_ptr, ycol, nbc, keep, tmp, s, &out->row_ptr,
                            &out->col, &total));
    out->nbr = nbr;
    out->nbc = nbc;
    out->br = br;
    out->bc = bc;
    out->nnzb = total;
    out->val = nullptr;
    tmp.release(xrp);
    tmp.release(xcol);
    tmp.release(ycol);
    return AMG_OK;
}

// Block (I, J) of S: for each of its br scalar rows, the entries in columns
// J bc .. J bc + bc - 1 (located by binary search in the sorted row); absent
// scalars are explicit zeros.  One thread per block.
__global__ void block_values_kernel(const int *__restrict__ brow, const int *__restrict__ bcol,
                                    int64_t nnzb, int br, int bc, const int *__restrict__ srp,
                                    const int *__restrict__ scol, const double *__restrict__ sval,
                                    double *__restrict__ bval)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nnzb) return;
    const int I = brow[k], c0 = bcol[k] * bc;
    double *dst = bval + k * br * bc;
    for (int r = 0; r < br; ++r) {
        const int row = I * br + r, hi = srp[row + 1];
        int p = find_sorted(scol, srp[row], hi, c0);
        for (int c = 0; c < bc; ++c) {
            double v = 0.0;
            if (p < hi && scol[p] == c0 + c) v = sval[p++];
            dst[r * bc + c] = v;
        }
    }
}

// Squared Frobenius norm of node block (I, J), its scalars summed in
// row-major order without FMA contraction (the order of the block strength
// kernel; absent scalars add nothing).  One thread per node-graph entry.
__global__ void node_norm2_kernel(const int *__restrict__ brow, const int *__restrict__ bcol,
                                  int64_t nnzb, int b, const int *__restrict__ srp,
                                  const int *__restrict__ scol, const double *__restrict__ sval,
                                  double *__restrict__ norm2)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nnzb) return;
    const int I = brow[k], c0 = bcol[k] * b;
    double acc = 0.0;
    for (int r = 0; r < b; ++r) {
        const int row = I * b + r, hi = srp[row + 1];
        for (int p = find_sorted(scol, srp[row], hi, c0); p < hi && scol[p] < c0 + b; ++p)
            acc = __dadd_rn(acc, __dmul_rn(sval[p], sval[p]));
    }
    norm2[k] = acc;
}

__global__ void node_diag_norm_kernel(const int *__restrict__ rp, const int *__restrict__ col,
                                      const double *__restrict__ norm2, int nn,
                                      double *__restrict__ dn)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nn) return;
    double v = 0.0;
    for (int p = rp[I]; p < rp[I + 1]; ++p)
        if (col[p] == I) v = __dsqrt_rn(norm2[p]);
    dn[I] = v;
}

// the block strength test on the node graph's norms (same operations)
__global__ void node_strength_kernel(const int *__restrict__ brow, const int *__restrict__ bcol,
                                     int64_t nnzb, const double *__restrict__ norm2,
                                     const double *__restrict__ dn, double e2,
                                     uint8_t *__restrict__ strong)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nnzb) return;
    const int I = brow[k], J = bcol[k];
    uint8_t st = 0;
    if (J != I) {
        double thr = __dmul_rn(e2, dn[I]);
        thr = __dmul_rn(thr, dn[J]);
        st = norm2[k] > thr ? 1 : 0;
    }
    strong[k] = st;
}

int scalar_to_block(const BsrD &S, int br, int bc, DevArena &keep, DevArena &tmp, cudaStream_t s,
                    BsrD *out)
{
    AMG_TRY(condense_pattern(S, br, bc, keep, tmp, s, out));
    AMG_TRY(keep.alloc_n(&out->val, (size_t)std::max<int64_t>(out->nnzb, 1) * br * bc));
    if (out->nnzb > 0) {
        int *brow = nullptr;
        AMG_TRY(tmp.alloc_n(&brow, (size_t)out->nnzb));
        block_rows_kernel<<<nblk(out->nbr), T1D, 0, s>>>(out->row_ptr, out->nbr, brow);
        block_values_kernel<<<nblk(out->nnzb), T1D, 0, s>>>(brow, out->col, out->nnzb, br, bc,
                                                            S.row_ptr, S.col, S.val, out->val);
        ::amg::count_launch(2);
        AMG_TRY_CUDA(cudaGetLastError());
        tmp.release(brow);
    }
    return AMG_OK;
}

int scalar_strength(const BsrD &S, int b, double eps, DevArena &keep, DevArena &tmp,
                    cudaStream_t s, BsrD *graph, uint8_t **strong)
{
    AMG_TRY(condense_pattern(S, b, b, keep, tmp, s, graph));
    const int nn = graph->nbr;
    AMG_TRY(keep.alloc_n(strong, (size_t)std::max<int64_t>(graph->nnzb, 1)));
    if (graph->nnzb == 0) return AMG_OK;
    int *brow = nullptr;
    double *norm2 = nullptr, *dn = nullptr;
    AMG_TRY(tmp.alloc_n(&brow, (size_t)graph->nnzb));
    AMG_TRY(tmp.alloc_n(&norm2, (size_t)graph->nnzb));
    AMG_TRY(tmp.alloc_n(&dn, (size_t)std::max(nn, 1)));
    block_rows_kernel<<<nblk(nn), T1D, 0, s>>>(graph->row_ptr, nn, brow);
    node_norm2_kernel<<<nblk(graph->nnzb), T1D, 0, s>>>(brow, graph->col, graph->nnzb, b,
                                                         S.row_ptr, S.col, S.val, norm2);
    node_diag_norm_kernel<<<nblk(nn), T1D, 0, s>>>(graph->row_ptr, graph->col, norm2, nn, dn);
    node_strength_kernel<<<nblk(graph->nnzb), T1D, 0, s>>>(brow, graph->col, graph->nnzb, norm2,
                                                            dn, eps * eps, *strong);
    ::amg::count_launch(4);
    AMG_TRY_CUDA(cudaGetLastError());
    tmp.release(brow);
    tmp.release(norm2);
    tmp.release(dn);
    return AMG_OK;
}

// tentative prolongation rows: scalar row i of an aggregated node holds the
// ns columns of its aggregate (all stored, zeros included)
__global__ void ptent_count_kernel(const int *__restrict__ agg, int n, int b, int ns,
                                   int *__restrict__ cnt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cnt[i] = agg[i / b] >= 0 ? ns : 0;
}

__global__ void ptent_fill_kernel(const int *__restrict__ agg, int n, int b, int ns,
                                  const int *__restrict__ rp, const double *__restrict__ ptent,
                                  int *__restrict__ col, double *__restrict__ val)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int a = agg[i / b];
    if (a < 0) return;
    for (int k = 0; k < ns; ++k) {
        col[rp[i] + k] = ns * a + k;
        val[rp[i] + k] = ptent[(int64_t)i * ns + k];
    }
}

// P = P_tent - omega D^-1 (A P_tent) in place on A P_tent's entries (its
// pattern holds P_tent's: A keeps its diagonal): s_i = omega / d_i (0 when
// d_i = 0), then p_ij - s_i (A P_tent)_ij, p_ij = 0 outside P_tent.
__global__ void scalar_smooth_p_kernel(const int *__restrict__ prow, const int *__restrict__ pcol,
                                       int64_t nnz, const int *__restrict__ agg, int b, int ns,
                                       const double *__restrict__ ptent,
                                       const double *__restrict__ d, double omega,
                                       double *__restrict__ val)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nnz) return;
    const int i = prow[k], j = pcol[k], a = agg[i / b];
    const double pt = (a >= 0 && j / ns == a) ? ptent[(int64_t)i * ns + (j - ns * a)] : 0.0;
    const double di = d[i];
    const double sc = di != 0.0 ? __ddiv_rn(omega, di) : 0.0;
    val[k] = __dsub_rn(pt, __dmul_rn(sc, val[k]));
}

int scalar_transfer(const BsrD &S, int b, const double *B, int ns, const int *agg_h, int nagg,
                    double relax, DevArena &keep, DevArena &tmp, cudaStream_t s, LevelBuild *out)
{
    const int n = S.nbr, nn = n / b;
    std::vector<int> aptr(nagg + 1, 0), mem;
    for (int I = 0; I < nn; ++I)
        if (agg_h[I] >= 0) aptr[agg_h[I] + 1]++;
    for (int a = 0; a < nagg; ++a) aptr[a + 1] += aptr[a];
    mem.resize(std::max(aptr[nagg], 1));
    {
        std::vector<int> fill(aptr.begin(), aptr.end() - 1);
        for (int I = 0; I < nn; ++I)
            if (agg_h[I] >= 0) mem[fill[agg_h[I]]++] = I;
    }
    int *d_aptr = nullptr, *d_mem = nullptr, *cnt = nullptr;
    double *Qs = nullptr, *ptent = nullptr, *d = nullptr;
    unsigned long long *rho_bits = nullptr;
    AMG_TRY(tmp.alloc_n(&d_aptr, nagg + 1));
    AMG_TRY(tmp.alloc_n(&d_mem, mem.size()));
    AMG_TRY(keep.alloc_n(&out->agg, std::max(nn, 1)));
    AMG_TRY(tmp.alloc_n(&Qs, (size_t)std::max(aptr[nagg], 1) * b * ns));
    AMG_TRY(tmp.alloc_n(&ptent, (size_t)std::max(n, 1) * ns));
    AMG_TRY(tmp.alloc_n(&d, (size_t)std::max(n, 1)));
    AMG_TRY(tmp.alloc_n(&rho_bits, 1));
    AMG_TRY(tmp.alloc_n(&cnt, (size_t)n + 1));
    AMG_TRY(keep.alloc_n(&out->Bc, (size_t)std::max(nagg, 1) * ns * ns));
    AMG_TRY_CUDA(cudaMemcpyAsync(d_aptr, aptr.data(), sizeof(int) * (nagg + 1),
                                 cudaMemcpyHostToDevice, s));
    AMG_TRY_CUDA(cudaMemcpyAsync(d_mem, mem.data(), sizeof(int) * mem.size(),
                                 cudaMemcpyHostToDevice, s));
    AMG_TRY_CUDA(cudaMemcpyAsync(out->agg, agg_h, sizeof(int) * nn, cudaMemcpyHostToDevice, s));
    AMG_TRY_CUDA(cudaMemsetAsync(ptent, 0, sizeof(double) * (size_t)n * ns, s));
    AMG_TRY_CUDA(cudaMemsetAsync(rho_bits, 0, sizeof(unsigned long long), s));
    out->nagg = nagg;
    // per-aggregate QR of the stacked near-nullspace rows (the same kernel
    // as the block setup: it is scalar arithmetic in either setup)
    if (nagg > 0) {
        if (ns == 6)
            tentative_kernel<6><<<nblk((int64_t)nagg * 32), T1D, 0, s>>>(nagg, b, d_aptr, d_mem, B,
                                                                          Qs, ptent, out->Bc);
        else
            tentative_kernel<3><<<nblk((int64_t)nagg * 32), T1D, 0, s>>>(nagg, b, d_aptr, d_mem, B,
                                                                          Qs, ptent, out->Bc);
        ::amg::count_launch(1);
    }
    // scalar rows: d_i and the Gershgorin bound, columns ascending
    jacobi_rho_kernel<<<nblk(n), T1D, 0, s>>>(S.row_ptr, S.col, S.val, n, 1, d, rho_bits);
    ptent_count_kernel<<<nblk(n), T1D, 0, s>>>(out->agg, n, b, ns, cnt);
    ::amg::count_launch(2);
    AMG_TRY_CUDA(cudaGetLastError());
    unsigned long long rb = 0;
    AMG_TRY_CUDA(cudaMemcpyAsync(&rb, rho_bits, sizeof(rb), cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));  // host vectors above go out of scope after this
    double rho;
    std::memcpy(&rho, &rb, sizeof rho);
    out->rho = rho;
    out->omega = (rho > 0.0) ? relax * (4.0 / 3.0) / rho : 0.0;
    // P_tent as scalar CSR
    BsrD Pt;
    Pt.nbr = n;
    Pt.nbc = nagg * ns;
    Pt.br = Pt.bc = 1;
    int total = 0;
    AMG_TRY(tmp.alloc_n(&Pt.row_ptr, (size_t)n + 1));
    AMG_TRY(exclusive_scan_i32(cnt, Pt.row_ptr, n, &total, tmp, s));
    Pt.nnzb = total;
    AMG_TRY(tmp.alloc_n(&Pt.col, (size_t)std::max(total, 1)));
    AMG_TRY(tmp.alloc_n(&Pt.val, (size_t)std::max(total, 1)));
    ptent_fill_kernel<<<nblk(n), T1D, 0, s>>>(out->agg, n, b, ns, Pt.row_ptr, ptent, Pt.col,
                                              Pt.val);
    ::amg::count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    // A P_tent (scalar SpGEMM), then P in place on its entries
    BsrD &P = out->P;
    AMG_TRY(spgemm(S, Pt, keep, tmp, s, &P));
    if (P.nnzb > 0) {
        int *prow = nullptr;
        AMG_TRY(tmp.alloc_n(&prow, (size_t)P.nnzb));
        block_rows_kernel<<<nblk(n), T1D, 0, s>>>(P.row_ptr, n, prow);
        scalar_smooth_p_kernel<<<nblk(P.nnzb), T1D, 0, s>>>(prow, P.col, P.nnzb, out->agg, b, ns,
                                                            ptent, d, out->omega, P.val);
        ::amg::count_launch(2);
        AMG_TRY_CUDA(cudaGetLastError());
        AMG_TRY(transpose_bsr(P, prow, keep, tmp, s, &out->R));
        tmp.release(prow);
    } else {
        AMG_TRY(transpose_bsr(P, nullptr, keep, tmp, s, &out->R));
    }
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    for (void *q : {(void *)d_aptr, (void *)d_mem, (void *)Qs, (void *)ptent, (void *)d,
                    (void *)rho_bits, (void *)cnt, (void *)Pt.row_ptr, (void *)Pt.col,
                    (void *)Pt.val})
        tmp.release(q);
    return AMG_OK;
}

}  // namespace amg
