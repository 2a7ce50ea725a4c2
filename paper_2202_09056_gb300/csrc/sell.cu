// Sliced block-ELL (SELL) layout and SpMV kernels for the V-cycle and CG.
//
// Why this layout on GB300: the FP64 pipe of sm_103a issues about two FP64
// lane-operations per clock per SM, 1/64 of the FP32 rate, so a 3x3 FP64
// block SpMV is bounded by its multiply-adds almost as much as by HBM
// (9 DFMA per 72 value bytes).  A kernel that splits a block row across all
// lanes of a warp pays for cross-lane FP64 reductions and predicated
// accumulations in that same pipe.  Here a row belongs to G lanes (G = 1 on
// the fine level, where rows are many and short; up to 128 on the coarse
// levels, where they are few and long): each lane does exactly br*bc DFMAs
// per block it owns and the G partial sums meet in a log2(G)-step butterfly
// (G <= 32), or a full-warp butterfly followed by a fixed-order sum of the
// G/32 warps' totals in shared memory (G = 64, 128: the row's slices are
// consecutive and always handled by warps of one CTA).
// To keep the loads coalesced, the 32 lanes of a slice store their blocks
// interleaved: entry e of the block at depth d of lane t sits at
// (slice_base + 32 d) * bb + 32 e + t, so every value load of a warp is one
// contiguous 256-byte segment; FP64 values go in lane pairs instead (entries
// 2p and 2p+1 of lane t at (slice_base + 32 d) * bb + 64 p + 2 t, an odd last
// entry after the pairs), one contiguous 512-byte segment per 16-byte load.  A slice is as deep as its longest lane;
// shorter lanes are padded with zero blocks pointing at column 0 (the padding
// is overhead, not algorithmic bytes).
//
// The epilogues (residual, smoothing, prolongation-correction, restriction
// with the next pre-smoothing, fused dot products) run on the first lane of
// each row group; dots are reduced per CTA in a fixed order, so results are
// bitwise reproducible for a fixed launch.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "amg_internal.cuh"

namespace amg {

__device__ __forceinline__ double sldv(const double *p) { return __ldcs(p); }
__device__ __forceinline__ float sldv(const float *p) { return __ldcs(p); }
__device__ __forceinline__ float sldv(const __nv_bfloat16 *p)
{
    unsigned short bits = __ldcs(reinterpret_cast<const unsigned short *>(p));
    return __uint_as_float(((unsigned int)bits) << 16);
}

template <int NT> __device__ __forceinline__ double cta_sum_d(double v)
{
    __shared__ double red[NT / 32];
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
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

constexpr int SELL_THREADS = 128;

// Register budget: the kernel is compiled for minb resident CTAs per SM
// (65536 / (128 x minb) registers per thread): 12 (40 registers) for 3x3
// blocks, 8 (64) for the others (6 for FP64 6x6, below), whose paired FP64
// loads hold 18-36 values (at 10 CTAs the 6x3 restriction spilled and ran
// 7 % slower).  Grid: up to cap CTAs per SM,
// measured on the 80^3 hierarchy.  The fine-level shapes (3-row blocks, one
// lane per row, uniform slices) run fastest oversubscribed, one slice group
// per CTA with the hardware scheduler balancing; the 6x6 coarse operators
// (few, long rows in widest-first order) fastest as exactly one resident
// wave with the warp-strided loop balancing.
__host__ __device__ constexpr int sell_minb(int br, int bc) { return br == 6 ? 8 : (bc == 6 ? 8 : 12); }
__host__ __device__ constexpr int sell_cap(int br, int bc) { return br == 6 ? (bc == 6 ? 8 : 16) : 32; }
// FP32-pair values hold hi and lo of every entry plus the pair accumulators:
// 64 registers for 3x3 (8 CTAs), 80 for 3x6 / 6x3 (6), 128 for 6x6 (4, and
// one resident wave of 4 CTAs per SM)
template <class VT> __host__ __device__ constexpr int sell_minb_t(int br, int bc)
{
    return std::is_same<VT, df32>::value ? (br == 6 && bc == 6 ? 4 : (br == 6 || bc == 6 ? 6 : 8))
                                         : sell_minb(br, bc);
}
template <class VT> __host__ __device__ constexpr int sell_cap_t(int br, int bc)
{
    return std::is_same<VT, df32>::value && br == 6 && bc == 6 ? 4 : sell_cap(br, bc);
}

// The FP64 3x3 kernels with a fused dot (the CG's q = A p with p.q, the
// post-smoothing with r.z, the true residual) keep one more double live: at
// 12 CTAs per SM (40 registers) they spilled 8 bytes, at 10 (48) none.
template <class VT> __host__ __device__ constexpr int sell_minb_dot(int br, int bc, int dot)
{
    return (dot != 0 && br == 3 && bc == 3 && std::is_same<VT, double>::value)
               ? 10
               : sell_minb_t<VT>(br, bc);
}

// A 6x6 FP64 block is 72 registers of values: those kernels are compiled
// for 6 resident CTAs per SM (80 registers) rather than 8 (64), which took
// level-1 A 113 -> 111 us, level-1 P 35 -> 33 us and the level-2 P and R
// 17-18 -> 15-17 us at 80^3 (the rows' arithmetic unchanged); 5 CTAs (96
// registers) gained nothing more.  The FP64 6x3 restriction (36 registers
// of values) likewise runs at 6: 112.7 -> 110.8 us.  Launches whose rows
// span several warps, and the 6x6 prolongations, size their grid to that
// one resident wave; the other launches keep their grid (8 or 16 CTAs per
// SM), the CTAs past the first wave taking the tail of the work.
template <class VT> __host__ __device__ constexpr bool sell_roomy(int br, int bc)
{
    return std::is_same<VT, double>::value && br == 6 && bc == 6;
}
template <class VT> __host__ __device__ constexpr int sell_minb_k(int br, int bc, int dot)
{
    return (sell_roomy<VT>(br, bc) || (std::is_same<VT, double>::value && br == 6 && bc == 3))
               ? 6
               : sell_minb_dot<VT>(br, bc, dot);
}

template <int BR, int BC, class VT, class TV, int MODE, int DOT, bool WIDE>
__global__ void __launch_bounds__(SELL_THREADS, sell_minb_k<VT>(BR, BC, DOT)) sell_spmv_kernel(SellArgs<TV> a)
{
    using Acc = TV;
    constexpr int BB = BR * BC;
    __shared__ Acc wsum[WIDE ? SELL_THREADS / 32 : 1][BR];
    if (a.stop && *a.stop) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int G = a.G;
    constexpr bool wide = WIDE;                // a row spans G/32 slices (G > 32)
    const int spr = wide ? G >> 5 : 1;
    const int sub = wide ? 0 : lane & (G - 1);
    const int rows_per_slice = wide ? 1 : 32 / G;
    const int nw = (int)((gridDim.x * (unsigned)blockDim.x) >> 5);
    const VT *__restrict__ val = static_cast<const VT *>(a.val);
    const int *__restrict__ col = a.col;
    const TV *__restrict__ x = a.x;
    double dot = 0.0;
    // nslices is a multiple of 4 when wide, so every warp of a CTA runs the
    // same number of iterations (the loop holds __syncthreads)
    for (int s = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5); s < a.nslices;
         s += nw) {
        const int slot = wide ? s / spr : s * rows_per_slice + lane / G;
        const int row = a.perm ? a.perm[slot] : slot;
        const int64_t base = a.slice_ptr[s];
        const int w = (int)((a.slice_ptr[s + 1] - base) >> 5);
        const VT *vp = val + base * BB + lane;
        const int *cp = col + base + lane;
        Acc acc[BR];
#pragma unroll
        for (int r = 0; r < BR; ++r) acc[r] = Acc(0);
        float sh[BR], sl[BR];  // FP32-pair accumulators (VT = df32)
#pragma unroll
        for (int r = 0; r < BR; ++r) sh[r] = sl[r] = 0.0f;
        int jn = (w > 0) ? __ldg(cp) : 0;
#pragma unroll(std::is_same<VT, df32>::value ? 1 : 2)
        for (int k = 0; k < w; ++k) {
            const int j = jn;
            if (k + 1 < w) jn = __ldg(cp + (k + 1) * 32);
            Acc xv[BC];
#pragma unroll
            for (int c = 0; c < BC; ++c) xv[c] = (Acc)__ldg(x + (int64_t)j * BC + c);
            if constexpr (std::is_same<VT, double>::value) {
                // FP64 values are stored in lane pairs: one 16-byte load
                // brings two entries of a lane's block (half the load
                // instructions of the per-entry layout)
                const double *vg = val + (base + (int64_t)k * 32) * BB;
                double v[BB];
#pragma unroll
                for (int p = 0; p < BB / 2; ++p) {
                    const double2 t2 = __ldcs(reinterpret_cast<const double2 *>(vg + p * 64) + lane);
                    v[2 * p] = t2.x;
                    v[2 * p + 1] = t2.y;
                }
                if constexpr (BB % 2 == 1) v[BB - 1] = __ldcs(vg + (BB / 2) * 64 + lane);
#pragma unroll
                for (int r = 0; r < BR; ++r)
#pragma unroll
                    for (int c = 0; c < BC; ++c) acc[r] = fma(v[r * BC + c], xv[c], acc[r]);
            } else if constexpr (std::is_same<VT, df32>::value) {
                // FP64 on FP32 pairs, stored like the FP64 lane pairs (one
                // 16-byte load brings two entries, hi and lo each); x split
                // on the bits.  Per entry: the error-free FP32 product of the
                // his with the cross terms added to its error, then the
                // double-float sum: two-sum of the his, the los added to its
                // error, a fast two-sum to renormalise (|sl| <= ulp(sh) / 2)
                // -- every rounded operation written out, nothing contracted
                const df32 *vg = val + (base + (int64_t)k * 32) * BB;
                float vh[BB], vl[BB];
#pragma unroll
                for (int p = 0; p < BB / 2; ++p) {
                    const float4 t4 = __ldcs(reinterpret_cast<const float4 *>(vg + p * 64) + lane);
                    vh[2 * p] = t4.x;
                    vl[2 * p] = t4.y;
                    vh[2 * p + 1] = t4.z;
                    vl[2 * p + 1] = t4.w;
                }
                if constexpr (BB % 2 == 1) {
                    const float2 t2 = __ldcs(reinterpret_cast<const float2 *>(vg + (BB / 2) * 64) + lane);
                    vh[BB - 1] = t2.x;
                    vl[BB - 1] = t2.y;
                }
                float xh[BC], xl[BC];
#pragma unroll
                for (int c = 0; c < BC; ++c) split_f64((double)xv[c], xh[c], xl[c]);
#pragma unroll
                for (int r = 0; r < BR; ++r)
#pragma unroll
                    for (int c = 0; c < BC; ++c) {
                        const float ah = vh[r * BC + c], al = vl[r * BC + c];
                        const float pr = __fmul_rn(ah, xh[c]);
                        float er = __fmaf_rn(ah, xh[c], -pr);
                        er = __fmaf_rn(ah, xl[c], er);
                        er = __fmaf_rn(al, xh[c], er);
                        const float sn = __fadd_rn(sh[r], pr);
                        const float bv = __fsub_rn(sn, sh[r]);
                        float te = __fadd_rn(__fsub_rn(sh[r], __fsub_rn(sn, bv)),
                                             __fsub_rn(pr, bv));
                        te = __fadd_rn(te, __fadd_rn(sl[r], er));
                        sh[r] = __fadd_rn(sn, te);
                        sl[r] = __fsub_rn(te, __fsub_rn(sh[r], sn));
                    }
            } else {
                const VT *vb = vp + (int64_t)k * 32 * BB;
#pragma unroll
                for (int r = 0; r < BR; ++r)
#pragma unroll
                    for (int c = 0; c < BC; ++c)
                        acc[r] = fma((Acc)sldv(vb + (r * BC + c) * 32), xv[c], acc[r]);
            }
        }
        if constexpr (std::is_same<VT, df32>::value)
#pragma unroll
            for (int r = 0; r < BR; ++r) acc[r] = f32_to_f64(sh[r]) + f32_to_f64(sl[r]);
        // rows split over G lanes: fixed-order butterfly within the group
        bool owner;
        if constexpr (!wide) {
            for (int m = G >> 1; m >= 1; m >>= 1)
#pragma unroll
                for (int r = 0; r < BR; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], m);
            owner = sub == 0;
        } else {
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1)
#pragma unroll
                for (int r = 0; r < BR; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], m);
            if (lane == 0)
#pragma unroll
                for (int r = 0; r < BR; ++r) wsum[warp][r] = acc[r];
            __syncthreads();
            owner = lane == 0 && warp % spr == 0;
            if (owner)
#pragma unroll
                for (int r = 0; r < BR; ++r) {
                    Acc t = wsum[warp][r];
                    for (int q = 1; q < spr; ++q) t += wsum[warp + q][r];
                    acc[r] = t;
                }
            __syncthreads();
        }
        if (MODE == SPMV_SMOOTHB && owner && row >= 0 && row < a.nrows) {
            // u + Mb (f - A u) with the row's BR x BR block
            Acc res[BR];
#pragma unroll
            for (int r = 0; r < BR; ++r) res[r] = a.f[(int64_t)row * BR + r] - acc[r];
            const TV *mb = a.Mb + (int64_t)row * BR * BR;
#pragma unroll
            for (int r = 0; r < BR; ++r) {
                const int64_t i = (int64_t)row * BR + r;
                Acc corr = Acc(0);
#pragma unroll
                for (int c = 0; c < BR; ++c) corr = fma((Acc)mb[r * BR + c], res[c], corr);
                const Acc out = x[i] + corr;
                a.y[i] = out;
                if (DOT == DOT_FY) dot += (double)a.f[i] * (double)out;
            }
        } else if (owner && row >= 0 && row < a.nrows) {
#pragma unroll
            for (int r = 0; r < BR; ++r) {
                const int64_t i = (int64_t)row * BR + r;
                Acc out;
                if (MODE == SPMV_PLAIN) out = acc[r];
                else if (MODE == SPMV_RESID) out = a.f[i] - acc[r];
                else if (MODE == SPMV_SMOOTH) out = x[i] + a.M[i] * (a.f[i] - acc[r]);
                else if (MODE == SPMV_AXPY) out = a.u[i] + acc[r];
                else out = acc[r];
                a.y[i] = out;
                if (MODE == SPMV_RESTRICT && a.y2 && !a.Mbn) a.y2[i] = a.M ? a.M[i] * out : Acc(0);
                if (DOT == DOT_XY) dot += (double)x[i] * (double)out;
                if (DOT == DOT_FY) dot += (double)a.f[i] * (double)out;
                if (DOT == DOT_YY) dot += (double)out * (double)out;
            }
            if (MODE == SPMV_RESTRICT && a.y2 && a.Mbn) {
                // the next level's pre-smoothing from zero with its blocks:
                // y2 = Mbn y on this block row (the BR outputs are acc[])
                const TV *mb = a.Mbn + (int64_t)row * BR * BR;
#pragma unroll
                for (int r = 0; r < BR; ++r) {
                    Acc v = Acc(0);
#pragma unroll
                    for (int c = 0; c < BR; ++c) v = fma((Acc)mb[r * BR + c], acc[c], v);
                    a.y2[(int64_t)row * BR + r] = v;
                }
            }
        }
    }
    if (DOT != DOT_NONE) {
        const double t = cta_sum_d<SELL_THREADS>(dot);
        if (threadIdx.x == 0) a.partials[blockIdx.x] = t;
    }
}

static int sell_grid_cap(int nslices, int cap_per_sm, const Geom &g)
{
    const int per_cta = SELL_THREADS / 32;
    int grid = (nslices + per_cta - 1) / per_cta;
    const int cap = g.num_sms * cap_per_sm;  // <= Geom::max_partials
    if (grid > cap) grid = cap;
    return std::max(grid, 1);
}

int sell_grid(int nslices, int br, int bc, const Geom &g)
{
    const int per_cta = SELL_THREADS / 32;
    int grid = (nslices + per_cta - 1) / per_cta;
    const int cap = g.num_sms * sell_cap(br, bc);  // <= Geom::max_partials
    if (grid > cap) grid = cap;
    return std::max(grid, 1);
}

template <int BR, int BC, class VT, class TV, int MODE, int DOT>
static int sell_go(const SellArgs<TV> &a, int grid, cudaStream_t s)
{
    if (a.G <= 32) {
        sell_spmv_kernel<BR, BC, VT, TV, MODE, DOT, false><<<grid, SELL_THREADS, 0, s>>>(a);
    } else if constexpr (BR == 6) {
        sell_spmv_kernel<BR, BC, VT, TV, MODE, DOT, true><<<grid, SELL_THREADS, 0, s>>>(a);
    } else {
        set_error("rows over several warps need 6-row blocks");
        return AMG_ERR_ARG;
    }
    count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    return AMG_OK;
}

// The (mode, dot) pairs the solver uses; FP64-only dots for the CG products.
template <int BR, int BC, class VT, class TV, int MODE>
static int sell_dot(int dot, const SellArgs<TV> &a, int grid, cudaStream_t s)
{
    constexpr bool f64 = std::is_same<TV, double>::value;
    if (dot == DOT_NONE) return sell_go<BR, BC, VT, TV, MODE, DOT_NONE>(a, grid, s);
    if constexpr (MODE == SPMV_SMOOTH || MODE == SPMV_SMOOTHB)
        if (dot == DOT_FY) return sell_go<BR, BC, VT, TV, MODE, DOT_FY>(a, grid, s);
    if constexpr (f64 && BR == BC && MODE == SPMV_PLAIN)
        if (dot == DOT_XY) return sell_go<BR, BC, VT, TV, MODE, DOT_XY>(a, grid, s);
    if constexpr (f64 && BR == BC && MODE == SPMV_RESID)
        if (dot == DOT_YY) return sell_go<BR, BC, VT, TV, MODE, DOT_YY>(a, grid, s);
    set_error("unsupported dot %d for spmv mode %d", dot, MODE);
    return AMG_ERR_ARG;
}

// Only the (mode, dot) pairs the solver records are instantiated.
template <int BR, int BC, class VT, class TV>
static int sell_mode(int mode, int dot, const SellArgs<TV> &a, int grid, cudaStream_t s)
{
    switch (mode) {
    case SPMV_PLAIN: return sell_dot<BR, BC, VT, TV, SPMV_PLAIN>(dot, a, grid, s);
    case SPMV_RESID: return sell_dot<BR, BC, VT, TV, SPMV_RESID>(dot, a, grid, s);
    case SPMV_SMOOTH: return sell_dot<BR, BC, VT, TV, SPMV_SMOOTH>(dot, a, grid, s);
    case SPMV_AXPY: return sell_dot<BR, BC, VT, TV, SPMV_AXPY>(dot, a, grid, s);
    case SPMV_RESTRICT: return sell_dot<BR, BC, VT, TV, SPMV_RESTRICT>(dot, a, grid, s);
    case SPMV_SMOOTHB:
        if constexpr (BR == BC && BR > 1)
            return sell_dot<BR, BC, VT, TV, SPMV_SMOOTHB>(dot, a, grid, s);
        set_error("block smoothing needs square node blocks");
        return AMG_ERR_ARG;
    default: set_error("bad spmv mode %d", mode); return AMG_ERR_ARG;
    }
}

template <class VT, class TV>
int launch_sell(const Sell<VT> &A, int mode, int dot, SellArgs<TV> a, const Geom &g,
                cudaStream_t s, int *grid_out, int max_grid)
{
    a.nrows = A.nrows;
    a.nslices = A.nslices;
    a.G = A.G;
    a.slice_ptr = A.slice_ptr;
    a.col = A.col;
    a.val = A.val;
    a.perm = A.perm;
    int grid = sell_grid_cap(A.nslices,
                             sell_roomy<VT>(A.br, A.bc) && (A.G > 32 || mode == SPMV_AXPY)
                                 ? 6
                                 : sell_cap_t<VT>(A.br, A.bc),
                             g);
    if (max_grid > 0 && grid > max_grid) grid = max_grid;
    if (((uintptr_t)a.x & (sizeof(TV) - 1)) != 0) {
        set_error("the sliced SpMV needs x aligned to its element size");
        return AMG_ERR_ARG;
    }
    if (grid_out) *grid_out = grid;
    if (dot != DOT_NONE && grid > g.max_partials) {
        set_error("fused dot needs %d partial sums, the buffer holds %d", grid, g.max_partials);
        return AMG_ERR_LIMIT;
    }
    if (A.nrows == 0) {
        if (dot != DOT_NONE) AMG_TRY_CUDA(cudaMemsetAsync(a.partials, 0, sizeof(double), s));
        return AMG_OK;
    }
    const int br = A.br, bc = A.bc;
    if (br == 1 && bc == 1) return sell_mode<1, 1, VT, TV>(mode, dot, a, grid, s);
    if (br == 3 && bc == 3) return sell_mode<3, 3, VT, TV>(mode, dot, a, grid, s);
    if (br == 6 && bc == 6) return sell_mode<6, 6, VT, TV>(mode, dot, a, grid, s);
    if (br == 3 && bc == 6) return sell_mode<3, 6, VT, TV>(mode, dot, a, grid, s);
    if (br == 6 && bc == 3) return sell_mode<6, 3, VT, TV>(mode, dot, a, grid, s);
    set_error("unsupported block shape %dx%d", br, bc);
    return AMG_ERR_ARG;
}

template int launch_sell<double, double>(const Sell<double> &, int, int, SellArgs<double>,
                                         const Geom &, cudaStream_t, int *, int);
template int launch_sell<float, float>(const Sell<float> &, int, int, SellArgs<float>,
                                       const Geom &, cudaStream_t, int *, int);
template int launch_sell<__nv_bfloat16, float>(const Sell<__nv_bfloat16> &, int, int,
                                               SellArgs<float>, const Geom &, cudaStream_t, int *,
                                               int);
template int launch_sell<df32, double>(const Sell<df32> &, int, int, SellArgs<double>,
                                       const Geom &, cudaStream_t, int *, int);

// ---------------------------------------------------------------- conversion
template <class T>
__global__ void sell_fill_kernel(const int *__restrict__ rp, const int *__restrict__ bcol,
                                 const double *__restrict__ bval, int nrows, int nslices, int bb,
                                 int G, const int *__restrict__ perm,
                                 const int64_t *__restrict__ sp, int *__restrict__ col,
                                 T *__restrict__ val)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nslices * 32) return;
    const int s = t >> 5, lane = t & 31;
    const bool wide = G > 32;
    const int slot = wide ? s / (G >> 5) : s * (32 / G) + lane / G;
    const int sub = wide ? (s % (G >> 5)) * 32 + lane : lane & (G - 1);
    const int row = perm ? perm[slot] : slot;
    const bool live = row >= 0 && row < nrows;
    const int len = live ? rp[row + 1] - rp[row] : 0;
    const int64_t base = sp[s];
    const int w = (int)((sp[s + 1] - base) >> 5);
    for (int d = 0; d < w; ++d) {
        const int k = d * G + sub;  // block k of the row sits at depth k / G of lane k % G
        const int64_t q = base + (int64_t)d * 32 + lane;
        const bool have = k < len;
        const int64_t src = have ? (int64_t)rp[row] + k : 0;
        col[q] = have ? bcol[src] : 0;
        T *vg = val + (base + (int64_t)d * 32) * bb;
        for (int e = 0; e < bb; ++e) {
            // FP64: entries 2p, 2p + 1 of a lane side by side (pair p of the
            // 32 lanes is one 512-byte run), an odd last entry per lane after
            // the pairs; other types: entry e of the 32 lanes is one run
            const int64_t off = sizeof(T) == 8 ? (e < (bb & ~1) ? (int64_t)(e >> 1) * 64 + 2 * lane + (e & 1)
                                                                 : (int64_t)(bb >> 1) * 64 + lane)
                                               : (int64_t)e * 32 + lane;
            vg[off] = have ? (T)bval[src * bb + e] : (T)0.0;
        }
    }
}

// Slot order of a sliced copy.  A row group is one slice of 32/G rows
// (G <= 32) or the G/32 consecutive slices of one row (G > 32).  Slice
// widths follow the longest lane, so rows of uneven length (P and R, whose
// length is the number of aggregates a node's neighbourhood touches; coarse
// A) waste slots.  When the natural order pads more than 5 %, rows are sorted
// by length, longest first (ties: ascending row), inside windows of 32 groups
// (SELL-C-sigma); a window keeps rows that are close in the numbering
// together, so the x gather keeps its locality.  The groups are then ordered
// by width, widest first (ties: ascending group): CTAs take them in that
// order (longest processing time first), so no SM is left with a tail of long
// rows while the others idle.  The sorting runs on the device; only the
// slice widths and group costs cross to the host.

// widths of every group's slices for the slot -> row map rowof (null: the
// natural order); total += the slots they take
__global__ void sell_group_width_kernel(const int *__restrict__ rp, int nrows, int G, int rpg,
                                        int spg, int ngroups, const int *__restrict__ rowof,
                                        int *__restrict__ w, unsigned long long *__restrict__ total)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ngroups) return;
    auto row_of = [&](int slot) { return rowof ? rowof[slot] : (slot < nrows ? slot : -1); };
    auto len = [&](int row) { return row < 0 || row >= nrows ? 0 : rp[row + 1] - rp[row]; };
    unsigned long long slots = 0;
    if (G > 32) {
        const int L = len(row_of(g));
        for (int q = 0; q < spg; ++q) {
            const int wq = max(0, (L - 32 * q + G - 1) / G);
            w[g * spg + q] = wq;
            slots += 32ull * wq;
        }
    } else {
        int m = 0;
        for (int t = 0; t < rpg; ++t) m = max(m, (len(row_of(g * rpg + t)) + G - 1) / G);
        w[g] = m;
        slots = 32ull * m;
    }
    atomicAdd(total, slots);
}

// one CTA per window of `win` rows: every row's rank by (length descending,
// row ascending) among the window's rows, pw[window start + rank] = row
constexpr int SELL_WIN_MAX = 1024;
__global__ void __launch_bounds__(256) sell_window_rank_kernel(const int *__restrict__ rp, int nrows,
                                                               int win, int *__restrict__ pw)
{
    __shared__ int ln[SELL_WIN_MAX];
    const int r0 = blockIdx.x * win, n = min(win, nrows - r0);
    for (int i = threadIdx.x; i < n; i += blockDim.x) ln[i] = rp[r0 + i + 1] - rp[r0 + i];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int li = ln[i];
        int rank = 0;
        for (int j = 0; j < n; ++j) rank += (ln[j] > li) || (ln[j] == li && j < i);
        pw[r0 + rank] = r0 + i;
    }
}

// perm[k rpg + t] = pw[order[k] rpg + t]
__global__ void sell_gather_groups_kernel(const int *__restrict__ order, const int *__restrict__ pw,
                                          int ngroups, int rpg, int *__restrict__ perm)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ngroups) return;
    const int g = order[k];
    for (int t = 0; t < rpg; ++t) perm[(int64_t)k * rpg + t] = pw[(int64_t)g * rpg + t];
}

template <class T>
int bsr_to_sell(const BsrD &B, DevArena &keep, cudaStream_t s, Sell<T> *out, double *padding,
                int max_lanes)
{
    Sell<T> S;
    S.nrows = B.nbr;
    S.nbc = B.nbc;
    S.br = B.br;
    S.bc = B.bc;
    // lanes per row: enough threads to fill the GPU (rows x G >= 160k, about
    // 32 warps per SM) while every lane keeps two blocks on average (one
    // when the operator has so few rows that fewer than 40k threads would
    // work on it); measured on the 80^3 hierarchy, each choice is within a
    // few percent of the best power of two
    const double avg = B.nbr ? (double)B.nnzb / B.nbr : 0.0;
    if (B.br != 6) max_lanes = std::min(max_lanes, 32);  // wide rows: 6-row blocks only
    int G = 1;
    while (G < max_lanes && (int64_t)B.nbr * G < 160000 &&
           avg / (2 * G) >= ((int64_t)B.nbr * G < 40000 ? 1.0 : 2.0))
        G <<= 1;
    S.G = G;
    const int bb = B.br * B.bc;
    const bool wide = G > 32;
    const int nrows = B.nbr, rpg = wide ? 1 : 32 / G, spg = wide ? G / 32 : 1;
    int ngroups = (nrows + rpg - 1) / rpg;
    while (wide && (int64_t)ngroups * spg % 4 != 0) ++ngroups;
    S.nslices = nrows > 0 ? ngroups * spg : 0;
    const int nslots = ngroups * rpg;
    std::vector<int> wh(std::max(S.nslices, 1), 0);
    if (S.nslices > 0) {
        int *w = nullptr, *pw = nullptr;
        unsigned long long *tot = nullptr;
        DevArena tmp;  // temporaries of this conversion (same supplier as the handle's)
        tmp.stream = s;
        struct Release {
            DevArena &a;
            ~Release() { a.release_all(); }
        } release_tmp{tmp};
        AMG_TRY(tmp.alloc_n(&w, (size_t)S.nslices));
        AMG_TRY(tmp.alloc_n(&tot, 2));
        AMG_TRY_CUDA(cudaMemsetAsync(tot, 0, sizeof(unsigned long long) * 2, s));
        sell_group_width_kernel<<<(ngroups + 255) / 256, 256, 0, s>>>(B.row_ptr, nrows, G, rpg, spg,
                                                                      ngroups, nullptr, w, tot);
        count_launch(1);
        AMG_TRY_CUDA(cudaGetLastError());
        unsigned long long ht[2] = {0, 0};
        AMG_TRY_CUDA(cudaMemcpyAsync(ht, tot, sizeof(ht[0]), cudaMemcpyDeviceToHost, s));
        AMG_TRY_CUDA(cudaStreamSynchronize(s));
        const int64_t nat = (int64_t)ht[0];
        bool sorted = false;
        if (B.nnzb > 0 && (double)(nat - B.nnzb) > 0.05 * (double)B.nnzb) {
            const int win = 32 * rpg;
            AMG_TRY(tmp.alloc_n(&pw, (size_t)nslots));
            AMG_TRY_CUDA(cudaMemsetAsync(pw, 0xff, sizeof(int) * nslots, s));  // -1: padding slots
            sell_window_rank_kernel<<<(nrows + win - 1) / win, 256, 0, s>>>(B.row_ptr, nrows, win, pw);
            sell_group_width_kernel<<<(ngroups + 255) / 256, 256, 0, s>>>(
                B.row_ptr, nrows, G, rpg, spg, ngroups, pw, w, tot + 1);
            count_launch(2);
            AMG_TRY_CUDA(cudaGetLastError());
            AMG_TRY_CUDA(cudaMemcpyAsync(ht + 1, tot + 1, sizeof(ht[1]), cudaMemcpyDeviceToHost, s));
            AMG_TRY_CUDA(cudaStreamSynchronize(s));
            sorted = (int64_t)ht[1] < nat;
        }
        if (!sorted && pw) {  // the sort does not pay: natural widths again
            AMG_TRY_CUDA(cudaMemsetAsync(tot, 0, sizeof(unsigned long long), s));
            sell_group_width_kernel<<<(ngroups + 255) / 256, 256, 0, s>>>(
                B.row_ptr, nrows, G, rpg, spg, ngroups, nullptr, w, tot);
            count_launch(1);
            AMG_TRY_CUDA(cudaGetLastError());
        }
        AMG_TRY_CUDA(cudaMemcpyAsync(wh.data(), w, sizeof(int) * S.nslices, cudaMemcpyDeviceToHost, s));
        AMG_TRY_CUDA(cudaStreamSynchronize(s));
        if (sorted) {
            // widest groups first, ties in ascending group order (a stable
            // counting sort on the group widths)
            std::vector<int> cost(ngroups, 0);
            int cmax = 0;
            for (int g = 0; g < ngroups; ++g) {
                for (int q = 0; q < spg; ++q) cost[g] += wh[(size_t)g * spg + q];
                cmax = std::max(cmax, cost[g]);
            }
            std::vector<int> start(cmax + 2, 0), order(ngroups);
            for (int g = 0; g < ngroups; ++g) start[cmax - cost[g] + 1]++;
            for (int c = 0; c <= cmax; ++c) start[c + 1] += start[c];
            for (int g = 0; g < ngroups; ++g) order[start[cmax - cost[g]]++] = g;
            std::vector<int> w2(wh);
            for (int k = 0; k < ngroups; ++k)
                for (int q = 0; q < spg; ++q) wh[(size_t)k * spg + q] = w2[(size_t)order[k] * spg + q];
            int *dorder = nullptr;
            AMG_TRY(tmp.alloc_n(&dorder, (size_t)ngroups));
            AMG_TRY_CUDA(cudaMemcpyAsync(dorder, order.data(), sizeof(int) * ngroups,
                                         cudaMemcpyHostToDevice, s));
            AMG_TRY(keep.alloc_n(&S.perm, (size_t)nslots));
            sell_gather_groups_kernel<<<(ngroups + 255) / 256, 256, 0, s>>>(dorder, pw, ngroups, rpg,
                                                                            S.perm);
            count_launch(1);
            AMG_TRY_CUDA(cudaGetLastError());
            AMG_TRY_CUDA(cudaStreamSynchronize(s));  // order is host memory
        }
    }
    std::vector<int64_t> sp(S.nslices + 1, 0);
    for (int i = 0; i < S.nslices; ++i) sp[i + 1] = sp[i] + 32LL * wh[i];
    S.nslots = sp[S.nslices];
    AMG_TRY(keep.alloc_n(&S.slice_ptr, S.nslices + 1));
    AMG_TRY(keep.alloc_n(&S.col, (size_t)std::max<int64_t>(S.nslots, 1)));
    AMG_TRY(keep.alloc_n(&S.val, (size_t)std::max<int64_t>(S.nslots, 1) * bb));
    AMG_TRY_CUDA(cudaMemcpyAsync(S.slice_ptr, sp.data(), sizeof(int64_t) * (S.nslices + 1),
                                 cudaMemcpyHostToDevice, s));
    if (S.nslices > 0) {
        sell_fill_kernel<T><<<(S.nslices * 32 + 127) / 128, 128, 0, s>>>(
            B.row_ptr, B.col, B.val, B.nbr, S.nslices, bb, G, S.perm, S.slice_ptr, S.col, S.val);
        count_launch(1);
        AMG_TRY_CUDA(cudaGetLastError());
    }
    AMG_TRY_CUDA(cudaStreamSynchronize(s));  // sp is host memory
    if (padding) *padding = B.nnzb ? (double)(S.nslots - B.nnzb) / (double)B.nnzb : 0.0;
    *out = S;
    return AMG_OK;
}

template <class T> int64_t sell_bytes(const Sell<T> &S)
{
    if (!S.slice_ptr) return 0;
    const int rslots = S.G > 32 ? S.nslices / (S.G / 32) : S.nslices * (32 / S.G);
    return S.nslots * (int64_t)(S.br * S.bc * sizeof(T) + sizeof(int)) +
           (int64_t)(S.nslices + 1) * (int64_t)sizeof(int64_t) +
           (S.perm ? (int64_t)rslots * (int64_t)sizeof(int) : 0);
}
template int64_t sell_bytes<double>(const Sell<double> &);
template int64_t sell_bytes<float>(const Sell<float> &);
template int64_t sell_bytes<__nv_bfloat16>(const Sell<__nv_bfloat16> &);
template int64_t sell_bytes<df32>(const Sell<df32> &);

template int bsr_to_sell<double>(const BsrD &, DevArena &, cudaStream_t, Sell<double> *, double *,
                                 int);
template int bsr_to_sell<float>(const BsrD &, DevArena &, cudaStream_t, Sell<float> *, double *,
                                int);
template int bsr_to_sell<__nv_bfloat16>(const BsrD &, DevArena &, cudaStream_t,
                                        Sell<__nv_bfloat16> *, double *, int);
template int bsr_to_sell<df32>(const BsrD &, DevArena &, cudaStream_t, Sell<df32> *, double *,
                               int);

}  // namespace amg
