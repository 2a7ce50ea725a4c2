// Batched form: many independent elasticity instances, each with several
// load cases, solved together by one graph launch.
//
// Every instance gets its own hierarchy from the single-instance setup
// (Alg. 1 with the same parameters), so its levels, omega and smoother are
// exactly those of a solve of that instance alone.  For the solve, level l of
// all instances that still smooth on level l is gathered into one
// concatenated sliced operator (A_l, P_l, R_l): the slices of each instance
// keep their own layout (their lanes-per-row G) and carry the instance id, so
// one kernel launch serves the level of every instance.  Vectors hold the K
// right-hand sides of an instance interleaved (row-major [dof][K]), and the
// SpMM loads every block once per tile of KT right-hand sides.  KT is chosen
// per operator at setup by timing the candidates (the autotuner).
//
// Each (instance, right-hand side) pair runs its own preconditioned CG
// (Sec. 4) with its own scalars; a pair that has converged stops updating,
// and an instance whose pairs have all converged drops out of the kernels.
// Dot products are reduced per instance in a fixed order over fixed chunks,
// so an instance solved inside a batch gives bitwise the same iterates as the
// same instance solved alone through this path.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <system_error>
#include <thread>

#include "amg_internal.cuh"

namespace amg {

constexpr int BKMAX = 16;       // right-hand sides per instance
constexpr int BCHUNK = 2048;    // dofs per dot-product chunk
constexpr int BT = 128;         // default threads of the SpMM CTAs (autotuned: 64, 128, 256)
constexpr int BT_MAX = 256;
constexpr int BSETUP_THREADS = 8;  // host threads setting up instances at once
// the block smoother's two epilogues (block damped Jacobi): SPMV_SMOOTHB for
// u + M_I (f - A u) and this one for the restriction whose next-level
// pre-smoothing is a block product (y2 = M_I y)
constexpr int BMODE_RESTRICTB = 6;

// Concatenated sliced operator of one level.
struct BSell {
    int nslices = 0, br = 0, bc = 0, kt = 1;
    int cta = BT, cap = 32;      // launch shape: threads per CTA (32 / G block rows per warp),
                                 // at most cap CTAs per SM
    int64_t *slice_ptr = nullptr;
    int *col = nullptr;
    double *val = nullptr;
    df32 *eval = nullptr;        // the same values as FP32 pairs (AMG_PREC_DF64 V-cycle)
    float *fval = nullptr;       // the same values rounded to FP32 (AMG_PREC_FP32 V-cycle)
    int *s_inst = nullptr, *s_local = nullptr, *s_G = nullptr;
    int *perm = nullptr;         // concatenated slot -> row maps of the sorted parts
    int64_t *s_pbase = nullptr;  // per slice: its first slot in perm, or -1 (natural order)
    int *order = nullptr;        // slices widest first over all instances
};

struct BArgs {
    int nslices;
    const int64_t *slice_ptr;
    const int *col;
    const double *val;
    const df32 *eval;
    const float *fval;
    const int *s_inst, *s_local, *s_G;
    const int *perm;
    const int64_t *s_pbase;
    const int *order;
    const int *K;           // right-hand sides per instance
    const int *nrows;       // block rows of the output space per instance
    const int64_t *xoff;    // instance offsets of x's space
    const int64_t *yoff;    // instance offsets of y's space (and of f, u)
    const int64_t *moff;    // instance offsets of the smoother diagonal (-1: none)
    const int *enable;      // per instance: run this instance
    const double *x, *f, *u, *M;
    const double *Mb;       // smoother blocks (SPMV_SMOOTHB: this level's; BMODE_RESTRICTB:
                            // the next level's), instance i's from moff[i] * BR
    double *y, *y2;
};

// VK: values and arithmetic of the block products -- 0 FP64, 1 FP32 pairs
// (emulated FP64), 2 FP32 (x rounded to FP32, FP32 FMAs); vectors FP64.
template <int BR, int BC, int KT, int MODE, int VK>
__global__ void __launch_bounds__(BT_MAX) bspmm_kernel(BArgs a)
{
    constexpr bool DF = VK == 1, F32 = VK == 2;
    constexpr int BB = BR * BC;
    const int lane = threadIdx.x & 31;
    const int nw = (int)((gridDim.x * (unsigned)blockDim.x) >> 5);
    for (int k = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5); k < a.nslices;
         k += nw) {
        const int s = a.order[k];
        const int inst = a.s_inst[s];
        if (!a.enable[inst]) continue;
        const int G = a.s_G[s], sub = lane & (G - 1);
        const int64_t pb = a.s_pbase[s];
        const int row = pb >= 0 ? a.perm[pb + lane / G] : a.s_local[s] * (32 / G) + lane / G;
        const int K = a.K[inst];
        const bool live = row >= 0 && row < a.nrows[inst];
        const int64_t base = a.slice_ptr[s];
        const int w = (int)((a.slice_ptr[s + 1] - base) >> 5);
        const double *vp = a.val + base * BB + lane;
        const int *cp = a.col + base + lane;
        const double *xb = a.x + a.xoff[inst];
        const int64_t yo = a.yoff[inst];
        for (int k0 = 0; k0 < K; k0 += KT) {
            double acc[BR][KT];
            float sh[BR][KT], sl[BR][KT];  // FP32-pair accumulators (DF); sh alone for F32
#pragma unroll
            for (int r = 0; r < BR; ++r)
#pragma unroll
                for (int t = 0; t < KT; ++t) {
                    acc[r][t] = 0.0;
                    sh[r][t] = sl[r][t] = 0.0f;
                }
            for (int d = 0; d < w; ++d) {
                const int j = __ldg(cp + d * 32);
                double xv[BC][KT];
#pragma unroll
                for (int c = 0; c < BC; ++c)
#pragma unroll
                    for (int t = 0; t < KT; ++t)
                        xv[c][t] = (k0 + t < K) ? __ldg(xb + ((int64_t)j * BC + c) * K + k0 + t) : 0.0;
                if constexpr (F32) {
                    // FP32 values in the FP64 lane-pair layout (one 8-byte
                    // load per two entries), x rounded to FP32, FP32 FMAs
                    const float *fg = a.fval + (base + (int64_t)d * 32) * BB;
                    float vf[BB];
#pragma unroll
                    for (int pr = 0; pr < BB / 2; ++pr) {
                        const float2 t2 = __ldg(reinterpret_cast<const float2 *>(fg + pr * 64) + lane);
                        vf[2 * pr] = t2.x;
                        vf[2 * pr + 1] = t2.y;
                    }
                    if constexpr (BB % 2 == 1) vf[BB - 1] = __ldg(fg + (BB / 2) * 64 + lane);
                    float xf[BC][KT];
#pragma unroll
                    for (int c = 0; c < BC; ++c)
#pragma unroll
                        for (int t = 0; t < KT; ++t) xf[c][t] = f64_to_f32_rn(xv[c][t]);
#pragma unroll
                    for (int r = 0; r < BR; ++r)
#pragma unroll
                        for (int c = 0; c < BC; ++c)
#pragma unroll
                            for (int t = 0; t < KT; ++t)
                                sh[r][t] = fmaf(vf[r * BC + c], xf[c][t], sh[r][t]);
                    continue;
                }
                if constexpr (DF) {
                    // FP64 emulated on FP32 pairs, as in the single-instance
                    // SELL kernel: hi/lo value pairs in the FP64 lane-pair
                    // layout, x split on the bits, error-free FP32 products
                    // and a renormalised double-float sum per (row, rhs)
                    const df32 *eg = a.eval + (base + (int64_t)d * 32) * BB;
                    float vh[BB], vl[BB];
#pragma unroll
                    for (int pr = 0; pr < BB / 2; ++pr) {
                        const float4 t4 = __ldg(reinterpret_cast<const float4 *>(eg + pr * 64) + lane);
                        vh[2 * pr] = t4.x;
                        vl[2 * pr] = t4.y;
                        vh[2 * pr + 1] = t4.z;
                        vl[2 * pr + 1] = t4.w;
                    }
                    if constexpr (BB % 2 == 1) {
                        const float2 t2 = __ldg(reinterpret_cast<const float2 *>(eg + (BB / 2) * 64) + lane);
                        vh[BB - 1] = t2.x;
                        vl[BB - 1] = t2.y;
                    }
                    float xh[BC][KT], xl[BC][KT];
#pragma unroll
                    for (int c = 0; c < BC; ++c)
#pragma unroll
                        for (int t = 0; t < KT; ++t) split_f64(xv[c][t], xh[c][t], xl[c][t]);
#pragma unroll
                    for (int r = 0; r < BR; ++r)
#pragma unroll
                        for (int c = 0; c < BC; ++c)
#pragma unroll
                            for (int t = 0; t < KT; ++t) {
                                const float ah = vh[r * BC + c], al = vl[r * BC + c];
                                const float pv = __fmul_rn(ah, xh[c][t]);
                                float er = __fmaf_rn(ah, xh[c][t], -pv);
                                er = __fmaf_rn(ah, xl[c][t], er);
                                er = __fmaf_rn(al, xh[c][t], er);
                                const float sn = __fadd_rn(sh[r][t], pv);
                                const float bv = __fsub_rn(sn, sh[r][t]);
                                float te = __fadd_rn(__fsub_rn(sh[r][t], __fsub_rn(sn, bv)),
                                                     __fsub_rn(pv, bv));
                                te = __fadd_rn(te, __fadd_rn(sl[r][t], er));
                                sh[r][t] = __fadd_rn(sn, te);
                                sl[r][t] = __fsub_rn(te, __fsub_rn(sh[r][t], sn));
                            }
                    continue;
                }
                // FP64 sliced values: entries 2p, 2p+1 of a lane side by
                // side (one 16-byte load), an odd last entry after the pairs
                // (the layout of sell.cu)
                const double *vg = vp - lane + (int64_t)d * 32 * BB;
                double v[BB];
#pragma unroll
                for (int pr = 0; pr < BB / 2; ++pr) {
                    const double2 t2 = __ldg(reinterpret_cast<const double2 *>(vg + pr * 64) + lane);
                    v[2 * pr] = t2.x;
                    v[2 * pr + 1] = t2.y;
                }
                if constexpr (BB % 2 == 1) v[BB - 1] = __ldg(vg + (BB / 2) * 64 + lane);
#pragma unroll
                for (int r = 0; r < BR; ++r)
#pragma unroll
                    for (int c = 0; c < BC; ++c)
#pragma unroll
                        for (int t = 0; t < KT; ++t)
                            acc[r][t] = fma(v[r * BC + c], xv[c][t], acc[r][t]);
            }
            if constexpr (DF)
#pragma unroll
                for (int r = 0; r < BR; ++r)
#pragma unroll
                    for (int t = 0; t < KT; ++t) acc[r][t] = f32_to_f64(sh[r][t]) + f32_to_f64(sl[r][t]);
            if constexpr (F32)
#pragma unroll
                for (int r = 0; r < BR; ++r)
#pragma unroll
                    for (int t = 0; t < KT; ++t) acc[r][t] = f32_to_f64(sh[r][t]);
            for (int m = G >> 1; m >= 1; m >>= 1)
#pragma unroll
                for (int r = 0; r < BR; ++r)
#pragma unroll
                    for (int t = 0; t < KT; ++t)
                        acc[r][t] += __shfl_xor_sync(0xffffffffu, acc[r][t], m);
            if (sub != 0 || !live) continue;
            if constexpr (MODE == SPMV_SMOOTHB || MODE == BMODE_RESTRICTB) {
                // block epilogues: the row's BR x BR block times its BR residuals
                // (smoothing) or its BR outputs (the next level's pre-smoothing)
                const int64_t mo = a.moff[inst];
                const double *mb = mo >= 0 ? a.Mb + (mo + (int64_t)row * BR) * BR : nullptr;
#pragma unroll
                for (int t = 0; t < KT; ++t) {
                    const int k = k0 + t;
                    if (k >= K) continue;
                    double v[BR];
#pragma unroll
                    for (int c = 0; c < BR; ++c) {
                        const int64_t i = yo + ((int64_t)row * BR + c) * K + k;
                        v[c] = MODE == SPMV_SMOOTHB ? a.f[i] - acc[c][t] : acc[c][t];
                        if (MODE == BMODE_RESTRICTB) a.y[i] = acc[c][t];
                    }
#pragma unroll
                    for (int r = 0; r < BR; ++r) {
                        const int64_t i = yo + ((int64_t)row * BR + r) * K + k;
                        double corr = 0.0;
                        if (mb)
#pragma unroll
                            for (int c = 0; c < BR; ++c) corr = fma(mb[r * BR + c], v[c], corr);
                        if (MODE == SPMV_SMOOTHB) a.y[i] = a.x[i] + corr;
                        else if (a.y2) a.y2[i] = corr;
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < BR; ++r)
#pragma unroll
                    for (int t = 0; t < KT; ++t) {
                        const int k = k0 + t;
                        if (k >= K) continue;
                        const int64_t i = yo + ((int64_t)row * BR + r) * K + k;
                        double out;
                        if (MODE == SPMV_PLAIN) out = acc[r][t];
                        else if (MODE == SPMV_RESID) out = a.f[i] - acc[r][t];
                        else if (MODE == SPMV_SMOOTH)
                            out = a.x[i] + a.M[a.moff[inst] + (int64_t)row * BR + r] * (a.f[i] - acc[r][t]);
                        else if (MODE == SPMV_AXPY) out = a.u[i] + acc[r][t];
                        else out = acc[r][t];
                        a.y[i] = out;
                        if (MODE == SPMV_RESTRICT && a.y2) {
                            const int64_t mo = a.moff[inst];
                            a.y2[i] = (mo >= 0) ? a.M[mo + (int64_t)row * BR + r] * out : 0.0;
                        }
                    }
            }
        }
    }
}

template <int BR, int BC, int MODE>
static int bspmm_kt(const BSell &S, int kt, const BArgs &a, int grid, cudaStream_t s)
{
    const int vk = a.eval ? 1 : (a.fval ? 2 : 0);
#define AMG_BSPMM(KT_)                                                                        \
    do {                                                                                      \
        if (vk == 1) bspmm_kernel<BR, BC, KT_, MODE, 1><<<grid, S.cta, 0, s>>>(a);            \
        else if (vk == 2) bspmm_kernel<BR, BC, KT_, MODE, 2><<<grid, S.cta, 0, s>>>(a);       \
        else bspmm_kernel<BR, BC, KT_, MODE, 0><<<grid, S.cta, 0, s>>>(a);                    \
    } while (0)
    switch (kt) {
    case 1: AMG_BSPMM(1); break;
    case 2: AMG_BSPMM(2); break;
    default: AMG_BSPMM(4); break;
    }
#undef AMG_BSPMM
    count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    return AMG_OK;
}

template <int BR, int BC>
static int bspmm_mode(const BSell &S, int kt, int mode, const BArgs &a, int grid, cudaStream_t s)
{
    switch (mode) {
    case SPMV_PLAIN: return bspmm_kt<BR, BC, SPMV_PLAIN>(S, kt, a, grid, s);
    case SPMV_RESID: return bspmm_kt<BR, BC, SPMV_RESID>(S, kt, a, grid, s);
    case SPMV_SMOOTH:
        if constexpr (BR == BC) return bspmm_kt<BR, BC, SPMV_SMOOTH>(S, kt, a, grid, s);
        break;
    case SPMV_AXPY: return bspmm_kt<BR, BC, SPMV_AXPY>(S, kt, a, grid, s);
    case SPMV_RESTRICT: return bspmm_kt<BR, BC, SPMV_RESTRICT>(S, kt, a, grid, s);
    case SPMV_SMOOTHB:
        if constexpr (BR == BC) return bspmm_kt<BR, BC, SPMV_SMOOTHB>(S, kt, a, grid, s);
        break;
    case BMODE_RESTRICTB:
        if constexpr (BR == 6) return bspmm_kt<BR, BC, BMODE_RESTRICTB>(S, kt, a, grid, s);
        break;
    default: break;
    }
    set_error("unsupported batched spmm mode %d", mode);
    return AMG_ERR_ARG;
}

// vk: the copy of the values to use -- 0 FP64, 1 FP32 pairs (the V-cycle of
// an AMG_PREC_DF64 batch), 2 FP32 (the V-cycle of an AMG_PREC_FP32 batch)
static int launch_bspmm(const BSell &S, int kt, int mode, BArgs a, const Geom &g, cudaStream_t s,
                        int vk = 0)
{
    if (S.nslices == 0) return AMG_OK;
    if ((vk == 1 && !S.eval) || (vk == 2 && !S.fval)) {
        set_error("no reduced copy of this batched operator");
        return AMG_ERR_STATE;
    }
    a.nslices = S.nslices;
    a.slice_ptr = S.slice_ptr;
    a.col = S.col;
    a.val = S.val;
    a.eval = vk == 1 ? S.eval : nullptr;
    a.fval = vk == 2 ? S.fval : nullptr;
    a.s_inst = S.s_inst;
    a.s_local = S.s_local;
    a.s_G = S.s_G;
    a.perm = S.perm;
    a.s_pbase = S.s_pbase;
    a.order = S.order;
    // one warp per slice, widest slices first, up to S.cap CTAs per SM (the
    // warp-strided loop covers the rest): the hardware scheduler balances the
    // instances' uneven rows
    const int wpc = S.cta / 32;
    int grid = (S.nslices + wpc - 1) / wpc;
    grid = std::min(grid, g.num_sms * S.cap);
    if (S.br == 3 && S.bc == 3) return bspmm_mode<3, 3>(S, kt, mode, a, grid, s);
    if (S.br == 6 && S.bc == 6) return bspmm_mode<6, 6>(S, kt, mode, a, grid, s);
    if (S.br == 3 && S.bc == 6) return bspmm_mode<3, 6>(S, kt, mode, a, grid, s);
    if (S.br == 6 && S.bc == 3) return bspmm_mode<6, 3>(S, kt, mode, a, grid, s);
    set_error("unsupported block shape");
    return AMG_ERR_ARG;
}

// ---------------------------------------------------------------- vectors
// Instance of element e of a level-0 batch vector (offsets ascending).
__device__ __forceinline__ int inst_of(const int64_t *off, int ninst, int64_t e)
{
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct BVec {
    int ninst;
    int64_t n;                 // total elements
    const int64_t *off;        // [ninst + 1] element offsets (level 0)
    const int *K;
    const int *goff;           // first global rhs index of each instance
};

// Dot products x . y per (instance, rhs): CTA per (instance, chunk of BCHUNK
// dofs); per-thread partial sums per rhs, then a fixed tree per rhs.
__global__ void __launch_bounds__(256) bdot_kernel(BVec v, const int *__restrict__ chunk_inst,
                                                   const int *__restrict__ chunk_first,
                                                   int nchunks, const int *__restrict__ enable,
                                                   const double *__restrict__ x,
                                                   const double *__restrict__ y,
                                                   double *__restrict__ part)
{
    __shared__ double red[256];
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int inst = chunk_inst[c];
        if (!enable[inst]) continue;
        const int K = v.K[inst];
        const int64_t off = v.off[inst];
        const int64_t ndof = (v.off[inst + 1] - off) / K;
        const int64_t d0 = (int64_t)(c - chunk_first[inst]) * BCHUNK;
        const int64_t d1 = min(d0 + BCHUNK, ndof);
        double acc[BKMAX];
#pragma unroll
        for (int k = 0; k < BKMAX; ++k) acc[k] = 0.0;
        for (int64_t dd = d0 + threadIdx.x; dd < d1; dd += 256)
#pragma unroll
            for (int k = 0; k < BKMAX; ++k)
                if (k < K) acc[k] += x[off + dd * K + k] * y[off + dd * K + k];
        for (int k = 0; k < K; ++k) {
            red[threadIdx.x] = acc[k];
            __syncthreads();
            for (int w = 128; w > 0; w >>= 1) {
                if (threadIdx.x < (unsigned)w) red[threadIdx.x] += red[threadIdx.x + w];
                __syncthreads();
            }
            if (threadIdx.x == 0) part[(int64_t)c * BKMAX + k] = red[0];
            __syncthreads();
        }
    }
}

// Sum of an instance's chunk partials, in chunk order: one thread per rhs.
__global__ void bseg_kernel(int ngl, const int *__restrict__ g_inst, const int *__restrict__ goff,
                            const int *__restrict__ chunk_first, const int *__restrict__ enable,
                            const double *__restrict__ part, double *__restrict__ out)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ngl) return;
    const int inst = g_inst[g];
    if (!enable[inst]) return;
    const int k = g - goff[inst];
    double s = 0.0;
    for (int c = chunk_first[inst]; c < chunk_first[inst + 1]; ++c) s += part[(int64_t)c * BKMAX + k];
    out[g] = s;
}

// Per-rhs CG state.
struct BState {
    double *nf, *rz, *pq, *alpha, *beta, *res, *res_true, *dot;
    int *it, *active, *check, *replace, *status;
    int *inst_active, *inst_check, *any_active;
};

// elementwise: p = z + beta p (active rhs); beta = 0 only on a pair's first
// iteration (a zero r.z later stops the pair as a breakdown), where p = z
// without reading p, which holds no earlier direction
__global__ void bdirection_kernel(BVec v, const int *__restrict__ active, const double *__restrict__ beta,
                                  const double *__restrict__ z, double *__restrict__ p)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < v.n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int inst = inst_of(v.off, v.ninst, e);
        const int g = v.goff[inst] + (int)((e - v.off[inst]) % v.K[inst]);
        if (active[g]) p[e] = beta[g] == 0.0 ? z[e] : z[e] + beta[g] * p[e];
    }
}

// u += alpha p ; r -= alpha q ; t0 = M r  (active rhs)
__global__ void bupdate_kernel(BVec v, const int *__restrict__ active, const double *__restrict__ alpha,
                               double *__restrict__ u, double *__restrict__ r,
                               const double *__restrict__ p, const double *__restrict__ q,
                               const double *__restrict__ M, const int64_t *__restrict__ moff,
                               double *__restrict__ t0)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < v.n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int inst = inst_of(v.off, v.ninst, e);
        const int K = v.K[inst];
        const int64_t le = e - v.off[inst];
        const int g = v.goff[inst] + (int)(le % K);
        if (!active[g]) continue;
        const double al = alpha[g];
        u[e] += al * p[e];
        const double ri = r[e] - al * q[e];
        r[e] = ri;
        if (t0) t0[e] = (moff[inst] >= 0) ? M[moff[inst] + le / K] * ri : 0.0;
    }
}

// r = rt ; t0 = M r (rhs whose residual is replaced)
__global__ void breplace_kernel(BVec v, const int *__restrict__ replace,
                                double *__restrict__ r, const double *__restrict__ rt,
                                const double *__restrict__ M, const int64_t *__restrict__ moff,
                                double *__restrict__ t0)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < v.n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int inst = inst_of(v.off, v.ninst, e);
        const int K = v.K[inst];
        const int64_t le = e - v.off[inst];
        const int g = v.goff[inst] + (int)(le % K);
        if (!replace[g]) continue;
        const double ri = rt[e];
        r[e] = ri;
        if (t0) t0[e] = (moff[inst] >= 0) ? M[moff[inst] + le / K] * ri : 0.0;
    }
}

// t0 = M_I r on level 0 with the block smoother (3 x 3 blocks per node), for
// every entry of the enabled instances: the next V-cycle's pre-smoothing from
// zero.  Vectors interleave an instance's K right-hand sides ([dof][K]);
// instance i's blocks start at moff[i] * 3.
__global__ void bblock_apply_kernel(BVec v, const int *__restrict__ enable,
                                    const double *__restrict__ Mb,
                                    const int64_t *__restrict__ moff,
                                    const double *__restrict__ r, double *__restrict__ t0)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < v.n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int inst = inst_of(v.off, v.ninst, e);
        if (!enable[inst]) continue;
        const int K = v.K[inst];
        const int64_t le = e - v.off[inst];
        const int64_t dof = le / K;
        const int k = (int)(le % K);
        const int64_t node = dof / 3;
        const int rr = (int)(dof % 3);
        const int64_t mo = moff[inst];
        if (mo < 0) {
            t0[e] = 0.0;
            continue;
        }
        const double *m = Mb + (mo + node * 3) * 3 + rr * 3;
        const double *rb = r + v.off[inst] + node * 3 * K + k;
        double val = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) val = fma(m[c], rb[(int64_t)c * K], val);
        t0[e] = val;
    }
}

// t0 = M r for all rhs (start of the solve)
__global__ void bscale_kernel(BVec v, const double *__restrict__ r, const double *__restrict__ M,
                              const int64_t *__restrict__ moff, double *__restrict__ t0)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < v.n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int inst = inst_of(v.off, v.ninst, e);
        const int64_t le = e - v.off[inst];
        t0[e] = (moff[inst] >= 0) ? M[moff[inst] + le / v.K[inst]] * r[e] : 0.0;
    }
}

// RHS-major user vectors <-> interleaved batch vectors (one instance)
__global__ void interleave_kernel(const double *__restrict__ src, double *__restrict__ dst,
                                  int64_t ndof, int K)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ndof * K;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = e / K;
        const int k = (int)(e % K);
        dst[e] = src[(int64_t)k * ndof + d];
    }
}

__global__ void deinterleave_kernel(const double *__restrict__ src, double *__restrict__ dst,
                                    int64_t ndof, int K)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ndof * K;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = e / K;
        const int k = (int)(e % K);
        dst[(int64_t)k * ndof + d] = src[e];
    }
}

// Per-rhs scalar steps, one CTA of 1024 threads over all rhs.
constexpr int BS_T = 1024;

__global__ void __launch_bounds__(BS_T) bstart_kernel(int ngl, BState st, const double *ff2,
                                                      const double *rr2, double tol)
{
    for (int g = threadIdx.x; g < ngl; g += BS_T) {
        const double nf = sqrt(ff2[g]);
        st.nf[g] = nf;
        const double res = nf > 0.0 ? sqrt(rr2[g]) / nf : 0.0;
        st.res[g] = res;
        st.res_true[g] = res;
        st.it[g] = 0;
        st.rz[g] = st.pq[g] = st.alpha[g] = st.beta[g] = 0.0;
        st.active[g] = (nf > 0.0 && res > tol) ? 1 : 0;
        st.check[g] = st.replace[g] = 0;
        st.status[g] = st.active[g] ? AMG_NOT_CONVERGED : AMG_OK;
    }
}

// per-instance flags from per-rhs flags (and the global any-active)
__device__ void bflags(int ninst, const int *goff, const int *flag, int *inst_flag, int *any)
{
    __shared__ int anyv;
    if (threadIdx.x == 0) anyv = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < ninst; i += BS_T) {
        int f = 0;
        for (int g = goff[i]; g < goff[i + 1]; ++g) f |= flag[g];
        inst_flag[i] = f;
        if (f) atomicOr(&anyv, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0 && any) *any = anyv;
}

__global__ void __launch_bounds__(BS_T) binit_flags_kernel(int ninst, const int *goff, BState st)
{
    bflags(ninst, goff, st.active, st.inst_active, st.any_active);
    for (int i = threadIdx.x; i < ninst; i += BS_T) st.inst_check[i] = 0;
}

__global__ void __launch_bounds__(BS_T) bbeta_kernel(int ngl, BState st, const double *rz)
{
    for (int g = threadIdx.x; g < ngl; g += BS_T) {
        if (!st.active[g]) continue;
        const double v = rz[g];
        if (!(v > 0.0) || !isfinite(v)) {
            st.status[g] = AMG_ERR_BREAKDOWN;
            st.active[g] = 0;
            continue;
        }
        st.beta[g] = (st.it[g] == 0) ? 0.0 : v / st.rz[g];
        st.rz[g] = v;
    }
}

__global__ void __launch_bounds__(BS_T) balpha_kernel(int ngl, BState st, const double *pq)
{
    for (int g = threadIdx.x; g < ngl; g += BS_T) {
        if (!st.active[g]) continue;
        const double v = pq[g];
        if (!(v > 0.0) || !isfinite(v)) {
            st.status[g] = AMG_ERR_BREAKDOWN;
            st.active[g] = 0;
            continue;
        }
        st.pq[g] = v;
        st.alpha[g] = st.rz[g] / v;
    }
}

__global__ void __launch_bounds__(BS_T) bres_kernel(int ngl, int ninst, const int *goff, BState st,
                                                    const double *rr, double tol)
{
    for (int g = threadIdx.x; g < ngl; g += BS_T) {
        st.check[g] = 0;
        if (!st.active[g]) continue;
        st.res[g] = sqrt(rr[g]) / st.nf[g];
        st.it[g] += 1;
        st.check[g] = st.res[g] <= tol ? 1 : 0;
    }
    __syncthreads();
    bflags(ninst, goff, st.check, st.inst_check, nullptr);
}

__global__ void __launch_bounds__(BS_T) bdecide_kernel(int ngl, int ninst, const int *goff, BState st,
                                                       const double *rtt, double tol, int maxiter,
                                                       cudaGraphConditionalHandle cond, int use_cond)
{
    for (int g = threadIdx.x; g < ngl; g += BS_T) {
        st.replace[g] = 0;
        if (!st.active[g]) continue;
        if (st.check[g]) {
            const double tr = sqrt(rtt[g]) / st.nf[g];
            st.res_true[g] = tr;
            if (tr <= tol) {
                st.active[g] = 0;
                st.status[g] = AMG_OK;
                continue;
            }
            st.replace[g] = 1;
        }
        if (st.it[g] >= maxiter) {
            st.active[g] = 0;
            st.status[g] = AMG_NOT_CONVERGED;
            st.replace[g] = 0;
        }
    }
    __syncthreads();
    bflags(ninst, goff, st.active, st.inst_active, st.any_active);
    __syncthreads();
    if (threadIdx.x == 0 && use_cond && !*st.any_active) cudaGraphSetConditional(cond, 0);
}

// Coarse right-hand sides of every enabled instance rounded to FP32 (VK 2)
// or split into FP32 pairs (VK 1), once per V-cycle, into one array indexed
// by coff (instance i's n_i K_i values from coff[i]): the coarse GEMV's inner
// loop then reads them as they are, without a conversion per product.
template <int VK>
__global__ void bcoarse_prep_kernel(int ninst, const int64_t *__restrict__ coff,
                                    const int *__restrict__ enable,
                                    double *const *__restrict__ fptr, void *__restrict__ out)
{
    const int64_t total = coff[ninst];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        int lo = 0, hi = ninst;  // coff[lo] <= e < coff[hi] (offsets strictly increase)
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (coff[mid] <= e) lo = mid;
            else hi = mid;
        }
        if (!enable[lo]) continue;
        const double v = fptr[lo][e - coff[lo]];
        if constexpr (VK == 2) static_cast<float *>(out)[e] = f64_to_f32_rn(v);
        else static_cast<df32 *>(out)[e] = df32(v);
    }
}

// Coarse solves of every instance at its own coarsest level: y_i = Ainv_i f_i
// for the instance's K right-hand sides; one warp per (instance, row).  The
// arithmetic follows the batch's V-cycle: FP64 (VK 0), FP64 emulated on FP32
// pairs (VK 1: the inverse as hi/lo pairs, the double-float product and sum
// of the SpMMs) or FP32 (VK 2: an FP32 copy of the inverse, FP32 FMAs); in
// the reduced forms the right-hand sides come from bcoarse_prep_kernel.
template <int VK>
__global__ void bcoarse_kernel(int nitems, const int *__restrict__ item_inst,
                               const int *__restrict__ item_row, const int *__restrict__ enable,
                               const int *__restrict__ nc, const int64_t *__restrict__ aoff,
                               const void *__restrict__ Ainv, const int64_t *__restrict__ coff,
                               const void *__restrict__ fconv, const int *__restrict__ K,
                               double *const *__restrict__ fptr, double *const *__restrict__ zptr)
{
    const int lane = threadIdx.x & 31;
    const int nw = (int)((gridDim.x * (unsigned)blockDim.x) >> 5);
    for (int t = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5); t < nitems; t += nw) {
        const int inst = item_inst[t];
        if (!enable[inst]) continue;
        const int row = item_row[t], n = nc[inst], Ki = K[inst];
        const int64_t r0 = aoff[inst] + (int64_t)row * n;
        // one pass over the row: each entry feeds the Ki right-hand sides'
        // sums (the row is read once, Ki independent chains); every sum runs
        // over the row in the same order whatever Ki is, so a pair's result
        // does not depend on how many right-hand sides share its instance
        double out[BKMAX];
        if constexpr (VK == 0) {
            const double *ar = static_cast<const double *>(Ainv) + r0;
            const double *f = fptr[inst];
            double acc[BKMAX];
#pragma unroll
            for (int k = 0; k < BKMAX; ++k) acc[k] = 0.0;
            for (int j = lane; j < n; j += 32) {
                const double a = ar[j];
                const double *fj = f + (int64_t)j * Ki;
#pragma unroll
                for (int k = 0; k < BKMAX; ++k)
                    if (k < Ki) acc[k] = fma(a, fj[k], acc[k]);
            }
#pragma unroll
            for (int k = 0; k < BKMAX; ++k) out[k] = acc[k];
        } else if constexpr (VK == 2) {
            const float *ar = static_cast<const float *>(Ainv) + r0;
            const float *f = static_cast<const float *>(fconv) + coff[inst];
            float acc[BKMAX];
#pragma unroll
            for (int k = 0; k < BKMAX; ++k) acc[k] = 0.0f;
            for (int j = lane; j < n; j += 32) {
                const float a = ar[j];
                const float *fj = f + (int64_t)j * Ki;
#pragma unroll
                for (int k = 0; k < BKMAX; ++k)
                    if (k < Ki) acc[k] = fmaf(a, fj[k], acc[k]);
            }
            // FP32 butterfly, then exactly to FP64
#pragma unroll
            for (int k = 0; k < BKMAX; ++k) {
                if (k >= Ki) break;
                float v = acc[k];
#pragma unroll
                for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
                out[k] = f32_to_f64(v);
            }
        } else {
            const df32 *ar = static_cast<const df32 *>(Ainv) + r0;
            const df32 *f = static_cast<const df32 *>(fconv) + coff[inst];
            float sh[BKMAX], sl[BKMAX];
#pragma unroll
            for (int k = 0; k < BKMAX; ++k) sh[k] = sl[k] = 0.0f;
            for (int j = lane; j < n; j += 32) {
                const df32 a = ar[j];
                const df32 *fj = f + (int64_t)j * Ki;
#pragma unroll
                for (int k = 0; k < BKMAX; ++k) {
                    if (k >= Ki) break;
                    const df32 x = fj[k];
                    // error-free product of the his plus the cross terms,
                    // then the renormalised double-float sum (nothing
                    // contracted: every rounding written out)
                    const float pv = __fmul_rn(a.h, x.h);
                    float er = __fmaf_rn(a.h, x.h, -pv);
                    er = __fmaf_rn(a.h, x.l, er);
                    er = __fmaf_rn(a.l, x.h, er);
                    const float sn = __fadd_rn(sh[k], pv);
                    const float bv = __fsub_rn(sn, sh[k]);
                    float te = __fadd_rn(__fsub_rn(sh[k], __fsub_rn(sn, bv)), __fsub_rn(pv, bv));
                    te = __fadd_rn(te, __fadd_rn(sl[k], er));
                    sh[k] = __fadd_rn(sn, te);
                    sl[k] = __fsub_rn(te, __fsub_rn(sh[k], sn));
                }
            }
#pragma unroll
            for (int k = 0; k < BKMAX; ++k) out[k] = f32_to_f64(sh[k]) + f32_to_f64(sl[k]);
        }
#pragma unroll
        for (int k = 0; k < BKMAX; ++k) {
            if (k >= Ki) break;
            double v = out[k];
            if constexpr (VK != 2)
#pragma unroll
                for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
            if (lane == 0) zptr[inst][(int64_t)row * Ki + k] = v;
        }
    }
}

}  // namespace amg

using namespace amg;

// One level of the batch: the concatenated operators of the instances that
// smooth on it, and the instance offsets of its vectors.
struct BLevelData {
    BSell A, P, R;
    double *M = nullptr;                 // concatenated smoother diagonals
    double *Mb = nullptr;                // ... and blocks (block damped Jacobi; from moff * br)
    int64_t *moff = nullptr;             // instance offsets into M (-1: none)
    int64_t *voff = nullptr;             // instance offsets of this level's vectors (-1: absent)
    int64_t *moff_next = nullptr;        // offsets of the next level's M (restriction epilogue)
    int *nrows = nullptr;                // block rows per instance (0 if absent)
    int *smooth = nullptr;               // instance smooths on this level (1) or not
    double *f = nullptr, *u = nullptr, *e = nullptr, *z = nullptr;
    int64_t len = 0;                     // vector length
};

struct amg_batch_s {
    amg_params prm;
    amg_allocator alloc{};               // copy of *prm.allocator (alloc == nullptr: none)
    const amg_allocator *allocator() const { return alloc.alloc ? &alloc : nullptr; }
    cudaStream_t stream = nullptr;
    Geom geom;
    DevArena mem;
    int ninst = 0, ngl = 0, nlev = 0;
    std::vector<amg_handle> inst;        // per-instance hierarchies (during setup only)
    std::vector<int> Kh, goffh, depth;   // host copies
    std::vector<int64_t> ndof0;
    std::vector<BLevelData> lv;
    int *K = nullptr, *goff = nullptr, *g_inst = nullptr;
    int64_t *off0 = nullptr;             // level-0 element offsets [ninst + 1]
    int *chunk_inst = nullptr, *chunk_first = nullptr;
    int nchunks = 0;
    // coarse
    double *Ainv = nullptr;              // FP64 inverses (FP64 V-cycle)
    void *AinvR = nullptr;               // ... rounded to FP32 or split into FP32 pairs
    int64_t *coff = nullptr;             // reduced forms: offsets of the converted rhs
    void *fconv = nullptr;               // ... and the converted coarse right-hand sides
    int64_t ctot = 0;
    int64_t *aoff = nullptr;
    int *nc = nullptr, *item_inst = nullptr, *item_row = nullptr;
    int nitems = 0;
    double **fptr = nullptr, **zptr = nullptr;
    // CG vectors (level 0 layout) and per-rhs state
    double *ff = nullptr, *uu = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *rt = nullptr,
           *part = nullptr;
    BState st{};
    int *all_on = nullptr;               // enable array with every instance on
    int *all_off = nullptr;              // ... and with every instance off (warm-up launches)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long body_kernels = 0;
    int host_loop = 0;  // exec is one iteration, launched by the host (loop_mode 1)
    int tol_maxiter_key = 0;
    double tol = 0;
    int maxiter = 0;
    double setup_seconds = 0;
    double phase_s[4] = {0, 0, 0, 0};  // instances, operators, coarse + state, autotune
    std::vector<int> kt_choice;          // autotuned RHS tile per (level, operator)
    std::vector<int> cta_choice, cap_choice;  // autotuned launch shape per (level, operator)
    int vk = 0;                          // V-cycle values: 0 FP64, 1 FP32 pairs, 2 FP32
};

static BVec bvec(amg_batch h)
{
    BVec v;
    v.ninst = h->ninst;
    v.n = h->lv[0].len;
    v.off = h->off0;
    v.K = h->K;
    v.goff = h->goff;
    return v;
}

static int bgrid(amg_batch h, int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g > h->geom.max_ctas) g = h->geom.max_ctas;
    return (int)std::max<int64_t>(g, 1);
}

static BArgs bargs(amg_batch h, const BLevelData &L, const int64_t *xoff, const int64_t *yoff,
                   const int *nrows, const int *enable)
{
    BArgs a{};
    a.K = h->K;
    a.nrows = nrows;
    a.xoff = xoff;
    a.yoff = yoff;
    a.enable = enable;
    (void)L;
    return a;
}

// batched dot x . y per rhs into out[g]
static int record_bdot(amg_batch h, const double *x, const double *y, const int *enable, double *out,
                       cudaStream_t s)
{
    int grid = std::min(h->nchunks, h->geom.num_sms * 8);
    bdot_kernel<<<std::max(grid, 1), 256, 0, s>>>(bvec(h), h->chunk_inst, h->chunk_first,
                                                  h->nchunks, enable, x, y, h->part);
    count_launch(1);
    bseg_kernel<<<(h->ngl + 127) / 128, 128, 0, s>>>(h->ngl, h->g_inst, h->goff, h->chunk_first,
                                                    enable, h->part, out);
    count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    return AMG_OK;
}

// Batched V-cycle: z0 = V(f0) for every enabled instance and rhs; level 0's u
// holds M_0 f0.
static int record_bvcycle(amg_batch h, const double *f0, double *z0, const int *enable,
                          cudaStream_t s)
{
    const Geom &g = h->geom;
    const int L = h->nlev - 1;
    int kti = 0;
    for (int l = 0; l < L; ++l) {
        BLevelData &C = h->lv[l];
        BLevelData &N = h->lv[l + 1];
        const double *f = (l == 0) ? f0 : C.f;
        {  // e = f - A u
            BArgs a = bargs(h, C, C.voff, C.voff, C.nrows, enable);
            a.x = C.u;
            a.f = f;
            a.y = C.e;
            AMG_TRY(launch_bspmm(C.A, C.A.kt, SPMV_RESID, a, g, s, h->vk));
        }
        {  // f_{l+1} = R e ; u_{l+1} = M_{l+1} f_{l+1}
            BArgs a = bargs(h, C, C.voff, N.voff, N.nrows, enable);
            a.x = C.e;
            a.y = N.f;
            a.y2 = N.u;
            a.M = N.M;
            a.Mb = N.Mb;
            a.moff = C.moff_next;
            AMG_TRY(launch_bspmm(C.R, C.R.kt, N.Mb ? BMODE_RESTRICTB : SPMV_RESTRICT, a, g, s,
                                 h->vk));
        }
        kti += 3;
    }
    {
        const int grid = std::max(std::min((h->nitems + 7) / 8, g.max_ctas), 1);
        if (h->vk) {
            const int pg = (int)std::max<int64_t>(1, std::min<int64_t>((h->ctot + 255) / 256,
                                                                       g.max_ctas));
            if (h->vk == 1)
                bcoarse_prep_kernel<1><<<pg, 256, 0, s>>>(h->ninst, h->coff, enable, h->fptr, h->fconv);
            else
                bcoarse_prep_kernel<2><<<pg, 256, 0, s>>>(h->ninst, h->coff, enable, h->fptr, h->fconv);
            count_launch(1);
        }
#define BCOARSE_ARGS h->nitems, h->item_inst, h->item_row, enable, h->nc, h->aoff, \
                     h->vk ? h->AinvR : (const void *)h->Ainv, h->coff, h->fconv, h->K, h->fptr, h->zptr
        if (h->vk == 1) bcoarse_kernel<1><<<grid, 256, 0, s>>>(BCOARSE_ARGS);
        else if (h->vk == 2) bcoarse_kernel<2><<<grid, 256, 0, s>>>(BCOARSE_ARGS);
        else bcoarse_kernel<0><<<grid, 256, 0, s>>>(BCOARSE_ARGS);
#undef BCOARSE_ARGS
        count_launch(1);
        AMG_TRY_CUDA(cudaGetLastError());
    }
    for (int l = L - 1; l >= 0; --l) {
        BLevelData &C = h->lv[l];
        BLevelData &N = h->lv[l + 1];
        const double *f = (l == 0) ? f0 : C.f;
        double *zl = (l == 0) ? z0 : C.z;
        {  // u += P z_{l+1}
            BArgs a = bargs(h, C, N.voff, C.voff, C.nrows, enable);
            a.x = N.z;
            a.u = C.u;
            a.y = C.u;
            AMG_TRY(launch_bspmm(C.P, C.P.kt, SPMV_AXPY, a, g, s, h->vk));
        }
        {  // z = u + M (f - A u)
            BArgs a = bargs(h, C, C.voff, C.voff, C.nrows, enable);
            a.x = C.u;
            a.f = f;
            a.M = C.M;
            a.Mb = C.Mb;
            a.moff = C.moff;
            a.y = zl;
            AMG_TRY(launch_bspmm(C.A, C.A.kt, C.Mb ? SPMV_SMOOTHB : SPMV_SMOOTH, a, g, s, h->vk));
        }
    }
    return AMG_OK;
}

static int record_biteration(amg_batch h, cudaStream_t s, cudaGraphConditionalHandle cond,
                             int use_cond)
{
    BLevelData &L0 = h->lv[0];
    const Geom &g = h->geom;
    const int64_t n = L0.len;
    BState &st = h->st;
    const int ngl = h->ngl;
    AMG_TRY(record_bvcycle(h, h->r, L0.z, st.inst_active, s));
    AMG_TRY(record_bdot(h, h->r, L0.z, st.inst_active, st.dot, s));
    bbeta_kernel<<<1, BS_T, 0, s>>>(ngl, st, st.dot);
    count_launch(1);
    bdirection_kernel<<<bgrid(h, n), 256, 0, s>>>(bvec(h), st.active, st.beta, L0.z, h->p);
    count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    {  // q = A p
        BArgs a = bargs(h, L0, L0.voff, L0.voff, L0.nrows, st.inst_active);
        a.x = h->p;
        a.y = h->q;
        AMG_TRY(launch_bspmm(L0.A, L0.A.kt, SPMV_PLAIN, a, g, s));
    }
    AMG_TRY(record_bdot(h, h->p, h->q, st.inst_active, st.dot, s));
    balpha_kernel<<<1, BS_T, 0, s>>>(ngl, st, st.dot);
    count_launch(1);
    // the next pre-smoothing M r fused into the update (diagonal smoother) or,
    // with smoother blocks, one block product after the residual replacement
    const bool blocks = L0.Mb != nullptr;
    bupdate_kernel<<<bgrid(h, n), 256, 0, s>>>(bvec(h), st.active, st.alpha, h->uu, h->r, h->p,
                                               h->q, L0.M, L0.moff,
                                               (h->nlev > 1 && !blocks) ? L0.u : nullptr);
    count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    AMG_TRY(record_bdot(h, h->r, h->r, st.inst_active, st.dot, s));
    bres_kernel<<<1, BS_T, 0, s>>>(ngl, h->ninst, h->goff, st, st.dot, h->tol);
    count_launch(1);
    {  // true residual of the rhs that reached the tolerance
        BArgs a = bargs(h, L0, L0.voff, L0.voff, L0.nrows, st.inst_check);
        a.x = h->uu;
        a.f = h->ff;
        a.y = h->rt;
        AMG_TRY(launch_bspmm(L0.A, L0.A.kt, SPMV_RESID, a, g, s));
    }
    AMG_TRY(record_bdot(h, h->rt, h->rt, st.inst_check, st.dot, s));
    bdecide_kernel<<<1, BS_T, 0, s>>>(ngl, h->ninst, h->goff, st, st.dot, h->tol, h->maxiter, cond,
                                      use_cond);
    count_launch(1);
    breplace_kernel<<<bgrid(h, n), 256, 0, s>>>(bvec(h), st.replace, h->r, h->rt, L0.M, L0.moff,
                                                (h->nlev > 1 && !blocks) ? L0.u : nullptr);
    count_launch(1);
    if (h->nlev > 1 && blocks) {
        bblock_apply_kernel<<<bgrid(h, n), 256, 0, s>>>(bvec(h), st.inst_active, L0.Mb, L0.moff,
                                                        h->r, L0.u);
        count_launch(1);
    }
    AMG_TRY_CUDA(cudaGetLastError());
    return AMG_OK;
}

static int build_bgraph(amg_batch h)
{
    if (h->exec) {
        cudaGraphExecDestroy(h->exec);
        cudaGraphDestroy(h->graph);
        h->exec = nullptr;
        h->graph = nullptr;
    }
    if (h->prm.loop_mode == 1) {
        // one captured iteration, launched by the host until no pair is
        // active (for profilers that cannot look inside conditional graphs;
        // same kernels, same results)
        cudaStream_t cs;
        AMG_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        AMG_TRY_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        long long nbody = 0;
        begin_launch_capture(&nbody);
        int st = record_biteration(h, cs, cudaGraphConditionalHandle{}, 0);
        end_launch_capture();
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &graph);
        cudaStreamDestroy(cs);
        if (st < 0 || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            if (st >= 0) set_error("graph capture: %s", cudaGetErrorString(e));
            return st < 0 ? st : AMG_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&h->exec, graph, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            h->exec = nullptr;
            set_error("graph instantiate: %s", cudaGetErrorString(e));
            return AMG_ERR_CUDA;
        }
        h->graph = graph;
        h->body_kernels = nbody;
        h->host_loop = 1;
        return AMG_OK;
    }
    h->host_loop = 0;
    cudaGraph_t graph = nullptr;
    AMG_TRY_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle cond;
    AMG_TRY_CUDA(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    AMG_TRY_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t cs;
    AMG_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    AMG_TRY_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal));
    long long nbody = 0;
    begin_launch_capture(&nbody);
    int st = record_biteration(h, cs, cond, 1);
    end_launch_capture();
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &captured);
    cudaStreamDestroy(cs);
    if (st < 0 || e != cudaSuccess) {
        cudaGraphDestroy(graph);
        if (st >= 0) set_error("graph capture: %s", cudaGetErrorString(e));
        return st < 0 ? st : AMG_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&h->exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        h->exec = nullptr;
        set_error("graph instantiate: %s", cudaGetErrorString(e));
        return AMG_ERR_CUDA;
    }
    h->graph = graph;
    h->body_kernels = nbody;
    return AMG_OK;
}

// ---------------------------------------------------------------- setup
template <class T> static int upload(DevArena &m, const std::vector<T> &v, T **out, cudaStream_t s)
{
    AMG_TRY(m.alloc_n(out, std::max<size_t>(v.size(), 1)));
    if (!v.empty())
        AMG_TRY_CUDA(cudaMemcpyAsync(*out, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s));
    return AMG_OK;
}

// Concatenate the sliced operators `which` (0 A, 1 P, 2 R) of level l over the
// instances that smooth on level l.
__global__ void to_df32_kernel(const double *__restrict__ v, df32 *__restrict__ e, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) e[i] = df32(v[i]);
}

__global__ void to_f32_kernel(const double *__restrict__ v, float *__restrict__ f, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) f[i] = (float)v[i];
}

// The sliced operator `which` (0 A, 1 P, 2 R) of level l of instance i.
static const Sell<double> &inst_sell(amg_batch h, int i, int l, int which)
{
    const Level &L = h->inst[i]->lv[l];
    return which == 0 ? L.sA : which == 1 ? L.sP : L.sR;
}
// Concatenate sliced parts (null: the instance does not smooth on this
// level) into one operator held by the batch.
static int concat_parts(amg_batch h, const std::vector<const Sell<double> *> &parts, BSell *out)
{
    cudaStream_t s = h->stream;
    BSell S;
    std::vector<int> s_inst, s_local, s_G;
    std::vector<int64_t> sp(1, 0), s_pbase;
    int64_t nslots = 0, nperm = 0;
    int bb = 0;
    for (int i = 0; i < h->ninst; ++i) {
        if (!parts[i]) continue;
        const Sell<double> &X = *parts[i];
        S.br = X.br;
        S.bc = X.bc;
        bb = X.br * X.bc;
        std::vector<int64_t> xsp(X.nslices + 1);
        AMG_TRY_CUDA(cudaMemcpyAsync(xsp.data(), X.slice_ptr, sizeof(int64_t) * (X.nslices + 1),
                                     cudaMemcpyDeviceToHost, s));
        AMG_TRY_CUDA(cudaStreamSynchronize(s));
        const int rps = 32 / X.G;
        for (int k = 0; k < X.nslices; ++k) {
            s_inst.push_back(i);
            s_local.push_back(k);
            s_G.push_back(X.G);
            sp.push_back(nslots + xsp[k + 1]);
            s_pbase.push_back(X.perm ? nperm + (int64_t)k * rps : -1);
        }
        nslots += X.nslots;
        if (X.perm) nperm += (int64_t)X.nslices * rps;
    }
    S.nslices = (int)s_inst.size();
    if (S.nslices == 0) {
        *out = S;
        return AMG_OK;
    }
    AMG_TRY(upload(h->mem, sp, &S.slice_ptr, s));
    AMG_TRY(upload(h->mem, s_inst, &S.s_inst, s));
    AMG_TRY(upload(h->mem, s_local, &S.s_local, s));
    AMG_TRY(upload(h->mem, s_G, &S.s_G, s));
    AMG_TRY(upload(h->mem, s_pbase, &S.s_pbase, s));
    {
        std::vector<int> order(S.nslices);
        for (int k = 0; k < S.nslices; ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            return sp[x + 1] - sp[x] > sp[y + 1] - sp[y];
        });
        AMG_TRY(upload(h->mem, order, &S.order, s));
    }
    AMG_TRY(h->mem.alloc_n(&S.perm, (size_t)std::max<int64_t>(nperm, 1)));
    AMG_TRY(h->mem.alloc_n(&S.col, (size_t)nslots));
    AMG_TRY(h->mem.alloc_n(&S.val, (size_t)nslots * bb));
    int64_t at = 0, pat = 0;
    for (int i = 0; i < h->ninst; ++i) {
        if (!parts[i]) continue;
        const Sell<double> &X = *parts[i];
        if (X.perm) {
            const int64_t np = (int64_t)X.nslices * (32 / X.G);
            AMG_TRY_CUDA(cudaMemcpyAsync(S.perm + pat, X.perm, sizeof(int) * np,
                                         cudaMemcpyDeviceToDevice, s));
            pat += np;
        }
        AMG_TRY_CUDA(cudaMemcpyAsync(S.col + at, X.col, sizeof(int) * X.nslots,
                                     cudaMemcpyDeviceToDevice, s));
        AMG_TRY_CUDA(cudaMemcpyAsync(S.val + at * bb, X.val, sizeof(double) * X.nslots * bb,
                                     cudaMemcpyDeviceToDevice, s));
        at += X.nslots;
    }
    if (h->vk) {  // the values as FP32 pairs or FP32, element by element (same layout)
        const int64_t ne = nslots * bb;
        const unsigned grid = (unsigned)((ne + 255) / 256);
        if (h->vk == 1) AMG_TRY(h->mem.alloc_n(&S.eval, (size_t)std::max<int64_t>(ne, 1)));
        else AMG_TRY(h->mem.alloc_n(&S.fval, (size_t)std::max<int64_t>(ne, 1)));
        if (ne > 0) {
            if (h->vk == 1) to_df32_kernel<<<grid, 256, 0, s>>>(S.val, S.eval, ne);
            else to_f32_kernel<<<grid, 256, 0, s>>>(S.val, S.fval, ne);
            count_launch(1);
            AMG_TRY_CUDA(cudaGetLastError());
        }
    }
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    *out = S;
    return AMG_OK;
}

static int concat_sell(amg_batch h, int l, int which, BSell *out)
{
    std::vector<const Sell<double> *> parts(h->ninst, nullptr);
    for (int i = 0; i < h->ninst; ++i)
        if (l < h->depth[i] - 1) parts[i] = &inst_sell(h, i, l, which);  // smoothing levels only
    return concat_parts(h, parts, out);
}

// Time the RHS tiles 1, 2, 4 of an operator in PLAIN mode, one launch each
// after a launch with every instance disabled (which loads the kernel and
// does no work); return the best (and its time in *best_ms, if asked).
static int autotune_kt(amg_batch h, const BSell &S, const int64_t *xoff, const int64_t *yoff,
                       const int *nrows, const double *x, double *y, int *best,
                       float *best_ms = nullptr)
{
    *best = 1;
    if (best_ms) *best_ms = 0.f;
    if (S.nslices == 0) return AMG_OK;
    int kmax = *std::max_element(h->Kh.begin(), h->Kh.end());
    cudaStream_t s = h->stream;
    cudaEvent_t e0, e1;
    AMG_TRY_CUDA(cudaEventCreate(&e0));
    AMG_TRY_CUDA(cudaEventCreate(&e1));
    float bestt = 1e30f;
    for (int kt : {1, 2, 4}) {
        if (kt > 1 && kt > kmax) break;
        BArgs a{};
        a.K = h->K;
        a.nrows = nrows;
        a.xoff = xoff;
        a.yoff = yoff;
        a.enable = h->all_on;
        a.x = x;
        a.y = y;
        // a reduced-precision batch tunes the tile of the V-cycle's kernels
        a.enable = h->all_off;
        AMG_TRY(launch_bspmm(S, kt, SPMV_PLAIN, a, h->geom, s, h->vk));  // warm-up
        a.enable = h->all_on;
        AMG_TRY_CUDA(cudaEventRecord(e0, s));
        AMG_TRY(launch_bspmm(S, kt, SPMV_PLAIN, a, h->geom, s, h->vk));
        AMG_TRY_CUDA(cudaEventRecord(e1, s));
        AMG_TRY_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        AMG_TRY_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < bestt) {
            bestt = ms;
            *best = kt;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms) *best_ms = bestt;
    return AMG_OK;
}

// Time one launch of an operator in PLAIN mode with its own launch shape and
// RHS tile (the kernels are warm from the RHS-tile tuning).
static int time_shape(amg_batch h, const BSell &S, const int64_t *xoff, const int64_t *yoff,
                      const int *nrows, const double *x, double *y, cudaEvent_t e0,
                      cudaEvent_t e1, float *ms)
{
    BArgs a{};
    a.K = h->K;
    a.nrows = nrows;
    a.xoff = xoff;
    a.yoff = yoff;
    a.enable = h->all_on;
    a.x = x;
    a.y = y;
    cudaStream_t s = h->stream;
    AMG_TRY_CUDA(cudaEventRecord(e0, s));
    AMG_TRY(launch_bspmm(S, S.kt, SPMV_PLAIN, a, h->geom, s, h->vk));
    AMG_TRY_CUDA(cudaEventRecord(e1, s));
    AMG_TRY_CUDA(cudaEventSynchronize(e1));
    AMG_TRY_CUDA(cudaEventElapsedTime(ms, e0, e1));
    return AMG_OK;
}

// Block-row tiling of one concatenated operator (the autotuner's second
// axis): the launch shape, i.e. how many warps (each one slice of 32 / G
// block rows) a CTA holds -- 64, 128 or 256 threads -- and how many CTAs an
// SM may take before the warp-strided loop wraps -- 16 or 32.  The RHS tile
// is tuned at the default shape (128 threads, 32 CTAs per SM); every other
// shape is then timed with that tile, and the fastest replaces the default
// when it is more than 3 % faster.  The shape only schedules the same
// per-row work, so results do not depend on the choice (lanes per row, which
// would change each row's summation split, stay the size heuristic's).
static int autotune_tiling(amg_batch h, BSell *cur, const int64_t *xoff, const int64_t *yoff,
                           const int *nrows, const double *x, double *y)
{
    if (cur->nslices == 0) return AMG_OK;
    cur->cta = BT;
    cur->cap = 32;
    float best = 0.f;  // the default shape's time at the chosen tile
    AMG_TRY(autotune_kt(h, *cur, xoff, yoff, nrows, x, y, &cur->kt, &best));
    cudaEvent_t e0, e1;
    AMG_TRY_CUDA(cudaEventCreate(&e0));
    AMG_TRY_CUDA(cudaEventCreate(&e1));
    int st = AMG_OK;
    const BSell base = *cur;
    for (int cta : {64, 128, 256})
        for (int cap : {16, 32}) {
            if (st < 0 || (cta == BT && cap == 32)) continue;
            BSell cand = base;
            cand.cta = cta;
            cand.cap = cap;
            float ms = 0.f;
            st = time_shape(h, cand, xoff, yoff, nrows, x, y, e0, e1, &ms);
            if (st >= 0 && ms < 0.97f * best) {
                best = ms;
                cur->cta = cta;
                cur->cap = cap;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

static void bdestroy(amg_batch h)
{
    if (!h) return;
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    for (amg_handle x : h->inst) destroy_handle(x);
    if (h->mem.has_custom()) {
        cudaDeviceSynchronize();  // see destroy_handle
        h->mem.release_all();
    } else {
        h->mem.release_all();
        if (h->stream) cudaStreamSynchronize(h->stream);
        else cudaDeviceSynchronize();
    }
    delete h;
}

// Streams of the setup threads: BSETUP_THREADS non-blocking streams per
// device, created on first use and kept for the life of the process.  A
// caller-supplied allocator receives the stream an allocation is made for,
// and a caching allocator (PyTorch's) keeps freed blocks for reuse on that
// stream only: streams that outlive one setup let the next setup reuse them,
// where a fresh stream per setup would leave them stranded.
static int setup_stream(int dev, int w, cudaStream_t *out)
{
    constexpr int kDev = 64;
    static cudaStream_t table[kDev][BSETUP_THREADS] = {};
    static std::mutex mu;
    if (dev < 0 || dev >= kDev || w < 0 || w >= BSETUP_THREADS) {
        set_error("setup stream: device %d, thread %d out of range", dev, w);
        return AMG_ERR_LIMIT;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!table[dev][w]) AMG_TRY_CUDA(cudaStreamCreateWithFlags(&table[dev][w], cudaStreamNonBlocking));
    *out = table[dev][w];
    return AMG_OK;
}

// The instances' hierarchies are independent problems: up to BSETUP_THREADS
// host threads take instances in index order, each setting them up on a
// setup stream of its own that first waits for the caller's stream (where
// the inputs were written).  One instance's host aggregation and
// synchronisations then overlap the kernels of the others.  Every instance
// runs the same kernels on the same inputs as when it is set up alone, so
// its hierarchy does not depend on the thread or on the other instances.
// Once a thread has finished, the instance's memory and later work belong to
// the caller's stream.  On failure the lowest-numbered failing instance is
// reported, its number before its message (instances are started in index
// order, so every lower one has been set up); no thread starts an instance
// after a failure.
static int setup_instances(amg_batch h, const amg_bsr *A, const double *const *B)
{
    const int ni = h->ninst;
    cudaStream_t s = h->stream;
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    const int nw = std::min(ni, std::min(BSETUP_THREADS, hw));
    if (nw <= 1) {
        for (int i = 0; i < ni; ++i) {
            const int st = setup_impl(h->inst[i], &A[i], B[i]);
            if (st < 0) {
                const std::string m = last_error();
                set_error("instance %d: %s", i, m.c_str());
                return st;
            }
        }
        return AMG_OK;
    }
    int dev = 0;
    AMG_TRY_CUDA(cudaGetDevice(&dev));
    cudaEvent_t ready;
    AMG_TRY_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    if (cudaEventRecord(ready, s) != cudaSuccess) {
        cudaEventDestroy(ready);
        AMG_TRY_CUDA(cudaGetLastError());
    }
    std::vector<int> status(ni, 1);  // 1 = not started
    std::vector<std::string> msg(ni);
    std::atomic<int> next{0};
    std::atomic<bool> failed{false};
    const amg_allocator *alloc = h->allocator();
    auto worker = [&](int w) {
        cudaStream_t ws = nullptr;
        int ok = cudaSetDevice(dev) == cudaSuccess ? setup_stream(dev, w, &ws) : AMG_ERR_CUDA;
        if (ok >= 0 && cudaStreamWaitEvent(ws, ready, 0) != cudaSuccess) ok = AMG_ERR_CUDA;
        const std::string why = ok >= 0 ? std::string() : std::string(last_error());
        AllocScope scope(alloc);
        for (;;) {
            if (failed.load()) break;
            const int i = next.fetch_add(1);
            if (i >= ni) break;
            amg_handle x = h->inst[i];
            int st;
            if (ok < 0) {
                set_error("instance setup stream: %s", why.c_str());
                st = ok;
            } else {
                x->stream = ws;
                x->mem.stream = ws;
                st = no_throw([&] { return setup_impl(x, &A[i], B[i]); });
                cudaStreamSynchronize(ws);  // nothing of the instance stays queued on ws
                x->stream = s;
                x->mem.stream = s;
            }
            status[i] = st < 0 ? st : 0;
            if (st < 0) {
                msg[i] = last_error();
                failed.store(true);
            }
        }
    };
    std::vector<std::thread> pool;
    pool.reserve(nw);
    for (int w = 0; w < nw; ++w) {
        try {
            pool.emplace_back(worker, w);
        } catch (const std::system_error &) {
            break;  // fewer threads: those started take every instance
        }
    }
    if (pool.empty()) worker(0);  // no thread could be started: this one does the work
    for (std::thread &t : pool) t.join();
    cudaEventDestroy(ready);
    for (int i = 0; i < ni; ++i)
        if (status[i] < 0) {
            set_error("instance %d: %s", i, msg[i].c_str());
            return status[i];
        }
    return AMG_OK;
}

static int bsetup_impl(amg_batch h, const amg_bsr *A, const double *const *B, const int32_t *nrhs)
{
    if (h->prm.storage != AMG_STORAGE_BLOCK || h->prm.setup != AMG_SETUP_BLOCK) {
        set_error("the batched solve uses block storage and the block setup");
        return AMG_ERR_ARG;
    }
    cudaStream_t s = h->stream;
    AMG_TRY(query_geom(&h->geom));
    const int ni = h->ninst;
    h->Kh.assign(nrhs, nrhs + ni);
    h->goffh.assign(ni + 1, 0);
    for (int i = 0; i < ni; ++i) h->goffh[i + 1] = h->goffh[i] + h->Kh[i];
    h->ngl = h->goffh[ni];
    // per-instance hierarchies (Alg. 1), FP64 sliced copies for every level
    for (int i = 0; i < ni; ++i) {
        amg_handle x = new amg_handle_s();
        x->prm = h->prm;
        x->alloc = h->alloc;
        x->prm.precision = AMG_PREC_FP64;  // FP64 sliced copies; the batch makes its pair copies
        x->stream = s;
        x->mem.stream = s;
        x->max_lanes = 32;  // the batched SpMM keeps each row within one warp
        h->inst.push_back(x);
    }
    auto tp = std::chrono::steady_clock::now();
    auto lap = [&](int k) {  // wall time of phase k (the stream drained first)
        cudaStreamSynchronize(s);
        const auto now = std::chrono::steady_clock::now();
        h->phase_s[k] = std::chrono::duration<double>(now - tp).count();
        tp = now;
    };
    AMG_TRY(setup_instances(h, A, B));
    lap(0);
    for (int i = 0; i < ni; ++i) {
        h->depth.push_back((int)h->inst[i]->lv.size());
        h->ndof0.push_back((int64_t)h->inst[i]->lv[0].n());
    }
    h->nlev = *std::max_element(h->depth.begin(), h->depth.end());
    std::vector<int> gi(h->ngl);
    for (int i = 0; i < ni; ++i)
        for (int g = h->goffh[i]; g < h->goffh[i + 1]; ++g) gi[g] = i;
    AMG_TRY(upload(h->mem, h->Kh, &h->K, s));
    AMG_TRY(upload(h->mem, h->goffh, &h->goff, s));
    AMG_TRY(upload(h->mem, gi, &h->g_inst, s));
    std::vector<int> on(ni, 1), off(ni, 0);
    AMG_TRY(upload(h->mem, on, &h->all_on, s));
    AMG_TRY(upload(h->mem, off, &h->all_off, s));
    // levels: vector offsets, smoother diagonals, concatenated operators
    h->lv.resize(h->nlev);
    for (int l = 0; l < h->nlev; ++l) {
        BLevelData &D = h->lv[l];
        std::vector<int64_t> voff(ni, -1), moff(ni, -1);
        std::vector<int> nrows(ni, 0), smooth(ni, 0);
        int64_t len = 0, mlen = 0;
        for (int i = 0; i < ni; ++i) {
            if (l >= h->depth[i]) continue;
            const Level &L = h->inst[i]->lv[l];
            voff[i] = len;
            len += (int64_t)L.n() * h->Kh[i];
            nrows[i] = L.A.nbr;
            if (l < h->depth[i] - 1) {
                smooth[i] = 1;
                moff[i] = mlen;
                mlen += L.n();
            }
        }
        D.len = len;
        AMG_TRY(upload(h->mem, voff, &D.voff, s));
        AMG_TRY(upload(h->mem, moff, &D.moff, s));
        AMG_TRY(upload(h->mem, nrows, &D.nrows, s));
        AMG_TRY(upload(h->mem, smooth, &D.smooth, s));
        AMG_TRY(h->mem.alloc_n(&D.M, (size_t)std::max<int64_t>(mlen, 1)));
        for (int i = 0; i < ni; ++i)
            if (moff[i] >= 0)
                AMG_TRY_CUDA(cudaMemcpyAsync(D.M + moff[i], h->inst[i]->lv[l].M,
                                             sizeof(double) * h->inst[i]->lv[l].n(),
                                             cudaMemcpyDeviceToDevice, s));
        if (h->prm.smoother == AMG_SMOOTH_BJACOBI) {
            // the instances' block damped Jacobi blocks, br x br per block row
            // (br = 3 on level 0, 6 below), instance i's from moff[i] * br
            int br = 0;
            for (int i = 0; i < ni; ++i)
                if (moff[i] >= 0) br = h->inst[i]->lv[l].A.br;
            if (br > 0) {
                AMG_TRY(h->mem.alloc_n(&D.Mb, (size_t)std::max<int64_t>(mlen * br, 1)));
                for (int i = 0; i < ni; ++i) {
                    if (moff[i] < 0) continue;
                    const Level &Li = h->inst[i]->lv[l];
                    if (!Li.Mb || Li.A.br != br) {
                        set_error("instance %d: level %d has no %dx%d smoother blocks", i, l, br, br);
                        return AMG_ERR_STATE;
                    }
                    AMG_TRY_CUDA(cudaMemcpyAsync(D.Mb + moff[i] * br, Li.Mb,
                                                 sizeof(double) * Li.n() * br,
                                                 cudaMemcpyDeviceToDevice, s));
                }
            }
        }
        const size_t vl = (size_t)std::max<int64_t>(len, 1);
        if (l > 0) AMG_TRY(h->mem.alloc_n(&D.f, vl));
        AMG_TRY(h->mem.alloc_n(&D.u, vl));
        AMG_TRY(h->mem.alloc_n(&D.e, vl));
        AMG_TRY(h->mem.alloc_n(&D.z, vl));
        AMG_TRY(concat_sell(h, l, 0, &D.A));
        AMG_TRY(concat_sell(h, l, 1, &D.P));
        AMG_TRY(concat_sell(h, l, 2, &D.R));
    }
    for (int l = 0; l + 1 < h->nlev; ++l) h->lv[l].moff_next = h->lv[l + 1].moff;
    if (h->nlev > 0) {
        std::vector<int64_t> none(ni, -1);
        AMG_TRY(upload(h->mem, none, &h->lv[h->nlev - 1].moff_next, s));
    }
    // level-0 element offsets and dot chunks
    std::vector<int64_t> off0(ni + 1, 0);
    std::vector<int> cinst, cfirst(ni + 1, 0);
    for (int i = 0; i < ni; ++i) {
        off0[i + 1] = off0[i] + h->ndof0[i] * h->Kh[i];
        const int nch = (int)((h->ndof0[i] + BCHUNK - 1) / BCHUNK);
        cfirst[i + 1] = cfirst[i] + nch;
        for (int c = 0; c < nch; ++c) cinst.push_back(i);
    }
    h->nchunks = cfirst[ni];
    AMG_TRY(upload(h->mem, off0, &h->off0, s));
    AMG_TRY(upload(h->mem, cinst, &h->chunk_inst, s));
    AMG_TRY(upload(h->mem, cfirst, &h->chunk_first, s));
    AMG_TRY(h->mem.alloc_n(&h->part, (size_t)std::max(h->nchunks, 1) * BKMAX));
    lap(1);
    // coarse solves: each instance's dense inverse at its own coarsest level
    std::vector<int64_t> aoff(ni, 0);
    std::vector<int> nc(ni), iinst, irow;
    std::vector<double *> fp(ni), zp(ni);
    int64_t atot = 0;
    for (int i = 0; i < ni; ++i) {
        amg_handle x = h->inst[i];
        nc[i] = x->nc;
        aoff[i] = atot;
        atot += (int64_t)x->nc * x->nc;
        const int Li = h->depth[i] - 1;
        BLevelData &D = h->lv[Li];
        int64_t vo = 0;
        AMG_TRY_CUDA(cudaMemcpyAsync(&vo, D.voff + i, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        AMG_TRY_CUDA(cudaStreamSynchronize(s));
        fp[i] = (Li == 0) ? nullptr : D.f + vo;
        zp[i] = D.z + vo;
        for (int r = 0; r < x->nc; ++r) {
            iinst.push_back(i);
            irow.push_back(r);
        }
    }
    AMG_TRY(h->mem.alloc_n(&h->Ainv, (size_t)std::max<int64_t>(atot, 1)));
    for (int i = 0; i < ni; ++i)
        AMG_TRY_CUDA(cudaMemcpyAsync(h->Ainv + aoff[i], h->inst[i]->Ainv,
                                     sizeof(double) * h->inst[i]->nc * h->inst[i]->nc,
                                     cudaMemcpyDeviceToDevice, s));
    if (h->vk) {
        // the reduced V-cycles solve their coarse levels in their own
        // arithmetic: the inverses rounded to FP32 or split into FP32 pairs
        // (the FP64 copy goes), and room for the converted right-hand sides
        const int64_t ne = std::max<int64_t>(atot, 1);
        const unsigned cg = (unsigned)((ne + 255) / 256);
        if (h->vk == 1) {
            df32 *e = nullptr;
            AMG_TRY(h->mem.alloc_n(&e, (size_t)ne));
            to_df32_kernel<<<cg, 256, 0, s>>>(h->Ainv, e, atot);
            h->AinvR = e;
        } else {
            float *f = nullptr;
            AMG_TRY(h->mem.alloc_n(&f, (size_t)ne));
            to_f32_kernel<<<cg, 256, 0, s>>>(h->Ainv, f, atot);
            h->AinvR = f;
        }
        count_launch(1);
        AMG_TRY_CUDA(cudaGetLastError());
        AMG_TRY_CUDA(cudaStreamSynchronize(s));
        h->mem.release(h->Ainv);
        h->Ainv = nullptr;
        std::vector<int64_t> coff(ni + 1, 0);
        for (int i = 0; i < ni; ++i) coff[i + 1] = coff[i] + (int64_t)nc[i] * h->Kh[i];
        h->ctot = coff[ni];
        AMG_TRY(upload(h->mem, coff, &h->coff, s));
        const size_t nconv = (size_t)std::max<int64_t>(h->ctot, 1);
        if (h->vk == 1) {
            df32 *e = nullptr;
            AMG_TRY(h->mem.alloc_n(&e, nconv));
            h->fconv = e;
        } else {
            float *f = nullptr;
            AMG_TRY(h->mem.alloc_n(&f, nconv));
            h->fconv = f;
        }
    }
    h->nitems = (int)iinst.size();
    AMG_TRY(upload(h->mem, aoff, &h->aoff, s));
    AMG_TRY(upload(h->mem, nc, &h->nc, s));
    AMG_TRY(upload(h->mem, iinst, &h->item_inst, s));
    AMG_TRY(upload(h->mem, irow, &h->item_row, s));
    // CG vectors and state
    const size_t n0 = (size_t)std::max<int64_t>(h->lv[0].len, 1);
    AMG_TRY(h->mem.alloc_n(&h->ff, n0));
    AMG_TRY(h->mem.alloc_n(&h->uu, n0));
    AMG_TRY(h->mem.alloc_n(&h->r, n0));
    AMG_TRY(h->mem.alloc_n(&h->p, n0));
    AMG_TRY(h->mem.alloc_n(&h->q, n0));
    AMG_TRY(h->mem.alloc_n(&h->rt, n0));
    const size_t G = (size_t)std::max(h->ngl, 1);
    BState &st = h->st;
    for (double **pp : {&st.nf, &st.rz, &st.pq, &st.alpha, &st.beta, &st.res, &st.res_true, &st.dot})
        AMG_TRY(h->mem.alloc_n(pp, G));
    for (int **pp : {&st.it, &st.active, &st.check, &st.replace, &st.status})
        AMG_TRY(h->mem.alloc_n(pp, G));
    AMG_TRY(h->mem.alloc_n(&st.inst_active, (size_t)ni));
    AMG_TRY(h->mem.alloc_n(&st.inst_check, (size_t)ni));
    AMG_TRY(h->mem.alloc_n(&st.any_active, 1));
    // level-0 coarse pointer: an instance whose only level is level 0 solves
    // from the CG residual directly (f pointer filled per solve below)
    AMG_TRY(upload(h->mem, fp, &h->fptr, s));
    AMG_TRY(upload(h->mem, zp, &h->zptr, s));
    lap(2);
    // autotune the block-row tiling and the RHS tile of every concatenated
    // operator (PLAIN mode, on zeroed vectors)
    AMG_TRY_CUDA(cudaMemsetAsync(h->p, 0, sizeof(double) * n0, s));
    for (int l = 0; l < h->nlev; ++l) {
        BLevelData &D = h->lv[l];
        const bool has_next = l + 1 < h->nlev;
        for (double *v : {D.z, D.e})
            if (v) AMG_TRY_CUDA(cudaMemsetAsync(v, 0, sizeof(double) * (size_t)std::max<int64_t>(D.len, 1), s));
        AMG_TRY(autotune_tiling(h, &D.A, D.voff, D.voff, D.nrows, D.z, D.e));
        if (has_next) {
            BLevelData &N = h->lv[l + 1];
            for (double *v : {N.z, N.e})
                if (v) AMG_TRY_CUDA(cudaMemsetAsync(v, 0, sizeof(double) * (size_t)std::max<int64_t>(N.len, 1), s));
            AMG_TRY(autotune_tiling(h, &D.P, N.voff, D.voff, D.nrows, N.z, D.e));
            AMG_TRY(autotune_tiling(h, &D.R, D.voff, N.voff, N.nrows, D.z, N.e));
        }
        for (const BSell *op : {&D.A, &D.P, &D.R}) {
            h->kt_choice.push_back(op->kt);
            h->cta_choice.push_back(op->nslices ? op->cta : 0);
            h->cap_choice.push_back(op->nslices ? op->cap : 0);
        }
    }
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    lap(3);
    // the batch holds copies of everything its solve reads (operators,
    // smoother diagonals, coarse inverses): the instances' own hierarchies go
    for (amg_handle x : h->inst) destroy_handle(x);
    h->inst.clear();
    return AMG_OK;
}

extern "C" {

int amg_batch_setup(int32_t ninst, const amg_bsr *A, const double *const *B, const int32_t *nrhs,
                    const amg_params *prm, void *stream, amg_batch *out)
{
    clear_error();
    if (!out || ninst < 1 || !A || !B || !nrhs) {
        set_error("amg_batch_setup: bad argument");
        return AMG_ERR_ARG;
    }
    *out = nullptr;
    for (int i = 0; i < ninst; ++i) {
        if (nrhs[i] < 1 || nrhs[i] > BKMAX) {
            set_error("instance %d: nrhs must be in 1..%d", i, BKMAX);
            return AMG_ERR_ARG;
        }
        if (!B[i] || A[i].bs_r != 3 || A[i].bs_c != 3 || A[i].nbrows < 1 ||
            A[i].nbrows != A[i].nbcols || !A[i].row_ptr || !A[i].col || !A[i].val) {
            set_error("instance %d: expects a non-empty square 3x3 BSR matrix and B", i);
            return AMG_ERR_ARG;
        }
    }
    amg_params p;
    amg_params_default(&p);
    if (prm) p = *prm;
    if (p.precision == AMG_PREC_BF16 || p.npre != 1 || p.npost != 1 ||
        (p.smoother != AMG_SMOOTH_SPAI0 && p.smoother != AMG_SMOOTH_BJACOBI)) {
        set_error("the batched solve runs FP64, emulated-FP64 or FP32 V(1,1) cycles with the "
                  "SPAI0 or block Jacobi smoother");
        return AMG_ERR_ARG;
    }
    auto t0 = std::chrono::steady_clock::now();
    if (p.allocator && (!p.allocator->alloc || !p.allocator->free)) {
        set_error("amg_params.allocator needs both alloc and free");
        return AMG_ERR_ARG;
    }
    amg_batch h = new amg_batch_s();
    h->prm = p;
    if (p.allocator) h->alloc = *p.allocator;
    h->prm.allocator = nullptr;
    AllocScope scope(h->allocator());
    h->vk = p.precision == AMG_PREC_DF64 ? 1 : (p.precision == AMG_PREC_FP32 ? 2 : 0);
    h->stream = (cudaStream_t)stream;
    h->mem.stream = h->stream;
    h->ninst = ninst;
    int st = no_throw([&] { return bsetup_impl(h, A, B, nrhs); });
    if (st < 0) {
        std::string msg = amg::last_error();
        bdestroy(h);
        set_error("%s", msg.c_str());
        return st;
    }
    h->setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return AMG_OK;
}

void amg_batch_free(amg_batch h) { bdestroy(h); }

int amg_batch_solve(amg_batch h, const double *const *F, double *const *U, double tol,
                    int32_t maxiter, int32_t *iters, double *rel_resid, void *stream)
{
    clear_error();
    if (!h || !F || !U || !(tol > 0.0) || maxiter < 1 || maxiter > 1000000) {
        set_error("amg_batch_solve: bad argument");
        return AMG_ERR_ARG;
    }
    AllocScope scope(h->allocator());
    cudaStream_t s = (cudaStream_t)stream;
    const int ni = h->ninst;
    BLevelData &L0 = h->lv[0];
    // user vectors (rhs-major per instance) -> interleaved batch vectors
    std::vector<int64_t> off0(ni + 1, 0);
    for (int i = 0; i < ni; ++i) off0[i + 1] = off0[i] + h->ndof0[i] * h->Kh[i];
    for (int i = 0; i < ni; ++i) {
        if (!F[i] || !U[i]) {
            set_error("instance %d: null vector", i);
            return AMG_ERR_ARG;
        }
        interleave_kernel<<<bgrid(h, h->ndof0[i] * h->Kh[i]), 256, 0, s>>>(F[i], h->ff + off0[i],
                                                                          h->ndof0[i], h->Kh[i]);
        interleave_kernel<<<bgrid(h, h->ndof0[i] * h->Kh[i]), 256, 0, s>>>(U[i], h->uu + off0[i],
                                                                          h->ndof0[i], h->Kh[i]);
        count_launch(2);
    }
    AMG_TRY_CUDA(cudaGetLastError());
    // instances with a single level solve from r directly
    bool fp_dirty = false;
    std::vector<double *> fp(ni);
    AMG_TRY_CUDA(cudaMemcpyAsync(fp.data(), h->fptr, sizeof(double *) * ni, cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < ni; ++i)
        if (h->depth[i] == 1 && fp[i] != h->r + off0[i]) {
            fp[i] = h->r + off0[i];
            fp_dirty = true;
        }
    if (fp_dirty)
        AMG_TRY_CUDA(cudaMemcpyAsync(h->fptr, fp.data(), sizeof(double *) * ni, cudaMemcpyHostToDevice, s));
    // r = f - A u, norms, state
    BState &st = h->st;
    {
        BArgs a{};
        a.K = h->K;
        a.nrows = L0.nrows;
        a.xoff = L0.voff;
        a.yoff = L0.voff;
        a.enable = h->all_on;
        a.x = h->uu;
        a.f = h->ff;
        a.y = h->r;
        AMG_TRY(launch_bspmm(L0.A, L0.A.kt, SPMV_RESID, a, h->geom, s));
    }
    AMG_TRY(record_bdot(h, h->ff, h->ff, h->all_on, st.nf, s));
    AMG_TRY(record_bdot(h, h->r, h->r, h->all_on, st.res, s));
    bstart_kernel<<<1, BS_T, 0, s>>>(h->ngl, st, st.nf, st.res, tol);
    binit_flags_kernel<<<1, BS_T, 0, s>>>(ni, h->goff, st);
    count_launch(2);
    if (h->nlev > 1 && L0.Mb) {
        bblock_apply_kernel<<<bgrid(h, L0.len), 256, 0, s>>>(bvec(h), h->all_on, L0.Mb, L0.moff,
                                                             h->r, L0.u);
        count_launch(1);
    } else if (h->nlev > 1) {
        bscale_kernel<<<bgrid(h, L0.len), 256, 0, s>>>(bvec(h), h->r, L0.M, L0.moff, L0.u);
        count_launch(1);
    }
    AMG_TRY_CUDA(cudaGetLastError());
    int any = 0;
    AMG_TRY_CUDA(cudaMemcpyAsync(&any, st.any_active, sizeof(int), cudaMemcpyDeviceToHost, s));
    {  // a non-finite f or u would otherwise read as a zero right-hand side
        std::vector<double> nf0(h->ngl), res0(h->ngl);
        AMG_TRY_CUDA(cudaMemcpyAsync(nf0.data(), st.nf, sizeof(double) * h->ngl,
                                     cudaMemcpyDeviceToHost, s));
        AMG_TRY_CUDA(cudaMemcpyAsync(res0.data(), st.res, sizeof(double) * h->ngl,
                                     cudaMemcpyDeviceToHost, s));
        AMG_TRY_CUDA(cudaStreamSynchronize(s));
        for (int g = 0; g < h->ngl; ++g)
            if (!std::isfinite(nf0[g]) || !std::isfinite(res0[g])) {
                const int i = (int)(std::upper_bound(h->goffh.begin(), h->goffh.end(), g) -
                                    h->goffh.begin()) - 1;
                set_error("instance %d, right-hand side %d: f or u holds a non-finite value", i,
                          g - h->goffh[i]);
                return AMG_ERR_ARG;
            }
    }
    if (any) {
        if (!h->exec || h->tol != tol || h->maxiter != maxiter) {
            h->tol = tol;
            h->maxiter = maxiter;
            AMG_TRY(build_bgraph(h));
        }
        if (!h->host_loop) {
            AMG_TRY_CUDA(cudaGraphLaunch(h->exec, s));
        } else {
            for (int k = 0; k <= maxiter && any; ++k) {
                AMG_TRY_CUDA(cudaGraphLaunch(h->exec, s));
                AMG_TRY_CUDA(cudaMemcpyAsync(&any, st.any_active, sizeof(int),
                                             cudaMemcpyDeviceToHost, s));
                AMG_TRY_CUDA(cudaStreamSynchronize(s));
            }
        }
    }
    // u of a zero right-hand side is zero
    std::vector<double> nf(h->ngl), res(h->ngl), rest(h->ngl);
    std::vector<int> it(h->ngl), stat(h->ngl);
    AMG_TRY_CUDA(cudaMemcpyAsync(nf.data(), st.nf, sizeof(double) * h->ngl, cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaMemcpyAsync(res.data(), st.res, sizeof(double) * h->ngl, cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaMemcpyAsync(rest.data(), st.res_true, sizeof(double) * h->ngl, cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaMemcpyAsync(it.data(), st.it, sizeof(int) * h->ngl, cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaMemcpyAsync(stat.data(), st.status, sizeof(int) * h->ngl, cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    long long steps = 0;
    for (int g = 0; g < h->ngl; ++g) steps = std::max<long long>(steps, it[g]);
    count_launch(h->body_kernels * steps);
    // true residual of every rhs for the report
    {
        BArgs a{};
        a.K = h->K;
        a.nrows = L0.nrows;
        a.xoff = L0.voff;
        a.yoff = L0.voff;
        a.enable = h->all_on;
        a.x = h->uu;
        a.f = h->ff;
        a.y = h->rt;
        AMG_TRY(launch_bspmm(L0.A, L0.A.kt, SPMV_RESID, a, h->geom, s));
    }
    AMG_TRY(record_bdot(h, h->rt, h->rt, h->all_on, st.dot, s));
    std::vector<double> rr(h->ngl);
    AMG_TRY_CUDA(cudaMemcpyAsync(rr.data(), st.dot, sizeof(double) * h->ngl, cudaMemcpyDeviceToHost, s));
    for (int i = 0; i < ni; ++i) {
        deinterleave_kernel<<<bgrid(h, h->ndof0[i] * h->Kh[i]), 256, 0, s>>>(h->uu + off0[i], U[i],
                                                                            h->ndof0[i], h->Kh[i]);
        count_launch(1);
    }
    AMG_TRY_CUDA(cudaGetLastError());
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    int worst = AMG_OK;
    for (int g = 0; g < h->ngl; ++g) {
        const bool zero = nf[g] == 0.0;
        if (iters) iters[g] = it[g];
        if (rel_resid) rel_resid[g] = zero ? 0.0 : std::sqrt(rr[g]) / nf[g];
        if (zero) continue;
        if (stat[g] < 0) worst = std::min(worst, stat[g]);
        else if (stat[g] == AMG_NOT_CONVERGED && worst == AMG_OK) worst = AMG_NOT_CONVERGED;
    }
    // zero right-hand sides: u = 0
    for (int i = 0; i < ni; ++i)
        for (int k = 0; k < h->Kh[i]; ++k)
            if (nf[h->goffh[i] + k] == 0.0)
                AMG_TRY_CUDA(cudaMemsetAsync(U[i] + (int64_t)k * h->ndof0[i], 0,
                                             sizeof(double) * h->ndof0[i], s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    if (worst == AMG_ERR_BREAKDOWN) set_error("CG breakdown in at least one right-hand side");
    return worst;
}

int amg_batch_info(amg_batch h, amg_batch_desc *out)
{
    if (!h || !out) return AMG_ERR_ARG;
    std::memset(out, 0, sizeof *out);
    out->ninst = h->ninst;
    out->nrhs_total = h->ngl;
    out->nlevels = h->nlev;
    out->setup_seconds = h->setup_seconds;
    for (int k = 0; k < 4; ++k) out->setup_phase_seconds[k] = h->phase_s[k];
    int64_t dofs = 0;
    for (int i = 0; i < h->ninst; ++i) dofs += h->ndof0[i];
    out->dofs_total = dofs;
    const int nk = std::min<int>((int)h->kt_choice.size(), 48);
    for (int k = 0; k < nk; ++k) out->rhs_tile[k] = h->kt_choice[k];
    for (int k = 0; k < nk; ++k) {
        out->cta_threads[k] = h->cta_choice[k];
        out->ctas_per_sm[k] = h->cap_choice[k];
    }
    out->bytes_total = (int64_t)h->mem.bytes;
    for (amg_handle x : h->inst) out->bytes_total += (int64_t)x->mem.bytes;
    return AMG_OK;
}

}  // extern "C"
