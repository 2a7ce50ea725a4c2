// Learned fine-level smoother: a small MLP per block row in place of SPAI0.
//
// For every fine node I the network sees unit-free features of its block row
// (the diagonal block divided by its Frobenius norm, the sum of the squared
// neighbour-block norms and the largest neighbour-block norm relative to it,
// the number of blocks / 27), computes h = relu(W1 x + b1) (64 units) and
// o = W2 h + b2 (6 outputs), and the smoother block is
//     M_I = S_I L_I L_I^T S_I,   S_I = diag(sqrt(m_I)),
// m_I the damped SPAI0 diagonal of the node's three rows and L_I the lower
// triangular factor [[1+o0,0,0],[o3,1+o1,0],[o4,o5,1+o2]].  A zero output
// layer is exactly SPAI0; M_I is symmetric positive semidefinite for every
// output, so the V-cycle stays symmetric for CG; a block with a zero on the
// diagonal of L_I (singular) makes the whole smoother fall back to SPAI0.
//
// The two dense layers run on the tensor cores (mma.sync m16n8k16, BF16
// operands, FP32 accumulation): one warp per 16-row tile, the first layer's
// accumulator fragments re-packed in registers as the second layer's A
// operand.  Training minimises the energy-norm error reduction of one
// smoothing step, L = mean_s ||e_s - M A e_s||_A^2 / ||e_s||_A^2, over error
// samples the method itself produces (errors left by a V-cycle, and white
// noise, which carries the top of the spectrum); the loss gradient
// uses the solve's own sliced SpMV kernels, the MLP backward is FP32 with
// per-CTA partial sums reduced in a fixed order, and Adam updates FP32
// master weights from which the BF16 copies are refreshed.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "amg_internal.cuh"

namespace amg {

constexpr int LF = 12, LFP = 16, LH = 64, LO = 6, LOP = 8;
constexpr int LNPARAM = LH * LF + LH + LO * LH + LO;  // 1222, order W1 b1 W2 b2

// ---------------------------------------------------------------- block apply
template <class T>
__global__ void block_apply_kernel(const T *__restrict__ Mb, const T *__restrict__ r,
                                   T *__restrict__ out, int nrows)
{
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nrows; I += gridDim.x * blockDim.x) {
        const T *m = Mb + (int64_t)I * 9;
        const T r0 = r[3 * (int64_t)I], r1 = r[3 * (int64_t)I + 1], r2 = r[3 * (int64_t)I + 2];
#pragma unroll
        for (int a = 0; a < 3; ++a) out[3 * (int64_t)I + a] = m[3 * a] * r0 + m[3 * a + 1] * r1 + m[3 * a + 2] * r2;
    }
}

template <class T>
int launch_block_apply(const T *Mb, const T *r, T *out, int nrows, const Geom &g, cudaStream_t s)
{
    if (nrows == 0) return AMG_OK;
    int grid = std::min((nrows + 255) / 256, g.max_ctas);
    block_apply_kernel<T><<<grid, 256, 0, s>>>(Mb, r, out, nrows);
    count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    return AMG_OK;
}
template int launch_block_apply<double>(const double *, const double *, double *, int, const Geom &,
                                        cudaStream_t);
template int launch_block_apply<float>(const float *, const float *, float *, int, const Geom &,
                                       cudaStream_t);

__global__ void narrow9_kernel(const double *__restrict__ a, float *__restrict__ b, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// ---------------------------------------------------------------- features
__global__ void features_kernel(const int *__restrict__ rp, const int *__restrict__ col,
                                const double *__restrict__ val, int nrows,
                                __nv_bfloat16 *__restrict__ X)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nrows) return;
    int pd = rp[I];
    for (int p = rp[I]; p < rp[I + 1]; ++p)
        if (col[p] == I) pd = p;
    double d2 = 0.0;
    for (int e = 0; e < 9; ++e) d2 += val[(int64_t)pd * 9 + e] * val[(int64_t)pd * 9 + e];
    const double nI = sqrt(d2);
    double s2 = 0.0, mx = 0.0;
    for (int p = rp[I]; p < rp[I + 1]; ++p) {
        if (p == pd) continue;
        double b2 = 0.0;
        for (int e = 0; e < 9; ++e) b2 += val[(int64_t)p * 9 + e] * val[(int64_t)p * 9 + e];
        s2 += b2;
        mx = fmax(mx, sqrt(b2));
    }
    __nv_bfloat16 *x = X + (int64_t)I * LFP;
    for (int e = 0; e < 9; ++e) x[e] = __double2bfloat16(val[(int64_t)pd * 9 + e] / nI);
    x[9] = __double2bfloat16(s2 / d2);
    x[10] = __double2bfloat16(mx / nI);
    x[11] = __double2bfloat16((rp[I + 1] - rp[I]) / 27.0);
    for (int e = LF; e < LFP; ++e) x[e] = __float2bfloat16(0.0f);
}

// ---------------------------------------------------------------- MLP forward
struct MlpDev {
    const __nv_bfloat16 *W1;  // [64][16]
    const float *b1;          // [64]
    const __nv_bfloat16 *W2;  // [8][64], rows 6 and 7 zero
    const float *b2;          // [8]
};

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16 *p)
{
    return *reinterpret_cast<const uint32_t *>(p);
}

__device__ __forceinline__ uint32_t pack_pair(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4],
                                               const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One warp per 16-row tile.  Fragment layout of m16n8k16 (g = lane / 4,
// t = lane % 4): A regs {row g, cols 2t..2t+1}, {row g+8, same}, {row g,
// cols 2t+8..}, {row g+8, cols 2t+8..}; B regs {k 2t..2t+1, n g},
// {k 2t+8.., n g}; C {row g, cols 2t, 2t+1}, {row g+8, cols 2t, 2t+1}.
__global__ void mlp_forward_kernel(const __nv_bfloat16 *__restrict__ X, int nrows, int ntiles,
                                   MlpDev w, float *__restrict__ O, float *__restrict__ H)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int nw = (int)((gridDim.x * (unsigned)blockDim.x) >> 5);
    for (int tile = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5); tile < ntiles;
         tile += nw) {
        const int r0 = tile * 16 + g, r1 = r0 + 8;
        const __nv_bfloat16 *x0 = X + (int64_t)r0 * LFP, *x1 = X + (int64_t)r1 * LFP;
        uint32_t a[4] = {ld_pair(x0 + 2 * t), ld_pair(x1 + 2 * t), ld_pair(x0 + 2 * t + 8),
                         ld_pair(x1 + 2 * t + 8)};
        float c[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.0f;
            const __nv_bfloat16 *wr = w.W1 + (8 * j + g) * LFP;
            uint32_t b[2] = {ld_pair(wr + 2 * t), ld_pair(wr + 2 * t + 8)};
            mma_bf16_16816(c[j], a, b);
            const float bb0 = w.b1[8 * j + 2 * t], bb1 = w.b1[8 * j + 2 * t + 1];
            c[j][0] = fmaxf(c[j][0] + bb0, 0.0f);
            c[j][1] = fmaxf(c[j][1] + bb1, 0.0f);
            c[j][2] = fmaxf(c[j][2] + bb0, 0.0f);
            c[j][3] = fmaxf(c[j][3] + bb1, 0.0f);
            if (H) {
                if (r0 < nrows) {
                    H[(int64_t)r0 * LH + 8 * j + 2 * t] = c[j][0];
                    H[(int64_t)r0 * LH + 8 * j + 2 * t + 1] = c[j][1];
                }
                if (r1 < nrows) {
                    H[(int64_t)r1 * LH + 8 * j + 2 * t] = c[j][2];
                    H[(int64_t)r1 * LH + 8 * j + 2 * t + 1] = c[j][3];
                }
            }
        }
        float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t a2[4] = {pack_pair(c[2 * q][0], c[2 * q][1]), pack_pair(c[2 * q][2], c[2 * q][3]),
                              pack_pair(c[2 * q + 1][0], c[2 * q + 1][1]),
                              pack_pair(c[2 * q + 1][2], c[2 * q + 1][3])};
            const __nv_bfloat16 *wr = w.W2 + g * LH + 16 * q;
            uint32_t b2[2] = {ld_pair(wr + 2 * t), ld_pair(wr + 2 * t + 8)};
            mma_bf16_16816(d, a2, b2);
        }
        if (r0 < nrows) {
            O[(int64_t)r0 * LOP + 2 * t] = d[0] + w.b2[2 * t];
            O[(int64_t)r0 * LOP + 2 * t + 1] = d[1] + w.b2[2 * t + 1];
        }
        if (r1 < nrows) {
            O[(int64_t)r1 * LOP + 2 * t] = d[2] + w.b2[2 * t];
            O[(int64_t)r1 * LOP + 2 * t + 1] = d[3] + w.b2[2 * t + 1];
        }
    }
}

// M_I = S L L^T S and the check that L (hence M_I) is nonsingular.
__global__ void mblocks_kernel(const float *__restrict__ O, const double *__restrict__ m, int nrows,
                               double *__restrict__ Mb, int *__restrict__ bad)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nrows) return;
    const float *o = O + (int64_t)I * LOP;
    const double L[3][3] = {{1.0 + o[0], 0.0, 0.0}, {o[3], 1.0 + o[1], 0.0}, {o[4], o[5], 1.0 + o[2]}};
    const double S[3] = {sqrt(m[3 * (int64_t)I]), sqrt(m[3 * (int64_t)I + 1]), sqrt(m[3 * (int64_t)I + 2])};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            // K_ab = sum_k L_ak L_bk in k order, (S_a S_b) K_ab: bitwise symmetric
            double k = 0.0;
            for (int c = 0; c < 3; ++c) k += L[a][c] * L[b][c];
            Mb[(int64_t)I * 9 + a * 3 + b] = (S[a] * S[b]) * k;
        }
    const double det = L[0][0] * L[1][1] * L[2][2];
    if (!(det * det > 0.0)) atomicOr(bad, 1);
}

// ---------------------------------------------------------------- training kernels
// s = r - t, partial sum of s^2 per CTA
__global__ void __launch_bounds__(256) lresid_kernel(const double *__restrict__ r,
                                                     const double *__restrict__ t,
                                                     double *__restrict__ s, int64_t n,
                                                     double *__restrict__ part)
{
    double v = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double si = r[i] - t[i];
        s[i] = si;
        v += si * si;
    }
    __shared__ double red[256];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < (unsigned)w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// partial sums of x . y per CTA
__global__ void __launch_bounds__(256) ldot_kernel(const double *__restrict__ x,
                                                   const double *__restrict__ y, int64_t n,
                                                   double *__restrict__ part)
{
    double v = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v += x[i] * y[i];
    __shared__ double red[256];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < (unsigned)w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// loss += num / den / S ; coef = -2 / (S den)   (one thread)
__global__ void lloss_kernel(const double *ss, const double *rr, double inv_s, double *loss,
                             double *coef)
{
    *loss += (*ss / *rr) * inv_s;
    *coef = -2.0 * inv_s / *rr;
}

// G_I += coef g_I r_I^T
__global__ void lgrad_kernel(const double *__restrict__ g, const double *__restrict__ r,
                             const double *__restrict__ coef, int nrows, double *__restrict__ G)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nrows) return;
    const double c = *coef;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) G[(int64_t)I * 9 + a * 3 + b] += c * g[3 * (int64_t)I + a] * r[3 * (int64_t)I + b];
}

// dL/do from dL/dM: dK = S G S (K = L L^T), dL/dL = (dK + dK^T) L, and each
// output takes the entry of dL/dL at its place in L.
__global__ void ldo_kernel(const double *__restrict__ G, const double *__restrict__ m,
                           const float *__restrict__ O, int nrows, float *__restrict__ dO)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nrows) return;
    double S[3];
    for (int a = 0; a < 3; ++a) S[a] = sqrt(m[3 * (int64_t)I + a]);
    const float *o = O + (int64_t)I * LOP;
    const double L[3][3] = {{1.0 + o[0], 0.0, 0.0}, {o[3], 1.0 + o[1], 0.0}, {o[4], o[5], 1.0 + o[2]}};
    const double *gm = G + (int64_t)I * 9;
    double Gs[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            Gs[a][b] = S[a] * gm[a * 3 + b] * S[b] + S[b] * gm[b * 3 + a] * S[a];
    auto gl = [&](int a, int b) {
        double v = 0.0;
        for (int c = 0; c < 3; ++c) v += Gs[a][c] * L[c][b];
        return v;
    };
    float *d = dO + (int64_t)I * LOP;
    d[0] = (float)gl(0, 0);
    d[1] = (float)gl(1, 1);
    d[2] = (float)gl(2, 2);
    d[3] = (float)gl(1, 0);
    d[4] = (float)gl(2, 0);
    d[5] = (float)gl(2, 1);
    d[6] = d[7] = 0.0f;
}

// Backward through the MLP: per-CTA partial sums of every parameter's
// gradient over a contiguous range of rows (fixed order).
constexpr int BW_T = 256;
constexpr int BW_PER = (LNPARAM + BW_T - 1) / BW_T;

__global__ void __launch_bounds__(BW_T) lbackward_kernel(int nrows, const __nv_bfloat16 *__restrict__ X,
                                                         const float *__restrict__ H,
                                                         const float *__restrict__ dO,
                                                         const __nv_bfloat16 *__restrict__ W2,
                                                         float *__restrict__ part)
{
    __shared__ float sx[LFP], sh[LH], sdo[LOP], sdh[LH];
    float acc[BW_PER];
#pragma unroll
    for (int q = 0; q < BW_PER; ++q) acc[q] = 0.0f;
    const int per = (nrows + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * per, i1 = min(nrows, i0 + per);
    const int tid = threadIdx.x;
    for (int I = i0; I < i1; ++I) {
        if (tid < LFP) sx[tid] = __bfloat162float(X[(int64_t)I * LFP + tid]);
        if (tid < LH) sh[tid] = H[(int64_t)I * LH + tid];
        if (tid < LOP) sdo[tid] = dO[(int64_t)I * LOP + tid];
        __syncthreads();
        if (tid < LH) {
            float v = 0.0f;
            for (int j = 0; j < LO; ++j) v += __bfloat162float(W2[j * LH + tid]) * sdo[j];
            sdh[tid] = sh[tid] > 0.0f ? v : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < BW_PER; ++q) {
            const int p = tid + q * BW_T;
            if (p >= LNPARAM) continue;
            float c;
            if (p < LH * LF) c = sdh[p / LF] * sx[p % LF];
            else if (p < LH * LF + LH) c = sdh[p - LH * LF];
            else if (p < LH * LF + LH + LO * LH) {
                const int q2 = p - LH * LF - LH;
                c = sdo[q2 / LH] * sh[q2 % LH];
            } else c = sdo[p - (LH * LF + LH + LO * LH)];
            acc[q] += c;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < BW_PER; ++q) {
        const int p = tid + q * BW_T;
        if (p < LNPARAM) part[(int64_t)blockIdx.x * LNPARAM + p] = acc[q];
    }
}

// grad[p] += sum over CTAs (fixed order) of the partials
__global__ void lreduce_kernel(const float *__restrict__ part, int nparts, float *__restrict__ grad)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= LNPARAM) return;
    float s = 0.0f;
    for (int c = 0; c < nparts; ++c) s += part[(int64_t)c * LNPARAM + p];
    grad[p] += s;
}

// BF16 / FP32 working copies of the flat FP32 parameters (W1 b1 W2 b2).
__global__ void lpack_kernel(const float *__restrict__ w, __nv_bfloat16 *__restrict__ W1,
                             float *__restrict__ b1, __nv_bfloat16 *__restrict__ W2,
                             float *__restrict__ b2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < LH * LFP) {
        const int k = i / LFP, f = i % LFP;
        W1[i] = __float2bfloat16(f < LF ? w[k * LF + f] : 0.0f);
    }
    if (i < LH) b1[i] = w[LH * LF + i];
    if (i < LOP * LH) {
        const int j = i / LH, k = i % LH;
        W2[i] = __float2bfloat16(j < LO ? w[LH * LF + LH + j * LH + k] : 0.0f);
    }
    if (i < LOP) b2[i] = i < LO ? w[LH * LF + LH + LO * LH + i] : 0.0f;
}

// Adam on the flat FP32 parameters; the gradient is averaged over `count`.
__global__ void ladam_kernel(float *__restrict__ w, const float *__restrict__ grad,
                             float *__restrict__ m1, float *__restrict__ m2, float lr, float b1,
                             float b2, float eps, int step, float count)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= LNPARAM) return;
    const float g = grad[p] / count;
    m1[p] = b1 * m1[p] + (1.0f - b1) * g;
    m2[p] = b2 * m2[p] + (1.0f - b2) * g * g;
    const float mh = m1[p] / (1.0f - powf(b1, (float)step));
    const float vh = m2[p] / (1.0f - powf(b2, (float)step));
    w[p] -= lr * mh / (sqrtf(vh) + eps);
}

// counter-based uniform(-1, 1) (SplitMix64 of seed + index)
__global__ void lrandom_kernel(double *__restrict__ x, int64_t n, unsigned long long seed)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long z = seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)(i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        x[i] = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
    }
}

// the network's working copies on the device
struct Net {
    __nv_bfloat16 *W1 = nullptr, *W2 = nullptr;
    float *b1 = nullptr, *b2 = nullptr, *w = nullptr;
    MlpDev dev() const { return MlpDev{W1, b1, W2, b2}; }
};

static int net_alloc(DevArena &mem, Net *n)
{
    AMG_TRY(mem.alloc_n(&n->W1, LH * LFP));
    AMG_TRY(mem.alloc_n(&n->W2, LOP * LH));
    AMG_TRY(mem.alloc_n(&n->b1, LH));
    AMG_TRY(mem.alloc_n(&n->b2, LOP));
    AMG_TRY(mem.alloc_n(&n->w, LNPARAM));
    return AMG_OK;
}

static int net_pack(const Net &n, cudaStream_t s)
{
    lpack_kernel<<<(LH * LFP + 255) / 256, 256, 0, s>>>(n.w, n.W1, n.b1, n.W2, n.b2);
    count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    return AMG_OK;
}

// features + forward + blocks for the fine level of a hierarchy
static int learned_blocks(amg_handle h, const Net &net, DevArena &tmp, double *Mb, int *bad_dev,
                          float **O_out, float **H_out, __nv_bfloat16 **X_out, cudaStream_t s)
{
    const Level &L0 = h->lv[0];
    const int n = L0.A.nbr, ntiles = (n + 15) / 16;
    __nv_bfloat16 *X = X_out && *X_out ? *X_out : nullptr;
    if (!X) {
        AMG_TRY(tmp.alloc_n(&X, (size_t)ntiles * 16 * LFP));
        AMG_TRY_CUDA(cudaMemsetAsync(X, 0, sizeof(__nv_bfloat16) * ntiles * 16 * LFP, s));
        features_kernel<<<(n + 255) / 256, 256, 0, s>>>(L0.A.row_ptr, L0.A.col, L0.A.val, n, X);
        count_launch(1);
    }
    float *O = O_out && *O_out ? *O_out : nullptr;
    if (!O) AMG_TRY(tmp.alloc_n(&O, (size_t)n * LOP));
    float *Hh = H_out ? *H_out : nullptr;
    const int grid = std::min((ntiles + 7) / 8, h->geom.num_sms * 8);
    mlp_forward_kernel<<<std::max(grid, 1), 256, 0, s>>>(X, n, ntiles, net.dev(), O, Hh);
    mblocks_kernel<<<(n + 255) / 256, 256, 0, s>>>(O, L0.M, n, Mb, bad_dev);
    count_launch(2);
    AMG_TRY_CUDA(cudaGetLastError());
    if (X_out) *X_out = X;
    if (O_out) *O_out = O;
    return AMG_OK;
}

__global__ void lscale_kernel(double *__restrict__ x, int64_t n, const double *__restrict__ nrm2)
{
    const double inv = 1.0 / sqrt(*nrm2);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] *= inv;
}

// lambda_max(Mb A) on level 0 by 20 power iterations from a fixed random
// vector (Mb A is similar to the symmetric Mb^1/2 A Mb^1/2, real spectrum).
// The smoothing iteration u += M (f - A u) contracts the energy norm only if
// this is below 2.
static int smoother_lambda_max(amg_handle h, const double *Mb, DevArena &tmp, cudaStream_t s,
                               double *out)
{
    const Level &L0 = h->lv[0];
    const int64_t n = L0.n();
    const int grid = std::min((int)((n + 255) / 256), h->geom.max_ctas);
    double *x = nullptr, *y = nullptr, *zero = nullptr, *sc = nullptr, *part = nullptr;
    AMG_TRY(tmp.alloc_n(&x, (size_t)n));
    AMG_TRY(tmp.alloc_n(&y, (size_t)n));
    AMG_TRY(tmp.alloc_n(&zero, (size_t)n));
    AMG_TRY(tmp.alloc_n(&sc, 2));
    AMG_TRY(tmp.alloc_n(&part, (size_t)h->geom.max_ctas + 1));
    AMG_TRY_CUDA(cudaMemsetAsync(zero, 0, sizeof(double) * n, s));
    lrandom_kernel<<<grid, 256, 0, s>>>(x, n, 0x5eedULL);
    count_launch(1);
    auto norm2 = [&](const double *v, double *dst) -> int {
        lresid_kernel<<<grid, 256, 0, s>>>(v, zero, y, n, part);  // y = v, partial |v|^2
        count_launch(1);
        return launch_reduce_sum(part, grid, dst, s);
    };
    AMG_TRY(norm2(x, sc));
    lscale_kernel<<<grid, 256, 0, s>>>(x, n, sc);
    count_launch(1);
    for (int k = 0; k < 20; ++k) {
        SellArgs<double> a{};
        a.x = x;
        a.y = y;
        AMG_TRY((launch_sell<double, double>(L0.sA, SPMV_PLAIN, DOT_NONE, a, h->geom, s)));
        AMG_TRY(launch_block_apply(Mb, y, x, L0.A.nbr, h->geom, s));  // x = M A x
        AMG_TRY(norm2(x, sc));
        lscale_kernel<<<grid, 256, 0, s>>>(x, n, sc);
        count_launch(1);
    }
    AMG_TRY_CUDA(cudaGetLastError());
    double nrm2 = 0.0;
    AMG_TRY_CUDA(cudaMemcpyAsync(&nrm2, sc, sizeof(double), cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    *out = std::sqrt(nrm2);  // |M A x_19| for the unit vector x_19
    return AMG_OK;
}

}  // namespace amg

using namespace amg;

// ---------------------------------------------------------------- trainer
struct LProblem {
    amg_handle h;
    int n = 0, nrows = 0, ntiles = 0, S = 0;
    __nv_bfloat16 *X = nullptr;
    float *O = nullptr, *H = nullptr, *dO = nullptr;
    double *E = nullptr;   // error samples [S][n]
    double *R = nullptr;   // A E
    double *rr = nullptr;  // e . A e per sample
    double *Mb = nullptr, *G = nullptr;
    double *v = nullptr, *t = nullptr, *sv = nullptr, *g = nullptr;
};

struct amg_trainer_s {
    DevArena mem;
    Net net;
    float *m1 = nullptr, *m2 = nullptr, *grad = nullptr, *part = nullptr;
    double *loss = nullptr, *coef = nullptr, *scal = nullptr, *dpart = nullptr;
    int *bad = nullptr;
    int nparts = 0, step = 0;
    double lr = 1e-3;
    Geom geom;
    std::vector<LProblem> probs;
};

static int trainer_eval(amg_trainer t, cudaStream_t s)
{
    AMG_TRY_CUDA(cudaMemsetAsync(t->grad, 0, sizeof(float) * LNPARAM, s));
    AMG_TRY_CUDA(cudaMemsetAsync(t->loss, 0, sizeof(double), s));
    for (LProblem &P : t->probs) {
        const Level &L0 = P.h->lv[0];
        AMG_TRY(learned_blocks(P.h, t->net, t->mem, P.Mb, t->bad, &P.O, &P.H, &P.X, s));
        AMG_TRY_CUDA(cudaMemsetAsync(P.G, 0, sizeof(double) * (size_t)P.nrows * 9, s));
        for (int k = 0; k < P.S; ++k) {
            const double *r = P.R + (int64_t)k * P.n;
            const double *e = P.E + (int64_t)k * P.n;
            const int grid = std::min((P.n + 255) / 256, t->geom.max_ctas);
            AMG_TRY(launch_block_apply(P.Mb, r, P.v, P.nrows, t->geom, s));  // v = M A e
            lresid_kernel<<<grid, 256, 0, s>>>(e, P.v, P.sv, P.n, t->dpart);   // e' = e - v
            count_launch(1);
            SellArgs<double> a{};
            a.x = P.sv;
            a.y = P.g;
            AMG_TRY((launch_sell<double, double>(L0.sA, SPMV_PLAIN, DOT_NONE, a, t->geom, s)));
            ldot_kernel<<<grid, 256, 0, s>>>(P.sv, P.g, P.n, t->dpart);        // e' . A e'
            count_launch(1);
            AMG_TRY(launch_reduce_sum(t->dpart, grid, t->scal, s));
            lloss_kernel<<<1, 1, 0, s>>>(t->scal, P.rr + k, 1.0 / P.S, t->loss, t->coef);
            lgrad_kernel<<<(P.nrows + 255) / 256, 256, 0, s>>>(P.g, r, t->coef, P.nrows, P.G);
            count_launch(2);
            AMG_TRY_CUDA(cudaGetLastError());
        }
        ldo_kernel<<<(P.nrows + 255) / 256, 256, 0, s>>>(P.G, L0.M, P.O, P.nrows, P.dO);
        lbackward_kernel<<<t->nparts, BW_T, 0, s>>>(P.nrows, P.X, P.H, P.dO, t->net.W2, t->part);
        lreduce_kernel<<<(LNPARAM + 255) / 256, 256, 0, s>>>(t->part, t->nparts, t->grad);
        count_launch(3);
        AMG_TRY_CUDA(cudaGetLastError());
    }
    return AMG_OK;
}

extern "C" {

int amg_trainer_create(const float *params, double lr, void *stream, amg_trainer *out)
{
    clear_error();
    if (!params || !out || !(lr > 0.0)) {
        set_error("amg_trainer_create: bad argument");
        return AMG_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    amg_trainer t = new amg_trainer_s();
    t->mem.stream = s;
    t->lr = lr;
    int st = query_geom(&t->geom);
    t->nparts = t->geom.num_sms * 2;
    if (st >= 0) st = net_alloc(t->mem, &t->net);
    if (st >= 0) st = t->mem.alloc_n(&t->m1, LNPARAM);
    if (st >= 0) st = t->mem.alloc_n(&t->m2, LNPARAM);
    if (st >= 0) st = t->mem.alloc_n(&t->grad, LNPARAM);
    if (st >= 0) st = t->mem.alloc_n(&t->part, (size_t)t->nparts * LNPARAM);
    if (st >= 0) st = t->mem.alloc_n(&t->loss, 1);
    if (st >= 0) st = t->mem.alloc_n(&t->coef, 1);
    if (st >= 0) st = t->mem.alloc_n(&t->scal, 1);
    if (st >= 0) st = t->mem.alloc_n(&t->dpart, (size_t)t->geom.max_ctas + 1);
    if (st >= 0) st = t->mem.alloc_n(&t->bad, 1);
    if (st < 0) {
        t->mem.release_all();
        delete t;
        return st;
    }
    cudaMemcpyAsync(t->net.w, params, sizeof(float) * LNPARAM, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(t->m1, 0, sizeof(float) * LNPARAM, s);
    cudaMemsetAsync(t->m2, 0, sizeof(float) * LNPARAM, s);
    st = net_pack(t->net, s);
    if (st >= 0 && cudaStreamSynchronize(s) != cudaSuccess) st = AMG_ERR_CUDA;
    if (st < 0) {
        t->mem.release_all();
        delete t;
        return st;
    }
    *out = t;
    return AMG_OK;
}

void amg_trainer_free(amg_trainer t)
{
    if (!t) return;
    t->mem.release_all();
    cudaStreamSynchronize(t->mem.stream);
    delete t;
}

static int add_problem(amg_trainer t, amg_handle h, int S, cudaStream_t s, LProblem **out)
{
    if (!t || !h || S < 1 || h->lv.size() < 2 || h->prm.precision != AMG_PREC_FP64 ||
        h->lv[0].A.br != 3) {
        set_error("amg_trainer: needs a multi-level FP64 hierarchy and at least one sample");
        return AMG_ERR_ARG;
    }
    LProblem P;
    P.h = h;
    P.n = h->lv[0].n();
    P.nrows = h->lv[0].A.nbr;
    P.ntiles = (P.nrows + 15) / 16;
    P.S = S;
    DevArena &m = t->mem;
    m.stream = s;
    AMG_TRY(m.alloc_n(&P.E, (size_t)S * P.n));
    AMG_TRY(m.alloc_n(&P.R, (size_t)S * P.n));
    AMG_TRY(m.alloc_n(&P.rr, (size_t)S));
    AMG_TRY(m.alloc_n(&P.Mb, (size_t)P.nrows * 9));
    AMG_TRY(m.alloc_n(&P.G, (size_t)P.nrows * 9));
    AMG_TRY(m.alloc_n(&P.H, (size_t)P.ntiles * 16 * LH));
    AMG_TRY(m.alloc_n(&P.dO, (size_t)P.nrows * LOP));
    for (double **pp : {&P.v, &P.t, &P.sv, &P.g}) AMG_TRY(m.alloc_n(pp, (size_t)P.n));
    t->probs.push_back(P);
    *out = &t->probs.back();
    return AMG_OK;
}

static int finish_problem(amg_trainer t, LProblem *P, cudaStream_t s)
{
    // R = A E and the energy norms e . A e
    const Level &L0 = P->h->lv[0];
    for (int k = 0; k < P->S; ++k) {
        const int grid = std::min((P->n + 255) / 256, t->geom.max_ctas);
        const double *e = P->E + (int64_t)k * P->n;
        double *r = P->R + (int64_t)k * P->n;
        SellArgs<double> a{};
        a.x = e;
        a.y = r;
        AMG_TRY((launch_sell<double, double>(L0.sA, SPMV_PLAIN, DOT_NONE, a, t->geom, s)));
        ldot_kernel<<<grid, 256, 0, s>>>(e, r, P->n, t->dpart);
        count_launch(1);
        AMG_TRY(launch_reduce_sum(t->dpart, grid, P->rr + k, s));
    }
    AMG_TRY_CUDA(cudaGetLastError());
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    return AMG_OK;
}

int amg_trainer_add_samples(amg_trainer t, amg_handle h, const double *R, int32_t nsamples,
                            void *stream)
{
    clear_error();
    cudaStream_t s = (cudaStream_t)stream;
    if (!R) {
        set_error("null samples");
        return AMG_ERR_ARG;
    }
    LProblem *P = nullptr;
    AMG_TRY(add_problem(t, h, nsamples, s, &P));
    AMG_TRY_CUDA(cudaMemcpyAsync(P->E, R, sizeof(double) * (size_t)nsamples * P->n,
                                 cudaMemcpyDeviceToDevice, s));
    return finish_problem(t, P, s);
}

int amg_trainer_add_generated(amg_trainer t, amg_handle h, int32_t nsamples, uint64_t seed,
                              void *stream)
{
    clear_error();
    cudaStream_t s = (cudaStream_t)stream;
    if (h && h->learned) {
        set_error("samples come from the SPAI0 V-cycle: use a hierarchy without learned blocks");
        return AMG_ERR_ARG;
    }
    LProblem *P = nullptr;
    AMG_TRY(add_problem(t, h, nsamples, s, &P));
    const Level &L0 = h->lv[0];
    for (int k = 0; k < nsamples; ++k) {
        // e0 random; even samples: e = (I - V A) e0, the error one V-cycle
        // leaves; odd samples: e = e0 (white noise carries the top of the
        // spectrum, which a smoother must not amplify)
        double *e = P->E + (int64_t)k * P->n;
        const int grid = std::min((P->n + 255) / 256, t->geom.max_ctas);
        lrandom_kernel<<<grid, 256, 0, s>>>(e, P->n,
                                            (unsigned long long)seed * 1000003ULL + (unsigned long long)k);
        count_launch(1);
        if (k % 2 == 0) {
            SellArgs<double> a{};
            a.x = e;
            a.y = P->v;
            AMG_TRY((launch_sell<double, double>(L0.sA, SPMV_PLAIN, DOT_NONE, a, t->geom, s)));
            AMG_TRY(amg_apply_vcycle(h, P->v, P->g, stream));            // g = V A e0
            lresid_kernel<<<grid, 256, 0, s>>>(e, P->g, P->sv, P->n, t->dpart);
            count_launch(1);
            AMG_TRY_CUDA(cudaMemcpyAsync(e, P->sv, sizeof(double) * P->n, cudaMemcpyDeviceToDevice, s));
        }
    }
    return finish_problem(t, P, s);
}

int amg_trainer_eval(amg_trainer t, double *loss, float *grad, void *stream)
{
    clear_error();
    if (!t || t->probs.empty()) {
        set_error("trainer has no problems");
        return AMG_ERR_STATE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    AMG_TRY(trainer_eval(t, s));
    double l = 0.0;
    std::vector<float> gh(LNPARAM);
    AMG_TRY_CUDA(cudaMemcpyAsync(&l, t->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaMemcpyAsync(gh.data(), t->grad, sizeof(float) * LNPARAM, cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    const double np = (double)t->probs.size();
    if (loss) *loss = l / np;
    if (grad)
        for (int p = 0; p < LNPARAM; ++p) grad[p] = (float)(gh[p] / np);
    return AMG_OK;
}

int amg_trainer_step(amg_trainer t, int32_t nsteps, double *loss, void *stream)
{
    clear_error();
    if (!t || t->probs.empty() || nsteps < 1) {
        set_error("trainer has no problems or bad step count");
        return AMG_ERR_STATE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < nsteps; ++k) {
        AMG_TRY(trainer_eval(t, s));
        ++t->step;
        ladam_kernel<<<(LNPARAM + 255) / 256, 256, 0, s>>>(t->net.w, t->grad, t->m1, t->m2,
                                                           (float)t->lr, 0.9f, 0.999f, 1e-8f,
                                                           t->step, (float)t->probs.size());
        count_launch(1);
        AMG_TRY(net_pack(t->net, s));
    }
    double l = 0.0;
    AMG_TRY_CUDA(cudaMemcpyAsync(&l, t->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    if (loss) *loss = l / (double)t->probs.size();
    return AMG_OK;
}

int amg_trainer_params(amg_trainer t, float *out)
{
    if (!t || !out) return AMG_ERR_ARG;
    AMG_TRY_CUDA(cudaMemcpy(out, t->net.w, sizeof(float) * LNPARAM, cudaMemcpyDeviceToHost));
    return AMG_OK;
}

int amg_set_learned_smoother(amg_handle h, const float *params, int32_t *fell_back, void *stream)
{
    clear_error();
    if (!h || !params) {
        set_error("null argument");
        return AMG_ERR_ARG;
    }
    AllocScope scope(h->allocator());
    cudaStream_t s = (cudaStream_t)stream;
    if (h->lv.size() < 2 || h->lv[0].A.br != 3 || h->prm.storage != AMG_STORAGE_BLOCK) {
        set_error("the learned smoother needs a multi-level hierarchy in block storage");
        return AMG_ERR_ARG;
    }
    if (h->ilu || h->prm.smoother != AMG_SMOOTH_SPAI0) {
        set_error("the hierarchy smooths with ILU(0) or block Jacobi; the learned smoother "
                  "replaces SPAI0 only");
        return AMG_ERR_STATE;
    }
    DevArena tmp;
    tmp.stream = s;
    Net net;
    int *bad = nullptr;
    int st = net_alloc(tmp, &net);
    if (st >= 0) st = tmp.alloc_n(&bad, 1);
    Level &L0 = h->lv[0];
    if (st >= 0 && !L0.Mb) st = h->mem.alloc_n(&L0.Mb, (size_t)L0.A.nbr * 9);
    if (st >= 0 && cudaMemcpyAsync(net.w, params, sizeof(float) * LNPARAM, cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = AMG_ERR_CUDA;
    if (st >= 0 && cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess) st = AMG_ERR_CUDA;
    if (st >= 0) st = net_pack(net, s);
    if (st >= 0) st = learned_blocks(h, net, tmp, L0.Mb, bad, nullptr, nullptr, nullptr, s);
    int hb = 1;
    if (st >= 0 && (cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess))
        st = AMG_ERR_CUDA;
    double lam = 0.0;
    if (st >= 0 && !hb) st = smoother_lambda_max(h, L0.Mb, tmp, s, &lam);
    if (st >= 0 && !hb && h->spai0_lambda == 0.0) {
        // the same estimate for SPAI0: blocks from a zero network output
        float *O0 = nullptr;
        double *M0 = nullptr;
        st = tmp.alloc_n(&O0, (size_t)L0.A.nbr * LOP);
        if (st >= 0) st = tmp.alloc_n(&M0, (size_t)L0.A.nbr * 9);
        if (st >= 0 && cudaMemsetAsync(O0, 0, sizeof(float) * L0.A.nbr * LOP, s) != cudaSuccess)
            st = AMG_ERR_CUDA;
        if (st >= 0) {
            mblocks_kernel<<<(L0.A.nbr + 255) / 256, 256, 0, s>>>(O0, L0.M, (int)L0.A.nbr, M0, bad);
            count_launch(1);
            if (cudaGetLastError() != cudaSuccess) st = AMG_ERR_CUDA;
        }
        double lam0 = 0.0;
        if (st >= 0) st = smoother_lambda_max(h, M0, tmp, s, &lam0);
        if (st >= 0) h->spai0_lambda = lam0;
    }
    tmp.release_all();
    cudaStreamSynchronize(s);
    if (st < 0) return st;
    // back to SPAI0 when a block is singular (1) or when the learned smoother
    // is less stable than both the bound 1.9 and SPAI0 itself (2): the
    // smoothing step contracts the energy norm only while lambda_max(M A) < 2
    const int fb = hb ? 1 : (lam >= std::max(1.9, h->spai0_lambda) ? 2 : 0);
    if (!fb && (h->prm.precision == AMG_PREC_FP32 || h->prm.precision == AMG_PREC_BF16)) {
        // the FP32 / BF16 V-cycles apply the blocks in FP32
        if (!L0.Mbf) AMG_TRY(h->mem.alloc_n(&L0.Mbf, (size_t)L0.A.nbr * 9));
        const int64_t n9 = (int64_t)L0.A.nbr * 9;
        narrow9_kernel<<<(int)std::min<int64_t>((n9 + 255) / 256, h->geom.max_ctas), 256, 0, s>>>(
            L0.Mb, L0.Mbf, n9);
        count_launch(1);
        AMG_TRY_CUDA(cudaGetLastError());
        AMG_TRY_CUDA(cudaStreamSynchronize(s));
    }
    h->learned = fb ? 0 : 1;
    h->learned_lambda = lam;
    if (fell_back) *fell_back = fb;
    if (h->exec) {  // the recorded iteration changes
        cudaGraphExecDestroy(h->exec);
        cudaGraphDestroy(h->graph);
        h->exec = nullptr;
        h->graph = nullptr;
    }
    return AMG_OK;
}

int amg_clear_learned_smoother(amg_handle h)
{
    if (!h) return AMG_ERR_ARG;
    h->learned = 0;
    if (h->exec) {
        cudaGraphExecDestroy(h->exec);
        cudaGraphDestroy(h->graph);
        h->exec = nullptr;
        h->graph = nullptr;
    }
    return AMG_OK;
}

}  // extern "C"
