// Block ILU(0) smoother: the relaxation of the paper's experiments (Sec. 4
// runs CG + SA-AMG with ILU(0) smoothing), in b x b block arithmetic on each
// level's own block pattern.
//
// Factorisation.  Row I of the factor is, in order over its blocks K < I:
// L_IK = A_IK U_KK^-1, then A_IJ -= L_IK U_KJ for every later block J of row
// I that row K's upper part also holds; what remains on and above the
// diagonal is U, and U_II is inverted (Gauss-Jordan without pivoting; an
// exactly zero row of the block -- a coarse DOF whose near-nullspace column
// was dropped -- gets a unit pivot and a zero row and column in the inverse).
// Row I depends on the rows K < I it holds, so the rows are grouped into
// dependency levels (level(I) = 1 + the largest level of those K, from the
// pattern alone, on the host) and each level is one launch with a warp per
// row: the K loop runs in order, the updates of one K spread over the lanes.
//
// Application.  ILU^-1 r is approximated by a fixed number of Jacobi sweeps
// per triangular factor, the data-parallel form of the substitutions:
//   y <- r - L_s y from y = r (L_s = the strict lower part, unit diagonal),
//   x <- U_D^-1 (y - U_s x) from x = U_D^-1 y (U_s = the strict upper part),
// each sweep one sliced SpMV in residual form (the V-cycle's kernel) plus,
// for U, a block-diagonal product with the inverses.
#include <algorithm>
#include <climits>
#include <vector>

#include "amg_internal.cuh"

namespace amg {

namespace {

constexpr int FT = 256;  // factor / split kernels: 8 rows (warps) per CTA

// Gauss-Jordan inverse of a B x B block without pivoting; false on a zero or
// non-finite pivot.
template <int B> __device__ bool block_inverse(const double *a, double *inv)
{
    double m[B][2 * B];
    bool zero[B];
#pragma unroll
    for (int r = 0; r < B; ++r) {
        zero[r] = true;
#pragma unroll
        for (int c = 0; c < B; ++c) zero[r] = zero[r] && a[r * B + c] == 0.0;
    }
#pragma unroll
    for (int r = 0; r < B; ++r)
#pragma unroll
        for (int c = 0; c < 2 * B; ++c)
            m[r][c] = c < B ? (zero[r] ? (c == r ? 1.0 : 0.0) : a[r * B + c])
                            : (c - B == r ? 1.0 : 0.0);
#pragma unroll
    for (int p = 0; p < B; ++p) {
        const double piv = m[p][p];
        if (!(fabs(piv) > 0.0) || !isfinite(piv)) return false;
#pragma unroll
        for (int c = 0; c < 2 * B; ++c) m[p][c] /= piv;
#pragma unroll
        for (int r = 0; r < B; ++r) {
            if (r == p) continue;
            const double f = m[r][p];
#pragma unroll
            for (int c = 0; c < 2 * B; ++c) m[r][c] -= f * m[p][c];
        }
    }
#pragma unroll
    for (int r = 0; r < B; ++r)
#pragma unroll
        for (int c = 0; c < B; ++c) inv[r * B + c] = (zero[r] || zero[c]) ? 0.0 : m[r][B + c];
    return true;
}

// One dependency level of the factorisation: rows[0..nrows) are independent
// of each other and every row they depend on is final.  One CTA of W warps
// per row, so that the few rows of a deep level spread over the SMs and a
// long row's updates over W * 32 threads.  F holds A's values on entry and
// the factor on exit; *status receives the lowest row whose diagonal block
// could not be inverted.
template <int B, int W>
__global__ void __launch_bounds__(W * 32) ilu_factor_rows_kernel(const int *__restrict__ rp,
                                                                 const int *__restrict__ col,
                                                                 const int *__restrict__ diag,
                                                                 double *__restrict__ F,
                                                                 double *__restrict__ Dinv,
                                                                 const int *__restrict__ rows,
                                                                 int *__restrict__ status)
{
    constexpr int BB = B * B, NT = W * 32;
    static_assert(BB <= NT + 32, "L_IK is computed by at most two entries per thread");
    __shared__ double lsh[BB];  // L_IK of the current K
    const int tid = threadIdx.x;
    const int I = rows[blockIdx.x];
    const int e0 = rp[I + 1], dI = diag[I];
    for (int pk = rp[I]; pk < dI; ++pk) {
        const int K = col[pk];
        double *lik = F + (int64_t)pk * BB;
        const double *dk = Dinv + (int64_t)K * BB;
        double l0 = 0.0, l1 = 0.0;  // entries tid and tid + NT of L_IK = A_IK U_KK^-1
        if (tid < BB) {
            const int r = tid / B, c = tid % B;
#pragma unroll
            for (int k = 0; k < B; ++k) l0 += lik[r * B + k] * dk[k * B + c];
        }
        if (tid + NT < BB) {
            const int r = (tid + NT) / B, c = (tid + NT) % B;
#pragma unroll
            for (int k = 0; k < B; ++k) l1 += lik[r * B + k] * dk[k * B + c];
        }
        __syncthreads();
        if (tid < BB) {
            lik[tid] = l0;
            lsh[tid] = l0;
        }
        if (tid + NT < BB) {
            lik[tid + NT] = l1;
            lsh[tid + NT] = l1;
        }
        __syncthreads();
        // A_IJ -= L_IK U_KJ for the later blocks J of row I that row K's
        // upper part holds; U_KJ is final, read into registers before any
        // store to row I
        const int kb = diag[K] + 1, ke = rp[K + 1];
        for (int pj = pk + 1 + tid; pj < e0; pj += NT) {
            const int J = col[pj];
            int lo = kb, hi = ke;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (col[mid] < J) lo = mid + 1;
                else hi = mid;
            }
            if (lo < ke && col[lo] == J) {
                double u[BB];
                const double *ukj = F + (int64_t)lo * BB;
#pragma unroll
                for (int e = 0; e < BB; ++e) u[e] = ukj[e];
                double *aij = F + (int64_t)pj * BB;
#pragma unroll
                for (int r = 0; r < B; ++r) {
                    double lr[B];
#pragma unroll
                    for (int k = 0; k < B; ++k) lr[k] = lsh[r * B + k];
#pragma unroll
                    for (int c = 0; c < B; ++c) {
                        double v = 0.0;
#pragma unroll
                        for (int k = 0; k < B; ++k) v += lr[k] * u[k * B + c];
                        aij[r * B + c] -= v;
                    }
                }
            }
        }
        __syncthreads();
    }
    if (tid == 0 && !block_inverse<B>(F + (int64_t)dI * BB, Dinv + (int64_t)I * BB))
        atomicMin(status, I);
}

// Strict lower and strict upper parts of the factor as their own BSR
// matrices (row pointers built on the host); one warp per row.
template <int B>
__global__ void __launch_bounds__(FT) ilu_split_kernel(const int *__restrict__ rp,
                                                       const int *__restrict__ col,
                                                       const int *__restrict__ diag,
                                                       const double *__restrict__ F, int nbr,
                                                       const int *__restrict__ lrp,
                                                       int *__restrict__ lcol,
                                                       double *__restrict__ lval,
                                                       const int *__restrict__ urp,
                                                       int *__restrict__ ucol,
                                                       double *__restrict__ uval)
{
    constexpr int BB = B * B;
    const int lane = threadIdx.x & 31;
    const int I = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (I >= nbr) return;
    const int b0 = rp[I], d = diag[I], e0 = rp[I + 1];
    const int nl = d - b0, nu = e0 - d - 1;
    for (int k = lane; k < nl; k += 32) lcol[lrp[I] + k] = col[b0 + k];
    for (int k = lane; k < nu; k += 32) ucol[urp[I] + k] = col[d + 1 + k];
    for (int64_t k = lane; k < (int64_t)nl * BB; k += 32)
        lval[(int64_t)lrp[I] * BB + k] = F[(int64_t)b0 * BB + k];
    for (int64_t k = lane; k < (int64_t)nu * BB; k += 32)
        uval[(int64_t)urp[I] * BB + k] = F[(int64_t)(d + 1) * BB + k];
}

// y = D x with D block diagonal (B x B blocks, row-major), one thread per row.
template <int B>
__global__ void block_diag_apply_kernel(const double *__restrict__ D, const double *__restrict__ x,
                                        double *__restrict__ y, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t I = i / B;
    const int r = (int)(i % B);
    const double *d = D + I * B * B + r * B;
    const double *xi = x + I * B;
    double v = 0.0;
#pragma unroll
    for (int c = 0; c < B; ++c) v += d[c] * xi[c];
    y[i] = v;
}

__global__ void vec_add_kernel(const double *__restrict__ a, const double *__restrict__ b,
                               double *__restrict__ y, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a[i] + b[i];
}

int block_diag_apply(int b, const double *D, const double *x, double *y, int64_t n, cudaStream_t s)
{
    if (n == 0) return AMG_OK;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (b == 3) block_diag_apply_kernel<3><<<grid, 256, 0, s>>>(D, x, y, n);
    else if (b == 6) block_diag_apply_kernel<6><<<grid, 256, 0, s>>>(D, x, y, n);
    else {
        set_error("ILU(0): block size %d not supported", b);
        return AMG_ERR_ARG;
    }
    count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    return AMG_OK;
}

}  // namespace

int launch_vec_add(const double *a, const double *b, double *y, int64_t n, cudaStream_t s)
{
    if (n == 0) return AMG_OK;
    vec_add_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, b, y, n);
    count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    return AMG_OK;
}

int ilu0_factor(const BsrD &A, int max_lanes, DevArena &keep, DevArena &tmp, cudaStream_t s,
                Ilu *out)
{
    const int nbr = A.nbr, b = A.br;
    if (A.nbc != nbr || A.bc != b || (b != 3 && b != 6)) {
        set_error("ILU(0) needs a square matrix of 3x3 or 6x6 blocks");
        return AMG_ERR_ARG;
    }
    const int64_t bb = (int64_t)b * b;
    // pattern on the host: diagonal positions and dependency levels
    std::vector<int> rp(nbr + 1), cl(std::max<int64_t>(A.nnzb, 1));
    AMG_TRY_CUDA(cudaMemcpyAsync(rp.data(), A.row_ptr, sizeof(int) * (nbr + 1),
                                 cudaMemcpyDeviceToHost, s));
    if (A.nnzb > 0)
        AMG_TRY_CUDA(cudaMemcpyAsync(cl.data(), A.col, sizeof(int) * A.nnzb,
                                     cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    std::vector<int> diag(std::max(nbr, 1)), lev(std::max(nbr, 1), 0);
    int depth = 0;
    for (int I = 0; I < nbr; ++I) {
        int d = -1, lv = 0;
        for (int p = rp[I]; p < rp[I + 1]; ++p) {
            const int K = cl[p];
            if (K < I) lv = std::max(lv, lev[K] + 1);
            else if (K == I) d = p;
        }
        if (d < 0) {
            set_error("ILU(0): block row %d has no diagonal block", I);
            return AMG_ERR_ARG;
        }
        diag[I] = d;
        lev[I] = lv;
        depth = std::max(depth, lv + 1);
    }
    std::vector<int> lptr(depth + 1, 0), order(std::max(nbr, 1));
    for (int I = 0; I < nbr; ++I) lptr[lev[I] + 1]++;
    for (int k = 0; k < depth; ++k) lptr[k + 1] += lptr[k];
    {
        std::vector<int> fill(lptr.begin(), lptr.end() - 1);
        for (int I = 0; I < nbr; ++I) order[fill[lev[I]]++] = I;
    }
    std::vector<int> lrp(nbr + 1, 0), urp(nbr + 1, 0);
    for (int I = 0; I < nbr; ++I) {
        lrp[I + 1] = lrp[I] + (diag[I] - rp[I]);
        urp[I + 1] = urp[I] + (rp[I + 1] - diag[I] - 1);
    }
    out->depth = depth;
    out->b = b;
    out->nbr = nbr;
    AMG_TRY(keep.alloc_n(&out->F, (size_t)std::max<int64_t>(A.nnzb, 1) * bb));
    AMG_TRY(keep.alloc_n(&out->Dinv, (size_t)std::max(nbr, 1) * bb));
    AMG_TRY(keep.alloc_n(&out->y0, (size_t)std::max(nbr, 1) * b));
    AMG_TRY(keep.alloc_n(&out->y1, (size_t)std::max(nbr, 1) * b));
    int *d_diag = nullptr, *d_order = nullptr, *d_status = nullptr;
    AMG_TRY(tmp.alloc_n(&d_diag, (size_t)std::max(nbr, 1)));
    AMG_TRY(tmp.alloc_n(&d_order, (size_t)std::max(nbr, 1)));
    AMG_TRY(tmp.alloc_n(&d_status, 1));
    AMG_TRY_CUDA(cudaMemcpyAsync(out->F, A.val, sizeof(double) * A.nnzb * bb,
                                 cudaMemcpyDeviceToDevice, s));
    AMG_TRY_CUDA(cudaMemcpyAsync(d_diag, diag.data(), sizeof(int) * nbr, cudaMemcpyHostToDevice, s));
    AMG_TRY_CUDA(cudaMemcpyAsync(d_order, order.data(), sizeof(int) * nbr, cudaMemcpyHostToDevice,
                                 s));
    const int big = INT_MAX;
    AMG_TRY_CUDA(cudaMemcpyAsync(d_status, &big, sizeof(int), cudaMemcpyHostToDevice, s));
    for (int k = 0; k < depth; ++k) {  // one launch per dependency level, a CTA per row
        const unsigned cnt = (unsigned)(lptr[k + 1] - lptr[k]);
        if (b == 3)
            ilu_factor_rows_kernel<3, 1><<<cnt, 32, 0, s>>>(A.row_ptr, A.col, d_diag, out->F,
                                                            out->Dinv, d_order + lptr[k], d_status);
        else
            ilu_factor_rows_kernel<6, 4><<<cnt, 128, 0, s>>>(A.row_ptr, A.col, d_diag, out->F,
                                                             out->Dinv, d_order + lptr[k],
                                                             d_status);
        count_launch(1);
    }
    AMG_TRY_CUDA(cudaGetLastError());
    int bad = big;
    AMG_TRY_CUDA(cudaMemcpyAsync(&bad, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));  // host vectors above are still in use until here
    if (bad != big) {
        set_error("ILU(0) breakdown: the diagonal block of row %d cannot be inverted", bad);
        return AMG_ERR_BREAKDOWN;
    }
    // strict triangles as BSR, then their sliced copies
    BsrD Lb, Ub;
    Lb.nbr = Ub.nbr = nbr;
    Lb.nbc = Ub.nbc = nbr;
    Lb.br = Lb.bc = Ub.br = Ub.bc = b;
    Lb.nnzb = lrp[nbr];
    Ub.nnzb = urp[nbr];
    AMG_TRY(tmp.alloc_n(&Lb.row_ptr, (size_t)nbr + 1));
    AMG_TRY(tmp.alloc_n(&Ub.row_ptr, (size_t)nbr + 1));
    AMG_TRY(tmp.alloc_n(&Lb.col, (size_t)std::max<int64_t>(Lb.nnzb, 1)));
    AMG_TRY(tmp.alloc_n(&Ub.col, (size_t)std::max<int64_t>(Ub.nnzb, 1)));
    AMG_TRY(tmp.alloc_n(&Lb.val, (size_t)std::max<int64_t>(Lb.nnzb, 1) * bb));
    AMG_TRY(tmp.alloc_n(&Ub.val, (size_t)std::max<int64_t>(Ub.nnzb, 1) * bb));
    AMG_TRY_CUDA(cudaMemcpyAsync(Lb.row_ptr, lrp.data(), sizeof(int) * (nbr + 1),
                                 cudaMemcpyHostToDevice, s));
    AMG_TRY_CUDA(cudaMemcpyAsync(Ub.row_ptr, urp.data(), sizeof(int) * (nbr + 1),
                                 cudaMemcpyHostToDevice, s));
    if (nbr > 0) {
        const unsigned grid = (unsigned)(((int64_t)nbr + FT / 32 - 1) / (FT / 32));
        if (b == 3)
            ilu_split_kernel<3><<<grid, FT, 0, s>>>(A.row_ptr, A.col, d_diag, out->F, nbr,
                                                    Lb.row_ptr, Lb.col, Lb.val, Ub.row_ptr, Ub.col,
                                                    Ub.val);
        else
            ilu_split_kernel<6><<<grid, FT, 0, s>>>(A.row_ptr, A.col, d_diag, out->F, nbr,
                                                    Lb.row_ptr, Lb.col, Lb.val, Ub.row_ptr, Ub.col,
                                                    Ub.val);
        count_launch(1);
        AMG_TRY_CUDA(cudaGetLastError());
    }
    double pad = 0.0;
    out->has_L = Lb.nnzb > 0;
    out->has_U = Ub.nnzb > 0;
    if (out->has_L) AMG_TRY(bsr_to_sell<double>(Lb, keep, s, &out->sL, &pad, max_lanes));
    if (out->has_U) AMG_TRY(bsr_to_sell<double>(Ub, keep, s, &out->sU, &pad, max_lanes));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));  // lrp / urp are host memory
    tmp.release(Ub.val);
    tmp.release(Lb.val);
    tmp.release(Ub.col);
    tmp.release(Lb.col);
    tmp.release(Ub.row_ptr);
    tmp.release(Lb.row_ptr);
    tmp.release(d_status);
    tmp.release(d_order);
    tmp.release(d_diag);
    return AMG_OK;
}

int ilu0_apply(const Ilu &F, int sweeps, const double *r, double *x, const Geom &g, cudaStream_t s)
{
    const int64_t n = (int64_t)F.nbr * F.b;
    // lower triangle: y <- r - L_s y from y = r
    const double *y = r;
    for (int k = 0; k < sweeps && F.has_L; ++k) {
        double *nxt = (y == F.y0) ? F.y1 : F.y0;
        SellArgs<double> a{};
        a.x = y;
        a.f = r;
        a.y = nxt;
        AMG_TRY((launch_sell<double, double>(F.sL, SPMV_RESID, DOT_NONE, a, g, s)));
        y = nxt;
    }
    double *w = (y == F.y0) ? F.y1 : F.y0;
    // upper triangle: x <- U_D^-1 (y - U_s x) from x = U_D^-1 y
    AMG_TRY(block_diag_apply(F.b, F.Dinv, y, x, n, s));
    for (int k = 0; k < sweeps && F.has_U; ++k) {
        SellArgs<double> a{};
        a.x = x;
        a.f = y;
        a.y = w;
        AMG_TRY((launch_sell<double, double>(F.sU, SPMV_RESID, DOT_NONE, a, g, s)));
        AMG_TRY(block_diag_apply(F.b, F.Dinv, w, x, n, s));
    }
    return AMG_OK;
}

}  // namespace amg
