// Block damped Jacobi smoother (AMG_SMOOTH_BJACOBI): the damped Jacobi
// relaxation that Sec. 2 names among the smoothers, taken over the node
// blocks of every smoothing level, M_I = (2 w_s / lambda) A_II^{-1}.
//
// Setup per level, on the device:
//   1. W_I = A_II^{-1} per node block (b x b: 3 on the finest level, 6
//      below), by Gauss-Jordan elimination without pivoting on the rows and
//      columns of A_II that are not entirely zero (a near-nullspace column
//      dropped on the level above leaves a zero row and column, which stay
//      zero in W_I); each product and sum rounded on its own (no contracted
//      multiply-adds), then symmetrised exactly, W_ab = W_ba = (X_ab + X_ba)/2.
//   2. lambda, an estimate of lambda_max(D_b^{-1} A) (D_b = block diagonal of
//      A): 20 power iterations x <- W A x / |W A x| from a hashed start
//      vector (the solve's sliced A), then the Rayleigh quotient (x, A x) /
//      (x, D_b x).  The quotient is a generalised eigenvalue estimate of
//      (A, D_b) and never exceeds lambda_max, so the damped operator M A peaks near 2 w_s (1.6
//      with w_s = 0.8) on any material: undamped block Jacobi has
//      lambda_max(D_b^{-1} A) of 2.6-3.9 on Q1 elasticity (nu 0.2-0.45), and
//      a damping above 2 / lambda_max makes the symmetric V-cycle indefinite.
//   3. M_I = (2 w_s / lambda) W_I, plus an FP32 copy for the FP32 and BF16
//      V-cycles.
// The V-cycle applies the blocks in the SpMV epilogue (smoothing), in the
// restriction's epilogue (the next level's pre-smoothing from zero) and, on
// the finest level, in a block multiply after the CG update.
#include <cmath>

#include "amg_internal.cuh"

namespace amg {

constexpr int BJ_THREADS = 128;

// W_I for every node block I of the BSR matrix A (b x b blocks, one thread
// per block row); bad[0] records 1 + the first block row with a
// non-positive pivot.
template <int B>
__global__ void __launch_bounds__(BJ_THREADS) bjacobi_blocks_kernel(
    const int *__restrict__ rp, const int *__restrict__ col, const double *__restrict__ val,
    int nbr, double *__restrict__ W, int *__restrict__ bad)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nbr) return;
    double blk[B][B];
#pragma unroll
    for (int r = 0; r < B; ++r)
#pragma unroll
        for (int c = 0; c < B; ++c) blk[r][c] = 0.0;
    // the diagonal block: columns ascend within the row
    int lo = rp[I], hi = rp[I + 1];
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (col[mid] < I) lo = mid + 1;
        else hi = mid;
    }
    if (lo < rp[I + 1] && col[lo] == I) {
        const double *a = val + (int64_t)lo * B * B;
#pragma unroll
        for (int r = 0; r < B; ++r)
#pragma unroll
            for (int c = 0; c < B; ++c) blk[r][c] = a[r * B + c];
    }
    int keep[B], k = 0;
#pragma unroll
    for (int r = 0; r < B; ++r) {
        bool z = true;
#pragma unroll
        for (int c = 0; c < B; ++c) z = z && blk[r][c] == 0.0;
        keep[r] = -1;
        if (!z) keep[k++] = r;
    }
    // compact the kept rows and columns into X (k x k, upper-left)
    double X[B][B];
#pragma unroll
    for (int x = 0; x < B; ++x)
#pragma unroll
        for (int y = 0; y < B; ++y) {
            double v = 0.0;
            if (x < k && y < k) {
                // keep[] indices are runtime values: select without indexing
#pragma unroll
                for (int r = 0; r < B; ++r)
#pragma unroll
                    for (int c = 0; c < B; ++c)
                        if (keep[x] == r && keep[y] == c) v = blk[r][c];
            }
            X[x][y] = v;
        }
    bool ok = true;
#pragma unroll
    for (int j = 0; j < B; ++j) {
        if (j >= k) break;
        const double piv = X[j][j];
        if (!(piv > 0.0)) {
            ok = false;
            break;
        }
        const double inv = 1.0 / piv;
        X[j][j] = 1.0;
#pragma unroll
        for (int c = 0; c < B; ++c)
            if (c < k) X[j][c] = __dmul_rn(X[j][c], inv);
#pragma unroll
        for (int i = 0; i < B; ++i) {
            if (i >= k || i == j) continue;
            const double f = X[i][j];
            X[i][j] = 0.0;
#pragma unroll
            for (int c = 0; c < B; ++c)
                if (c < k) X[i][c] = __dsub_rn(X[i][c], __dmul_rn(f, X[j][c]));
        }
    }
    if (!ok) atomicMin(bad, I + 1);
    double *w = W + (int64_t)I * B * B;
#pragma unroll
    for (int r = 0; r < B; ++r)
#pragma unroll
        for (int c = 0; c < B; ++c) {
            double v = 0.0;
#pragma unroll
            for (int x = 0; x < B; ++x)
#pragma unroll
                for (int y = 0; y < B; ++y)
                    if (x < k && y < k && keep[x] == r && keep[y] == c)
                        v = ok ? __dmul_rn(__dadd_rn(X[x][y], X[y][x]), 0.5) : 0.0;
            w[r * B + c] = v;
        }
}

// x_0[i] = h(i) / 2^32 - 1/2 with h(i) = (i + 1) * 2654435761 mod 2^32
__global__ void bjacobi_start_kernel(double *__restrict__ x, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t h = (uint32_t)((uint64_t)(i + 1) * 2654435761u);
        x[i] = (double)h / 4294967296.0 - 0.5;
    }
}

// y_I = Wb_I t_I / sqrt(*prev) for b x b blocks (one thread per block row;
// prev = null: no division), with per-CTA partial sums of |y|^2 in a fixed
// order: one power-iteration step on the unnormalised iterate t = A y_k, its
// normalisation by |y_k| folded in
template <int B>
__global__ void __launch_bounds__(256) bjacobi_apply_kernel(const double *__restrict__ Wb,
                                                            const double *__restrict__ t,
                                                            double *__restrict__ y, int nbr,
                                                            const double *__restrict__ prev,
                                                            double *__restrict__ part)
{
    __shared__ double sm[256];
    const double pv = prev ? *prev : 1.0;
    const double inv = pv > 0.0 ? 1.0 / sqrt(pv) : 0.0;  // a zero iterate stays zero
    double acc = 0.0;
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nbr; I += gridDim.x * blockDim.x) {
        const double *w = Wb + (int64_t)I * B * B;
        double tv[B];
#pragma unroll
        for (int c = 0; c < B; ++c) tv[c] = t[(int64_t)I * B + c] * inv;
#pragma unroll
        for (int r = 0; r < B; ++r) {
            double v = 0.0;
#pragma unroll
            for (int c = 0; c < B; ++c) v += w[r * B + c] * tv[c];
            y[(int64_t)I * B + r] = v;
            acc += v * v;
        }
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w >= 1; w >>= 1) {
        if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

// y_I = A_II x_I (the block diagonal of A)
template <int B>
__global__ void bjacobi_diag_kernel(const int *__restrict__ rp, const int *__restrict__ col,
                                    const double *__restrict__ val, int nbr,
                                    const double *__restrict__ x, double *__restrict__ y)
{
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nbr; I += gridDim.x * blockDim.x) {
        int lo = rp[I], hi = rp[I + 1];
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (col[mid] < I) lo = mid + 1;
            else hi = mid;
        }
        const bool has = lo < rp[I + 1] && col[lo] == I;
        const double *a = val + (int64_t)lo * B * B;
#pragma unroll
        for (int r = 0; r < B; ++r) {
            double v = 0.0;
            if (has)
#pragma unroll
                for (int c = 0; c < B; ++c) v += a[r * B + c] * x[(int64_t)I * B + c];
            y[(int64_t)I * B + r] = v;
        }
    }
}

// per-CTA partial sums of x . y in a fixed order (grid-stride, then a tree)
__global__ void __launch_bounds__(256) bjacobi_dot_kernel(const double *__restrict__ x,
                                                          const double *__restrict__ y, int64_t n,
                                                          double *__restrict__ part)
{
    __shared__ double sm[256];
    double v = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v += x[i] * y[i];
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int w = 128; w >= 1; w >>= 1) {
        if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void bjacobi_damp_kernel(double *__restrict__ M, float *__restrict__ Mf, int64_t n,
                                    double w)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = w * M[i];
        M[i] = v;
        if (Mf) Mf[i] = (float)v;
    }
}

template <int B>
static int bjacobi_level(amg_handle h, Level &L, int l, const Sell<double> &S, DevArena &tmp,
                         cudaStream_t s)
{
    const Geom &g = h->geom;
    const int nbr = L.A.nbr;
    const int64_t n = L.n(), nb = (int64_t)nbr * B * B;
    const bool narrow = h->prm.precision == AMG_PREC_FP32 || h->prm.precision == AMG_PREC_BF16;
    AMG_TRY(h->mem.alloc_n(&L.Mb, (size_t)std::max<int64_t>(nb, 1)));
    if (narrow) AMG_TRY(h->mem.alloc_n(&L.Mbf, (size_t)std::max<int64_t>(nb, 1)));
    int *bad = nullptr;
    double *x = nullptr, *t = nullptr, *y = nullptr, *sc = nullptr, *part = nullptr;
    AMG_TRY(tmp.alloc_n(&bad, 1));
    AMG_TRY(tmp.alloc_n(&x, (size_t)std::max<int64_t>(n, 1)));
    AMG_TRY(tmp.alloc_n(&t, (size_t)std::max<int64_t>(n, 1)));
    AMG_TRY(tmp.alloc_n(&y, (size_t)std::max<int64_t>(n, 1)));
    AMG_TRY(tmp.alloc_n(&sc, 3));
    const int vg = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, g.max_ctas));
    const int bg = std::max(1, std::min((nbr + 255) / 256, g.max_ctas));
    AMG_TRY(tmp.alloc_n(&part, (size_t)std::max(vg, bg) + 1));
    const int big = 0x7fffffff;
    AMG_TRY_CUDA(cudaMemcpyAsync(bad, &big, sizeof(int), cudaMemcpyHostToDevice, s));
    if (nbr > 0) {
        bjacobi_blocks_kernel<B><<<(nbr + BJ_THREADS - 1) / BJ_THREADS, BJ_THREADS, 0, s>>>(
            L.A.row_ptr, L.A.col, L.A.val, nbr, L.Mb, bad);
        count_launch(1);
    }
    AMG_TRY_CUDA(cudaGetLastError());
    // lambda: 20 power iterations on unnormalised iterates (each step divides
    // by the previous norm), then the Rayleigh quotient of the last one
    auto spmv = [&](const double *in, double *out) -> int {
        SellArgs<double> a{};
        a.x = in;
        a.y = out;
        return launch_sell<double, double>(S, SPMV_PLAIN, DOT_NONE, a, g, s);
    };
    bjacobi_start_kernel<<<vg, 256, 0, s>>>(x, n);
    count_launch(1);
    double *cur = x, *nxt = y;
    for (int it = 0; it < 20; ++it) {
        AMG_TRY(spmv(cur, t));
        bjacobi_apply_kernel<B><<<bg, 256, 0, s>>>(L.Mb, t, nxt, nbr, it ? sc : nullptr, part);
        count_launch(1);
        AMG_TRY(launch_reduce_sum(part, bg, sc, s));
        std::swap(cur, nxt);
    }
    AMG_TRY(spmv(cur, t));
    bjacobi_dot_kernel<<<vg, 256, 0, s>>>(cur, t, n, part);
    count_launch(1);
    AMG_TRY(launch_reduce_sum(part, vg, sc + 1, s));
    bjacobi_diag_kernel<B><<<bg, 256, 0, s>>>(L.A.row_ptr, L.A.col, L.A.val, nbr, cur, nxt);
    count_launch(1);
    bjacobi_dot_kernel<<<vg, 256, 0, s>>>(cur, nxt, n, part);
    count_launch(1);
    AMG_TRY(launch_reduce_sum(part, vg, sc + 2, s));
    AMG_TRY_CUDA(cudaGetLastError());
    int hbad = big;
    double hs[3] = {0, 0, 0};
    AMG_TRY_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaMemcpyAsync(hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    if (hbad != big) {
        set_error("block Jacobi: node block %d of level %d is not positive definite", hbad - 1, l);
        return AMG_ERR_ARG;
    }
    const double lam = hs[2] > 0.0 ? hs[1] / hs[2] : 0.0;
    L.bj_lambda = lam;
    const double w = lam > 0.0 ? 2.0 * h->prm.smooth_relax / lam : 0.0;
    if (nb > 0) {
        const int dg = (int)std::min<int64_t>((nb + 255) / 256, g.max_ctas);
        bjacobi_damp_kernel<<<dg, 256, 0, s>>>(L.Mb, narrow ? L.Mbf : nullptr, nb, w);
        count_launch(1);
    }
    AMG_TRY_CUDA(cudaGetLastError());
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    for (void *p : {(void *)bad, (void *)x, (void *)t, (void *)y, (void *)sc, (void *)part})
        tmp.release(p);
    return AMG_OK;
}

// Runs after the solve's sliced copies exist: the power iteration multiplies
// with the level's FP64 sliced A (the reduced-precision V-cycles keep one
// for level 0 only; coarser levels get a temporary FP64 copy).
int bjacobi_setup(amg_handle h, DevArena &tmp, cudaStream_t s)
{
    for (size_t l = 0; l + 1 < h->lv.size(); ++l) {
        Level &L = h->lv[l];
        Sell<double> own;
        const Sell<double> *S = &L.sA;
        if (L.sA.nslices == 0 && L.A.nbr > 0) {
            double pad = 0.0;
            AMG_TRY(bsr_to_sell<double>(L.A, tmp, s, &own, &pad, h->max_lanes));
            S = &own;
        }
        int st;
        if (L.A.br == 3) st = bjacobi_level<3>(h, L, (int)l, *S, tmp, s);
        else if (L.A.br == 6) st = bjacobi_level<6>(h, L, (int)l, *S, tmp, s);
        else {
            set_error("block Jacobi needs 3x3 or 6x6 node blocks (level %d has %d)", (int)l, L.A.br);
            st = AMG_ERR_ARG;
        }
        if (S == &own) {
            AMG_TRY_CUDA(cudaStreamSynchronize(s));
            for (void *p : {(void *)own.slice_ptr, (void *)own.col, (void *)own.val, (void *)own.perm})
                if (p) tmp.release(p);
        }
        if (st < 0) return st;
    }
    return AMG_OK;
}

}  // namespace amg
