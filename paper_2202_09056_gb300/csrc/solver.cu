// The hierarchy handle, the setup loop (Alg. 1), the V-cycle (Alg. 2) and the
// device-resident preconditioned CG of Sec. 4, and the C ABI around them.
//
// The CG loop is one CUDA graph: a conditional WHILE node whose body holds
// one full iteration (V-cycle, direction update, A p with the fused p.Ap,
// u/r updates with the fused ||r||^2, the true-residual confirmation).  All
// scalars (alpha, beta, norms, counters, flags) live in device memory; the
// last kernel of the body clears the loop condition once the solve has
// converged, reached maxiter or broken down.  The host synchronises only
// before the loop (initial residual) and after it.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "amg_internal.cuh"

namespace amg {
const char *last_error();

constexpr int FIN_THREADS = 256;

template <int NT> __device__ __forceinline__ double block_sum_fixed(const double *p, int n)
{
    __shared__ double red[NT];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += NT) v += p[i];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = NT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < (unsigned)w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    return red[0];
}

template <class TV>
__global__ void __launch_bounds__(256) vec_dot_kernel(const TV *__restrict__ x,
                                                      const TV *__restrict__ y, int64_t n,
                                                      double *__restrict__ partials)
{
    double v = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v += (double)x[i] * (double)y[i];
    __shared__ double red[256];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < (unsigned)w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

// First pre-smoothing sweep from a zero guess in the V-cycle's precision:
// t = M r (or 0 without pre-smoothing); rv receives r in that precision when
// the V-cycle does not run in FP64.
template <class TV>
__global__ void scale_kernel(const TV *__restrict__ M, const double *__restrict__ r,
                             TV *__restrict__ t, TV *__restrict__ rv, int64_t n, int zero)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const TV ri = (TV)r[i];
        if (rv) rv[i] = ri;
        if (t) t[i] = zero ? TV(0) : M[i] * ri;
    }
}

// z (V-cycle precision) -> double
template <class TV>
__global__ void widen_kernel(const TV *__restrict__ a, double *__restrict__ b, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}

__global__ void narrow_kernel(const double *__restrict__ a, float *__restrict__ b, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

__global__ void cg_start_kernel(CgState *st, const double *__restrict__ scal, double tol,
                                int maxiter)
{
    const double nf = sqrt(scal[0]);
    st->tol = tol;
    st->maxiter = maxiter;
    st->nf = nf;
    st->res = nf > 0.0 ? sqrt(scal[1]) / nf : 0.0;
    st->res_true = st->res;
    st->rz = st->pq = st->alpha = st->beta = 0.0;
    st->it = 0;
    st->check = st->replace = st->converged = st->stop = 0;
    st->no_check = 1;
    st->no_replace = 1;
    st->status = AMG_NOT_CONVERGED;
}

// beta = (r.z)_new / (r.z)_old (0 on the first iteration)
__global__ void __launch_bounds__(FIN_THREADS) cg_beta_kernel(CgState *st,
                                                             const double *__restrict__ part,
                                                             int np)
{
    const double rz = block_sum_fixed<FIN_THREADS>(part, np);
    if (threadIdx.x != 0 || st->stop) return;
    if (!(rz > 0.0) || !isfinite(rz)) {
        st->status = AMG_ERR_BREAKDOWN;
        st->stop = 1;
        st->no_check = 1;
        st->no_replace = 1;
        return;
    }
    st->beta = (st->it == 0) ? 0.0 : rz / st->rz;
    st->rz = rz;
}

template <class TV>
__global__ void cg_direction_kernel(const TV *__restrict__ z, double *__restrict__ p,
                                    const CgState *__restrict__ st, int64_t n)
{
    if (st->stop) return;
    // the first direction is z itself: p holds no earlier direction to scale
    // (0 * p would carry whatever its memory held, NaN included)
    const double beta = st->beta;
    const bool first = st->it == 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = first ? (double)z[i] : (double)z[i] + beta * p[i];
}

__global__ void __launch_bounds__(FIN_THREADS) cg_alpha_kernel(CgState *st,
                                                              const double *__restrict__ part,
                                                              int np)
{
    const double pq = block_sum_fixed<FIN_THREADS>(part, np);
    if (threadIdx.x != 0 || st->stop) return;
    if (!(pq > 0.0) || !isfinite(pq)) {
        st->status = AMG_ERR_BREAKDOWN;
        st->stop = 1;
        st->no_check = 1;
        st->no_replace = 1;
        return;
    }
    st->pq = pq;
    st->alpha = st->rz / pq;
}

// u += alpha p ; r -= alpha q ; t0 = M r (next pre-smoothing, in the V-cycle's
// precision; rv = r in that precision when it is not FP64) ; partial r.r
template <class TV>
__global__ void __launch_bounds__(256) cg_update_kernel(double *__restrict__ u, double *__restrict__ r,
                                                        const double *__restrict__ p,
                                                        const double *__restrict__ q,
                                                        const TV *__restrict__ M,
                                                        TV *__restrict__ t0, TV *__restrict__ rv,
                                                        const CgState *__restrict__ st, int64_t n,
                                                        int pre, double *__restrict__ partials)
{
    if (st->stop) return;
    const double alpha = st->alpha;
    double v = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        u[i] += alpha * p[i];
        const double ri = r[i] - alpha * q[i];
        r[i] = ri;
        const TV rr = (TV)ri;
        if (rv) rv[i] = rr;
        if (t0) t0[i] = pre ? M[i] * rr : TV(0);
        v += ri * ri;
    }
    __shared__ double red[256];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < (unsigned)w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(FIN_THREADS) cg_resnorm_kernel(CgState *st,
                                                                const double *__restrict__ part,
                                                                int np)
{
    const double rr = block_sum_fixed<FIN_THREADS>(part, np);
    if (threadIdx.x != 0 || st->stop) return;
    st->res = sqrt(rr) / st->nf;
    st->it += 1;
    st->no_check = (st->res <= st->tol) ? 0 : 1;
}

// Confirmation with the true residual and the loop decision.
__global__ void __launch_bounds__(FIN_THREADS) cg_decide_kernel(CgState *st,
                                                               const double *__restrict__ part,
                                                               int np,
                                                               cudaGraphConditionalHandle cond,
                                                               int use_cond)
{
    const double rr = block_sum_fixed<FIN_THREADS>(part, np);
    if (threadIdx.x != 0) return;
    if (!st->stop) {
        st->replace = 0;
        if (!st->no_check) {
            const double tr = sqrt(rr) / st->nf;
            st->res_true = tr;
            if (tr <= st->tol) {
                st->converged = 1;
                st->stop = 1;
                st->status = AMG_OK;
            } else {
                st->replace = 1;
            }
        }
        st->no_replace = st->replace ? 0 : 1;
        if (!st->stop && st->it >= st->maxiter) {
            st->stop = 1;
            st->status = AMG_NOT_CONVERGED;
        }
    }
    if (st->stop) {
        st->no_replace = 1;
        if (use_cond) cudaGraphSetConditional(cond, 0);
    }
}

// r = r_true (residual replacement) and the matching pre-smoothed t0.
template <class TV>
__global__ void cg_replace_kernel(double *__restrict__ r, const double *__restrict__ rt,
                                  const TV *__restrict__ M, TV *__restrict__ t0,
                                  TV *__restrict__ rv, const CgState *__restrict__ st, int64_t n,
                                  int pre)
{
    if (st->no_replace) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double ri = rt[i];
        r[i] = ri;
        const TV rr = (TV)ri;
        if (rv) rv[i] = rr;
        if (t0) t0[i] = pre ? M[i] * rr : TV(0);
    }
}

}  // namespace amg

using namespace amg;

static int vgrid(amg_handle h, int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g > h->geom.max_ctas) g = h->geom.max_ctas;
    return (int)std::max<int64_t>(g, 1);
}

// One level of the V-cycle in the precision it runs in.
template <class VT, class TV> struct VLevel {
    const Sell<VT> *A = nullptr, *P = nullptr, *R = nullptr;
    const TV *M = nullptr;
    TV *f = nullptr, *u = nullptr, *e = nullptr, *z = nullptr, *t = nullptr;
    int n = 0;
};

template <class VT, class TV> static VLevel<VT, TV> view(Level &L);
template <> VLevel<double, double> view<double, double>(Level &L)
{
    VLevel<double, double> v;
    v.A = &L.sA; v.P = &L.sP; v.R = &L.sR; v.M = L.M;
    v.f = L.f; v.u = L.u; v.e = L.e; v.z = L.z; v.t = L.t; v.n = L.n();
    return v;
}
template <> VLevel<df32, double> view<df32, double>(Level &L)
{
    VLevel<df32, double> v;
    v.A = &L.eA; v.P = &L.eP; v.R = &L.eR; v.M = L.M;
    v.f = L.f; v.u = L.u; v.e = L.e; v.z = L.z; v.t = L.t; v.n = L.n();
    return v;
}
template <> VLevel<float, float> view<float, float>(Level &L)
{
    VLevel<float, float> v;
    v.A = &L.fA; v.P = &L.fP; v.R = &L.fR; v.M = L.Mf;
    v.f = L.vf; v.u = L.vu; v.e = L.ve; v.z = L.vz; v.t = L.vt; v.n = L.n();
    return v;
}
template <> VLevel<__nv_bfloat16, float> view<__nv_bfloat16, float>(Level &L)
{
    VLevel<__nv_bfloat16, float> v;
    v.A = &L.bA; v.P = &L.bP; v.R = &L.bR; v.M = L.Mf;
    v.f = L.vf; v.u = L.vu; v.e = L.ve; v.z = L.vz; v.t = L.vt; v.n = L.n();
    return v;
}

template <class TV>
static int launch_vec_dot(amg_handle h, const TV *x, const TV *y, int64_t n, double *part,
                          cudaStream_t s, int *grid_out = nullptr);

// Block ILU(0) smoothing step x = ILU_l^-1 r and y = a + b (FP64 V-cycle only).
template <class TV> static int ilu_smooth(amg_handle h, int l, const TV *r, TV *x, cudaStream_t s);
template <> int ilu_smooth<double>(amg_handle h, int l, const double *r, double *x, cudaStream_t s)
{
    return ilu0_apply(h->lv[l].ilu, h->prm.ilu_sweeps, r, x, h->geom, s);
}
template <> int ilu_smooth<float>(amg_handle, int, const float *, float *, cudaStream_t)
{
    set_error("the ILU(0) smoother runs in the FP64 V-cycle only");
    return AMG_ERR_STATE;
}
template <class TV> static int vec_add(const TV *a, const TV *b, TV *y, int64_t n, cudaStream_t s);
template <> int vec_add<double>(const double *a, const double *b, double *y, int64_t n,
                                cudaStream_t s)
{
    return launch_vec_add(a, b, y, n, s);
}
template <> int vec_add<float>(const float *, const float *, float *, int64_t, cudaStream_t)
{
    set_error("the ILU(0) smoother runs in the FP64 V-cycle only");
    return AMG_ERR_STATE;
}

// One V-cycle (Alg. 2) from a zero initial guess: z0 = V(f0), matrices stored
// in VT and vectors in TV.  Level 0's u must already hold the first
// pre-smoothing sweep M_0 f0 (or zero without pre-smoothing).  With
// rz_partials, the last level-0 kernel also leaves the per-CTA partial sums
// of f0 . z0 (accumulated in FP64), and *rz_np their number (the grid of
// the kernel that wrote them).
// The learned blocks in the V-cycle's vector precision.
// The smoother blocks of level l, in the V-cycle vectors' precision, or null
// when the level smooths with the SPAI0 diagonal: block damped Jacobi blocks
// on every smoothing level, or the learned 3x3 blocks on level 0.
template <class TV> static const TV *blocks_ptr(const amg_handle h, size_t l);
template <> const double *blocks_ptr<double>(const amg_handle h, size_t l)
{
    if (l + 1 >= h->lv.size()) return nullptr;
    const bool on = h->prm.smoother == AMG_SMOOTH_BJACOBI || (l == 0 && h->learned);
    return on ? h->lv[l].Mb : nullptr;
}
template <> const float *blocks_ptr<float>(const amg_handle h, size_t l)
{
    if (l + 1 >= h->lv.size()) return nullptr;
    const bool on = h->prm.smoother == AMG_SMOOTH_BJACOBI || (l == 0 && h->learned);
    return on ? h->lv[l].Mbf : nullptr;
}

template <class VT, class TV>
static int record_vcycle(amg_handle h, const TV *f0, TV *z0, double *rz_partials, cudaStream_t s,
                         int *rz_np = nullptr)
{
    const int L = (int)h->lv.size() - 1;
    const int npre = h->prm.npre, npost = h->prm.npost;
    const Geom &g = h->geom;
    std::vector<VLevel<VT, TV>> V;
    for (auto &lev : h->lv) V.push_back(view<VT, TV>(lev));
    std::vector<TV *> ucur(L + 1, nullptr), spare(L + 1, nullptr);
    const bool ilu = h->ilu != 0;  // FP64 V-cycle only (checked at setup)
    const bool ilu_pre = ilu && npre > 0;
    for (int l = 0; l < L; ++l) {
        VLevel<VT, TV> &C = V[l];
        VLevel<VT, TV> &N = V[l + 1];
        const TV *f = (l == 0) ? f0 : C.f;
        TV *u = C.u, *t = C.t;
        if (ilu_pre) {  // first pre-smoothing sweep from zero: u = ILU^-1 f
            AMG_TRY(ilu_smooth<TV>(h, l, f, u, s));
            for (int sweep = 1; sweep < npre; ++sweep) {  // u += ILU^-1 (f - A u)
                SellArgs<TV> a{};
                a.x = u;
                a.f = f;
                a.y = C.e;
                AMG_TRY((launch_sell<VT, TV>(*C.A, SPMV_RESID, DOT_NONE, a, g, s)));
                AMG_TRY(ilu_smooth<TV>(h, l, C.e, t, s));
                AMG_TRY(vec_add<TV>(u, t, u, C.n, s));
            }
        }
        for (int sweep = 1; sweep < npre && !ilu; ++sweep) {  // further pre-smoothing sweeps
            const TV *mb = blocks_ptr<TV>(h, l);
            const bool blocks = mb != nullptr;
            SellArgs<TV> a{};
            a.x = u;
            a.f = f;
            a.M = C.M;
            a.Mb = mb;
            a.y = t;
            AMG_TRY((launch_sell<VT, TV>(*C.A, blocks ? SPMV_SMOOTHB : SPMV_SMOOTH, DOT_NONE, a, g,
                                         s)));
            std::swap(u, t);
        }
        ucur[l] = u;
        spare[l] = t;
        {  // e = f - A u
            SellArgs<TV> a{};
            a.x = u;
            a.f = f;
            a.y = C.e;
            AMG_TRY((launch_sell<VT, TV>(*C.A, SPMV_RESID, DOT_NONE, a, g, s)));
        }
        {  // f_{l+1} = R e ; u_{l+1} = M_{l+1} f_{l+1}
            SellArgs<TV> a{};
            a.x = C.e;
            a.y = N.f;
            const bool next_smooths = (l + 1 < L);
            // with ILU(0) the next level pre-smooths itself (npre = 0: zero u)
            a.y2 = (next_smooths && !ilu_pre) ? N.u : nullptr;
            a.M = (next_smooths && npre > 0) ? N.M : nullptr;
            // with smoother blocks on the next level, its pre-smoothing is
            // the block product (npre = 0: zero u, written by a null M)
            if (next_smooths && npre > 0) a.Mbn = blocks_ptr<TV>(h, l + 1);
            AMG_TRY((launch_sell<VT, TV>(*C.R, SPMV_RESTRICT, DOT_NONE, a, g, s)));
        }
    }
    {  // coarsest: direct solve with the dense FP64 inverse
        VLevel<VT, TV> &Cc = V[L];
        const TV *fL = (L == 0) ? f0 : Cc.f;
        TV *zL = (L == 0) ? z0 : Cc.z;
        AMG_TRY(launch_coarse_gemv<TV>(h->Ainv, h->nc, fL, zL, g, s));
        if (L == 0 && rz_partials)
            AMG_TRY(launch_vec_dot<TV>(h, f0, z0, h->nc, rz_partials, s, rz_np));
    }
    for (int l = L - 1; l >= 0; --l) {
        VLevel<VT, TV> &C = V[l];
        VLevel<VT, TV> &N = V[l + 1];
        const TV *f = (l == 0) ? f0 : C.f;
        TV *u = ucur[l], *t = spare[l];
        TV *zl = (l == 0) ? z0 : C.z;
        {  // u += P z_{l+1}
            SellArgs<TV> a{};
            a.x = N.z;
            a.u = u;
            a.y = u;
            AMG_TRY((launch_sell<VT, TV>(*C.P, SPMV_AXPY, DOT_NONE, a, g, s)));
        }
        if (ilu) {  // u += ILU^-1 (f - A u), the last sweep written to z_l
            for (int sweep = 0; sweep < npost; ++sweep) {
                SellArgs<TV> a{};
                a.x = u;
                a.f = f;
                a.y = C.e;
                AMG_TRY((launch_sell<VT, TV>(*C.A, SPMV_RESID, DOT_NONE, a, g, s)));
                AMG_TRY(ilu_smooth<TV>(h, l, C.e, t, s));
                AMG_TRY(vec_add<TV>(u, t, sweep == npost - 1 ? zl : u, C.n, s));
            }
            if (npost > 0 && l == 0 && rz_partials)
                AMG_TRY(launch_vec_dot<TV>(h, f0, z0, C.n, rz_partials, s, rz_np));
        }
        const TV *w = u;
        const TV *mb = blocks_ptr<TV>(h, l);
        const bool blocks = mb != nullptr;
        for (int sweep = 0; sweep < npost && !ilu; ++sweep) {  // u += M (f - A u)
            const bool last = (sweep == npost - 1);
            TV *out = last ? zl : t;
            SellArgs<TV> a{};
            a.x = w;
            a.f = f;
            a.M = C.M;
            a.Mb = mb;
            a.y = out;
            a.partials = rz_partials;
            const int dot = (l == 0 && last && rz_partials) ? DOT_FY : DOT_NONE;
            AMG_TRY((launch_sell<VT, TV>(*C.A, blocks ? SPMV_SMOOTHB : SPMV_SMOOTH, dot, a, g, s,
                                         dot != DOT_NONE ? rz_np : nullptr)));
            w = out;
            t = (out == t) ? u : t;  // ping-pong between u and t
        }
        if (npost == 0) {
            AMG_TRY_CUDA(cudaMemcpyAsync(zl, u, sizeof(TV) * C.n, cudaMemcpyDeviceToDevice, s));
            if (l == 0 && rz_partials)
                AMG_TRY(launch_vec_dot<TV>(h, f0, z0, C.n, rz_partials, s, rz_np));
        }
    }
    return AMG_OK;
}

// One CG iteration, as recorded into the body of the graph.  The outer
// recurrences, dots and the fine A p product are FP64; the V-cycle runs with
// matrices in VT and vectors in TV (FP64 or FP32), its input r and output z
// converted at the boundary.
template <class VT, class TV>
static int record_cg_iteration_t(amg_handle h, cudaStream_t s, cudaGraphConditionalHandle cond,
                                 int use_cond)
{
    constexpr bool f64 = std::is_same<TV, double>::value;
    Level &L0 = h->lv[0];
    VLevel<VT, TV> V0 = view<VT, TV>(L0);
    const int64_t n = L0.n();
    const int npre = h->prm.npre;
    const bool multi = h->lv.size() > 1;
    const Geom &g = h->geom;
    const TV *f0 = f64 ? (const TV *)h->r : (const TV *)h->rv;
    TV *z0 = f64 ? (TV *)h->z : (TV *)h->zv;
    TV *rv = f64 ? nullptr : (TV *)h->rv;
    // z = V(r), partial r.z
    int rz_np = 0;
    AMG_TRY((record_vcycle<VT, TV>(h, f0, z0, h->partials, s, &rz_np)));
    if (rz_np < 1) {
        set_error("the V-cycle left no partial sums of r.z");
        return AMG_ERR_STATE;
    }
    cg_beta_kernel<<<1, FIN_THREADS, 0, s>>>(h->st, h->partials, rz_np); ::amg::count_launch(1);
    cg_direction_kernel<TV><<<vgrid(h, n), 256, 0, s>>>(z0, h->p, h->st, n); ::amg::count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    int grid = 0;
    {  // q = A p, partial p.q (FP64 in every precision form: the CG's attainable
       // accuracy follows the error of A p relative to |A| |p|)
        SellArgs<double> a{};
        a.x = h->p;
        a.y = h->q;
        a.partials = h->partials;
        a.stop = &h->st->stop;
        AMG_TRY((launch_sell<double, double>(L0.sA, SPMV_PLAIN, DOT_XY, a, g, s, &grid)));
    }
    cg_alpha_kernel<<<1, FIN_THREADS, 0, s>>>(h->st, h->partials, grid); ::amg::count_launch(1);
    const bool blocks = blocks_ptr<TV>(h, 0) != nullptr && multi && npre > 0;
    // the next pre-smoothing M r fused into the update (ILU(0) smooths inside the V-cycle)
    const bool fuse_pre = multi && !blocks && !(h->ilu && npre > 0);
    cg_update_kernel<TV><<<vgrid(h, n), 256, 0, s>>>(h->uu, h->r, h->p, h->q, V0.M,
                                                     fuse_pre ? V0.u : nullptr, rv, h->st,
                                                     n, npre > 0, h->partials); ::amg::count_launch(1);
    cg_resnorm_kernel<<<1, FIN_THREADS, 0, s>>>(h->st, h->partials, vgrid(h, n)); ::amg::count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    {  // true residual, only when the recurrence residual reached tol: every
       // other iteration the launch exits at once, so a small grid (4 CTAs
       // per SM, warp-strided over the slices) keeps that cheap
        SellArgs<double> a{};
        a.x = h->uu;
        a.f = h->ff;
        a.y = h->rt;
        a.partials = h->partials;
        a.stop = &h->st->no_check;
        AMG_TRY((launch_sell<double, double>(L0.sA, SPMV_RESID, DOT_YY, a, g, s, &grid,
                                             g.num_sms * 4)));
    }
    cg_decide_kernel<<<1, FIN_THREADS, 0, s>>>(h->st, h->partials, grid, cond, use_cond); ::amg::count_launch(1);
    cg_replace_kernel<TV><<<vgrid(h, n), 256, 0, s>>>(h->r, h->rt, V0.M,
                                                      fuse_pre ? V0.u : nullptr, rv, h->st,
                                                      n, npre > 0); ::amg::count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    if (blocks)  // next pre-smoothing with the level-0 blocks: u0 = Mb r
        AMG_TRY(launch_block_apply<TV>(blocks_ptr<TV>(h, 0), f0, V0.u, L0.A.nbr, g, s));
    return AMG_OK;
}

static int record_cg_iteration(amg_handle h, cudaStream_t s, cudaGraphConditionalHandle cond,
                               int use_cond)
{
    switch (h->prm.precision) {
    case AMG_PREC_FP32: return record_cg_iteration_t<float, float>(h, s, cond, use_cond);
    case AMG_PREC_DF64: return record_cg_iteration_t<df32, double>(h, s, cond, use_cond);
    case AMG_PREC_BF16: return record_cg_iteration_t<__nv_bfloat16, float>(h, s, cond, use_cond);
    default: return record_cg_iteration_t<double, double>(h, s, cond, use_cond);
    }
}

template <class TV>
static int launch_vec_dot(amg_handle h, const TV *x, const TV *y, int64_t n, double *part,
                          cudaStream_t s, int *grid_out)
{
    const int grid = vgrid(h, n);
    vec_dot_kernel<TV><<<grid, 256, 0, s>>>(x, y, n, part); ::amg::count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    if (grid_out) *grid_out = grid;
    return AMG_OK;
}

// Host-loop variant: the same iteration captured as a plain graph.
static int build_step_graph(amg_handle h)
{
    if (h->exec) return AMG_OK;
    cudaStream_t cs;
    AMG_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    AMG_TRY_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    long long nbody = 0;
    begin_launch_capture(&nbody);
    cudaGraphConditionalHandle none = 0;
    int st = record_cg_iteration(h, cs, none, 0);
    end_launch_capture();
    h->body_kernels = nbody;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (st < 0) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) {
        set_error("graph capture: %s", cudaGetErrorString(e));
        return AMG_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&h->exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        h->exec = nullptr;
        set_error("graph instantiate: %s", cudaGetErrorString(e));
        return AMG_ERR_CUDA;
    }
    h->graph = graph;
    return AMG_OK;
}

static int build_graph(amg_handle h)
{
    if (h->prm.loop_mode == 1) return build_step_graph(h);
    if (h->exec) return AMG_OK;
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
    int st = record_cg_iteration(h, cs, cond, 1);
    end_launch_capture();
    h->body_kernels = nbody;
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &captured);
    cudaStreamDestroy(cs);
    if (st < 0) {
        cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        set_error("graph capture: %s", cudaGetErrorString(e));
        return AMG_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&h->exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        h->exec = nullptr;
        set_error("graph instantiate: %s", cudaGetErrorString(e));
        return AMG_ERR_CUDA;
    }
    h->graph = graph;
    return AMG_OK;
}

// ---------------------------------------------------------------- C ABI
extern "C" {

int amg_params_default(amg_params *prm)
{
    if (!prm) return AMG_ERR_ARG;
    std::memset(prm, 0, sizeof *prm);
    prm->eps_strong = 0.08;
    prm->relax = 2.0;
    prm->smooth_relax = 0.8;
    prm->coarse_enough = 3000;
    prm->max_levels = 15;
    prm->npre = 1;
    prm->npost = 1;
    prm->precision = AMG_PREC_FP64;
    prm->ilu_sweeps = 2;
    return AMG_OK;
}

const char *amg_last_error(void) { return amg::last_error(); }

}  // extern "C"

void amg::destroy_handle(amg_handle h)
{
    if (!h) return;
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->mem.has_custom()) {
        // the caller's supplier may hand the buffers to work on any stream:
        // nothing of this handle may still be queued when they go back
        cudaDeviceSynchronize();
        h->mem.release_all();
    } else {
        h->mem.release_all();
        if (h->stream) cudaStreamSynchronize(h->stream);
        else cudaDeviceSynchronize();
    }
    if (h->st_h) cudaFreeHost(h->st_h);
    delete h;
}

// Input pattern check, one thread per block row: bad[0] |= 1 (row pointers),
// 2 (columns not ascending or out of range), 4 (no diagonal block), 8 (the
// pattern is not symmetric: block (I, J) without (J, I); A is SPD, and the
// Galerkin products rely on it); bad[1] = the lowest offending row.  Rows are
// first checked on their own (codes 1, 2, 4); only a fully valid pattern is
// searched for the transposed blocks, so no search reads a bad row.
// bad[0] |= 16 if any of the n values is NaN or infinite
__global__ void finite_check_kernel(const double *__restrict__ v, int64_t n, int *__restrict__ bad)
{
    int nonfinite = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        nonfinite |= !isfinite(v[i]);
    if (__any_sync(0xffffffffu, nonfinite) && (threadIdx.x & 31) == 0) atomicOr(bad, 16);
}

__global__ void validate_symmetry_kernel(const int *__restrict__ rp, const int *__restrict__ col,
                                         int nbr, int *__restrict__ bad)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nbr || bad[0] != 0) return;
    for (int k = rp[I]; k < rp[I + 1]; ++k) {
        const int J = col[k];
        int lo = rp[J], hi = rp[J + 1];
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (col[mid] < I) lo = mid + 1;
            else hi = mid;
        }
        if (lo >= rp[J + 1] || col[lo] != I) {
            atomicOr(bad + 2, 8);
            atomicMin(bad + 1, I);
            return;
        }
    }
}

__global__ void validate_pattern_kernel(const int *__restrict__ rp, const int *__restrict__ col,
                                        int nbr, int nbc, int64_t nnzb, int *__restrict__ bad)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nbr) return;
    const int64_t a = rp[I], b = rp[I + 1];
    int code = 0;
    if (a < 0 || b < a || b > nnzb || (I == 0 && a != 0) || (I == nbr - 1 && b != nnzb)) {
        code = 1;
    } else {
        bool diag = false;
        for (int64_t k = a; k < b; ++k) {
            const int c = col[k];
            if (c < 0 || c >= nbc || (k > a && c <= col[k - 1])) {
                code = 2;
                break;
            }
            diag |= c == I;
        }
        if (!code && !diag) code = 4;
    }
    if (code) {
        atomicOr(bad, code);
        atomicMin(bad + 1, I);
    }
}

// Stop rule of the coarsening loop after level `nlev - 1` (n rows, nn nodes)
// was aggregated into nagg aggregates: no aggregates, or too few nodes
// merged (aggregates >= 0.9 x nodes); and a level below the finest that is
// already small (at most 2 coarse_enough rows) stays the coarsest rather
// than being coarsened into a tiny level (fewer than coarse_enough / 4 rows,
// aggregated from a dense operator: such a last step doubles the CG
// iterations or worse on these meshes).
static bool stop_coarsening(const amg_params &prm, int nlev, int64_t n, int nn, int nagg, int ns)
{
    if (nagg == 0 || (double)nagg >= 0.9 * (double)nn) return true;
    return nlev > 1 && n <= 2 * (int64_t)prm.coarse_enough &&
           4 * (int64_t)nagg * ns < (int64_t)prm.coarse_enough;
}

// Alg. 1 in scalar arithmetic (AMG_SETUP_SCALAR): level 0 unblocked, then
// per level the node graph's strength, aggregation (host greedy passes or
// device MIS-2 on the node graph), the scalar transfer operators, the scalar
// Galerkin product and SPAI0; the coarsest scalar matrix is factored; last,
// every level is converted into blocks (level 0 keeps the input blocks).
// The scalar matrices stay in L.xA, L.xP, L.xR for the solve copies.
template <class Lap>
static int setup_levels_scalar(amg_handle h, DevArena &tmp, Lap &lap)
{
    cudaStream_t s = h->stream;
    const amg_params &prm = h->prm;
    AMG_TRY(unblock_bsr(h->lv[0].A, h->mem, s, &h->lv[0].xA));
    lap(0);
    for (;;) {
        Level &C = h->lv.back();
        const int b = h->lv.size() == 1 ? 3 : h->ns;
        const BsrD &S = C.xA;
        const int n = S.nbr, nn = n / b;
        if (n <= prm.coarse_enough || (int)h->lv.size() >= prm.max_levels) break;
        BsrD G;
        AMG_TRY(scalar_strength(S, b, C.eps, h->mem, tmp, s, &G, &C.strong));
        std::vector<int> agg(std::max(nn, 1));
        int nagg = 0;
        if (prm.aggregation == AMG_AGG_MIS2) {
            int *dagg = nullptr;
            AMG_TRY(tmp.alloc_n(&dagg, (size_t)nn));
            AMG_TRY(aggregate_mis2(G, C.strong, dagg, &nagg, nullptr, tmp, s));
            AMG_TRY_CUDA(cudaMemcpyAsync(agg.data(), dagg, sizeof(int) * nn,
                                         cudaMemcpyDeviceToHost, s));
            AMG_TRY_CUDA(cudaStreamSynchronize(s));
            tmp.release(dagg);
        } else {
            HostStrongGraph hg;
            AMG_TRY(strong_graph_to_host(G, C.strong, tmp, s, &hg));
            AMG_TRY(aggregate_host(nn, hg.srp.get(), hg.scol.get(), agg.data(), &nagg));
        }
        h->mem.release(G.row_ptr);
        h->mem.release(G.col);
        lap(1);
        if (stop_coarsening(prm, (int)h->lv.size(), n, nn, nagg, h->ns)) break;
        LevelBuild lb;
        AMG_TRY(scalar_transfer(S, b, C.B, h->ns, agg.data(), nagg, prm.relax, h->mem, tmp, s,
                                &lb));
        lap(2);
        C.xP = lb.P;
        C.xR = lb.R;
        C.agg = lb.agg;
        C.nagg = nagg;
        C.omega = lb.omega;
        C.rho = lb.rho;
        Level N;
        AMG_TRY(galerkin(S, C.xP, C.xR, h->mem, tmp, s, &N.xA));
        lap(3);
        N.B = lb.Bc;
        N.eps = C.eps * 0.5;
        AMG_TRY(h->mem.alloc_n(&C.M, (size_t)std::max(n, 1)));
        AMG_TRY(spai0_diag(S, prm.smooth_relax, C.M, s));
        lap(4);
        h->lv.push_back(N);
    }
    Level &Cc = h->lv.back();
    Cc.coarsest = true;
    AMG_TRY(coarse_inverse(Cc.xA, h->mem, tmp, s, &h->Ainv));
    h->nc = Cc.xA.nbr;
    lap(5);
    for (size_t l = 0; l < h->lv.size(); ++l) {
        Level &L = h->lv[l];
        const int b = l == 0 ? 3 : h->ns;
        if (l > 0) AMG_TRY(scalar_to_block(L.xA, b, b, h->mem, tmp, s, &L.A));
        if (!L.coarsest) {
            AMG_TRY(scalar_to_block(L.xP, b, h->ns, h->mem, tmp, s, &L.P));
            AMG_TRY(scalar_to_block(L.xR, h->ns, b, h->mem, tmp, s, &L.R));
        }
    }
    return AMG_OK;
}

int amg::setup_impl(amg_handle h, const amg_bsr *Ain, const double *B)
{
    cudaStream_t s = h->stream;
    const amg_params &prm = h->prm;
    DevArena tmp;
    tmp.stream = s;
    struct TmpGuard {
        DevArena &t;
        ~TmpGuard() { t.release_all(); }
    } guard{tmp};
    AMG_TRY(query_geom(&h->geom));
    // wall time per setup phase (each lap ends with the stream synchronised)
    auto tp = std::chrono::steady_clock::now();
    auto lap = [&](int k) {
        cudaStreamSynchronize(s);
        const auto t = std::chrono::steady_clock::now();
        h->setup_phase[k] += std::chrono::duration<double>(t - tp).count();
        tp = t;
    };
    {  // level 0: own copy of A and B
        Level L0;
        BsrD &A = L0.A;
        A.nbr = Ain->nbrows;
        A.nbc = Ain->nbcols;
        A.br = Ain->bs_r;
        A.bc = Ain->bs_c;
        A.nnzb = Ain->nnzb;
        AMG_TRY(h->mem.alloc_n(&A.row_ptr, (size_t)A.nbr + 1));
        AMG_TRY(h->mem.alloc_n(&A.col, (size_t)std::max<int64_t>(A.nnzb, 1)));
        AMG_TRY(h->mem.alloc_n(&A.val, (size_t)std::max<int64_t>(A.nnzb, 1) * 9));
        AMG_TRY(h->mem.alloc_n(&L0.B, (size_t)A.nbr * 3 * h->ns));
        AMG_TRY_CUDA(cudaMemcpyAsync(A.row_ptr, Ain->row_ptr, sizeof(int) * (A.nbr + 1),
                                     cudaMemcpyDeviceToDevice, s));
        AMG_TRY_CUDA(cudaMemcpyAsync(A.col, Ain->col, sizeof(int) * A.nnzb,
                                     cudaMemcpyDeviceToDevice, s));
        AMG_TRY_CUDA(cudaMemcpyAsync(A.val, Ain->val, sizeof(double) * 9 * A.nnzb,
                                     cudaMemcpyDeviceToDevice, s));
        AMG_TRY_CUDA(cudaMemcpyAsync(L0.B, B, sizeof(double) * 3 * h->ns * A.nbr,
                                     cudaMemcpyDeviceToDevice, s));
        L0.eps = prm.eps_strong;
        // validate the pattern before any other kernel indexes with it: the
        // checking kernel reads a row's columns only after its own row
        // pointers were found inside [0, nnzb]
        int *bad = nullptr;
        AMG_TRY(tmp.alloc_n(&bad, 3));
        const int init[3] = {0, INT32_MAX, 0};
        AMG_TRY_CUDA(cudaMemcpyAsync(bad, init, sizeof(init), cudaMemcpyHostToDevice, s));
        if (A.nbr > 0) {
            validate_pattern_kernel<<<(A.nbr + 255) / 256, 256, 0, s>>>(A.row_ptr, A.col, A.nbr,
                                                                        A.nbc, A.nnzb, bad);
            // square matrices only reach here (nbc == nbr); runs only when
            // every row passed (each thread reads bad[0] first)
            validate_symmetry_kernel<<<(A.nbr + 255) / 256, 256, 0, s>>>(A.row_ptr, A.col, A.nbr,
                                                                         bad);
            ::amg::count_launch(2);
            AMG_TRY_CUDA(cudaGetLastError());
        }
        {  // non-finite values in A or B
            const int64_t nv = A.nnzb * 9, nb = (int64_t)A.nbr * 3 * h->ns;
            const int g1 = (int)std::min<int64_t>((nv + 255) / 256, h->geom.max_ctas);
            const int g2 = (int)std::min<int64_t>((nb + 255) / 256, h->geom.max_ctas);
            if (nv > 0) finite_check_kernel<<<g1, 256, 0, s>>>(A.val, nv, bad + 2);
            if (nb > 0) finite_check_kernel<<<g2, 256, 0, s>>>(L0.B, nb, bad + 2);
            ::amg::count_launch((nv > 0) + (nb > 0));
            AMG_TRY_CUDA(cudaGetLastError());
        }
        int hb[3] = {0, 0, 0};
        AMG_TRY_CUDA(cudaMemcpyAsync(hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, s));
        AMG_TRY_CUDA(cudaStreamSynchronize(s));
        tmp.release(bad);
        if (hb[0] & 1) {
            set_error("row_ptr must start at 0, end at nnzb and not decrease (block row %d)", hb[1]);
            return AMG_ERR_ARG;
        }
        if (hb[0] & 2) {
            set_error("block row %d: columns must be ascending and in range", hb[1]);
            return AMG_ERR_ARG;
        }
        if (hb[0] & 4) {
            set_error("block row %d has no diagonal block", hb[1]);
            return AMG_ERR_ARG;
        }
        if (hb[2] & 8) {
            set_error("the block pattern is not symmetric (block row %d)", hb[1]);
            return AMG_ERR_ARG;
        }
        if (hb[2] & 16) {
            set_error("A or B holds a non-finite value");
            return AMG_ERR_ARG;
        }
        h->lv.push_back(L0);
    }
    lap(0);
    if (prm.setup == AMG_SETUP_SCALAR) {
        AMG_TRY(setup_levels_scalar(h, tmp, lap));
    } else for (;;) {
        Level &C = h->lv.back();
        const int nn = C.A.nbr, n = C.n();
        if (n <= prm.coarse_enough || (int)h->lv.size() >= prm.max_levels) break;
        AMG_TRY(h->mem.alloc_n(&C.strong, (size_t)std::max<int64_t>(C.A.nnzb, 1)));
        AMG_TRY(compute_strength(C.A, C.eps, C.strong, s));
        std::vector<int> agg(std::max(nn, 1));
        int nagg = 0;
        if (prm.aggregation == AMG_AGG_MIS2) {
            // parallel aggregation on the device; only the map comes back
            int *dagg = nullptr;
            AMG_TRY(tmp.alloc_n(&dagg, (size_t)nn));
            AMG_TRY(aggregate_mis2(C.A, C.strong, dagg, &nagg, nullptr, tmp, s));
            AMG_TRY_CUDA(cudaMemcpyAsync(agg.data(), dagg, sizeof(int) * nn,
                                         cudaMemcpyDeviceToHost, s));
            AMG_TRY_CUDA(cudaStreamSynchronize(s));
            tmp.release(dagg);
        } else {
            HostStrongGraph hg;
            AMG_TRY(strong_graph_to_host(C.A, C.strong, tmp, s, &hg));
            AMG_TRY(aggregate_host(nn, hg.srp.get(), hg.scol.get(), agg.data(), &nagg));
        }
        lap(1);
        if (stop_coarsening(prm, (int)h->lv.size(), n, nn, nagg, h->ns)) break;
        LevelBuild lb;
        AMG_TRY(build_transfer(C.A, C.B, h->ns, C.strong, agg.data(), nagg, prm.relax, h->mem, tmp, s,
                               &lb));
        lap(2);
        C.P = lb.P;
        C.R = lb.R;
        C.agg = lb.agg;
        C.nagg = nagg;
        C.omega = lb.omega;
        C.rho = lb.rho;
        Level N;
        AMG_TRY(galerkin(C.A, C.P, C.R, h->mem, tmp, s, &N.A));
        lap(3);
        N.B = lb.Bc;
        N.eps = C.eps * 0.5;
        AMG_TRY(h->mem.alloc_n(&C.M, (size_t)std::max(n, 1)));
        AMG_TRY(spai0_diag(C.A, prm.smooth_relax, C.M, s));
        lap(4);
        h->lv.push_back(N);
    }
    if (prm.setup != AMG_SETUP_SCALAR) {
        Level &Cc = h->lv.back();
        Cc.coarsest = true;
        AMG_TRY(coarse_inverse(Cc.A, h->mem, tmp, s, &h->Ainv));
        h->nc = Cc.n();
        lap(5);
    }
    if (prm.smoother == AMG_SMOOTH_ILU0) {  // block ILU(0) of every smoothing level
        for (size_t l = 0; l + 1 < h->lv.size(); ++l)
            AMG_TRY(ilu0_factor(h->lv[l].A, h->max_lanes, h->mem, tmp, s, &h->lv[l].ilu));
        h->ilu = 1;
        lap(4);
    }
    // V-cycle operators in the sliced layout, in the V-cycle's precision; the
    // fine A is also kept in FP64 for the CG products.
    const int prec = prm.precision;
    const bool scalar = prm.storage == AMG_STORAGE_SCALAR;
    for (size_t l = 0; l < h->lv.size(); ++l) {
        Level &L = h->lv[l];
        const bool vc = !L.coarsest;
        // the operators as stored for the solve: the block BSR itself, or its
        // scalar unblocking (temporary; only the sliced copies are kept)
        BsrD uA, uP, uR;
        const BsrD *oA = &L.A, *oP = &L.P, *oR = &L.R;
        if (scalar && L.xA.row_ptr) {  // the scalar setup's own matrices
            oA = &L.xA;
            if (vc) {
                oP = &L.xP;
                oR = &L.xR;
            }
        } else if (scalar) {
            if (l == 0 || vc) {
                AMG_TRY(unblock_bsr(L.A, tmp, s, &uA));
                oA = &uA;
            }
            if (vc) {
                AMG_TRY(unblock_bsr(L.P, tmp, s, &uP));
                AMG_TRY(unblock_bsr(L.R, tmp, s, &uR));
                oP = &uP;
                oR = &uR;
            }
        }
        if (l == 0 || (vc && prec == AMG_PREC_FP64))
            AMG_TRY(bsr_to_sell<double>(*oA, h->mem, s, &L.sA, &L.pad_A, h->max_lanes));
        if (vc && prec == AMG_PREC_FP64) {
            AMG_TRY(bsr_to_sell<double>(*oP, h->mem, s, &L.sP, &L.pad_P, h->max_lanes));
            AMG_TRY(bsr_to_sell<double>(*oR, h->mem, s, &L.sR, &L.pad_R, h->max_lanes));
        }
        if (prec == AMG_PREC_DF64 && (l == 0 || vc))
            AMG_TRY(bsr_to_sell<df32>(*oA, h->mem, s, &L.eA, &L.pad_A, h->max_lanes));
        if (vc && prec == AMG_PREC_DF64) {
            AMG_TRY(bsr_to_sell<df32>(*oP, h->mem, s, &L.eP, &L.pad_P, h->max_lanes));
            AMG_TRY(bsr_to_sell<df32>(*oR, h->mem, s, &L.eR, &L.pad_R, h->max_lanes));
        }
        if (vc && prec == AMG_PREC_FP32) {
            AMG_TRY(bsr_to_sell<float>(*oA, h->mem, s, &L.fA, &L.pad_A, h->max_lanes));
            AMG_TRY(bsr_to_sell<float>(*oP, h->mem, s, &L.fP, &L.pad_P, h->max_lanes));
            AMG_TRY(bsr_to_sell<float>(*oR, h->mem, s, &L.fR, &L.pad_R, h->max_lanes));
        }
        if (vc && prec == AMG_PREC_BF16) {
            AMG_TRY(bsr_to_sell<__nv_bfloat16>(*oA, h->mem, s, &L.bA, &L.pad_A, h->max_lanes));
            AMG_TRY(bsr_to_sell<__nv_bfloat16>(*oP, h->mem, s, &L.bP, &L.pad_P, h->max_lanes));
            AMG_TRY(bsr_to_sell<__nv_bfloat16>(*oR, h->mem, s, &L.bR, &L.pad_R, h->max_lanes));
        }
        if (scalar) {
            AMG_TRY_CUDA(cudaStreamSynchronize(s));
            for (BsrD *u : {&uA, &uP, &uR}) {
                if (u->row_ptr) tmp.release(u->row_ptr);
                if (u->col) tmp.release(u->col);
                if (u->val) tmp.release(u->val);
            }
        }
    }
    if (prm.smoother == AMG_SMOOTH_BJACOBI) {  // block damped Jacobi of every smoothing level
        lap(6);                                // (its power iteration uses the sliced copies)
        AMG_TRY(bjacobi_setup(h, tmp, s));
        lap(4);
    }
    // the scalar setup's matrices are not kept past the solve copies
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    for (Level &L : h->lv)
        for (BsrD *x : {&L.xA, &L.xP, &L.xR}) {
            h->mem.release(x->row_ptr);
            h->mem.release(x->col);
            h->mem.release(x->val);
            *x = BsrD();
        }
    for (size_t l = 0; l < h->lv.size(); ++l) {
        Level &L = h->lv[l];
        const size_t n = (size_t)std::max(L.n(), 1);
        if (prec == AMG_PREC_FP64 || prec == AMG_PREC_DF64) {
            if (l > 0) AMG_TRY(h->mem.alloc_n(&L.f, n));
            AMG_TRY(h->mem.alloc_n(&L.u, n));
            AMG_TRY(h->mem.alloc_n(&L.e, n));
            AMG_TRY(h->mem.alloc_n(&L.z, n));
            AMG_TRY(h->mem.alloc_n(&L.t, n));
        } else {
            if (l > 0) AMG_TRY(h->mem.alloc_n(&L.vf, n));
            AMG_TRY(h->mem.alloc_n(&L.vu, n));
            AMG_TRY(h->mem.alloc_n(&L.ve, n));
            AMG_TRY(h->mem.alloc_n(&L.vz, n));
            AMG_TRY(h->mem.alloc_n(&L.vt, n));
            if (L.M) {
                AMG_TRY(h->mem.alloc_n(&L.Mf, n));
                narrow_kernel<<<vgrid(h, L.n()), 256, 0, s>>>(L.M, L.Mf, L.n());
                count_launch(1);
                AMG_TRY_CUDA(cudaGetLastError());
            }
        }
    }
    if (prec == AMG_PREC_FP32 || prec == AMG_PREC_BF16) {
        const size_t n0 = (size_t)std::max(h->lv[0].n(), 1);
        AMG_TRY(h->mem.alloc_n(&h->rv, n0));
        AMG_TRY(h->mem.alloc_n(&h->zv, n0));
    }
    const size_t n0 = (size_t)std::max(h->lv[0].n(), 1);
    AMG_TRY(h->mem.alloc_n(&h->ff, n0));
    AMG_TRY(h->mem.alloc_n(&h->uu, n0));
    AMG_TRY(h->mem.alloc_n(&h->r, n0));
    AMG_TRY(h->mem.alloc_n(&h->p, n0));
    AMG_TRY(h->mem.alloc_n(&h->q, n0));
    AMG_TRY(h->mem.alloc_n(&h->z, n0));
    AMG_TRY(h->mem.alloc_n(&h->rt, n0));
    AMG_TRY(h->mem.alloc_n(&h->partials,
                           (size_t)std::max(h->geom.max_ctas, h->geom.max_partials) + 1));
    AMG_TRY(h->mem.alloc_n(&h->scal, 8));
    AMG_TRY(h->mem.alloc_n(&h->st, 1));
    AMG_TRY_CUDA(cudaMallocHost((void **)&h->st_h, sizeof(CgState)));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    lap(6);
    return AMG_OK;
}

extern "C" {

int amg_setup(const amg_bsr *A, const double *B, int32_t nb_ns, const amg_params *prm,
              void *stream, amg_handle *out)
{
    clear_error();
    if (!out) {
        set_error("null output handle");
        return AMG_ERR_ARG;
    }
    *out = nullptr;
    AMG_TRY(check_bsr(A, 1));
    if (A->bs_r != 3 || A->nbrows < 1) {
        set_error("amg_setup expects a non-empty 3x3 block matrix");
        return AMG_ERR_ARG;
    }
    if ((nb_ns != 6 && nb_ns != 3) || !B) {
        set_error("amg_setup expects the six rigid-body modes (nb_ns = 6) or three translations (3)");
        return AMG_ERR_ARG;
    }
    amg_params p;
    amg_params_default(&p);
    if (prm) p = *prm;
    if (p.npre < 0 || p.npost < 0 || p.max_levels < 1 || p.coarse_enough < 0 ||
        !(p.eps_strong >= 0.0) || p.precision < AMG_PREC_FP64 || p.precision > AMG_PREC_DF64 ||
        p.loop_mode < 0 || p.loop_mode > 1 || p.storage < AMG_STORAGE_BLOCK ||
        p.storage > AMG_STORAGE_SCALAR || p.aggregation < AMG_AGG_GREEDY ||
        p.aggregation > AMG_AGG_MIS2 || p.smoother < AMG_SMOOTH_SPAI0 ||
        p.smoother > AMG_SMOOTH_BJACOBI || p.ilu_sweeps < 0 || p.ilu_sweeps > 64 ||
        p.setup < AMG_SETUP_BLOCK || p.setup > AMG_SETUP_SCALAR || p.reserved != 0) {
        set_error("bad parameters");
        return AMG_ERR_ARG;
    }
    if (p.setup == AMG_SETUP_SCALAR && p.smoother != AMG_SMOOTH_SPAI0) {
        set_error("the scalar setup builds the SPAI0 smoother");
        return AMG_ERR_ARG;
    }
    if (p.smoother == AMG_SMOOTH_ILU0 &&
        (p.precision != AMG_PREC_FP64 || p.storage != AMG_STORAGE_BLOCK)) {
        set_error("the ILU(0) smoother runs in the FP64 V-cycle with block storage");
        return AMG_ERR_ARG;
    }
    if (p.smoother == AMG_SMOOTH_BJACOBI &&
        (p.storage != AMG_STORAGE_BLOCK || !(p.smooth_relax > 0.0))) {
        set_error("the block Jacobi smoother needs block storage and smooth_relax > 0");
        return AMG_ERR_ARG;
    }
    auto t0 = std::chrono::steady_clock::now();
    amg_handle h = new amg_handle_s();
    h->prm = p;
    if (p.allocator) {
        if (!p.allocator->alloc || !p.allocator->free) {
            delete h;
            set_error("amg_params.allocator needs both alloc and free");
            return AMG_ERR_ARG;
        }
        h->alloc = *p.allocator;
    }
    h->prm.allocator = nullptr;  // the caller's struct is not kept; h->alloc is the copy
    h->ns = nb_ns;
    h->stream = (cudaStream_t)stream;
    h->mem.stream = h->stream;
    AllocScope scope(h->allocator());
    int st = no_throw([&] { return setup_impl(h, A, B); });
    if (st < 0) {
        std::string msg = amg::last_error();
        destroy_handle(h);
        set_error("%s", msg.c_str());
        return st;
    }
    h->setup_seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return AMG_OK;
}

void amg_free(amg_handle h) { destroy_handle(h); }

int amg_apply_vcycle(amg_handle h, const double *r, double *z, void *stream)
{
    clear_error();
    if (!h || !r || !z) {
        set_error("null argument");
        return AMG_ERR_ARG;
    }
    AllocScope scope(h->allocator());
    cudaStream_t s = (cudaStream_t)stream;
    Level &L0 = h->lv[0];
    const int64_t n = L0.n();
    const bool multi = h->lv.size() > 1;
    const int zero = h->prm.npre == 0;
    if (h->prm.precision == AMG_PREC_FP64 || h->prm.precision == AMG_PREC_DF64) {
        if (multi && blocks_ptr<double>(h, 0) && !zero) {
            AMG_TRY(launch_block_apply(L0.Mb, r, L0.u, L0.A.nbr, h->geom, s));
        } else if (multi && !(h->ilu && !zero)) {  // ILU(0) pre-smooths inside the V-cycle
            scale_kernel<double><<<vgrid(h, n), 256, 0, s>>>(L0.M, r, L0.u, nullptr, n, zero);
            count_launch(1);
            AMG_TRY_CUDA(cudaGetLastError());
        }
        if (h->prm.precision == AMG_PREC_DF64) return record_vcycle<df32, double>(h, r, z, nullptr, s);
        return record_vcycle<double, double>(h, r, z, nullptr, s);
    }
    const bool lb = multi && blocks_ptr<float>(h, 0) && !zero;
    scale_kernel<float><<<vgrid(h, n), 256, 0, s>>>(L0.Mf, r, (multi && !lb) ? L0.vu : nullptr,
                                                    h->rv, n, zero);
    count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    if (lb) AMG_TRY(launch_block_apply<float>(L0.Mbf, h->rv, L0.vu, L0.A.nbr, h->geom, s));
    if (h->prm.precision == AMG_PREC_FP32)
        AMG_TRY((record_vcycle<float, float>(h, h->rv, h->zv, nullptr, s)));
    else
        AMG_TRY((record_vcycle<__nv_bfloat16, float>(h, h->rv, h->zv, nullptr, s)));
    widen_kernel<float><<<vgrid(h, n), 256, 0, s>>>(h->zv, z, n);
    count_launch(1);
    AMG_TRY_CUDA(cudaGetLastError());
    return AMG_OK;
}

int amg_solve(amg_handle h, const double *f, double *u, double tol, int32_t maxiter,
              int32_t *iters, double *rel_resid, void *stream)
{
    clear_error();
    if (!h || !f || !u) {
        set_error("null argument");
        return AMG_ERR_ARG;
    }
    if (!(tol > 0.0) || maxiter < 0 || maxiter > 1000000) {
        set_error("bad tolerance or iteration limit");
        return AMG_ERR_ARG;
    }
    AllocScope scope(h->allocator());
    cudaStream_t s = (cudaStream_t)stream;
    Level &L0 = h->lv[0];
    const int64_t n = L0.n();
    const bool multi = h->lv.size() > 1;
    AMG_TRY_CUDA(cudaMemcpyAsync(h->ff, f, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    AMG_TRY_CUDA(cudaMemcpyAsync(h->uu, u, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    vec_dot_kernel<double><<<vgrid(h, n), 256, 0, s>>>(h->ff, h->ff, n, h->partials); ::amg::count_launch(1);
    AMG_TRY(launch_reduce_sum(h->partials, vgrid(h, n), h->scal, s));
    int grid = 0;
    {
        SellArgs<double> a{};
        a.x = h->uu;
        a.f = h->ff;
        a.y = h->r;
        a.partials = h->partials;
        AMG_TRY((launch_sell<double, double>(L0.sA, SPMV_RESID, DOT_YY, a, h->geom, s, &grid)));
    }
    AMG_TRY(launch_reduce_sum(h->partials, grid, h->scal + 1, s));
    cg_start_kernel<<<1, 1, 0, s>>>(h->st, h->scal, tol, maxiter); ::amg::count_launch(1);
    if (h->prm.precision == AMG_PREC_FP64 || h->prm.precision == AMG_PREC_DF64) {
        if (multi && blocks_ptr<double>(h, 0) && h->prm.npre > 0) {
            AMG_TRY(launch_block_apply(L0.Mb, h->r, L0.u, L0.A.nbr, h->geom, s));
        } else if (multi && !(h->ilu && h->prm.npre > 0)) {  // ILU(0) pre-smooths in the V-cycle
            scale_kernel<double><<<vgrid(h, n), 256, 0, s>>>(L0.M, h->r, L0.u, nullptr, n,
                                                             h->prm.npre == 0);
            count_launch(1);
        }
    } else {
        const bool lb = multi && blocks_ptr<float>(h, 0) && h->prm.npre > 0;
        scale_kernel<float><<<vgrid(h, n), 256, 0, s>>>(L0.Mf, h->r,
                                                        (multi && !lb) ? L0.vu : nullptr, h->rv,
                                                        n, h->prm.npre == 0);
        count_launch(1);
        if (lb) AMG_TRY(launch_block_apply<float>(L0.Mbf, h->rv, L0.vu, L0.A.nbr, h->geom, s));
    }
    AMG_TRY_CUDA(cudaGetLastError());
    AMG_TRY_CUDA(cudaMemcpyAsync(h->st_h, h->st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    int status;
    if (!std::isfinite(h->st_h->nf) || !std::isfinite(h->st_h->res)) {
        set_error("f or the initial guess u holds a non-finite value");
        return AMG_ERR_ARG;
    }
    if (h->st_h->nf == 0.0) {
        AMG_TRY_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * n, s));
        AMG_TRY_CUDA(cudaStreamSynchronize(s));
        if (iters) *iters = 0;
        if (rel_resid) *rel_resid = 0.0;
        return AMG_OK;
    }
    if (h->st_h->res <= tol || maxiter == 0) {
        if (iters) *iters = 0;
        if (rel_resid) *rel_resid = h->st_h->res;
        return h->st_h->res <= tol ? AMG_OK : AMG_NOT_CONVERGED;
    }
    AMG_TRY(build_graph(h));
    if (h->prm.loop_mode == 1) {
        // one graph launch per CG step; the state is polled every 8 steps and
        // the kernels of steps launched after the stop return at once
        for (int it = 0; it < maxiter; it += 8) {
            for (int k = 0; k < 8 && it + k < maxiter; ++k)
                AMG_TRY_CUDA(cudaGraphLaunch(h->exec, s));
            AMG_TRY_CUDA(cudaMemcpyAsync(h->st_h, h->st, sizeof(CgState),
                                         cudaMemcpyDeviceToHost, s));
            AMG_TRY_CUDA(cudaStreamSynchronize(s));
            if (h->st_h->stop) break;
        }
    } else {
        AMG_TRY_CUDA(cudaGraphLaunch(h->exec, s));
    }
    AMG_TRY_CUDA(cudaMemcpyAsync(h->st_h, h->st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    status = h->st_h->status;
    count_launch(h->body_kernels * (long long)h->st_h->it);
    double res = h->st_h->res_true;
    if (status != AMG_OK) {  // report the true residual of the returned iterate
        SellArgs<double> a{};
        a.x = h->uu;
        a.f = h->ff;
        a.y = h->rt;
        a.partials = h->partials;
        AMG_TRY((launch_sell<double, double>(L0.sA, SPMV_RESID, DOT_YY, a, h->geom, s, &grid)));
        AMG_TRY(launch_reduce_sum(h->partials, grid, h->scal + 2, s));
        double rr = 0.0;
        AMG_TRY_CUDA(cudaMemcpyAsync(&rr, h->scal + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
        AMG_TRY_CUDA(cudaStreamSynchronize(s));
        res = std::sqrt(rr) / h->st_h->nf;
    }
    AMG_TRY_CUDA(cudaMemcpyAsync(u, h->uu, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    if (iters) *iters = h->st_h->it;
    if (rel_resid) *rel_resid = res;
    if (status == AMG_ERR_BREAKDOWN) set_error("CG breakdown at iteration %d", h->st_h->it);
    return status;
}

int amg_get_stats(amg_handle h, amg_stats *out)
{
    if (!h || !out) return AMG_ERR_ARG;
    std::memset(out, 0, sizeof *out);
    out->nlevels = (int)h->lv.size();
    out->coarse_n = h->nc;
    out->setup_seconds = h->setup_seconds;
    int64_t bytes = 0, nnz0 = 0, nnz = 0;
    auto bsr_bytes = [](const BsrD &m) -> int64_t {
        if (!m.row_ptr) return 0;
        return (int64_t)(m.nbr + 1) * 4 + m.nnzb * 4 + m.nnzb * m.br * m.bc * 8;
    };
    for (size_t l = 0; l < h->lv.size(); ++l) {
        const Level &L = h->lv[l];
        bytes += bsr_bytes(L.A) + bsr_bytes(L.P) + bsr_bytes(L.R);
        if (L.M) bytes += (int64_t)L.n() * 8;
        const int64_t z = L.A.nnzb * L.A.br * L.A.bc;
        if (l == 0) nnz0 = z;
        nnz += z;
    }
    bytes += (int64_t)h->nc * h->nc * 8;
    out->bytes_matrices = bytes;
    out->bytes_total = (int64_t)h->mem.bytes;
    out->operator_complexity = nnz0 ? (double)nnz / (double)nnz0 : 0.0;
    out->learned = h->learned;
    out->learned_lambda = h->learned_lambda;
    int64_t sb = 0;
    for (const Level &L : h->lv)
        sb += sell_bytes(L.sA) + sell_bytes(L.sP) + sell_bytes(L.sR) + sell_bytes(L.fA) +
              sell_bytes(L.fP) + sell_bytes(L.fR) + sell_bytes(L.bA) + sell_bytes(L.bP) +
              sell_bytes(L.bR) + sell_bytes(L.eA) + sell_bytes(L.eP) + sell_bytes(L.eR);
    out->bytes_solve = sb;
    for (int k = 0; k < 7; ++k) out->setup_phase_seconds[k] = h->setup_phase[k];
    out->spai0_lambda = h->spai0_lambda;
    return AMG_OK;
}

int amg_level_info(amg_handle h, int32_t level, amg_level_desc *out)
{
    if (!h || !out || level < 0 || level >= (int)h->lv.size()) {
        set_error("bad level");
        return AMG_ERR_ARG;
    }
    const Level &L = h->lv[level];
    std::memset(out, 0, sizeof *out);
    out->nbrows = L.A.nbr;
    out->bs = L.A.br;
    out->nnzb_A = L.A.nnzb;
    out->nnzb_P = L.P.nnzb;
    out->nagg = L.nagg;
    out->is_coarsest = L.coarsest;
    out->eps = L.eps;
    out->omega = L.omega;
    out->rho = L.rho;
    out->smoother_lambda = L.bj_lambda;
    return AMG_OK;
}

static int export_bsr(const BsrD &m, int32_t *rp, int32_t *cl, double *vl, cudaStream_t s)
{
    if (!m.row_ptr) {
        set_error("operator not present on this level");
        return AMG_ERR_STATE;
    }
    if (rp) AMG_TRY_CUDA(cudaMemcpyAsync(rp, m.row_ptr, sizeof(int) * (m.nbr + 1), cudaMemcpyDeviceToHost, s));
    if (cl) AMG_TRY_CUDA(cudaMemcpyAsync(cl, m.col, sizeof(int) * m.nnzb, cudaMemcpyDeviceToHost, s));
    if (vl)
        AMG_TRY_CUDA(cudaMemcpyAsync(vl, m.val, sizeof(double) * m.nnzb * m.br * m.bc,
                                     cudaMemcpyDeviceToHost, s));
    return AMG_OK;
}

int amg_level_export(amg_handle h, int32_t level, int32_t which, int32_t *row_ptr, int32_t *col,
                     double *val)
{
    clear_error();
    if (!h || level < 0 || level >= (int)h->lv.size()) {
        set_error("bad level");
        return AMG_ERR_ARG;
    }
    AllocScope scope(h->allocator());
    const Level &L = h->lv[level];
    cudaStream_t s = h->stream;
    switch (which) {
    case 0: AMG_TRY(export_bsr(L.A, row_ptr, col, val, s)); break;
    case 1: AMG_TRY(export_bsr(L.P, row_ptr, col, val, s)); break;
    case 2: AMG_TRY(export_bsr(L.R, row_ptr, col, val, s)); break;
    case 3:
        if (!L.agg) { set_error("no aggregates on this level"); return AMG_ERR_STATE; }
        if (row_ptr) AMG_TRY_CUDA(cudaMemcpyAsync(row_ptr, L.agg, sizeof(int) * L.A.nbr, cudaMemcpyDeviceToHost, s));
        break;
    case 4:
        if (!L.M) { set_error("no smoother on this level"); return AMG_ERR_STATE; }
        if (val) AMG_TRY_CUDA(cudaMemcpyAsync(val, L.M, sizeof(double) * L.n(), cudaMemcpyDeviceToHost, s));
        break;
    case 5:
        if (val) AMG_TRY_CUDA(cudaMemcpyAsync(val, L.B, sizeof(double) * L.n() * h->ns, cudaMemcpyDeviceToHost, s));
        break;
    case 7: {
        const double *mb = blocks_ptr<double>(h, (size_t)level);
        if (!mb) { set_error("no smoother blocks on this level"); return AMG_ERR_STATE; }
        if (val)
            AMG_TRY_CUDA(cudaMemcpyAsync(val, mb, sizeof(double) * L.A.nbr * L.A.br * L.A.br,
                                         cudaMemcpyDeviceToHost, s));
        break;
    }
    case 8:
    case 9:
        if (!L.ilu.F) { set_error("no ILU(0) factor on this level"); return AMG_ERR_STATE; }
        if (val && which == 8)
            AMG_TRY_CUDA(cudaMemcpyAsync(val, L.ilu.F, sizeof(double) * L.A.nnzb * L.A.br * L.A.br,
                                         cudaMemcpyDeviceToHost, s));
        if (val && which == 9)
            AMG_TRY_CUDA(cudaMemcpyAsync(val, L.ilu.Dinv, sizeof(double) * L.A.nbr * L.A.br * L.A.br,
                                         cudaMemcpyDeviceToHost, s));
        break;
    case 6:
        if (!L.strong) { set_error("no strength flags on this level"); return AMG_ERR_STATE; }
        if (row_ptr) AMG_TRY_CUDA(cudaMemcpyAsync(row_ptr, L.strong, L.A.nnzb, cudaMemcpyDeviceToHost, s));
        break;
    default: set_error("bad operator id %d", which); return AMG_ERR_ARG;
    }
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    return AMG_OK;
}

int amg_level_spmv(amg_handle h, int32_t level, int32_t which, const double *x, double *y,
                   void *stream)
{
    clear_error();
    if (!h || level < 0 || level >= (int)h->lv.size() || which < 0 || which > 5 || !x || !y) {
        set_error("bad argument");
        return AMG_ERR_ARG;
    }
    AllocScope scope(h->allocator());
    const Level &L = h->lv[level];
    if (which >= 3) {  // the FP32-pair copies of an AMG_PREC_DF64 hierarchy
        const Sell<df32> &E = which == 3 ? L.eA : which == 4 ? L.eP : L.eR;
        if (!E.slice_ptr) {
            set_error("no FP32-pair copy of this operator (AMG_PREC_DF64 only)");
            return AMG_ERR_STATE;
        }
        SellArgs<double> a{};
        a.x = x;
        a.y = y;
        return launch_sell<df32, double>(E, SPMV_PLAIN, DOT_NONE, a, h->geom, (cudaStream_t)stream);
    }
    const Sell<double> &S = which == 0 ? L.sA : which == 1 ? L.sP : L.sR;
    if (!S.slice_ptr) {
        set_error("operator not present on this level");
        return AMG_ERR_STATE;
    }
    SellArgs<double> a{};
    a.x = x;
    a.y = y;
    return launch_sell<double, double>(S, SPMV_PLAIN, DOT_NONE, a, h->geom, (cudaStream_t)stream);
}

// Element-wise comparison of two matrices with the same shape: red[0] = 1 if
// the row pointers or columns differ; red[1], red[2] = the bits of the
// largest |a - b| and |a| (non-negative doubles order like their bits).
__global__ void compare_bsr_kernel(const int *__restrict__ rp1, const int *__restrict__ rp2,
                                   int64_t nrp, const int *__restrict__ c1,
                                   const int *__restrict__ c2, int64_t nc,
                                   const double *__restrict__ v1, const double *__restrict__ v2,
                                   int64_t nv, unsigned long long *__restrict__ red)
{
    double dm = 0.0, am = 0.0;
    int diff = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv || i < nc || i < nrp;
         i += stride) {
        if (i < nrp) diff |= rp1[i] != rp2[i];
        if (i < nc) diff |= c1[i] != c2[i];
        if (i < nv) {
            dm = fmax(dm, fabs(v1[i] - v2[i]));
            am = fmax(am, fabs(v1[i]));
        }
    }
    if (diff) atomicOr(&red[0], 1ull);
    atomicMax(&red[1], (unsigned long long)__double_as_longlong(dm));
    atomicMax(&red[2], (unsigned long long)__double_as_longlong(am));
}

int amg_level_galerkin(amg_handle h, int32_t level, int32_t storage, double *seconds,
                       double *rel_diff)
{
    clear_error();
    if (!h || !seconds || !rel_diff || level < 0 || level + 1 >= (int)h->lv.size() ||
        (storage != AMG_STORAGE_BLOCK && storage != AMG_STORAGE_SCALAR)) {
        set_error("bad argument (level must have a coarser level)");
        return AMG_ERR_ARG;
    }
    AllocScope scope(h->allocator());
    const Level &L = h->lv[level];
    const BsrD &Ac0 = h->lv[level + 1].A;
    cudaStream_t s = h->stream;
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    DevArena keep, tmp;
    keep.stream = tmp.stream = s;
    BsrD C;
    const auto t0 = std::chrono::steady_clock::now();
    int st = storage == AMG_STORAGE_SCALAR ? galerkin_scalar(L.A, L.P, L.R, keep, tmp, s, &C)
                                           : galerkin(L.A, L.P, L.R, keep, tmp, s, &C);
    if (st >= 0 && cudaStreamSynchronize(s) != cudaSuccess) st = AMG_ERR_CUDA;
    *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    // compare with the hierarchy's A_{l+1} (unblocked for the scalar product),
    // on the device: pattern flag, largest |difference| and largest |entry|
    BsrD ref = Ac0;
    if (st >= 0 && storage == AMG_STORAGE_SCALAR) st = unblock_bsr(Ac0, tmp, s, &ref);
    if (st >= 0) {
        *rel_diff = -1.0;  // patterns differ
        if (C.nbr == ref.nbr && C.nnzb == ref.nnzb && C.br == ref.br && C.bc == ref.bc) {
            unsigned long long *red = nullptr;  // [0] pattern differs, [1] max |d|, [2] max |a|
            if (tmp.alloc_n(&red, 3) < 0) st = AMG_ERR_CUDA;
            if (st >= 0) {
                const int64_t nv = ref.nnzb * ref.br * ref.bc;
                const int64_t nidx = std::max<int64_t>(ref.nnzb, (int64_t)ref.nbr + 1);
                const int grid = (int)std::min<int64_t>((std::max(nv, nidx) + 255) / 256,
                                                        h->geom.max_ctas);
                cudaMemsetAsync(red, 0, sizeof(unsigned long long) * 3, s);
                compare_bsr_kernel<<<std::max(grid, 1), 256, 0, s>>>(
                    ref.row_ptr, C.row_ptr, ref.nbr + 1, ref.col, C.col, ref.nnzb, ref.val, C.val,
                    nv, red);
                count_launch(1);
                unsigned long long hr[3] = {0, 0, 0};
                if (cudaMemcpyAsync(hr, red, sizeof(hr), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess)
                    st = AMG_ERR_CUDA;
                if (st >= 0 && !hr[0]) {
                    double dmax, vmax;
                    std::memcpy(&dmax, &hr[1], sizeof dmax);
                    std::memcpy(&vmax, &hr[2], sizeof vmax);
                    *rel_diff = vmax > 0.0 ? dmax / vmax : dmax;
                }
            }
        }
    }
    cudaStreamSynchronize(s);
    keep.release_all();
    tmp.release_all();
    if (st < 0) return st;
    AMG_TRY_CUDA(cudaStreamSynchronize(s));
    return AMG_OK;
}

int amg_level_padding(amg_handle h, int32_t level, double *pad3)
{
    if (!h || !pad3 || level < 0 || level >= (int)h->lv.size()) return AMG_ERR_ARG;
    const Level &L = h->lv[level];
    pad3[0] = L.pad_A;
    pad3[1] = L.pad_P;
    pad3[2] = L.pad_R;
    return AMG_OK;
}

int amg_bsr_spmv(const amg_bsr *A, const double *x, double *y, void *stream)
{
    clear_error();
    AMG_TRY(check_bsr(A, 0));
    if (A->nbrows == 0) return AMG_OK;
    if (!y || (A->nnzb > 0 && !x)) {
        set_error("null vector");
        return AMG_ERR_ARG;
    }
    Geom g;
    AMG_TRY(query_geom(&g));
    SpmvArgs<double> a{};
    a.row_ptr = A->row_ptr;
    a.col = A->col;
    a.val = A->val;
    a.nbr = A->nbrows;
    a.x = x;
    a.y = y;
    return launch_spmv<double, double>(A->bs_r, A->bs_c, SPMV_PLAIN, DOT_NONE, a, g,
                                       (cudaStream_t)stream);
}

int amg_bsr_spmv_dot(const amg_bsr *A, const double *x, double *y, double *dot_out, void *stream)
{
    clear_error();
    AMG_TRY(check_bsr(A, 1));
    if (!x || !y || !dot_out) {
        set_error("null argument");
        return AMG_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Geom g;
    AMG_TRY(query_geom(&g));
    DevArena tmp;
    tmp.stream = s;
    double *part = nullptr;
    AMG_TRY(tmp.alloc_n(&part, (size_t)g.max_ctas + 1));
    SpmvArgs<double> a{};
    a.row_ptr = A->row_ptr;
    a.col = A->col;
    a.val = A->val;
    a.nbr = A->nbrows;
    a.x = x;
    a.y = y;
    a.partials = part;
    int grid = 0;
    int st = launch_spmv<double, double>(A->bs_r, A->bs_c, SPMV_PLAIN, DOT_XY, a, g, s, &grid);
    if (st >= 0) st = launch_reduce_sum(part, grid, part + g.max_ctas, s);
    if (st >= 0) {
        cudaError_t e = cudaMemcpyAsync(dot_out, part + g.max_ctas, sizeof(double),
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error("%s", cudaGetErrorString(e));
            st = AMG_ERR_CUDA;
        }
    }
    tmp.release_all();
    cudaStreamSynchronize(s);
    return st;
}

}  // extern "C"
