// Internal declarations shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <exception>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/amg_gb300.h"

namespace amg {

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
void clear_error();
const char *last_error();

// f() with any C++ exception (host memory exhausted in a std::vector, a
// thread that cannot start) turned into an error status: nothing unwinds
// through the C ABI or out of a worker thread.
template <class F> int no_throw(F &&f)
{
    try {
        return f();
    } catch (const std::bad_alloc &) {
        set_error("host memory exhausted");
        return AMG_ERR_LIMIT;
    } catch (const std::exception &e) {
        set_error("%s", e.what());
        return AMG_ERR_STATE;
    } catch (...) {
        set_error("unexpected exception");
        return AMG_ERR_STATE;
    }
}

// Kernel launch accounting: every launch site reports itself; launches
// recorded into a graph under capture are counted per graph execution.
void count_launch(long long n);
void begin_launch_capture(long long *counter);
void end_launch_capture();

#define AMG_TRY_CUDA(call)                                                              \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            ::amg::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,                 \
                             cudaGetErrorString(e_));                                   \
            return AMG_ERR_CUDA;                                                        \
        }                                                                               \
    } while (0)

#define AMG_TRY(call)                                                                   \
    do {                                                                                \
        int s_ = (call);                                                                \
        if (s_ < 0) return s_;                                                          \
    } while (0)

// ---------------------------------------------------------------- device memory
// The caller's device memory supplier for the duration of a library call on
// a handle (amg_params.allocator); null = the library's own stream-ordered
// cudaMallocAsync.  Scoped per thread: entry points install their handle's.
struct AllocScope {
    const amg_allocator *prev;
    explicit AllocScope(const amg_allocator *a);
    ~AllocScope();
};
const amg_allocator *current_allocator();

// Device allocations owned by a handle (or a call).  Each pointer remembers
// the supplier it came from (the scope's at allocation time) and goes back
// to it.
struct DevArena {
    struct Rec {
        void *p;
        size_t n;
        amg_allocator al;   // al.alloc == nullptr: cudaMallocAsync
    };
    cudaStream_t stream = nullptr;
    std::vector<Rec> recs;
    size_t bytes = 0;
    int alloc(void **p, size_t n);
    template <class T> int alloc_n(T **p, size_t n) { return alloc((void **)p, n * sizeof(T)); }
    void release(void *p);   // free one pointer early
    void release_all();
    bool has_custom() const;
};

// A device BSR matrix owned by the library.  Values are stored in T.
template <class T> struct Bsr {
    int nbr = 0, nbc = 0, br = 0, bc = 0;
    int64_t nnzb = 0;
    int *row_ptr = nullptr;
    int *col = nullptr;
    T *val = nullptr;
};
using BsrD = Bsr<double>;

// Argument check of a borrowed BSR matrix (dimensions, nnzb within int32,
// pointers; square with square blocks when want_square).
int check_bsr(const amg_bsr *A, int want_square);

// ---------------------------------------------------------------- launch geometry
struct Geom {
    int num_sms = 0;
    int max_ctas = 0;       // grid cap of the 256-thread grid-stride kernels
    int max_partials = 0;   // largest grid of any kernel with a fused dot (per-CTA partials)
};
int query_geom(Geom *g);

// ---------------------------------------------------------------- CG device state
struct CgState {
    double tol, nf;        // tolerance, ||f||
    double rz, pq, alpha, beta, res, res_true;
    int it, maxiter;
    int check;             // recurrence residual reached tol: confirm with the true one
    int replace;           // true residual failed: replace r by it
    int converged;
    int stop;              // loop ends after this iteration (converged, maxiter, breakdown)
    int no_check;          // early-exit flag of the true-residual kernel (= !check)
    int no_replace;        // early-exit flag of the replacement kernel
    int status;            // AMG_OK / AMG_NOT_CONVERGED / AMG_ERR_BREAKDOWN
};

// ---------------------------------------------------------------- kernels (spmv.cu)
enum SpmvMode {
    SPMV_PLAIN = 0,   // y = A x
    SPMV_RESID = 1,   // y = f - A x
    SPMV_SMOOTH = 2,  // y = x + M (f - A x)           (x = u, square A)
    SPMV_AXPY = 3,    // y = u + A x                  (prolongation, y may alias u)
    SPMV_RESTRICT = 4,// y = A x ; y2 = M y           (restriction + next pre-smoothing)
    SPMV_SMOOTHB = 5, // y = x + Mb (f - A x)          (block smoother, b x b per block row)
};

enum DotMode {
    DOT_NONE = 0,
    DOT_XY = 1,       // sum_i x_i y_i over the output rows (square A: q = A p, p.q)
    DOT_FY = 2,       // sum_i f_i y_i                (post-smoothing on level 0: r.z)
    DOT_YY = 3,       // sum_i y_i y_i                (true residual norm)
};

// Vector element type of the V-cycle (double, or float for the reduced-precision forms).
template <class TV> struct SpmvArgs {
    const int *row_ptr;
    const int *col;
    const void *val;     // value type chosen by the launcher
    int nbr;
    const TV *x;
    const TV *f;
    const TV *u;
    const TV *M;
    TV *y;
    TV *y2;
    double *partials;    // one per CTA when a dot is fused
    const int *stop;     // early exit when *stop != 0 (may be null)
};

// Launch y = op(A) x with the given mode.  VT = value type of the blocks.
int spmv_grid(int nbr, const Geom &g);

template <class VT, class TV>
int launch_spmv(int br, int bc, int mode, int dot, const SpmvArgs<TV> &a, const Geom &g,
                cudaStream_t s, int *grid_out = nullptr);

// Deterministic reduction of `n` partials into out[0] (single CTA), with an
// optional finisher applied by one thread.
int launch_reduce_sum(const double *partials, int n, double *out, cudaStream_t s);

// Dense GEMV on the coarsest level: y = Ainv * x (n x n row-major).
template <class TV>
int launch_coarse_gemv(const double *Ainv, int n, const TV *x, TV *y, const Geom &g,
                       cudaStream_t s);

// ---------------------------------------------------------------- FP64 on FP32 pairs
// A double held as the unevaluated sum of two floats, hi + lo (about 48
// significant bits).  GB300 issues FP32 at 64x its FP64 rate, so products of
// such pairs computed with FP32 operations (an error-free product plus a
// compensated sum) move the FP64-bound SpMV onto the FP32 pipe.  The
// conversions are done on the bits (integer operations), so that no step
// runs on the FP64 pipe.
//
// split: hi = x with its significand truncated to 24 bits, lo = the next 24
// of the 29 bits below (truncated); |x - (hi + lo)| < 2^-47 |x|.  Values
// outside FP32's normal range (|x| < 2^-126 or > 2^128) are flushed to zero
// or infinity; a lo part below that range is dropped.
__device__ __forceinline__ void split_f64(double x, float &h, float &l)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned int sgn = (unsigned int)(u >> 63) << 31;
    const int e = (int)((u >> 52) & 0x7ff);
    const unsigned long long m = u & 0xfffffffffffffull;
    const int fe = e - 1023 + 127;  // FP32 biased exponent of x
    l = __uint_as_float(sgn);
    if (e == 0 || fe <= 0) {
        h = __uint_as_float(sgn);
        return;
    }
    if (fe >= 255) {
        h = __uint_as_float(sgn | 0x7f800000u | ((e == 0x7ff && m) ? 0x400000u : 0u));
        return;
    }
    h = __uint_as_float(sgn | ((unsigned int)fe << 23) | (unsigned int)(m >> 29));
    const unsigned long long rem = m & 0x1fffffffull;  // x - hi = rem * 2^(e - 1075)
    if (rem == 0) return;
    const int top = 63 - __clzll((long long)rem);  // rem in [2^top, 2^(top+1)), top <= 28
    const int le = e - 1075 + top + 127;
    if (le <= 0) return;
    const unsigned int mant =
        top >= 23 ? (unsigned int)(rem >> (top - 23)) : (unsigned int)(rem << (23 - top));
    l = __uint_as_float(sgn | ((unsigned int)le << 23) | (mant & 0x7fffffu));
}

// exact float -> double on the bits (subnormal floats flushed to zero)
__device__ __forceinline__ double f32_to_f64(float f)
{
    const unsigned int u = __float_as_uint(f);
    const unsigned long long sgn = (unsigned long long)(u >> 31) << 63;
    const unsigned int e = (u >> 23) & 0xff;
    const unsigned long long m = (unsigned long long)(u & 0x7fffffu) << 29;
    if (e == 0) return __longlong_as_double((long long)sgn);
    if (e == 0xff) return __longlong_as_double((long long)(sgn | 0x7ff0000000000000ull | m));
    return __longlong_as_double((long long)(sgn | ((unsigned long long)(e + 896) << 52) | m));
}

// double -> float rounded to nearest (ties to even) on the bits; values
// outside FP32's normal range are flushed to zero or infinity
__device__ __forceinline__ float f64_to_f32_rn(double x)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned int sgn = (unsigned int)(u >> 63) << 31;
    const int e = (int)((u >> 52) & 0x7ff);
    const unsigned long long m = u & 0xfffffffffffffull;
    const int fe = e - 896;  // FP32 biased exponent
    if (e == 0 || fe <= 0) return __uint_as_float(sgn);
    if (fe >= 255)
        return __uint_as_float(sgn | 0x7f800000u | ((e == 0x7ff && m) ? 0x400000u : 0u));
    unsigned int bits = ((unsigned int)fe << 23) | (unsigned int)(m >> 29);
    const unsigned long long rem = m & 0x1fffffffull, half = 0x10000000ull;
    if (rem > half || (rem == half && (bits & 1u))) ++bits;  // a carry may round up to infinity
    return __uint_as_float(sgn | bits);
}

struct __align__(8) df32 {
    float h, l;
    __host__ __device__ df32() : h(0.0f), l(0.0f) {}
    __device__ explicit df32(double v) { split_f64(v, h, l); }
};

// ---------------------------------------------------------------- SELL-32 (sell.cu)
// Sliced block-ELL: 32 lanes per slice, G lanes per block row (32/G rows per
// slice); block k of a row belongs to lane k % G of its group at depth k / G,
// and the blocks of a slice are interleaved so that every warp-wide load is
// contiguous.
template <class T> struct Sell {
    int nrows = 0, nbc = 0, br = 0, bc = 0, nslices = 0;
    int G = 1;                   // lanes per block row (power of two, <= 128); 32/G rows
                                 // per slice, or G/32 slices per row when G > 32
    int64_t nslots = 0;          // block slots including padding (multiple of 32)
    int64_t *slice_ptr = nullptr;// [nslices + 1] slot offsets
    int *col = nullptr;          // [nslots]
    T *val = nullptr;            // [nslots * br * bc]
    int *perm = nullptr;         // optional row of each row slot (-1 = padding)
};

template <class TV> struct SellArgs {
    const TV *Mb;        // b x b smoother blocks (SPMV_SMOOTHB), in the vectors' precision
    const TV *Mbn;       // SPMV_RESTRICT: the next level's blocks, y2 = Mbn y per block row
    int nrows, nslices, G;
    const int64_t *slice_ptr;
    const int *col;
    const void *val;
    const int *perm;
    const TV *x;
    const TV *f;
    const TV *u;
    const TV *M;
    TV *y;
    TV *y2;
    double *partials;
    const int *stop;
};

int sell_grid(int nslices, int br, int bc, const Geom &g);
// bytes a sliced copy holds on the device
template <class T> int64_t sell_bytes(const Sell<T> &S);
// max_grid > 0 caps the grid (the warp-strided loop covers every slice): for
// launches that usually exit at once on their stop flag
template <class VT, class TV>
int launch_sell(const Sell<VT> &A, int mode, int dot, SellArgs<TV> a, const Geom &g,
                cudaStream_t s, int *grid_out = nullptr, int max_grid = 0);
template <class T>
int bsr_to_sell(const BsrD &B, DevArena &keep, cudaStream_t s, Sell<T> *out, double *padding,
                int max_lanes = 128);

// ---------------------------------------------------------------- setup (setup.cu)
struct LevelBuild {
    // outputs of one coarsening step on device
    BsrD P, R, Ac;
    double *Bc = nullptr;
    int *agg = nullptr;
    int nagg = 0;
    double omega = 0, rho = 0;
};

int exclusive_scan_i32(const int *in, int *out, int n, int *total_host, DevArena &tmp,
                       cudaStream_t s);
int compute_strength(const BsrD &A, double eps, uint8_t *strong, cudaStream_t s);
// Parallel MIS-2 aggregation on the device (mis2.cu): agg[nbr] device, the
// aggregate count (and, if asked, the number of rounds) to the host.
int aggregate_mis2(const BsrD &A, const uint8_t *strong, int *agg, int *nagg_host, int *rounds_host,
                   DevArena &tmp, cudaStream_t s);
// The strong links of a level's node graph on the host: per node its strong
// neighbours in column order (CSR, host memory, not zero-filled).
struct HostStrongGraph {
    int nn = 0;
    std::unique_ptr<int[]> srp, scol;
};
int strong_graph_to_host(const BsrD &A, const uint8_t *strong, DevArena &tmp, cudaStream_t s,
                         HostStrongGraph *out);
// greedy aggregation (aggregate.cpp) on the strong graph; agg[nn] host
int aggregate_host(int nn, const int *srp, const int *scol, int *agg, int *nagg);
int build_transfer(const BsrD &A, const double *B, int ns, const uint8_t *strong,
                   const int *agg_h, int nagg, double relax, DevArena &keep, DevArena &tmp,
                   cudaStream_t s, LevelBuild *out);
// scalar CSR (1x1 blocks) copy of a BSR matrix, allocated in mem
int unblock_bsr(const BsrD &B, DevArena &mem, cudaStream_t s, BsrD *out);
int galerkin(const BsrD &A, const BsrD &P, const BsrD &R, DevArena &keep, DevArena &tmp,
             cudaStream_t s, BsrD *Ac);
int galerkin_scalar(const BsrD &A, const BsrD &P, const BsrD &R, DevArena &keep, DevArena &tmp,
                    cudaStream_t s, BsrD *Ac);
int spai0_diag(const BsrD &A, double scale, double *M, cudaStream_t s);
// scalar setup (the Sec. 3/4 scalar and hybrid solvers): S is scalar CSR
// (1x1 blocks), nodes are b consecutive rows.  The node graph (pattern in
// `graph`, flags in *strong, allocated in keep) with the block setup's
// strength test; the transfer operators P, R as scalar CSR; a scalar CSR
// matrix converted into br x bc blocks (explicit zeros where absent).
int scalar_strength(const BsrD &S, int b, double eps, DevArena &keep, DevArena &tmp,
                    cudaStream_t s, BsrD *graph, uint8_t **strong);
int scalar_transfer(const BsrD &S, int b, const double *B, int ns, const int *agg_h, int nagg,
                    double relax, DevArena &keep, DevArena &tmp, cudaStream_t s, LevelBuild *out);
int scalar_to_block(const BsrD &S, int br, int bc, DevArena &keep, DevArena &tmp, cudaStream_t s,
                    BsrD *out);
// Block damped Jacobi blocks of every smoothing level (bjacobi.cu).
int bjacobi_setup(amg_handle h, DevArena &tmp, cudaStream_t s);

int coarse_inverse(const BsrD &A, DevArena &keep, DevArena &tmp, cudaStream_t s,
                   double **Ainv_out);

// ---------------------------------------------------------------- block ILU(0) (ilu.cu)
struct Ilu {
    int nbr = 0, b = 0, depth = 0;  // depth = dependency levels of the factorisation
    double *F = nullptr;            // factor on A's block pattern: L below, U on/above the diagonal
    double *Dinv = nullptr;         // [nbr][b][b] inverses of U's diagonal blocks
    Sell<double> sL, sU;            // strict lower / strict upper parts, sliced
    bool has_L = false, has_U = false;
    double *y0 = nullptr, *y1 = nullptr;  // sweep vectors
};
int ilu0_factor(const BsrD &A, int max_lanes, DevArena &keep, DevArena &tmp, cudaStream_t s,
                Ilu *out);
// x = ILU^-1 r with `sweeps` Jacobi sweeps per triangle (x must not alias r)
int ilu0_apply(const Ilu &F, int sweeps, const double *r, double *x, const Geom &g, cudaStream_t s);
int launch_vec_add(const double *a, const double *b, double *y, int64_t n, cudaStream_t s);

// ---------------------------------------------------------------- hierarchy (solver.cu)
struct Level {
    BsrD A, P, R;
    Sell<double> sA, sP, sR;  // V-cycle copies of A, P, R in the SELL layout (FP64)
    Sell<float> fA, fP, fR;   // FP32 copies (precision form)
    Sell<__nv_bfloat16> bA, bP, bR;  // BF16-stored copies (precision form)
    Sell<df32> eA, eP, eR;    // FP64 values as FP32 pairs (AMG_PREC_DF64)
    double pad_A = 0, pad_P = 0, pad_R = 0;
    float *Mf = nullptr;      // smoother diagonal for the reduced-precision V-cycle
    float *vf = nullptr, *vu = nullptr, *ve = nullptr, *vz = nullptr, *vt = nullptr;
    double *M = nullptr;      // damped SPAI0 diagonal (scalar rows)
    double *B = nullptr;      // near-nullspace, n x 6
    int *agg = nullptr;       // aggregate of each node (device)
    uint8_t *strong = nullptr;
    int nagg = 0;
    bool coarsest = false;
    double eps = 0, omega = 0, rho = 0;
    double *f = nullptr, *u = nullptr, *e = nullptr, *z = nullptr, *t = nullptr;
    double *Mb = nullptr;     // smoother blocks, replacing M when set: learned 3x3 (level
                              // 0) or block damped Jacobi (b x b, every smoothing level)
    float *Mbf = nullptr;     // FP32 copy of Mb for the FP32 / BF16 V-cycles
    double bj_lambda = 0;     // block Jacobi: the lambda_max(D_b^-1 A) estimate
    Ilu ilu;                  // block ILU(0) smoother (when selected), replaces M
    BsrD xA, xP, xR;          // scalar CSR of A, P, R built by the scalar setup (kept until
                              // the solve's copies are made)
    int n() const { return A.nbr * A.br; }
};

}  // namespace amg

// The hierarchy handle behind the C ABI's opaque amg_handle.
struct amg_handle_s {
    amg_params prm;
    amg_allocator alloc{};        // copy of *prm.allocator (alloc == nullptr: none)
    const amg_allocator *allocator() const { return alloc.alloc ? &alloc : nullptr; }
    cudaStream_t stream = nullptr;
    amg::Geom geom;
    int max_lanes = 128;          // cap on lanes per row of the sliced copies
    int ns = 6;                   // near-nullspace columns = DOFs of a coarse node (6 or 3)
    amg::DevArena mem;
    std::vector<amg::Level> lv;
    double *Ainv = nullptr;
    int nc = 0;
    double *ff = nullptr, *uu = nullptr, *r = nullptr, *p = nullptr, *q = nullptr,
           *z = nullptr, *rt = nullptr, *partials = nullptr, *scal = nullptr;
    float *rv = nullptr, *zv = nullptr;   // r and z in the reduced-precision V-cycle
    amg::CgState *st = nullptr;
    amg::CgState *st_h = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long body_kernels = 0;   // kernels in one iteration of the graph body
    double setup_seconds = 0.0;
    double setup_phase[7] = {0, 0, 0, 0, 0, 0, 0};  // see amg_stats.setup_phase_seconds
    int learned = 0;              // level 0 smooths with the learned blocks
    int ilu = 0;                  // every smoothing level uses its block ILU(0)
    double learned_lambda = 0.0;  // estimated lambda_max(M A) of the learned smoother
    double spai0_lambda = 0.0;    // the same estimate for SPAI0 (0 until first needed)
};


namespace amg {
int setup_impl(amg_handle h, const amg_bsr *Ain, const double *B);
void destroy_handle(amg_handle h);
// out_I = Mb_I r_I for every 3-row node (learned smoother, learned.cu)
template <class T>
int launch_block_apply(const T *Mb, const T *r, T *out, int nrows, const Geom &g, cudaStream_t s);
}  // namespace amg
