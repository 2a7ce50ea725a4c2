// Error reporting, device memory (the library's stream-ordered allocations or
// the caller's supplier) and launch geometry.
#include <atomic>
#include <cstdarg>
#include <cstring>

#include "amg_internal.cuh"

namespace amg {

static thread_local char g_last_error[1024] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
}

void clear_error() { g_last_error[0] = '\0'; }

const char *last_error() { return g_last_error; }

static std::atomic<long long> g_launches{0};
static thread_local long long *t_capture = nullptr;

void count_launch(long long n)
{
    if (t_capture) *t_capture += n;
    else g_launches += n;
}
void begin_launch_capture(long long *counter) { t_capture = counter; }
void end_launch_capture() { t_capture = nullptr; }
long long launches() { return g_launches.load(); }

static thread_local const amg_allocator *t_allocator = nullptr;

AllocScope::AllocScope(const amg_allocator *a) : prev(t_allocator) { t_allocator = a; }
AllocScope::~AllocScope() { t_allocator = prev; }
const amg_allocator *current_allocator() { return t_allocator; }

int DevArena::alloc(void **p, size_t n)
{
    *p = nullptr;
    if (n == 0) n = 16;
    const amg_allocator *a = t_allocator;
    Rec r{nullptr, n, amg_allocator{}};
    if (a && a->alloc) {
        r.p = a->alloc(a->ctx, n, (void *)stream);
        if (!r.p) {
            set_error("the caller's allocator returned NULL for %zu bytes", n);
            return AMG_ERR_CUDA;
        }
        if (((uintptr_t)r.p & 255u) != 0) {
            if (a->free) a->free(a->ctx, r.p, n, (void *)stream);
            set_error("the caller's allocator returned a pointer that is not 256-byte aligned");
            return AMG_ERR_ARG;
        }
        r.al = *a;
    } else {
        cudaError_t e = cudaMallocAsync(&r.p, n, stream);
        if (e != cudaSuccess) {
            set_error("cudaMallocAsync(%zu bytes): %s", n, cudaGetErrorString(e));
            return AMG_ERR_CUDA;
        }
    }
    *p = r.p;
    recs.push_back(r);
    bytes += n;
    return AMG_OK;
}

static void give_back(const DevArena::Rec &r, cudaStream_t s)
{
    if (r.al.alloc) {
        if (r.al.free) r.al.free(r.al.ctx, r.p, r.n, (void *)s);
    } else {
        cudaFreeAsync(r.p, s);
    }
}

void DevArena::release(void *p)
{
    if (!p) return;
    for (size_t i = 0; i < recs.size(); ++i)
        if (recs[i].p == p) {
            give_back(recs[i], stream);
            bytes -= recs[i].n;
            recs[i] = recs.back();
            recs.pop_back();
            return;
        }
}

void DevArena::release_all()
{
    for (const Rec &r : recs) give_back(r, stream);
    recs.clear();
    bytes = 0;
}

bool DevArena::has_custom() const
{
    for (const Rec &r : recs)
        if (r.al.alloc) return true;
    return false;
}

int check_bsr(const amg_bsr *A, int want_square)
{
    if (!A) {
        set_error("null matrix");
        return AMG_ERR_ARG;
    }
    if (A->nbrows < 0 || A->nbcols < 0 || A->nnzb < 0 || A->nnzb > 2147483647LL) {
        set_error("bad matrix dimensions");
        return AMG_ERR_ARG;
    }
    if (want_square && (A->nbrows != A->nbcols || A->bs_r != A->bs_c)) {
        set_error("matrix must be square with square blocks");
        return AMG_ERR_ARG;
    }
    if (!A->row_ptr || (A->nnzb > 0 && (!A->col || !A->val))) {
        set_error("null matrix array");
        return AMG_ERR_ARG;
    }
    return AMG_OK;
}

int query_geom(Geom *g)
{
    int dev = 0;
    AMG_TRY_CUDA(cudaGetDevice(&dev));
    AMG_TRY_CUDA(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, dev));
    g->max_ctas = g->num_sms * 8;  // 8 CTAs of 256 threads fill an SM's 2048 thread slots
    // the sliced SpMV runs up to 16 CTAs of 128 threads per SM; every kernel
    // that leaves one partial sum per CTA stays within this many
    g->max_partials = g->num_sms * 32;  // largest SELL grid (sell_cap)
    return AMG_OK;
}

}  // namespace amg

extern "C" int64_t amg_kernel_launches(void) { return (int64_t)amg::launches(); }
