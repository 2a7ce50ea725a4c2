// Error reporting, stream-ordered device memory and launch geometry.
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

int DevArena::alloc(void **p, size_t n)
{
    *p = nullptr;
    if (n == 0) n = 16;
    cudaError_t e = cudaMallocAsync(p, n, stream);
    if (e != cudaSuccess) {
        set_error("cudaMallocAsync(%zu bytes): %s", n, cudaGetErrorString(e));
        *p = nullptr;
        return AMG_ERR_CUDA;
    }
    ptrs.push_back(*p);
    bytes += n;
    return AMG_OK;
}

void DevArena::release(void *p)
{
    if (!p) return;
    for (size_t i = 0; i < ptrs.size(); ++i)
        if (ptrs[i] == p) {
            cudaFreeAsync(p, stream);
            ptrs[i] = ptrs.back();
            ptrs.pop_back();
            return;
        }
}

void DevArena::release_all()
{
    for (void *p : ptrs) cudaFreeAsync(p, stream);
    ptrs.clear();
    bytes = 0;
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
