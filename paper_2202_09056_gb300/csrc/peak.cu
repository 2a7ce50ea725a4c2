// Measured FP64 FMA rate of the device: the denominator of the FP64 SpMV's
// arithmetic roofline.  Every thread runs CH independent chains
// a <- a * m + c (m slightly below 1, so the values stay bounded and
// normal), which keeps the FP64 pipe supplied with independent instructions;
// the chains' sum is stored so that the work is observable.  Several chain
// counts and occupancies are timed and the fastest is reported: the pipe's
// rate is the best any of them sustains.
#include "amg_internal.cuh"

namespace amg {

constexpr int FMA_THREADS = 256;

template <int CH>
__global__ void fp64_fma_chains_kernel(double *__restrict__ sink, int iters, double m, double c)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;  // < sink_len (checked on the host)
    double a[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) a[k] = 1.0 + 1e-3 * k + 1e-9 * (double)(t & 1023);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < CH; ++k) a[k] = fma(a[k], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CH; ++k) s += a[k];
    sink[t] = s;
}

template <int CH>
static int time_chains(int grid, int64_t fmas_per_thread, double *sink, cudaStream_t s,
                       cudaEvent_t e0, cudaEvent_t e1, double *rate)
{
    const int iters = (int)std::max<int64_t>(1, fmas_per_thread / (4 * CH));
    fp64_fma_chains_kernel<CH><<<grid, FMA_THREADS, 0, s>>>(sink, iters / 16 + 1, 0.9999999,
                                                            1e-7);  // warm-up
    AMG_TRY_CUDA(cudaEventRecord(e0, s));
    fp64_fma_chains_kernel<CH><<<grid, FMA_THREADS, 0, s>>>(sink, iters, 0.9999999, 1e-7);
    AMG_TRY_CUDA(cudaEventRecord(e1, s));
    count_launch(2);
    AMG_TRY_CUDA(cudaGetLastError());
    AMG_TRY_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    AMG_TRY_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    *rate = (double)grid * FMA_THREADS * 4.0 * CH * (double)iters / (ms * 1e-3);
    return AMG_OK;
}

}  // namespace amg

using namespace amg;

extern "C" int amg_fp64_fma_rate(double *sink, int64_t sink_len, int32_t iters,
                                 double *fma_per_second, double *seconds, int32_t *num_sms,
                                 void *stream)
{
    clear_error();
    if (!sink || sink_len <= 0 || iters <= 0 || !fma_per_second) {
        set_error("amg_fp64_fma_rate: bad argument");
        return AMG_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Geom g;
    AMG_TRY(query_geom(&g));
    if (sink_len < (int64_t)g.num_sms * 8 * FMA_THREADS) {
        set_error("amg_fp64_fma_rate: sink holds %lld doubles, the largest grid writes %lld",
                  (long long)sink_len, (long long)g.num_sms * 8 * FMA_THREADS);
        return AMG_ERR_ARG;
    }
    cudaEvent_t e0, e1;
    AMG_TRY_CUDA(cudaEventCreate(&e0));
    AMG_TRY_CUDA(cudaEventCreate(&e1));
    // the same total FMAs per configuration: iters x 8 per thread of a
    // 4-CTA-per-SM grid
    const int64_t total = (int64_t)g.num_sms * 4 * FMA_THREADS * 8 * (int64_t)iters;
    double best = 0.0;
    int st = AMG_OK;
    for (int per_sm : {2, 4, 8}) {
        const int grid = g.num_sms * per_sm;
        const int64_t fpt = total / ((int64_t)grid * FMA_THREADS);
        double r4 = 0, r8 = 0, r16 = 0;
        if (st >= 0) st = time_chains<4>(grid, fpt, sink, s, e0, e1, &r4);
        if (st >= 0) st = time_chains<8>(grid, fpt, sink, s, e0, e1, &r8);
        if (st >= 0) st = time_chains<16>(grid, fpt, sink, s, e0, e1, &r16);
        best = std::max(best, std::max(r4, std::max(r8, r16)));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st < 0) return st;
    *fma_per_second = best;
    if (seconds) *seconds = (double)total / best;
    if (num_sms) *num_sms = g.num_sms;
    return AMG_OK;
}
