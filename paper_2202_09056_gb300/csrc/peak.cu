// Measured FP64 FMA rate of the device: the denominator of the FP64 SpMV's
// arithmetic roofline.  Every thread runs FMA_CHAINS independent chains
// a <- a * m + c (m slightly below 1, so the values stay bounded and
// normal), which keeps the FP64 pipe supplied with independent instructions;
// the chains' sum is stored so that the work is observable.  The grid fills
// every SM with FMA_CTAS_PER_SM CTAs of FMA_THREADS threads.
#include "amg_internal.cuh"

namespace amg {

constexpr int FMA_CHAINS = 8;
constexpr int FMA_THREADS = 256;
constexpr int FMA_CTAS_PER_SM = 4;

__global__ void __launch_bounds__(FMA_THREADS) fp64_fma_chains_kernel(double *__restrict__ sink,
                                                                      int64_t sink_len,
                                                                      int iters, double m,
                                                                      double c)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double a[FMA_CHAINS];
#pragma unroll
    for (int k = 0; k < FMA_CHAINS; ++k) a[k] = 1.0 + 1e-3 * k + 1e-9 * (double)(t & 1023);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < FMA_CHAINS; ++k) a[k] = fma(a[k], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < FMA_CHAINS; ++k) s += a[k];
    sink[t % sink_len] = s;
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
    const int grid = g.num_sms * FMA_CTAS_PER_SM;
    cudaEvent_t e0, e1;
    AMG_TRY_CUDA(cudaEventCreate(&e0));
    AMG_TRY_CUDA(cudaEventCreate(&e1));
    // one short launch first (clocks up, module loaded), then the timed one
    fp64_fma_chains_kernel<<<grid, FMA_THREADS, 0, s>>>(sink, sink_len, iters / 16 + 1,
                                                         0.9999999, 1e-7);
    count_launch(1);
    AMG_TRY_CUDA(cudaEventRecord(e0, s));
    fp64_fma_chains_kernel<<<grid, FMA_THREADS, 0, s>>>(sink, sink_len, iters, 0.9999999, 1e-7);
    count_launch(1);
    AMG_TRY_CUDA(cudaEventRecord(e1, s));
    AMG_TRY_CUDA(cudaGetLastError());
    AMG_TRY_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    AMG_TRY_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double fmas = (double)grid * FMA_THREADS * FMA_CHAINS * (double)iters;
    *fma_per_second = fmas / (ms * 1e-3);
    if (seconds) *seconds = ms * 1e-3;
    if (num_sms) *num_sms = g.num_sms;
    return AMG_OK;
}
