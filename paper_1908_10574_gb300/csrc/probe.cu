// cm_dpx_rate: the issue rate of the packed 16-bit DPX max-add instructions on this GPU, in
// lane-operations per clock per SM -- the denominator of the Smith-Waterman kernel's roofline
// (peak cells/s = SMs x clock x rate x 2 cells / ops per packed cell).
//
// One CTA of 1,024 threads per SM; every thread runs `iters` rounds of independent chains of
// the instructions the cell update issues most (__viaddmax_s16x2, then __vimax3_s16x2), on
// values that depend on runtime inputs so nothing folds away, and thread 0 of every CTA reads
// clock64() around the loop (between barriers).  The rate is the total lane-operations over
// the summed per-SM cycles.  The mix measures the two forms as the kernel uses them: three
// max-adds and one three-way max per step of a chain.
#include <cstdint>
#include <vector>

#include "ctx.h"

namespace cm {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(kProbeThreads, 1) dpx_rate_kernel(uint32_t seed, int32_t iters,
                                                                    long long* cycles,
                                                                    uint32_t* sink)
{
    uint32_t a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = seed * (threadIdx.x + 7 * k + 1);
    const uint32_t b = seed ^ 0x00050003u, c = seed | 0x00100010u;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) {
            a[k] = __viaddmax_s16x2(a[k], b, c);
            a[k] = __viaddmax_s16x2(a[k], c, b);
            a[k] = __viaddmax_s16x2(a[k], b, a[(k + 1) % kProbeChains]);
            a[k] = __vimax3_s16x2(a[k], b, a[(k + 3) % kProbeChains]);
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    uint32_t x = 0;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x ^= a[k];
    if (x == 0x9e3779b9u) sink[threadIdx.x] = x;       // keeps the chains live
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace
}  // namespace cm

using namespace cm;

extern "C" int cm_dpx_rate(cm_ctx* c, double* lane_ops_per_clk_per_sm)
{
    if (!c || !lane_ops_per_clk_per_sm) return c ? fail(c, CM_ERR_ARG, "null output") : CM_ERR_ARG;
    CUDA_TRY(cudaSetDevice(c->device));
    const int nsm = c->num_sms;
    long long* d_cyc;
    uint32_t* d_sink;
    ENSURE(B_RES, (size_t)nsm * 2 + 1, d_cyc);
    ENSURE(B_SCRATCH, (size_t)kProbeThreads, d_sink);
    const int32_t iters = 4096;
    std::vector<long long> cyc((size_t)nsm);
    for (int rep = 0; rep < 2; ++rep) {                   // the first launch warms up
        dpx_rate_kernel<<<nsm, kProbeThreads, 0, c->stream>>>(0x12345u + rep, iters, d_cyc, d_sink);
        CUDA_TRY(cudaGetLastError());
        c->stats.launches += 1;
    }
    CUDA_TRY(cudaMemcpyAsync(cyc.data(), d_cyc, (size_t)nsm * sizeof(long long),
                             cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    double cycles = 0;
    for (long long x : cyc) cycles += (double)x;
    const double ops = (double)nsm * kProbeThreads * iters * kProbeChains * 4.0;
    *lane_ops_per_clk_per_sm = cycles > 0 ? ops / cycles : 0.0;
    return CM_OK;
}
