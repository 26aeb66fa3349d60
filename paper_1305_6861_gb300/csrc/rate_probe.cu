// rate_probe.cu -- measured arithmetic rates of the device, the denominators of the roofline
// fractions the benchmark reports.
//
// The simulation is bound by the FP32 pipe (float32 path) or the float64 pipe (float64 path and
// the adjoint), not by memory.  A unit-count figure (SMs x lanes x clock) says what the pipe could
// do in principle; this probe says what a stream of independent fused multiply-adds actually
// reaches on this device: every thread runs 8 independent chains a <- a*m + c (no loads, no
// stores in the loop), the grid fills every SM with 2048 threads, and the kernel is timed with
// CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "../../include/mrsim.h"
#include "handles.h"
#include "packed.cuh"

using namespace mrsim;

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_BLOCKS_PER_SM = 8;
constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_UNROLL = 4;

// KIND 0: float32 fmaf; 1: float32 pairs, fma.rn.f32x2 (two lanes per instruction); 2: float64 fma.
// The chains converge to c / (1 - m) and stay finite; the store happens only for a NaN, which the
// compiler cannot rule out, so the chains are kept.
template <int KIND>
__global__ void __launch_bounds__(PROBE_THREADS) fma_rate_kernel(int64_t iters, int *sink) {
    const float s = 1.0f + 1e-7f * (float)(threadIdx.x & 31);
    if constexpr (KIND == 0) {
        float a[PROBE_CHAINS];
        const float m = 0.999999f * s, c = 1e-6f * s;
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = (float)j * s;
        for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
                for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = fmaf(a[j], m, c);
        }
        float t = 0.0f;
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j) t += a[j];
        if (isnan(t)) *sink = 1;
    } else if constexpr (KIND == 1) {
        dev::f2 a[PROBE_CHAINS];
        const dev::f2 m = dev::pk2(0.999999f * s, 0.9999995f * s), c = dev::pk2(1e-6f * s, 2e-6f * s);
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = dev::pk2((float)j * s, (float)j + s);
        for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
                for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = dev::vfma(a[j], m, c);
        }
        float t = 0.0f;
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j) t += dev::hsum(a[j]);
        if (isnan(t)) *sink = 1;
    } else {
        double a[PROBE_CHAINS];
        const double m = 0.999999 * s, c = 1e-6 * s;
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = (double)j * s;
        for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
                for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = fma(a[j], m, c);
        }
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j) t += a[j];
        if (isnan(t)) *sink = 1;
    }
}

cudaError_t launch_probe(int kind, int grid, int64_t iters, int *sink, cudaStream_t st) {
    switch (kind) {
    case 0: fma_rate_kernel<0><<<grid, PROBE_THREADS, 0, st>>>(iters, sink); break;
    case 1: fma_rate_kernel<1><<<grid, PROBE_THREADS, 0, st>>>(iters, sink); break;
    default: fma_rate_kernel<2><<<grid, PROBE_THREADS, 0, st>>>(iters, sink); break;
    }
    return cudaGetLastError();
}

// One timed launch; *ms receives its duration.
cudaError_t timed_probe(int kind, int grid, int64_t iters, int *sink, cudaStream_t st, float *ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = launch_probe(kind, grid, iters, sink, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

}  // namespace

extern "C" mrsim_status mrsim_measure_fma_rate(mrsim_ctx *ctx, int32_t kind, double target_ms, void *stream,
                                               double *lane_ops_per_s, double *kernel_ms) {
    if (!ctx) return MRSIM_EINVAL;
    if (kind < 0 || kind > 2 || !(target_ms >= 1.0 && target_ms <= 10000.0) || !lane_ops_per_s) {
        ctx->err = "mrsim_measure_fma_rate: kind must be 0..2, target_ms in [1, 1e4], lane_ops_per_s non-NULL";
        return MRSIM_EINVAL;
    }
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = ctx->num_sms * PROBE_BLOCKS_PER_SM;
    const double lanes_per_iter = (double)grid * PROBE_THREADS * PROBE_CHAINS * PROBE_UNROLL * (kind == 1 ? 2 : 1);
    // calibration launch (also loads the kernel), then one launch sized to the target duration
    int64_t iters = kind == 2 ? 256 : 4096;
    float ms = 0.0f;
    cudaError_t e = timed_probe(kind, grid, iters, ctx->d_bad, st, &ms);
    if (e == cudaSuccess) {
        const double scale = target_ms / std::max((double)ms, 1e-3);
        iters = std::max<int64_t>(1, (int64_t)((double)iters * std::min(scale, 1e6)));
        e = timed_probe(kind, grid, iters, ctx->d_bad, st, &ms);
    }
    if (e != cudaSuccess) {
        ctx->err = std::string("fma rate probe: ") + cudaGetErrorString(e);
        return MRSIM_ECUDA;
    }
    *lane_ops_per_s = lanes_per_iter * (double)iters / ((double)ms * 1e-3);
    if (kernel_ms) *kernel_ms = ms;
    return MRSIM_OK;
}
