// Throughput of the special-function unit (MUFU) for the approximate functions the
// backprojection update evaluates: rsqrt.approx.ftz, sin.approx.ftz, cos.approx.ftz, and
// the update's own mix (one reciprocal square root whose result feeds one sine and one
// cosine).  The MUFU rate bounds every kernel that sums (sample, position) updates (Eq. 3),
// so the rooflines of those kernels are taken against this measured rate rather than a
// nominal per-clock figure.
//
// Every thread runs eight independent dependency chains, and the grid fills every SM with
// 2048 threads, so that neither latency nor occupancy limits the rate.  The values stay
// normal and bounded: x <- rsqrt(x) tends to 1, x <- sin(x) decays slowly from below 1.5,
// x <- cos(x) tends to 0.739; the mix maps x in [1, 3] to 1 + sin(y)^2 + cos(y) with
// y = rsqrt(x), again in [1, 3).

#include <cuda_runtime.h>

#include <cstdint>

#include "hh_internal.h"
#include "hhffbp.h"

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;

__device__ __forceinline__ float probe_rsqrt(float x) {
    float y;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float probe_sin(float x) {
    float y;
    asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float probe_cos(float x) {
    float y;
    asm volatile("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int OP>
__global__ void __launch_bounds__(kProbeThreads) k_mufu_rate(float* __restrict__ out, int iters) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.25f + 0.03125f * (float)c + 1e-4f * (float)(threadIdx.x & 63);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if constexpr (OP == HH_MUFU_RSQRT) {
                x[c] = probe_rsqrt(x[c]);
            } else if constexpr (OP == HH_MUFU_SIN) {
                x[c] = probe_sin(x[c]);
            } else if constexpr (OP == HH_MUFU_COS) {
                x[c] = probe_cos(x[c]);
            } else {
                const float y = probe_rsqrt(x[c]);
                const float s = probe_sin(y), co = probe_cos(y);
                x[c] = fmaf(s, s, 1.f + co);
            }
        }
    }
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += x[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

template <int OP>
cudaError_t launch_probe(float* out, int blocks, int iters, cudaStream_t s) {
    k_mufu_rate<OP><<<blocks, kProbeThreads, 0, s>>>(out, iters);
    hh::note_launch();
    return cudaGetLastError();
}

cudaError_t launch_op(int op, float* out, int blocks, int iters, cudaStream_t s) {
    switch (op) {
        case HH_MUFU_RSQRT: return launch_probe<HH_MUFU_RSQRT>(out, blocks, iters, s);
        case HH_MUFU_SIN: return launch_probe<HH_MUFU_SIN>(out, blocks, iters, s);
        case HH_MUFU_COS: return launch_probe<HH_MUFU_COS>(out, blocks, iters, s);
        default: return launch_probe<HH_MUFU_UPDATE_MIX>(out, blocks, iters, s);
    }
}

}  // namespace

extern "C" int hh_mufu_throughput(int32_t op, int32_t iters, void* cuda_stream, int64_t* mufu_ops, float* ms) {
    if (!mufu_ops || !ms || iters <= 0 || iters > (1 << 20)) return HH_ERR_ARG;
    if (op != HH_MUFU_RSQRT && op != HH_MUFU_SIN && op != HH_MUFU_COS && op != HH_MUFU_UPDATE_MIX) return HH_ERR_ARG;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return hh::note_cuda_error((int)e);
    const int blocks = sms * kProbeBlocksPerSm;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    float* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void**>(&out), sizeof(float) * (size_t)blocks * kProbeThreads, s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = launch_op(op, out, blocks, iters, s);  // warm-up: clocks, module load
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch_op(op, out, blocks, iters, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (out) cudaFreeAsync(out, s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return hh::note_cuda_error((int)e);
    const int64_t per_iter = op == HH_MUFU_UPDATE_MIX ? 3 : 1;
    *mufu_ops = (int64_t)blocks * kProbeThreads * kChains * (int64_t)iters * per_iter;
    return HH_OK;
}
