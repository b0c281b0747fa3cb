// Arithmetic-pipe probes (mrcm_probe_peak): the throughput ceilings the
// roofline of the MRCM kernels is quoted against, measured on the device the
// library runs on rather than taken from a datasheet.
//
// Each probe keeps every scheduler of every SM busy with independent chains
// of one instruction kind and counts its flops:
//   DFMA  FP64 fused multiply-add, 8 independent chains per thread (2 flops)
//   DMMA  FP64 mma.sync m8n8k4, 4 independent accumulators per warp (512)
//   FFMA  FP32 fused multiply-add, 8 chains per thread (2 flops)
//   TF32  mma.sync m16n8k8 tf32 -> f32, 4 accumulators per warp (2048)
//   BF16  mma.sync m16n8k16 bf16 -> f32, 4 accumulators per warp (4096)
//   DFMA_DMMA  half the warps DFMA, half DMMA (do the two FP64 paths add up?)
// The results never leave the registers except through a store guarded by a
// comparison with a runtime NaN (never true), which keeps the compiler from
// dropping the chains.
#include <algorithm>

#include "mrcm_internal.h"
#include "../../include/mrcm.h"

namespace mrcm {
namespace {

__device__ double g_probe_sink;

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSM = 4;

__device__ __forceinline__ void dfma_chains(double (&a)[8], double b, double c) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
}
__global__ void __launch_bounds__(kProbeThreads) probe_dfma(int iters, double b, double never) {
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 1e-3 + k;
    const double c = b * 1e-9;
    // four iterations per loop trip: the loop's own instructions stay far
    // below the FP64 issue rate
    int it = 0;
    for (; it + 3 < iters; it += 4) {
        dfma_chains(a, b, c);
        dfma_chains(a, b, c);
        dfma_chains(a, b, c);
        dfma_chains(a, b, c);
    }
    for (; it < iters; ++it) dfma_chains(a, b, c);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == never) g_probe_sink = s;
}

// Half of the warps of each CTA run FP64 FMA chains and half FP64 MMA
// chains (the same per-warp flops per iteration as the two probes above
// divided evenly): shows whether the two FP64 paths share one unit.
__global__ void __launch_bounds__(kProbeThreads) probe_dfma_dmma(int iters, double b, double never) {
    double s = 0.0;
    if ((threadIdx.x >> 5) & 1) {
        double a[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 1e-3 + k;
        const double c = b * 1e-9;
        for (int it = 0; it < iters; ++it) dfma_chains(a, b, c);
#pragma unroll
        for (int k = 0; k < 8; ++k) s += a[k];
    } else {
        const double av = threadIdx.x * 1e-3;
        double c[4][2];
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k][0] = c[k][1] = 0.0;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                             : "+d"(c[k][0]), "+d"(c[k][1])
                             : "d"(av), "d"(b));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) s += c[k][0] + c[k][1];
    }
    if (s == never) g_probe_sink = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_ffma(int iters, float b, double never) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 1e-3f + k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], b, 1e-9f);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if ((double)s == never) g_probe_sink = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_dmma(int iters, double b, double never) {
    const double av = threadIdx.x * 1e-3, bv = b;
    double c[4][2];
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k][0] = c[k][1] = 0.0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(c[k][0]), "+d"(c[k][1])
                         : "d"(av), "d"(bv));
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) s += c[k][0] + c[k][1];
    if (s == never) g_probe_sink = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_tf32(int iters, float b, double never) {
    const unsigned a = __float_as_uint(threadIdx.x * 1e-3f), bb = __float_as_uint(b);
    float c[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int r = 0; r < 4; ++r) c[k][r] = 0.f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            asm volatile(
                "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                "{%8, %9}, {%0, %1, %2, %3};"
                : "+f"(c[k][0]), "+f"(c[k][1]), "+f"(c[k][2]), "+f"(c[k][3])
                : "r"(a), "r"(a), "r"(a), "r"(a), "r"(bb), "r"(bb));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) s += c[k][0] + c[k][1] + c[k][2] + c[k][3];
    if ((double)s == never) g_probe_sink = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_bf16(int iters, float b, double never) {
    // two bf16 values per 32-bit register
    const unsigned short hb = (unsigned short)(__float_as_uint(b) >> 16);
    const unsigned a = ((unsigned)hb << 16) | hb;
    float c[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int r = 0; r < 4; ++r) c[k][r] = 0.f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                "{%8, %9}, {%0, %1, %2, %3};"
                : "+f"(c[k][0]), "+f"(c[k][1]), "+f"(c[k][2]), "+f"(c[k][3])
                : "r"(a), "r"(a), "r"(a), "r"(a), "r"(a), "r"(a));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) s += c[k][0] + c[k][1] + c[k][2] + c[k][3];
    if ((double)s == never) g_probe_sink = s;
}

// flops of one iteration of one thread (mma: per warp / 32)
double probe_flops_per_thread_iter(int kind) {
    switch (kind) {
        case MRCM_PROBE_DFMA: return 16.0;
        case MRCM_PROBE_DMMA: return 4.0 * 512.0 / 32.0;
        case MRCM_PROBE_FFMA: return 16.0;
        case MRCM_PROBE_TF32: return 4.0 * 2048.0 / 32.0;
        case MRCM_PROBE_BF16: return 4.0 * 4096.0 / 32.0;
        case MRCM_PROBE_DFMA_DMMA: return 0.5 * 16.0 + 0.5 * (4.0 * 512.0 / 32.0);
        default: return 0.0;
    }
}

cudaError_t probe_launch(int kind, int grid, int iters, cudaStream_t s) {
    const double never = __builtin_nan("");
    switch (kind) {
        case MRCM_PROBE_DFMA: probe_dfma<<<grid, kProbeThreads, 0, s>>>(iters, 0.999999, never); break;
        case MRCM_PROBE_DMMA: probe_dmma<<<grid, kProbeThreads, 0, s>>>(iters, 0.999999, never); break;
        case MRCM_PROBE_FFMA: probe_ffma<<<grid, kProbeThreads, 0, s>>>(iters, 0.999999f, never); break;
        case MRCM_PROBE_TF32: probe_tf32<<<grid, kProbeThreads, 0, s>>>(iters, 0.999999f, never); break;
        case MRCM_PROBE_BF16: probe_bf16<<<grid, kProbeThreads, 0, s>>>(iters, 0.999999f, never); break;
        case MRCM_PROBE_DFMA_DMMA: probe_dfma_dmma<<<grid, kProbeThreads, 0, s>>>(iters, 0.999999, never); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace
}  // namespace mrcm

using namespace mrcm;

extern "C" int mrcm_probe_peak(int kind, double seconds, double* tflops, void* cuda_stream) {
    if (!tflops || !(seconds > 0.0) || seconds > 10.0) return MRCM_ERR_INVALID_ARG;
    if (probe_flops_per_thread_iter(kind) == 0.0) return MRCM_ERR_INVALID_ARG;
    *tflops = 0.0;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0, rc;
    if ((rc = cuda_status(cudaGetDevice(&dev))) != MRCM_OK) return rc;
    if ((rc = cuda_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) != MRCM_OK) return rc;
    const int grid = sms * kProbeBlocksPerSM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((rc = cuda_status(cudaEventCreate(&e0))) != MRCM_OK) return rc;
    if ((rc = cuda_status(cudaEventCreate(&e1))) != MRCM_OK) {
        cudaEventDestroy(e0);
        return rc;
    }
    // calibrate the iteration count on a short run, then time three runs of
    // about `seconds` / 3 each and keep the fastest
    double best = 0.0;
    int iters = 256;
    for (int run = 0; run < 5 && rc == MRCM_OK; ++run) {
        float ms = 0.f;
        if ((rc = cuda_status(cudaEventRecord(e0, s))) != MRCM_OK) break;
        if ((rc = cuda_status(probe_launch(kind, grid, iters, s))) != MRCM_OK) break;
        if ((rc = cuda_status(cudaEventRecord(e1, s))) != MRCM_OK) break;
        if ((rc = cuda_status(cudaEventSynchronize(e1))) != MRCM_OK) break;
        if ((rc = cuda_status(cudaEventElapsedTime(&ms, e0, e1))) != MRCM_OK) break;
        const double flops = probe_flops_per_thread_iter(kind) * (double)grid * kProbeThreads * iters;
        if (run >= 2) best = std::max(best, flops / (ms * 1e-3) / 1e12);
        if (run < 2) {
            // next iteration count for a run of seconds / 3
            const double scale = (seconds / 3.0) / std::max(ms * 1e-3, 1e-6);
            const double next = std::min(std::max((double)iters * scale, 256.0), 2.0e9);
            iters = (int)next;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MRCM_OK) return rc;
    *tflops = best;
    return MRCM_OK;
}
