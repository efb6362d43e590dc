// Integer issue-rate microbenchmark: the ceiling against which the fused
// tail's integer throughput is reported.  The tail's work is bit logic,
// population counts and integer adds on 32-bit words; this kernel issues the
// same instruction kinds in independent dependent chains (eight per thread,
// enough to hide the pipeline latency) and reports operations per second.
#include <cuda_runtime.h>

#include <cstdint>

#include "mapa_ctx.h"
#include "mapa_engine.h"

namespace mapa {
namespace {

constexpr int kProbeChains = 8;

// kind 0: per chain and iteration one lop3 and one add (2 ops);
// kind 1: one lop3, one popc and one add (3 ops, a third of them popc, about
// the share of population counts in the score increment).
template <int Kind>
__global__ void __launch_bounds__(256) k_int_mix(uint32_t seed, int iters, uint32_t *sink) {
    uint32_t a[kProbeChains];
    const uint32_t b = seed * 2654435761u + blockIdx.x, c = seed ^ 0x5bd1e995u;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) a[j] = (threadIdx.x + 1u) * (2u * j + 1u) ^ seed;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) {
            uint32_t t;
            asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[j]) : "r"(b), "r"(c));
            if constexpr (Kind == 1) {
                asm volatile("popc.b32 %0, %1;" : "=r"(t) : "r"(a[j]));
            } else {
                t = b;
            }
            asm volatile("add.u32 %0, %0, %1;" : "+r"(a[j]) : "r"(t));
        }
    }
    uint32_t x = 0u;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) x ^= a[j];
    if (x == 0x9E3779B9u) sink[0] = x;  // keeps the chains live
}

}  // namespace
}  // namespace mapa

int mapa_measure_int_peak(mapa_ctx ctx, int32_t kind, double *ops_per_s) {
    if (!ctx || !ops_per_s || (kind != 0 && kind != 1)) return MAPA_E_INVALID;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return MAPA_E_CUDA;
    cudaStream_t st = mapa::engine_stream(ctx->engine);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const unsigned grid = static_cast<unsigned>(sms > 0 ? sms : 1) * 8u;  // 8 blocks of 256 per SM: 64 warps
    const int iters = 8192;
    uint32_t *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = MAPA_OK;
    if (cudaMalloc(&sink, 4) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        rc = MAPA_E_CUDA;
    }
    float best = 0.f;
    for (int rep = 0; rc == MAPA_OK && rep < 4; ++rep) {
        cudaEventRecord(e0, st);
        if (kind == 0) mapa::k_int_mix<0><<<grid, 256, 0, st>>>(12345u + rep, iters, sink);
        else mapa::k_int_mix<1><<<grid, 256, 0, st>>>(12345u + rep, iters, sink);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = MAPA_E_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;  // the first launch warms up
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (rc != MAPA_OK) return rc;
    const double ops = static_cast<double>(grid) * 256.0 * mapa::kProbeChains * iters * (kind == 0 ? 2.0 : 3.0);
    *ops_per_s = best > 0.f ? ops / (best * 1e-3) : 0.0;
    return MAPA_OK;
}
