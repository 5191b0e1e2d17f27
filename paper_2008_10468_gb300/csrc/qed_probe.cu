// Peak probes of the arithmetic the event kernels run on (sm_103a): the rate
// of 32 x 32 -> 64-bit multiplies as Philox4x32-10 issues them (the high and
// the low word of each product, the hot pass's dominant work), of binary32
// fused multiply-adds, of special-function exp2 and of plain integer ALU
// operations.  Each thread runs eight independent chains, so that the rate
// is the pipe's, not one chain's latency.  Not part of the paper's method:
// the denominators of the event kernels' roofline, measured on the GPU at
// hand instead of taken from unit counts.
#include <cstdint>
#include <cuda_runtime.h>

#include "qed.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

// Operations counted per chain step: mul 2 (high and low word), fma 2 (flops),
// ex2 1, alu 2 (an xor-add pair).
template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_probe(long long iters, uint32_t seed,
                                                         unsigned int* sink) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (KIND == QED_PROBE_MUL32) {
        uint32_t a[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = t * 0x9E3779B9u + seed + (uint32_t)c;
        for (long long k = 0; k < iters; ++k) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                const uint32_t hi = __umulhi(0xD2511F53u, a[c]);
                const uint32_t lo = 0xD2511F53u * a[c];
                a[c] = hi ^ lo;
            }
        }
        uint32_t r = 0;
#pragma unroll
        for (int c = 0; c < kChains; ++c) r ^= a[c];
        if (r == 0x12345678u) atomicAdd(sink, 1u);
    } else if (KIND == QED_PROBE_FMA32) {
        float x[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = 1.0f + 1e-6f * (float)((t + c) & 1023);
        for (long long k = 0; k < iters; ++k) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], 0.9999999f, 1e-7f);
        }
        float r = 0.0f;
#pragma unroll
        for (int c = 0; c < kChains; ++c) r += x[c];
        if (r == 12345.0f) atomicAdd(sink, 1u);
    } else if (KIND == QED_PROBE_EX2) {
        float x[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = -1e-3f * (float)((t + c) & 1023);
        for (long long k = 0; k < iters; ++k) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                float y;
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[c]));
                x[c] = -y;   // stays in [-1, 0): the chain never over- or underflows
            }
        }
        float r = 0.0f;
#pragma unroll
        for (int c = 0; c < kChains; ++c) r += x[c];
        if (r == 12345.0f) atomicAdd(sink, 1u);
    } else {
        uint32_t a[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = t + seed * (uint32_t)(c + 1);
        for (long long k = 0; k < iters; ++k) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = (a[c] ^ 0x5bd1e995u) + (uint32_t)c;
        }
        uint32_t r = 0;
#pragma unroll
        for (int c = 0; c < kChains; ++c) r ^= a[c];
        if (r == 0x12345678u) atomicAdd(sink, 1u);
    }
}

template <int KIND>
double ops_per_step() {
    return KIND == QED_PROBE_EX2 ? 1.0 : 2.0;
}

template <int KIND>
qed_status run_probe(long long iters, int blocks, cudaStream_t s, unsigned int* sink,
                     double* ops_per_s, double* ms_out) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return QED_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return QED_ERR_CUDA;
    }
    k_probe<KIND><<<blocks, kProbeThreads, 0, s>>>(iters / 16, 1u, sink);   // warm-up
    cudaEventRecord(e0, s);
    k_probe<KIND><<<blocks, kProbeThreads, 0, s>>>(iters, 2u, sink);
    cudaEventRecord(e1, s);
    qed_status st = QED_OK;
    float ms = 0.0f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        st = QED_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != QED_OK) return st;
    const double ops = (double)blocks * kProbeThreads * kChains * (double)iters * ops_per_step<KIND>();
    *ops_per_s = ops / ((double)ms * 1e-3);
    if (ms_out) *ms_out = (double)ms;
    return QED_OK;
}

}  // namespace

extern "C" qed_status qed_peak_probe(int kind, int64_t iters, double* ops_per_s, double* ms,
                                     void* stream) {
    if (!ops_per_s || iters <= 0 || kind < 0 || kind > QED_PROBE_ALU) return QED_ERR_ARG;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return QED_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe<QED_PROBE_MUL32>,
                                                      kProbeThreads, 0) != cudaSuccess)
        return QED_ERR_CUDA;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    // the probes allocate nothing but this one word
    unsigned int* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(unsigned int)) != cudaSuccess) return QED_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    qed_status st;
    switch (kind) {
        case QED_PROBE_MUL32: st = run_probe<QED_PROBE_MUL32>(iters, blocks, s, sink, ops_per_s, ms); break;
        case QED_PROBE_FMA32: st = run_probe<QED_PROBE_FMA32>(iters, blocks, s, sink, ops_per_s, ms); break;
        case QED_PROBE_EX2: st = run_probe<QED_PROBE_EX2>(iters, blocks, s, sink, ops_per_s, ms); break;
        default: st = run_probe<QED_PROBE_ALU>(iters, blocks, s, sink, ops_per_s, ms); break;
    }
    cudaFree(sink);
    return st;
}
