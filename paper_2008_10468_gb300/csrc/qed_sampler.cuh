// Learned inverse-CDF sampler for the photon energy fraction (sm_103a).
//
// The network maps (log10 chi, u) to x = delta^{1/3}, the variable of
// Algorithm 1: 2 -> 64 -> 64 -> 64 -> 1, SiLU hidden layers, logistic output
// anchored at the uniform's logit L = ln(u / (1 - u)):
//   v  = (log10 chi / 2, L / 8)
//   h1 = silu(W1 v + b1), h2 = silu(W2 h1 + b2), h3 = silu(W3 h2 + b3)
//   x  = sigmoid(w4 . h3 + b4 + L)
// The anchor gives x(u -> 0) = 0 and x(u -> 1) = 1 exactly, the end points of
// every inverse CDF of x, and the logit input stretches both tails of u, where
// the inverse CDF is steepest, so that the network sees them on the scale of
// the bulk.
// Parameters are packed W1, b1, W2, b2, W3, b3, w4, b4 (W[out][in] row-major,
// 8577 floats).  Training keeps FP32 master weights and Adam moments; the
// event kernels use a BF16 copy with FP32 accumulation.
//
// Training targets come from the exact inverse CDF of the emission spectrum,
// tabulated on the GPU from the library's acceptance function 3x^2 P(x^3)
// (Eq. 1) on a fine grid of chi and x.  The same table gives the total
// per-sub-step probability per c (the integral bounded by f(b), Sec. 3.1.1),
// which decides events when the sampler replaces the rejection step.
#pragma once
#include <cuda_bf16.h>

#include "qed_device.cuh"

namespace qed {

constexpr int kMlpW = 64;
constexpr int kMlpOffW1 = 0, kMlpOffB1 = 128, kMlpOffW2 = 192, kMlpOffB2 = 4288;
constexpr int kMlpOffW3 = 4352, kMlpOffB3 = 8448, kMlpOffW4 = 8512, kMlpOffB4 = 8576;
constexpr int kMlpParams = 8577;
constexpr float kMlpLog10Lo = -2.0f, kMlpLog10Hi = 2.0f;  // trained chi range

__device__ __forceinline__ float sigmoidf_(float z) { return 1.0f / (1.0f + __expf(-z)); }
// Logit of a uniform in (0, 1) (1 - u is exact for u >= 1/2), the network's
// second input (scaled) and its output anchor.
constexpr float kMlpLogitScale = 0.125f;
__device__ __forceinline__ float logitf_(float u) { return logf(u) - logf(1.0f - u); }
__device__ __forceinline__ float mlp_input_u(float u) { return logitf_(u) * kMlpLogitScale; }
__device__ __forceinline__ float anchor_of_v1(float v1) { return v1 * (1.0f / kMlpLogitScale); }
__device__ __forceinline__ float siluf_(float z) { return z * sigmoidf_(z); }

// ---------------------------------------------------------------------------
// Exact CDF rows.  Row i has chi_i = 10^(lo + i (hi - lo)/(n - 1)); node m has
// x_m = m / M.  cdf[i][m] = int_0^{x_m} P / int_0^1 P (trapezoid rule, FP64
// prefix sums), total[i] = int_0^1 P dx / c.  P is the acceptance function
// of Algorithm 1 (emission, x = delta^{1/3}) or, with `pair`, of Algorithm 2
// (x = delta_e, the electron's energy fraction).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_cdf_rows(float log10_lo, float log10_hi, int nrows,
                                                  int M, int pair, float* __restrict__ cdf,
                                                  float* __restrict__ total) {
    __shared__ SynTable tbl;
    __shared__ double warp_sums[8];
    __shared__ double carry;
    stage_syn_table(tbl);
    __syncthreads();
    const int row = blockIdx.x;
    if (row >= nrows) return;
    const float l10 = log10_lo + (log10_hi - log10_lo) * (float)row / (float)(nrows - 1);
    const float b = 1.5f * exp10f(l10);
    const float b23 = exp2f(__log2f(b) * (2.0f / 3.0f));
    const float dx = 1.0f / (float)M;
    if (threadIdx.x == 0) carry = 0.0;
    __syncthreads();
    float* out = cdf + (size_t)row * (M + 1);
    // chunks of 256 nodes: node m = base + tid, interval [x_{m-1}, x_m]
    for (int base = 1; base <= M; base += 256) {
        const int m = base + threadIdx.x;
        float pm = 0.0f, pprev = 0.0f;
        if (m <= M) {
            float d;
            // emission: x = delta^{1/3}, the density at x -> 0 is kSmallF c b^{2/3};
            // pair production: x = delta_e, the density vanishes at both ends
            pm = m < M ? acceptance(tbl, pair != 0, b, 1.0f, (float)m * dx, &d) : 0.0f;
            pprev = m - 1 == 0 ? (pair ? 0.0f : kSmallF * b23)
                               : acceptance(tbl, pair != 0, b, 1.0f, (float)(m - 1) * dx, &d);
        }
        double a = (m <= M) ? 0.5 * ((double)pm + (double)pprev) * (double)dx : 0.0;
        // inclusive scan within the block
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        double v = a;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) warp_sums[w] = v;
        __syncthreads();
        double off = carry;
        for (int k = 0; k < w; ++k) off += warp_sums[k];
        const double incl = off + v;
        if (m <= M) out[m] = (float)incl;   // unnormalised for now
        __syncthreads();
        if (threadIdx.x == 255) carry = incl;
        __syncthreads();
    }
    const double tot = carry;
    if (threadIdx.x == 0) {
        out[0] = 0.0f;
        total[row] = (float)tot;
    }
    __syncthreads();
    // a row whose probability underflows binary32 (pairs at small chi) keeps
    // total 0 and a uniform CDF, and its bin is never usable
    const float inv = tot > 0.0 ? (float)(1.0 / tot) : 0.0f;
    for (int m = 1 + threadIdx.x; m <= M; m += 256)
        out[m] = tot > 0.0 ? fminf(out[m] * inv, 1.0f) : (float)m / (float)M;
}

// Inverse of one CDF row at u: the node interval by binary search, then
// linear interpolation.
__device__ __forceinline__ float cdf_row_inverse(const float* __restrict__ row, int M, float u) {
    int lo = 0, hi = M;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (row[mid] <= u) lo = mid;
        else hi = mid;
    }
    const float c0 = row[lo], c1 = row[hi];
    const float w = c1 > c0 ? (u - c0) / (c1 - c0) : 0.5f;
    return ((float)lo + w) / (float)M;
}

// CDF of one row at x (linear interpolation between nodes).
__device__ __forceinline__ float cdf_row_at(const float* __restrict__ row, int M, float x) {
    const float p = fminf(fmaxf(x, 0.0f), 1.0f) * (float)M;
    const int m = min((int)p, M - 1);
    const float w = p - (float)m;
    return row[m] + w * (row[m + 1] - row[m]);
}

// Density of one row at x (difference quotient of the node interval).
__device__ __forceinline__ float cdf_row_density(const float* __restrict__ row, int M, float x) {
    const int m = min(max((int)(x * (float)M), 0), M - 1);
    return (row[m + 1] - row[m]) * (float)M;
}

// Training samples: log10 chi uniform in [l10_lo, l10_hi]; u uniform for
// half of the samples and, for the other half, logit u uniform in [-16, 16]
// (the tails of u, where the inverse CDF is steepest, get their own share);
// target x from the two neighbouring CDF rows (linear in log10 chi), and the
// weight p(x), the density of x at the target: with it the squared error
// p^2 (x - t)^2 is, to first order, the squared error of the CDF.
__global__ void k_sampler_batch(uint32_t k0, uint32_t k1, uint32_t batch_index, int B,
                                float l10_lo, float l10_hi,
                                const float* __restrict__ cdf, int nrows, int M,
                                float* __restrict__ v, float* __restrict__ target,
                                float* __restrict__ weight) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    const uint4 r = philox4x32_10(make_uint4((uint32_t)s, batch_index, 0x5A4D4C50u, 0u), k0, k1);
    const float l10 = l10_lo + (l10_hi - l10_lo) * u01(r.x);
    float u, L;
    if (r.z & 1u) {
        u = u01(r.y);
        L = logitf_(u);
    } else {
        L = (2.0f * u01(r.w) - 1.0f) * 16.0f;
        u = 1.0f / (1.0f + expf(-L));
    }
    const float pos = (l10 - kMlpLog10Lo) / (kMlpLog10Hi - kMlpLog10Lo) * (float)(nrows - 1);
    const int i = min((int)pos, nrows - 2);
    const float w = pos - (float)i;
    const float* ra = cdf + (size_t)i * (M + 1);
    const float* rb = cdf + (size_t)(i + 1) * (M + 1);
    const float xa = cdf_row_inverse(ra, M, u);
    const float xb = cdf_row_inverse(rb, M, u);
    const float x = xa + w * (xb - xa);
    v[2 * s] = l10 * 0.5f;
    v[2 * s + 1] = L * kMlpLogitScale;
    target[s] = x;
    if (weight)
        weight[s] = (1.0f - w) * cdf_row_density(ra, M, x) + w * cdf_row_density(rb, M, x);
}

// ---------------------------------------------------------------------------
// Training: forward and backward over tiles of 64 samples per block, weights
// in shared memory with rows padded to 65 floats (conflict-free for both the
// row and the column access), per-block partial gradients.
// ---------------------------------------------------------------------------
constexpr int kTileS = 64;
constexpr int kPad = kMlpW + 1;

struct TrainSmem {
    float W2[kMlpW * kPad], W3[kMlpW * kPad];
    float A1[kTileS * kMlpW], A2[kTileS * kMlpW], A3[kTileS * kMlpW];  // activations
    float Z1[kTileS * kMlpW], Z2[kTileS * kMlpW], Z3[kTileS * kMlpW];  // pre-activations
    float W1[kMlpW * 2], b1[kMlpW], b2[kMlpW], b3[kMlpW], w4[kMlpW];
    float v[kTileS * 2], tgt[kTileS], wgt[kTileS], dout[kTileS];
    float b4;
};

// out[s][n] = bias[n] + sum_j W[n][j] in[s][j] for the tile; thread t owns
// n = t % 64 and 16 consecutive samples.
__device__ __forceinline__ void tile_forward(const float* W, const float* bias, const float* in,
                                             float* z, float* a) {
    const int n = threadIdx.x & 63;
    const int s0 = (threadIdx.x >> 6) * 16;
    float acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = bias[n];
    for (int j = 0; j < kMlpW; ++j) {
        const float w = W[n * kPad + j];
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[k] = fmaf(w, in[(s0 + k) * kMlpW + j], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        z[(s0 + k) * kMlpW + n] = acc[k];
        a[(s0 + k) * kMlpW + n] = siluf_(acc[k]);
    }
}

__device__ __forceinline__ float dsiluf_(float z) {
    const float s = sigmoidf_(z);
    return s * (1.0f + z * (1.0f - s));
}

// Weights as used by the forward pass: with `qat` rounded to BF16 (the form
// the event kernels evaluate), the gradient flowing straight to the FP32
// master weight.
__device__ __forceinline__ float train_weight(float w, int qat) {
    return qat ? __bfloat162float(__float2bfloat16_rn(w)) : w;
}

// CDF and density of the exact spectrum at (log10 chi, x), bilinear in the
// table rows.
__device__ __forceinline__ void cdf_at(const float* __restrict__ cdf, int nrows, int M, float l10,
                                       float x, float* c, float* p) {
    const float pos = (fminf(fmaxf(l10, kMlpLog10Lo), kMlpLog10Hi) - kMlpLog10Lo) /
                      (kMlpLog10Hi - kMlpLog10Lo) * (float)(nrows - 1);
    const int i = min((int)pos, nrows - 2);
    const float w = pos - (float)i;
    const float* ra = cdf + (size_t)i * (M + 1);
    const float* rb = ra + (M + 1);
    *c = (1.0f - w) * cdf_row_at(ra, M, x) + w * cdf_row_at(rb, M, x);
    *p = (1.0f - w) * cdf_row_density(ra, M, x) + w * cdf_row_density(rb, M, x);
}

// Loss modes: targets given (cdf == nullptr): mean(w^2 (x - t)^2); exact CDF
// given: mean((CDF(chi, x) - u)^2), the squared error of the sampler's CDF,
// with its x-derivative p(x) from the table.
__global__ void __launch_bounds__(256) k_mlp_grad(const float* __restrict__ theta,
                                                  const float* __restrict__ v,
                                                  const float* __restrict__ target,
                                                  const float* __restrict__ weight, int B,
                                                  int qat, const float* __restrict__ cdf,
                                                  int nrows, int M, float* __restrict__ partial,
                                                  float* __restrict__ loss_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
    const int t = threadIdx.x;
    for (int i = t; i < kMlpW * kMlpW; i += 256) {
        const int n = i / kMlpW, j = i % kMlpW;
        S.W2[n * kPad + j] = train_weight(theta[kMlpOffW2 + i], qat);
        S.W3[n * kPad + j] = train_weight(theta[kMlpOffW3 + i], qat);
    }
    for (int i = t; i < 128; i += 256) S.W1[i] = train_weight(theta[kMlpOffW1 + i], qat);
    if (t < 64) {
        S.b1[t] = train_weight(theta[kMlpOffB1 + t], qat);
        S.b2[t] = train_weight(theta[kMlpOffB2 + t], qat);
        S.b3[t] = train_weight(theta[kMlpOffB3 + t], qat);
        S.w4[t] = train_weight(theta[kMlpOffW4 + t], qat);
    }
    if (t == 0) S.b4 = train_weight(theta[kMlpOffB4], qat);
    // per-thread gradient accumulators for the entries this thread owns
    // (n = t % 64, a block of 16 in-indices), kept across tiles
    const int n = t & 63;
    const int jb = (t >> 6) * 16;
    float gW3[16], gW2[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) gW3[k] = gW2[k] = 0.0f;
    float gW1[2] = {0.0f, 0.0f};
    float gb1 = 0.0f, gb2 = 0.0f, gb3 = 0.0f, gw4 = 0.0f, gb4 = 0.0f, lsum = 0.0f;
    __syncthreads();
    const int ntiles = (B + kTileS - 1) / kTileS;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int base = tile * kTileS;
        for (int i = t; i < kTileS; i += 256) {
            const int s = base + i;
            const bool ok = s < B;
            S.v[2 * i] = ok ? v[2 * s] : 0.0f;
            S.v[2 * i + 1] = ok ? v[2 * s + 1] : 0.0f;
            S.tgt[i] = ok ? target[s] : -1.0f;  // -1 marks padding
            S.wgt[i] = ok ? (weight ? weight[s] : 1.0f) : 0.0f;
        }
        __syncthreads();
        // layer 1 (2 inputs)
        for (int i = t; i < kTileS * kMlpW; i += 256) {
            const int s = i / kMlpW, m = i % kMlpW;
            const float z = fmaf(S.W1[2 * m], S.v[2 * s], fmaf(S.W1[2 * m + 1], S.v[2 * s + 1], S.b1[m]));
            S.Z1[i] = z;
            S.A1[i] = siluf_(z);
        }
        __syncthreads();
        tile_forward(S.W2, S.b2, S.A1, S.Z2, S.A2);
        __syncthreads();
        tile_forward(S.W3, S.b3, S.A2, S.Z3, S.A3);
        __syncthreads();
        // output and loss: one warp
        if (t < kTileS) {
            float o = S.b4 + anchor_of_v1(S.v[2 * t + 1]);
            for (int j = 0; j < kMlpW; ++j) o = fmaf(S.w4[j], S.A3[t * kMlpW + j], o);
            const float x = sigmoidf_(o);
            const bool ok = S.tgt[t] >= 0.0f;
            float r, slope;
            if (cdf) {
                // residual in CDF space at the network's output
                float c, p;
                cdf_at(cdf, nrows, M, 2.0f * S.v[2 * t], x, &c, &p);
                const float u = 1.0f / (1.0f + expf(-anchor_of_v1(S.v[2 * t + 1])));
                r = ok ? c - u : 0.0f;
                slope = p;
            } else {
                r = ok ? S.wgt[t] * (x - S.tgt[t]) : 0.0f;
                slope = S.wgt[t];
            }
            lsum += r * r;
            S.dout[t] = (2.0f / (float)B) * r * slope * x * (1.0f - x);
        }
        __syncthreads();
        // dZ3 = dout * w4 * silu'(Z3), in place of Z3; output-layer gradients
        for (int i = t; i < kTileS * kMlpW; i += 256) {
            const int s = i / kMlpW, m = i % kMlpW;
            S.Z3[i] = S.dout[s] * S.w4[m] * dsiluf_(S.Z3[i]);
        }
        if (t < kMlpW) {
            float a = 0.0f;
            for (int s = 0; s < kTileS; ++s) a = fmaf(S.dout[s], S.A3[s * kMlpW + t], a);
            gw4 += a;
        }
        if (t == 0)
            for (int s = 0; s < kTileS; ++s) gb4 += S.dout[s];
        __syncthreads();
        // dW3[n][j] = sum_s dZ3[s][n] A2[s][j]; db3
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float a = 0.0f;
            for (int s = 0; s < kTileS; ++s) a = fmaf(S.Z3[s * kMlpW + n], S.A2[s * kMlpW + jb + k], a);
            gW3[k] += a;
        }
        if (t < kMlpW)
            for (int s = 0; s < kTileS; ++s) gb3 += S.Z3[s * kMlpW + t];
        // dA2[s][j] = sum_n W3[n][j] dZ3[s][n] -> dZ2 = dA2 * silu'(Z2), into A1's
        // partner buffer: use A3 (no longer needed) as dZ2
        {
            const int j = t & 63;
            const int s0 = (t >> 6) * 16;
            for (int k = 0; k < 16; ++k) {
                const int s = s0 + k;
                float a = 0.0f;
                for (int m = 0; m < kMlpW; ++m) a = fmaf(S.W3[m * kPad + j], S.Z3[s * kMlpW + m], a);
                S.A3[s * kMlpW + j] = a * dsiluf_(S.Z2[s * kMlpW + j]);
            }
        }
        __syncthreads();
        // dW2[n][j] = sum_s dZ2[s][n] A1[s][j]; db2
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float a = 0.0f;
            for (int s = 0; s < kTileS; ++s) a = fmaf(S.A3[s * kMlpW + n], S.A1[s * kMlpW + jb + k], a);
            gW2[k] += a;
        }
        if (t < kMlpW)
            for (int s = 0; s < kTileS; ++s) gb2 += S.A3[s * kMlpW + t];
        // dA1[s][j] = sum_n W2[n][j] dZ2[s][n] -> dZ1 into Z2 (no longer needed)
        {
            const int j = t & 63;
            const int s0 = (t >> 6) * 16;
            for (int k = 0; k < 16; ++k) {
                const int s = s0 + k;
                float a = 0.0f;
                for (int m = 0; m < kMlpW; ++m) a = fmaf(S.W2[m * kPad + j], S.A3[s * kMlpW + m], a);
                S.Z2[s * kMlpW + j] = a * dsiluf_(S.Z1[s * kMlpW + j]);
            }
        }
        __syncthreads();
        // dW1[m][0..1] = sum_s dZ1[s][m] v[s][0..1]; db1
        if (t < kMlpW) {
            float a0 = 0.0f, a1 = 0.0f, bb = 0.0f;
            for (int s = 0; s < kTileS; ++s) {
                const float d = S.Z2[s * kMlpW + t];
                a0 = fmaf(d, S.v[2 * s], a0);
                a1 = fmaf(d, S.v[2 * s + 1], a1);
                bb += d;
            }
            gW1[0] += a0;
            gW1[1] += a1;
            gb1 += bb;
        }
        __syncthreads();
    }
    float* out = partial + (size_t)blockIdx.x * kMlpParams;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        out[kMlpOffW3 + n * kMlpW + jb + k] = gW3[k];
        out[kMlpOffW2 + n * kMlpW + jb + k] = gW2[k];
    }
    if (t < kMlpW) {
        out[kMlpOffW1 + 2 * t] = gW1[0];
        out[kMlpOffW1 + 2 * t + 1] = gW1[1];
        out[kMlpOffB1 + t] = gb1;
        out[kMlpOffB2 + t] = gb2;
        out[kMlpOffB3 + t] = gb3;
        out[kMlpOffW4 + t] = gw4;
    }
    if (t == 0) out[kMlpOffB4] = gb4;
    // loss: sum over the tile's first warp (threads 0..63 held samples)
    float l = lsum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((t & 31) == 0 && t < kTileS && loss_out) atomicAdd(loss_out, l / (float)B);
}

// Sum the partial gradients; optionally apply one Adam step and refresh the
// BF16 copy.  grad_out (nullable) receives the summed gradient.
__global__ void k_mlp_adam(const float* __restrict__ partial, int nparts, float* __restrict__ theta,
                           float* __restrict__ m1, float* __restrict__ m2,
                           __nv_bfloat16* __restrict__ wbf, float lr, float beta1, float beta2,
                           float eps, float bc1, float bc2, int apply, float* __restrict__ grad_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    float g = 0.0f;
    for (int p = 0; p < nparts; ++p) g += partial[(size_t)p * kMlpParams + i];
    if (grad_out) grad_out[i] = g;
    if (!apply) return;
    const float a = beta1 * m1[i] + (1.0f - beta1) * g;
    const float b = beta2 * m2[i] + (1.0f - beta2) * g * g;
    m1[i] = a;
    m2[i] = b;
    const float th = theta[i] - lr * (a / bc1) / (sqrtf(b / bc2) + eps);
    theta[i] = th;
    wbf[i] = __float2bfloat16_rn(th);
}

// ---------------------------------------------------------------------------
// Inference with BF16 weights and FP32 accumulation.  Each output neuron is a
// dot product taken in the order j = 0..63, the same in the warp-cooperative
// and the per-thread forms, so both give the same result.  The hidden-layer
// weights are staged once as FP32 (the BF16 values, converted exactly), so
// that the dot products take no conversion per weight.
// ---------------------------------------------------------------------------
constexpr int kWPad = kMlpW + 4;   // FP32 row stride: 68 (16-byte rows; the
                                   // 128-bit loads of 8 lanes hit distinct banks)

struct SamplerSmem {
    __align__(16) float W2[kMlpW * kWPad];
    __align__(16) float W3[kMlpW * kWPad];
    float W1[kMlpW * 2], b1[kMlpW], b2[kMlpW], b3[kMlpW], w4[kMlpW];
    float b4;
    float wtot[1024];                 // total probability per c along log10 chi
    unsigned long long bin_ok;        // bit k: chi bin k within the error limit
    int nrows;
    __align__(16) float h[8][kMlpW];  // per-warp activation buffer (up to 8 warps)
};

__device__ __forceinline__ void stage_sampler(SamplerSmem& S, const __nv_bfloat16* __restrict__ w,
                                              const float* __restrict__ wtot, int nrows,
                                              unsigned long long bin_ok) {
    for (int i = threadIdx.x; i < kMlpW * kMlpW; i += blockDim.x) {
        const int n = i / kMlpW, j = i % kMlpW;
        S.W2[n * kWPad + j] = __bfloat162float(w[kMlpOffW2 + i]);
        S.W3[n * kWPad + j] = __bfloat162float(w[kMlpOffW3 + i]);
    }
    for (int i = threadIdx.x; i < 128; i += blockDim.x) S.W1[i] = __bfloat162float(w[kMlpOffW1 + i]);
    for (int i = threadIdx.x; i < kMlpW; i += blockDim.x) {
        S.b1[i] = __bfloat162float(w[kMlpOffB1 + i]);
        S.b2[i] = __bfloat162float(w[kMlpOffB2 + i]);
        S.b3[i] = __bfloat162float(w[kMlpOffB3 + i]);
        S.w4[i] = __bfloat162float(w[kMlpOffW4 + i]);
    }
    for (int i = threadIdx.x; i < nrows && i < 1024; i += blockDim.x) S.wtot[i] = wtot[i];
    if (threadIdx.x == 0) {
        S.b4 = __bfloat162float(w[kMlpOffB4]);
        S.bin_ok = bin_ok;
        S.nrows = nrows;
    }
}

__device__ __forceinline__ float neuron_dot(const float* __restrict__ row,
                                            const float* __restrict__ h, float acc) {
#pragma unroll 8
    for (int j = 0; j < kMlpW; ++j) acc = fmaf(row[j], h[j], acc);
    return acc;
}

// Two neurons of one lane, sharing the activation loads: weights and
// activations read four at a time (128-bit loads), products accumulated in
// FP32 in the order j = 0..63 (the order of neuron_dot, so both forms give
// identical results).
__device__ __forceinline__ void neuron_dot2(const float* __restrict__ row0,
                                            const float* __restrict__ row1,
                                            const float* __restrict__ h, float& acc0,
                                            float& acc1) {
#pragma unroll 4
    for (int j = 0; j < kMlpW; j += 4) {
        const float4 hv = *reinterpret_cast<const float4*>(h + j);
        const float4 w0 = *reinterpret_cast<const float4*>(row0 + j);
        const float4 w1 = *reinterpret_cast<const float4*>(row1 + j);
        acc0 = fmaf(w0.x, hv.x, acc0);
        acc0 = fmaf(w0.y, hv.y, acc0);
        acc0 = fmaf(w0.z, hv.z, acc0);
        acc0 = fmaf(w0.w, hv.w, acc0);
        acc1 = fmaf(w1.x, hv.x, acc1);
        acc1 = fmaf(w1.y, hv.y, acc1);
        acc1 = fmaf(w1.z, hv.z, acc1);
        acc1 = fmaf(w1.w, hv.w, acc1);
    }
}

// All 32 lanes of a warp evaluate x(v0, v1) together; every lane gets x.
// Lane l owns neurons l and l + 32 of each hidden layer.
__device__ __forceinline__ float mlp_infer_warp(SamplerSmem& S, float v0, float v1) {
    const int lane = threadIdx.x & 31;
    float* h = S.h[(threadIdx.x >> 5) & 7];
    float a0 = siluf_(fmaf(S.W1[2 * lane], v0, fmaf(S.W1[2 * lane + 1], v1, S.b1[lane])));
    float a1 = siluf_(fmaf(S.W1[2 * (lane + 32)], v0,
                           fmaf(S.W1[2 * (lane + 32) + 1], v1, S.b1[lane + 32])));
    __syncwarp();
    h[lane] = a0;
    h[lane + 32] = a1;
    __syncwarp();
    a0 = S.b2[lane];
    a1 = S.b2[lane + 32];
    neuron_dot2(S.W2 + lane * kWPad, S.W2 + (lane + 32) * kWPad, h, a0, a1);
    a0 = siluf_(a0);
    a1 = siluf_(a1);
    __syncwarp();
    h[lane] = a0;
    h[lane + 32] = a1;
    __syncwarp();
    a0 = S.b3[lane];
    a1 = S.b3[lane + 32];
    neuron_dot2(S.W3 + lane * kWPad, S.W3 + (lane + 32) * kWPad, h, a0, a1);
    float o = fmaf(S.w4[lane], siluf_(a0), 0.0f);
    o = fmaf(S.w4[lane + 32], siluf_(a1), o);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) o += __shfl_xor_sync(0xffffffffu, o, off);
    __syncwarp();
    return sigmoidf_(o + S.b4 + anchor_of_v1(v1));
}

// Tabulated total probability per c at b = 3 chi / 2 (linear in log10 chi,
// on the logarithm of the table values); chi must be inside the trained range.
__device__ __forceinline__ float wtot_at(const float* wtot, int nrows, float chi) {
    const float pos = (log10f(chi) - kMlpLog10Lo) / (kMlpLog10Hi - kMlpLog10Lo) * (float)(nrows - 1);
    const int i = min(max((int)pos, 0), nrows - 2);
    const float w = pos - (float)i;
    return __expf((1.0f - w) * __logf(wtot[i]) + w * __logf(wtot[i + 1]));
}
__device__ __forceinline__ float sampler_wtot(const SamplerSmem& S, float chi) {
    return wtot_at(S.wtot, S.nrows, chi);
}

// ---------------------------------------------------------------------------
// Tensor-core form of the inference: the 32 lanes of a warp evaluate their 32
// samples together, one sample (row) per lane, as two tiles of 16 rows through
// mma.sync m16n8k16 (BF16 x BF16 -> FP32).  The weights are the BF16 values
// themselves.  Each activation enters the next layer as two BF16 numbers,
// hi = bf16(a) and lo = bf16(a - hi), with two products per tile, so that the
// activations keep ~16 significant bits (BF16 activations alone gave a CDF
// error of 2e-3).  The accumulator fragment of one layer (rows g, g + 8,
// columns 2t, 2t + 1 of each 8-column tile, g = lane / 4, t = lane % 4) is the
// A fragment of the next one for the same rows, so activations stay in
// registers between layers.  A row's result depends on that row's inputs only.
// ---------------------------------------------------------------------------
constexpr int kHPad = 72;   // BF16 row stride of W2, W3 ([n][k], 64 + 8): the
                            // 32-bit fragment loads of a warp hit 32 banks

struct SamplerMma {
    __align__(16) __nv_bfloat16 W2[kMlpW * kHPad];
    __align__(16) __nv_bfloat16 W3[kMlpW * kHPad];
    float W1[kMlpW * 2], b1[kMlpW], b2[kMlpW], b3[kMlpW], w4[kMlpW];
    float b4;
    float wtot[1024];
    unsigned long long bin_ok;
    int nrows;
};

__device__ __forceinline__ void stage_sampler_mma(SamplerMma& S, const __nv_bfloat16* __restrict__ w,
                                                  const float* __restrict__ wtot, int nrows,
                                                  unsigned long long bin_ok) {
    for (int i = threadIdx.x; i < kMlpW * kMlpW; i += blockDim.x) {
        const int n = i / kMlpW, k = i % kMlpW;
        S.W2[n * kHPad + k] = w[kMlpOffW2 + i];
        S.W3[n * kHPad + k] = w[kMlpOffW3 + i];
    }
    for (int i = threadIdx.x; i < 128; i += blockDim.x) S.W1[i] = __bfloat162float(w[kMlpOffW1 + i]);
    for (int i = threadIdx.x; i < kMlpW; i += blockDim.x) {
        S.b1[i] = __bfloat162float(w[kMlpOffB1 + i]);
        S.b2[i] = __bfloat162float(w[kMlpOffB2 + i]);
        S.b3[i] = __bfloat162float(w[kMlpOffB3 + i]);
        S.w4[i] = __bfloat162float(w[kMlpOffW4 + i]);
    }
    for (int i = threadIdx.x; i < nrows && i < 1024; i += blockDim.x) S.wtot[i] = wtot[i];
    if (threadIdx.x == 0) {
        S.b4 = __bfloat162float(w[kMlpOffB4]);
        S.bin_ok = bin_ok;
        S.nrows = nrows;
    }
}

// D += A B for one m16n8k16 tile (A: 4 registers of BF16 pairs, B: 2).
__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                          uint32_t b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// (x0, x1) as BF16 pairs: hi rounds each value, lo rounds what hi leaves.
__device__ __forceinline__ void split_bf16x2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);   // .x (low half) = x0
    const __nv_bfloat162 l =
        __floats2bfloat162_rn(x0 - __low2float(h), x1 - __high2float(h));
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ float silu_fast(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

// One hidden layer for one 16-row tile: C = W a + b from the A fragments
// (hi, lo) of the layer below, then SiLU; the result replaces (hi, lo).
// upper = false: rows 8..15 of the tile hold no sample; their activations are
// left at 0 instead of going through SiLU (rows do not mix in the products, so
// the other rows' results are unchanged).
__device__ __forceinline__ void mma_hidden(const __nv_bfloat16* __restrict__ W,
                                           const float* __restrict__ bias, uint32_t (&Ah)[4][4],
                                           uint32_t (&Al)[4][4], bool upper) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float C[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float b0 = bias[8 * nt + 2 * t], b1 = bias[8 * nt + 2 * t + 1];
        C[nt][0] = b0;
        C[nt][1] = b1;
        C[nt][2] = b0;
        C[nt][3] = b1;
    }
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const __nv_bfloat16* row = W + (8 * nt + g) * kHPad + 16 * kt + 2 * t;
            const uint32_t b0 = *reinterpret_cast<const uint32_t*>(row);
            const uint32_t b1 = *reinterpret_cast<const uint32_t*>(row + 8);
            mma_16816(C[nt], Ah[kt], b0, b1);
            mma_16816(C[nt], Al[kt], b0, b1);
        }
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int kt = nt >> 1, q = (nt & 1) * 2;
        split_bf16x2(silu_fast(C[nt][0]), silu_fast(C[nt][1]), Ah[kt][q], Al[kt][q]);
    }
    if (upper) {
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int kt = nt >> 1, q = (nt & 1) * 2;
            split_bf16x2(silu_fast(C[nt][2]), silu_fast(C[nt][3]), Ah[kt][q + 1], Al[kt][q + 1]);
        }
    } else {
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            Ah[kt][1] = Ah[kt][3] = 0u;
            Al[kt][1] = Al[kt][3] = 0u;
        }
    }
}

// The network's output logit (before b4 and the anchor) for rows g and g + 8
// of one tile, whose inputs are (v0a, v1a) and (v0b, v1b); every lane of the
// group g gets both (upper = false: rows g + 8 hold no sample, ob is 0).
__device__ __forceinline__ void mma_tile(const SamplerMma& S, float v0a, float v1a, float v0b,
                                         float v1b, float& oa, float& ob, bool upper = true) {
    const int lane = threadIdx.x & 31, t = lane & 3;
    uint32_t Ah[4][4], Al[4][4];
    // layer 1 (two inputs) on the CUDA cores, in the fragment layout
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int n = 8 * nt + 2 * t;
        const float w00 = S.W1[2 * n], w01 = S.W1[2 * n + 1];
        const float w10 = S.W1[2 * n + 2], w11 = S.W1[2 * n + 3];
        const float za0 = fmaf(w00, v0a, fmaf(w01, v1a, S.b1[n]));
        const float za1 = fmaf(w10, v0a, fmaf(w11, v1a, S.b1[n + 1]));
        const int kt = nt >> 1, q = (nt & 1) * 2;
        split_bf16x2(silu_fast(za0), silu_fast(za1), Ah[kt][q], Al[kt][q]);
        Ah[kt][q + 1] = Al[kt][q + 1] = 0u;
        if (upper) {
            const float zb0 = fmaf(w00, v0b, fmaf(w01, v1b, S.b1[n]));
            const float zb1 = fmaf(w10, v0b, fmaf(w11, v1b, S.b1[n + 1]));
            split_bf16x2(silu_fast(zb0), silu_fast(zb1), Ah[kt][q + 1], Al[kt][q + 1]);
        }
    }
    mma_hidden(S.W2, S.b2, Ah, Al, upper);
    // layer 3 and the output dot product with w4
    const int g = lane >> 2;
    float C[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float b0 = S.b3[8 * nt + 2 * t], b1 = S.b3[8 * nt + 2 * t + 1];
        C[nt][0] = b0;
        C[nt][1] = b1;
        C[nt][2] = b0;
        C[nt][3] = b1;
    }
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const __nv_bfloat16* row = S.W3 + (8 * nt + g) * kHPad + 16 * kt + 2 * t;
            const uint32_t b0 = *reinterpret_cast<const uint32_t*>(row);
            const uint32_t b1 = *reinterpret_cast<const uint32_t*>(row + 8);
            mma_16816(C[nt], Ah[kt], b0, b1);
            mma_16816(C[nt], Al[kt], b0, b1);
        }
    }
    float pa = 0.0f, pb = 0.0f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float w0 = S.w4[8 * nt + 2 * t], w1 = S.w4[8 * nt + 2 * t + 1];
        pa = fmaf(w0, silu_fast(C[nt][0]), fmaf(w1, silu_fast(C[nt][1]), pa));
    }
    if (upper) {
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float w0 = S.w4[8 * nt + 2 * t], w1 = S.w4[8 * nt + 2 * t + 1];
            pb = fmaf(w0, silu_fast(C[nt][2]), fmaf(w1, silu_fast(C[nt][3]), pb));
        }
    }
    pa += __shfl_xor_sync(0xffffffffu, pa, 1);
    pa += __shfl_xor_sync(0xffffffffu, pa, 2);
    pb += __shfl_xor_sync(0xffffffffu, pb, 1);
    pb += __shfl_xor_sync(0xffffffffu, pb, 2);
    oa = pa;
    ob = pb;
}

// x(v0, v1) for the lanes with `want` set, the others get 0; called by all 32
// lanes together.  The wanted samples are packed into the first rows (in lane
// order), so that a warp with at most 16 of them runs one tile: the result of
// a sample does not depend on its row or on the other rows.  `buf` is this
// warp's staging area in shared memory.
struct MmaBuf {
    float2 in[32];
    float out[32];
};
__device__ __forceinline__ float mlp_infer_mma_some(const SamplerMma& S, MmaBuf& buf, bool want,
                                                    float v0, float v1) {
    constexpr unsigned int kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const unsigned int m = __ballot_sync(kAll, want);
    const int n = __popc(m);
    const int rank = __popc(m & ((1u << lane) - 1u));
    if (want) buf.in[rank] = make_float2(v0, v1);
    __syncwarp();
    const int tiles = (n + 15) >> 4;
#pragma unroll 1
    for (int mt = 0; mt < tiles; ++mt) {
        const int ra = 16 * mt + g, rb = ra + 8;
        const float2 a = ra < n ? buf.in[ra] : make_float2(0.0f, 0.0f);
        const float2 b = rb < n ? buf.in[rb] : make_float2(0.0f, 0.0f);
        float oa, ob;
        mma_tile(S, a.x, a.y, b.x, b.y, oa, ob, n - 16 * mt > 8);
        if (t == 0) {
            buf.out[ra] = oa;
            buf.out[rb] = ob;
        }
    }
    __syncwarp();
    const float o = want ? buf.out[rank] : 0.0f;
    __syncwarp();   // buf is reused by the next call
    return want ? sigmoidf_(o + S.b4 + anchor_of_v1(v1)) : 0.0f;
}

// One sample through the tensor-core form, for a warp that steps one particle
// (lane 0's inputs; every lane gets x).  Out of line, so that the kernels that
// call it do not carry its registers on their other paths.
__device__ __noinline__ float mlp_infer_mma_one(const SamplerMma& S, MmaBuf& buf, float v0,
                                                float v1) {
    const float x = mlp_infer_mma_some(S, buf, (threadIdx.x & 31) == 0, v0, v1);
    return __shfl_sync(0xffffffffu, x, 0);
}

// Dynamic shared memory of the event kernels in a sampler mode: mode 1 the
// FP32 form (SamplerSmem), mode 2 the tensor-core form (SamplerMma) of the
// emission and the pair networks followed by one MmaBuf per warp (up to 8
// warps per block).
// Mode 2 holds the emission network, then the pair network, then the buffers.
constexpr size_t kMmaSmemBytes = 2 * sizeof(SamplerMma) + 8 * sizeof(MmaBuf);
constexpr size_t kNetSmemBytes =
    sizeof(SamplerSmem) > kMmaSmemBytes ? sizeof(SamplerSmem) : kMmaSmemBytes;
__device__ __forceinline__ SamplerMma& pair_mma(unsigned char* dyn) {
    return *reinterpret_cast<SamplerMma*>(dyn + sizeof(SamplerMma));
}
__device__ __forceinline__ MmaBuf& warp_mma_buf(unsigned char* dyn) {
    return reinterpret_cast<MmaBuf*>(dyn + 2 * sizeof(SamplerMma))[(threadIdx.x >> 5) & 7];
}

// x(v0, v1) for the sample of every lane; called by all 32 lanes together.
__device__ __forceinline__ float mlp_infer_mma(const SamplerMma& S, float v0, float v1) {
    constexpr unsigned int kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31, g = lane >> 2;
    float out = 0.0f;
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
        // rows 16 mt + g and 16 mt + g + 8 are the samples of those lanes
        const int ra = 16 * mt + g, rb = ra + 8;
        const float v0a = __shfl_sync(kAll, v0, ra), v1a = __shfl_sync(kAll, v1, ra);
        const float v0b = __shfl_sync(kAll, v0, rb), v1b = __shfl_sync(kAll, v1, rb);
        float oa, ob;
        mma_tile(S, v0a, v1a, v0b, v1b, oa, ob);
        // lane 16 mt + r takes its row from lane 4 (r % 8), first of group r % 8
        const int src = 4 * (lane & 7);
        const float ga = __shfl_sync(kAll, oa, src), gb = __shfl_sync(kAll, ob, src);
        if ((lane >> 4) == mt) out = (lane & 8) ? gb : ga;
    }
    return sigmoidf_(out + S.b4 + anchor_of_v1(v1));
}

}  // namespace qed
