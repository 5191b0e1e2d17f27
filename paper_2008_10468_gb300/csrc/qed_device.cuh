// Device building blocks of the QED event generator (sm_103a).
//
//   - Philox4x32-10 (Salmon et al., SC'11) and the open-interval uniform;
//   - the quantum parameter chi (Sec. 2.2) in float-float arithmetic;
//   - the synchrotron functions F and G (Sec. 3.2.1) from the octave tables of
//     synchro_coeffs.h, staged in shared memory;
//   - the rate bounds f(b) of Sec. 3.1.1 and the sub-step planner;
//   - the acceptance functions of Algorithms 1 and 2.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define QED_TABLE_ATTR __device__
#include "synchro_coeffs.h"

namespace qed {

// ---------------------------------------------------------------------------
// Philox4x32-10: ten rounds of two 32x32->64 multiplies with key bumps by the
// Weyl constants (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// ((r >> 9) + 1/2) * 2^-23: open interval (0, 1), exact in binary32.
__device__ __forceinline__ float u01(uint32_t r) {
    return fmaf((float)(r >> 9), 0x1p-23f, 0x1p-24f);
}

// Domain-separation constants of the child-id stream (the draw stream uses
// the seed itself as key).
constexpr uint32_t kChildKeyLo = 0xA511E9B3u;
constexpr uint32_t kChildKeyHi = 0x63C1D2F5u;

// ---------------------------------------------------------------------------
// Float-float arithmetic (error-free transformations with FMA).  Explicit
// _rn intrinsics keep the compiler from contracting or reassociating.
// ---------------------------------------------------------------------------
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = two_sum(a.hi, b.hi);
    const float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, lo);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    ff p = two_prod(a.hi, b.hi);
    const float lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, lo);
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    ff p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
__device__ __forceinline__ ff ff_sqrt(ff a) {
    if (!(a.hi > 0.0f)) return {0.0f, 0.0f};
    const float s = __fsqrt_rn(a.hi);
    // one Newton correction: (a - s^2) / (2 s)
    const ff s2 = two_prod(s, s);
    const float r = __fadd_rn(__fadd_rn(__fsub_rn(a.hi, s2.hi), -s2.lo), a.lo);
    return fast_two_sum(s, __fdiv_rn(r, __fmul_rn(2.0f, s)));
}

// chi = sqrt((eps E + p x B)^2 - (p . E)^2) / E_s with eps = sqrt(1 + p^2)
// (e+-) or |p| (photon), Sec. 2.2.  The difference of squares cancels for
// particles co-moving with a crossed field, so every product is kept exact.
// Returns chi; *eps_out receives eps rounded to binary32.
__device__ __forceinline__ float chi_ff(bool photon, float px, float py, float pz, float Ex,
                                        float Ey, float Ez, float Bx, float By, float Bz,
                                        float inv_Es, float* eps_out) {
    const ff p2 = ff_add(ff_add(two_prod(px, px), two_prod(py, py)), two_prod(pz, pz));
    const ff g2 = photon ? p2 : ff_add(p2, ff{1.0f, 0.0f});
    const ff eps = ff_sqrt(g2);
    const ff ax = ff_add(ff_mul_f(eps, Ex), ff_add(two_prod(py, Bz), ff_neg(two_prod(pz, By))));
    const ff ay = ff_add(ff_mul_f(eps, Ey), ff_add(two_prod(pz, Bx), ff_neg(two_prod(px, Bz))));
    const ff az = ff_add(ff_mul_f(eps, Ez), ff_add(two_prod(px, By), ff_neg(two_prod(py, Bx))));
    const ff pe = ff_add(ff_add(two_prod(px, Ex), two_prod(py, Ey)), two_prod(pz, Ez));
    const ff a2 = ff_add(ff_add(ff_mul(ax, ax), ff_mul(ay, ay)), ff_mul(az, az));
    const ff q = ff_add(a2, ff_neg(ff_mul(pe, pe)));
    const float qv = __fadd_rn(q.hi, q.lo);
    *eps_out = __fadd_rn(eps.hi, eps.lo);
    return qv > 0.0f ? __fsqrt_rn(qv) * inv_Es : 0.0f;
}

// ---------------------------------------------------------------------------
// Synchrotron functions F (first) and G (second), Sec. 3.2.1:
//   F(x) = x^{1/3} exp(-lam_k x) P_k(t),  t = log2 x - k on [2^k, 2^(k+1)),
//   t = x^{2/3} on the piece below 2^KMIN.  `tbl` is the table of
//   synchro_coeffs.h as float4 rows of 16 floats (F c0..c5, G c0..c5, lam).
// ---------------------------------------------------------------------------
constexpr int kSynRows = QED_SYN_NPIECE * 4;  // float4 per table

__device__ __forceinline__ void synchrotron_FG(const float4* __restrict__ tbl, float x, float& F,
                                               float& G) {
    const float l2 = __log2f(x);
    const float u = exp2f(l2 * (1.0f / 3.0f));                 // x^{1/3}
    const int e = ((__float_as_int(x) >> 23) & 0xff) - 127;   // floor(log2 x), normal x
    const bool small = e < QED_SYN_KMIN;
    const int k = min(e, QED_SYN_KMAX);
    const int piece = small ? 0 : k - QED_SYN_KMIN + 1;
    float t = small ? u * u : l2 - (float)k;
    t = fminf(t, 1.02f);
    const float4* row = tbl + 4 * piece;
    const float4 a = row[0], b = row[1], c = row[2], d = row[3];
    float pf = fmaf(b.y, t, b.x);
    pf = fmaf(pf, t, a.w);
    pf = fmaf(pf, t, a.z);
    pf = fmaf(pf, t, a.y);
    pf = fmaf(pf, t, a.x);
    float pg = fmaf(c.w, t, c.z);
    pg = fmaf(pg, t, c.y);
    pg = fmaf(pg, t, c.x);
    pg = fmaf(pg, t, b.w);
    pg = fmaf(pg, t, b.z);
    const float env = u * expf(-d.x * x);
    const bool ok = (x > 0.0f) && (x < 88.0f);
    F = ok ? env * pf : 0.0f;
    G = ok ? env * pg : 0.0f;
}

// Copy the synchrotron table into shared memory (call with all threads of
// the block, then __syncthreads()).
__device__ __forceinline__ void stage_syn_table(float4* dst) {
    // the __device__ source array is only 4-byte aligned: copy float by float
    const float* src = &qed_syn_table[0][0];
    float* d = reinterpret_cast<float*>(dst);
    for (int i = threadIdx.x; i < 4 * kSynRows; i += blockDim.x) d[i] = src[i];
}

// ---------------------------------------------------------------------------
// Rate bounds f(b), Sec. 3.1.1, with c the prefactor for the time interval
// (c = sqrt3 R t / (pi gamma)) and b = 3 chi / 2.  Pieces [0,0.1) [0.1,0.5)
// [0.5,10) [10,inf).
// ---------------------------------------------------------------------------
constexpr float kPi = 3.14159265358979f;

__device__ __forceinline__ float bound_emission(float b, float c) {
    float lead;
    if (b < 0.1f) lead = 0.56f * kPi * b;
    else if (b < 0.5f) lead = 0.45f * kPi * powf(b, 11.0f / 12.0f);
    else if (b < 10.0f) lead = 0.42f * kPi * powf(b, 19.0f / 24.0f);
    else lead = 0.55f * kPi * powf(b, 2.0f / 3.0f);
    return c * (lead + 0.1f * b);
}

// x -> 0 limit of 3 x^2 P(x^3) over c b^{2/3}:  4 pi / (sqrt3 Gamma(1/3) 2^{1/3}).
constexpr float kSmallF = 2.14952824153447863f;

struct Plan {
    uint32_t N;      // sub-steps for the remaining time
    float b;         // 3 chi / 2
    float c_h;       // sqrt3 R h / (pi gamma) for one sub-step
    uint32_t T;      // squeeze threshold on (r >> 9): candidates have (r >> 9) < T
    double h;        // sub-step length (periods)
    bool guard;      // N raised by the validity guard
};

struct StepParams {
    uint64_t seed;
    double dt;           // global step (periods)
    float K;             // sqrt3 R / pi  (1 / period)
    float inv_Es;        // 1 / Schwinger field (code units)
    float p_max;
    float pair_coeff;
    uint32_t step;       // global step index (Philox counter word 2)
    uint32_t process_mask;
    int recoil;
    int cascade;
};

// Squeeze: an upper bound of the acceptance function over all x, from the
// tabulated sup_x P / (c b^{2/3}) of the octave of b.
__device__ __forceinline__ float squeeze_bound(const float* __restrict__ sqz_e,
                                               const float* __restrict__ sqz_p, bool photon,
                                               float b, float c_h, float b23) {
    if (!(b > 0.0f)) return 0.0f;
    const int j = ((__float_as_int(b) >> 23) & 0xff) - 127;
    float H;
    if (!photon) {
        if (j < QED_SQZ_E_JMIN) H = QED_SQZ_E_SMALL;
        else if (j >= QED_SQZ_E_JMAX) return 2.0f;  // no squeeze
        else H = sqz_e[j - QED_SQZ_E_JMIN];
    } else {
        if (j < QED_SQZ_P_JMIN) H = sqz_p[0];
        else if (j >= QED_SQZ_P_JMAX) return 2.0f;
        else H = sqz_p[j - QED_SQZ_P_JMIN];
    }
    return c_h * H * b23;
}

__device__ __forceinline__ uint32_t squeeze_threshold(float B) {
    // y = ((r>>9) * 2 + 1) 2^-24 < B  <=>  (r>>9) < (B 2^24 - 1) / 2
    if (!(B < 1.0f)) return 1u << 23;
    const float t = ceilf(fmaf(B, 0x1p23f, -0.5f)) + 1.0f;
    return t <= 0.0f ? 0u : (t >= 0x1p23f ? (1u << 23) : (uint32_t)t);
}

// Plan the sub-steps of the remaining time t_rem (Algorithms 1/2, line 1).
__device__ __forceinline__ Plan make_plan(const StepParams& P, const float* __restrict__ sqz_e,
                                          const float* __restrict__ sqz_p, bool photon, float chi,
                                          float eps, double t_rem) {
    Plan pl;
    pl.b = 1.5f * chi;
    const float inv_eps = 1.0f / eps;
    const float c_rem = P.K * (float)t_rem * inv_eps;
    const float b = pl.b;
    float f = photon ? P.pair_coeff * c_rem * b : bound_emission(b, c_rem);
    float q = f / P.p_max;
    float N = fmaxf(1.0f, ceilf(q));
    float b23 = 0.0f;
    if (b > 0.0f) b23 = exp2f(__log2f(b) * (2.0f / 3.0f));
    pl.guard = false;
    if (!photon) {
        const float g = ceilf(kSmallF * c_rem * b23);
        if (g > N) { N = g; pl.guard = true; }
    }
    N = fminf(N, 1073741824.0f);  // 2^30: keeps the 32-bit sub-step counter from wrapping
    pl.N = (uint32_t)N;
    pl.h = t_rem / (double)pl.N;
    pl.c_h = P.K * (float)pl.h * inv_eps;
    pl.T = squeeze_threshold(squeeze_bound(sqz_e, sqz_p, photon, b, pl.c_h, b23));
    return pl;
}

// Acceptance function of Algorithm 1 (emission, delta = x^3, Eq. 1):
//   3 x^2 P(x^3) = (c b / x) [(1 - delta) F(z) + delta^2 G(z)],  z = delta / (b (1-delta)).
// Algorithm 2 (pair, delta = x, Eq. 2 with the positive bracket):
//   P_p = (c b / 3) [G(z) - delta (1 - delta) F(z)],  z = 1 / (b delta (1 - delta)).
__device__ __forceinline__ float acceptance(const float4* __restrict__ tbl, bool photon, float b,
                                            float c_h, float x, float* delta_out) {
    float F, G;
    if (!photon) {
        const float d = x * x * x;
        const float omd = 1.0f - d;
        const float z = d / (b * omd);
        synchrotron_FG(tbl, z, F, G);
        *delta_out = d;
        return (c_h * b / x) * (omd * F + d * d * G);
    } else {
        const float dd = x * (1.0f - x);
        const float z = 1.0f / (b * dd);
        synchrotron_FG(tbl, z, F, G);
        *delta_out = x;
        return (c_h * b * (1.0f / 3.0f)) * (G - dd * F);
    }
}

}  // namespace qed
