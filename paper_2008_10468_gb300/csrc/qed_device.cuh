// Device building blocks of the QED event generator (sm_103a).
//
//   - Philox4x32-10 (Salmon et al., SC'11) and the open-interval uniform;
//   - the quantum parameter chi (Sec. 2.2) in float-float arithmetic;
//   - the synchrotron functions F and G (Sec. 3.2.1) from the octave tables of
//     synchro_coeffs.h, staged in shared memory;
//   - the rate bounds f(b) of Sec. 3.1.1 and the sub-step planner;
//   - the acceptance functions of Algorithms 1 and 2;
//   - the Boris push of Algorithm 1 on the binary32 momentum.
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

// The same with the round keys given: round r uses (k0 + r 0x9E3779B9,
// k1 + r 0xBB67AE85) from K.k[2r], K.k[2r+1].  The event kernels take them
// from their parameter block, computed once on the host (philox_keys), so a
// block costs only its multiplies and xors.
struct PhiloxKeys {
    uint32_t k[20];
};

__host__ __device__ inline PhiloxKeys philox_keys(uint32_t k0, uint32_t k1) {
    PhiloxKeys K;
    for (int r = 0; r < 10; ++r) {
        K.k[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
        K.k[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
    return K;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys& K) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ K.k[2 * r], lo1, hi0 ^ c.w ^ K.k[2 * r + 1], lo0);
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
// ... and of the event-driven sampler's waiting-time stream.
constexpr uint32_t kWaitKeyLo = 0x3C6EF372u;
constexpr uint32_t kWaitKeyHi = 0xDAA66D2Bu;

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
// particles co-moving with a crossed field, so every product is kept exact:
// chi_sq_ff returns (chi E_s)^2 and eps as float-float pairs.
__device__ __forceinline__ void chi_sq_ff(bool photon, float px, float py, float pz, float Ex,
                                          float Ey, float Ez, float Bx, float By, float Bz,
                                          ff* q_out, ff* eps_out) {
    const ff p2 = ff_add(ff_add(two_prod(px, px), two_prod(py, py)), two_prod(pz, pz));
    const ff g2 = photon ? p2 : ff_add(p2, ff{1.0f, 0.0f});
    const ff eps = ff_sqrt(g2);
    const ff ax = ff_add(ff_mul_f(eps, Ex), ff_add(two_prod(py, Bz), ff_neg(two_prod(pz, By))));
    const ff ay = ff_add(ff_mul_f(eps, Ey), ff_add(two_prod(pz, Bx), ff_neg(two_prod(px, Bz))));
    const ff az = ff_add(ff_mul_f(eps, Ez), ff_add(two_prod(px, By), ff_neg(two_prod(py, Bx))));
    const ff pe = ff_add(ff_add(two_prod(px, Ex), two_prod(py, Ey)), two_prod(pz, Ez));
    const ff a2 = ff_add(ff_add(ff_mul(ax, ax), ff_mul(ay, ay)), ff_mul(az, az));
    *q_out = ff_add(a2, ff_neg(ff_mul(pe, pe)));
    *eps_out = eps;
}

// chi from chi_sq_ff, rounded to binary32; *eps_out receives eps rounded to
// binary32.
__device__ __forceinline__ float chi_ff(bool photon, float px, float py, float pz, float Ex,
                                        float Ey, float Ez, float Bx, float By, float Bz,
                                        float inv_Es, float* eps_out) {
    ff q, eps;
    chi_sq_ff(photon, px, py, pz, Ex, Ey, Ez, Bx, By, Bz, &q, &eps);
    const float qv = __fadd_rn(q.hi, q.lo);
    *eps_out = __fadd_rn(eps.hi, eps.lo);
    return qv > 0.0f ? __fsqrt_rn(qv) * inv_Es : 0.0f;
}

// chi in binary32 (Sec. 2.2).  Sets *well_conditioned when the rounding
// error of chi is certainly below 7.5 u kappa_max relative (u = 2^-24): the
// error of the computed chi^2 is at most ~15 u M^2 with M = eps|E| + |p||B|
// (a bound on |eps E + p x B| and |p.E|), and kappa = 2 (eps^2 E^2 + p^2 B^2)
// / chi^2 >= M^2 / chi^2 (*kappa_out, if asked).  Both the planner and the
// push mode's chi of each sub-step accept kappa < 8 (3.6e-6); the planner
// widens its count's safety band with kappa.  Otherwise use chi_ff.
__device__ __forceinline__ float chi_f32(bool photon, float px, float py, float pz, float Ex,
                                         float Ey, float Ez, float Bx, float By, float Bz,
                                         float inv_Es, float* eps_out, bool* well_conditioned,
                                         float kappa_max = 8.0f, float* kappa_out = nullptr) {
    const float p2 = fmaf(px, px, fmaf(py, py, pz * pz));
    const float eps = photon ? sqrtf(p2) : sqrtf(1.0f + p2);
    const float cx = fmaf(py, Bz, -pz * By);
    const float cy = fmaf(pz, Bx, -px * Bz);
    const float cz = fmaf(px, By, -py * Bx);
    const float ax = fmaf(eps, Ex, cx), ay = fmaf(eps, Ey, cy), az = fmaf(eps, Ez, cz);
    const float s = fmaf(px, Ex, fmaf(py, Ey, pz * Ez));
    const float q = fmaf(-s, s, fmaf(ax, ax, fmaf(ay, ay, az * az)));
    const float E2 = fmaf(Ex, Ex, fmaf(Ey, Ey, Ez * Ez));
    const float B2 = fmaf(Bx, Bx, fmaf(By, By, Bz * Bz));
    const float M2 = 2.0f * fmaf(eps * eps, E2, p2 * B2);
    *eps_out = eps;
    *well_conditioned = q * kappa_max > M2;
    if (kappa_out) *kappa_out = __fdividef(M2, q);
    return q > 0.0f ? sqrtf(q) * inv_Es : 0.0f;
}

// chi and eps of a momentum: binary32 when well conditioned (kappa < 8),
// else float-float.
__device__ __forceinline__ float chi_any(bool photon, float px, float py, float pz, float Ex,
                                         float Ey, float Ez, float Bx, float By, float Bz,
                                         float inv_Es, float* eps_out) {
    bool wc;
    const float chi = chi_f32(photon, px, py, pz, Ex, Ey, Ez, Bx, By, Bz, inv_Es, eps_out, &wc);
    if (wc) return chi;
    return chi_ff(photon, px, py, pz, Ex, Ey, Ez, Bx, By, Bz, inv_Es, eps_out);
}

// Boris push (Algorithm 1: the particle moves by one sub-step before the
// draw).  In code units (p in m c, fields in m c omega / e, time in laser
// periods) the Lorentz force is dp/dt = 2 pi q (E + p x B / gamma); with
// a = pi q h for a sub-step h:
//   p- = p + a E,  t = (a / gamma(p-)) B,  s = 2 t / (1 + t^2),
//   p+ = p- + (p- + p- x t) x s,  p(h) = p+ + a E.
// t and s share one denominator: with u = a B, g^2 = 1 + |p-|^2,
// w = g^2 + |u|^2 and D = g w, t = u (w / D) and s = u (2 g^2 / D), so one
// division serves both (the push is the serial part of the push-mode step).
// Each operation is an explicit round-to-nearest binary32 intrinsic, in this
// order: the result is the IEEE binary32 evaluation of these formulas, not
// subject to contraction into FMAs.
__device__ __forceinline__ void boris_push(float& px, float& py, float& pz, float a, float Ex,
                                           float Ey, float Ez, float Bx, float By, float Bz) {
    const float mx = __fadd_rn(px, __fmul_rn(a, Ex));
    const float my = __fadd_rn(py, __fmul_rn(a, Ey));
    const float mz = __fadd_rn(pz, __fmul_rn(a, Ez));
    const float ux = __fmul_rn(a, Bx), uy = __fmul_rn(a, By), uz = __fmul_rn(a, Bz);
    const float m2 = __fadd_rn(__fadd_rn(__fmul_rn(mx, mx), __fmul_rn(my, my)), __fmul_rn(mz, mz));
    const float u2 = __fadd_rn(__fadd_rn(__fmul_rn(ux, ux), __fmul_rn(uy, uy)), __fmul_rn(uz, uz));
    const float g2 = __fadd_rn(1.0f, m2);
    const float g = __fsqrt_rn(g2);
    const float w = __fadd_rn(g2, u2);
    const float R = __fdiv_rn(1.0f, __fmul_rn(g, w));
    const float ct = __fmul_rn(w, R);
    const float cs = __fmul_rn(__fmul_rn(2.0f, g2), R);
    const float tx = __fmul_rn(ct, ux), ty = __fmul_rn(ct, uy), tz = __fmul_rn(ct, uz);
    const float sx = __fmul_rn(cs, ux), sy = __fmul_rn(cs, uy), sz = __fmul_rn(cs, uz);
    const float qx = __fadd_rn(mx, __fsub_rn(__fmul_rn(my, tz), __fmul_rn(mz, ty)));
    const float qy = __fadd_rn(my, __fsub_rn(__fmul_rn(mz, tx), __fmul_rn(mx, tz)));
    const float qz = __fadd_rn(mz, __fsub_rn(__fmul_rn(mx, ty), __fmul_rn(my, tx)));
    const float rx = __fadd_rn(mx, __fsub_rn(__fmul_rn(qy, sz), __fmul_rn(qz, sy)));
    const float ry = __fadd_rn(my, __fsub_rn(__fmul_rn(qz, sx), __fmul_rn(qx, sz)));
    const float rz = __fadd_rn(mz, __fsub_rn(__fmul_rn(qx, sy), __fmul_rn(qy, sx)));
    px = __fadd_rn(rx, __fmul_rn(a, Ex));
    py = __fadd_rn(ry, __fmul_rn(a, Ey));
    pz = __fadd_rn(rz, __fmul_rn(a, Ez));
}

// ---------------------------------------------------------------------------
// Synchrotron functions F (first) and G (second), Sec. 3.2.1:
//   F(x) = x^{1/3} exp(-lam_k x) P_k(t),  t = log2 x - k on [2^k, 2^(k+1)),
//   t = x^{2/3} on the piece below 2^KMIN.  `tbl` is the table of
//   synchro_coeffs.h as float4 rows of 16 floats (F c0..c5, G c0..c5, lam).
// ---------------------------------------------------------------------------
constexpr int kSynCoef = 2 * (QED_SYN_DEG + 1);   // F and G coefficients per piece
constexpr int kSynStride = 32;                     // pieces padded to one bank row

// Shared-memory form of the table: coefficient-major, c[j][p] is power j of
// piece p (F in rows 0..DEG, G in rows DEG+1..2DEG+1).  Lanes of a warp
// reading power j of different pieces hit different banks (22 pieces fit in
// one row of 32 banks); 64-bit (F, G) pairs would share 16 bank pairs among
// 22 pieces and conflict.
struct SynTable {
    float c[kSynCoef][kSynStride];
    unsigned int lam_mask;   // bit p set: piece p carries the exp(-x) envelope
};

__device__ __forceinline__ void synchrotron_FG(const SynTable& tb, float x, float& F, float& G) {
    const float l2 = __log2f(x);
    const float u = exp2f(l2 * (1.0f / 3.0f));                 // x^{1/3}
    const int e = ((__float_as_int(x) >> 23) & 0xff) - 127;   // floor(log2 x), normal x
    const bool small = e < QED_SYN_KMIN;
    const int k = min(e, QED_SYN_KMAX);
    const int piece = small ? 0 : k - QED_SYN_KMIN + 1;
    float t = small ? u * u : l2 - (float)k;
    t = fminf(t, 1.02f);
    float pf = tb.c[QED_SYN_DEG][piece];
    float pg = tb.c[2 * QED_SYN_DEG + 1][piece];
#pragma unroll
    for (int j = QED_SYN_DEG - 1; j >= 0; --j) {
        pf = fmaf(pf, t, tb.c[j][piece]);
        pg = fmaf(pg, t, tb.c[QED_SYN_DEG + 1 + j][piece]);
    }
    const float lam = ((tb.lam_mask >> piece) & 1u) ? 1.0f : 0.0f;
    const float env = u * expf(-lam * x);
    const bool ok = (x > 0.0f) && (x < 88.0f);
    F = ok ? env * pf : 0.0f;
    G = ok ? env * pg : 0.0f;
}

// Copy the synchrotron table into shared memory (call with all threads of
// the block, then __syncthreads()).
__device__ __forceinline__ void stage_syn_table(SynTable& tb) {
    for (int i = threadIdx.x; i < kSynCoef * kSynStride; i += blockDim.x) {
        const int j = i / kSynStride, p = i % kSynStride;
        tb.c[j][p] = p < QED_SYN_NPIECE ? qed_syn_table[p][j] : 0.0f;
    }
    if (threadIdx.x == 0) {
        unsigned int m = 0;
        for (int p = 0; p < QED_SYN_NPIECE; ++p)
            if (qed_syn_table[p][kSynCoef] > 0.0f) m |= 1u << p;
        tb.lam_mask = m;
    }
}

// ---------------------------------------------------------------------------
// Rate bounds f(b), Sec. 3.1.1, with c the prefactor for the time interval
// (c = sqrt3 R t / (pi gamma)) and b = 3 chi / 2.  Pieces [0,0.1) [0.1,0.5)
// [0.5,10) [10,inf).
// ---------------------------------------------------------------------------
constexpr float kPi = 3.14159265358979f;

// The emission bound from l2b = log2(b) (b > 0): the powers as exp2(a l2b) on
// the special-function unit (error budget in make_plan).
__device__ __forceinline__ float bound_emission_l2(float b, float l2b, float c) {
    float lead;
    if (b < 0.1f) lead = 0.56f * kPi * b;
    else if (b < 0.5f) lead = 0.45f * kPi * exp2f(l2b * (11.0f / 12.0f));
    else if (b < 10.0f) lead = 0.42f * kPi * exp2f(l2b * (19.0f / 24.0f));
    else lead = 0.55f * kPi * exp2f(l2b * (2.0f / 3.0f));
    return c * (lead + 0.1f * b);
}

// x -> 0 limit of 3 x^2 P(x^3) over c b^{2/3}:  4 pi / (sqrt3 Gamma(1/3) 2^{1/3}).
constexpr float kSmallF = 2.14952824153447863f;

// Remaining time of a particle within the global step, in laser periods, as a
// float-float pair (about 48 significant bits).  Sub-steps have length
// h = t / N and the time after sub-step k of a plan is t - (k + 1) h, the
// last sub-step ending the plan exactly.  The pair keeps this accumulator on
// the FP32 pipe: FP64, and 64-bit integer conversions and divisions (which
// this GPU runs on its FP64 pipe, at 1/64 of the FP32 rate), stay off the
// sub-step path.
struct ftime {
    float hi, lo;
};

__device__ __forceinline__ bool time_positive(ftime t) { return t.hi > 0.0f; }

// An integer below 2^31 as the exact sum of two binary32 numbers: the
// rounded value and the (signed, small) rest.
__device__ __forceinline__ ff int_ff(uint32_t n) {
    const float hi = (float)n;   // exact up to 2^24
    const float lo = (float)(int)(n - (uint32_t)hi);
    return {hi, lo};
}

// t / N for an integer N >= 1, to float-float precision: an approximate
// reciprocal of N's leading part, one exact-residual correction of the
// leading part of the quotient, then the trailing part from the remainder
// t - q N (the product with N's leading part error-free via FMA; N's rest,
// nonzero only above 2^24, times q as a small correction).
__device__ __forceinline__ ftime time_div(ftime t, uint32_t N) {
    const ff n = int_ff(N);
    const float r = __fdividef(1.0f, n.hi);
    float q = t.hi * r;
    q = __fmaf_rn(__fmaf_rn(-q, n.hi, t.hi), r, q);
    const ff qn = two_prod(q, n.hi);
    const float rem = __fadd_rn(
        __fsub_rn(__fsub_rn(__fsub_rn(t.hi, qn.hi), qn.lo), __fmul_rn(q, n.lo)), t.lo);
    const ff out = fast_two_sum(q, rem * r);
    return {out.hi, out.lo};
}

// t - m h for an integer m (exact as a float-float pair up to 2^31).
__device__ __forceinline__ ftime time_sub_mul(ftime t, uint32_t m, ftime h) {
    const ff mf = int_ff(m);
    const ff mh = ff_add(two_prod(h.hi, mf.hi),
                         ff{__fmaf_rn(h.hi, mf.lo, __fmul_rn(h.lo, mf.hi)), 0.0f});
    const ff d = ff_add(ff{t.hi, t.lo}, ff_neg(mh));
    return {d.hi, d.lo};
}

struct Plan {
    uint32_t N;      // sub-steps for the remaining time
    float b;         // 3 chi / 2
    float c_h;       // sqrt3 R h / (pi gamma) for one sub-step
    uint32_t T;      // squeeze threshold on (r >> 9): candidates have (r >> 9) < T
    ftime h;         // sub-step length (periods)
    bool guard;      // N raised by the validity guard
    bool safe;       // N is certain (the count of the exact q)
    float chi, eps;  // quantum parameter and energy the plan was made from
};

// The step constants the planner reads, passed by value so that the
// out-of-line slow path takes them in registers (a reference to the kernel's
// parameter block would make the whole block addressable, i.e. a local copy).
struct PlanConst {
    float K, inv_Es, inv_p_max, pair_coeff, p_max;
    double lambda_m;   // laser wavelength (m): the binary64 constants of near-tie plans
};

// Physical constants (CODATA 2022) and the binary64 forms of K = sqrt3 R / pi
// and 1 / E_s for wavelength lambda_m, evaluated in the same order on the host
// and the device.
constexpr double kAlphaD = 7.2973525643e-3;           // fine-structure constant
constexpr double kTauCD = 1.2880886664441626e-21;     // hbar / (m c^2), s
constexpr double kCLightD = 299792458.0;              // m / s
constexpr double kPiD64 = 3.14159265358979323846;
__host__ __device__ __forceinline__ double rate_K64(double lambda_m) {
    const double R = kAlphaD / kTauCD * (lambda_m / kCLightD);   // 1 / period
    return 1.7320508075688772 / kPiD64 * R;
}
__host__ __device__ __forceinline__ double inv_schwinger64(double lambda_m) {
    return 2.0 * kPiD64 * kCLightD / lambda_m * kTauCD;
}

struct StepParams {
    uint64_t seed;
    double dt;           // global step (periods)
    float K;             // sqrt3 R / pi  (1 / period)
    float inv_Es;        // 1 / Schwinger field (code units)
    float p_max;
    float inv_p_max;     // 1 / p_max
    float pair_coeff;
    double lambda_m;     // laser wavelength (m)
    PhiloxKeys draw_keys;   // round keys of the draw stream (key: seed)
    PhiloxKeys child_keys;  // ... of the child-id stream (key: seed ^ kChildKey)
    unsigned long long wait_ns;  // tail pass: longest bounded wait before QED_ERR_TIMEOUT
    ftime t_step;        // dt as float-float
    const uint32_t* step_base;  // graph runs: device step base added to `step`
    uint32_t hot_min;           // plans with at least this many sub-steps go to the hot pass
    uint32_t long_min;          // ... and with at least this many to its warp mode
    int sampler;                // learned sampler on (e+- in usable bins)
    int net_rows;               // rows of the total-probability table
    unsigned long long net_bins;  // usable bins (64, uniform in log10 chi over [-2, 2))
    const void* net_w;          // BF16 network weights (8577)
    const float* net_wtot;      // total probability per c along log10 chi
    unsigned long long pnet_bins;  // pair sampler (event-driven mode): usable bins (0: off)
    const void* pnet_w;            // its BF16 weights
    const float* pnet_wtot;        // its total probability per c along log10 chi
    uint32_t step;       // global step index (Philox counter word 2)
    uint32_t process_mask;
    int recoil;
    int cascade;
    const uint32_t* cell;        // push mode with per-cell counts: cell of each initial row
    const unsigned int* N_cell;  // ... and the count of each cell (NULL: per-particle plans)
    long long ncells;
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

__device__ __forceinline__ int emission_piece(float b) {
    return b < 0.1f ? 0 : (b < 0.5f ? 1 : (b < 10.0f ? 2 : 3));
}

// log2 b within 5e-7 for every b > 0: the exponent exactly, plus __log2f of
// the mantissa in [1, 2), where its absolute error is at most 2^-22 (for a
// subnormal or zero b, __log2f of b itself).
__device__ __forceinline__ float log2_split(float b) {
    const int bits = __float_as_int(b);
    const int e = ((bits >> 23) & 0xff) - 127;
    const float m = __int_as_float((bits & 0x007fffff) | 0x3f800000);
    return e > -127 ? (float)e + __log2f(m) : __log2f(b);
}

// Plan the sub-steps of the remaining time T (Algorithms 1/2, planning).
// `safe` reports whether N is certain.  The binary32 q = f / P_max carries a
// relative error below 1.2e-6 + e_chi: c 3.6e-7 (1/eps by the fast divide, K
// and t rounded, two products), b^e 2.6e-7 (log2_split) plus 2.9e-7 (exp2f and
// the product in its argument), the constants A pi and 0.1 in binary32
// 1.2e-7, the last three roundings 1.5e-7; and chi's error e_chi passes on at
// most linearly (every f(b) piece grows at most linearly in b).  With chi in
// binary32, e_chi <= 7.5 u kappa + u (chi_f32), so the band is
// d = 1.5e-6 + 5e-7 kappa; with chi from float-float, d = 1.5e-6.  N =
// max(1, ceil(q), ceil(g)) is certain when it is the same at q (1 -+ d) and
// g (1 -+ d) and b stays in its f piece within d; otherwise plan_slow
// recomputes it.
__device__ __forceinline__ PlanConst plan_const(const StepParams& P) {
    return PlanConst{P.K, P.inv_Es, P.inv_p_max, P.pair_coeff, P.p_max, P.lambda_m};
}

__device__ __forceinline__ Plan make_plan(const PlanConst& P, const float* __restrict__ sqz_e,
                                          const float* __restrict__ sqz_p, bool photon, float chi,
                                          float eps, ftime T, float d) {
    Plan pl;
    pl.chi = chi;
    pl.eps = eps;
    pl.b = 1.5f * chi;
    const float inv_eps = __fdividef(1.0f, eps);
    const float c_rem = P.K * T.hi * inv_eps;
    const float b = pl.b;
    const float l2b = log2_split(b);
    const float f = photon ? P.pair_coeff * c_rem * b
                           : (b > 0.0f ? bound_emission_l2(b, l2b, c_rem) : 0.0f);
    const float q = f * P.inv_p_max;
    float N = fmaxf(1.0f, ceilf(q));
    float b23 = 0.0f;
    if (b > 0.0f) b23 = exp2f(l2b * (2.0f / 3.0f));
    pl.guard = false;
    float graw = 0.0f;
    if (!photon) {
        graw = kSmallF * c_rem * b23;
        const float g = ceilf(graw);
        if (g > N) { N = g; pl.guard = true; }
    }
    // N = max(1, ceil(q), ceil(g)) is monotone in q and g: it is certain when
    // it is the same at both ends of the band (and b stays in its f piece)
    const float n_lo = fmaxf(1.0f, fmaxf(ceilf(q * (1.0f - d)), ceilf(graw * (1.0f - d))));
    const float n_hi = fmaxf(1.0f, fmaxf(ceilf(q * (1.0f + d)), ceilf(graw * (1.0f + d))));
    bool safe = n_lo == n_hi;
    if (!photon)
        safe = safe && emission_piece(b * (1.0f - d)) == emission_piece(b * (1.0f + d));
    N = fminf(N, 1073741824.0f);  // 2^30: keeps the 32-bit sub-step counter from wrapping
    pl.N = (uint32_t)N;
    pl.safe = safe;
    pl.h = time_div(T, pl.N);
    pl.c_h = P.K * pl.h.hi * inv_eps;
    pl.T = squeeze_threshold(squeeze_bound(sqz_e, sqz_p, photon, b, pl.c_h, b23));
    return pl;
}

// f(b) of Sec. 3.1.1 in binary64, in the order the products are written
// there: A pi c b^e + 0.1 c b.
__device__ __forceinline__ double bound_emission64(double b, double c) {
    double lead;
    if (b < 0.1) lead = 0.56 * 3.14159265358979323846 * c * b;
    else if (b < 0.5) lead = 0.45 * 3.14159265358979323846 * c * pow(b, 11.0 / 12.0);
    else if (b < 10.0) lead = 0.42 * 3.14159265358979323846 * c * pow(b, 19.0 / 24.0);
    else lead = 0.55 * 3.14159265358979323846 * c * pow(b, 2.0 / 3.0);
    return lead + 0.1 * c * b;
}

// Slow path of plan_particle, for plans whose binary32 count is not certain
// (chi ill-conditioned, or f / P_max within 3e-6 of an integer, or b at a
// piece edge): chi in float-float and the binary32 plan from it; if its count
// is still not certain, the count N = max(1, ceil(f/P_max), guard) in
// binary64, so that N is the exact count unless f / P_max lies within ~1e-13
// of an integer.  The binary64 step is rare (0.6% of the longest plans,
// fewer of the others), so it stays off the sub-step path.  Kept out of line
// so that the common path does not carry its registers.
__device__ __noinline__ Plan plan_slow(PlanConst P, const float* __restrict__ sqz_e,
                                       const float* __restrict__ sqz_p, bool photon, float px,
                                       float py, float pz, float Ex, float Ey, float Ez, float Bx,
                                       float By, float Bz, ftime T) {
    ff q2, epsf;
    chi_sq_ff(photon, px, py, pz, Ex, Ey, Ez, Bx, By, Bz, &q2, &epsf);
    const double q2d = (double)q2.hi + (double)q2.lo;
    const double chi_d = q2d > 0.0 ? sqrt(q2d) * inv_schwinger64(P.lambda_m) : 0.0;
    const double eps_d = (double)epsf.hi + (double)epsf.lo;
    Plan pl;
    pl.chi = (float)chi_d;
    pl.eps = (float)eps_d;
    if (!(pl.eps > 0.0f)) {
        pl.N = 0;
        return pl;
    }
    // the binary32 plan from the float-float chi (chi now within 1 ulp): when
    // its count is certain, that is the plan (an ill-conditioned chi, the
    // common reason to be here, needs no binary64)
    pl = make_plan(P, sqz_e, sqz_p, photon, pl.chi, pl.eps, T, 1.5e-6f);
    if (pl.safe) return pl;
    const double b = 1.5 * chi_d;
    const double c_rem = rate_K64(P.lambda_m) * ((double)T.hi + (double)T.lo) / eps_d;  // hi + lo exact
    const double f = photon ? (double)P.pair_coeff * c_rem * b
                            : (b > 0.0 ? bound_emission64(b, c_rem) : 0.0);
    double N = fmax(1.0, ceil(f / (double)P.p_max));
    pl.guard = false;
    if (!photon && b > 0.0) {
        const double g = ceil(2.14952824153447863 * c_rem * pow(b, 2.0 / 3.0));
        if (g > N) { N = g; pl.guard = true; }
    }
    N = fmin(N, 1073741824.0);   // 2^30
    pl.N = (uint32_t)N;
    pl.safe = true;
    pl.b = 1.5f * pl.chi;
    pl.h = time_div(T, pl.N);
    pl.c_h = P.K * pl.h.hi * __fdividef(1.0f, pl.eps);
    const float b23 = pl.b > 0.0f ? exp2f(__log2f(pl.b) * (2.0f / 3.0f)) : 0.0f;
    pl.T = squeeze_threshold(squeeze_bound(sqz_e, sqz_p, photon, pl.b, pl.c_h, b23));
    return pl;
}

// One sub-step per cell (Algorithms 1 and 2 start by fixing the cell's
// sub-step): with per-cell counts, the first plan (s = 0) of an initial row
// (i < n_init) takes its cell's count N_cell when that is larger than its own,
// i.e. the sub-step T / N_cell; h, c_h and the squeeze threshold follow.
// The plain step's kernels call it only in their cell-count instantiations
// (kCells): with the test at run time, the kernels' register allocation
// changed and the step without cell counts took 2-3% longer.
__device__ __forceinline__ Plan cell_count_plan(Plan pl, const float* __restrict__ sqz_e,
                                             const float* __restrict__ sqz_p, float K,
                                             bool photon, uint32_t Nc, ftime T, float eps) {
    pl.N = Nc;
    pl.h = time_div(T, Nc);
    pl.c_h = K * pl.h.hi * __fdividef(1.0f, eps);
    const float b23 = pl.b > 0.0f ? exp2f(__log2f(pl.b) * (2.0f / 3.0f)) : 0.0f;
    pl.T = squeeze_threshold(squeeze_bound(sqz_e, sqz_p, photon, pl.b, pl.c_h, b23));
    return pl;
}

__device__ __forceinline__ void apply_cell_count(const StepParams& SP, Plan& pl,
                                                 const float* __restrict__ sqz_e,
                                                 const float* __restrict__ sqz_p, bool photon,
                                                 long long i, long long n_init, uint32_t s,
                                                 ftime T, float eps) {
    if (!SP.N_cell || s != 0u || i >= n_init || !(eps > 0.0f)) return;
    const uint32_t c = SP.cell[i];
    const uint32_t Nc = (long long)c < SP.ncells ? SP.N_cell[c] : 0u;
    if (Nc > pl.N) pl = cell_count_plan(pl, sqz_e, sqz_p, SP.K, photon, Nc, T, eps);
}

// chi and the plan of a particle: binary32 chi when it is well conditioned and
// the plan is safe, otherwise chi in float-float (and the plan again).
__device__ __forceinline__ Plan plan_particle(const StepParams& SP, const float* __restrict__ sqz_e,
                                              const float* __restrict__ sqz_p, bool photon,
                                              float px, float py, float pz, float Ex, float Ey,
                                              float Ez, float Bx, float By, float Bz, ftime T,
                                              float* chi_out, float* eps_out) {
    const PlanConst P = plan_const(SP);
    bool wc;
    float eps, kappa;
    const float chi = chi_f32(photon, px, py, pz, Ex, Ey, Ez, Bx, By, Bz, P.inv_Es, &eps, &wc,
                              8.0f, &kappa);
    if (wc && eps > 0.0f) {
        const Plan pl =
            make_plan(P, sqz_e, sqz_p, photon, chi, eps, T, fmaf(5e-7f, kappa, 1.5e-6f));
        if (pl.safe) {
            *chi_out = chi;
            *eps_out = eps;
            return pl;
        }
    }
    const Plan pl = plan_slow(P, sqz_e, sqz_p, photon, px, py, pz, Ex, Ey, Ez, Bx, By, Bz, T);
    *chi_out = pl.chi;
    *eps_out = pl.eps;
    return pl;
}

// Acceptance function of Algorithm 1 (emission, delta = x^3, Eq. 1):
//   3 x^2 P(x^3) = (c b / x) [(1 - delta) F(z) + delta^2 G(z)],  z = delta / (b (1-delta)).
// Algorithm 2 (pair, delta = x, Eq. 2 with the positive bracket):
//   P_p = (c b / 3) [G(z) - delta (1 - delta) F(z)],  z = 1 / (b delta (1 - delta)).
// The quotients use the fast divide (within 2 ulp): P moves by a few 1e-7
// relative, inside the band |y - P| <= 1e-5 P within which a decision y < P
// counts as a tie.
__device__ __forceinline__ float acceptance(const SynTable& tbl, bool photon, float b,
                                            float c_h, float x, float* delta_out) {
    float F, G;
    if (!photon) {
        const float d = x * x * x;
        const float omd = (1.0f - x) * fmaf(x, x + 1.0f, 1.0f);  // 1 - x^3 without cancellation
        const float z = __fdividef(d, b * omd);
        synchrotron_FG(tbl, z, F, G);
        *delta_out = d;
        return __fdividef(c_h * b, x) * (omd * F + d * d * G);
    } else {
        const float dd = x * (1.0f - x);
        const float z = __fdividef(1.0f, b * dd);
        synchrotron_FG(tbl, z, F, G);
        *delta_out = x;
        return (c_h * b * (1.0f / 3.0f)) * (G - dd * F);
    }
}

}  // namespace qed
