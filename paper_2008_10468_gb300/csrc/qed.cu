// GB300 (sm_103a) implementation of the C ABI in include/qed.h.
//
// Kernels
//   k_sweep / k_generate   synchrotron functions over an array or over
//                          in-kernel arguments (Sec. 3.2.1)
//   k_plan                 chi and the sub-step count (Algorithms 1/2 line 1)
//   k_cold                 one thread per particle: plan, sub-step loop,
//                          events, children; particles whose plan exceeds
//                          kHotMin sub-steps are pushed to the hot queue
//   k_hot                  persistent kernel: one warp per queued particle,
//                          64 sub-steps per iteration (lane l draws the
//                          Philox block of sub-steps 2l, 2l+1), first accepted
//                          sub-step found with ballots
//   k_advance              closes a cascade generation
//
// Every sub-step draws (x, y) from Philox4x32-10 at counter
// (id_lo, id_hi, step, s/2) under key = seed (even s: words 0,1; odd s:
// words 2,3).  Before evaluating the acceptance function the kernels compare
// y with an upper bound of that function over all x (the squeeze); this
// changes no decision and skips the synchrotron functions for most sub-steps.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "qed.h"
#include "qed_device.cuh"

using namespace qed;

namespace {

constexpr double kAlpha = 7.2973525643e-3;          // CODATA 2022
constexpr double kTauC = 1.2880886664441626e-21;    // hbar / (m c^2), s
constexpr double kCLight = 299792458.0;             // m / s
constexpr double kPiD = 3.14159265358979323846;

constexpr uint32_t kHotMin = 64;       // plans with N >= kHotMin go to the warp path
constexpr int kColdThreads = 256;
constexpr int kHotThreads = 128;
constexpr int kSweepThreads = 256;

struct DevCtl {
    unsigned long long substeps, emissions, pairs, children, guard_hits, plans, candidates;
    unsigned int max_N;
    int status;
    long long required;
    long long pass_begin, pass_end;
    unsigned int hot_tail, hot_head;
    int more, passes;
    long long log_count_unused;
};

struct HotItem {
    uint32_t idx;
    uint32_t s;
    double t_rem;
};

struct DevParticles {
    float *px, *py, *pz, *Ex, *Ey, *Ez, *Bx, *By, *Bz, *w;
    uint64_t* id;
    uint8_t* type;
    long long* count;
    long long capacity;
};

struct Scratch {
    double* t_rem;          // remaining time of appended children (capacity)
    HotItem* hot;           // queue of warp-path particles (capacity)
    qed_event_record* log;  // optional
    long long log_cap;
    long long* log_count;
};

struct Stats {
    unsigned long long substeps = 0, emissions = 0, pairs = 0, children = 0, guard = 0, plans = 0,
                       cand = 0;
    unsigned int max_N = 0;
};

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ unsigned int warp_max(unsigned int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ void flush_stats(const Stats& st, DevCtl* ctl) {
    const unsigned long long a = warp_sum(st.substeps), b = warp_sum(st.emissions),
                             c = warp_sum(st.pairs), d = warp_sum(st.children),
                             e = warp_sum(st.guard), f = warp_sum(st.plans), g = warp_sum(st.cand);
    const unsigned int m = warp_max(st.max_N);
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd(&ctl->substeps, a);
        if (b) atomicAdd(&ctl->emissions, b);
        if (c) atomicAdd(&ctl->pairs, c);
        if (d) atomicAdd(&ctl->children, d);
        if (e) atomicAdd(&ctl->guard_hits, e);
        if (f) atomicAdd(&ctl->plans, f);
        if (g) atomicAdd(&ctl->candidates, g);
        if (m) atomicMax(&ctl->max_N, m);
    }
}

struct SharedTables {
    float4 syn[kSynRows];
    float sqz_e[QED_SQZ_E_JMAX - QED_SQZ_E_JMIN];
    float sqz_p[QED_SQZ_P_JMAX - QED_SQZ_P_JMIN];
};

__device__ __forceinline__ void stage_tables(SharedTables& sm) {
    stage_syn_table(sm.syn);
    for (int i = threadIdx.x; i < QED_SQZ_E_JMAX - QED_SQZ_E_JMIN; i += blockDim.x)
        sm.sqz_e[i] = qed_sqz_emission[i];
    for (int i = threadIdx.x; i < QED_SQZ_P_JMAX - QED_SQZ_P_JMIN; i += blockDim.x)
        sm.sqz_p[i] = qed_sqz_pair[i];
}

// ---------------------------------------------------------------------------
// Synchrotron sweep
// ---------------------------------------------------------------------------
template <bool W1, bool W2>
__global__ void __launch_bounds__(kSweepThreads) k_sweep(const float* __restrict__ y,
                                                         float* __restrict__ F1,
                                                         float* __restrict__ F2, long long n,
                                                         int vec) {
    __shared__ float4 tbl[kSynRows];
    stage_syn_table(tbl);
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long done = 0;
    if (vec) {
        const long long n4 = n >> 2;
        const float4* y4 = reinterpret_cast<const float4*>(y);
        for (long long i = t; i < n4; i += stride) {
            const float4 v = __ldcs(y4 + i);
            float4 a, b;
            synchrotron_FG(tbl, v.x, a.x, b.x);
            synchrotron_FG(tbl, v.y, a.y, b.y);
            synchrotron_FG(tbl, v.z, a.z, b.z);
            synchrotron_FG(tbl, v.w, a.w, b.w);
            if (W1) __stcs(reinterpret_cast<float4*>(F1) + i, a);
            if (W2) __stcs(reinterpret_cast<float4*>(F2) + i, b);
        }
        done = n4 << 2;
    }
    for (long long i = done + t; i < n; i += stride) {
        float a, b;
        synchrotron_FG(tbl, y[i], a, b);
        if (W1) F1[i] = a;
        if (W2) F2[i] = b;
    }
}

__global__ void __launch_bounds__(kSweepThreads) k_generate(uint32_t k0, uint32_t k1, long long n,
                                                            float lo, float log2_ratio,
                                                            float* checksum, float* y_out,
                                                            float* F1_out, float* F2_out) {
    __shared__ float4 tbl[kSynRows];
    stage_syn_table(tbl);
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long nblk = (n + 3) >> 2;
    float acc = 0.0f;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < nblk; j += stride) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)(j >> 32), 0u, 0u), k0, k1);
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long i = 4 * j + q;
            const float yv = lo * exp2f(u01(w[q]) * log2_ratio);
            float a, b;
            synchrotron_FG(tbl, yv, a, b);
            if (i < n) {
                acc += a + b;
                if (y_out) y_out[i] = yv;
                if (F1_out) F1_out[i] = a;
                if (F2_out) F2_out[i] = b;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (checksum && (threadIdx.x & 31) == 0) atomicAdd(checksum, acc);
}

// ---------------------------------------------------------------------------
// Planner
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kColdThreads) k_plan(DevParticles P, StepParams SP, long long n,
                                                       float* chi_out, uint32_t* N_out) {
    __shared__ SharedTables sm;
    stage_tables(sm);
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint8_t type = P.type[i];
        const bool photon = type == QED_PHOTON;
        float chi = 0.0f;
        uint32_t N = 0;
        const bool active = type <= QED_PHOTON &&
                            (photon ? (SP.process_mask & QED_PROC_PAIR)
                                    : (SP.process_mask & QED_PROC_EMISSION));
        float eps;
        chi = chi_ff(photon, P.px[i], P.py[i], P.pz[i], P.Ex[i], P.Ey[i], P.Ez[i], P.Bx[i],
                     P.By[i], P.Bz[i], SP.inv_Es, &eps);
        if (active && eps > 0.0f) {
            const Plan pl = make_plan(SP, sm.sqz_e, sm.sqz_p, photon, chi, eps, SP.dt);
            N = pl.N;
        }
        if (chi_out) chi_out[i] = chi;
        if (N_out) N_out[i] = N;
    }
}

// ---------------------------------------------------------------------------
// Events
// ---------------------------------------------------------------------------
struct PState {
    float px, py, pz;
};

// Reserve rows for children; on overflow mark the reserved rows removed and
// record the capacity error.
__device__ __forceinline__ long long reserve_rows(const DevParticles& P, DevCtl* ctl, int n) {
    const long long slot =
        (long long)atomicAdd(reinterpret_cast<unsigned long long*>(P.count), (unsigned long long)n);
    if (slot + n > P.capacity) {
        for (long long j = slot; j < slot + n && j < P.capacity; ++j) {
            P.type[j] = QED_REMOVED;
            P.id[j] = 0;
        }
        atomicMax(&ctl->required, slot + n);
        atomicExch(&ctl->status, (int)QED_ERR_CAPACITY);
        return -1;
    }
    return slot;
}

__device__ __forceinline__ void write_child(const DevParticles& P, const Scratch& S, long long j,
                                            long long parent, float px, float py, float pz,
                                            uint64_t id, uint8_t type, double t_rem) {
    P.px[j] = px;
    P.py[j] = py;
    P.pz[j] = pz;
    P.Ex[j] = P.Ex[parent];
    P.Ey[j] = P.Ey[parent];
    P.Ez[j] = P.Ez[parent];
    P.Bx[j] = P.Bx[parent];
    P.By[j] = P.By[parent];
    P.Bz[j] = P.Bz[parent];
    P.w[j] = P.w[parent];
    P.id[j] = id;
    P.type[j] = type;
    S.t_rem[j] = t_rem;
}

// Apply an accepted event (recoil or decay, children, log).  Returns true if
// the particle was removed (photon decay).
__device__ bool apply_event(const DevParticles& P, const Scratch& S, const StepParams& SP,
                            DevCtl* ctl, long long i, uint64_t id, bool photon, float x,
                            float eps, float chi, uint32_t s, double t_after, PState& st,
                            Stats& stats, bool write_rows) {
    const uint4 cid = philox4x32_10(make_uint4((uint32_t)id, (uint32_t)(id >> 32), SP.step, s),
                                    (uint32_t)SP.seed ^ kChildKeyLo,
                                    (uint32_t)(SP.seed >> 32) ^ kChildKeyHi);
    const uint64_t id0 = ((uint64_t)cid.x | ((uint64_t)cid.y << 32)) | (1ull << 63);
    const uint64_t id1 = ((uint64_t)cid.z | ((uint64_t)cid.w << 32)) | (1ull << 63);
    float delta;
    bool removed = false;
    if (!photon) {
        delta = x * x * x;
        if (write_rows) {
            const long long j = reserve_rows(P, ctl, 1);
            if (j >= 0)
                write_child(P, S, j, i, delta * st.px, delta * st.py, delta * st.pz, id0,
                            QED_PHOTON, t_after);
        }
        if (SP.recoil) {
            if (delta < 1e-6f && eps > 1e4f) {
                const double f = 1.0 - (double)delta;
                st.px = (float)(f * (double)st.px);
                st.py = (float)(f * (double)st.py);
                st.pz = (float)(f * (double)st.pz);
            } else if (delta < 0.5f) {
                st.px = fmaf(-delta, st.px, st.px);
                st.py = fmaf(-delta, st.py, st.py);
                st.pz = fmaf(-delta, st.pz, st.pz);
            } else {
                const float omd = (1.0f - x) * (1.0f + x + x * x);
                st.px *= omd;
                st.py *= omd;
                st.pz *= omd;
            }
        }
        stats.emissions++;
        stats.children++;
    } else {
        delta = x;
        if (write_rows) {
            const long long j = reserve_rows(P, ctl, 2);
            if (j >= 0) {
                const float omd = 1.0f - x;
                write_child(P, S, j, i, x * st.px, x * st.py, x * st.pz, id0, QED_ELECTRON,
                            t_after);
                write_child(P, S, j + 1, i, omd * st.px, omd * st.py, omd * st.pz, id1,
                            QED_POSITRON, t_after);
            }
        }
        removed = SP.recoil != 0;
        stats.pairs++;
        stats.children += 2;
    }
    if (write_rows && S.log) {
        const long long k = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(S.log_count), 1ull);
        if (k < S.log_cap) {
            qed_event_record r;
            r.parent_id = id;
            r.child_id0 = id0;
            r.child_id1 = photon ? id1 : 0ull;
            r.s = s;
            r.kind = photon ? 2u : 1u;
            r.delta = delta;
            r.chi = chi;
            S.log[k] = r;
        }
    }
    return removed;
}

__device__ __forceinline__ bool process_enabled(const StepParams& SP, bool photon) {
    return photon ? (SP.process_mask & QED_PROC_PAIR) != 0
                  : (SP.process_mask & QED_PROC_EMISSION) != 0;
}

__device__ __forceinline__ void push_hot(const Scratch& S, DevCtl* ctl, long long i, uint32_t s,
                                         double t_rem) {
    const unsigned int k = atomicAdd(&ctl->hot_tail, 1u);
    HotItem it;
    it.idx = (uint32_t)i;
    it.s = s;
    it.t_rem = t_rem;
    S.hot[k] = it;
}

// One thread per particle.  first_pass: rows [0, pass_end) with the full step;
// otherwise rows [pass_begin, pass_end) (children) with their stored time.
__global__ void __launch_bounds__(kColdThreads) k_cold(DevParticles P, StepParams SP, Scratch S,
                                                       DevCtl* ctl, int first_pass) {
    __shared__ SharedTables sm;
    stage_tables(sm);
    __syncthreads();
    if (ctl->status == (int)QED_ERR_TIMEOUT) return;
    const long long begin = first_pass ? 0 : ctl->pass_begin;
    const long long end = ctl->pass_end;
    const long long stride = (long long)gridDim.x * blockDim.x;
    Stats stats;
    const uint32_t k0 = (uint32_t)SP.seed, k1 = (uint32_t)(SP.seed >> 32);
    for (long long i = begin + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < end;
         i += stride) {
        const uint8_t type = P.type[i];
        if (type > QED_PHOTON) continue;
        const bool photon = type == QED_PHOTON;
        if (!process_enabled(SP, photon)) continue;
        double t_rem = first_pass ? SP.dt : S.t_rem[i];
        if (!(t_rem > 0.0)) continue;
        const uint64_t id = P.id[i];
        PState st{P.px[i], P.py[i], P.pz[i]};
        const float Ex = P.Ex[i], Ey = P.Ey[i], Ez = P.Ez[i];
        const float Bx = P.Bx[i], By = P.By[i], Bz = P.Bz[i];
        bool changed = false, removed = false;
        uint32_t s = 0;
        uint4 blk = make_uint4(0, 0, 0, 0);
        uint32_t blk_idx = 0xffffffffu;
        while (t_rem > 0.0) {
            float eps;
            const float chi = chi_ff(photon, st.px, st.py, st.pz, Ex, Ey, Ez, Bx, By, Bz,
                                     SP.inv_Es, &eps);
            if (!(eps > 0.0f)) break;
            const Plan pl = make_plan(SP, sm.sqz_e, sm.sqz_p, photon, chi, eps, t_rem);
            stats.plans++;
            stats.guard += pl.guard ? 1 : 0;
            stats.max_N = max(stats.max_N, pl.N);
            if (pl.N >= kHotMin) {
                if (changed) {
                    P.px[i] = st.px;
                    P.py[i] = st.py;
                    P.pz[i] = st.pz;
                    changed = false;
                }
                stats.plans--;  // the warp path re-plans and counts it
                push_hot(S, ctl, i, s, t_rem);
                t_rem = 0.0;
                break;
            }
            bool event = false;
            for (uint32_t k = 0; k < pl.N; ++k) {
                const uint32_t b = s >> 1;
                if (b != blk_idx) {
                    blk = philox4x32_10(make_uint4((uint32_t)id, (uint32_t)(id >> 32), SP.step, b),
                                        k0, k1);
                    blk_idx = b;
                }
                const uint32_t rx = (s & 1u) ? blk.z : blk.x;
                const uint32_t ry = (s & 1u) ? blk.w : blk.y;
                stats.substeps++;
                if ((ry >> 9) < pl.T) {
                    stats.cand++;
                    const float x = u01(rx);
                    float delta;
                    const float Pa = acceptance(sm.syn, photon, pl.b, pl.c_h, x, &delta);
                    if (u01(ry) < Pa) {
                        const double t_after =
                            (k + 1 == pl.N) ? 0.0
                                            : __dsub_rn(t_rem, __dmul_rn((double)(k + 1), pl.h));
                        removed = apply_event(P, S, SP, ctl, i, id, photon, x, eps, chi, s,
                                              t_after, st, stats, true);
                        changed = true;
                        ++s;
                        t_rem = t_after;
                        event = true;
                        break;
                    }
                }
                ++s;
            }
            if (removed) break;
            if (!event) t_rem = 0.0;
        }
        if (removed) {
            P.type[i] = QED_REMOVED;
        } else if (changed) {
            P.px[i] = st.px;
            P.py[i] = st.py;
            P.pz[i] = st.pz;
        }
    }
    flush_stats(stats, ctl);
}

// One warp per queued particle.
__global__ void __launch_bounds__(kHotThreads) k_hot(DevParticles P, StepParams SP, Scratch S,
                                                     DevCtl* ctl) {
    __shared__ SharedTables sm;
    stage_tables(sm);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned int tail = ctl->hot_tail;
    const uint32_t k0 = (uint32_t)SP.seed, k1 = (uint32_t)(SP.seed >> 32);
    Stats stats;  // counted on lane 0 only
    while (true) {
        unsigned int q = 0;
        if (lane == 0) q = atomicAdd(&ctl->hot_head, 1u);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= tail) break;
        const HotItem it = S.hot[q];
        const long long i = it.idx;
        const uint8_t type = P.type[i];
        const bool photon = type == QED_PHOTON;
        const uint64_t id = P.id[i];
        PState st{P.px[i], P.py[i], P.pz[i]};
        const float Ex = P.Ex[i], Ey = P.Ey[i], Ez = P.Ez[i];
        const float Bx = P.Bx[i], By = P.By[i], Bz = P.Bz[i];
        uint32_t s = it.s;
        double t_rem = it.t_rem;
        bool removed = false, changed = false;
        while (t_rem > 0.0) {
            float eps;
            const float chi = chi_ff(photon, st.px, st.py, st.pz, Ex, Ey, Ez, Bx, By, Bz,
                                     SP.inv_Es, &eps);
            if (!(eps > 0.0f)) break;
            const Plan pl = make_plan(SP, sm.sqz_e, sm.sqz_p, photon, chi, eps, t_rem);
            if (lane == 0) {
                stats.plans++;
                stats.guard += pl.guard ? 1 : 0;
                stats.max_N = max(stats.max_N, pl.N);
            }
            uint32_t kdone = 0;
            bool event = false;
            while (kdone < pl.N) {
                const uint32_t sb = s;
                const uint32_t sa = sb & ~1u;
                const uint32_t lim = sb + (pl.N - kdone);
                const uint32_t s0 = sa + 2u * (uint32_t)lane;
                const uint4 r = philox4x32_10(
                    make_uint4((uint32_t)id, (uint32_t)(id >> 32), SP.step, (sa >> 1) + lane), k0, k1);
                const bool v0 = s0 >= sb && s0 < lim;
                const bool v1 = s0 + 1 >= sb && s0 + 1 < lim;
                const bool c0 = v0 && (r.y >> 9) < pl.T;
                const bool c1 = v1 && (r.w >> 9) < pl.T;
                bool a0 = false, a1 = false;
                float dtmp;
                if (c0) a0 = u01(r.y) < acceptance(sm.syn, photon, pl.b, pl.c_h, u01(r.x), &dtmp);
                if (c1) a1 = u01(r.w) < acceptance(sm.syn, photon, pl.b, pl.c_h, u01(r.z), &dtmp);
                const unsigned int m0 = __ballot_sync(0xffffffffu, a0);
                const unsigned int m1 = __ballot_sync(0xffffffffu, a1);
                const unsigned int nc =
                    __popc(__ballot_sync(0xffffffffu, c0)) + __popc(__ballot_sync(0xffffffffu, c1));
                if (lane == 0) stats.cand += nc;
                if ((m0 | m1) == 0u) {
                    const uint32_t chunk_end = min(sa + 64u, lim);
                    if (lane == 0) stats.substeps += chunk_end - sb;
                    kdone += chunk_end - sb;
                    s = chunk_end;
                    continue;
                }
                const int p0 = m0 ? 2 * (__ffs(m0) - 1) : 1 << 30;
                const int p1 = m1 ? 2 * (__ffs(m1) - 1) + 1 : 1 << 30;
                const int pos = min(p0, p1);
                const uint32_t s_ev = sa + (uint32_t)pos;
                const float xo = (pos & 1) ? u01(r.z) : u01(r.x);
                const float x = __shfl_sync(0xffffffffu, xo, pos >> 1);
                const uint32_t k_ev = kdone + (s_ev - sb);
                if (lane == 0) stats.substeps += s_ev - sb + 1;
                const double t_after =
                    (k_ev + 1 == pl.N) ? 0.0 : __dsub_rn(t_rem, __dmul_rn((double)(k_ev + 1), pl.h));
                removed = apply_event(P, S, SP, ctl, i, id, photon, x, eps, chi, s_ev, t_after,
                                      st, stats, lane == 0);
                changed = true;
                s = s_ev + 1;
                t_rem = t_after;
                event = true;
                break;
            }
            if (removed) break;
            if (!event) t_rem = 0.0;
        }
        if (lane == 0) {
            if (removed) P.type[i] = QED_REMOVED;
            else if (changed) {
                P.px[i] = st.px;
                P.py[i] = st.py;
                P.pz[i] = st.pz;
            }
        }
    }
    if (lane != 0) stats = Stats();
    flush_stats(stats, ctl);
}

__global__ void k_step_init(DevCtl* ctl, long long* count, long long capacity) {
    DevCtl c;
    memset(&c, 0, sizeof c);
    long long n = *count;
    if (n < 0) n = 0;
    if (n > capacity) n = capacity;
    *count = n;
    c.pass_begin = 0;
    c.pass_end = n;
    *ctl = c;
}

__global__ void k_advance(DevCtl* ctl, long long* count, long long capacity, int more_allowed) {
    long long n = *count;
    if (n > capacity) {
        n = capacity;
        *count = capacity;
    }
    ctl->pass_begin = ctl->pass_end;
    ctl->pass_end = n;
    ctl->hot_head = 0;
    ctl->hot_tail = 0;
    ctl->passes += 1;
    ctl->more = (more_allowed && n > ctl->pass_begin && ctl->status == 0) ? 1 : 0;
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct qed_ctx {
    qed_config cfg;
    cudaStream_t stream;
    int device;
    int sms;
    DevCtl* d_ctl;
    DevCtl* h_ctl;          // pinned
    double* d_trem;
    HotItem* d_hot;
    long long scratch_cap;
    qed_event_record* log;
    long long log_cap;
    long long* log_count;
    int cold_blocks, hot_blocks;
    char err[512];
};

namespace {

qed_status set_err(qed_ctx* ctx, qed_status st, const char* what) {
    if (ctx) snprintf(ctx->err, sizeof ctx->err, "%s", what);
    return st;
}

qed_status cuda_check(qed_ctx* ctx, cudaError_t e, const char* where) {
    if (e == cudaSuccess) return QED_OK;
    if (ctx) snprintf(ctx->err, sizeof ctx->err, "%s: %s", where, cudaGetErrorString(e));
    return QED_ERR_CUDA;
}

#define QED_CUDA(ctx, call)                                         \
    do {                                                            \
        qed_status _s = cuda_check((ctx), (call), #call);           \
        if (_s != QED_OK) return _s;                                \
    } while (0)

StepParams make_params(const qed_config& c, uint64_t step) {
    StepParams P;
    P.seed = c.seed;
    P.dt = c.dt_periods;
    const double period = c.lambda_m / kCLight;
    const double R = kAlpha / kTauC * period;                 // 1 / period
    P.K = (float)(1.7320508075688772 / kPiD * R);
    const double omega = 2.0 * kPiD * kCLight / c.lambda_m;
    P.inv_Es = (float)(omega * kTauC);                        // 1 / E_s in code units
    P.p_max = c.p_max;
    P.pair_coeff = c.pair_bound_coeff;
    P.step = (uint32_t)step;
    P.process_mask = c.process_mask;
    P.recoil = c.recoil;
    P.cascade = c.cascade_in_step;
    return P;
}

DevParticles to_dev(const qed_particles* p) {
    DevParticles d;
    d.px = p->px; d.py = p->py; d.pz = p->pz;
    d.Ex = p->Ex; d.Ey = p->Ey; d.Ez = p->Ez;
    d.Bx = p->Bx; d.By = p->By; d.Bz = p->Bz;
    d.w = p->w; d.id = p->id; d.type = p->type;
    d.count = reinterpret_cast<long long*>(p->count);
    d.capacity = p->capacity;
    return d;
}

bool particles_ok(const qed_particles* p) {
    return p && p->px && p->py && p->pz && p->Ex && p->Ey && p->Ez && p->Bx && p->By && p->Bz &&
           p->w && p->id && p->type && p->count && p->capacity > 0 && p->capacity < (1ll << 32);
}

qed_status ensure_scratch(qed_ctx* ctx, long long cap) {
    if (ctx->scratch_cap >= cap) return QED_OK;
    if (ctx->d_trem) cudaFree(ctx->d_trem);
    if (ctx->d_hot) cudaFree(ctx->d_hot);
    ctx->d_trem = nullptr;
    ctx->d_hot = nullptr;
    ctx->scratch_cap = 0;
    QED_CUDA(ctx, cudaMalloc(&ctx->d_trem, sizeof(double) * cap));
    QED_CUDA(ctx, cudaMalloc(&ctx->d_hot, sizeof(HotItem) * cap));
    ctx->scratch_cap = cap;
    return QED_OK;
}

void fill_stats(const DevCtl& c, qed_step_stats* out, long long count) {
    out->substeps = c.substeps;
    out->emissions = c.emissions;
    out->pairs = c.pairs;
    out->children = c.children;
    out->guard_hits = c.guard_hits;
    out->plans = c.plans;
    out->candidates = c.candidates;
    out->max_N = c.max_N;
    out->status = c.status;
    out->required_capacity = c.required;
    out->count = count;
    out->passes = c.passes;
    out->reserved = 0;
}

}  // namespace

extern "C" {

void qed_config_default(qed_config* c) {
    if (!c) return;
    c->seed = 20081046ull;
    c->dt_periods = 0.1;
    c->lambda_m = 1e-6;
    c->p_max = 0.01f;
    c->pair_bound_coeff = 0.1f;
    c->process_mask = QED_PROC_EMISSION | QED_PROC_PAIR;
    c->cascade_in_step = 1;
    c->recoil = 1;
    c->max_passes = 64;
}

qed_status qed_init(qed_ctx** out, const qed_config* cfg, void* stream) {
    if (!out || !cfg) return QED_ERR_ARG;
    *out = nullptr;
    if (!(cfg->p_max > 0.0f && cfg->p_max <= 1.0f) || !(cfg->dt_periods > 0.0) ||
        !(cfg->lambda_m > 0.0) || !(cfg->pair_bound_coeff > 0.0f))
        return QED_ERR_ARG;
    qed_ctx* ctx = new (std::nothrow) qed_ctx();
    if (!ctx) return QED_ERR_ARG;
    ctx->cfg = *cfg;
    if (ctx->cfg.max_passes <= 0) ctx->cfg.max_passes = 64;
    ctx->stream = (cudaStream_t)stream;
    qed_status st = cuda_check(ctx, cudaGetDevice(&ctx->device), "cudaGetDevice");
    if (st == QED_OK)
        st = cuda_check(ctx, cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount,
                                                    ctx->device), "sm count");
    if (st == QED_OK) st = cuda_check(ctx, cudaMalloc(&ctx->d_ctl, sizeof(DevCtl)), "cudaMalloc");
    if (st == QED_OK)
        st = cuda_check(ctx, cudaHostAlloc(&ctx->h_ctl, sizeof(DevCtl), cudaHostAllocDefault),
                        "cudaHostAlloc");
    if (st == QED_OK) st = cuda_check(ctx, cudaMemset(ctx->d_ctl, 0, sizeof(DevCtl)), "memset");
    if (st == QED_OK) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cold, kColdThreads, 0);
        ctx->cold_blocks = ctx->sms * (per_sm > 0 ? per_sm : 1);
        per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hot, kHotThreads, 0);
        ctx->hot_blocks = ctx->sms * (per_sm > 0 ? per_sm : 1);
        st = cuda_check(ctx, cudaGetLastError(), "occupancy");
    }
    if (st != QED_OK) {
        qed_destroy(ctx);
        return st;
    }
    *out = ctx;
    return QED_OK;
}

qed_status qed_destroy(qed_ctx* ctx) {
    if (!ctx) return QED_ERR_ARG;
    if (ctx->stream || ctx->d_ctl) cudaStreamSynchronize(ctx->stream);
    if (ctx->d_ctl) cudaFree(ctx->d_ctl);
    if (ctx->h_ctl) cudaFreeHost(ctx->h_ctl);
    if (ctx->d_trem) cudaFree(ctx->d_trem);
    if (ctx->d_hot) cudaFree(ctx->d_hot);
    delete ctx;
    return QED_OK;
}

const char* qed_last_error(const qed_ctx* ctx) { return ctx ? ctx->err : "null context"; }

qed_status qed_synchrotron_F1F2(qed_ctx* ctx, const float* y, float* F1, float* F2, int64_t n) {
    if (!ctx) return QED_ERR_ARG;
    if (!y || n < 0) return set_err(ctx, QED_ERR_ARG, "qed_synchrotron_F1F2: bad argument");
    if (n == 0 || (!F1 && !F2)) return QED_OK;
    const int vec = ((((uintptr_t)y) | ((uintptr_t)F1) | ((uintptr_t)F2)) & 15u) == 0 ? 1 : 0;
    long long work = vec ? (n + 3) / 4 : n;
    long long blocks = (work + kSweepThreads - 1) / kSweepThreads;
    const long long max_blocks = (long long)ctx->sms * 8;
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    if (F1 && F2)
        k_sweep<true, true><<<(int)blocks, kSweepThreads, 0, ctx->stream>>>(y, F1, F2, n, vec);
    else if (F1)
        k_sweep<true, false><<<(int)blocks, kSweepThreads, 0, ctx->stream>>>(y, F1, F2, n, vec);
    else
        k_sweep<false, true><<<(int)blocks, kSweepThreads, 0, ctx->stream>>>(y, F1, F2, n, vec);
    return cuda_check(ctx, cudaGetLastError(), "k_sweep");
}

qed_status qed_synchrotron_generate(qed_ctx* ctx, uint64_t seed, int64_t n, float lo, float hi,
                                    float* checksum, float* y_out, float* F1_out, float* F2_out) {
    if (!ctx) return QED_ERR_ARG;
    if (n < 0 || !(lo > 0.0f) || !(hi >= lo))
        return set_err(ctx, QED_ERR_ARG, "qed_synchrotron_generate: bad argument");
    if (n == 0) return QED_OK;
    long long blocks = ((n + 3) / 4 + kSweepThreads - 1) / kSweepThreads;
    const long long max_blocks = (long long)ctx->sms * 8;
    if (blocks > max_blocks) blocks = max_blocks;
    k_generate<<<(int)blocks, kSweepThreads, 0, ctx->stream>>>(
        (uint32_t)seed, (uint32_t)(seed >> 32), n, lo, log2f(hi / lo), checksum, y_out, F1_out,
        F2_out);
    return cuda_check(ctx, cudaGetLastError(), "k_generate");
}

qed_status qed_plan(qed_ctx* ctx, const qed_particles* p, int64_t n, float* chi, uint32_t* N) {
    if (!ctx) return QED_ERR_ARG;
    if (!particles_ok(p) || n < 0 || n > p->capacity)
        return set_err(ctx, QED_ERR_ARG, "qed_plan: bad argument");
    if (n == 0) return QED_OK;
    const StepParams SP = make_params(ctx->cfg, 0);
    long long blocks = (n + kColdThreads - 1) / kColdThreads;
    if (blocks > ctx->cold_blocks) blocks = ctx->cold_blocks;
    k_plan<<<(int)blocks, kColdThreads, 0, ctx->stream>>>(to_dev(p), SP, n, chi, N);
    return cuda_check(ctx, cudaGetLastError(), "k_plan");
}

qed_status qed_set_event_log(qed_ctx* ctx, qed_event_record* records, int64_t capacity,
                             int64_t* count) {
    if (!ctx) return QED_ERR_ARG;
    if (records && (capacity < 0 || !count))
        return set_err(ctx, QED_ERR_ARG, "qed_set_event_log: bad argument");
    ctx->log = records;
    ctx->log_cap = records ? capacity : 0;
    ctx->log_count = records ? reinterpret_cast<long long*>(count) : nullptr;
    return QED_OK;
}

qed_status qed_event_step(qed_ctx* ctx, const qed_particles* p, uint64_t step_index,
                          qed_step_stats* out) {
    if (!ctx) return QED_ERR_ARG;
    if (!particles_ok(p) || step_index > 0xffffffffull)
        return set_err(ctx, QED_ERR_ARG, "qed_event_step: bad argument");
    qed_status st = ensure_scratch(ctx, p->capacity);
    if (st != QED_OK) return st;
    const StepParams SP = make_params(ctx->cfg, step_index);
    const DevParticles D = to_dev(p);
    Scratch S;
    S.t_rem = ctx->d_trem;
    S.hot = ctx->d_hot;
    S.log = ctx->log;
    S.log_cap = ctx->log_cap;
    S.log_count = ctx->log_count;
    const bool cascade = ctx->cfg.cascade_in_step &&
                         (ctx->cfg.process_mask & (QED_PROC_EMISSION | QED_PROC_PAIR)) ==
                             (QED_PROC_EMISSION | QED_PROC_PAIR);
    k_step_init<<<1, 1, 0, ctx->stream>>>(ctx->d_ctl, D.count, D.capacity);
    for (int pass = 0; pass < ctx->cfg.max_passes; ++pass) {
        k_cold<<<ctx->cold_blocks, kColdThreads, 0, ctx->stream>>>(D, SP, S, ctx->d_ctl,
                                                                    pass == 0 ? 1 : 0);
        k_hot<<<ctx->hot_blocks, kHotThreads, 0, ctx->stream>>>(D, SP, S, ctx->d_ctl);
        k_advance<<<1, 1, 0, ctx->stream>>>(ctx->d_ctl, D.count, D.capacity, cascade ? 1 : 0);
        QED_CUDA(ctx, cudaGetLastError());
        if (!cascade) break;
        QED_CUDA(ctx, cudaMemcpyAsync(ctx->h_ctl, ctx->d_ctl, sizeof(DevCtl),
                                      cudaMemcpyDeviceToHost, ctx->stream));
        QED_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (!ctx->h_ctl->more) break;
    }
    if (out) return qed_read_stats(ctx, out);
    return QED_OK;
}

qed_status qed_read_stats(qed_ctx* ctx, qed_step_stats* out) {
    if (!ctx || !out) return QED_ERR_ARG;
    QED_CUDA(ctx, cudaMemcpyAsync(ctx->h_ctl, ctx->d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    QED_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    fill_stats(*ctx->h_ctl, out, ctx->h_ctl->pass_end);
    return (qed_status)ctx->h_ctl->status;
}

size_t qed_abi_struct_size(const char* name) {
    if (!name) return 0;
    if (!strcmp(name, "qed_config")) return sizeof(qed_config);
    if (!strcmp(name, "qed_particles")) return sizeof(qed_particles);
    if (!strcmp(name, "qed_step_stats")) return sizeof(qed_step_stats);
    if (!strcmp(name, "qed_event_record")) return sizeof(qed_event_record);
    return 0;
}

}  // extern "C"
