// GB300 (sm_103a) implementation of the C ABI in include/qed.h.
//
// Kernels
//   k_sweep / k_generate   synchrotron functions over an array or over
//                          in-kernel arguments (Sec. 3.2.1)
//   k_plan                 chi and the sub-step count (planning, Algorithms 1/2)
//   k_cold                 thread pass: one lane per row for the plan and
//                          events, the warp's lanes together for the draws;
//                          plans of at least hot_min sub-steps are queued
//   k_hot_lanes            hot pass (persistent): long plans one warp each
//                          (64 sub-steps per iteration, lane l drawing the
//                          Philox block of sub-steps 2l, 2l+1), medium plans
//                          one lane each with warp-shared draws; in sampler
//                          mode the warp of a sampler particle evaluates the
//                          network for its events
//   k_advance              closes a cascade generation; below tail_rows rows
//                          it hands the rest of the step to the tail pass
//   k_tail_begin / k_step / k_tail_end
//                          tail pass: after one more thread pass, a persistent
//                          kernel takes the queue and every child appended
//                          later (no generations), children published by
//                          their writers
//
// Every sub-step draws (x, y) from Philox4x32-10 at counter
// (id_lo, id_hi, step, s/2) under key = seed (even s: words 0,1; odd s:
// words 2,3).  Before evaluating the acceptance function the kernels compare
// y with an upper bound of that function over all x (the squeeze); this
// changes no decision and skips the synchrotron functions for most sub-steps.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>
#include <vector>

#include "qed.h"
#include "qed_device.cuh"
#include "qed_sampler.cuh"

using namespace qed;

namespace {


// Defaults measured on the 2^24 clumped population (coordinate search over
// hot_min 32..128 and long_min 128..2048)
constexpr uint32_t kHotMinDefault = 32;    // plans with N >= hot_min go to the hot pass
constexpr uint32_t kLongMinDefault = 256;  // ... and with N >= long_min to its warp mode
constexpr long long kTailRowsDefault = 1ll << 17;   // generations below this go to the tail pass

// Minimum resident blocks per SM requested from the register allocator:
// 3 x 256 threads hold the thread and hot passes at 80 registers (24 warps
// per SM).
#ifndef QED_COLD_MIN_BLOCKS
#define QED_COLD_MIN_BLOCKS 3
#endif
#ifndef QED_LANES_MIN_BLOCKS
#define QED_LANES_MIN_BLOCKS 3
#endif
constexpr int kColdThreads = 256;
constexpr int kLaneThreads = 256;
constexpr int kSweepThreads = 256;

struct DevCtl {
    unsigned long long substeps, emissions, pairs, children, guard_hits, plans, candidates;
    unsigned long long substeps_warp;
    unsigned long long sampler_events;
    unsigned long long sampler_pairs;
    unsigned int max_N;
    int status;
    long long required;
    long long pass_begin, pass_end;
    unsigned int hot_tail, hot_head;   // long plans: front of the queue array
    unsigned int med_tail, med_head;   // medium plans: back of the queue array
    int more, passes;
    int first_pass;      // 1 until the first generation of the step is done
    int sticky;          // first error of a multi-step graph run: later steps do nothing
    long long live;      // rows kept by the last compaction
    int compact_needed;  // the last compaction found removed rows
    int tail;            // the generations stopped below tail_rows: the tail pass finishes the step
    unsigned int hot_hw;            // long-plan queue entries written by this step's generations
    // tail pass (persistent kernel)
    long long n0;                   // first child row of the tail (rows before it are done)
    unsigned long long child_head;  // next child row (from n0) to take
    unsigned long long finished;    // work units (queue entries, children) complete
    unsigned int step_tail;         // long plans queued by the persistent kernel, stored
                                    // after the thread pass's hot_tail entries
    int skip;                       // the tail pass does nothing
    unsigned long long push_head;   // push mode: next row of the generation to take
    unsigned int samp_tail, samp_head;   // event-driven sampler: its queue of this generation
    long long n_init;               // rows at the start of the step (the rest are children)
    unsigned long long beat;        // persistent passes: progress of long chains, so that
                                    // idle warps tell a long chain from a stalled step
};

// Type byte of a child row that has been reserved but not yet written: in the
// tail pass the writer stores the row, fences, then stores its real type.
constexpr uint8_t kNotReady = 0xFF;
// Row index of a long-plan queue entry that has not been written yet.
constexpr uint32_t kNoItem = 0xFFFFFFFFu;

struct HotItem {
    uint32_t idx;
    uint32_t s;
    ftime t_rem;     // remaining time (periods)
};

struct DevParticles {
    float *px, *py, *pz, *Ex, *Ey, *Ez, *Bx, *By, *Bz, *w;
    uint64_t* id;
    uint8_t* type;
    long long* count;
    long long capacity;
};

struct Scratch {
    ftime* t_rem;           // remaining time of appended children (capacity)
    HotItem* hot;           // queue of hot-pass particles (hot_cap entries), filled
                            // from both ends: long plans from the front,
                            // medium plans from the back
    long long hot_cap;
    HotItem* samp;          // event-driven sampler's queue (capacity entries; null when off)
    qed_event_record* log;  // optional
    long long log_cap;
    long long* log_count;
};

// Per-thread counters of one launch (32-bit: a thread's share of one launch
// stays far below 2^32); summed per warp and added to the control block.
struct Stats {
    unsigned int substeps = 0, emissions = 0, pairs = 0, children = 0, guard = 0, plans = 0,
                 cand = 0, warp_substeps = 0, sampled = 0, sampled_p = 0;
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
                             e = warp_sum(st.guard), f = warp_sum(st.plans), g = warp_sum(st.cand),
                             h = warp_sum(st.warp_substeps),  // 64-bit sums of 32-bit counters
                             q = warp_sum(st.sampled), qp = warp_sum(st.sampled_p);
    const unsigned int m = warp_max(st.max_N);
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd(&ctl->substeps, a);
        if (b) atomicAdd(&ctl->emissions, b);
        if (c) atomicAdd(&ctl->pairs, c);
        if (d) atomicAdd(&ctl->children, d);
        if (e) atomicAdd(&ctl->guard_hits, e);
        if (f) atomicAdd(&ctl->plans, f);
        if (g) atomicAdd(&ctl->candidates, g);
        if (h) atomicAdd(&ctl->substeps_warp, h);
        if (q) atomicAdd(&ctl->sampler_events, q);
        if (qp) atomicAdd(&ctl->sampler_pairs, qp);
        if (m) atomicMax(&ctl->max_N, m);
    }
}

struct SharedTables {
    SynTable syn;
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
    __shared__ SynTable tbl;
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
    __shared__ SynTable tbl;
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
// The fields the planner reads from a row.
struct PlanRow {
    uint8_t type;
    float px, py, pz, Ex, Ey, Ez, Bx, By, Bz;
};

__device__ __forceinline__ PlanRow load_plan_row(const DevParticles& P, long long i) {
    return PlanRow{P.type[i], P.px[i], P.py[i], P.pz[i], P.Ex[i],
                   P.Ey[i],   P.Ez[i], P.Bx[i], P.By[i], P.Bz[i]};
}

// One row of k_plan: its plan, the outputs, and its cell's count.
__device__ __forceinline__ void plan_row(const StepParams& SP, const SharedTables& sm,
                                         const PlanRow& r, long long i, uint32_t c,
                                         float* chi_out, uint32_t* N_out, long long ncells,
                                         unsigned int* N_cell) {
    const bool photon = r.type == QED_PHOTON;
    float chi = 0.0f;
    uint32_t N = 0;
    const bool active = r.type <= QED_PHOTON &&
                        (photon ? (SP.process_mask & QED_PROC_PAIR)
                                : (SP.process_mask & QED_PROC_EMISSION));
    float eps;
    const ftime T0{(float)SP.dt, (float)(SP.dt - (double)(float)SP.dt)};
    const Plan pl = plan_particle(SP, sm.sqz_e, sm.sqz_p, photon, r.px, r.py, r.pz, r.Ex, r.Ey,
                                  r.Ez, r.Bx, r.By, r.Bz, T0, &chi, &eps);
    if (active && eps > 0.0f) N = pl.N;
    if (chi_out) chi_out[i] = chi;
    if (N_out) N_out[i] = N;
    if (N_cell) {
        const bool in = (long long)c < ncells;
        const uint32_t key = in ? c : 0xffffffffu;
        bool one_cell = false;
        if (__activemask() == 0xffffffffu)
            one_cell = __all_sync(0xffffffffu, __shfl_sync(0xffffffffu, key, 0) == key);
        if (one_cell) {
            const uint32_t m = __reduce_max_sync(0xffffffffu, N);
            if ((threadIdx.x & 31) == 0 && in && m > 0u) atomicMax(N_cell + c, m);
        } else if (in && N > 0u) {
            atomicMax(N_cell + c, N);
        }
    }
}

// cell / N_cell (optional): per-cell planning (Algorithm 1 and 2 fix one
// sub-step per cell): N_cell[c] becomes the largest N of the rows of cell c
// (N_cell zeroed by the caller; rows whose cell index is >= ncells are left
// out of it).  Rows of a cell usually sit together in the store: when the 32
// rows of a warp share one cell, their largest count goes to it in one
// atomic.  Each thread loads its next row (one grid stride on) before it
// plans the current one, so that twice the loads are in flight.
__global__ void __launch_bounds__(kColdThreads) k_plan(DevParticles P, StepParams SP, long long n,
                                                       float* chi_out, uint32_t* N_out,
                                                       const uint32_t* __restrict__ cell,
                                                       long long ncells, unsigned int* N_cell,
                                                       const long long* n_dev) {
    __shared__ SharedTables sm;
    stage_tables(sm);
    __syncthreads();
    if (n_dev && *n_dev < n) n = *n_dev;   // rows in use (the store's count)
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PlanRow cur = load_plan_row(P, i);
    uint32_t c_cur = N_cell ? cell[i] : 0u;
    for (; i < n; i += stride) {
        // the next row's loads go out before this row is planned
        const long long nx = i + stride;
        PlanRow nxt = cur;
        uint32_t c_nxt = 0u;
        if (nx < n) {
            nxt = load_plan_row(P, nx);
            c_nxt = N_cell ? cell[nx] : 0u;
        }
        plan_row(SP, sm, cur, i, c_cur, chi_out, N_out, ncells, N_cell);
        cur = nxt;
        c_cur = c_nxt;
    }
}

// ---------------------------------------------------------------------------
// Events
// ---------------------------------------------------------------------------
struct PState {
    float px, py, pz;
};

// Rows stored so far (the count, capped at the capacity), read afresh.
__device__ __forceinline__ unsigned long long stored_rows(const DevParticles& P) {
    const long long c = *reinterpret_cast<volatile long long*>(P.count);
    return (unsigned long long)min(c, P.capacity);
}

// Reserve n rows for children.  `aggregate`: the lanes of the warp that reach
// this call together share one atomic (ballots of the active lanes give each
// lane its offset, the first lane adds the total, the base is broadcast).  On overflow
// the reserved rows are marked removed and the capacity error is recorded.
__device__ __forceinline__ long long reserve_rows(const DevParticles& P, DevCtl* ctl, int n,
                                                  bool aggregate) {
    long long slot;
    if (aggregate) {
        // n is 1 (photon) or 2 (pair): the prefix over the active lanes is
        // exact from two ballots, whatever lanes are active
        const unsigned int act = __activemask();
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(act) - 1;
        const unsigned int m1 = __ballot_sync(act, n == 1);
        const unsigned int m2 = __ballot_sync(act, n == 2);
        const unsigned int below = (1u << lane) - 1u;
        const int offset = __popc(m1 & below) + 2 * __popc(m2 & below);
        const int total = __popc(m1) + 2 * __popc(m2);
        unsigned long long base = 0;
        if (lane == leader)
            base = atomicAdd(reinterpret_cast<unsigned long long*>(P.count),
                             (unsigned long long)total);
        base = __shfl_sync(act, base, leader);
        slot = (long long)base + offset;
    } else {
        slot = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(P.count),
                                    (unsigned long long)n);
    }
    if (slot + n > P.capacity) {
        for (long long j = slot; j < slot + n && j < P.capacity; ++j) {
            P.id[j] = 0;
            __threadfence();   // a tail-pass lane may be waiting for this row
            *reinterpret_cast<volatile uint8_t*>(P.type + j) = QED_REMOVED;
        }
        atomicMax(&ctl->required, slot + n);
        atomicExch(&ctl->status, (int)QED_ERR_CAPACITY);
        return -1;
    }
    return slot;
}

// The parent's fields, copied to its children.
struct Fields {
    float Ex, Ey, Ez, Bx, By, Bz;
};

// Every field of a child row but its type byte, which the caller stores last.
__device__ __forceinline__ void write_child_fields(const DevParticles& P, const Scratch& S,
                                                   long long j, const Fields& F, float w,
                                                   float px, float py, float pz, uint64_t id,
                                                   ftime t_rem) {
    P.px[j] = px;
    P.py[j] = py;
    P.pz[j] = pz;
    P.Ex[j] = F.Ex;
    P.Ey[j] = F.Ey;
    P.Ez[j] = F.Ez;
    P.Bx[j] = F.Bx;
    P.By[j] = F.By;
    P.Bz[j] = F.Bz;
    P.w[j] = w;
    P.id[j] = id;
    S.t_rem[j] = t_rem;
}


constexpr long long kReserveHere = -2;   // apply_event reserves the child rows itself

// Apply an accepted event (recoil or decay, children, log).  Returns true if
// the particle was removed (photon decay).  Thread callers (write_rows) do
// everything themselves, sharing one reservation atomic per warp; warp
// callers (all 32 lanes, identical arguments) reserve and store on lane 0
// (13 stores from one lane measured faster than a 13-way divergent split of
// the stores across lanes).  The reservation is issued first so that its
// latency overlaps the child-id computation.
__device__ __forceinline__ bool apply_event(const DevParticles& P, const Scratch& S, const StepParams& SP,
                            DevCtl* ctl, long long i, uint64_t id, bool photon, float x,
                            float eps, float chi, uint32_t step, uint32_t s, ftime t_after, PState& st,
                            Stats& stats, bool write_rows, bool warp_caller, const Fields& F,
                            bool publish, long long j_pre = kReserveHere) {
    const int nch = photon ? 2 : 1;
    const int lane = threadIdx.x & 31;
    long long j = -1;
    if (j_pre != kReserveHere) {
        j = j_pre;   // reserved by the caller (-1: it did not fit)
    } else if (warp_caller) {
        // lane 0 reserves and stores; its result is first needed at the stores
        if (lane == 0) j = reserve_rows(P, ctl, nch, false);
    } else if (write_rows) {
        j = reserve_rows(P, ctl, nch, true);
    }
    const uint4 cid = philox4x32_10(make_uint4((uint32_t)id, (uint32_t)(id >> 32), step, s),
                                    SP.child_keys);
    const uint64_t id0 = ((uint64_t)cid.x | ((uint64_t)cid.y << 32)) | (1ull << 63);
    const uint64_t id1 = ((uint64_t)cid.z | ((uint64_t)cid.w << 32)) | (1ull << 63);
    float delta;
    bool removed = false;
    float cp[2][3];
    if (!photon) {
        delta = x * x * x;
        cp[0][0] = delta * st.px;
        cp[0][1] = delta * st.py;
        cp[0][2] = delta * st.pz;
        cp[1][0] = cp[1][1] = cp[1][2] = 0.0f;
    } else {
        delta = x;
        const float omd = 1.0f - x;
        cp[0][0] = x * st.px;
        cp[0][1] = x * st.py;
        cp[0][2] = x * st.pz;
        cp[1][0] = omd * st.px;
        cp[1][1] = omd * st.py;
        cp[1][2] = omd * st.pz;
    }
    if (j >= 0) {
        const uint64_t cids[2] = {id0, id1};
        const uint8_t ctypes[2] = {photon ? (uint8_t)QED_ELECTRON : (uint8_t)QED_PHOTON,
                                   (uint8_t)QED_POSITRON};
        if (!warp_caller || lane == 0) {
            const float w = P.w[i];
            for (int r = 0; r < nch; ++r)
                write_child_fields(P, S, j + r, F, w, cp[r][0], cp[r][1], cp[r][2], cids[r],
                                   t_after);
            // in the tail pass another warp may be waiting for these rows:
            // one fence for the event's children, then their type bytes
            if (publish) __threadfence();
            for (int r = 0; r < nch; ++r)
                *reinterpret_cast<volatile uint8_t*>(P.type + j + r) = ctypes[r];
        }
    }
    if (!photon) {
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
        if (!warp_caller || lane == 0) {   // a warp caller counts on lane 0
            stats.emissions++;
            stats.children++;
        }
    } else {
        removed = SP.recoil != 0;
        if (!warp_caller || lane == 0) {
            stats.pairs++;
            stats.children += 2;
        }
    }
    const bool logger = warp_caller ? lane == 0 : write_rows;
    if (logger && S.log) {
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
                                         ftime t_rem, bool long_plan) {
    HotItem it;
    it.idx = (uint32_t)i;
    it.s = s;
    it.t_rem = t_rem;
    if (long_plan) {
        S.hot[atomicAdd(&ctl->hot_tail, 1u)] = it;
    } else {
        S.hot[S.hot_cap - 1 - (long long)atomicAdd(&ctl->med_tail, 1u)] = it;
    }
}

// With the learned sampler on, e+- whose chi lies in a usable bin of its
// range (64 bins uniform in log10 chi over [-2, 2)) are stepped in the hot
// pass's warp mode, where the network is evaluated.
__device__ __forceinline__ bool sampler_bin_ok(const StepParams& SP, float chi) {
    if (!SP.sampler || !(chi >= 1e-2f && chi < 1e2f)) return false;
    const int bin = min(max((int)((log10f(chi) - kMlpLog10Lo) * 16.0f), 0), 63);
    return (SP.net_bins >> bin) & 1ull;
}

// With the event-driven sampler, photons whose plan has candidates (a nonzero
// squeeze threshold) and whose chi_gamma lies in a usable bin of the pair
// sampler decide their decay from the tabulated total pair probability and
// take delta_e from the pair network.
__device__ __forceinline__ bool pair_sampler_ok(const StepParams& SP, float chi, uint32_t T) {
    if (!SP.pnet_bins || T == 0u || !(chi >= 1e-2f && chi < 1e2f)) return false;
    const int bin = min(max((int)((log10f(chi) - kMlpLog10Lo) * 16.0f), 0), 63);
    return (SP.pnet_bins >> bin) & 1ull;
}

// Graph runs keep the global step index as a device base plus the node's
// offset, so that relaunching a graph continues with new step indices.
__device__ __forceinline__ uint32_t step_index(const StepParams& SP) {
    return SP.step_base ? SP.step + *SP.step_base : SP.step;
}

// One round of warp-shared draws.  Every active lane has the sub-steps
// [s, s_end) of its current plan to test; the Philox blocks of those ranges
// are laid end to end (prefix sum of the per-lane block counts) and drawn 32
// at a time, lane f of a round taking block f.  Its owner is the last lane
// whose first block index is <= f (5-step binary search over the lanes), whose
// plan parameters come by shuffle.  Accepted sub-steps are reduced per owner
// with a shared-memory minimum: on return facc[lane] holds the lane's earliest
// accepted sub-step in its range, or kNoEvent.  Called by all 32 lanes.
constexpr uint32_t kNoEvent = 0xffffffffu;
__device__ __forceinline__ void warp_draw_round(const SharedTables& sm, uint32_t* facc,
                                                bool active, uint32_t s, uint32_t s_end,
                                                uint32_t T, float b, float c_h, uint64_t id,
                                                bool photon, uint32_t step, const PhiloxKeys& K,
                                                unsigned int& cand) {
    constexpr unsigned int kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t b0 = s >> 1;
    const uint32_t nblk = (active && s_end > s) ? ((s_end - 1u) >> 1) - b0 + 1u : 0u;
    uint32_t incl = nblk;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kAll, incl, o);
        if (lane >= o) incl += t;
    }
    const uint32_t total = __shfl_sync(kAll, incl, 31);
    const uint32_t excl = incl - nblk;
    facc[lane] = kNoEvent;
    __syncwarp();
    for (uint32_t fb = 0; fb < total; fb += 32) {
        const uint32_t f = fb + (uint32_t)lane;
        int owner = 0;
#pragma unroll
        for (int stp = 16; stp > 0; stp >>= 1) {
            const uint32_t e = __shfl_sync(kAll, excl, owner + stp);
            if (e <= f) owner += stp;
        }
        const uint32_t blk = __shfl_sync(kAll, b0, owner) + (f - __shfl_sync(kAll, excl, owner));
        const uint32_t o_s = __shfl_sync(kAll, s, owner);
        const uint32_t o_end = __shfl_sync(kAll, s_end, owner);
        const uint32_t o_T = __shfl_sync(kAll, T, owner);
        const float o_b = __shfl_sync(kAll, b, owner);
        const float o_ch = __shfl_sync(kAll, c_h, owner);
        const uint32_t o_lo = __shfl_sync(kAll, (uint32_t)id, owner);
        const uint32_t o_hi = __shfl_sync(kAll, (uint32_t)(id >> 32), owner);
        const bool o_photon = __shfl_sync(kAll, photon ? 1 : 0, owner) != 0;
        if (f < total) {
            const uint4 r = philox4x32_10(make_uint4(o_lo, o_hi, step, blk), K);
            const uint32_t sA = 2u * blk;
            const bool cA = sA >= o_s && sA < o_end && (r.y >> 9) < o_T;
            const bool cB = sA + 1u >= o_s && sA + 1u < o_end && (r.w >> 9) < o_T;
            cand += (unsigned)cA + (unsigned)cB;
            bool aA = false, aB = false;
            float dtmp;
            if (cA || cB) {
                // one acceptance evaluation per lane: the earlier candidate of
                // the pair; the later one only if the earlier is rejected
                const bool first = cA;
                const float y = u01(first ? r.y : r.w);
                const bool acc =
                    y < acceptance(sm.syn, o_photon, o_b, o_ch, u01(first ? r.x : r.z), &dtmp);
                aA = first && acc;
                aB = !first && acc;
            }
            if (cA && cB && !aA)
                aB = u01(r.w) < acceptance(sm.syn, o_photon, o_b, o_ch, u01(r.z), &dtmp);
            if (aA) atomicMin(&facc[owner], sA);
            else if (aB) atomicMin(&facc[owner], sA + 1u);
        }
    }
    __syncwarp();
}

// x of sub-step s (the first word of its draw pair).
__device__ __forceinline__ float draw_x(uint64_t id, uint32_t step, uint32_t s,
                                        const PhiloxKeys& K) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)id, (uint32_t)(id >> 32), step, s >> 1), K);
    return u01((s & 1u) ? r.z : r.x);
}

// Thread pass: one lane per row for planning and events, the warp's lanes
// together for the draws (warp_draw_round).  First generation of a step:
// rows [0, pass_end) with the full step; later generations: rows
// [pass_begin, pass_end) (children) with their stored remaining time.  Each
// lane plans its row; particles whose plan reaches hot_min sub-steps (or,
// with the sampler, e+- in a usable chi bin) go to the hot queue.  A round
// draws every remaining planned sub-step of the warp's rows, so that a warp
// whose particles plan 1 to 30 sub-steps keeps its lanes busy; each particle
// takes its earliest accepted sub-step, the decision of testing its
// sub-steps in order and stopping at the first acceptance.  Lanes with an
// event apply it, re-plan the remaining time and join the next round.
template <bool kCells = false>
__global__ void __launch_bounds__(kColdThreads, QED_COLD_MIN_BLOCKS) k_cold(DevParticles P, StepParams SP, Scratch S,
                                                       DevCtl* ctl) {
    const uint32_t step = step_index(SP);
    __shared__ SharedTables sm;
    __shared__ uint32_t first_acc[kColdThreads];
    stage_tables(sm);
    __syncthreads();
    if (ctl->status == (int)QED_ERR_TIMEOUT || ctl->skip) return;
    const int first_pass = ctl->first_pass;
    const long long begin = first_pass ? 0 : ctl->pass_begin;
    const long long end = ctl->pass_end;
    const long long n_init = kCells ? ctl->n_init : 0;
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    uint32_t* facc = first_acc + (threadIdx.x & ~31);
    constexpr unsigned int kAll = 0xffffffffu;
    Stats stats;
    for (long long base = begin + warp * 32; base < end; base += nwarps * 32) {
        const long long i = base + lane;
        bool active = false, photon = false, changed = false, removed = false;
        uint64_t id = 0;
        PState st{0.0f, 0.0f, 0.0f};
        float Ex = 0.0f, Ey = 0.0f, Ez = 0.0f, Bx = 0.0f, By = 0.0f, Bz = 0.0f;
        ftime t_rem{0.0f, 0.0f};
        if (i < end) {
            const uint8_t type = P.type[i];
            photon = type == QED_PHOTON;
            if (type <= QED_PHOTON && process_enabled(SP, photon)) {
                t_rem = first_pass ? SP.t_step : S.t_rem[i];
                if (time_positive(t_rem)) {
                    active = true;
                    id = P.id[i];
                    st = PState{P.px[i], P.py[i], P.pz[i]};
                    Ex = P.Ex[i]; Ey = P.Ey[i]; Ez = P.Ez[i];
                    Bx = P.Bx[i]; By = P.By[i]; Bz = P.Bz[i];
                }
            }
        }
        Plan pl;
        pl.N = 0;
        pl.T = 0;
        pl.b = pl.c_h = 0.0f;
        float chi = 0.0f, eps = 0.0f;
        uint32_t s = 0;
        bool need_plan = active;
        while (__any_sync(kAll, active)) {
            if (need_plan) {
                need_plan = false;
                pl = plan_particle(SP, sm.sqz_e, sm.sqz_p, photon, st.px, st.py, st.pz, Ex, Ey, Ez,
                                   Bx, By, Bz, t_rem, &chi, &eps);
                if (kCells)
                    apply_cell_count(SP, pl, sm.sqz_e, sm.sqz_p, photon, i, n_init, s, t_rem, eps);
                if (!(eps > 0.0f)) {
                    active = false;
                } else {
                    stats.max_N = max(stats.max_N, pl.N);
                    if (pl.N >= SP.hot_min || (!photon && sampler_bin_ok(SP, chi))) {
                        if (changed) {
                            P.px[i] = st.px;
                            P.py[i] = st.py;
                            P.pz[i] = st.pz;
                            changed = false;
                        }
                        // the hot pass plans again; long plans and the
                        // sampler's particles are stepped by a whole warp,
                        // the others by a lane (the event-driven sampler's
                        // particles one lane each, in their own queue)
                        const bool net = photon ? pair_sampler_ok(SP, chi, pl.T)
                                                : sampler_bin_ok(SP, chi);
                        if (net && S.samp) {
                            HotItem it;
                            it.idx = (uint32_t)i;
                            it.s = s;
                            it.t_rem = t_rem;
                            S.samp[atomicAdd(&ctl->samp_tail, 1u)] = it;
                        } else {
                            push_hot(S, ctl, i, s, t_rem, pl.N >= SP.long_min || net);
                        }
                        active = false;
                    } else {
                        stats.plans++;
                        stats.guard += pl.guard ? 1 : 0;
                        if (pl.T == 0u) {
                            // a zero squeeze threshold admits no candidate:
                            // the sub-steps pass without an event
                            stats.substeps += pl.N;
                            s += pl.N;
                            active = false;
                        }
                    }
                }
            }
            const uint32_t s_end = active ? s + pl.N : 0u;
            warp_draw_round(sm, facc, active, s, s_end, pl.T, pl.b, pl.c_h, id, photon, step, SP.draw_keys, stats.cand);
            if (active) {
                const uint32_t s_ev = facc[lane];
                if (s_ev == kNoEvent) {
                    stats.substeps += pl.N;
                    s = s_end;
                    active = false;   // the plan ran out without an event
                } else {
                    const uint32_t k = s_ev - s;
                    stats.substeps += k + 1u;
                    const float x = draw_x(id, step, s_ev, SP.draw_keys);
                    const ftime t_after = (k + 1u == pl.N) ? ftime{0.0f, 0.0f}
                                                           : time_sub_mul(t_rem, k + 1u, pl.h);
                    removed = apply_event(P, S, SP, ctl, i, id, photon, x, eps, chi, step, s_ev,
                                          t_after, st, stats, true, false,
                                          Fields{Ex, Ey, Ez, Bx, By, Bz}, false);
                    changed = true;
                    s = s_ev + 1u;
                    t_rem = t_after;
                    if (removed || !time_positive(t_rem)) active = false;
                    else need_plan = true;
                }
            }
            __syncwarp();   // facc is reset by the next round
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

// ---------------------------------------------------------------------------
// Push mode: Algorithm 1 with the Boris push before every e+- draw
// ---------------------------------------------------------------------------
constexpr int kPushGroupMax = 16;   // busy lanes of a drained warp that switch to group mode
constexpr int kPushPlanBatch = 8;   // lanes wanting a plan before the warp plans
constexpr int kPushClaimBatch = 8;  // free lanes before the warp claims rows
// A push-mode step.  The push makes every sub-step depend on the one before,
// so a lane steps one particle through its sub-steps in order; a lane whose
// particle is done takes the next row (the idle lanes of a warp share one
// atomic on ctl->push_head, which starts at 0).  Per sub-step of an e+-: the
// push over h, chi and eps of the new momentum, the squeeze bound for that
// chi, the draw of sub-step s and the test.  A photon flies straight: its
// momentum, chi and plan stay, as in the other kernels.  After an event the
// particle is re-planned over the time that remains, from its state after
// the push and the recoil.
//
// kStream = false: one cascade generation, the rows [pass_begin, pass_end).
// kStream = true: the whole step in one launch.  Rows are taken in store
// order as they come: the step's initial rows, then every child as soon as
// it is reserved, so that a generation does not wait for the longest push
// chain of the one before.  The rows past the initial ones start "not
// written" (k_push_begin); a child's writer stores the row, fences, then its
// type byte, and a lane that took the row waits for that byte.  Each warp
// takes child indices into a pending range with one atomic and hands a lane
// only an index whose row is reserved already (indices never reserved are
// void at the end).  The step ends when the rows completed equal the rows
// stored.  Every wait is bounded: a warp that sees no progress anywhere
// (rows stored, rows completed, the beats of long chains) for SP.wait_ns
// records QED_ERR_TIMEOUT and returns.
//
// Divergence control (both forms): a lane that wants a plan (a new row, or
// after an event) waits until kPushPlanBatch lanes of its warp want one, or
// until no busy lane is left to step; an accepted event is applied with the
// lane's next plan; in the persistent form free lanes claim rows only once
// kPushClaimBatch of them are free (or none is busy).  When the warp finds
// no row to take and at most kPushGroupMax lanes are busy, it switches to
// group mode (below).
constexpr unsigned int kBeatRounds = 1024;   // rounds of a warp between two beats
template <bool kStream>
__global__ void __launch_bounds__(kLaneThreads) k_push(DevParticles P, StepParams SP, Scratch S,
                                                       DevCtl* ctl) {
    const uint32_t step = step_index(SP);
    __shared__ SharedTables sm;
    stage_tables(sm);
    __syncthreads();
    if (ctl->status == (int)QED_ERR_TIMEOUT) return;
    const bool first_pass = kStream || ctl->first_pass != 0;
    const long long begin = kStream ? 0 : (first_pass ? 0 : ctl->pass_begin);
    const long long n = kStream ? 0 : ctl->pass_end - begin;
    const long long n_init = ctl->n_init;
    const bool cascade = SP.cascade != 0;
    constexpr unsigned int kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const PlanConst PC = plan_const(SP);
    Stats stats;
    bool busy = false, drained = kStream ? false : n <= 0, photon = false, electron = false;
    bool need_plan = false, removed = false;
    bool waiting = false;                          // kStream: the lane's row is still being written
    bool ev = false;                               // an accepted event not yet applied
    float ev_x = 0.0f, ev_eps = 0.0f, ev_chi = 0.0f;
    unsigned int units = 0;                        // kStream: rows this lane completed, not yet added
    unsigned long long pend_lo = 0, pend_hi = 0;   // kStream: the warp's pending child indices
    unsigned long long idle_ns = 0, seen = 0;      // kStream: bounded wait
    unsigned int idle = 0, rounds = 0;
    bool timed_out = false;
    long long i = 0;
    uint64_t id = 0;
    PState st{0.0f, 0.0f, 0.0f};
    Fields F{0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    ftime t_rem{0.0f, 0.0f};
    Plan pl;
    pl.N = 0;
    pl.T = 0;
    pl.b = pl.c_h = 0.0f;
    pl.h = ftime{0.0f, 0.0f};
    float chi = 0.0f, eps = 0.0f, a = 0.0f;
    uint32_t k = 0, s = 0, blk = kNoEvent;
    uint4 r = make_uint4(0u, 0u, 0u, 0u);
    // a row the lane holds: start its particle, or count the row as done
    auto take_row = [&](long long row) {
        const uint8_t type = P.type[row];
        photon = type == QED_PHOTON;
        if (type <= QED_PHOTON && process_enabled(SP, photon)) {
            t_rem = (kStream ? row < n_init : first_pass) ? SP.t_step : S.t_rem[row];
            if (time_positive(t_rem)) {
                busy = true;
                need_plan = true;
                removed = false;
                electron = type == QED_ELECTRON;
                id = P.id[row];
                st = PState{P.px[row], P.py[row], P.pz[row]};
                F = Fields{P.Ex[row], P.Ey[row], P.Ez[row], P.Bx[row], P.By[row], P.Bz[row]};
                s = 0;
                blk = kNoEvent;
                return;
            }
        }
        if (kStream) ++units;
    };
    while (true) {
        const unsigned int free_lanes = __ballot_sync(kAll, !busy && !waiting);
        if (kStream) {
            // rows for the free lanes: indices below the rows stored now.  A
            // claim is a round trip to the control block: the free lanes wait
            // until kPushClaimBatch of them want a row (or no lane is busy),
            // and the stored count is read only for indices past the
            // initial rows.
            int got = 0;
            unsigned long long base = 0;
            const bool claim = free_lanes != 0 &&
                               (__popc(free_lanes) >= kPushClaimBatch ||
                                __ballot_sync(kAll, busy) == 0u);
            if (claim) {
                const int want = __popc(free_lanes);
                if (lane == 0) {
                    const unsigned long long n0 = (unsigned long long)n_init;
                    if (pend_lo == pend_hi) {
                        const unsigned long long h =
                            *reinterpret_cast<volatile unsigned long long*>(&ctl->push_head);
                        const unsigned long long lim =
                            (cascade && h + (unsigned long long)want > n0) ? max(stored_rows(P), n0)
                                                                           : n0;
                        if (h < lim) {
                            const unsigned long long kk = min((unsigned long long)want, lim - h);
                            pend_lo = atomicAdd(&ctl->push_head, kk);
                            pend_hi = pend_lo + kk;
                        }
                    }
                    if (pend_lo < pend_hi) {
                        const unsigned long long lim =
                            (cascade && pend_hi > n0) ? max(stored_rows(P), n0) : n0;
                        if (pend_lo < lim) {
                            got = (int)min((unsigned long long)want, min(pend_hi, lim) - pend_lo);
                            base = pend_lo;
                            pend_lo += (unsigned long long)got;
                        }
                    }
                }
                got = __shfl_sync(kAll, got, 0);
                base = __shfl_sync(kAll, base, 0);
                const int rank = __popc(free_lanes & ((1u << lane) - 1u));
                if (!busy && !waiting && rank < got) {
                    i = (long long)(base + (unsigned long long)rank);
                    waiting = true;
                }
            }
            // the warp is starved when a claim left free lanes without a row
            drained = claim && got < __popc(free_lanes);
            if (waiting) {
                const uint8_t ty = *reinterpret_cast<volatile uint8_t*>(P.type + i);
                if (ty != kNotReady) {
                    __threadfence();   // the row was stored before its type byte
                    waiting = false;
                    take_row(i);
                }
            }
        } else if (free_lanes && !drained) {
            const int leader = __ffs(free_lanes) - 1;
            unsigned long long base = 0;
            if (lane == leader)
                base = atomicAdd(&ctl->push_head, (unsigned long long)__popc(free_lanes));
            base = __shfl_sync(kAll, base, leader);
            if ((long long)base + __popc(free_lanes) >= n) drained = true;
            if (!busy) {
                const long long row = (long long)base + __popc(free_lanes & ((1u << lane) - 1u));
                if (row < n) {
                    i = begin + row;
                    take_row(i);
                }
            }
        }
        const unsigned int bm = __ballot_sync(kAll, busy);
        if (!bm) {
            if (!kStream) {
                if (drained) break;
                continue;
            }
            // nothing to step: wait for rows, or finish
            const bool hold = __any_sync(kAll, waiting);
            bool finish = false;
            unsigned long long progress = 0;
            if (!hold) {
                const unsigned long long sum = warp_sum(units);
                units = 0;
                if (lane == 0) {
                    __threadfence();   // this warp's reservations before its completions
                    if (sum) atomicAdd(&ctl->finished, sum);
                    const unsigned long long c1 = cascade ? stored_rows(P) : (unsigned long long)n_init;
                    const unsigned long long f =
                        *reinterpret_cast<volatile unsigned long long*>(&ctl->finished);
                    const unsigned long long c2 = cascade ? stored_rows(P) : (unsigned long long)n_init;
                    finish = f == c1 && c1 == c2;
                    progress = f + c2 + *reinterpret_cast<volatile unsigned long long*>(&ctl->beat);
                }
                finish = __shfl_sync(kAll, finish ? 1 : 0, 0) != 0;
                progress = __shfl_sync(kAll, progress, 0);
            }
            if (finish) break;
            // idle: back off from 256 ns to 4 us (64 ns while a row is being
            // written); the idle time counts from the last progress seen
            if (!hold && progress != seen) {
                seen = progress;
                idle_ns = 0;
            }
            const unsigned int nap = hold ? 64u : 256u << min(idle, 4u);
            ++idle;
            idle_ns += nap;
            if (idle_ns > SP.wait_ns) {
                timed_out = true;
                break;
            }
            __nanosleep(nap);
            continue;
        }
        if (kStream) {
            idle = 0;
            idle_ns = 0;
            if (++rounds == kBeatRounds) {   // a long chain shows its progress
                rounds = 0;
                if (lane == 0) atomicAdd(&ctl->beat, 1ull);
            }
        }
        // plan the lane's particle (Algorithms 1/2, planning); true if it is
        // done.  An accepted event of the lane's last sub-step is applied
        // first (recoil or decay, children), so that the lanes of a warp
        // apply their events together with their plans.
        auto plan_now = [&]() -> bool {
            need_plan = false;
            if (ev) {
                ev = false;
                removed = apply_event(P, S, SP, ctl, i, id, photon, ev_x, ev_eps, ev_chi, step, s,
                                      t_rem, st, stats, true, false, F, kStream);
                ++s;
                if (removed || !time_positive(t_rem)) return true;
            }
            pl = plan_particle(SP, sm.sqz_e, sm.sqz_p, photon, st.px, st.py, st.pz, F.Ex, F.Ey,
                               F.Ez, F.Bx, F.By, F.Bz, t_rem, &chi, &eps);
            if (!(eps > 0.0f)) return true;
            // per-cell counts: an initial row's first plan takes its cell's
            // count when that is larger (the cell's sub-step)
            apply_cell_count(SP, pl, sm.sqz_e, sm.sqz_p, photon, i, n_init, s, t_rem, eps);
            stats.plans++;
            stats.guard += pl.guard ? 1 : 0;
            stats.max_N = max(stats.max_N, pl.N);
            k = 0;
            const float ah = __fmul_rn(kPi, pl.h.hi);
            a = electron ? -ah : ah;
            if (photon && pl.T == 0u) {
                // a zero squeeze threshold admits no candidate
                stats.substeps += pl.N;
                s += pl.N;
                return true;
            }
            return false;
        };
        const int m = __popc(bm);
        bool done = false;
        if (drained && m <= kPushGroupMax) {
            // Group mode: no rows are left and m <= kPushGroupMax lanes are
            // busy.  The g-th busy lane's particle gets the G = 32 / m lanes
            // [g G, (g+1) G):
            // every lane of the group runs the same push chain from the
            // owner's state and keeps the state after push j + 1 (j its place
            // in the group), then tests sub-step s + j; the first accepted
            // sub-step of the group decides, as in the sequential loop.  Only
            // the pushes stay serial.
            const int G = 32 / m;
            const int g = lane / G, j = lane - g * G;
            int owner = lane;
            if (g < m) {
                unsigned int mm = bm;
                for (int t = 0; t < g; ++t) mm &= mm - 1u;
                owner = __ffs(mm) - 1;
            }
            const bool ready = busy && !need_plan;
            if (busy && need_plan) done = plan_now();   // its group waits this round
            const bool g_ready = (__shfl_sync(kAll, ready ? 1 : 0, owner) != 0) && g < m;
            const float ox = __shfl_sync(kAll, st.px, owner), oy = __shfl_sync(kAll, st.py, owner),
                        oz = __shfl_sync(kAll, st.pz, owner);
            const float oa = __shfl_sync(kAll, a, owner);
            const float oEx = __shfl_sync(kAll, F.Ex, owner), oEy = __shfl_sync(kAll, F.Ey, owner),
                        oEz = __shfl_sync(kAll, F.Ez, owner), oBx = __shfl_sync(kAll, F.Bx, owner),
                        oBy = __shfl_sync(kAll, F.By, owner), oBz = __shfl_sync(kAll, F.Bz, owner);
            const float ohh = __shfl_sync(kAll, pl.h.hi, owner), ob = __shfl_sync(kAll, pl.b, owner),
                        och = __shfl_sync(kAll, pl.c_h, owner), ochi = __shfl_sync(kAll, chi, owner),
                        oeps = __shfl_sync(kAll, eps, owner);
            const uint32_t oT = __shfl_sync(kAll, pl.T, owner), oN = __shfl_sync(kAll, pl.N, owner),
                           ok = __shfl_sync(kAll, k, owner), os = __shfl_sync(kAll, s, owner);
            const uint32_t oid0 = __shfl_sync(kAll, (uint32_t)id, owner),
                           oid1 = __shfl_sync(kAll, (uint32_t)(id >> 32), owner);
            const bool oph = __shfl_sync(kAll, photon ? 1 : 0, owner) != 0;
            const uint32_t valid = g_ready ? min((uint32_t)G, oN - ok) : 0u;
            PState q{ox, oy, oz}, mine = q;
            const bool do_push = g_ready && !oph;
            for (int t = 0; t < G; ++t) {
                if (do_push && (uint32_t)t < valid)
                    boris_push(q.px, q.py, q.pz, oa, oEx, oEy, oEz, oBx, oBy, oBz);
                if (t == j) mine = q;
            }
            bool acc = false, cnd = false;
            float cj = ochi, ej = oeps, xj = 0.0f;
            if ((uint32_t)j < valid) {
                float b = ob, c_h = och;
                uint32_t T = oT;
                if (!oph) {
                    cj = chi_any(false, mine.px, mine.py, mine.pz, oEx, oEy, oEz, oBx, oBy, oBz,
                                 PC.inv_Es, &ej);
                    b = 1.5f * cj;
                    c_h = PC.K * ohh * __fdividef(1.0f, ej);
                    const float b23 = b > 0.0f ? exp2f(__log2f(b) * (2.0f / 3.0f)) : 0.0f;
                    T = squeeze_threshold(squeeze_bound(sm.sqz_e, sm.sqz_p, false, b, c_h, b23));
                }
                const uint32_t sj = os + (uint32_t)j;
                const uint4 r = philox4x32_10(make_uint4(oid0, oid1, step, sj >> 1), SP.draw_keys);
                const uint32_t yw = (sj & 1u) ? r.w : r.y;
                xj = u01((sj & 1u) ? r.z : r.x);
                if ((yw >> 9) < T) {
                    cnd = true;
                    float dtmp;
                    acc = u01(yw) < acceptance(sm.syn, oph, b, c_h, xj, &dtmp);
                }
            }
            const unsigned int am = __ballot_sync(kAll, acc);
            const unsigned int gmask = G == 32 ? kAll : (((1u << G) - 1u) << (g * G));
            const unsigned int ga = am & gmask;
            const int jstar = ga ? __ffs(ga) - 1 - g * G : -1;
            const uint32_t used = jstar >= 0 ? (uint32_t)jstar + 1u : valid;
            if (cnd && (uint32_t)j < used) stats.cand++;
            // each busy lane takes the outcome of the group it owns
            const int my_g = __popc(bm & ((1u << lane) - 1u));
            const int gl = (busy ? my_g : 0) * G;
            const uint32_t used_o = __shfl_sync(kAll, used, gl);
            const int jstar_o = __shfl_sync(kAll, jstar, gl);
            const int src = gl + (used_o > 0u ? (int)used_o - 1 : 0);
            const float nx = __shfl_sync(kAll, mine.px, src), ny = __shfl_sync(kAll, mine.py, src),
                        nz = __shfl_sync(kAll, mine.pz, src);
            const float nchi = __shfl_sync(kAll, cj, src), neps = __shfl_sync(kAll, ej, src),
                        nxd = __shfl_sync(kAll, xj, src);
            if (ready) {
                stats.substeps += used_o;
                st = PState{nx, ny, nz};
                if (jstar_o >= 0) {
                    const uint32_t kk = k + used_o;
                    const ftime t_after = (kk == pl.N) ? ftime{0.0f, 0.0f}
                                                       : time_sub_mul(t_rem, kk, pl.h);
                    removed = apply_event(P, S, SP, ctl, i, id, photon, nxd, neps, nchi, step,
                                          s + (uint32_t)jstar_o, t_after, st, stats, true, false, F,
                                          kStream);
                    s += used_o;
                    t_rem = t_after;
                    if (removed || !time_positive(t_rem)) done = true;
                    else need_plan = true;
                } else {
                    s += used_o;
                    k += used_o;
                    if (k == pl.N) done = true;
                }
            }
        } else {
            // A plan taken by one or two lanes at a time would make the warp
            // run the planner in most rounds while the others wait: a lane
            // that wants a plan waits until kPushPlanBatch lanes want one, or
            // until no busy lane is left to step, and then steps its first
            // sub-step in the same round.
            const unsigned int pm = __ballot_sync(kAll, busy && need_plan);
            if ((__popc(pm) >= kPushPlanBatch || pm == bm) && busy && need_plan) done = plan_now();
        }
        if (!(drained && m <= kPushGroupMax) && busy && !need_plan && !done) {
            float b = pl.b, c_h = pl.c_h, chi_k = chi, eps_k = eps;
            uint32_t T = pl.T;
            if (!photon) {
                boris_push(st.px, st.py, st.pz, a, F.Ex, F.Ey, F.Ez, F.Bx, F.By, F.Bz);
                chi_k = chi_any(false, st.px, st.py, st.pz, F.Ex, F.Ey, F.Ez, F.Bx, F.By, F.Bz,
                                PC.inv_Es, &eps_k);
                b = 1.5f * chi_k;
                c_h = PC.K * pl.h.hi * __fdividef(1.0f, eps_k);
                const float b23 = b > 0.0f ? exp2f(__log2f(b) * (2.0f / 3.0f)) : 0.0f;
                T = squeeze_threshold(squeeze_bound(sm.sqz_e, sm.sqz_p, false, b, c_h, b23));
            }
            if ((s >> 1) != blk) {
                blk = s >> 1;
                r = philox4x32_10(make_uint4((uint32_t)id, (uint32_t)(id >> 32), step, blk), SP.draw_keys);
            }
            const uint32_t yw = (s & 1u) ? r.w : r.y;
            const float x = u01((s & 1u) ? r.z : r.x);
            stats.substeps++;
            bool acc = false;
            if ((yw >> 9) < T) {
                stats.cand++;
                float dtmp;
                acc = u01(yw) < acceptance(sm.syn, photon, b, c_h, x, &dtmp);
            }
            if (acc) {
                // the event is applied with the next plan (plan_now), s and
                // the pushed state stay until then
                t_rem = (k + 1u == pl.N) ? ftime{0.0f, 0.0f} : time_sub_mul(t_rem, k + 1u, pl.h);
                ev = true;
                ev_x = x;
                ev_eps = eps_k;
                ev_chi = chi_k;
                need_plan = true;
            } else {
                ++s;
                if (++k == pl.N) done = true;
            }
        }
        if (done) {
            busy = false;
            if (removed) {
                P.type[i] = QED_REMOVED;
            } else if (!photon) {
                P.px[i] = st.px;
                P.py[i] = st.py;
                P.pz[i] = st.pz;
            }
            if (kStream) ++units;
        }
    }
    if (kStream) {
        if (timed_out && lane == 0) atomicExch(&ctl->status, (int)QED_ERR_TIMEOUT);
        const unsigned long long sum = warp_sum(units);
        if (lane == 0 && sum) {
            __threadfence();
            atomicAdd(&ctl->finished, sum);
        }
    }
    flush_stats(stats, ctl);
}

// One queued particle stepped by the whole warp (all 32 lanes, identical
// arguments): 64 sub-steps per iteration (lane l draws the Philox block of
// sub-steps 2l and 2l+1), the first accepted sub-step found with two ballots.
// Statistics are counted on lane 0, candidates per lane.
// kSampler: an e+- in a usable bin of the sampler's chi range decides events
// from the tabulated total probability c_h W(b) and takes the energy fraction
// from the network at the event's uniform, evaluated by the warp (FP32).
template <int kSampler, bool kCells = false>
__device__ __forceinline__ void warp_item(const DevParticles& P, const Scratch& S,
                                          const StepParams& SP, DevCtl* ctl,
                                          const SharedTables& sm, unsigned char* net_smem,
                                          const HotItem& it, uint32_t step, uint32_t k0,
                                          uint32_t k1, Stats& stats, unsigned int& cand,
                                          bool publish) {
    const int lane = threadIdx.x & 31;
    SamplerSmem& net = *reinterpret_cast<SamplerSmem*>(net_smem);      // mode 1
    SamplerMma& mma = *reinterpret_cast<SamplerMma*>(net_smem);        // mode 2
    const long long i = it.idx;
    const bool photon = P.type[i] == QED_PHOTON;
    const uint64_t id = P.id[i];
    PState st{P.px[i], P.py[i], P.pz[i]};
    const float Ex = P.Ex[i], Ey = P.Ey[i], Ez = P.Ez[i];
    const float Bx = P.Bx[i], By = P.By[i], Bz = P.Bz[i];
    uint32_t s = it.s;
    ftime t_rem = it.t_rem;
    bool removed = false, changed = false;
    unsigned int rounds = 0;   // publish (persistent pass): beats of a long chain
    const long long n_init = kCells ? ctl->n_init : 0;
    while (time_positive(t_rem)) {
        float eps, chi;
        Plan pl = plan_particle(SP, sm.sqz_e, sm.sqz_p, photon, st.px, st.py, st.pz, Ex, Ey, Ez,
                                Bx, By, Bz, t_rem, &chi, &eps);
        if (kCells) apply_cell_count(SP, pl, sm.sqz_e, sm.sqz_p, photon, i, n_init, s, t_rem, eps);
        if (!(eps > 0.0f)) break;
        if (lane == 0) {
            stats.plans++;
            stats.guard += pl.guard ? 1 : 0;
            stats.max_N = max(stats.max_N, pl.N);
        }
        // event-driven mode: photons in a usable bin of the pair sampler too
        const bool use_pnet =
            kSampler == 2 && photon && pl.N >= SP.hot_min && pair_sampler_ok(SP, chi, pl.T);
        const bool use_net = (kSampler != 0 && !photon && sampler_bin_ok(SP, chi)) || use_pnet;
        const SamplerMma& tab = use_pnet ? pair_mma(net_smem) : mma;
        const float thr =
            use_net ? fminf(pl.c_h * (kSampler == 2 ? wtot_at(tab.wtot, tab.nrows, chi)
                                                    : sampler_wtot(net, chi)),
                            1.0f)
                    : 0.0f;
        uint32_t kdone = 0;
        bool event = false;
        if (!use_net && pl.T == 0u) {   // no candidates: count without drawing
            if (lane == 0) stats.substeps += pl.N;
            s += pl.N;
            kdone = pl.N;
        }
        if (kSampler == 2 && use_net) {
            // Event-driven: with chi and the plan fixed until the next event,
            // each sub-step is an event with probability thr on its own, so
            // the sub-steps before the next event are geometric, drawn by
            // inversion: floor(ln u / ln(1 - thr)).  One Philox block per
            // segment (counter: the segment's first sub-step, own key); its
            // second word gives the network's uniform.
            const uint32_t left = pl.N - kdone;
            const uint4 r = philox4x32_10(make_uint4((uint32_t)id, (uint32_t)(id >> 32), step, s),
                                          k0 ^ kWaitKeyLo, k1 ^ kWaitKeyHi);
            const float wait = floorf(logf(u01(r.y)) / log1pf(-thr));
            if (!(wait < (float)left)) {   // no event in the rest of the plan
                if (lane == 0) stats.substeps += left;
                s += left;
                kdone = pl.N;
            } else {
                const uint32_t k = (uint32_t)wait;
                const uint32_t s_ev = s + k;
                const uint32_t k_ev = kdone + k;
                // the tensor-core form, as in k_samp (one sample: one tile)
                const float x = mlp_infer_mma_one(tab, warp_mma_buf(net_smem),
                                                  log10f(chi) * 0.5f, mlp_input_u(u01(r.x)));
                if (lane == 0) {
                    stats.substeps += k + 1;
                    if (photon) stats.sampled_p++;
                    else stats.sampled++;
                }
                const ftime t_after = (k_ev + 1 == pl.N) ? ftime{0.0f, 0.0f}
                                                         : time_sub_mul(t_rem, k_ev + 1, pl.h);
                removed = apply_event(P, S, SP, ctl, i, id, photon, x, eps, chi, step, s_ev,
                                      t_after, st, stats, lane == 0, true,
                                      Fields{Ex, Ey, Ez, Bx, By, Bz}, publish);
                changed = true;
                s = s_ev + 1;
                t_rem = t_after;
                event = true;
                kdone = pl.N;   // skips the sub-step loop below
            }
        }
        while (kdone < pl.N) {
            const uint32_t sb = s;
            const uint32_t sa = sb & ~1u;
            const uint32_t lim = sb + (pl.N - kdone);
            const uint32_t s0 = sa + 2u * (uint32_t)lane;
            const uint4 r = philox4x32_10(
                make_uint4((uint32_t)id, (uint32_t)(id >> 32), step, (sa >> 1) + lane), SP.draw_keys);
            const bool v0 = s0 >= sb && s0 < lim;
            const bool v1 = s0 + 1 >= sb && s0 + 1 < lim;
            bool c0, c1, a0 = false, a1 = false;
            if (kSampler == 1 && use_net) {
                c0 = c1 = false;
                a0 = v0 && u01(r.y) < thr;
                a1 = v1 && u01(r.w) < thr;
            } else {
                c0 = v0 && (r.y >> 9) < pl.T;
                c1 = v1 && (r.w >> 9) < pl.T;
                // one acceptance evaluation per lane: the earlier candidate
                // of the pair; the later one only if the earlier is rejected
                float dtmp;
                if (c0 || c1) {
                    const bool first = c0;
                    const float y = u01(first ? r.y : r.w);
                    const bool acc =
                        y < acceptance(sm.syn, photon, pl.b, pl.c_h, u01(first ? r.x : r.z), &dtmp);
                    a0 = first && acc;
                    a1 = !first && acc;
                }
                if (c0 && c1 && !a0)
                    a1 = u01(r.w) < acceptance(sm.syn, photon, pl.b, pl.c_h, u01(r.z), &dtmp);
            }
            const unsigned int m0 = __ballot_sync(0xffffffffu, a0);
            const unsigned int m1 = __ballot_sync(0xffffffffu, a1);
            cand += (unsigned)c0 + (unsigned)c1;
            if ((m0 | m1) == 0u) {
                const uint32_t chunk_end = min(sa + 64u, lim);
                if (lane == 0) stats.substeps += chunk_end - sb;
                kdone += chunk_end - sb;
                s = chunk_end;
                if (publish && ++rounds == kBeatRounds) {
                    rounds = 0;
                    if (lane == 0) atomicAdd(&ctl->beat, 1ull);
                }
                continue;
            }
            const int p0 = m0 ? 2 * (__ffs(m0) - 1) : 1 << 30;
            const int p1 = m1 ? 2 * (__ffs(m1) - 1) + 1 : 1 << 30;
            const int pos = min(p0, p1);
            const uint32_t s_ev = sa + (uint32_t)pos;
            const float xo = (pos & 1) ? u01(r.z) : u01(r.x);
            float x = __shfl_sync(0xffffffffu, xo, pos >> 1);
            if (kSampler == 1 && use_net) {
                // inverse sampling: the event's uniform through the network
                x = mlp_infer_warp(net, log10f(chi) * 0.5f, mlp_input_u(x));
                if (lane == 0) stats.sampled++;
            }
            const uint32_t k_ev = kdone + (s_ev - sb);
            if (lane == 0) stats.substeps += s_ev - sb + 1;
            const ftime t_after = (k_ev + 1 == pl.N) ? ftime{0.0f, 0.0f}
                                                     : time_sub_mul(t_rem, k_ev + 1, pl.h);
            removed = apply_event(P, S, SP, ctl, i, id, photon, x, eps, chi, step, s_ev, t_after,
                                  st, stats, lane == 0, true, Fields{Ex, Ey, Ez, Bx, By, Bz},
                                  publish);
            changed = true;
            s = s_ev + 1;
            t_rem = t_after;
            event = true;
            break;
        }
        if (removed) break;
        if (!event) t_rem = ftime{0.0f, 0.0f};
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


// Event-driven sampler, one lane per particle (sampler mode 2; reading of
// Sec. 2.2's inverse sampling, with the sub-steps to the next event drawn at
// once).  A lane holds one of the sampler's particles (e+- in a usable chi
// bin, queued by the thread pass).  Per round, every busy lane draws the
// sub-steps to its next event, geometric with the per-sub-step probability
// c_h W(b) of its plan: floor(ln u / ln(1 - p)) from one Philox block at
// counter (id, step, first sub-step of the plan) under the waiting-time key.
// If the event falls beyond the plan, the particle's time runs out without an
// event; otherwise the lanes with an event evaluate the network together on
// the tensor cores (mlp_infer_mma, the block's other word as the uniform), and
// apply their events (recoil, photon child, one reservation atomic per warp)
// and re-plan from the remaining time.  A particle whose new chi leaves the
// sampler's usable bins continues with rejection: its state goes back to the
// store and it joins the hot pass's queue (the hot pass runs after this
// kernel).  Idle lanes take queue entries, one atomic per warp.  Persistent.
__global__ void __launch_bounds__(kLaneThreads) k_samp(DevParticles P, StepParams SP, Scratch S,
                                                       DevCtl* ctl) {
    const uint32_t step = step_index(SP);
    __shared__ SharedTables sm;
    __shared__ float fld[6][kLaneThreads];   // E, B at the lane's row
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    SamplerMma& net = *reinterpret_cast<SamplerMma*>(dyn_smem);   // emission
    SamplerMma& pnet = pair_mma(dyn_smem);                           // pair production
    stage_tables(sm);
    stage_sampler_mma(net, reinterpret_cast<const __nv_bfloat16*>(SP.net_w), SP.net_wtot,
                      SP.net_rows, SP.net_bins);
    if (SP.pnet_bins)
        stage_sampler_mma(pnet, reinterpret_cast<const __nv_bfloat16*>(SP.pnet_w), SP.pnet_wtot,
                          SP.net_rows, SP.pnet_bins);
    __syncthreads();
    if (ctl->status == (int)QED_ERR_TIMEOUT) return;
    constexpr unsigned int kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t kw0 = (uint32_t)SP.seed ^ kWaitKeyLo, kw1 = (uint32_t)(SP.seed >> 32) ^ kWaitKeyHi;
    const unsigned int tail = ctl->samp_tail;
    Stats stats;
    bool active = false, more = true, photon = false;
    uint32_t i = 0, s = 0;
    uint64_t id = 0;
    PState st{0.0f, 0.0f, 0.0f};
    ftime t_rem{0.0f, 0.0f};
    Plan pl;
    pl.N = 0;
    float chi = 0.0f, eps = 0.0f, thr = 0.0f;
    bool removed = false;
    // after a load or an event: plan the remaining time; false if the lane
    // is done with the particle (no time left, or handed to rejection)
    auto plan_lane = [&]() -> bool {
        pl = plan_particle(SP, sm.sqz_e, sm.sqz_p, photon, st.px, st.py, st.pz,
                           fld[0][threadIdx.x], fld[1][threadIdx.x], fld[2][threadIdx.x],
                           fld[3][threadIdx.x], fld[4][threadIdx.x], fld[5][threadIdx.x], t_rem,
                           &chi, &eps);
        if (!(eps > 0.0f)) return false;
        stats.max_N = max(stats.max_N, pl.N);
        const bool usable = photon ? pl.N >= SP.hot_min && pair_sampler_ok(SP, chi, pl.T)
                                   : sampler_bin_ok(SP, chi);
        if (!usable) {
            // rejection from here on: the hot pass plans again from the store
            if (!photon) {
                P.px[i] = st.px;
                P.py[i] = st.py;
                P.pz[i] = st.pz;
            }
            push_hot(S, ctl, i, s, t_rem, pl.N >= SP.long_min);
            return false;
        }
        stats.plans++;
        stats.guard += pl.guard ? 1 : 0;
        const SamplerMma& tab = photon ? pnet : net;
        thr = fminf(pl.c_h * wtot_at(tab.wtot, tab.nrows, chi), 1.0f);
        return true;
    };
    while (true) {
        if (more) {
            const unsigned int idle = __ballot_sync(kAll, !active);
            if (idle) {
                unsigned int base = 0;
                if (lane == 0) base = atomicAdd(&ctl->samp_head, (unsigned int)__popc(idle));
                base = __shfl_sync(kAll, base, 0);
                if (base + (unsigned int)__popc(idle) >= tail) more = false;
                if (!active) {
                    const unsigned int q = base + (unsigned int)__popc(idle & ((1u << lane) - 1u));
                    if (q < tail) {
                        const HotItem it = S.samp[q];
                        i = it.idx;
                        s = it.s;
                        t_rem = it.t_rem;
                        photon = P.type[i] == QED_PHOTON;
                        id = P.id[i];
                        st = PState{P.px[i], P.py[i], P.pz[i]};
                        fld[0][threadIdx.x] = P.Ex[i];
                        fld[1][threadIdx.x] = P.Ey[i];
                        fld[2][threadIdx.x] = P.Ez[i];
                        fld[3][threadIdx.x] = P.Bx[i];
                        fld[4][threadIdx.x] = P.By[i];
                        fld[5][threadIdx.x] = P.Bz[i];
                        active = plan_lane();
                    }
                }
            }
        }
        if (!__any_sync(kAll, active)) {
            if (!more) break;
            continue;
        }
        // the sub-steps to the next event
        bool ev = false, done = false;
        uint32_t k = 0;
        float u_net = 0.5f;
        if (active) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)id, (uint32_t)(id >> 32), step, s),
                                          kw0, kw1);
            const float wait = floorf(logf(u01(r.y)) / log1pf(-thr));
            if (!(wait < (float)pl.N && thr > 0.0f)) {   // no event in the rest of the plan
                stats.substeps += pl.N;
                s += pl.N;
                done = true;
            } else {
                k = (uint32_t)wait;
                ev = true;
                u_net = u01(r.x);
            }
        }
        if (__any_sync(kAll, ev)) {
            // the child rows (one photon, or an e- and an e+), reserved first
            // (one atomic for the warp's events) so that the atomic's latency
            // overlaps the network
            long long j = -1;
            if (ev) j = reserve_rows(P, ctl, photon ? 2 : 1, true);
            // the emission and the pair network for the lanes with such an
            // event, each packed into one tile when at most 16 have one
            const float v0 = log10f(chi) * 0.5f, v1 = mlp_input_u(u_net);
            float x = 0.0f;
            if (__any_sync(kAll, ev && !photon))
                x = mlp_infer_mma_some(net, warp_mma_buf(dyn_smem), ev && !photon, v0, v1);
            if (__any_sync(kAll, ev && photon)) {
                const float xp = mlp_infer_mma_some(pnet, warp_mma_buf(dyn_smem), ev && photon,
                                                    v0, v1);
                if (photon) x = xp;
            }
            if (ev) {
                const uint32_t s_ev = s + k;
                stats.substeps += k + 1;
                if (photon) stats.sampled_p++;
                else stats.sampled++;
                const ftime t_after = (k + 1 == pl.N) ? ftime{0.0f, 0.0f}
                                                      : time_sub_mul(t_rem, k + 1, pl.h);
                removed = apply_event(P, S, SP, ctl, i, id, photon, x, eps, chi, step, s_ev,
                                      t_after, st, stats, true, false,
                                      Fields{fld[0][threadIdx.x], fld[1][threadIdx.x],
                                             fld[2][threadIdx.x], fld[3][threadIdx.x],
                                             fld[4][threadIdx.x], fld[5][threadIdx.x]},
                                      false, j);
                s = s_ev + 1;
                t_rem = t_after;
                if (removed || !time_positive(t_rem)) {
                    done = true;
                } else if (!plan_lane()) {
                    active = false;   // handed to rejection, or no energy left
                }
            }
        }
        if (done) {
            if (removed) {
                P.type[i] = QED_REMOVED;   // a decayed photon (Algorithm 2)
            } else if (!photon) {
                P.px[i] = st.px;
                P.py[i] = st.py;
                P.pz[i] = st.pz;
            }
            removed = false;
            active = false;
        }
    }
    stats.warp_substeps = stats.substeps;
    flush_stats(stats, ctl);
}

// Hot pass (rejection).  Long plans (N >= long_min, front of the queue) first,
// one warp each (warp_item), so that their long chains start early; then the
// medium plans (back of the queue), one lane each, with the same warp-shared
// draws as the thread pass but at most kWindow sub-steps per lane and round,
// so that the draws wasted after an event stay short.  Lanes with an event in
// the round apply it and re-plan together, so that the event path is paid
// once per round rather than once per event; lanes whose particle is done
// take the next queue entries (one atomic per warp).  Persistent: the grid is
// the resident block count, and a warp leaves when the queue is empty and its
// lanes are idle.
// kSampler = 1 (per-sub-step sampler): the sampler's particles (e+- in a
// usable bin of its chi range) are queued for the warp mode, which evaluates
// the network (warp_item).  Sampler mode 2 steps its particles in k_samp and
// runs this kernel's rejection form (kSampler = 0) for the others.
constexpr uint32_t kWindow = 64;

template <int kSampler, bool kCells = false>
__global__ void __launch_bounds__(kLaneThreads, QED_LANES_MIN_BLOCKS) k_hot_lanes(DevParticles P, StepParams SP,
                                                                 Scratch S, DevCtl* ctl) {
    const uint32_t step = step_index(SP);
    __shared__ SharedTables sm;
    __shared__ uint32_t first_acc[kLaneThreads];
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    // sampler mode 2 runs its network in k_samp; its generations use k_hot_lanes<0>
    static_assert(kSampler == 0 || kSampler == 1, "hot pass: rejection or sampler mode 1");
    stage_tables(sm);
    if (kSampler == 1)
        stage_sampler(*reinterpret_cast<SamplerSmem*>(dyn_smem),
                      reinterpret_cast<const __nv_bfloat16*>(SP.net_w), SP.net_wtot, SP.net_rows,
                      SP.net_bins);
    __syncthreads();
    if (ctl->status == (int)QED_ERR_TIMEOUT) return;
    constexpr unsigned int kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    uint32_t* facc = first_acc + (threadIdx.x & ~31);
    const uint32_t k0 = (uint32_t)SP.seed, k1 = (uint32_t)(SP.seed >> 32);
    Stats stats;
    {
        // long plans first, one warp each, so that their long chains start early
        const unsigned int long_tail = ctl->hot_tail;
        Stats wstats;                 // counted on lane 0
        unsigned int wcand = 0;
        while (true) {
            unsigned int q = 0;
            if (lane == 0) q = atomicAdd(&ctl->hot_head, 1u);
            q = __shfl_sync(kAll, q, 0);
            if (q >= long_tail) break;
            warp_item<kSampler, kCells>(P, S, SP, ctl, sm, dyn_smem, S.hot[q], step, k0, k1, wstats, wcand,
                                false);
        }
        if (lane == 0) stats = wstats;
        stats.cand = wcand;
    }
    // medium plans, one lane each, from the back of the queue array
    const unsigned int tail = ctl->med_tail;
    bool active = false, photon = false, changed = false, removed = false;
    long long i = 0;
    uint64_t id = 0;
    PState st{0.0f, 0.0f, 0.0f};
    float Ex = 0.0f, Ey = 0.0f, Ez = 0.0f, Bx = 0.0f, By = 0.0f, Bz = 0.0f;
    ftime t_rem{0.0f, 0.0f};
    uint32_t s = 0, k_done = 0;
    Plan pl;
    pl.N = 0;
    pl.T = 0;
    pl.b = pl.c_h = 0.0f;
    float chi = 0.0f, eps = 0.0f;
    bool more = true;   // the queue may hold entries (warp-uniform)
    while (true) {
        bool planned = false;
        if (more) {
            const unsigned int idle = __ballot_sync(kAll, !active);
            if (idle) {
                unsigned int base = 0;
                if (lane == 0) base = atomicAdd(&ctl->med_head, (unsigned int)__popc(idle));
                base = __shfl_sync(kAll, base, 0);
                if (base + (unsigned int)__popc(idle) >= tail) more = false;
                if (!active) {
                    const unsigned int q = base + (unsigned int)__popc(idle & ((1u << lane) - 1u));
                    if (q < tail) {
                        const HotItem it = S.hot[S.hot_cap - 1 - (long long)q];
                        i = it.idx;
                        s = it.s;
                        t_rem = it.t_rem;
                        photon = P.type[i] == QED_PHOTON;
                        id = P.id[i];
                        st = PState{P.px[i], P.py[i], P.pz[i]};
                        Ex = P.Ex[i]; Ey = P.Ey[i]; Ez = P.Ez[i];
                        Bx = P.Bx[i]; By = P.By[i]; Bz = P.Bz[i];
                        changed = removed = false;
                        planned = true;
                    }
                }
            }
        }
        if (planned) {
            pl = plan_particle(SP, sm.sqz_e, sm.sqz_p, photon, st.px, st.py, st.pz, Ex, Ey, Ez,
                               Bx, By, Bz, t_rem, &chi, &eps);
            if (kCells)
                apply_cell_count(SP, pl, sm.sqz_e, sm.sqz_p, photon, i, ctl->n_init, s, t_rem,
                                 eps);
            if (eps > 0.0f) {
                active = true;
                k_done = 0;
                stats.plans++;
                stats.guard += pl.guard ? 1 : 0;
                stats.max_N = max(stats.max_N, pl.N);
                if (pl.T == 0u) {   // no candidates: the plan passes without an event
                    stats.substeps += pl.N;
                    s += pl.N;
                    active = false;
                }
            }
        }
        if (!__any_sync(kAll, active)) {
            if (!more) break;
            continue;
        }
        const uint32_t n_win = active ? min(kWindow, pl.N - k_done) : 0u;
        const uint32_t s_end = s + n_win;
        warp_draw_round(sm, facc, active, s, s_end, pl.T, pl.b, pl.c_h, id, photon, step, SP.draw_keys,
                        stats.cand);
        if (active) {
            const uint32_t s_ev = facc[lane];
            bool done = false;
            if (s_ev == kNoEvent) {
                stats.substeps += n_win;
                s = s_end;
                k_done += n_win;
                done = k_done == pl.N;   // the plan ran out without an event
            } else {
                const uint32_t k = k_done + (s_ev - s);
                stats.substeps += s_ev - s + 1u;
                const float x = draw_x(id, step, s_ev, SP.draw_keys);
                const ftime t_after = (k + 1u == pl.N) ? ftime{0.0f, 0.0f}
                                                       : time_sub_mul(t_rem, k + 1u, pl.h);
                removed = apply_event(P, S, SP, ctl, i, id, photon, x, eps, chi, step, s_ev,
                                      t_after, st, stats, true, false,
                                      Fields{Ex, Ey, Ez, Bx, By, Bz}, false);
                changed = true;
                s = s_ev + 1u;
                t_rem = t_after;
                done = removed || !time_positive(t_rem);
                if (!done) {
                    pl = plan_particle(SP, sm.sqz_e, sm.sqz_p, photon, st.px, st.py, st.pz, Ex,
                                       Ey, Ez, Bx, By, Bz, t_rem, &chi, &eps);
                    k_done = 0;
                    if (!(eps > 0.0f)) {
                        done = true;
                    } else {
                        stats.plans++;
                        stats.guard += pl.guard ? 1 : 0;
                        stats.max_N = max(stats.max_N, pl.N);
                        if (pl.T == 0u) {
                            stats.substeps += pl.N;
                            s += pl.N;
                            done = true;
                        }
                    }
                }
            }
            if (done) {
                if (removed) {
                    P.type[i] = QED_REMOVED;
                } else if (changed) {
                    P.px[i] = st.px;
                    P.py[i] = st.py;
                    P.pz[i] = st.pz;
                }
                active = false;
            }
        }
        __syncwarp();   // facc is reset by the next round
    }
    stats.warp_substeps = stats.substeps;   // every sub-step of this kernel is a hot-pass one
    flush_stats(stats, ctl);
}

// ---------------------------------------------------------------------------
// Tail pass.  Once a cascade generation falls below tail_rows rows, the
// generations stop: a thread pass (k_cold) over that generation, then one
// launch of this persistent kernel finishes the step, taking the thread pass's
// queue and every child appended from then on (rows n0 and up) as they come.
// Each warp takes, in order,
//   1. a long plan from the queue (N >= long_min, or a sampler particle), stepped
//      by the whole warp (warp_item);
//   2. for its idle lanes, child rows appended so far, then the thread pass's
//      medium plans, one lane each, drawn with the warp-shared rounds in windows
//      of kWindow sub-steps.
// A child row is published by its writer (type byte last, after a fence); a
// lane that takes a row still being written waits for it.  Work units are the
// thread pass's queue entries and the child rows; the pass ends when every
// unit known so far (the children: the store count, capped at the capacity,
// less n0) is complete.  Warps add their completed units to the control block
// when they run out of work, so the count is exact whenever the test can
// succeed.  Idle warps back off (256 ns doubling to 4 us), so that their
// polls of the control words do not slow the atomics of the busy ones.  Every
// wait is bounded: past SP.wait_ns (1 s unless qed_set_wait_limit says
// otherwise) without progress anywhere (rows stored or completed, or a beat:
// warps stepping a long chain add one every kBeatRounds rounds), or as many
// 64 ns polls for a queue entry, the kernel records QED_ERR_TIMEOUT and
// returns.
// ---------------------------------------------------------------------------
constexpr unsigned long long kWaitNsDefault = 1000000000ull;   // idle time before giving up: 1 s

// Queue a long plan: the entry's row index is written last (readers wait for it).
__device__ __forceinline__ void push_long(const Scratch& S, DevCtl* ctl, unsigned int cold_long,
                                          long long i, uint32_t s, ftime t_rem) {
    const unsigned int k = cold_long + atomicAdd(&ctl->step_tail, 1u);
    HotItem* e = S.hot + k;
    e->s = s;
    e->t_rem = t_rem;
    __threadfence();
    *reinterpret_cast<volatile uint32_t*>(&e->idx) = (uint32_t)i;
}

template <int kSampler, bool kCells = false>
// Two resident blocks per SM (128 registers, no spills): the tail pass is
// bound by latency, not by the number of warps (three blocks at 80 registers
// spilled 434 bytes a thread and measured 0.8% slower per step).
__global__ void __launch_bounds__(kLaneThreads, 2) k_step(DevParticles P, StepParams SP,
                                                            Scratch S, DevCtl* ctl) {
    const uint32_t step = step_index(SP);
    __shared__ SharedTables sm;
    __shared__ uint32_t first_acc[kLaneThreads];
    __shared__ float fld[6][kLaneThreads];   // E, B at the lane's row (read at plans and events)
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    stage_tables(sm);
    if (kSampler == 1)
        stage_sampler(*reinterpret_cast<SamplerSmem*>(dyn_smem),
                      reinterpret_cast<const __nv_bfloat16*>(SP.net_w), SP.net_wtot, SP.net_rows,
                      SP.net_bins);
    else if (kSampler == 2) {
        stage_sampler_mma(*reinterpret_cast<SamplerMma*>(dyn_smem),
                          reinterpret_cast<const __nv_bfloat16*>(SP.net_w), SP.net_wtot,
                          SP.net_rows, SP.net_bins);
        if (SP.pnet_bins)
            stage_sampler_mma(pair_mma(dyn_smem), reinterpret_cast<const __nv_bfloat16*>(SP.pnet_w),
                              SP.pnet_wtot, SP.net_rows, SP.pnet_bins);
    }
    __syncthreads();
    if (ctl->skip) return;
    constexpr unsigned int kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    uint32_t* facc = first_acc + (threadIdx.x & ~31);
    const uint32_t k0 = (uint32_t)SP.seed, k1 = (uint32_t)(SP.seed >> 32);
    const unsigned long long n0 = (unsigned long long)ctl->n0;
    const bool cascade = SP.cascade != 0;
    // the thread pass's queue (fixed during this kernel)
    const unsigned int cold_long = ctl->hot_tail, cold_med = ctl->med_tail;
    const unsigned long long units0 = (unsigned long long)cold_long + cold_med;
    Stats stats;                 // per lane; the warp mode counts on lane 0
    unsigned int done = 0;       // units this lane completed, not yet added to ctl->finished
    bool active = false, waiting = false, child = false;
    bool photon = false, changed = false, removed = false;
    long long i = 0;
    uint64_t id = 0;
    PState st{0.0f, 0.0f, 0.0f};
    ftime t_rem{0.0f, 0.0f};
    uint32_t s = 0, k_done = 0;
    Plan pl;
    pl.N = 0;
    pl.T = 0;
    pl.b = pl.c_h = 0.0f;
    float chi = 0.0f, eps = 0.0f;
    unsigned int idle = 0, rounds = 0;
    unsigned long long idle_ns = 0, seen = 0;
    unsigned int ticket = kNoItem;   // lane 0: long-queue entry taken, not yet pushed
    unsigned long long pend_lo = 0, pend_hi = 0;   // lane 0: child indices taken, not handed out
    bool timed_out = false;
    while (true) {
        // ---- 1. a long plan, stepped by the whole warp.  Lane 0 takes a ticket
        // with one atomic add when the queue looks non-empty; a ticket past the
        // tail is kept until its entry is pushed (void if the step ends first).
        {
            int got = 0;
            unsigned int q = 0;
            if (lane == 0) {
                if (ticket == kNoItem &&
                    *reinterpret_cast<volatile unsigned int*>(&ctl->hot_head) <
                        cold_long + *reinterpret_cast<volatile unsigned int*>(&ctl->step_tail))
                    ticket = atomicAdd(&ctl->hot_head, 1u);
                if (ticket != kNoItem &&
                    ticket < cold_long + *reinterpret_cast<volatile unsigned int*>(&ctl->step_tail)) {
                    q = ticket;
                    ticket = kNoItem;
                    got = 1;
                }
            }
            got = __shfl_sync(kAll, got, 0);
            if (got) {
                q = __shfl_sync(kAll, q, 0);
                // the entry may still be being written: wait for its row index
                HotItem it;
                it.idx = kNoItem;
                if (lane == 0) {
                    const volatile uint32_t* vi = &S.hot[q].idx;
                    const unsigned long long polls = SP.wait_ns / 64 + 1;
                    for (unsigned long long w = 0; w < polls; ++w) {
                        if (*vi != kNoItem) break;
                        __nanosleep(64);
                    }
                    __threadfence();
                    it = S.hot[q];
                }
                it.idx = __shfl_sync(kAll, it.idx, 0);
                if (it.idx == kNoItem) {
                    timed_out = true;
                    break;
                }
                it.s = __shfl_sync(kAll, it.s, 0);
                it.t_rem.hi = __shfl_sync(kAll, it.t_rem.hi, 0);
                it.t_rem.lo = __shfl_sync(kAll, it.t_rem.lo, 0);
                warp_item<kSampler, kCells>(P, S, SP, ctl, sm, dyn_smem, it, step, k0, k1, stats, stats.cand,
                                    true);
                if (lane == 0) ++done;
                idle = 0;
                idle_ns = 0;
                continue;
            }
        }
        // ---- 2. rows for the idle lanes: children first, then the medium plans.
        // Lane 0 takes child indices with one atomic add into a pending range
        // and hands a lane only an index whose row is reserved already (the
        // rest stay pending; indices never reserved are void when the step
        // ends); medium plans come the same way, an index past their count is
        // dropped.
        {
            const unsigned int free_lanes = __ballot_sync(kAll, !active && !waiting);
            if (free_lanes) {
                const int want = __popc(free_lanes);
                unsigned long long base_c = 0, base_i = 0;
                int got_c = 0, got_i = 0;
                if (lane == 0) {
                    if (cascade) {
                        const unsigned long long stored = stored_rows(P);
                        if (pend_lo == pend_hi) {
                            const unsigned long long ch =
                                *reinterpret_cast<volatile unsigned long long*>(&ctl->child_head);
                            if (ch < stored) {
                                const unsigned long long k =
                                    min((unsigned long long)want, stored - ch);
                                pend_lo = atomicAdd(&ctl->child_head, k);
                                pend_hi = pend_lo + k;
                            }
                        }
                        if (pend_lo < pend_hi && pend_lo < stored) {
                            got_c = (int)min((unsigned long long)want, min(pend_hi, stored) - pend_lo);
                            base_c = pend_lo;
                            pend_lo += (unsigned long long)got_c;
                        }
                    }
                    if (got_c < want &&
                        *reinterpret_cast<volatile unsigned int*>(&ctl->med_head) < cold_med) {
                        const unsigned int k = (unsigned int)(want - got_c);
                        const unsigned int b = atomicAdd(&ctl->med_head, k);
                        base_i = b;
                        got_i = b < cold_med ? (int)min(k, cold_med - b) : 0;
                    }
                }
                got_c = __shfl_sync(kAll, got_c, 0);
                got_i = __shfl_sync(kAll, got_i, 0);
                if (got_c + got_i) {
                    base_c = __shfl_sync(kAll, base_c, 0);
                    base_i = __shfl_sync(kAll, base_i, 0);
                    const int rank = __popc(free_lanes & ((1u << lane) - 1u));
                    if (!active && !waiting && rank < got_c + got_i) {
                        // a child's row index, or a medium plan's queue position
                        child = rank < got_c;
                        i = (long long)(child ? base_c + rank : base_i + (rank - got_c));
                        waiting = true;
                    }
                }
            }
        }
        // ---- 3. lanes holding a row: load and plan it once it is written
        if (waiting) {
            uint32_t s0 = 0;
            if (!child) {   // a medium plan: its row, first sub-step and remaining time
                const HotItem it = S.hot[S.hot_cap - 1 - i];
                i = it.idx;
                s0 = it.s;
                t_rem = it.t_rem;
            }
            const uint8_t ty = *reinterpret_cast<volatile uint8_t*>(P.type + i);
            if (!child || ty != kNotReady) {
                if (child) {
                    __threadfence();
                    t_rem = S.t_rem[i];
                }
                waiting = false;
                photon = ty == QED_PHOTON;
                bool work = ty <= QED_PHOTON && process_enabled(SP, photon) && time_positive(t_rem);
                if (work) {
                    id = P.id[i];
                    st = PState{P.px[i], P.py[i], P.pz[i]};
                    fld[0][threadIdx.x] = P.Ex[i];
                    fld[1][threadIdx.x] = P.Ey[i];
                    fld[2][threadIdx.x] = P.Ez[i];
                    fld[3][threadIdx.x] = P.Bx[i];
                    fld[4][threadIdx.x] = P.By[i];
                    fld[5][threadIdx.x] = P.Bz[i];
                    s = s0;
                    changed = removed = false;
                    pl = plan_particle(SP, sm.sqz_e, sm.sqz_p, photon, st.px, st.py, st.pz,
                                       fld[0][threadIdx.x], fld[1][threadIdx.x],
                                       fld[2][threadIdx.x], fld[3][threadIdx.x],
                                       fld[4][threadIdx.x], fld[5][threadIdx.x], t_rem, &chi, &eps);
                    if (kCells)
                        apply_cell_count(SP, pl, sm.sqz_e, sm.sqz_p, photon, i, ctl->n_init, s,
                                         t_rem, eps);
                    work = eps > 0.0f;
                }
                if (!work) {
                    ++done;
                } else {
                    stats.max_N = max(stats.max_N, pl.N);
                    if (pl.N >= SP.long_min || (!photon && sampler_bin_ok(SP, chi)) ||
                        (kSampler == 2 && photon && pl.N >= SP.hot_min &&
                         pair_sampler_ok(SP, chi, pl.T))) {
                        push_long(S, ctl, cold_long, i, s, t_rem);   // the warp mode plans again
                    } else {
                        stats.plans++;
                        stats.guard += pl.guard ? 1 : 0;
                        if (pl.T == 0u) {   // no candidates: the plan passes without an event
                            stats.substeps += pl.N;
                            ++done;
                        } else {
                            active = true;
                            k_done = 0;
                        }
                    }
                }
            }
        }
        // ---- 4. nothing to draw: wait for work, or finish
        if (!__any_sync(kAll, active)) {
            // lanes waiting for a row still being written hold the warp
            const bool hold = __any_sync(kAll, waiting);
            bool finish = false;
            unsigned long long progress = 0;
            if (!hold) {
                // add this warp's finished rows, then test for the end of the step
                const unsigned long long sum = warp_sum(done);
                done = 0;
                if (lane == 0) {
                    __threadfence();   // this warp's reservations before its completions
                    if (sum) atomicAdd(&ctl->finished, sum);
                    // units to complete: the thread pass's queue, and every child
                    // reserved so far when children are stepped within the step
                    const unsigned long long c1 = units0 + (cascade ? stored_rows(P) - n0 : 0ull);
                    const unsigned long long f =
                        *reinterpret_cast<volatile unsigned long long*>(&ctl->finished);
                    const unsigned long long c2 = units0 + (cascade ? stored_rows(P) - n0 : 0ull);
                    finish = f == c1 && c1 == c2;
                    progress = f + c2 + *reinterpret_cast<volatile unsigned long long*>(&ctl->beat);
                }
                finish = __shfl_sync(kAll, finish ? 1 : 0, 0) != 0;
                progress = __shfl_sync(kAll, progress, 0);
            }
            if (finish) break;
            // idle: back off from 256 ns to 4 us (64 ns while a row is being
            // written); the idle time counts from the last progress seen
            // (rows stored or completed, beats of long chains)
            if (!hold && progress != seen) {
                seen = progress;
                idle_ns = 0;
            }
            const unsigned int nap = hold ? 64u : 256u << min(idle, 4u);
            ++idle;
            idle_ns += nap;
            if (idle_ns > SP.wait_ns) {
                timed_out = true;
                break;
            }
            __nanosleep(nap);
            continue;
        }
        idle = 0;
        idle_ns = 0;
        if (++rounds == kBeatRounds) {
            rounds = 0;
            if (lane == 0) atomicAdd(&ctl->beat, 1ull);
        }
        // ---- 5. one round of warp-shared draws for the active lanes
        const uint32_t n_win = active ? min(kWindow, pl.N - k_done) : 0u;
        const uint32_t s_end = s + n_win;
        warp_draw_round(sm, facc, active, s, s_end, pl.T, pl.b, pl.c_h, id, photon, step, SP.draw_keys,
                        stats.cand);
        if (active) {
            const uint32_t s_ev = facc[lane];
            bool fin = false;
            if (s_ev == kNoEvent) {
                stats.substeps += n_win;
                s = s_end;
                k_done += n_win;
                fin = k_done == pl.N;   // the plan ran out without an event
            } else {
                const uint32_t k = k_done + (s_ev - s);
                stats.substeps += s_ev - s + 1u;
                const float x = draw_x(id, step, s_ev, SP.draw_keys);
                const ftime t_after = (k + 1u == pl.N) ? ftime{0.0f, 0.0f}
                                                       : time_sub_mul(t_rem, k + 1u, pl.h);
                removed = apply_event(P, S, SP, ctl, i, id, photon, x, eps, chi, step, s_ev,
                                      t_after, st, stats, true, false,
                                      Fields{fld[0][threadIdx.x], fld[1][threadIdx.x],
                                             fld[2][threadIdx.x], fld[3][threadIdx.x],
                                             fld[4][threadIdx.x], fld[5][threadIdx.x]},
                                      true);
                changed = true;
                s = s_ev + 1u;
                t_rem = t_after;
                fin = removed || !time_positive(t_rem);
                if (!fin) {
                    pl = plan_particle(SP, sm.sqz_e, sm.sqz_p, photon, st.px, st.py, st.pz,
                                       fld[0][threadIdx.x], fld[1][threadIdx.x],
                                       fld[2][threadIdx.x], fld[3][threadIdx.x],
                                       fld[4][threadIdx.x], fld[5][threadIdx.x], t_rem, &chi,
                                       &eps);
                    k_done = 0;
                    if (!(eps > 0.0f)) {
                        fin = true;
                    } else {
                        stats.max_N = max(stats.max_N, pl.N);
                        if (pl.N >= SP.long_min || (!photon && sampler_bin_ok(SP, chi)) ||
                        (kSampler == 2 && photon && pl.N >= SP.hot_min &&
                         pair_sampler_ok(SP, chi, pl.T))) {
                            // continue in the warp mode; its state goes with the row
                            P.px[i] = st.px;
                            P.py[i] = st.py;
                            P.pz[i] = st.pz;
                            changed = false;
                            push_long(S, ctl, cold_long, i, s, t_rem);
                            active = false;
                        } else {
                            stats.plans++;
                            stats.guard += pl.guard ? 1 : 0;
                            if (pl.T == 0u) {
                                stats.substeps += pl.N;
                                s += pl.N;
                                fin = true;
                            }
                        }
                    }
                }
            }
            if (fin) {
                if (removed) {
                    P.type[i] = QED_REMOVED;
                } else if (changed) {
                    P.px[i] = st.px;
                    P.py[i] = st.py;
                    P.pz[i] = st.pz;
                }
                active = false;
                ++done;
            }
        }
        __syncwarp();   // facc is reset by the next round
    }
    if (timed_out && lane == 0) atomicExch(&ctl->status, (int)QED_ERR_TIMEOUT);
    const unsigned long long sum = warp_sum(done);
    if (lane == 0 && sum) atomicAdd(&ctl->finished, sum);
    stats.warp_substeps = stats.substeps;   // every sub-step of this kernel is a hot-pass one
    flush_stats(stats, ctl);
}

// Before the persistent step (cascading): rows [n0, capacity) are free; mark
// them not written, so that a lane taking a child row waits for its writer.

// Start a step.  keep_sticky: inside a multi-step graph, a step that follows
// a failed step does nothing (its range is empty and it keeps the status).
__global__ void k_step_init(DevCtl* ctl, long long* count, long long capacity, int keep_sticky) {
    const int sticky = keep_sticky ? ctl->sticky : 0;
    DevCtl c;
    memset(&c, 0, sizeof c);
    long long n = *count;
    if (n < 0) n = 0;
    if (n > capacity) n = capacity;
    *count = n;
    c.pass_begin = 0;
    c.pass_end = sticky ? 0 : n;
    c.n_init = n;
    c.first_pass = 1;
    c.sticky = sticky;
    c.status = sticky;
    *ctl = c;
}

// Close a cascade generation: the next generation is the rows appended during
// this one.  In a graph, the WHILE node's condition is set here.
// The hot-pass and tail-pass kernels for a sampler mode (0: off, 1: per
// sub-step, 2: event-driven), each its own instantiation so that a mode's
// code carries no other mode's path.
// cells: the step takes per-cell counts for the first plans (only without a
// learned sampler); its kernels are separate instantiations, so that the
// plain step carries none of that code.
const void* cold_kernel(bool cells) {
    return cells ? (const void*)k_cold<true> : (const void*)k_cold<false>;
}
const void* hot_kernel(int mode, bool cells = false) {
    // sampler mode 2 runs its network in k_samp: the hot pass of its
    // generations is rejection's (loop_hot_mode), so there is no k_hot_lanes<2>
    return mode == 1 ? (const void*)k_hot_lanes<1>
                     : cells ? (const void*)k_hot_lanes<0, true> : (const void*)k_hot_lanes<0>;
}
const void* step_kernel(int mode, bool cells = false) {
    return mode == 2 ? (const void*)k_step<2>
                     : mode ? (const void*)k_step<1>
                            : cells ? (const void*)k_step<0, true> : (const void*)k_step<0>;
}

// tail_rows > 0: a next generation of fewer rows goes to the tail pass
// instead (ctl->tail set, the loop ends).
__global__ void k_advance(DevCtl* ctl, long long* count, long long capacity, int more_allowed,
                          int max_passes, long long tail_rows, cudaGraphConditionalHandle handle,
                          int use_handle) {
    long long n = *count;
    if (n > capacity) {
        n = capacity;
        *count = capacity;
    }
    ctl->pass_begin = ctl->sticky ? 0 : ctl->pass_end;
    ctl->pass_end = ctl->sticky ? 0 : n;
    ctl->hot_hw = max(ctl->hot_hw, ctl->hot_tail);
    ctl->hot_head = 0;
    ctl->hot_tail = 0;
    ctl->med_head = 0;
    ctl->med_tail = 0;
    ctl->samp_head = 0;
    ctl->samp_tail = 0;
    ctl->passes += 1;
    ctl->first_pass = 0;
    int more = (more_allowed && ctl->pass_end > ctl->pass_begin && ctl->status == 0) ? 1 : 0;
    if (more && ctl->passes >= max_passes) {
        more = 0;
        ctl->status = (int)QED_ERR_STATE;  // cascade deeper than the configured passes
    }
    if (more && tail_rows > 0 && ctl->pass_end - ctl->pass_begin < tail_rows) {
        more = 0;
        ctl->tail = 1;
    }
    ctl->more = more;
    if (use_handle) cudaGraphSetConditional(handle, (unsigned int)more);
}

// Start of the tail pass (or nothing, when the generations ran to the end):
// rows from pass_end to the capacity are marked not written, so that a lane
// taking a child row waits for its writer, and the long-plan queue entries
// the generations wrote go back to "not written", so that a warp waiting for
// an entry the persistent kernel pushes never reads an older one.  The thread
// pass that follows runs over [pass_begin, pass_end) as one more generation.
__global__ void k_tail_begin(DevParticles P, Scratch S, DevCtl* ctl) {
    const bool on = ctl->tail != 0;
    const long long n0 = ctl->pass_end;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t0 == 0) {
        ctl->skip = on ? 0 : 1;
        ctl->n0 = n0;
        ctl->child_head = (unsigned long long)n0;
        ctl->finished = 0;
        ctl->step_tail = 0;
    }
    if (!on) return;
    for (long long r = n0 + t0; r < P.capacity; r += stride) P.type[r] = kNotReady;
    const long long used = min((long long)ctl->hot_hw, S.hot_cap);
    for (long long q = t0; q < used; q += stride) S.hot[q].idx = kNoItem;
}

// Start of a push step run as one persistent pass (k_push<true>): the rows
// past the initial ones are marked not written, so that a lane taking a child
// row waits for its writer, and the step is marked as a tail pass (k_tail_end
// then caps the count and clears the rows past it).
__global__ void k_push_begin(DevParticles P, DevCtl* ctl) {
    const long long n0 = ctl->n_init;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t0 == 0) ctl->tail = 1;
    for (long long r = n0 + t0; r < P.capacity; r += stride) P.type[r] = kNotReady;
}

// End of the step: after a tail pass the count is capped at the capacity
// (children that did not fit were dropped and the status says so) and rows
// past it go back to removed; in every step the long-plan queue entries used
// go back to "not written".
__global__ void k_tail_end(DevParticles P, Scratch S, DevCtl* ctl) {
    const bool on = ctl->tail != 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long c = min(*P.count, P.capacity);
    if (on) {
        for (long long r = c + t0; r < P.capacity; r += stride) P.type[r] = QED_REMOVED;
        if (t0 == 0) {
            *P.count = c;
            ctl->pass_begin = ctl->pass_end;
            ctl->pass_end = ctl->sticky ? 0 : c;   // the count the step reports
            ctl->passes += 1;
        }
    }
    const long long used =
        min(max((long long)ctl->hot_hw, (long long)ctl->hot_tail + ctl->step_tail), S.hot_cap);
    for (long long q = t0; q < used; q += stride) S.hot[q].idx = kNoItem;
}

// Write the statistics of the step into `rec` (if not null); an error becomes
// sticky for the following steps of a graph run.
__global__ void k_step_close(DevCtl* ctl, const long long* count, qed_step_stats* rec,
                             uint32_t* step_base, uint32_t advance) {
    const DevCtl c = *ctl;
    if (step_base && advance) *step_base += advance;
    if (rec) {
        qed_step_stats r;
        r.substeps = c.substeps;
        r.emissions = c.emissions;
        r.pairs = c.pairs;
        r.children = c.children;
        r.guard_hits = c.guard_hits;
        r.plans = c.plans;
        r.candidates = c.candidates;
        r.max_N = c.max_N;
        r.status = c.status;
        r.required_capacity = c.required;
        r.count = *count;
        r.passes = c.passes;
        r.tail = c.tail;
        r.substeps_warp = c.substeps_warp;
        r.sampler_events = c.sampler_events;
        r.sampler_pairs = c.sampler_pairs;
        *rec = r;
    }
    if (c.status != 0 && c.sticky == 0) ctl->sticky = c.status;
}

// Reset the sticky status at the start of a multi-step graph run.
__global__ void k_graph_begin(DevCtl* ctl) { ctl->sticky = 0; }

// ---------------------------------------------------------------------------
// Compaction: squeeze removed rows (decayed or drained photons) out of the
// store, keeping the order of the remaining rows.  Optionally drains photons
// whose chi is below `drain_chi` into a weighted log-energy spectrum first.
// Out of place through a mirror store, then copied back.
// ---------------------------------------------------------------------------
constexpr int kCompactThreads = 1024;
constexpr int kCompactRows = 4;                        // rows per thread per tile
constexpr int kTile = kCompactThreads * kCompactRows;  // rows per block

struct Mirror {
    float *px, *py, *pz, *Ex, *Ey, *Ez, *Bx, *By, *Bz, *w;
    uint64_t* id;
    uint8_t* type;
};

__device__ __forceinline__ long long clamp_count(const DevParticles& P) {
    long long n = *P.count;
    return n < 0 ? 0 : (n > P.capacity ? P.capacity : n);
}

__global__ void __launch_bounds__(kCompactThreads)
    k_compact_count(DevParticles P, StepParams SP, float drain_chi, double* hist,
                    unsigned int* block_live) {
    __shared__ unsigned int warp_tot[kCompactThreads / 32];
    // the block's drained weight per bin, added to the spectrum once per bin:
    // the drained photons crowd a few energy bins, and one global atomic per
    // photon serialised on them
    __shared__ double sh_hist[QED_SPECTRUM_BINS];
    for (int b = threadIdx.x; b < QED_SPECTRUM_BINS; b += blockDim.x) sh_hist[b] = 0.0;
    __syncthreads();
    const long long n = clamp_count(P);
    const long long base = (long long)blockIdx.x * kTile;
    unsigned int live = 0;
    if (base < n) {
#pragma unroll
        for (int k = 0; k < kCompactRows; ++k) {
            const long long i = base + (long long)k * kCompactThreads + threadIdx.x;
            if (i >= n) break;
            uint8_t t = P.type[i];
            if (t == QED_PHOTON && drain_chi > 0.0f) {
                float eps;
                const float chi = chi_ff(true, P.px[i], P.py[i], P.pz[i], P.Ex[i], P.Ey[i], P.Ez[i],
                                         P.Bx[i], P.By[i], P.Bz[i], SP.inv_Es, &eps);
                if (chi < drain_chi) {
                    if (hist) {
                        const float l = log10f(fmaxf(eps, 1e-30f));
                        int bin = (int)floorf((l - (float)QED_SPECTRUM_LOG10_MIN) *
                                              ((float)QED_SPECTRUM_BINS /
                                               (float)(QED_SPECTRUM_LOG10_MAX - QED_SPECTRUM_LOG10_MIN)));
                        bin = min(max(bin, 0), QED_SPECTRUM_BINS - 1);
                        atomicAdd(&sh_hist[bin], (double)P.w[i]);
                    }
                    P.type[i] = QED_REMOVED;
                    t = QED_REMOVED;
                }
            }
            live += t <= QED_PHOTON ? 1u : 0u;
        }
    }
    // block sum
    unsigned int v = live;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned int w = warp_tot[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (threadIdx.x == 0) block_live[blockIdx.x] = w;
    }
    if (hist)
        for (int b = threadIdx.x; b < QED_SPECTRUM_BINS; b += blockDim.x)
            if (sh_hist[b] != 0.0) atomicAdd(&hist[b], sh_hist[b]);
}

// Exclusive scan of the per-tile counts (one block); total -> ctl->live.
__global__ void __launch_bounds__(kCompactThreads)
    k_compact_scan(unsigned int* block_live, int nb, DevCtl* ctl, const long long* count) {
    __shared__ unsigned long long part[kCompactThreads];
    const int per = (nb + kCompactThreads - 1) / kCompactThreads;
    const int lo = threadIdx.x * per;
    const int hi = min(lo + per, nb);
    unsigned long long sum = 0;
    for (int i = lo; i < hi; ++i) sum += block_live[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    // Hillis-Steele inclusive scan over the 1024 partial sums
    for (int o = 1; o < kCompactThreads; o <<= 1) {
        const unsigned long long add = threadIdx.x >= o ? part[threadIdx.x - o] : 0ull;
        __syncthreads();
        part[threadIdx.x] += add;
        __syncthreads();
    }
    unsigned long long run = part[threadIdx.x] - sum;  // exclusive
    for (int i = lo; i < hi; ++i) {
        const unsigned int c = block_live[i];
        block_live[i] = (unsigned int)run;
        run += c;
    }
    if (threadIdx.x == kCompactThreads - 1) {
        const long long total = (long long)part[kCompactThreads - 1];
        long long n = *count;
        ctl->live = total;
        ctl->compact_needed = total != n ? 1 : 0;
    }
}

__global__ void __launch_bounds__(kCompactThreads)
    k_compact_scatter(DevParticles P, Mirror M, const unsigned int* block_off, const DevCtl* ctl) {
    if (!ctl->compact_needed) return;
    __shared__ unsigned int warp_tot[kCompactThreads / 32];
    __shared__ unsigned int carry;
    const long long n = clamp_count(P);
    const long long base = (long long)blockIdx.x * kTile;
    if (base >= n) return;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long off = block_off[blockIdx.x];
    for (int k = 0; k < kCompactRows; ++k) {
        const long long i = base + (long long)k * kCompactThreads + threadIdx.x;
        const bool keep = i < n && P.type[i] <= QED_PHOTON;
        const unsigned int b = __ballot_sync(0xffffffffu, keep);
        const unsigned int in_warp = __popc(b & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[warp] = __popc(b);
        __syncthreads();
        if (warp == 0) {
            const unsigned int v = warp_tot[lane];
            unsigned int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            warp_tot[lane] = incl - v;  // exclusive offsets of the warps
        }
        __syncthreads();
        if (keep) {
            const long long d = off + carry + warp_tot[warp] + in_warp;
            M.px[d] = P.px[i]; M.py[d] = P.py[i]; M.pz[d] = P.pz[i];
            M.Ex[d] = P.Ex[i]; M.Ey[d] = P.Ey[i]; M.Ez[d] = P.Ez[i];
            M.Bx[d] = P.Bx[i]; M.By[d] = P.By[i]; M.Bz[d] = P.Bz[i];
            M.w[d] = P.w[i]; M.id[d] = P.id[i]; M.type[d] = P.type[i];
        }
        __syncthreads();
        if (threadIdx.x == kCompactThreads - 1)
            carry += warp_tot[warp] + in_warp + (keep ? 1u : 0u);
        __syncthreads();
    }
}

__global__ void k_compact_copyback(DevParticles P, Mirror M, DevCtl* ctl) {
    if (!ctl->compact_needed) return;
    const long long live = ctl->live;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < live; i += stride) {
        P.px[i] = M.px[i]; P.py[i] = M.py[i]; P.pz[i] = M.pz[i];
        P.Ex[i] = M.Ex[i]; P.Ey[i] = M.Ey[i]; P.Ez[i] = M.Ez[i];
        P.Bx[i] = M.Bx[i]; P.By[i] = M.By[i]; P.Bz[i] = M.Bz[i];
        P.w[i] = M.w[i]; P.id[i] = M.id[i]; P.type[i] = M.type[i];
    }
}

__global__ void k_compact_finish(DevParticles P, const DevCtl* ctl) {
    if (ctl->compact_needed) *P.count = ctl->live;
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
// One learned sampler's state (context-owned).
struct NetState {
    float* d_theta;            // FP32 master parameters
    float* d_m1;               // Adam moments
    float* d_m2;
    __nv_bfloat16* d_wbf;      // BF16 copy used by the event kernels
    float* d_cdf;              // exact CDF rows (training targets)
    float* d_wtot;             // total probability per c along log10 chi
    int net_ready;             // parameters loaded or trained
    unsigned long long net_bins;
    long long adam_t;
};

struct qed_ctx {
    qed_config cfg;
    cudaStream_t stream;
    int device;
    int sms;
    DevCtl* d_ctl;
    DevCtl* h_ctl;          // pinned
    ftime* d_trem;
    HotItem* d_hot;
    long long scratch_cap;
    qed_event_record* log;
    long long log_cap;
    long long* log_count;
    int cold_blocks, hot_blocks;
    int cold_blocks_max, hot_blocks_max;
    int net_blocks;           // grid of the hot pass in sampler mode
    uint32_t hot_min, long_min;
    long long tail_rows;        // cascade generations below this size go to the tail pass
    unsigned long long wait_ns; // longest bounded wait of the tail pass
    int step_blocks, step_net_blocks;   // resident blocks of the tail pass's kernel
    int plan_blocks;                    // resident blocks of the planner (k_plan)
    int samp_blocks;            // resident blocks of the event-driven sampler kernel
    HotItem* d_samp;            // its queue (capacity entries), allocated on first use
    long long samp_cap;
    int push_blocks;            // resident blocks of the push-mode kernel
    unsigned int* d_Ncell;      // per-cell counts of the push mode with cells
    long long ncell_cap;
    unsigned char* d_hstore;    // device copy of a host store (qed_event_step_host)
    long long hstore_cap;
    // compaction
    Mirror mirror;
    long long mirror_cap;
    unsigned int* d_block_live;
    double* d_hist;
    // learned samplers: nets[0] emission (Eq. 1), nets[1] pair production
    // (Eq. 2); net_sel is the one the qed_sampler_* calls address
    NetState nets[2];
    int net_sel;
    float* d_partial;          // per-block partial gradients
    float* d_batch;            // training inputs (2 per sample), targets and weights
    int batch_cap;
    float* d_loss;
    // multi-step graph
    cudaGraph_t graph;
    cudaGraphExec_t graph_exec;
    // one event step as a graph (generations in a device-side loop), rebuilt
    // when its key (store, scratch, parameters, grids) changes
    cudaGraph_t step_graph;
    cudaGraphExec_t step_exec;
    uint64_t step_key[64];
    int step_key_n;
    uint32_t* d_step_idx;
    qed_step_stats* d_records;
    uint32_t* d_step_base;
    int graph_steps;
    // benchmark timing: event pairs recorded around launches
    int prof_on;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_kind;
    size_t prof_used;
    long long launches[QED_KERNEL_KINDS];
    char err[512];
};

namespace {
qed_status sampler_params(qed_ctx* ctx, StepParams* SP);
}  // namespace

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
    P.K = (float)rate_K64(c.lambda_m);                        // sqrt3 R / pi, 1 / period
    P.t_step.hi = (float)c.dt_periods;
    P.t_step.lo = (float)(c.dt_periods - (double)P.t_step.hi);
    P.inv_Es = (float)inv_schwinger64(c.lambda_m);            // 1 / E_s in code units
    P.p_max = c.p_max;
    P.inv_p_max = 1.0f / c.p_max;
    P.pair_coeff = c.pair_bound_coeff;
    P.lambda_m = c.lambda_m;
    P.draw_keys = philox_keys((uint32_t)c.seed, (uint32_t)(c.seed >> 32));
    P.child_keys = philox_keys((uint32_t)c.seed ^ kChildKeyLo, (uint32_t)(c.seed >> 32) ^ kChildKeyHi);
    P.wait_ns = kWaitNsDefault;
    P.step_base = nullptr;
    P.hot_min = kHotMinDefault;
    P.long_min = kLongMinDefault;
    P.sampler = 0;
    P.net_rows = 0;
    P.net_bins = 0;
    P.net_w = nullptr;
    P.net_wtot = nullptr;
    P.pnet_bins = 0;
    P.pnet_w = nullptr;
    P.pnet_wtot = nullptr;
    P.step = (uint32_t)step;
    P.process_mask = c.process_mask;
    P.recoil = c.recoil;
    P.cascade = c.cascade_in_step;
    P.cell = nullptr;
    P.N_cell = nullptr;
    P.ncells = 0;
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
    QED_CUDA(ctx, cudaMalloc(&ctx->d_trem, sizeof(ftime) * cap));
    // queue: long plans from the front, medium plans from the back.  Every
    // entry belongs to a row and a row has at most two entries per generation
    // (in the tail pass a medium plan may come back as a long plan), so 2 cap
    // entries never let the ends meet.  Long-plan entries start "not written"
    // (row index all ones) and each step resets the ones it used.
    QED_CUDA(ctx, cudaMalloc(&ctx->d_hot, sizeof(HotItem) * 2 * cap));
    QED_CUDA(ctx, cudaMemset(ctx->d_hot, 0xFF, sizeof(HotItem) * 2 * cap));
    ctx->scratch_cap = cap;
    return QED_OK;
}

// The event-driven sampler's queue (sampler mode 2): one entry per row at most
// per generation.  Sets S->samp.
qed_status ensure_samp(qed_ctx* ctx, long long cap, const StepParams& SP, Scratch* S) {
    if (SP.sampler != 2) return QED_OK;
    if (ctx->samp_cap < cap) {
        if (ctx->d_samp) cudaFree(ctx->d_samp);
        ctx->d_samp = nullptr;
        ctx->samp_cap = 0;
        QED_CUDA(ctx, cudaMalloc(&ctx->d_samp, sizeof(HotItem) * cap));
        ctx->samp_cap = cap;
    }
    S->samp = ctx->d_samp;
    return QED_OK;
}

// Sampler mode of the generations' hot pass: with the event-driven sampler its
// particles run in k_samp before the hot pass, which then steps rejection
// plans only.
int loop_hot_mode(const StepParams& SP) { return SP.sampler == 2 ? 0 : SP.sampler; }

// Generations below this size go to the tail pass.
long long tail_rows_for(const qed_ctx* ctx, const StepParams&) { return ctx->tail_rows; }

// Bracket a launch with timing events when profiling is on; count it always.
struct LaunchScope {
    qed_ctx* ctx;
    int kind;
    size_t slot;
    LaunchScope(qed_ctx* c, int k) : ctx(c), kind(k), slot((size_t)-1) {
        ctx->launches[kind]++;
        if (!ctx->prof_on) return;
        if (ctx->prof_used + 2 > ctx->prof_ev.size()) {
            size_t grow = ctx->prof_ev.size() ? ctx->prof_ev.size() : 512;
            for (size_t i = 0; i < grow; ++i) {
                cudaEvent_t e;
                if (cudaEventCreate(&e) != cudaSuccess) return;
                ctx->prof_ev.push_back(e);
            }
        }
        slot = ctx->prof_used;
        ctx->prof_used += 2;
        ctx->prof_kind.push_back(kind);
        cudaEventRecord(ctx->prof_ev[slot], ctx->stream);
    }
    ~LaunchScope() {
        if (slot != (size_t)-1) cudaEventRecord(ctx->prof_ev[slot + 1], ctx->stream);
    }
};

qed_status ensure_mirror(qed_ctx* ctx, long long cap) {
    if (!ctx->d_hist) {
        QED_CUDA(ctx, cudaMalloc(&ctx->d_hist, sizeof(double) * QED_SPECTRUM_BINS));
        QED_CUDA(ctx, cudaMemsetAsync(ctx->d_hist, 0, sizeof(double) * QED_SPECTRUM_BINS,
                                      ctx->stream));
    }
    if (ctx->mirror_cap >= cap) return QED_OK;
    float** f[] = {&ctx->mirror.px, &ctx->mirror.py, &ctx->mirror.pz, &ctx->mirror.Ex,
                   &ctx->mirror.Ey, &ctx->mirror.Ez, &ctx->mirror.Bx, &ctx->mirror.By,
                   &ctx->mirror.Bz, &ctx->mirror.w};
    for (float** a : f) {
        if (*a) cudaFree(*a);
        *a = nullptr;
    }
    if (ctx->mirror.id) cudaFree(ctx->mirror.id);
    if (ctx->mirror.type) cudaFree(ctx->mirror.type);
    if (ctx->d_block_live) cudaFree(ctx->d_block_live);
    ctx->mirror.id = nullptr;
    ctx->mirror.type = nullptr;
    ctx->d_block_live = nullptr;
    ctx->mirror_cap = 0;
    for (float** a : f) QED_CUDA(ctx, cudaMalloc(a, sizeof(float) * cap));
    QED_CUDA(ctx, cudaMalloc(&ctx->mirror.id, sizeof(uint64_t) * cap));
    QED_CUDA(ctx, cudaMalloc(&ctx->mirror.type, cap));
    const long long nb = (cap + kTile - 1) / kTile;
    QED_CUDA(ctx, cudaMalloc(&ctx->d_block_live, sizeof(unsigned int) * nb));
    ctx->mirror_cap = cap;
    return QED_OK;
}

void free_graph(qed_ctx* ctx) {
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    if (ctx->d_records) cudaFree(ctx->d_records);
    if (ctx->d_step_base) cudaFree(ctx->d_step_base);
    ctx->graph_exec = nullptr;
    ctx->graph = nullptr;
    ctx->d_records = nullptr;
    ctx->d_step_base = nullptr;
    ctx->graph_steps = 0;
}

bool cascade_enabled(const qed_config& c) {
    return c.cascade_in_step &&
           (c.process_mask & (QED_PROC_EMISSION | QED_PROC_PAIR)) ==
               (QED_PROC_EMISSION | QED_PROC_PAIR);
}

Scratch make_scratch(const qed_ctx* ctx) {
    Scratch S;
    S.t_rem = ctx->d_trem;
    S.hot = ctx->d_hot;
    S.hot_cap = 2 * ctx->scratch_cap;
    S.samp = nullptr;
    S.log = ctx->log;
    S.log_cap = ctx->log_cap;
    S.log_count = ctx->log_count;
    return S;
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
    out->tail = c.tail;
    out->substeps_warp = c.substeps_warp;
    out->sampler_events = c.sampler_events;
    out->sampler_pairs = c.sampler_pairs;
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
    c->drain_chi = 0.0f;
    c->sampler_mode = 0;
    c->sampler_max_err = 1e-3f;
}

qed_status qed_init(qed_ctx** out, const qed_config* cfg, void* stream) {
    if (!out || !cfg) return QED_ERR_ARG;
    *out = nullptr;
    if (!(cfg->p_max > 0.0f && cfg->p_max <= 1.0f) || !(cfg->dt_periods > 0.0) ||
        !(cfg->lambda_m > 0.0) || !(cfg->pair_bound_coeff > 0.0f) || !(cfg->drain_chi >= 0.0f) ||
        cfg->sampler_mode < 0 || cfg->sampler_mode > 2)
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
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cold<false>, kColdThreads, 0);
        ctx->cold_blocks = ctx->cold_blocks_max = ctx->sms * (per_sm > 0 ? per_sm : 1);
        per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hot_lanes<0>, kLaneThreads, 0);
        ctx->hot_blocks = ctx->hot_blocks_max = ctx->sms * (per_sm > 0 ? per_sm : 1);
        per_sm = 0;
        cudaFuncSetAttribute(hot_kernel(1), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kNetSmemBytes);
        for (int m = 1; m <= 2; ++m)
            cudaFuncSetAttribute(step_kernel(m), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kNetSmemBytes);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hot_lanes<1>, kLaneThreads,
                                                      kNetSmemBytes);
        ctx->net_blocks = ctx->sms * (per_sm > 0 ? per_sm : 1);
        per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step<0>, kLaneThreads, 0);
        ctx->step_blocks = ctx->sms * (per_sm > 0 ? per_sm : 1);
        per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_plan, kColdThreads, 0);
        ctx->plan_blocks = ctx->sms * (per_sm > 0 ? per_sm : 1);
        per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step<1>, kLaneThreads,
                                                      kNetSmemBytes);
        ctx->step_net_blocks = ctx->sms * (per_sm > 0 ? per_sm : 1);
        per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push<true>, kLaneThreads, 0);
        ctx->push_blocks = ctx->sms * (per_sm > 0 ? per_sm : 1);
        per_sm = 0;
        cudaFuncSetAttribute(k_samp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kMmaSmemBytes);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_samp, kLaneThreads,
                                                      kMmaSmemBytes);
        ctx->samp_blocks = ctx->sms * (per_sm > 0 ? per_sm : 1);
        ctx->hot_min = kHotMinDefault;
        ctx->long_min = kLongMinDefault;
        ctx->tail_rows = kTailRowsDefault;
        ctx->wait_ns = kWaitNsDefault;
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
    if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
    if (ctx->step_graph) cudaGraphDestroy(ctx->step_graph);
    if (ctx->d_step_idx) cudaFree(ctx->d_step_idx);
    for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
    if (ctx->stream || ctx->d_ctl) cudaStreamSynchronize(ctx->stream);
    if (ctx->d_ctl) cudaFree(ctx->d_ctl);
    if (ctx->h_ctl) cudaFreeHost(ctx->h_ctl);
    if (ctx->d_trem) cudaFree(ctx->d_trem);
    if (ctx->d_hot) cudaFree(ctx->d_hot);
    if (ctx->d_Ncell) cudaFree(ctx->d_Ncell);
    if (ctx->d_samp) cudaFree(ctx->d_samp);
    if (ctx->d_hstore) cudaFree(ctx->d_hstore);
    free_graph(ctx);
    float* f[] = {ctx->mirror.px, ctx->mirror.py, ctx->mirror.pz, ctx->mirror.Ex, ctx->mirror.Ey,
                  ctx->mirror.Ez, ctx->mirror.Bx, ctx->mirror.By, ctx->mirror.Bz, ctx->mirror.w};
    for (float* a : f)
        if (a) cudaFree(a);
    if (ctx->mirror.id) cudaFree(ctx->mirror.id);
    if (ctx->mirror.type) cudaFree(ctx->mirror.type);
    if (ctx->d_block_live) cudaFree(ctx->d_block_live);
    if (ctx->d_hist) cudaFree(ctx->d_hist);
    for (NetState& N : ctx->nets) {
        void* np[] = {N.d_theta, N.d_m1, N.d_m2, N.d_wbf, N.d_cdf, N.d_wtot};
        for (void* a : np)
            if (a) cudaFree(a);
    }
    void* sp[] = {ctx->d_partial, ctx->d_batch, ctx->d_loss};
    for (void* a : sp)
        if (a) cudaFree(a);
    delete ctx;
    return QED_OK;
}

const char* qed_last_error(const qed_ctx* ctx) { return ctx ? ctx->err : "null context"; }

qed_status qed_synchrotron_F1F2(qed_ctx* ctx, const float* y, float* F1, float* F2, int64_t n) {
    if (!ctx) return QED_ERR_ARG;
    if (n == 0 || (n > 0 && !F1 && !F2)) return QED_OK;
    if (!y || n < 0) return set_err(ctx, QED_ERR_ARG, "qed_synchrotron_F1F2: bad argument");
    const int vec = ((((uintptr_t)y) | ((uintptr_t)F1) | ((uintptr_t)F2)) & 15u) == 0 ? 1 : 0;
    long long work = vec ? (n + 3) / 4 : n;
    long long blocks = (work + kSweepThreads - 1) / kSweepThreads;
    const long long max_blocks = (long long)ctx->sms * 8;
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    LaunchScope ls(ctx, QED_KERNEL_SWEEP);
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
    LaunchScope ls(ctx, QED_KERNEL_GENERATE);
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
    if (blocks > ctx->plan_blocks) blocks = ctx->plan_blocks;
    LaunchScope ls(ctx, QED_KERNEL_PLAN);
    k_plan<<<(int)blocks, kColdThreads, 0, ctx->stream>>>(to_dev(p), SP, n, chi, N, nullptr, 0ll,
                                                          nullptr, nullptr);
    return cuda_check(ctx, cudaGetLastError(), "k_plan");
}

qed_status qed_plan_cells(qed_ctx* ctx, const qed_particles* p, int64_t n, const uint32_t* cell,
                          int64_t ncells, uint32_t* N_cell) {
    if (!ctx) return QED_ERR_ARG;
    if (!particles_ok(p) || n < 0 || n > p->capacity || ncells < 0 || (n > 0 && !cell) ||
        (ncells > 0 && !N_cell))
        return set_err(ctx, QED_ERR_ARG, "qed_plan_cells: bad argument");
    if (ncells == 0) return QED_OK;
    QED_CUDA(ctx, cudaMemsetAsync(N_cell, 0, sizeof(uint32_t) * (size_t)ncells, ctx->stream));
    if (n == 0) return QED_OK;
    const StepParams SP = make_params(ctx->cfg, 0);
    long long blocks = (n + kColdThreads - 1) / kColdThreads;
    if (blocks > ctx->plan_blocks) blocks = ctx->plan_blocks;
    LaunchScope ls(ctx, QED_KERNEL_PLAN);
    k_plan<<<(int)blocks, kColdThreads, 0, ctx->stream>>>(to_dev(p), SP, n, nullptr, nullptr, cell,
                                                          (long long)ncells,
                                                          reinterpret_cast<unsigned int*>(N_cell),
                                                          nullptr);
    return cuda_check(ctx, cudaGetLastError(), "k_plan (cells)");
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

}  // extern "C"
static qed_status run_step_graph(qed_ctx* ctx, const DevParticles& D, StepParams SP,
                                 const Scratch& S, uint32_t step);
// Per-cell counts (reading of Algorithms 1 and 2: one sub-step per cell) over
// the rows in use, before the step changes them: N_cell[c] = the largest
// count of cell c's rows (k_plan), then the step's parameters point at them.
static qed_status cell_counts(qed_ctx* ctx, const DevParticles& D, StepParams* SP,
                              const uint32_t* cell, int64_t ncells) {
    if (ncells > ctx->ncell_cap) {
        if (ctx->d_Ncell) cudaFree(ctx->d_Ncell);
        ctx->d_Ncell = nullptr;
        ctx->ncell_cap = 0;
        QED_CUDA(ctx, cudaMalloc(&ctx->d_Ncell, sizeof(unsigned int) * (size_t)ncells));
        ctx->ncell_cap = ncells;
    }
    QED_CUDA(ctx, cudaMemsetAsync(ctx->d_Ncell, 0, sizeof(unsigned int) * (size_t)ncells,
                                  ctx->stream));
    long long blocks = (D.capacity + kColdThreads - 1) / kColdThreads;
    if (blocks > ctx->plan_blocks) blocks = ctx->plan_blocks;
    {
        LaunchScope ls(ctx, QED_KERNEL_PLAN);
        k_plan<<<(int)blocks, kColdThreads, 0, ctx->stream>>>(D, *SP, D.capacity, nullptr,
                                                              nullptr, cell, (long long)ncells,
                                                              ctx->d_Ncell, D.count);
    }
    QED_CUDA(ctx, cudaGetLastError());
    SP->cell = cell;
    SP->N_cell = ctx->d_Ncell;
    SP->ncells = ncells;
    return QED_OK;
}

// The event step, with per-cell first-plan counts when cell != NULL.
static qed_status plain_step(qed_ctx* ctx, const qed_particles* p, uint64_t step_index,
                             qed_step_stats* out, const uint32_t* cell, int64_t ncells) {
    qed_status st = ensure_scratch(ctx, p->capacity);
    if (st != QED_OK) return st;
    StepParams SP = make_params(ctx->cfg, step_index);
    SP.hot_min = ctx->hot_min;
    SP.long_min = ctx->long_min;
    SP.wait_ns = ctx->wait_ns;
    st = sampler_params(ctx, &SP);
    if (st != QED_OK) return st;
    if (cell && SP.sampler)
        return set_err(ctx, QED_ERR_ARG,
                       "qed_event_step_cells: per-cell counts do not combine with the sampler");
    const DevParticles D = to_dev(p);
    Scratch S = make_scratch(ctx);
    st = ensure_samp(ctx, p->capacity, SP, &S);
    if (st != QED_OK) return st;
    if (cell && ncells > 0) {
        st = cell_counts(ctx, D, &SP, cell, ncells);
        if (st != QED_OK) return st;
    }
    const bool cascade = cascade_enabled(ctx->cfg);
    if (cascade && !ctx->prof_on) {
        // the generations run in a device-side loop: no host round trip per
        // generation (per-kernel timing needs the host loop below)
        st = run_step_graph(ctx, D, SP, S, (uint32_t)step_index);
        if (st != QED_OK) return st;
        if (out) return qed_read_stats(ctx, out);
        return QED_OK;
    }
    {
        LaunchScope ls(ctx, QED_KERNEL_CONTROL);
        k_step_init<<<1, 1, 0, ctx->stream>>>(ctx->d_ctl, D.count, D.capacity, 0);
    }
    for (int pass = 0; pass < ctx->cfg.max_passes; ++pass) {
        {
            LaunchScope ls(ctx, QED_KERNEL_COLD);
            if (SP.N_cell) k_cold<true><<<ctx->cold_blocks, kColdThreads, 0, ctx->stream>>>(D, SP, S, ctx->d_ctl);
            else k_cold<false><<<ctx->cold_blocks, kColdThreads, 0, ctx->stream>>>(D, SP, S, ctx->d_ctl);
        }
        if (SP.sampler == 2) {
            LaunchScope ls(ctx, QED_KERNEL_SAMPLER);
            k_samp<<<ctx->samp_blocks, kLaneThreads, kMmaSmemBytes, ctx->stream>>>(
                D, SP, S, ctx->d_ctl);
        }
        {
            LaunchScope ls(ctx, QED_KERNEL_HOT);
            DevParticles d = D;
            StepParams sp = SP;
            Scratch sc = S;
            DevCtl* c = ctx->d_ctl;
            void* a[] = {&d, &sp, &sc, &c};
            const int hm = loop_hot_mode(SP);
            QED_CUDA(ctx, cudaLaunchKernel(hot_kernel(hm, SP.N_cell != nullptr),
                                           dim3(hm ? ctx->net_blocks : ctx->hot_blocks),
                                           dim3(kLaneThreads), a, hm ? kNetSmemBytes : 0,
                                           ctx->stream));
        }
        {
            LaunchScope ls(ctx, QED_KERNEL_CONTROL);
            k_advance<<<1, 1, 0, ctx->stream>>>(ctx->d_ctl, D.count, D.capacity, cascade ? 1 : 0,
                                                ctx->cfg.max_passes, tail_rows_for(ctx, SP), 0ull,
                                                0);
        }
        QED_CUDA(ctx, cudaGetLastError());
        if (!cascade) break;
        QED_CUDA(ctx, cudaMemcpyAsync(ctx->h_ctl, ctx->d_ctl, sizeof(DevCtl),
                                      cudaMemcpyDeviceToHost, ctx->stream));
        QED_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (!ctx->h_ctl->more) break;
    }
    // the tail pass (its kernels do nothing when the generations ran to the end);
    // there the sampler's particles go to the warp mode
    S.samp = nullptr;
    {
        LaunchScope ls(ctx, QED_KERNEL_CONTROL);
        k_tail_begin<<<ctx->sms * 8, 256, 0, ctx->stream>>>(D, S, ctx->d_ctl);
    }
    {
        LaunchScope ls(ctx, QED_KERNEL_COLD);
        if (SP.N_cell) k_cold<true><<<ctx->cold_blocks, kColdThreads, 0, ctx->stream>>>(D, SP, S, ctx->d_ctl);
        else k_cold<false><<<ctx->cold_blocks, kColdThreads, 0, ctx->stream>>>(D, SP, S, ctx->d_ctl);
    }
    {
        LaunchScope ls(ctx, QED_KERNEL_HOT);
        DevParticles d = D;
        StepParams sp = SP;
        Scratch sc = S;
        DevCtl* c = ctx->d_ctl;
        void* a[] = {&d, &sp, &sc, &c};
        QED_CUDA(ctx, cudaLaunchKernel(step_kernel(SP.sampler, SP.N_cell != nullptr),
                                       dim3(SP.sampler ? ctx->step_net_blocks : ctx->step_blocks),
                                       dim3(kLaneThreads), a,
                                       SP.sampler ? kNetSmemBytes : 0, ctx->stream));
    }
    {
        LaunchScope ls(ctx, QED_KERNEL_CONTROL);
        k_tail_end<<<ctx->sms * 8, 256, 0, ctx->stream>>>(D, S, ctx->d_ctl);
    }
    QED_CUDA(ctx, cudaGetLastError());
    if (out) return qed_read_stats(ctx, out);
    return QED_OK;
}

extern "C" {

qed_status qed_event_step(qed_ctx* ctx, const qed_particles* p, uint64_t step_index,
                          qed_step_stats* out) {
    if (!ctx) return QED_ERR_ARG;
    if (!particles_ok(p) || step_index > 0xffffffffull)
        return set_err(ctx, QED_ERR_ARG, "qed_event_step: bad argument");
    return plain_step(ctx, p, step_index, out, nullptr, 0);
}

qed_status qed_event_step_cells(qed_ctx* ctx, const qed_particles* p, uint64_t step_index,
                                const uint32_t* cell, int64_t ncells, qed_step_stats* out) {
    if (!ctx) return QED_ERR_ARG;
    if (!particles_ok(p) || step_index > 0xffffffffull || !cell || ncells <= 0 ||
        ncells > 0xffffffffll)
        return set_err(ctx, QED_ERR_ARG, "qed_event_step_cells: bad argument");
    return plain_step(ctx, p, step_index, out, cell, ncells);
}

}  // extern "C"
static qed_status push_step(qed_ctx* ctx, const qed_particles* p, uint64_t step_index,
                            qed_step_stats* out, const uint32_t* cell, int64_t ncells) {
    qed_status st = ensure_scratch(ctx, p->capacity);
    if (st != QED_OK) return st;
    StepParams SP = make_params(ctx->cfg, step_index);   // the sampler is not used
    SP.wait_ns = ctx->wait_ns;
    const DevParticles D = to_dev(p);
    const Scratch S = make_scratch(ctx);
    const bool cascade = cascade_enabled(ctx->cfg);
    if (cell && ncells > 0) {
        st = cell_counts(ctx, D, &SP, cell, ncells);
        if (st != QED_OK) return st;
    }
    {
        LaunchScope ls(ctx, QED_KERNEL_CONTROL);
        k_step_init<<<1, 1, 0, ctx->stream>>>(ctx->d_ctl, D.count, D.capacity, 0);
    }
    if (cascade && ctx->tail_rows > 0) {
        // the whole step as one persistent pass: children are taken as they
        // are appended (no generation waits for the one before)
        {
            LaunchScope ls(ctx, QED_KERNEL_CONTROL);
            k_push_begin<<<ctx->sms * 8, 256, 0, ctx->stream>>>(D, ctx->d_ctl);
        }
        {
            LaunchScope ls(ctx, QED_KERNEL_HOT);
            k_push<true><<<ctx->push_blocks, kLaneThreads, 0, ctx->stream>>>(D, SP, S, ctx->d_ctl);
        }
        {
            LaunchScope ls(ctx, QED_KERNEL_CONTROL);
            k_tail_end<<<ctx->sms * 8, 256, 0, ctx->stream>>>(D, S, ctx->d_ctl);
        }
        QED_CUDA(ctx, cudaGetLastError());
        if (out) return qed_read_stats(ctx, out);
        return QED_OK;
    }
    for (int pass = 0; pass < ctx->cfg.max_passes; ++pass) {
        QED_CUDA(ctx, cudaMemsetAsync(&ctx->d_ctl->push_head, 0, sizeof(unsigned long long),
                                      ctx->stream));
        {
            LaunchScope ls(ctx, QED_KERNEL_HOT);
            k_push<false><<<ctx->push_blocks, kLaneThreads, 0, ctx->stream>>>(D, SP, S, ctx->d_ctl);
        }
        {
            LaunchScope ls(ctx, QED_KERNEL_CONTROL);
            // generation by generation (tail_rows 0, or no cascade)
            k_advance<<<1, 1, 0, ctx->stream>>>(ctx->d_ctl, D.count, D.capacity, cascade ? 1 : 0,
                                                ctx->cfg.max_passes, 0ll, 0ull, 0);
        }
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
extern "C" {

qed_status qed_event_step_push(qed_ctx* ctx, const qed_particles* p, uint64_t step_index,
                               qed_step_stats* out) {
    if (!ctx) return QED_ERR_ARG;
    if (!particles_ok(p) || step_index > 0xffffffffull)
        return set_err(ctx, QED_ERR_ARG, "qed_event_step_push: bad argument");
    return push_step(ctx, p, step_index, out, nullptr, 0);
}

qed_status qed_event_step_push_cells(qed_ctx* ctx, const qed_particles* p, uint64_t step_index,
                                     const uint32_t* cell, int64_t ncells, qed_step_stats* out) {
    if (!ctx) return QED_ERR_ARG;
    if (!particles_ok(p) || step_index > 0xffffffffull || !cell || ncells <= 0 ||
        ncells > 0xffffffffll)
        return set_err(ctx, QED_ERR_ARG, "qed_event_step_push_cells: bad argument");
    return push_step(ctx, p, step_index, out, cell, ncells);
}

}  // extern "C"
__global__ void k_set_count(long long* count, long long n) { *count = n; }
extern "C" {

// The store in host memory: its rows go to a device copy owned by the
// context (SoA, capacity rows: ten float arrays, the ids, the types, the
// count), the step runs there, and what the step changed comes back.
qed_status qed_event_step_host(qed_ctx* ctx, qed_host_particles* h, uint64_t step_index,
                               qed_step_stats* out) {
    if (!ctx) return QED_ERR_ARG;
    if (!h || !h->px || !h->py || !h->pz || !h->Ex || !h->Ey || !h->Ez || !h->Bx || !h->By ||
        !h->Bz || !h->w || !h->id || !h->type || h->capacity <= 0 || h->capacity >= (1ll << 32) ||
        h->count < 0 || h->count > h->capacity || step_index > 0xffffffffull)
        return set_err(ctx, QED_ERR_ARG, "qed_event_step_host: bad argument");
    const long long cap = h->capacity, n = h->count;
    const size_t f4 = sizeof(float) * (size_t)cap;
    const size_t id_off = 10 * f4, type_off = id_off + sizeof(uint64_t) * (size_t)cap;
    const size_t count_off = (type_off + (size_t)cap + 15) / 16 * 16;
    if (ctx->hstore_cap != cap) {
        if (ctx->d_hstore) cudaFree(ctx->d_hstore);
        ctx->d_hstore = nullptr;
        ctx->hstore_cap = 0;
        QED_CUDA(ctx, cudaMalloc(&ctx->d_hstore, count_off + sizeof(long long)));
        ctx->hstore_cap = cap;
    }
    unsigned char* base = ctx->d_hstore;
    float* dev_f[10];
    for (int k = 0; k < 10; ++k) dev_f[k] = reinterpret_cast<float*>(base + (size_t)k * f4);
    float* host_f[10] = {h->px, h->py, h->pz, h->Ex, h->Ey, h->Ez, h->Bx, h->By, h->Bz, h->w};
    qed_particles d;
    d.px = dev_f[0]; d.py = dev_f[1]; d.pz = dev_f[2];
    d.Ex = dev_f[3]; d.Ey = dev_f[4]; d.Ez = dev_f[5];
    d.Bx = dev_f[6]; d.By = dev_f[7]; d.Bz = dev_f[8];
    d.w = dev_f[9];
    d.id = reinterpret_cast<uint64_t*>(base + id_off);
    d.type = base + type_off;
    d.count = reinterpret_cast<int64_t*>(base + count_off);
    d.capacity = cap;
    cudaStream_t s = ctx->stream;
    const auto h2d = [&](void* dst, const void* src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
    };
    for (int k = 0; k < 10; ++k) QED_CUDA(ctx, h2d(dev_f[k], host_f[k], sizeof(float) * (size_t)n));
    QED_CUDA(ctx, h2d(d.id, h->id, sizeof(uint64_t) * (size_t)n));
    QED_CUDA(ctx, h2d(d.type, h->type, (size_t)n));
    QED_CUDA(ctx, cudaMemsetAsync(d.type + n, QED_REMOVED, (size_t)(cap - n), s));
    k_set_count<<<1, 1, 0, s>>>(reinterpret_cast<long long*>(d.count), n);
    QED_CUDA(ctx, cudaGetLastError());
    qed_step_stats st{};
    const qed_status r = qed_event_step(ctx, &d, step_index, &st);
    if (out) *out = st;
    if (r != QED_OK) return r;   // the host store is left as it was
    const long long m = st.count;
    const auto d2h = [&](void* dst, const void* src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s) : cudaSuccess;
    };
    // the step changes momenta and types of the rows it was given, and
    // writes every field of the rows it appends
    for (int k = 0; k < 10; ++k) {
        const long long lo = k < 3 ? 0 : n;
        QED_CUDA(ctx, d2h(host_f[k] + lo, dev_f[k] + lo, sizeof(float) * (size_t)(m - lo)));
    }
    QED_CUDA(ctx, d2h(h->id + n, d.id + n, sizeof(uint64_t) * (size_t)(m - n)));
    QED_CUDA(ctx, d2h(h->type, d.type, (size_t)m));
    QED_CUDA(ctx, cudaStreamSynchronize(s));
    h->count = m;
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

// Launch the compaction kernels (and the photon drain) on the context stream.
static qed_status launch_compaction(qed_ctx* ctx, const DevParticles& D, const StepParams& SP) {
    const long long nb = (D.capacity + kTile - 1) / kTile;
    if (nb > (1ll << 31) - 1) return set_err(ctx, QED_ERR_ARG, "capacity too large");
    {
        LaunchScope ls(ctx, QED_KERNEL_CONTROL);
        k_compact_count<<<(int)nb, kCompactThreads, 0, ctx->stream>>>(
            D, SP, ctx->cfg.drain_chi, ctx->d_hist, ctx->d_block_live);
        k_compact_scan<<<1, kCompactThreads, 0, ctx->stream>>>(ctx->d_block_live, (int)nb,
                                                               ctx->d_ctl, D.count);
        k_compact_scatter<<<(int)nb, kCompactThreads, 0, ctx->stream>>>(D, ctx->mirror,
                                                                        ctx->d_block_live, ctx->d_ctl);
        k_compact_copyback<<<ctx->sms * 8, 256, 0, ctx->stream>>>(D, ctx->mirror, ctx->d_ctl);
        k_compact_finish<<<1, 1, 0, ctx->stream>>>(D, ctx->d_ctl);
    }
    return cuda_check(ctx, cudaGetLastError(), "compaction");
}

qed_status qed_compact(qed_ctx* ctx, const qed_particles* p, int64_t* removed) {
    if (!ctx) return QED_ERR_ARG;
    if (!particles_ok(p)) return set_err(ctx, QED_ERR_ARG, "qed_compact: bad argument");
    qed_status st = ensure_mirror(ctx, p->capacity);
    if (st != QED_OK) return st;
    const DevParticles D = to_dev(p);
    const StepParams SP = make_params(ctx->cfg, 0);
    long long before = 0;
    if (removed) {
        QED_CUDA(ctx, cudaMemcpyAsync(&before, p->count, sizeof before, cudaMemcpyDeviceToHost,
                                      ctx->stream));
    }
    st = launch_compaction(ctx, D, SP);
    if (st != QED_OK) return st;
    if (removed) {
        long long after = 0;
        QED_CUDA(ctx, cudaMemcpyAsync(&after, p->count, sizeof after, cudaMemcpyDeviceToHost,
                                      ctx->stream));
        QED_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        *removed = before - after;
    }
    return QED_OK;
}

qed_status qed_read_spectrum(qed_ctx* ctx, double* out, int nbins, int reset) {
    if (!ctx || !out || nbins != QED_SPECTRUM_BINS) return QED_ERR_ARG;
    if (!ctx->d_hist) {
        for (int i = 0; i < nbins; ++i) out[i] = 0.0;
        return QED_OK;
    }
    QED_CUDA(ctx, cudaMemcpyAsync(out, ctx->d_hist, sizeof(double) * nbins,
                                  cudaMemcpyDeviceToHost, ctx->stream));
    if (reset)
        QED_CUDA(ctx, cudaMemsetAsync(ctx->d_hist, 0, sizeof(double) * nbins, ctx->stream));
    QED_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return QED_OK;
}

namespace {

// Append a kernel node with `args` to graph g after `deps`.
qed_status add_kernel(qed_ctx* ctx, cudaGraph_t g, cudaGraphNode_t* node, const void* func,
                      dim3 grid, dim3 block, void** args, const cudaGraphNode_t* deps, int ndeps,
                      size_t smem = 0) {
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof kp);
    kp.func = const_cast<void*>(func);
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = (unsigned int)smem;
    kp.kernelParams = args;
    kp.extra = nullptr;
    return cuda_check(ctx, cudaGraphAddKernelNode(node, g, deps, (size_t)ndeps, &kp),
                      "cudaGraphAddKernelNode");
}

// The tail pass after a step's generation loop (node `dep`): tail begin,
// thread pass, persistent kernel, tail end (`last`).  Its kernels do nothing
// when the generations ran to the end.
qed_status add_tail_nodes(qed_ctx* ctx, cudaGraph_t g, cudaGraphNode_t dep, const DevParticles& Din,
                          const StepParams& SPin, const Scratch& Sin, DevCtl* ctl_in,
                          cudaGraphNode_t* last) {
    DevParticles D = Din;
    StepParams SP = SPin;
    Scratch S = Sin;
    S.samp = nullptr;   // in the tail pass the sampler's particles go to the warp mode
    DevCtl* ctl = ctl_in;
    cudaGraphNode_t tb, tc, ts, te;
    qed_status st;
    {
        void* a[] = {&D, &S, &ctl};
        st = add_kernel(ctx, g, &tb, (const void*)k_tail_begin, dim3(ctx->sms * 8), dim3(256), a,
                        &dep, 1);
    }
    if (st == QED_OK) {
        void* a[] = {&D, &SP, &S, &ctl};
        st = add_kernel(ctx, g, &tc, cold_kernel(SP.N_cell != nullptr), dim3(ctx->cold_blocks),
                        dim3(kColdThreads), a, &tb, 1);
    }
    if (st == QED_OK) {
        void* a[] = {&D, &SP, &S, &ctl};
        st = add_kernel(ctx, g, &ts, step_kernel(SP.sampler, SP.N_cell != nullptr),
                        dim3(SP.sampler ? ctx->step_net_blocks : ctx->step_blocks),
                        dim3(kLaneThreads), a, &tc, 1, SP.sampler ? kNetSmemBytes : 0);
    }
    if (st == QED_OK) {
        void* a[] = {&D, &S, &ctl};
        st = add_kernel(ctx, g, &te, (const void*)k_tail_end, dim3(ctx->sms * 8), dim3(256), a,
                        &ts, 1);
    }
    *last = te;
    return st;
}

}  // namespace

qed_status qed_graph_capture(qed_ctx* ctx, const qed_particles* p, uint64_t first_step,
                             int nsteps) {
    if (!ctx) return QED_ERR_ARG;
    if (!particles_ok(p) || nsteps <= 0 || first_step + (uint64_t)nsteps > 0x100000000ull)
        return set_err(ctx, QED_ERR_ARG, "qed_graph_capture: bad argument");
    free_graph(ctx);
    qed_status st = ensure_scratch(ctx, p->capacity);
    if (st == QED_OK) st = ensure_mirror(ctx, p->capacity);
    if (st != QED_OK) return st;
    QED_CUDA(ctx, cudaMalloc(&ctx->d_records, sizeof(qed_step_stats) * nsteps));
    QED_CUDA(ctx, cudaMalloc(&ctx->d_step_base, sizeof(uint32_t)));
    {
        const uint32_t base = (uint32_t)first_step;
        QED_CUDA(ctx, cudaMemcpyAsync(ctx->d_step_base, &base, sizeof base, cudaMemcpyHostToDevice,
                                      ctx->stream));
        QED_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    uint32_t* step_base = ctx->d_step_base;
    QED_CUDA(ctx, cudaMemsetAsync(ctx->d_records, 0, sizeof(qed_step_stats) * nsteps, ctx->stream));
    QED_CUDA(ctx, cudaGraphCreate(&ctx->graph, 0));
    cudaGraph_t g = ctx->graph;
    DevParticles D = to_dev(p);
    Scratch S = make_scratch(ctx);
    {
        StepParams SP0 = make_params(ctx->cfg, 0);
        st = sampler_params(ctx, &SP0);
        if (st == QED_OK) st = ensure_samp(ctx, p->capacity, SP0, &S);
        if (st != QED_OK) {
            free_graph(ctx);
            return st;
        }
    }
    DevCtl* ctl = ctx->d_ctl;
    long long* count = D.count;
    long long capacity = D.capacity;
    int more_allowed = cascade_enabled(ctx->cfg) ? 1 : 0;
    int max_passes = ctx->cfg.max_passes;
    long long tail_rows = ctx->tail_rows;
    int keep_sticky = 1;
    float drain = ctx->cfg.drain_chi;
    double* hist = ctx->d_hist;
    Mirror M = ctx->mirror;
    unsigned int* block_live = ctx->d_block_live;
    const long long nbl = (capacity + kTile - 1) / kTile;
    int nb = (int)nbl;

    cudaGraphNode_t prev;
    {
        void* a[] = {&ctl};
        st = add_kernel(ctx, g, &prev, (const void*)k_graph_begin, dim3(1), dim3(1), a, nullptr, 0);
        if (st != QED_OK) return st;
    }
    for (int k = 0; k < nsteps && st == QED_OK; ++k) {
        StepParams SP = make_params(ctx->cfg, (uint64_t)k);   // offset from the device base
        SP.step_base = step_base;
        SP.hot_min = ctx->hot_min;
        SP.long_min = ctx->long_min;
        SP.wait_ns = ctx->wait_ns;
        st = sampler_params(ctx, &SP);
        if (st != QED_OK) break;
        qed_step_stats* rec = ctx->d_records + k;
        cudaGraphNode_t init, wnode, n1, n2, n3, n4, n5, close;
        {
            void* a[] = {&ctl, &count, &capacity, &keep_sticky};
            st = add_kernel(ctx, g, &init, (const void*)k_step_init, dim3(1), dim3(1), a, &prev, 1);
        }
        // WHILE node: one cascade generation per iteration
        cudaGraphConditionalHandle h;
        if (st == QED_OK)
            st = cuda_check(ctx, cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault),
                            "cudaGraphConditionalHandleCreate");
        if (st != QED_OK) break;
        cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
        memset(&cp.conditional, 0, sizeof cp.conditional);
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        st = cuda_check(ctx, cudaGraphAddNode(&wnode, g, &init, nullptr, 1, &cp), "cudaGraphAddNode");
        if (st != QED_OK) break;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaGraphNode_t bc, bs, bh, ba;
        int use_handle = 1;
        {
            void* a[] = {&D, &SP, &S, &ctl};
            st = add_kernel(ctx, body, &bc, cold_kernel(SP.N_cell != nullptr), dim3(ctx->cold_blocks),
                            dim3(kColdThreads), a, nullptr, 0);
        }
        bs = bc;
        if (st == QED_OK && SP.sampler == 2) {
            void* a[] = {&D, &SP, &S, &ctl};
            st = add_kernel(ctx, body, &bs, (const void*)k_samp, dim3(ctx->samp_blocks),
                            dim3(kLaneThreads), a, &bc, 1, kMmaSmemBytes);
        }
        if (st == QED_OK) {
            void* a[] = {&D, &SP, &S, &ctl};
            const int hm = loop_hot_mode(SP);
            st = add_kernel(ctx, body, &bh, hot_kernel(hm, SP.N_cell != nullptr),
                            dim3(hm ? ctx->net_blocks : ctx->hot_blocks), dim3(kLaneThreads), a,
                            &bs, 1, hm ? kNetSmemBytes : 0);
        }
        if (st == QED_OK) {
            void* a[] = {&ctl,        &count, &capacity, &more_allowed, &max_passes,
                         &tail_rows, &h,     &use_handle};
            st = add_kernel(ctx, body, &ba, (const void*)k_advance, dim3(1), dim3(1), a, &bh, 1);
        }
        cudaGraphNode_t tend;
        if (st == QED_OK) st = add_tail_nodes(ctx, g, wnode, D, SP, S, ctl, &tend);
        // compaction (and optional photon drain) after the cascade
        if (st == QED_OK) {
            void* a[] = {&D, &SP, &drain, &hist, &block_live};
            st = add_kernel(ctx, g, &n1, (const void*)k_compact_count, dim3(nb),
                            dim3(kCompactThreads), a, &tend, 1);
        }
        if (st == QED_OK) {
            void* a[] = {&block_live, &nb, &ctl, &count};
            st = add_kernel(ctx, g, &n2, (const void*)k_compact_scan, dim3(1), dim3(kCompactThreads),
                            a, &n1, 1);
        }
        if (st == QED_OK) {
            void* a[] = {&D, &M, &block_live, &ctl};
            st = add_kernel(ctx, g, &n3, (const void*)k_compact_scatter, dim3(nb),
                            dim3(kCompactThreads), a, &n2, 1);
        }
        if (st == QED_OK) {
            void* a[] = {&D, &M, &ctl};
            st = add_kernel(ctx, g, &n4, (const void*)k_compact_copyback, dim3(ctx->sms * 8),
                            dim3(256), a, &n3, 1);
        }
        if (st == QED_OK) {
            void* a[] = {&D, &ctl};
            st = add_kernel(ctx, g, &n5, (const void*)k_compact_finish, dim3(1), dim3(1), a, &n4, 1);
        }
        uint32_t advance = (k == nsteps - 1) ? (uint32_t)nsteps : 0u;
        if (st == QED_OK) {
            void* a[] = {&ctl, &count, &rec, &step_base, &advance};
            st = add_kernel(ctx, g, &close, (const void*)k_step_close, dim3(1), dim3(1), a, &n5, 1);
        }
        prev = close;
    }
    if (st == QED_OK)
        st = cuda_check(ctx, cudaGraphInstantiate(&ctx->graph_exec, g, 0), "cudaGraphInstantiate");
    if (st != QED_OK) {
        free_graph(ctx);
        return st;
    }
    ctx->graph_steps = nsteps;
    return QED_OK;
}

qed_status qed_graph_launch(qed_ctx* ctx) {
    if (!ctx) return QED_ERR_ARG;
    if (!ctx->graph_exec) return set_err(ctx, QED_ERR_STATE, "qed_graph_launch: no graph captured");
    ctx->launches[QED_KERNEL_CONTROL] += 1;
    return cuda_check(ctx, cudaGraphLaunch(ctx->graph_exec, ctx->stream), "cudaGraphLaunch");
}

qed_status qed_graph_read_stats(qed_ctx* ctx, qed_step_stats* out, int nsteps) {
    if (!ctx || !out || nsteps <= 0) return QED_ERR_ARG;
    if (!ctx->d_records || nsteps > ctx->graph_steps)
        return set_err(ctx, QED_ERR_STATE, "qed_graph_read_stats: no such steps");
    QED_CUDA(ctx, cudaMemcpyAsync(out, ctx->d_records, sizeof(qed_step_stats) * nsteps,
                                  cudaMemcpyDeviceToHost, ctx->stream));
    QED_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < nsteps; ++k)
        if (out[k].status != 0) return (qed_status)out[k].status;
    return QED_OK;
}

}  // extern "C"

__global__ void k_set_step(uint32_t* p, uint32_t v) { *p = v; }

// Build (when its key changed) and launch the one-step graph: step-init, then
// a conditional WHILE node whose body is one cascade generation (thread
// pass, hot pass, generation control; the control kernel sets the
// condition).  The step index reaches the kernels through a device word
// written by a kernel launched just before the graph.
static qed_status run_step_graph(qed_ctx* ctx, const DevParticles& Din, StepParams SPin,
                                 const Scratch& Sin, uint32_t step) {
    if (!ctx->d_step_idx) QED_CUDA(ctx, cudaMalloc(&ctx->d_step_idx, sizeof(uint32_t)));
    SPin.step = 0;
    SPin.step_base = ctx->d_step_idx;
    uint64_t key[64];
    int nk = 0;
    auto put = [&](uint64_t v) { if (nk < 64) key[nk++] = v; };
    auto putf = [&](float v) { uint32_t b; memcpy(&b, &v, 4); put(b); };
    auto putp = [&](const void* v) { put((uint64_t)(uintptr_t)v); };
    for (const void* q : {(const void*)Din.px, (const void*)Din.py, (const void*)Din.pz,
                          (const void*)Din.Ex, (const void*)Din.Ey, (const void*)Din.Ez,
                          (const void*)Din.Bx, (const void*)Din.By, (const void*)Din.Bz,
                          (const void*)Din.w, (const void*)Din.id, (const void*)Din.type,
                          (const void*)Din.count})
        putp(q);
    put((uint64_t)Din.capacity);
    putp(Sin.t_rem); putp(Sin.hot); put((uint64_t)Sin.hot_cap); putp(Sin.log);
    put((uint64_t)Sin.log_cap); putp(Sin.log_count); putp(Sin.samp);
    put(SPin.seed);
    { uint64_t b; memcpy(&b, &SPin.dt, 8); put(b); }
    putf(SPin.K); putf(SPin.inv_Es); putf(SPin.p_max); putf(SPin.inv_p_max); putf(SPin.pair_coeff);
    putf(SPin.t_step.hi); putf(SPin.t_step.lo);
    put(SPin.hot_min); put(SPin.long_min); put((uint64_t)SPin.sampler); put((uint64_t)SPin.net_rows);
    put(SPin.net_bins); putp(SPin.net_w); putp(SPin.net_wtot); put(SPin.process_mask);
    put(SPin.pnet_bins); putp(SPin.pnet_w); putp(SPin.pnet_wtot);
    put((uint64_t)SPin.recoil); put((uint64_t)SPin.cascade); put(SPin.wait_ns);
    putp(SPin.cell); putp(SPin.N_cell); put((uint64_t)SPin.ncells);
    { uint64_t b; memcpy(&b, &SPin.lambda_m, 8); put(b); }
    put((uint64_t)ctx->cold_blocks); put((uint64_t)ctx->hot_blocks); put((uint64_t)ctx->net_blocks);
    put((uint64_t)ctx->cfg.max_passes);
    put((uint64_t)ctx->tail_rows); put((uint64_t)ctx->step_blocks); put((uint64_t)ctx->step_net_blocks);
    put((uint64_t)ctx->samp_blocks);
    const bool same = ctx->step_exec && nk == ctx->step_key_n &&
                      memcmp(key, ctx->step_key, sizeof(uint64_t) * nk) == 0;
    if (!same) {
        if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
        if (ctx->step_graph) cudaGraphDestroy(ctx->step_graph);
        ctx->step_exec = nullptr;
        ctx->step_graph = nullptr;
        QED_CUDA(ctx, cudaGraphCreate(&ctx->step_graph, 0));
        cudaGraph_t g = ctx->step_graph;
        // node arguments live in this frame until the graph is instantiated
        DevParticles D = Din;
        StepParams SP = SPin;
        Scratch S = Sin;
        DevCtl* ctl = ctx->d_ctl;
        long long* count = D.count;
        long long capacity = D.capacity;
        int keep_sticky = 0, more_allowed = 1, max_passes = ctx->cfg.max_passes, use_handle = 1;
        long long tail_rows = tail_rows_for(ctx, SP);
        cudaGraphNode_t init, wnode, bc, bs, bh, ba, tend;
        qed_status st;
        {
            void* a[] = {&ctl, &count, &capacity, &keep_sticky};
            st = add_kernel(ctx, g, &init, (const void*)k_step_init, dim3(1), dim3(1), a, nullptr, 0);
        }
        cudaGraphConditionalHandle h;
        if (st == QED_OK)
            st = cuda_check(ctx, cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault),
                            "cudaGraphConditionalHandleCreate");
        cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
        if (st == QED_OK) {
            memset(&cp.conditional, 0, sizeof cp.conditional);
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            st = cuda_check(ctx, cudaGraphAddNode(&wnode, g, &init, nullptr, 1, &cp),
                            "cudaGraphAddNode");
        }
        if (st == QED_OK) {
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            void* a[] = {&D, &SP, &S, &ctl};
            st = add_kernel(ctx, body, &bc, cold_kernel(SP.N_cell != nullptr), dim3(ctx->cold_blocks),
                            dim3(kColdThreads), a, nullptr, 0);
            bs = bc;
            if (st == QED_OK && SP.sampler == 2)
                st = add_kernel(ctx, body, &bs, (const void*)k_samp, dim3(ctx->samp_blocks),
                                dim3(kLaneThreads), a, &bc, 1, kMmaSmemBytes);
            const int hm = loop_hot_mode(SP);
            if (st == QED_OK)
                st = add_kernel(ctx, body, &bh, hot_kernel(hm, SP.N_cell != nullptr),
                                dim3(hm ? ctx->net_blocks : ctx->hot_blocks), dim3(kLaneThreads),
                                a, &bs, 1, hm ? kNetSmemBytes : 0);
            if (st == QED_OK) {
                void* b[] = {&ctl,        &count, &capacity, &more_allowed, &max_passes,
                             &tail_rows, &h,     &use_handle};
                st = add_kernel(ctx, body, &ba, (const void*)k_advance, dim3(1), dim3(1), b, &bh, 1);
            }
        }
        if (st == QED_OK) st = add_tail_nodes(ctx, g, wnode, D, SP, S, ctl, &tend);
        if (st == QED_OK)
            st = cuda_check(ctx, cudaGraphInstantiate(&ctx->step_exec, g, 0), "cudaGraphInstantiate");
        if (st != QED_OK) {
            if (ctx->step_graph) cudaGraphDestroy(ctx->step_graph);
            ctx->step_graph = nullptr;
            ctx->step_exec = nullptr;
            return st;
        }
        memcpy(ctx->step_key, key, sizeof(uint64_t) * nk);
        ctx->step_key_n = nk;
    }
    k_set_step<<<1, 1, 0, ctx->stream>>>(ctx->d_step_idx, step);
    QED_CUDA(ctx, cudaGetLastError());
    ctx->launches[QED_KERNEL_CONTROL] += 1;
    return cuda_check(ctx, cudaGraphLaunch(ctx->step_exec, ctx->stream), "cudaGraphLaunch");
}

// ---------------------------------------------------------------------------
// Learned sampler
// ---------------------------------------------------------------------------
namespace {

constexpr int kCdfRows = 1024;      // rows of the exact CDF along log10 chi in [-2, 2]
constexpr float kPairLog10Lo = -0.60206f;   // log10 0.25: lower end of the pair network's training
constexpr int kCdfM = 4096;         // x intervals per row
constexpr int kEvalSub = 4;         // evaluation rows per error bin
constexpr int kEvalU = 1024;        // evaluation points in u per row

// The network the qed_sampler_* calls address (qed_sampler_process).
NetState& cur_net(qed_ctx* ctx) { return ctx->nets[ctx->net_sel]; }

qed_status sampler_alloc(qed_ctx* ctx, int max_batch) {
    if (!cur_net(ctx).d_theta) {
        QED_CUDA(ctx, cudaMalloc(&cur_net(ctx).d_theta, sizeof(float) * kMlpParams));
        QED_CUDA(ctx, cudaMalloc(&cur_net(ctx).d_m1, sizeof(float) * kMlpParams));
        QED_CUDA(ctx, cudaMalloc(&cur_net(ctx).d_m2, sizeof(float) * kMlpParams));
        QED_CUDA(ctx, cudaMalloc(&cur_net(ctx).d_wbf, sizeof(__nv_bfloat16) * kMlpParams));
        QED_CUDA(ctx, cudaMalloc(&ctx->d_partial, sizeof(float) * kMlpParams * ctx->sms * 2));
        QED_CUDA(ctx, cudaMalloc(&ctx->d_loss, sizeof(float)));
        QED_CUDA(ctx, cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sizeof(TrainSmem)));
    }
    if (!cur_net(ctx).d_cdf) {
        QED_CUDA(ctx, cudaMalloc(&cur_net(ctx).d_cdf, sizeof(float) * kCdfRows * (kCdfM + 1)));
        QED_CUDA(ctx, cudaMalloc(&cur_net(ctx).d_wtot, sizeof(float) * kCdfRows));
        k_cdf_rows<<<kCdfRows, 256, 0, ctx->stream>>>(kMlpLog10Lo, kMlpLog10Hi, kCdfRows, kCdfM,
                                                      ctx->net_sel, cur_net(ctx).d_cdf,
                                                      cur_net(ctx).d_wtot);
        QED_CUDA(ctx, cudaGetLastError());
    }
    if (max_batch > 0 && ctx->d_batch && ctx->batch_cap < max_batch) {
        cudaFree(ctx->d_batch);
        ctx->d_batch = nullptr;
    }
    if (max_batch > 0 && !ctx->d_batch) {
        QED_CUDA(ctx, cudaMalloc(&ctx->d_batch, sizeof(float) * 4 * (size_t)max_batch));
        ctx->batch_cap = max_batch;
    }
    return QED_OK;
}

qed_status sampler_params(qed_ctx* ctx, StepParams* SP) {
    if (!ctx->cfg.sampler_mode) return QED_OK;
    const NetState& E = ctx->nets[0];
    if (!E.net_ready || !E.d_wtot)
        return set_err(ctx, QED_ERR_STATE, "sampler_mode set but no sampler trained or loaded");
    SP->sampler = ctx->cfg.sampler_mode;   // 1: per sub-step, 2: event-driven
    SP->net_rows = kCdfRows;
    SP->net_bins = E.net_bins;
    SP->net_w = E.d_wbf;
    SP->net_wtot = E.d_wtot;
    // the pair sampler (event-driven mode only), once trained and evaluated
    const NetState& Q = ctx->nets[1];
    if (SP->sampler == 2 && Q.net_ready && Q.d_wtot && Q.net_bins) {
        SP->pnet_bins = Q.net_bins;
        SP->pnet_w = Q.d_wbf;
        SP->pnet_wtot = Q.d_wtot;
    }
    return QED_OK;
}

// Deterministic initial parameters: uniform(+-1/sqrt(fan_in)) from Philox on
// the host (the same recipe for every run with the same seed).
void sampler_init_host(uint64_t seed, float* th) {
    uint64_t state = seed * 0x9E3779B97F4A7C15ull + 1;
    auto next = [&state]() {
        state ^= state << 13;
        state ^= state >> 7;
        state ^= state << 17;
        return (double)(state >> 11) * 0x1p-53;
    };
    for (int i = 0; i < kMlpParams; ++i) {
        double fan = (i < kMlpOffB1 || i < kMlpOffW2) ? 2.0 : 64.0;
        const double lim = 1.0 / sqrt(fan);
        th[i] = (float)((2.0 * next() - 1.0) * lim);
    }
}

}  // namespace

// Per-thread evaluation form of the network (same operation order as the
// warp form, including the butterfly order of the output sum of lane 0).
__device__ float mlp_infer_thread(const SamplerSmem& S, float v0, float v1) {
    float h1[kMlpW], h2[kMlpW];
    for (int n = 0; n < kMlpW; ++n)
        h1[n] = siluf_(fmaf(S.W1[2 * n], v0, fmaf(S.W1[2 * n + 1], v1, S.b1[n])));
    for (int n = 0; n < kMlpW; ++n) h2[n] = siluf_(neuron_dot(S.W2 + n * kWPad, h1, S.b2[n]));
    float part[32];
    for (int l = 0; l < 32; ++l) {
        float o = 0.0f;
        for (int q = 0; q < 2; ++q) {
            const int n = l + 32 * q;
            o = fmaf(S.w4[n], siluf_(neuron_dot(S.W3 + n * kWPad, h2, S.b3[n])), o);
        }
        part[l] = o;
    }
    for (int off = 16; off > 0; off >>= 1) {
        float nxt[32];
        for (int l = 0; l < 32; ++l) nxt[l] = part[l] + part[l ^ off];
        for (int l = 0; l < 32; ++l) part[l] = nxt[l];
    }
    return sigmoidf_(part[0] + S.b4 + anchor_of_v1(v1));
}

// Max |CDF(chi, x_net(chi, u)) - u| per bin over kEvalSub rows per bin and a
// uniform grid of u; rows of `cdf` are the evaluation rows.
__global__ void k_sampler_eval(const __nv_bfloat16* __restrict__ w, const float* __restrict__ cdf,
                               const float* __restrict__ tot, int nrows, int M, float log10_lo,
                               float log10_hi, unsigned int* __restrict__ bin_err_bits) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    SamplerSmem& S = *reinterpret_cast<SamplerSmem*>(dyn_smem);
    stage_sampler(S, w, cdf, 0, 0ull);
    __syncthreads();
    const int row = blockIdx.x;
    if (row >= nrows) return;
    const float l10 = log10_lo + (log10_hi - log10_lo) * ((float)row + 0.5f) / (float)nrows;
    const int bin = min(max((int)((l10 - kMlpLog10Lo) * 16.0f), 0), 63);
    float worst = 0.0f;
    for (int k = threadIdx.x; k < kEvalU; k += blockDim.x) {
        const float u = ((float)k + 0.5f) / (float)kEvalU;
        const float x = mlp_infer_thread(S, l10 * 0.5f, mlp_input_u(u));
        const float c = cdf_row_at(cdf + (size_t)row * (M + 1), M, x);
        worst = fmaxf(worst, fabsf(c - u));
    }
    if (!(tot[row] > 0.0f)) worst = 1.0f;   // no probability to sample
    atomicMax(&bin_err_bits[bin], __float_as_uint(worst));
}

// The same error measurement for the tensor-core form of the network (the
// event-driven sampler's arithmetic): each lane evaluates its own u, the warp
// together.
__global__ void k_sampler_eval_mma(const __nv_bfloat16* __restrict__ w,
                                   const float* __restrict__ cdf, const float* __restrict__ tot,
                                   int nrows, int M, float log10_lo, float log10_hi,
                                   unsigned int* __restrict__ bin_err_bits) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    SamplerMma& S = *reinterpret_cast<SamplerMma*>(dyn_smem);
    stage_sampler_mma(S, w, nullptr, 0, 0ull);
    __syncthreads();
    const int row = blockIdx.x;
    if (row >= nrows) return;
    const float l10 = log10_lo + (log10_hi - log10_lo) * ((float)row + 0.5f) / (float)nrows;
    const int bin = min(max((int)((l10 - kMlpLog10Lo) * 16.0f), 0), 63);
    float worst = 0.0f;
    for (int k0 = 0; k0 < kEvalU; k0 += blockDim.x) {   // uniform trip count (kEvalU % blockDim == 0)
        const int k = k0 + threadIdx.x;
        const float u = ((float)k + 0.5f) / (float)kEvalU;
        const float x = mlp_infer_mma(S, l10 * 0.5f, mlp_input_u(u));
        const float c = cdf_row_at(cdf + (size_t)row * (M + 1), M, x);
        worst = fmaxf(worst, fabsf(c - u));
    }
    if (!(tot[row] > 0.0f)) worst = 1.0f;   // no probability to sample
    atomicMax(&bin_err_bits[bin], __float_as_uint(worst));
}

// x = Q(chi, u) through the tensor-core form of the network; every lane of a
// warp takes part in each round (indices past n compute and drop a value).
__global__ void k_sampler_quantile_mma(const __nv_bfloat16* __restrict__ w,
                                       const float* __restrict__ log10chi,
                                       const float* __restrict__ u, float* __restrict__ x,
                                       long long n) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    SamplerMma& S = *reinterpret_cast<SamplerMma*>(dyn_smem);
    stage_sampler_mma(S, w, nullptr, 0, 0ull);
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b = (long long)blockIdx.x * blockDim.x; b < n; b += stride) {
        const long long i = b + threadIdx.x;
        const bool ok = i < n;
        const float l10 = ok ? fminf(fmaxf(log10chi[i], kMlpLog10Lo), kMlpLog10Hi) : 0.0f;
        const float uu = ok ? u[i] : 0.5f;
        const float xv = mlp_infer_mma(S, l10 * 0.5f, mlp_input_u(uu));
        if (ok) x[i] = xv;
    }
}

// x = Q(chi, u): the exact table inverse (bilinear in log10 chi and the CDF
// node interval) or the network in its per-thread form.
__global__ void k_sampler_quantile(const __nv_bfloat16* __restrict__ w, const float* __restrict__ cdf,
                                   int nrows, int M, const float* __restrict__ log10chi,
                                   const float* __restrict__ u, float* __restrict__ x, long long n,
                                   int use_net) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    SamplerSmem& S = *reinterpret_cast<SamplerSmem*>(dyn_smem);
    if (use_net) stage_sampler(S, w, cdf, 0, 0ull);
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float l10 = fminf(fmaxf(log10chi[i], kMlpLog10Lo), kMlpLog10Hi);
        if (use_net) {
            x[i] = mlp_infer_thread(S, l10 * 0.5f, mlp_input_u(u[i]));
        } else {
            const float pos = (l10 - kMlpLog10Lo) / (kMlpLog10Hi - kMlpLog10Lo) * (float)(nrows - 1);
            const int r = min((int)pos, nrows - 2);
            const float wgt = pos - (float)r;
            const float xa = cdf_row_inverse(cdf + (size_t)r * (M + 1), M, u[i]);
            const float xb = cdf_row_inverse(cdf + (size_t)(r + 1) * (M + 1), M, u[i]);
            x[i] = xa + wgt * (xb - xa);
        }
    }
}

extern "C" {

qed_status qed_sampler_process(qed_ctx* ctx, uint32_t process) {
    if (!ctx || (process != QED_PROC_EMISSION && process != QED_PROC_PAIR))
        return set_err(ctx, QED_ERR_ARG, "qed_sampler_process: bad argument");
    ctx->net_sel = process == QED_PROC_PAIR ? 1 : 0;
    return QED_OK;
}

qed_status qed_sampler_quantile(qed_ctx* ctx, const float* log10chi, const float* u, float* x,
                                int64_t n, int use_net) {
    if (!ctx || n < 0 || (n > 0 && (!log10chi || !u || !x)))
        return set_err(ctx, QED_ERR_ARG, "qed_sampler_quantile: bad argument");
    if (use_net < 0 || use_net > 2) return set_err(ctx, QED_ERR_ARG, "qed_sampler_quantile: use_net");
    if (use_net && !cur_net(ctx).net_ready) return set_err(ctx, QED_ERR_STATE, "no sampler trained or loaded");
    qed_status st = sampler_alloc(ctx, 0);
    if (st != QED_OK || n == 0) return st;
    long long blocks = (n + 127) / 128;
    if (blocks > ctx->sms * 8) blocks = ctx->sms * 8;
    if (use_net == 2) {
        k_sampler_quantile_mma<<<(int)blocks, 128, sizeof(SamplerMma), ctx->stream>>>(
            cur_net(ctx).d_wbf, log10chi, u, x, n);
        return cuda_check(ctx, cudaGetLastError(), "qed_sampler_quantile");
    }
    k_sampler_quantile<<<(int)blocks, 128, use_net ? sizeof(SamplerSmem) : 0, ctx->stream>>>(
        cur_net(ctx).d_wbf, cur_net(ctx).d_cdf, kCdfRows, kCdfM, log10chi, u, x, n, use_net);
    return cuda_check(ctx, cudaGetLastError(), "qed_sampler_quantile");
}

qed_status qed_sampler_train(qed_ctx* ctx, uint64_t seed, int64_t samples, int batch, float lr,
                             float* final_loss) {
    if (!ctx) return QED_ERR_ARG;
    if (samples <= 0 || batch < kTileS || batch > (1 << 20) || !(lr > 0.0f))
        return set_err(ctx, QED_ERR_ARG, "qed_sampler_train: bad argument");
    qed_status st = sampler_alloc(ctx, batch);
    if (st != QED_OK) return st;
    if (!cur_net(ctx).net_ready) {
        float th[kMlpParams];
        sampler_init_host(seed, th);
        QED_CUDA(ctx, cudaMemcpyAsync(cur_net(ctx).d_theta, th, sizeof th, cudaMemcpyHostToDevice,
                                      ctx->stream));
        QED_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    QED_CUDA(ctx, cudaMemsetAsync(cur_net(ctx).d_m1, 0, sizeof(float) * kMlpParams, ctx->stream));
    QED_CUDA(ctx, cudaMemsetAsync(cur_net(ctx).d_m2, 0, sizeof(float) * kMlpParams, ctx->stream));
    const long long steps = (samples + batch - 1) / batch;
    const int ntiles = (batch + kTileS - 1) / kTileS;
    const int grid = std::min(ntiles, ctx->sms * 2);
    float* v = ctx->d_batch;
    float* tgt = ctx->d_batch + 2 * (size_t)batch;
    float* wgt = ctx->d_batch + 3 * (size_t)batch;
    const float b1 = 0.9f, b2 = 0.999f;
    double p1 = 1.0, p2 = 1.0;
    // the pair network learns chi_gamma >= 0.25 only: below, the pair rate
    // is negligible and the spectrum a spike at 1/2 (rejection keeps those)
    const float l10_lo = ctx->net_sel == 1 ? kPairLog10Lo : kMlpLog10Lo;
    for (long long k = 0; k < steps; ++k) {
        k_sampler_batch<<<(batch + 255) / 256, 256, 0, ctx->stream>>>(
            (uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)k, batch, l10_lo, kMlpLog10Hi,
            cur_net(ctx).d_cdf, kCdfRows, kCdfM, v, tgt, wgt);
        const bool last = k + 1 == steps;
        if (last) QED_CUDA(ctx, cudaMemsetAsync(ctx->d_loss, 0, sizeof(float), ctx->stream));
        k_mlp_grad<<<grid, 256, sizeof(TrainSmem), ctx->stream>>>(
            cur_net(ctx).d_theta, v, tgt, wgt, batch, 1, cur_net(ctx).d_cdf, kCdfRows, kCdfM, ctx->d_partial,
            last ? ctx->d_loss : nullptr);
        p1 *= b1;
        p2 *= b2;
        // cosine decay of the step size over the run
        const float lr_k = lr * 0.5f * (1.0f + cosf(3.14159265f * (float)k / (float)steps));
        k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, ctx->stream>>>(
            ctx->d_partial, grid, cur_net(ctx).d_theta, cur_net(ctx).d_m1, cur_net(ctx).d_m2, cur_net(ctx).d_wbf, lr_k, b1, b2,
            1e-8f, (float)(1.0 - p1), (float)(1.0 - p2), 1, nullptr);
        QED_CUDA(ctx, cudaGetLastError());
    }
    cur_net(ctx).adam_t += steps;
    cur_net(ctx).net_ready = 1;
    cur_net(ctx).net_bins = 0;   // evaluate before use
    if (final_loss) {
        QED_CUDA(ctx, cudaMemcpyAsync(final_loss, ctx->d_loss, sizeof(float), cudaMemcpyDeviceToHost,
                                      ctx->stream));
    }
    QED_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return QED_OK;
}

qed_status qed_sampler_evaluate(qed_ctx* ctx, float* bin_err, int nbins) {
    if (!ctx || !bin_err || nbins != QED_SAMPLER_BINS) return QED_ERR_ARG;
    if (!cur_net(ctx).net_ready) return set_err(ctx, QED_ERR_STATE, "no sampler trained or loaded");
    qed_status st = sampler_alloc(ctx, 0);
    if (st != QED_OK) return st;
    const int rows = QED_SAMPLER_BINS * kEvalSub;
    float* cdf = nullptr;
    float* tot = nullptr;
    unsigned int* bits = nullptr;
    QED_CUDA(ctx, cudaMalloc(&cdf, sizeof(float) * (size_t)rows * (kCdfM + 1)));
    QED_CUDA(ctx, cudaMalloc(&tot, sizeof(float) * rows));
    QED_CUDA(ctx, cudaMalloc(&bits, sizeof(unsigned int) * QED_SAMPLER_BINS));
    QED_CUDA(ctx, cudaMemsetAsync(bits, 0, sizeof(unsigned int) * QED_SAMPLER_BINS, ctx->stream));
    // rows at the centres of rows equal sub-intervals of [-2, 2]
    const float half = 0.5f * (kMlpLog10Hi - kMlpLog10Lo) / rows;
    k_cdf_rows<<<rows, 256, 0, ctx->stream>>>(kMlpLog10Lo + half, kMlpLog10Hi - half, rows, kCdfM,
                                              ctx->net_sel, cdf, tot);
    // both forms of the network the event kernels use: a bin's error is the
    // larger of the two
    k_sampler_eval<<<rows, 128, sizeof(SamplerSmem), ctx->stream>>>(
        cur_net(ctx).d_wbf, cdf, tot, rows, kCdfM, kMlpLog10Lo, kMlpLog10Hi, bits);
    k_sampler_eval_mma<<<rows, 128, sizeof(SamplerMma), ctx->stream>>>(
        cur_net(ctx).d_wbf, cdf, tot, rows, kCdfM, kMlpLog10Lo, kMlpLog10Hi, bits);
    unsigned int hb[QED_SAMPLER_BINS];
    st = cuda_check(ctx, cudaMemcpyAsync(hb, bits, sizeof hb, cudaMemcpyDeviceToHost, ctx->stream),
                    "copy bins");
    if (st == QED_OK) st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "evaluate");
    cudaFree(cdf);
    cudaFree(tot);
    cudaFree(bits);
    if (st != QED_OK) return st;
    unsigned long long ok = 0;
    for (int b = 0; b < QED_SAMPLER_BINS; ++b) {
        float e;
        memcpy(&e, &hb[b], sizeof e);
        bin_err[b] = e;
        if (e <= ctx->cfg.sampler_max_err) ok |= 1ull << b;
    }
    cur_net(ctx).net_bins = ok;
    return QED_OK;
}

qed_status qed_sampler_gradient(qed_ctx* ctx, const float* params, const float* v,
                                const float* target, const float* weight, int64_t B, float* grad,
                                float* loss) {
    if (!ctx || !params || !v || !target || !grad || B < 1 || B > (1 << 24))
        return set_err(ctx, QED_ERR_ARG, "qed_sampler_gradient: bad argument");
    qed_status st = sampler_alloc(ctx, 0);
    if (st != QED_OK) return st;
    const int ntiles = (int)((B + kTileS - 1) / kTileS);
    const int grid = std::min(ntiles, ctx->sms * 2);
    if (loss) QED_CUDA(ctx, cudaMemsetAsync(loss, 0, sizeof(float), ctx->stream));
    k_mlp_grad<<<grid, 256, sizeof(TrainSmem), ctx->stream>>>(params, v, target, weight, (int)B,
                                                              0, nullptr, 0, 0, ctx->d_partial,
                                                              loss);
    k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, ctx->stream>>>(
        ctx->d_partial, grid, nullptr, nullptr, nullptr, nullptr, 0.0f, 0.0f, 0.0f, 0.0f, 1.0f,
        1.0f, 0, grad);
    return cuda_check(ctx, cudaGetLastError(), "qed_sampler_gradient");
}

qed_status qed_sampler_load(qed_ctx* ctx, const float* params, int64_t n) {
    if (!ctx || !params || n != kMlpParams) return QED_ERR_ARG;
    qed_status st = sampler_alloc(ctx, 0);
    if (st != QED_OK) return st;
    QED_CUDA(ctx, cudaMemcpyAsync(cur_net(ctx).d_theta, params, sizeof(float) * kMlpParams,
                                  cudaMemcpyHostToDevice, ctx->stream));
    // refresh the BF16 copy with a zero-step Adam pass over a zero gradient
    QED_CUDA(ctx, cudaMemsetAsync(ctx->d_partial, 0, sizeof(float) * kMlpParams, ctx->stream));
    QED_CUDA(ctx, cudaMemsetAsync(cur_net(ctx).d_m1, 0, sizeof(float) * kMlpParams, ctx->stream));
    QED_CUDA(ctx, cudaMemsetAsync(cur_net(ctx).d_m2, 0, sizeof(float) * kMlpParams, ctx->stream));
    k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, ctx->stream>>>(
        ctx->d_partial, 1, cur_net(ctx).d_theta, cur_net(ctx).d_m1, cur_net(ctx).d_m2, cur_net(ctx).d_wbf, 0.0f, 0.9f, 0.999f, 1e-8f,
        1.0f, 1.0f, 1, nullptr);
    QED_CUDA(ctx, cudaGetLastError());
    QED_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cur_net(ctx).net_ready = 1;
    cur_net(ctx).net_bins = 0;
    return QED_OK;
}

qed_status qed_sampler_save(qed_ctx* ctx, float* params, int64_t n) {
    if (!ctx || !params || n != kMlpParams) return QED_ERR_ARG;
    if (!cur_net(ctx).net_ready) return set_err(ctx, QED_ERR_STATE, "no sampler trained or loaded");
    QED_CUDA(ctx, cudaMemcpyAsync(params, cur_net(ctx).d_theta, sizeof(float) * kMlpParams,
                                  cudaMemcpyDeviceToHost, ctx->stream));
    QED_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return QED_OK;
}

// ---------------------------------------------------------------------------
// Autotuning of the launch settings
// ---------------------------------------------------------------------------
namespace {

// Copy rows [0, n) of every array between the store and the mirror.
qed_status copy_store(qed_ctx* ctx, const qed_particles* p, long long n, bool to_mirror) {
    float* f_store[] = {p->px, p->py, p->pz, p->Ex, p->Ey, p->Ez, p->Bx, p->By, p->Bz, p->w};
    float* f_mirror[] = {ctx->mirror.px, ctx->mirror.py, ctx->mirror.pz, ctx->mirror.Ex,
                         ctx->mirror.Ey, ctx->mirror.Ez, ctx->mirror.Bx, ctx->mirror.By,
                         ctx->mirror.Bz, ctx->mirror.w};
    for (int k = 0; k < 10; ++k) {
        float* dst = to_mirror ? f_mirror[k] : f_store[k];
        const float* src = to_mirror ? f_store[k] : f_mirror[k];
        QED_CUDA(ctx, cudaMemcpyAsync(dst, src, sizeof(float) * n, cudaMemcpyDeviceToDevice,
                                      ctx->stream));
    }
    QED_CUDA(ctx, cudaMemcpyAsync(to_mirror ? ctx->mirror.id : p->id, to_mirror ? p->id : ctx->mirror.id,
                                  sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    QED_CUDA(ctx, cudaMemcpyAsync(to_mirror ? ctx->mirror.type : p->type,
                                  to_mirror ? p->type : ctx->mirror.type, n,
                                  cudaMemcpyDeviceToDevice, ctx->stream));
    if (!to_mirror)
        QED_CUDA(ctx, cudaMemcpyAsync(p->count, &n, sizeof n, cudaMemcpyHostToDevice, ctx->stream));
    QED_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return QED_OK;
}

}  // namespace

qed_status qed_set_launch(qed_ctx* ctx, uint32_t hot_min, uint32_t long_min,
                          int cold_blocks_per_sm, int hot_blocks_per_sm) {
    if (!ctx || cold_blocks_per_sm < 0 || hot_blocks_per_sm < 0) return QED_ERR_ARG;
    if (hot_min) ctx->hot_min = hot_min;
    if (long_min) ctx->long_min = long_min;
    if (cold_blocks_per_sm)
        ctx->cold_blocks = std::min(ctx->sms * cold_blocks_per_sm, ctx->cold_blocks_max);
    if (hot_blocks_per_sm)
        ctx->hot_blocks = std::min(ctx->sms * hot_blocks_per_sm, ctx->hot_blocks_max);
    return QED_OK;
}

qed_status qed_set_wait_limit(qed_ctx* ctx, uint64_t ns) {
    if (!ctx) return QED_ERR_ARG;
    ctx->wait_ns = ns ? (unsigned long long)ns : kWaitNsDefault;
    return QED_OK;
}

qed_status qed_set_tail(qed_ctx* ctx, int64_t tail_rows) {
    if (!ctx || tail_rows < 0) return QED_ERR_ARG;
    ctx->tail_rows = tail_rows;
    return QED_OK;
}

qed_status qed_autotune(qed_ctx* ctx, const qed_particles* p, uint64_t step_index,
                        const char* out_json) {
    if (!ctx) return QED_ERR_ARG;
    if (!particles_ok(p)) return set_err(ctx, QED_ERR_ARG, "qed_autotune: bad argument");
    qed_status st = ensure_mirror(ctx, p->capacity);
    if (st != QED_OK) return st;
    long long n = 0;
    QED_CUDA(ctx, cudaMemcpyAsync(&n, p->count, sizeof n, cudaMemcpyDeviceToHost, ctx->stream));
    QED_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (n < 0 || n > p->capacity) return set_err(ctx, QED_ERR_ARG, "qed_autotune: bad count");
    st = copy_store(ctx, p, n, true);
    if (st != QED_OK) return st;
    cudaEvent_t e0, e1;
    QED_CUDA(ctx, cudaEventCreate(&e0));
    QED_CUDA(ctx, cudaEventCreate(&e1));
    const int cold_max = ctx->cold_blocks_max / ctx->sms, hot_max = ctx->hot_blocks_max / ctx->sms;
    struct Setting { uint32_t hot_min, long_min; int cold, hot; long long tail; };
    struct Trial { Setting c; float ms; };
    std::vector<Trial> trials;
    auto run = [&](const Setting& c, float* ms) -> qed_status {
        qed_set_launch(ctx, c.hot_min, c.long_min, c.cold, c.hot);
        qed_set_tail(ctx, c.tail);
        qed_status s2 = copy_store(ctx, p, n, false);
        if (s2 != QED_OK) return s2;
        cudaEventRecord(e0, ctx->stream);
        qed_step_stats stt;
        s2 = qed_event_step(ctx, p, step_index, &stt);
        cudaEventRecord(e1, ctx->stream);
        cudaEventSynchronize(e1);
        if (s2 != QED_OK) return s2;
        cudaEventElapsedTime(ms, e0, e1);
        trials.push_back({c, *ms});
        return QED_OK;
    };
    float ms = 0.0f, best = 0.0f;
    Setting b{ctx->hot_min, ctx->long_min, cold_max, hot_max, ctx->tail_rows};
    st = run(b, &best);   // warm-up and reference
    if (st == QED_OK) st = run(b, &best);
    // coordinate search: one setting at a time, keeping the best so far
    auto sweep = [&](auto assign, const auto& values) {
        for (const auto v : values) {
            if (st != QED_OK) return;
            Setting c = b;
            assign(c, v);
            st = run(c, &ms);
            if (st == QED_OK && ms < best) { best = ms; b = c; }
        }
    };
    const uint32_t hot_mins[] = {16, 32, 64, 128, 256};
    const uint32_t long_mins[] = {128, 256, 512, 1024, 2048, 1u << 30};
    std::vector<int> colds, hots;
    for (int v = 1; v <= cold_max; ++v) colds.push_back(v);
    for (int v = 1; v <= hot_max; ++v) hots.push_back(v);
    sweep([](Setting& c, uint32_t v) { c.hot_min = v; }, hot_mins);
    sweep([](Setting& c, uint32_t v) { c.long_min = v; }, long_mins);
    sweep([](Setting& c, int v) { c.cold = v; }, colds);
    sweep([](Setting& c, int v) { c.hot = v; }, hots);
    const long long tails[] = {0, 1ll << 14, 1ll << 16, 1ll << 18, 1ll << 20, 1ll << 22};
    sweep([](Setting& c, long long v) { c.tail = v; }, tails);
    qed_set_launch(ctx, b.hot_min, b.long_min, b.cold, b.hot);
    qed_set_tail(ctx, b.tail);
    const qed_status st_restore = copy_store(ctx, p, n, false);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != QED_OK) return st;
    if (st_restore != QED_OK) return st_restore;
    if (out_json) {
        FILE* f = fopen(out_json, "w");
        if (!f) return set_err(ctx, QED_ERR_ARG, "qed_autotune: cannot write the JSON file");
        fprintf(f, "{\"hot_min\": %u, \"long_min\": %u, \"cold_blocks_per_sm\": %d, "
                   "\"hot_blocks_per_sm\": %d, \"tail_rows\": %lld, \"ms\": %.4f, \"trials\": [",
                b.hot_min, b.long_min, b.cold, b.hot, b.tail, best);
        for (size_t k = 0; k < trials.size(); ++k)
            fprintf(f, "%s{\"hot_min\": %u, \"long_min\": %u, \"cold\": %d, \"hot\": %d, "
                       "\"tail_rows\": %lld, \"ms\": %.4f}",
                    k ? ", " : "", trials[k].c.hot_min, trials[k].c.long_min, trials[k].c.cold,
                    trials[k].c.hot, trials[k].c.tail, trials[k].ms);
        fprintf(f, "]}\n");
        fclose(f);
    }
    return QED_OK;
}

qed_status qed_profile_enable(qed_ctx* ctx, int enable) {
    if (!ctx) return QED_ERR_ARG;
    ctx->prof_on = enable ? 1 : 0;
    return QED_OK;
}

qed_status qed_profile_read(qed_ctx* ctx, double* ms, int64_t* launches, int n) {
    if (!ctx || n < 0 || n > QED_KERNEL_KINDS) return QED_ERR_ARG;
    QED_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    double acc[QED_KERNEL_KINDS] = {0};
    for (size_t k = 0; k < ctx->prof_kind.size(); ++k) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, ctx->prof_ev[2 * k], ctx->prof_ev[2 * k + 1]) == cudaSuccess)
            acc[ctx->prof_kind[k]] += t;
    }
    for (int i = 0; i < n; ++i) {
        if (ms) ms[i] = acc[i];
        if (launches) launches[i] = ctx->launches[i];
    }
    ctx->prof_kind.clear();
    ctx->prof_used = 0;
    for (int i = 0; i < QED_KERNEL_KINDS; ++i) ctx->launches[i] = 0;
    return cuda_check(ctx, cudaGetLastError(), "qed_profile_read");
}

size_t qed_abi_struct_size(const char* name) {
    if (!name) return 0;
    if (!strcmp(name, "qed_config")) return sizeof(qed_config);
    if (!strcmp(name, "qed_particles")) return sizeof(qed_particles);
    if (!strcmp(name, "qed_step_stats")) return sizeof(qed_step_stats);
    if (!strcmp(name, "qed_event_record")) return sizeof(qed_event_record);
    if (!strcmp(name, "qed_host_particles")) return sizeof(qed_host_particles);
    return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The remaining-time arithmetic of the event kernels, exposed for validation
// ---------------------------------------------------------------------------
__global__ void k_time_split(const float* __restrict__ t_hi, const float* __restrict__ t_lo,
                             const uint32_t* __restrict__ N, const uint32_t* __restrict__ m,
                             long long n, double* __restrict__ h_out, double* __restrict__ t_out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const ftime t{t_hi[i], t_lo[i]};
        const ftime h = time_div(t, N[i]);
        const ftime r = m[i] >= N[i] ? ftime{0.0f, 0.0f} : time_sub_mul(t, m[i], h);
        h_out[i] = (double)h.hi + (double)h.lo;
        t_out[i] = (double)r.hi + (double)r.lo;
    }
}

extern "C" qed_status qed_time_split(const float* t_hi, const float* t_lo, const uint32_t* N,
                                     const uint32_t* m, int64_t n, double* h, double* t_after,
                                     void* stream) {
    if (n < 0 || (n > 0 && (!t_hi || !t_lo || !N || !m || !h || !t_after))) return QED_ERR_ARG;
    if (n == 0) return QED_OK;
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    k_time_split<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(t_hi, t_lo, N, m, n, h, t_after);
    return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Event step without allocation.
//
// For callers that may not allocate device memory: hosts that hand each
// component a fixed memory budget up front (a cudaMalloc of their own would
// fail, or take memory promised to another component), and plug-ins living
// inside another application's memory pool (which must not go around that
// pool to the CUDA allocator).  The scratch of the event step (control block,
// remaining times of children, queue of long sub-step chains) lives in one
// file-scope device array sized for QED_NOALLOC_MAX_ROWS rows; every GPU that
// loads this library keeps it until the process exits.  The first call on a
// device looks up the array's device address (cudaGetSymbolAddress) and the
// launch geometry with that device current; later calls reuse them.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocCtlBytes = 256;
constexpr size_t kNoAllocTremOffset = kNoAllocCtlBytes;
constexpr size_t kNoAllocHotOffset =
    kNoAllocTremOffset + sizeof(ftime) * (size_t)QED_NOALLOC_MAX_ROWS;
constexpr size_t kNoAllocBytes =
    kNoAllocHotOffset + sizeof(HotItem) * 2 * (size_t)QED_NOALLOC_MAX_ROWS;
static_assert(sizeof(DevCtl) <= kNoAllocCtlBytes, "control block does not fit");
static_assert(kNoAllocHotOffset % 16 == 0, "queue alignment");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocDevice {
    int ready;
    unsigned char* base;   // device address of g_noalloc_scratch on this device
    int sms, cold_blocks, hot_blocks, step_blocks;
};
constexpr int kNoAllocMaxDevices = 64;
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];
std::mutex g_noalloc_mutex;

qed_status noalloc_setup(int dev, NoAllocDevice* out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoAllocDevice& d = g_noalloc_dev[dev];
    if (!d.ready) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr)
            return QED_ERR_CUDA;
        int sms = 0, per_cold = 0, per_hot = 0, per_step = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return QED_ERR_CUDA;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_cold, k_cold<false>, kColdThreads, 0) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_hot, k_hot_lanes<0>, kLaneThreads, 0) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_step, k_step<0>, kLaneThreads, 0) !=
                cudaSuccess)
            return QED_ERR_CUDA;
        // long-plan queue entries start "not written"; each step resets the ones it used
        if (cudaMemset(static_cast<unsigned char*>(ptr) + kNoAllocHotOffset, 0xFF,
                       sizeof(HotItem) * 2 * (size_t)QED_NOALLOC_MAX_ROWS) != cudaSuccess ||
            cudaDeviceSynchronize() != cudaSuccess)
            return QED_ERR_CUDA;
        d.base = static_cast<unsigned char*>(ptr);
        d.sms = sms;
        d.cold_blocks = sms * (per_cold > 0 ? per_cold : 1);
        d.hot_blocks = sms * (per_hot > 0 ? per_hot : 1);
        d.step_blocks = sms * (per_step > 0 ? per_step : 1);
        d.ready = 1;
    }
    *out = d;
    return QED_OK;
}

}  // namespace

// After a failed launch the step may not have reached k_tail_end, which puts
// the long-plan queue entries it used back to "not written"; the next call on
// the device then clears the whole queue again in its set-up.
static qed_status noalloc_fail(int dev, qed_status st) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    g_noalloc_dev[dev].ready = 0;
    return st;
}

extern "C" qed_status qed_event_step_noalloc(const qed_config* cfg, const qed_particles* p,
                                             uint64_t step_index, void* stream,
                                             qed_step_stats* out) {
    if (!cfg || !particles_ok(p) || step_index > 0xffffffffull) return QED_ERR_ARG;
    if (p->capacity > (int64_t)QED_NOALLOC_MAX_ROWS) return QED_ERR_ARG;
    if (!(cfg->p_max > 0.0f && cfg->p_max <= 1.0f) || !(cfg->dt_periods > 0.0) ||
        !(cfg->lambda_m > 0.0) || !(cfg->pair_bound_coeff > 0.0f))
        return QED_ERR_ARG;
    if (cfg->sampler_mode != 0) return QED_ERR_ARG;   // the learned sampler needs a context
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QED_ERR_CUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return QED_ERR_ARG;
    NoAllocDevice nd;
    qed_status st = noalloc_setup(dev, &nd);
    if (st != QED_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int max_passes = cfg->max_passes > 0 ? cfg->max_passes : 64;
    const StepParams SP = make_params(*cfg, step_index);
    const DevParticles D = to_dev(p);
    DevCtl* ctl = reinterpret_cast<DevCtl*>(nd.base);
    Scratch S;
    S.t_rem = reinterpret_cast<ftime*>(nd.base + kNoAllocTremOffset);
    S.hot = reinterpret_cast<HotItem*>(nd.base + kNoAllocHotOffset);
    S.hot_cap = 2 * (long long)QED_NOALLOC_MAX_ROWS;
    S.log = nullptr;
    S.log_cap = 0;
    S.log_count = nullptr;
    const bool cascade = cascade_enabled(*cfg);
    // the step-init kernel resets the whole control block, so nothing left
    // from an earlier call is read
    k_step_init<<<1, 1, 0, s>>>(ctl, D.count, D.capacity, 0);
    DevCtl h;
    for (int pass = 0; pass < max_passes; ++pass) {
        k_cold<false><<<nd.cold_blocks, kColdThreads, 0, s>>>(D, SP, S, ctl);
        k_hot_lanes<0><<<nd.hot_blocks, kLaneThreads, 0, s>>>(D, SP, S, ctl);
        k_advance<<<1, 1, 0, s>>>(ctl, D.count, D.capacity, cascade ? 1 : 0, max_passes,
                                  kTailRowsDefault, 0ull, 0);
        if (cudaGetLastError() != cudaSuccess) return noalloc_fail(dev, QED_ERR_CUDA);
        if (!cascade) break;
        if (cudaMemcpyAsync(&h, ctl, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return noalloc_fail(dev, QED_ERR_CUDA);
        if (!h.more) break;
    }
    // the tail pass (its kernels do nothing when the generations ran to the end)
    k_tail_begin<<<nd.sms * 8, 256, 0, s>>>(D, S, ctl);
    k_cold<false><<<nd.cold_blocks, kColdThreads, 0, s>>>(D, SP, S, ctl);
    k_step<0><<<nd.step_blocks, kLaneThreads, 0, s>>>(D, SP, S, ctl);
    k_tail_end<<<nd.sms * 8, 256, 0, s>>>(D, S, ctl);
    if (cudaGetLastError() != cudaSuccess) return noalloc_fail(dev, QED_ERR_CUDA);
    if (!out) return QED_OK;
    if (cudaMemcpyAsync(&h, ctl, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return noalloc_fail(dev, QED_ERR_CUDA);
    fill_stats(h, out, h.pass_end);
    return (qed_status)h.status;
}
