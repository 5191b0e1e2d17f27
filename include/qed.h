/*
 * qed.h - C ABI of the GB300 QED Monte Carlo event generator.
 *
 * Implements the per-particle event generator of "Optimized routines for
 * event generators in QED-PIC codes" (Volokitin et al., arXiv:2008.10468):
 * hard-photon emission by electrons/positrons (Eq. 1, Algorithm 1) and
 * photon decay into pairs (Eq. 2, Algorithm 2), with local sub-stepping
 * planned from the rate bounds of Sec. 3.1.1 and the synchrotron functions
 * of Sec. 3.2.1.
 *
 * Conventions
 *   - Code units: momentum in m c, fields in m c omega / e (omega = 2 pi c /
 *     lambda), time in laser periods T = lambda / c.
 *   - Particle storage is structure-of-arrays in device memory, owned by the
 *     caller.  Row i of every array describes one macroparticle.  Types:
 *     0 electron, 1 positron, 2 photon, 3 removed (a photon that decayed).
 *   - All calls are asynchronous on the context's CUDA stream unless stated.
 *     Pointers documented as "device" must be device (or managed) memory.
 *   - Errors are return codes; nothing is thrown across the ABI.  A CUDA
 *     error is QED_ERR_CUDA and its text is kept for qed_last_error().
 *     Problems found inside a kernel (capacity exceeded, a bounded wait that
 *     gave up) are written to a device status word and reported by the next
 *     call that reads statistics back.
 *   - A context is not thread safe; use one per host thread.
 */
#ifndef QED_H
#define QED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QED_OK = 0,
    QED_ERR_ARG = 1,       /* invalid argument (null pointer, bad size, ...)  */
    QED_ERR_CUDA = 2,      /* a CUDA runtime call failed                       */
    QED_ERR_CAPACITY = 3,  /* children did not fit; see required_capacity     */
    QED_ERR_TIMEOUT = 4,   /* a bounded device-side wait gave up              */
    QED_ERR_STATE = 5      /* call out of order (e.g. launch before capture)  */
} qed_status;

enum { QED_PROC_EMISSION = 1u, QED_PROC_PAIR = 2u };

enum { QED_ELECTRON = 0, QED_POSITRON = 1, QED_PHOTON = 2, QED_REMOVED = 3 };

/* Run configuration.  qed_config_default() fills the values the paper
 * recommends (P_max = 0.01, Sec. 3.1.2) and the synthetic workloads use. */
typedef struct {
    uint64_t seed;             /* key of the Philox4x32-10 streams              */
    double dt_periods;         /* global PIC step in laser periods (0.1)        */
    double lambda_m;           /* laser wavelength in metres (1e-6)             */
    float p_max;               /* max per-sub-step event probability (0.01)     */
    float pair_bound_coeff;    /* photon bound f = coeff * c * b (0.1, Sec. 3.1.1) */
    uint32_t process_mask;     /* QED_PROC_EMISSION | QED_PROC_PAIR             */
    int32_t cascade_in_step;   /* 1: children are processed in the same step    */
    int32_t recoil;            /* 1: events change/remove the parent; 0 is a
                                  validation mode in which they do not          */
    int32_t max_passes;        /* cascade generations per step (0 -> 64)        */
    float drain_chi;           /* compaction drains photons with chi below this
                                  into the photon spectrum (0: never)           */
    int32_t sampler_mode;      /* 1: learned inverse-CDF sampler for e+- emission
                                  where usable (see qed_sampler_train): each
                                  sub-step is an event with the tabulated
                                  probability; 2: the same, event-driven: the
                                  sub-steps to the next event are drawn at once
                                  (geometric), with no per-sub-step draws; its
                                  particles run one per lane and each warp's
                                  events go through the network together on
                                  the tensor cores; in the tail pass of the
                                  cascade they are stepped a warp each and go
                                  through the network one at a time          */
    float sampler_max_err;     /* a chi bin is usable if its max CDF error <= this
                                  (1e-3)                                        */
} qed_config;

/* Photon spectrum filled by the drain: weight per bin of log10(photon
 * energy / m c^2), QED_SPECTRUM_BINS equal bins over [MIN, MAX). */
#define QED_SPECTRUM_BINS 240
#define QED_SPECTRUM_LOG10_MIN (-4)
#define QED_SPECTRUM_LOG10_MAX 8

/* Particle store (device pointers, caller-owned). */
typedef struct {
    float *px, *py, *pz;       /* momentum (m c); photon: |k| is its energy     */
    float *Ex, *Ey, *Ez;       /* electric field at the particle                */
    float *Bx, *By, *Bz;       /* magnetic field at the particle                */
    float *w;                  /* macroparticle weight                          */
    uint64_t *id;              /* unique id; children get ids with bit 63 set   */
    uint8_t *type;             /* 0 e-, 1 e+, 2 photon, 3 removed               */
    int64_t *count;            /* device int64: rows in use (updated by steps)  */
    int64_t capacity;          /* rows allocated in every array                 */
} qed_particles;

/* Particle store in host memory (host pointers, caller-owned), for
 * qed_event_step_host: the fields of qed_particles, with the row count on
 * the host. */
typedef struct {
    float *px, *py, *pz, *Ex, *Ey, *Ez, *Bx, *By, *Bz, *w;
    uint64_t *id;
    uint8_t *type;
    int64_t count;             /* rows in use: read before the step, written after */
    int64_t capacity;          /* rows every array holds                        */
} qed_host_particles;

/* Statistics of the last step (host struct). */
typedef struct {
    uint64_t substeps;         /* sub-steps executed (loop iterations of Alg. 1/2) */
    uint64_t emissions;        /* photon emission events                        */
    uint64_t pairs;            /* pair production events                        */
    uint64_t children;         /* rows appended                                 */
    uint64_t guard_hits;       /* plans raised by the validity guard            */
    uint64_t plans;            /* sub-step plans made (1 + one per event)       */
    uint64_t candidates;       /* sub-steps whose draw passed the squeeze test, so
                                  that the acceptance function decides (a work
                                  counter: the warp mode tests whole 64-sub-step
                                  windows, also past an event)                  */
    uint32_t max_N;            /* largest planned sub-step count                */
    int32_t status;            /* qed_status of the step                        */
    int64_t required_capacity; /* rows needed when status == QED_ERR_CAPACITY   */
    int64_t count;             /* rows in use after the step                    */
    int32_t passes;            /* cascade generations processed                 */
    int32_t tail;              /* 1: the step's last generations ran as the tail pass */
    uint64_t substeps_warp;    /* of `substeps`, those run by the hot pass and the tail pass's persistent kernel */
    uint64_t sampler_events;   /* emissions whose energy came from the learned sampler */
    uint64_t sampler_pairs;    /* pair events whose electron fraction came from the
                                  learned pair sampler */
} qed_step_stats;

/* One event, written to the optional device event log (validation). */
typedef struct {
    uint64_t parent_id;
    uint64_t child_id0;        /* photon (emission) or electron (pair)          */
    uint64_t child_id1;        /* positron (pair), 0 for emission               */
    uint32_t s;                /* sub-step index of the event in this step      */
    uint32_t kind;             /* 1 emission, 2 pair                            */
    float delta;               /* energy fraction: photon (1) or electron (2)   */
    float chi;                 /* parent chi at the event                       */
} qed_event_record;

typedef struct qed_ctx qed_ctx;

/* Fill *cfg with the defaults listed in qed_config.  Never fails. */
void qed_config_default(qed_config* cfg);

/* Create a context on the current CUDA device.  `stream` is a cudaStream_t
 * (NULL: the legacy default stream) on which every later call is ordered.
 * Copies *cfg.  Allocates nothing large; the per-step scratch is sized on
 * the first qed_event_step.  Errors: QED_ERR_ARG (null out/cfg, p_max not
 * in (0, 1], dt <= 0, lambda <= 0), QED_ERR_CUDA. */
qed_status qed_init(qed_ctx** out, const qed_config* cfg, void* stream);

/* Release the context and its device scratch (synchronises its stream). */
qed_status qed_destroy(qed_ctx* ctx);

/* Text of the last error of this context (static storage of the context). */
const char* qed_last_error(const qed_ctx* ctx);

/* Synchrotron functions, Sec. 3.2.1:
 *   F1[i] = F(y[i]) = y int_y^inf K_{5/3}(t) dt,
 *   F2[i] = G(y[i]) = y K_{2/3}(y),
 * in binary32 (relative error <= 4e-6 for y in [1e-4, 50]; 0 for y <= 0 or
 * y >= 88).  y, F1, F2 are device arrays of n floats; F1 or F2 may be NULL to
 * skip that output; n == 0 is a no-op whatever the pointers.  Errors:
 * QED_ERR_ARG (null ctx, null y with n > 0, n < 0). */
qed_status qed_synchrotron_F1F2(qed_ctx* ctx, const float* y, float* F1, float* F2, int64_t n);

/* The same functions in binary64, at the double-precision accuracy level of
 * Sec. 3.2.1 (Table 1: 1e-14): relative error below 1e-15 for y in
 * (0, 512), from three polynomials of degree 11 per octave (no difference of
 * large terms is formed); 0 for y <= 0, y >= 512 (where F, G < 1e-220) and
 * NaN.  y, F1, F2 are device arrays of n doubles; F1 or F2 may be NULL (not
 * both when n > 0); n == 0 is a no-op.  No context: runs on `stream` (a
 * cudaStream_t, NULL for the default stream), asynchronously.  Errors:
 * QED_ERR_ARG (n < 0, null y or both outputs null with n > 0), QED_ERR_CUDA. */
qed_status qed_synchrotron_F1F2_f64(const double* y, double* F1, double* F2, int64_t n,
                                    void* stream);

/* The same functions on arguments generated in the kernel:
 *   y_i = lo * (hi/lo)^u_i,  u_i the open-interval uniform of word (i mod 4)
 *   of Philox4x32-10 at counter (i/4 low, i/4 high, 0, 0), key `seed`.
 * Moves no argument bytes through memory (the arithmetic-bound mode of the
 * sweep).  *checksum (device float, may be NULL) receives sum(F1 + F2) by
 * atomic adds (order-dependent rounding).  y_out/F1_out/F2_out (device,
 * nullable) store the values for validation.  Errors: QED_ERR_ARG. */
qed_status qed_synchrotron_generate(qed_ctx* ctx, uint64_t seed, int64_t n, float lo, float hi,
                                    float* checksum, float* y_out, float* F1_out, float* F2_out);

/* The planning step of Algorithms 1/2 only: for rows [0, n) compute chi (Sec. 2.2) and
 * the sub-step count N of a full global step (bound f(b) of Sec. 3.1.1,
 * N = max(1, ceil(f / P_max)), validity guard for e+-).  chi and N are
 * device arrays of n entries (either may be NULL).  Rows that are removed, or
 * whose process is disabled, get N = 0.  Errors: QED_ERR_ARG. */
qed_status qed_plan(qed_ctx* ctx, const qed_particles* p, int64_t n, float* chi, uint32_t* N);

/* Per-cell planning (Sec. 2.2: Algorithms 1 and 2 start by fixing one
 * sub-step per cell): N_cell[c] = the largest sub-step count N of
 * qed_plan over the rows i < n with cell[i] == c (0 for a cell without an
 * active row), so that sub_t = dt / N_cell[c] keeps every particle of the
 * cell within P_max per sub-step.  cell: device array of n cell indices;
 * rows with cell[i] >= ncells are left out.  N_cell: device array of ncells
 * entries, overwritten.  qed_event_step itself plans per particle, a finer
 * form of the same bound; these counts are for callers that take one
 * sub-step per cell.  Errors: QED_ERR_ARG, QED_ERR_CUDA. */
qed_status qed_plan_cells(qed_ctx* ctx, const qed_particles* p, int64_t n, const uint32_t* cell,
                          int64_t ncells, uint32_t* N_cell);

/* One global step of the event generator (Algorithms 1 and 2) for every row
 * in use.  Each particle is planned, stepped through its sub-steps with
 * Philox4x32-10 draws keyed by (id, step_index, sub-step), emits photons /
 * decays (photons are marked removed, type 3), recoils, and is re-planned
 * after every event over the remaining time.  Children are appended at rows
 * count.. and, if cascade_in_step, processed in the same step: generation by
 * generation while the generations are large, then (qed_set_tail) the rest
 * in one tail pass.  If out != NULL the call synchronises the stream and fills *out; if NULL it
 * returns without waiting (statistics readable with qed_read_stats).
 * Capacity: if the children do not fit, status QED_ERR_CAPACITY is returned
 * (in *out and as the return value when out != NULL) with the rows needed;
 * the step is then incomplete (parents that emitted a dropped child have
 * recoiled) and the caller must restore its own copy of the store.
 * Errors: QED_ERR_ARG, QED_ERR_CUDA, QED_ERR_CAPACITY, QED_ERR_TIMEOUT. */
qed_status qed_event_step(qed_ctx* ctx, const qed_particles* p, uint64_t step_index,
                          qed_step_stats* out);

/* qed_event_step with one sub-step per cell for the first plans (Algorithms 1
 * and 2 start by fixing the sub-step of the particle's cell): the counts of
 * qed_plan_cells are taken over the rows in use at the start of the step
 * (cell: device array with a cell index for each of them; rows with
 * cell[i] >= ncells keep their own count), and each of those rows makes its
 * first plan with its cell's count when that is larger than its own.
 * Re-plans after events, and children, plan per particle.  The context owns
 * the ncells counts (allocated on first use).  Errors: as qed_event_step;
 * QED_ERR_ARG for a NULL cell, ncells outside [1, 2^32), or a learned
 * sampler in cfg.sampler_mode (the two do not combine). */
qed_status qed_event_step_cells(qed_ctx* ctx, const qed_particles* p, uint64_t step_index,
                                const uint32_t* cell, int64_t ncells, qed_step_stats* out);

/* qed_event_step on a store in host memory (the same step: Sec. 2,
 * Algorithms 1 and 2).  The context keeps a device copy of the store's
 * layout (capacity rows; allocated on first use and when the capacity
 * changes).  Rows [0, h->count) of every field are copied to it, the step
 * runs there, and what the step changed is copied back: momenta and types
 * of the rows it was given, every field of the rows it appended; h->count
 * becomes the rows in use after the step.  Copies are cudaMemcpyAsync on the
 * context stream: page-locked host arrays (cudaHostAlloc, cudaHostRegister)
 * copy at the host link's rate, pageable ones are staged by the driver.
 * Synchronises.  *out (nullable) receives the step's statistics.  If the
 * step does not succeed (QED_ERR_CAPACITY with the rows required,
 * QED_ERR_TIMEOUT, ...) nothing is copied back: the host store is left as it
 * was.  Errors: QED_ERR_ARG (a null array, capacity outside [1, 2^32),
 * count outside [0, capacity]), QED_ERR_CUDA, and the statuses of
 * qed_event_step. */
qed_status qed_event_step_host(qed_ctx* ctx, qed_host_particles* h, uint64_t step_index,
                               qed_step_stats* out);

/* The same step with the Boris push of Algorithm 1 (Sec. 2.2: the particle is
 * moved by a Boris step of one sub-step, then chi is recomputed and
 * the draw tested): before every draw an electron or positron moves its
 * momentum by one sub-step h under the Lorentz force of its own constant
 * fields, dp/dt = 2 pi q (E + p x B / gamma) in code units (q = -1 for e-,
 * +1 for e+), and the draw is tested at the chi of the pushed momentum.  A
 * photon flies straight (Algorithm 2): momentum and chi stay.  The sub-step
 * count is planned from the state at the start of the step and after each
 * event, as in qed_event_step.  The push is the IEEE binary32 evaluation of
 * the Boris formulas (the store's precision).  Positions are not stored, so
 * only momenta move.  On return every processed e+- row holds its momentum
 * after the step.  Same arguments, statistics, capacity rule and errors as
 * qed_event_step; the learned sampler is not used.  With the cascade, the
 * whole step runs as one persistent pass that takes each child as soon as it
 * is reserved (the generations do not wait for the longest push chain of the
 * one before), unless qed_set_tail(ctx, 0) asks for one launch per
 * generation; both give the same result. */
qed_status qed_event_step_push(qed_ctx* ctx, const qed_particles* p, uint64_t step_index,
                               qed_step_stats* out);

/* The push-mode step with one sub-step per cell, Algorithm 1 as the paper
 * states it: the counts of qed_plan_cells are taken over the rows in use at
 * the start of the step (cell: device array with a cell index for each of
 * them; rows with cell[i] >= ncells keep their own count), and each of those
 * rows makes its first plan with its cell's count when that is larger than
 * its own, i.e. with the cell's sub-step dt / N_cell.  Re-plans after events,
 * and children, plan per particle as in qed_event_step_push.  The context
 * owns the ncells counts (allocated on first use).  Errors: as
 * qed_event_step_push; QED_ERR_ARG for a NULL cell or ncells outside
 * [1, 2^32). */
qed_status qed_event_step_push_cells(qed_ctx* ctx, const qed_particles* p, uint64_t step_index,
                                     const uint32_t* cell, int64_t ncells, qed_step_stats* out);

/* Synchronise and read the statistics of the last step.  Errors: ARG, CUDA. */
qed_status qed_read_stats(qed_ctx* ctx, qed_step_stats* out);

/* Optional event log for validation: subsequent steps append one record per
 * event to `records` (device array of `capacity` entries) while *count
 * (device int64, caller-zeroed) counts the events seen; records beyond the
 * capacity are dropped.  Pass records == NULL to disable.  Errors: ARG. */
qed_status qed_set_event_log(qed_ctx* ctx, qed_event_record* records, int64_t capacity,
                             int64_t* count);

/* Remove the rows of removed particles (type 3) from the store, keeping the
 * order of the others, and set *count to the rows kept.  If cfg.drain_chi > 0,
 * photons with chi below it are first added (by weight) to the context's
 * photon spectrum and removed: the paper's method never needs them again,
 * since their pair probability is negligible.  Not part of the paper's
 * algorithm; a store-management step of this library.  *removed (host,
 * nullable) receives the rows removed (the call then synchronises).
 * Device scratch of 49 bytes per row of capacity is allocated on first use.
 * Errors: QED_ERR_ARG, QED_ERR_CUDA. */
qed_status qed_compact(qed_ctx* ctx, const qed_particles* p, int64_t* removed);

/* Copy the drained-photon spectrum (QED_SPECTRUM_BINS doubles) to `out`
 * (host) and, if reset, zero it.  Synchronises.  Errors: QED_ERR_ARG. */
qed_status qed_read_spectrum(qed_ctx* ctx, double* out, int nbins, int reset);

/* Record `nsteps` consecutive global steps (step indices first_step ..
 * first_step + nsteps - 1) on store `p` as one CUDA graph: per step, the
 * cascade generations run in a device-side loop (a conditional WHILE node
 * whose condition the last kernel of each generation sets), then the tail
 * pass (qed_set_tail), then the store is compacted (qed_compact), then the step's statistics are recorded on the
 * device.  No host synchronisation inside.  Each launch continues the step
 * numbering: the first launch runs steps first_step .. first_step + nsteps - 1,
 * the next one the following nsteps indices (fresh draws and child ids).
 * A step that fails (capacity,
 * cascade deeper than max_passes) makes the following steps no-ops; its
 * record carries the status.  Replaces any earlier graph of the context.
 * Errors: QED_ERR_ARG, QED_ERR_CUDA. */
qed_status qed_graph_capture(qed_ctx* ctx, const qed_particles* p, uint64_t first_step,
                             int nsteps);

/* Launch the captured graph on the context stream (asynchronous).
 * Errors: QED_ERR_STATE (nothing captured), QED_ERR_CUDA. */
qed_status qed_graph_launch(qed_ctx* ctx);

/* Synchronise and copy the per-step statistics of the last graph launch
 * (nsteps <= captured steps) to out[0..nsteps).  Returns the first non-zero
 * step status, else QED_OK.  Errors: QED_ERR_ARG, QED_ERR_STATE, CUDA. */
qed_status qed_graph_read_stats(qed_ctx* ctx, qed_step_stats* out, int nsteps);

/* Learned inverse-CDF sampler (the inverse-sampling event generator the
 * paper names as the classical alternative, Sec. 2.2, for the emission of
 * Eq. 1).  A 2-64-64-64-1 perceptron (SiLU; logistic output anchored at
 * logit u, so that x(0) = 0 and x(1) = 1; BF16 weights and FP32
 * accumulation in the event kernels) maps (log10 chi, u) to x, the cube
 * root of the photon energy fraction, for chi in [1e-2, 1e2).  With
 * cfg.sampler_mode, e+- in a usable chi bin decide events from the tabulated
 * total probability per sub-step c_h W(b) and take x from the network at the
 * event's uniform; all others keep rejection.  The 64 bins are uniform in
 * log10 chi; a bin is usable when its measured max |CDF(x_net(u)) - u| is at
 * most cfg.sampler_max_err. */
#define QED_SAMPLER_PARAMS 8577
#define QED_SAMPLER_BINS 64

/* The learned samplers are two networks of the same form: for photon emission
 * (x = delta^{1/3} of Eq. 1, the default) and for pair production (x =
 * delta_e, the electron's energy fraction of Eq. 2, a spectrum symmetric
 * about 1/2).  qed_sampler_train, _evaluate, _gradient, _quantile, _load and
 * _save address the network chosen here (QED_PROC_EMISSION or
 * QED_PROC_PAIR).  In sampler_mode 2 the event step uses the pair network,
 * once trained and evaluated, for photon plans with a nonzero squeeze
 * threshold, at least hot_min sub-steps and chi_gamma in a usable bin: the
 * sub-steps to the decay are drawn at once from the tabulated total pair
 * probability and delta_e comes from the network; all other photon plans
 * keep rejection.  Errors: QED_ERR_ARG. */
qed_status qed_sampler_process(qed_ctx* ctx, uint32_t process);

/* Train with Adam (cosine-decayed step `lr`) on `samples` pairs drawn in
 * batches of `batch` (64 <= batch <= 2^20): log10 chi and u uniform (chi in
 * [1e-2, 1e2) for the emission network, [0.25, 1e2) for the pair network,
 * whose spectrum underflows binary32 below), target x from the exact CDF of
 * the network's spectrum, tabulated on the GPU from the acceptance function
 * of Algorithm 1 or 2 (1024 chi rows x 4096 x intervals).
 * Loss: mean of (CDF(chi, x_net) - u)^2, the squared CDF error of the
 * sampler, with CDF and density from the same tables; the forward pass uses
 * the BF16-rounded weights the event kernels use, its gradient updating the
 * FP32 weights.
 * Starts from deterministic initial weights (seed) unless parameters were
 * trained or loaded before.  *final_loss (host, nullable): mean squared
 * error of the last batch.  Synchronises.  Errors: ARG, CUDA. */
qed_status qed_sampler_train(qed_ctx* ctx, uint64_t seed, int64_t samples, int batch, float lr,
                             float* final_loss);

/* Measure the max CDF error per bin (bin_err: host array of
 * QED_SAMPLER_BINS) on 4 chi rows x 1024 u per bin against exact CDF rows,
 * for both forms of the network the event kernels use (the larger error
 * counts), and mark the usable bins.  Required before an event step in
 * sampler mode.
 * Errors: ARG, STATE (no sampler), CUDA. */
qed_status qed_sampler_evaluate(qed_ctx* ctx, float* bin_err, int nbins);

/* Loss mean(w^2 (x - t)^2) of the network `params` (device,
 * QED_SAMPLER_PARAMS floats, used unrounded) on inputs v (device, B x 2:
 * log10 chi / 2, logit(u) / 8), targets t and weights w (device, B; weight NULL:
 * all 1), and its gradient into grad (device, QED_SAMPLER_PARAMS); *loss
 * (device, nullable).  For gradient checks.  Errors: ARG, CUDA. */
qed_status qed_sampler_gradient(qed_ctx* ctx, const float* params, const float* v,
                                const float* target, const float* weight, int64_t B, float* grad,
                                float* loss);

/* x = delta^{1/3} at (log10chi[i], u[i]) for i < n (device arrays; log10 chi
 * clamped to [-2, 2]; u in the open interval (0, 1)): use_net = 0 the exact
 * inverse CDF from the tables (bilinear in log10 chi and x), 1 the network
 * as the warp-mode event kernels evaluate it (FP32 activations), 2 the
 * network on the tensor cores as the event-driven sampler evaluates it
 * (mma.sync BF16 x BF16 -> FP32, activations as BF16 hi + lo pairs).
 * Errors: ARG, STATE, CUDA. */
qed_status qed_sampler_quantile(qed_ctx* ctx, const float* log10chi, const float* u, float* x,
                                int64_t n, int use_net);

/* Copy parameters in (host -> device, also refreshes the BF16 copy) or out. */
qed_status qed_sampler_load(qed_ctx* ctx, const float* params, int64_t n);
qed_status qed_sampler_save(qed_ctx* ctx, float* params, int64_t n);

/* Launch settings.  hot_min: plans of at least this many sub-steps leave the
 * thread pass for the hot pass (default 32); long_min: hot plans of at least
 * this many sub-steps are stepped by a whole warp each, the others one lane
 * each (default 256; the sampler mode steps every hot particle by a warp);
 * the resident blocks per SM of the thread and hot passes (default: the
 * occupancy maximum; larger values are clamped to it).  0 keeps a setting.
 * No setting changes a result.  Errors: QED_ERR_ARG. */
qed_status qed_set_launch(qed_ctx* ctx, uint32_t hot_min, uint32_t long_min,
                          int cold_blocks_per_sm, int hot_blocks_per_sm);

/* Tail pass of the cascade (Sec. 2: the events of one step form a cascade
 * whose generations shrink).  Once a generation has fewer than tail_rows rows
 * the generations stop: one thread pass over that generation, then one
 * persistent kernel takes its queue and every child appended after it as
 * they come, so that the step is not bound by the longest chain of each
 * small generation in turn.  0 turns it off; default 131072 rows.  No
 * setting changes a result (the passes count counts the tail as one).
 * Errors: QED_ERR_ARG (ctx null, tail_rows < 0). */
qed_status qed_set_tail(qed_ctx* ctx, int64_t tail_rows);

/* Longest bounded wait of the persistent passes (the tail pass, the push
 * step's pass), in nanoseconds (0: the default, 1 s).  Their kernels wait
 * for child rows that another warp is still writing and for queue entries
 * not yet pushed, and their idle warps wait for new work; a warp that has
 * waited this long without progress anywhere (rows stored or completed,
 * beats of long chains) gives up, and the step ends with QED_ERR_TIMEOUT
 * (in the statistics and as the return value when they are read) instead of
 * hanging; the context stays usable.  A short limit makes idle warps give
 * up early, so it is for tests of that path.  Applies to later steps and
 * graph captures.  Errors: QED_ERR_ARG (ctx null). */
qed_status qed_set_wait_limit(qed_ctx* ctx, uint64_t ns);

/* Time qed_event_step on `p` (step index step_index) for a coordinate search
 * over the launch settings (hot_min 16 ... 256, long_min 128 ... 2048 or
 * never, blocks per SM of each pass, tail_rows 0 or 2^14 ... 2^22), keep the
 * fastest, and restore the store from a snapshot
 * after every trial (the store is unchanged on return).  Writes the chosen
 * settings and all trial timings as JSON to out_json (host file path,
 * nullable).  Uses the compaction mirror as snapshot.  Synchronises.
 * Errors: ARG, CUDA and those of qed_event_step. */
qed_status qed_autotune(qed_ctx* ctx, const qed_particles* p, uint64_t step_index,
                        const char* out_json);

/* Kernel kinds for qed_profile_read. */
enum {
    QED_KERNEL_SWEEP = 0,      /* synchrotron functions over an array          */
    QED_KERNEL_GENERATE = 1,   /* synchrotron functions, in-kernel arguments   */
    QED_KERNEL_PLAN = 2,       /* planner                                      */
    QED_KERNEL_COLD = 3,       /* event step: thread-per-particle pass         */
    QED_KERNEL_HOT = 4,        /* event step: queue pass and tail pass         */
    QED_KERNEL_CONTROL = 5,    /* event step: per-step and per-pass bookkeeping */
    QED_KERNEL_SAMPLER = 6,    /* event step: event-driven sampler, one lane per particle */
    QED_KERNEL_KINDS = 8
};

/* Benchmark timing.  While enabled, every kernel this context launches is
 * bracketed by CUDA events recorded on the context stream (this adds a few
 * microseconds per launch).  Launch counts are kept whether or not timing is
 * enabled.  Errors: QED_ERR_ARG, QED_ERR_CUDA. */
qed_status qed_profile_enable(qed_ctx* ctx, int enable);

/* Synchronise the stream, write the milliseconds measured and the kernels
 * launched per kind since the last read into ms[0..n) and launches[0..n)
 * (host arrays, either may be NULL; n <= QED_KERNEL_KINDS), then reset both
 * accumulators.  Errors: QED_ERR_ARG, QED_ERR_CUDA. */
qed_status qed_profile_read(qed_ctx* ctx, double* ms, int64_t* launches, int n);

/* Validation of the remaining-time arithmetic the event kernels use (Sec. 2,
 * Algorithms 1 and 2: the global step split into N sub-steps of length
 * h = t / N; after an event at sub-step m - 1 the time left is t - m h).  The
 * kernels carry t as a float-float pair (t_hi + t_lo, about 48 significant
 * bits) on the FP32 pipe; for each i < n this computes h = t / N[i] and
 * t - m[i] h (0 when m[i] >= N[i], the plan's last sub-step ending it
 * exactly) that way and returns both as binary64 (h, t_after: device arrays
 * of n doubles; t_hi, t_lo: device floats, |t_lo| <= ulp(t_hi) / 2; N, m:
 * device uint32, N >= 1).  Asynchronous on `stream` (a cudaStream_t).
 * Errors: QED_ERR_ARG, QED_ERR_CUDA. */
qed_status qed_time_split(const float* t_hi, const float* t_lo, const uint32_t* N,
                          const uint32_t* m, int64_t n, double* h, double* t_after, void* stream);

/* Largest store (rows of capacity) that qed_event_step_noalloc accepts. */
#define QED_NOALLOC_MAX_ROWS 65536

/* qed_event_step for callers that cannot allocate device memory: hosts that
 * hand each component a fixed memory budget in advance (an allocation of its
 * own would fail, or take memory promised to another component), and plug-ins
 * living inside another program's memory pool (which must not go around that
 * pool to the CUDA allocator).  No context: the run configuration is passed
 * directly, and the step's scratch (about 2.5 MB) lives in a device array
 * built into this library, which every GPU that loads the library keeps until
 * the process exits.  The paper has no counterpart; this is a packaging of
 * the same step.
 *
 * Same arguments and results as qed_event_step (no event log, no learned
 * sampler: cfg->sampler_mode must be 0), on `stream` (a cudaStream_t, NULL:
 * the legacy default stream); with cfg->cascade_in_step it synchronises that
 * stream after every cascade generation, and if out != NULL at the end.
 * The first call on a device looks up the array and the launch geometry with
 * that device current; later calls on the device reuse them.  The array is shared by every call
 * and keeps the contents of the last one: each step starts by resetting what
 * it reads, but calls whose work overlaps on the GPU (other streams, other
 * host threads) race with each other; serialise them.
 * Calls no cudaMalloc, cudaFree or allocating library routine.
 * Errors: QED_ERR_ARG (bad argument, cfg->sampler_mode != 0, or
 * p->capacity > QED_NOALLOC_MAX_ROWS), QED_ERR_CUDA (the next call on the
 * device then repeats its set-up), and the statuses of qed_event_step. */
qed_status qed_event_step_noalloc(const qed_config* cfg, const qed_particles* p,
                                  uint64_t step_index, void* stream, qed_step_stats* out);

/* Peak probes: the rate, on the current device, of the arithmetic the event
 * kernels run on, for the denominators of their roofline (not part of the
 * paper's method).  Each thread of a full grid runs eight independent chains
 * of one operation for `iters` steps, timed with CUDA events on `stream`
 * (a cudaStream_t, NULL: the default stream) after a short warm-up:
 *   QED_PROBE_MUL32  32 x 32 -> 64-bit multiplies as Philox4x32-10 issues
 *                    them, counting the high and the low word (2 per step)
 *   QED_PROBE_FMA32  binary32 fused multiply-adds, 2 flops per step
 *   QED_PROBE_EX2    special-function exp2 (ex2.approx), 1 per step
 *   QED_PROBE_ALU    integer xor and add, 2 per step
 * *ops_per_s receives operations per second, *ms (nullable) the kernel's
 * time.  Synchronises.  Allocates one word of device memory.
 * Errors: QED_ERR_ARG (kind, iters <= 0, null ops_per_s), QED_ERR_CUDA. */
enum { QED_PROBE_MUL32 = 0, QED_PROBE_FMA32 = 1, QED_PROBE_EX2 = 2, QED_PROBE_ALU = 3 };
qed_status qed_peak_probe(int kind, int64_t iters, double* ops_per_s, double* ms, void* stream);

/* sizeof of a public struct by name ("qed_config", "qed_particles",
 * "qed_host_particles", "qed_step_stats", "qed_event_record"), or 0 for an
 * unknown name.  Host
 * only; lets bindings check their struct mirrors without a GPU. */
size_t qed_abi_struct_size(const char* name);

#ifdef __cplusplus
}
#endif

#endif /* QED_H */
