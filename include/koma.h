/*
 * koma.h - C ABI of libkoma, a CUDA (sm_103a) Bloch simulator.
 *
 * The library computes the complex MR signal of a phantom of independent
 * spins under a discretised pulse sequence, following the KomaMRI.jl paper
 * (Castillo-Passi et al., "KomaMRI.jl: An Open-Source Framework for General
 * MRI Simulations with GPU Acceleration"):
 *   - each spin obeys the Bloch equation in the rotating frame (Eq. Bloch)
 *     with effective field B = (B1x, B1y, G.x + dw/gamma) (Eq. "B definition");
 *   - time is split into steps solved by first-order operator splitting,
 *     rotation then relaxation (Eqs. rotation_Bloch, relax_Bloch);
 *   - steps with RF (B1 != 0) rotate by the Cayley-Klein spinor of the
 *     step's constant field (spinor equations, Eq. Rot_exc); steps without RF
 *     precess about z by the phase integrated with the trapezoid rule over
 *     the step's gradient vertices (Eq. Rotation_precession and the integral
 *     form in Section "Simulation blocks, Regime Switching, and
 *     Sequence-Aware Time Stepping");
 *   - relaxation: Mxy e^{-dt/T2}, Mz e^{-dt/T1} + M0 (1 - e^{-dt/T1});
 *   - the signal at every ADC time point is the sum of Mxy over all spins
 *     (Section "GPU/CPU Parallelization", the sig[t] matrix).
 *
 * Units: SI. Positions m, gradients T/m, B1 T, times s, off-resonance rad/s.
 * gamma = 2 pi x 42.577478518e6 rad/s/T (koma_gamma()).
 *
 * Conventions common to every entry point:
 *   - Return value: KOMA_OK or an error code; on error the call has no
 *     effect on its outputs and koma_last_error(ctx) describes the cause.
 *   - Host pointers ("host") are read synchronously during the call and may
 *     be freed afterwards. Device pointers ("device") are CUDA global-memory
 *     pointers of the context's device, owned by the caller.
 *   - Handles returned through an "out" pointer are owned by the caller and
 *     released with the matching *_free / koma_destroy.
 *   - A context is not thread-safe: use one per host thread or lock around it.
 *   - All entry points are callable without a GPU up to the first CUDA call:
 *     koma_init then fails with KOMA_E_CUDA.
 */
#ifndef KOMA_H
#define KOMA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KOMA_OK = 0,
    KOMA_E_INVALID = 1, /* bad argument (NULL, size, NaN, T1/T2 <= 0, dt <= 0, ...) */
    KOMA_E_NOMEM = 2,   /* device allocation failed or the memory budget is exceeded */
    KOMA_E_CUDA = 3,    /* a CUDA runtime call failed; see koma_last_error */
    KOMA_E_TIMEOUT = 4, /* a bounded device-side wait gave up (see koma_sync) */
    KOMA_E_BUSY = 5,    /* the object is in use by another request */
    KOMA_E_INTERNAL = 6 /* a kernel's own bounds check caught a record pointing outside its
                           launch's buffers (an inconsistent record stream); the access was
                           skipped and the result is not to be used (see koma_sync) */
} koma_status;

typedef enum {
    /* every operation in FP64 on the device */
    KOMA_FP64 = 0,
    /* rotation/relaxation in FP32; accumulated phase carried as a hi/lo FP32
     * pair (FP64-accurate); per-CTA signal sums in FP32, cross-CTA in FP64 */
    KOMA_FP32_SPLITPHASE = 1
} koma_precision;

typedef struct koma_ctx koma_ctx;
typedef struct koma_phantom koma_phantom;
typedef struct koma_sequence koma_sequence;

/* Launch description of the last koma_simulate call on a context (for
 * benchmarking and tests). */
typedef struct {
    int32_t kernels;          /* kernels launched by the call                */
    int32_t grid;             /* CTAs of the Bloch kernel                     */
    int32_t block;            /* threads per CTA                              */
    int32_t spins_per_thread; /* spins each thread steps                      */
    int64_t spins_per_cta;
    int64_t n_records;        /* step records the kernel walked              */
    int64_t partial_bytes;    /* scratch used for per-CTA signal partials     */
    void *bloch_stream;       /* stream the kernels were launched on          */
    int32_t split;            /* CTAs sharing a spin range, dividing its ADC
                                 runs (1: none; used when the spins fill few
                                 warps and sampling dominates the work)     */
    int32_t mma_grid;         /* CTAs of the tensor-core readout (0: not
                                 used by this call)                        */
    int32_t tile_records;     /* step records per shared-memory tile of the
                                 walking kernel                            */
    int32_t phase_mode;       /* how the walking kernel took the phase
                                 2 pi K.x: 0 the hi/lo fractional product;
                                 1 one FP32 product (the dictionary kernel
                                 for isochromats along z, when |z Kz| <= 1
                                 turn for every spin and record)            */
} koma_launch_info;

/* Counts of the uploaded sequence by step class (hot-path cost model). */
typedef struct {
    int64_t n_steps;     /* discretised steps                                 */
    int64_t n_rf;        /* steps with B1 != 0 (excitation regime)            */
    int64_t n_adc;       /* ADC time points                                   */
    int64_t n_precess;   /* steps without RF                                  */
    int64_t n_records;   /* kernel records: RF steps + precession materialise + ADC runs */
    int64_t n_adc_runs;  /* ADC records (each <= 128 uniformly spaced samples) */
    int64_t n_materialize;
    int64_t n_mma_groups; /* groups of ADC runs sharing their per-sample
                             rotator (same dK, dtau), summed as matrix
                             products on the tensor cores (FP32 path)      */
    int64_t n_mma_runs;   /* ADC runs in those groups                       */
    int64_t n_mma_samples; /* ADC samples in those runs                     */
    int64_t n_rf_maps;    /* repeated RF pulses taken by their maps (FP32
                             path): distinct pulses (runs of RF steps that
                             recur unchanged at least 3 times) ...          */
    int64_t n_rf_map_runs;  /* ... their occurrences ...                    */
    int64_t n_rf_map_steps; /* ... the RF steps of those occurrences ...     */
    int64_t n_rf_map_pulse_steps; /* ... and the steps of the distinct pulses
                             (what the map pre-pass steps per spin)          */
    int64_t z_dict;       /* 1: no RF step has a z gradient and every ADC
                             record holds one sample, so a grouped phantom of
                             isochromats along z (x = y = 0, no off-resonance,
                             one T1/T2 per group) takes the dictionary kernel */
    double z_kmax;        /* with z_dict: max |Kz| (turns/m) over the phase
                             records; max |z| x z_kmax <= 1 lets the
                             dictionary kernel take the phase as one FP32
                             product (0 without z_dict)                       */
} koma_sequence_info;

/* gamma used by the library, rad/s/T. */
double koma_gamma(void);

/* Library version string (static storage). */
const char *koma_version(void);

/*
 * Create a context on CUDA device `device`.
 * mem_budget_bytes: upper bound on device memory the context may hold
 *   (phantoms + sequences + scratch); 0 = unlimited.
 * out: receives the context. Errors: KOMA_E_INVALID (out NULL, device < 0),
 *   KOMA_E_CUDA (no such device / no GPU).
 */
koma_status koma_init(int device, size_t mem_budget_bytes, koma_ctx **out);

/* Release the context and its scratch. Phantoms and sequences must be freed
 * first (they hold a reference to the context). NULL is accepted. */
koma_status koma_destroy(koma_ctx *ctx);

/* Text of the last error on ctx ("" if none). Valid until the next call. */
const char *koma_last_error(const koma_ctx *ctx);

/* Device memory currently held by the context's objects, bytes. */
size_t koma_mem_used(const koma_ctx *ctx);

/*
 * Upload a phantom: n spins with (host, FP64, length n each)
 *   x, y, z   position, m                     (Phantom, Section "Overview")
 *   pd        proton density M0, >= 0
 *   t1, t2    relaxation times, s, > 0; +inf means no relaxation
 *   dw        off-resonance, rad/s
 * group_offsets: NULL, or host int64 [n_groups + 1], non-decreasing, from 0
 *   to n: spins [group_offsets[g], group_offsets[g+1]) form signal group g
 *   (e.g. the isochromats of one dictionary entry). NULL => one group.
 * The arrays are copied (and converted to the device layout) synchronously;
 * the library owns the device copy until koma_phantom_free.
 * Errors: KOMA_E_INVALID (NULL pointer, n < 0, non-finite value other than
 *   t1/t2 = +inf, t1 or t2 <= 0, pd < 0, bad group_offsets), KOMA_E_NOMEM,
 *   KOMA_E_CUDA.
 */
koma_status koma_phantom_upload(koma_ctx *ctx, int64_t n,
                                const double *x, const double *y, const double *z,
                                const double *pd, const double *t1, const double *t2,
                                const double *dw, const int64_t *group_offsets,
                                int64_t n_groups, koma_phantom **out);

/* Number of spins / groups of an uploaded phantom (-1 for NULL). */
int64_t koma_phantom_n_spins(const koma_phantom *ph);
int64_t koma_phantom_n_groups(const koma_phantom *ph);

koma_status koma_phantom_free(koma_phantom *ph);

/*
 * Motion (the phantom's motion field u(x, t), Section "Overview", entering
 * the field as G(t).x(t) in Eq. "B definition"; experiment (d) moves the
 * object at a constant 0.1 m/s): give every spin a constant velocity, so
 * that x_j(t) = x_j + v_j t with t measured from t_0 of the sequence.
 *   vx, vy, vz  host FP64 [n] (m/s), finite; all three NULL makes the
 *               phantom static again.
 * Copied synchronously; the library owns the device copy until
 * koma_phantom_free. A moving phantom runs on the motion kernels of
 * koma_simulate (FP32: the phase from t_ref to t is 2 pi (K.x + K1.v + df tau)
 * with the first gradient moment K1 = gammabar * integral of G(s) s ds; an RF
 * step takes the spin's position at the step midpoint; FP64 likewise).
 * koma_simulate_static and the server take static phantoms only.
 * Errors: KOMA_E_INVALID (NULL phantom, one or two NULL arrays, non-finite
 *   velocity), KOMA_E_NOMEM, KOMA_E_CUDA.
 */
koma_status koma_phantom_set_motion(koma_phantom *ph, const double *vx, const double *vy,
                                    const double *vz);

/*
 * Upload a discretised sequence (the DiscreteSequence of Section
 * "Simulation blocks, Regime Switching, and Sequence-Aware Time Stepping")
 * of n_steps steps between time points t_0 .. t_{n_steps}:
 *   dt        host FP64 [n_steps]      step length t_{n+1} - t_n, s, > 0
 *   gx,gy,gz  host FP64 [n_steps + 1]  gradient at each time point, T/m
 *             (piecewise linear between time points)
 *   b1_re, b1_im host FP64 [n_steps]   RF field, T, constant over the step;
 *             a step is in the excitation regime iff b1 != 0
 *   adc       host uint8 [n_steps + 1] 1 = the signal is sampled at t_i
 *             (state after step i-1; t_0 is the initial equilibrium state)
 * The host preprocesses it once (regime classification, FP64 cumulative
 * gradient moments since the last RF step split into hi/lo FP32, uniform
 * ADC runs) into step records and copies them to the device.
 * Errors: KOMA_E_INVALID (NULL, n_steps < 0, dt <= 0 or non-finite,
 *   non-finite G or B1, adc not 0/1), KOMA_E_NOMEM, KOMA_E_CUDA.
 */
koma_status koma_sequence_upload(koma_ctx *ctx, int64_t n_steps, const double *dt,
                                 const double *gx, const double *gy, const double *gz,
                                 const double *b1_re, const double *b1_im,
                                 const uint8_t *adc, koma_sequence **out);

/* Number of ADC samples / steps of an uploaded sequence (-1 for NULL). */
int64_t koma_sequence_n_adc(const koma_sequence *seq);
int64_t koma_sequence_n_steps(const koma_sequence *seq);
/* Step-class counts of an uploaded sequence. */
koma_status koma_sequence_get_info(const koma_sequence *seq, koma_sequence_info *info);

koma_status koma_sequence_free(koma_sequence *seq);

/*
 * Host-only planning (no device, no context): validate a sequence and run
 * the preprocessing of koma_sequence_upload, reporting the step-class
 * counts in `info`. If rec_out is not NULL it receives the FP64 step records,
 * 17 doubles each ([type, count, first sample, 14 payload values]), and
 * rec_capacity (records) must be at least info->n_records. Payload, times
 * relative to the reference time t_ref (end of the last RF step, or t_0):
 *   RF (0):   gammabar dt Gbar (3, turns/m), gammabar dt B1 (2, turns),
 *             dt, t_mid (the step's midpoint time, s)
 *   PREC (1): K (3, turns/m), tau (s), K1 (3, turns s/m)
 *   ADC (2):  K, tau of the first sample, dK (3), dtau, K1 of the first
 *             sample (3), dK1_0 (3): sample l sits at K + l dK,
 *             tau + l dtau, K1 + l dK1_0 + l (l - 1)/2 dtau dK
 * with K = gammabar * integral of G since t_ref and K1 = gammabar *
 * integral of G(s) s ds since t_ref (s absolute time from t_0). Record
 * types: 0 = RF step, 1 = move the reference time (materialise
 * precession), 2 = run of ADC samples. Errors: KOMA_E_INVALID as for
 * koma_sequence_upload, or capacity too small.
 */
koma_status koma_sequence_plan(int64_t n_steps, const double *dt, const double *gx,
                               const double *gy, const double *gz, const double *b1_re,
                               const double *b1_im, const uint8_t *adc,
                               koma_sequence_info *info, double *rec_out, int64_t rec_capacity);

/*
 * Simulate: enqueue the Bloch kernel and the signal reduction on `stream`
 * (a cudaStream_t of the context's device; NULL = legacy default stream).
 * Asynchronous: returns once the work is enqueued.
 *   sig_dev   device FP64 [n_groups][n_adc][2] (interleaved re, im; i.e. a
 *             complex128 [n_groups, n_adc] array), written completely.
 * The context's scratch (per-CTA partial sums, FP32) is grown on demand with
 * cudaMalloc, so the first call for a larger problem is not capturable.
 * Grouped phantoms (n_groups > 1) sum within each group. Many small groups
 * (at most 512 spins per group on average, e.g. the isochromats of MRF
 * dictionary entries) run on the work-item kernel: each group is split into
 * items of at most 32 x (spins per thread) spins, one warp per item, in one
 * persistent launch taking items longest first; larger groups are split into
 * whole CTAs. Both end with a fixed-order per-group sum (deterministic).
 * FP32 path, static ungrouped phantom: the ADC runs of the sequence's
 * matrix-form groups (koma_sequence_info.n_mma_groups > 0: runs sharing
 * their per-sample rotator, e.g. the readout lines of an EPI or a Cartesian
 * scan) are summed by a tensor-core kernel: sample l of run r is
 * sum_s E_s(r) z_s^l (E_s(r) the spin's Mxy at the run's first sample, z_s
 * its per-sample rotator), a complex matrix product over the spins taken in
 * FP16 hi/lo pairs (three products, ~22-bit operands) with FP32
 * accumulation. The Bloch kernel then stores E (8 bytes per spin and run, in
 * the scratch) instead of stepping those samples. koma_set_mma switches this
 * off and on.
 * Errors: KOMA_E_INVALID (NULL handles, objects of another context, bad
 *   precision), KOMA_E_NOMEM (scratch over budget), KOMA_E_CUDA (launch).
 * Device-side waits are bounded; a wait that gives up is reported by the
 * next koma_sync on the context.
 */
koma_status koma_simulate(koma_ctx *ctx, const koma_phantom *ph, const koma_sequence *seq,
                          koma_precision precision, double *sig_dev, void *stream);

/*
 * koma_simulate_static: the KOMA_FP32_SPLITPHASE simulation of koma_simulate
 * for callers that cannot allocate device memory at simulation time - for
 * example a host framework whose allocator has reserved the whole device, a
 * caller that must not trigger cudaMalloc's implicit device synchronisation
 * in a latency-critical loop, or code that has no allocator of its own. The
 * paper has no counterpart to this entry point; it is a deployment variant.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine: the per-CTA
 * partial sums live in a file-scope static device array of 4,194,304 FP32
 * complex values (32 MiB), which every GPU that loads libkoma holds until
 * the process exits.
 *   ph, seq   uploaded objects of one context (ungrouped phantom only)
 *   sig_dev   device FP64 [n_adc][2] (complex128), written completely
 *   stream    cudaStream_t of the context's device (NULL = legacy default)
 * Asynchronous like koma_simulate. The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current)
 * and caches it; make that first call before any stream capture. Every call
 * on a device shares the one array and leaves its contents behind (each
 * call overwrites every entry it reads, so nothing needs clearing): calls
 * whose kernels overlap on the GPU (different streams, no ordering) race
 * and give wrong results - order them on one stream or by events.
 * Errors: KOMA_E_INVALID (NULL handles, objects of different contexts, a
 *   grouped phantom, sig_dev NULL, or a problem needing more partial sums
 *   than the array holds: CTAs x ADC samples > 4,194,304, e.g. more than
 *   256 x 16,384 - use koma_simulate then), KOMA_E_CUDA. Messages via
 *   koma_last_error on the phantom's context.
 */
koma_status koma_simulate_static(const koma_phantom *ph, const koma_sequence *seq,
                                 double *sig_dev, void *stream);

/*
 * Autotune the FP32 launch for this (phantom, sequence) pair: times the
 * candidate configurations on the full problem (grouped phantoms: spins per
 * thread {2, 4} x block {128, 256} x sequence-tile length {64, 128, 256}
 * records of the work-item kernel, plus, for a dictionary of isochromats
 * along z, the dictionary kernel (spins_per_thread 8 in the launch info)
 * with tiles {128, 256} and block 128 (also 256 when it takes the hi/lo
 * phase); otherwise spins per thread {2, 4} of the Bloch kernel) and keeps
 * the fastest on the
 * phantom; later koma_simulate calls with this sequence use it. The choice
 * is also cached on the context by problem shape (kernel family and the
 * powers of two of spins, groups, records, ADC samples and RF steps), and
 * untuned launches of a cached shape use it. Synchronous (waits on
 * `stream`); overwrites sig_dev (device FP64 [n_groups][n_adc][2]).
 * chosen: NULL or receives the chosen launch. Errors as koma_simulate.
 */
koma_status koma_tune(koma_ctx *ctx, const koma_phantom *ph, const koma_sequence *seq,
                      double *sig_dev, void *stream, koma_launch_info *chosen);

/*
 * Self-check of the device-side timeout path (no counterpart in the paper).
 * Enqueues on `stream` a one-thread kernel that waits, with the bounded wait
 * the Bloch kernels use for their record tiles, on a barrier that nothing
 * completes; after limit_us microseconds (1 .. 2,000,000) it gives up and
 * sets the context's status word. The next koma_sync on the stream then
 * returns KOMA_E_TIMEOUT (clearing the word), and the context stays usable.
 * It faults and hangs nothing: the wait is bounded by the device's global
 * timer. Errors: KOMA_E_INVALID (limit out of range), KOMA_E_CUDA (launch).
 */
koma_status koma_check_bounded_wait(koma_ctx *ctx, int64_t limit_us, void *stream);

/*
 * Wait for `stream` and report device-side status: KOMA_E_TIMEOUT if a
 * bounded wait inside a kernel of this context gave up since the last
 * koma_sync, KOMA_E_INTERNAL if a kernel skipped a record that pointed
 * outside its buffers (an ADC run past the signal's end or out of order, a
 * map slot or readout snapshot row out of range: the kernels check every
 * index they take from a record before using it); the flags are then
 * cleared. KOMA_E_CUDA on an asynchronous CUDA error, else KOMA_OK.
 */
koma_status koma_sync(koma_ctx *ctx, void *stream);

/*
 * Kernel timing. With enable != 0, every later koma_simulate on ctx records
 * CUDA events on its stream before the Bloch kernel, after it, after the
 * tensor-core readout, and after the reduction. koma_get_timing waits for the last
 * call's final event and returns the two durations in milliseconds.
 * Errors: KOMA_E_INVALID (NULL, or no timed call yet), KOMA_E_CUDA.
 */
koma_status koma_set_timing(koma_ctx *ctx, int enable);
koma_status koma_get_timing(koma_ctx *ctx, float *bloch_ms, float *reduce_ms);
/* The same call split into its three stages: the Bloch kernel, the
 * tensor-core readout (0 when the call did not launch it) and the
 * reduction; bloch_ms + mma_ms is koma_get_timing's bloch_ms. */
koma_status koma_get_stage_timing(koma_ctx *ctx, float *bloch_ms, float *mma_ms, float *reduce_ms);

/* Matrix-form (tensor-core) readout on (enable != 0, the default) or off:
 * off, every ADC sample is stepped by the Bloch kernel. Errors:
 * KOMA_E_INVALID (NULL). */
koma_status koma_set_mma(koma_ctx *ctx, int enable);

/* Maps of repeated RF pulses on (enable != 0, the default) or off. On, the
 * FP32 path of koma_simulate (static phantoms, Bloch kernel) first computes
 * for every spin and every repeated pulse (koma_sequence_info.n_rf_maps) the
 * affine map M -> A M + c of the whole pulse - the composition of its steps'
 * rotations (Eq. Rot_exc) and relaxations, stepped in FP32 by a pre-pass
 * kernel (8 bytes x 6 per spin and pulse of scratch) - and the Bloch kernel
 * applies it at each occurrence instead of stepping the pulse again. Off,
 * every RF step is stepped. Errors: KOMA_E_INVALID (NULL). */
koma_status koma_set_rf_maps(koma_ctx *ctx, int enable);

/* Duration (ms) of the map pre-pass of the last timed koma_simulate on ctx
 * (0 if that call had none; koma_get_stage_timing's bloch_ms includes it).
 * Errors: KOMA_E_INVALID (NULL, or no timed call yet), KOMA_E_CUDA. */
koma_status koma_get_map_timing(koma_ctx *ctx, float *maps_ms);

/* Launch description of the last koma_simulate or koma_simulate_static on
 * ctx (after a static call, koma_get_timing reports no timed call: that entry
 * point records no stage events). */
koma_status koma_get_launch_info(const koma_ctx *ctx, koma_launch_info *info);

/*
 * One call from host arrays to host signal (end-to-end path): uploads the
 * phantom and the sequence, simulates on the context's internal stream,
 * copies the signal to `sig_host` (host FP64 [n_groups][n_adc][2]) and
 * frees the uploads. Synchronous. Arguments as for the three calls above.
 */
koma_status koma_simulate_host(koma_ctx *ctx, int64_t n,
                               const double *x, const double *y, const double *z,
                               const double *pd, const double *t1, const double *t2,
                               const double *dw, const int64_t *group_offsets, int64_t n_groups,
                               int64_t n_steps, const double *dt, const double *gx,
                               const double *gy, const double *gz, const double *b1_re,
                               const double *b1_im, const uint8_t *adc,
                               koma_precision precision, double *sig_host);

/* One simulation of a batch of host-buffer calls: the arguments of
 * koma_simulate_host after ctx (arrays borrowed for the duration of the batch
 * call; the caller owns them and sig_host). */
typedef struct {
    int64_t n;                      /* spins                                      */
    const double *x, *y, *z;        /* [n] positions (m)                          */
    const double *pd, *t1, *t2;     /* [n] proton density, T1, T2 (s)             */
    const double *dw;               /* [n] off-resonance (rad/s)                  */
    const int64_t *group_offsets;   /* NULL or [n_groups + 1]                     */
    int64_t n_groups;
    int64_t n_steps;                /* sequence, as for koma_sequence_upload       */
    const double *dt, *gx, *gy, *gz, *b1_re, *b1_im;
    const uint8_t *adc;
    double *sig_host;               /* out: host FP64 [n_groups][n_adc][2]        */
} koma_host_job;

/*
 * koma_simulate_host for each of jobs[0 .. n_jobs), with one job's host
 * work (checks, preprocessing of its sequence, uploads) overlapped with the
 * previous job's simulation on the device: jobs alternate between ctx and a
 * second context on the same device that the first batch call creates and
 * ctx keeps (same memory budget; destroyed with ctx). Every job's inputs are
 * copied to the device and its signal copied back, as in koma_simulate_host;
 * results are identical to one koma_simulate_host per job. Synchronous: all
 * signals are in place on return. Errors: as koma_simulate_host, the first
 * failing job's (jobs after it are not run; the message is ctx's), and
 * KOMA_E_INVALID for n_jobs < 0 or jobs NULL with n_jobs > 0.
 */
koma_status koma_simulate_host_batch(koma_ctx *ctx, int64_t n_jobs, const koma_host_job *jobs,
                                     koma_precision precision);

/* ------------------------------------------------------------------------
 * Serving: a continuous-batching simulation server.
 *
 * Not in the paper: a deployment form of the same simulation. A server owns
 * worker threads on one device. Submitted requests (host phantom, optionally
 * grouped, + host sequence: the arrays and checks of koma_phantom_upload and
 * koma_sequence_upload) are admitted in arrival order while the server's
 * device-memory budget allows. Two lanes share the GPU:
 *   - small ungrouped requests share launches of one persistent kernel that
 *     steps 512-spin batches of every admitted request (shortest remaining
 *     work first, two launches in flight), so requests arriving while others
 *     run join within one launch. A batch walks its sequence in chunks of
 *     step records, its spin state checkpointed in device memory between
 *     launches, so a long simulation never holds the GPU for long; repeated
 *     RF pulses are applied through their maps;
 *   - requests with at least `plain_spins` spins and grouped requests (a
 *     dictionary: one signal per group) run the koma_simulate path (maps of
 *     repeated pulses, the tensor-core readout, the grouped kernel) on four
 *     lane threads with a context and a stream each: one request's upload
 *     overlaps other requests' kernels, and requests that do not fill the
 *     GPU run side by side, next to the shared launches.
 * A request's result (KOMA_FP32_SPLITPHASE arithmetic) does not depend on
 * the other requests: it is bitwise the same alone and in any mix.
 * ---------------------------------------------------------------------- */
typedef struct koma_server koma_server;

typedef struct {
    int device;              /* CUDA device                                   */
    int max_active;          /* admitted requests at once; 0 = 64             */
    size_t mem_budget_bytes; /* device memory for admitted requests; 0 = none */
    double launch_work;      /* work per launch, RF spin-step units; 0 = default (~4 ms) */
    int64_t chunk_records;   /* a batch walks at most this many step records per launch and is
                                checkpointed between launches (long sequences do not hold the GPU);
                                0 = 4096 */
    int64_t plain_spins;     /* requests with at least this many spins run the koma_simulate
                                path in the server's second lane; 0 = 524288, < 0 = never
                                (grouped requests always do) */
} koma_server_config;

typedef struct {
    uint64_t id;
    int64_t n_spins, n_steps, n_adc;
    double submit_s, admit_s, done_s; /* seconds since the server started      */
    double latency_s;                 /* submit (incl. preprocessing) to result */
    int32_t launches;                 /* launches the request took part in (shared kernel launches,
                                         or 1 for the koma_simulate lane)       */
    koma_status status;
    int64_t n_groups;                 /* signal groups (1: ungrouped)           */
    int32_t lane;                     /* 0: shared launches, 1: koma_simulate lane */
    double prep_s;                    /* host time of the submit call (checks, preprocessing, copies) */
    double upload_s;                  /* koma_simulate lane: uploads (0 in the shared lane) */
    double run_s;                     /* koma_simulate lane: simulate, copy-back and wait (0 in the
                                         shared lane) */
} koma_request_info;

typedef struct {
    int64_t submitted, completed, failed, pending, active, launches, batches;
    size_t mem_used, mem_peak;
    int64_t lane_runs;  /* requests run by the koma_simulate lane */
} koma_server_stats;

/* Create a server (cfg NULL: device 0, defaults). Errors: KOMA_E_INVALID,
 * KOMA_E_CUDA (no device), KOMA_E_NOMEM. */
koma_status koma_server_create(const koma_server_config *cfg, koma_server **out);

/* Submit one simulation; validates and preprocesses on the calling thread,
 * then returns its id. group_offsets / n_groups as koma_phantom_upload (NULL:
 * one group). Requests of the shared lane keep no host arrays. For those of
 * the koma_simulate lane the calling thread copies the phantom into device
 * memory, where the conversion kernel checks every spin and builds the FP32
 * block (counted against the memory budget from then on); if the budget has
 * no room for it yet, the spins are checked on the host and a host copy is
 * kept until the lane uploads it. The sequence arrays are copied and checked
 * on the host. Thread-safe. Errors: KOMA_E_INVALID (as the uploads; message
 * via koma_server_last_error), KOMA_E_NOMEM, KOMA_E_CUDA, KOMA_E_BUSY (server
 * shutting down). */
koma_status koma_server_submit(koma_server *srv, int64_t n, const double *x, const double *y,
                               const double *z, const double *pd, const double *t1,
                               const double *t2, const double *dw, const int64_t *group_offsets,
                               int64_t n_groups, int64_t n_steps, const double *dt,
                               const double *gx, const double *gy, const double *gz,
                               const double *b1_re, const double *b1_im, const uint8_t *adc,
                               uint64_t *id_out);

/* Wait (timeout_s < 0: forever) for request `id`; on success writes its
 * signal to sig_host (host FP64 [n_groups][n_adc][2], capacity >= n_groups x
 * n_adc entries) and
 * `info` (may be NULL), then forgets the request. Errors: KOMA_E_TIMEOUT
 * (still running; call again), KOMA_E_INVALID (unknown id or capacity),
 * KOMA_E_NOMEM (larger than the whole budget), KOMA_E_CUDA, KOMA_E_BUSY
 * (shut down before admission). Thread-safe. */
koma_status koma_server_wait(koma_server *srv, uint64_t id, double timeout_s, double *sig_host,
                             int64_t capacity, koma_request_info *info);

koma_status koma_server_get_stats(koma_server *srv, koma_server_stats *out);
const char *koma_server_last_error(const koma_server *srv);

/* Finish admitted work, fail requests never admitted, release everything.
 * No wait may be in progress. */
koma_status koma_server_destroy(koma_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* KOMA_H */
