/*
 * rbm.h - C ABI of the GB300 (sm_103a) Random Batch Method library.
 *
 * The library advances an interacting particle system (Jin, Li & Liu,
 * arXiv:1812.10575, Sec. 1, eq. "interactingps")
 *
 *     dX^i = -grad V(X^i) dt + 1/(N-1) sum_{j != i} K(X^i - X^j) dt + sigma dB^i
 *
 * by RBM-1 (Sec. 2.1, Algorithm "randomdiv": each step a fresh random division
 * of the N particles into batches of size p, the interaction replaced by
 * 1/(p-1) times the in-batch sum, one Euler-Maruyama step) or by the direct
 * O(N^2) forward-Euler step the paper compares it with (Sec. 4.1).  All work
 * runs in the library's own CUDA kernels on the caller's stream.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Positions: row-major N x ld array of the run's dtype in device memory, with
 *   ld = d for d = 1, 2 and ld = 4 for d = 3 (the fourth lane is padding; the
 *   library preserves its bits).  The base address must be 16-byte aligned.
 *   The caller owns it and keeps it alive until rbm_free.
 * Stream: every call enqueues work on the stream given to rbm_init (a
 *   cudaStream_t passed as void*, NULL = the legacy default stream) and
 *   returns without waiting, except rbm_sync, rbm_step_host and the calls
 *   documented as synchronous.
 * Randomness: counter-based Philox4x32-10 keyed by the 64-bit seed.  Counter
 *   (id, m mod 2^32, replica, stream*256 + call): stream 0 gives the
 *   permutation key of particle id at step m, (w1 << 32) | w0; stream 1,
 *   call t, gives Box-Muller pair t of particle id's Brownian increment.  The
 *   increment depends on (id, m) only, so RBM and direct steps from the same
 *   state share it (the synchronous coupling of Sec. 3, eq. "coupling").
 *   Uniforms take the top 53 bits (FP64 runs) or 24 bits (FP32 runs) of each
 *   64-bit word w: u = ((w >> (64-b)) + 1) * 2^-b, in (0, 1].
 * Random division: particle ids sorted ascending by (key, id); batch q is
 *   sorted positions [q p, min(q p + p, N)).  The last batch has N mod p
 *   members when p does not divide N; a singleton batch feels no interaction.
 * K(0) := 0 for every kernel (coincident particles exert no force).
 * Errors: parameter errors return synchronously (RBM_ERR_INVALID, nothing is
 *   enqueued).  Device-side conditions (a non-finite position, a bounded wait
 *   that ran out) are latched in a device status word and returned by
 *   rbm_sync (and by the next rbm_step_host).  After any error other than
 *   RBM_ERR_INVALID the context accepts only rbm_get_step, rbm_sync and
 *   rbm_free.
 * Threads: a context is not thread-safe; distinct contexts are independent.
 */
#ifndef RBM_H
#define RBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rbm_ctx rbm_ctx; /* opaque; owned by the library */

typedef enum {
    RBM_OK = 0,
    RBM_ERR_INVALID = -1,     /* bad parameter or pointer; nothing enqueued   */
    RBM_ERR_CUDA = -2,        /* a CUDA runtime call failed                   */
    RBM_ERR_NOMEM = -3,       /* device or pinned allocation failed           */
    RBM_ERR_TIMEOUT = -4,     /* a bounded device-side wait ran out           */
    RBM_ERR_NONFINITE = -5,   /* a step produced a NaN or infinite position   */
    RBM_ERR_STATE = -6,       /* context unusable after an earlier error      */
    RBM_ERR_UNSUPPORTED = -7  /* valid request this build does not implement  */
} rbm_status;

typedef enum { RBM_F32 = 0, RBM_F64 = 1 } rbm_dtype;

/* Confining potential V (Sec. 1). */
typedef enum {
    RBM_V_ZERO = 0,      /* V = 0                                 */
    RBM_V_QUADRATIC = 1  /* V = v_coef |x|^2 / 2, -grad V = -v_coef x */
} rbm_potential;

/* Interaction kernel K, x = X^i - X^j (the paper's examples, Secs. 4-5). */
typedef enum {
    RBM_K_INV1D = 0,        /* 1/x, d = 1 only (Dyson Brownian motion, Sec. 4.2) */
    RBM_K_COULOMB = 1,      /* x/|x|^3 (Thomson problem, Sec. 5.1)              */
    RBM_K_BOUNDED_CONF = 2, /* -x if |x| < k_param else 0 (opinions, Sec. 5.2)  */
    RBM_K_GAUSS_AGG = 3,    /* -x exp(-|x|^2/2)                                  */
    RBM_K_REG_ATTRACT = 4,  /* -x / (|x|^2 + k_param)                            */
    RBM_K_SMOOTH_TEST = 5,  /* x / (1 + |x|^2) (test example, Sec. 4.1)          */
    RBM_K_LINEAR = 6        /* -k_param x                                        */
} rbm_kernel;

typedef enum {
    RBM_METHOD_RBM = 0,       /* RBM-1 step (Algorithm "randomdiv")            */
    RBM_METHOD_DIRECT = 1,    /* direct O(N^2) forward-Euler step (Sec. 4.1)   */
    RBM_METHOD_SURROGATE = 2, /* learned mean-field force with the RBM-1 step
                                 as fallback (see rbm_surrogate_config)        */
    RBM_METHOD_RBMR = 3       /* RBM-r: floor(N/p) iterations per step of
                                 Algorithm "fullyrandom" (see below)           */
} rbm_method;

/* Time scheme of the RBM step. */
typedef enum {
    RBM_SCHEME_EULER = 0, /* explicit Euler-Maruyama of eq. "firstalgorithm" */
    RBM_SCHEME_SPLIT = 1, /* splitting, Sec. 2.3 item 5: the p = 2 pair flow of
                             K solved exactly (K = 1/x: |delta|^2 += 4 dt;
                             K = x/|x|^3: |delta|^3 += 6 dt, Secs. 4.2, 5.1),
                             then Euler-Maruyama for -grad V and the noise.
                             K = LINEAR (-c x): the gap shrinks by
                             exp(-2 c dt) about the fixed mean (the wealth
                             model's exchange, Sec. 5.2).
                             Requires p = 2 and K = INV1D, COULOMB or LINEAR. */
    RBM_SCHEME_VERLET = 2 /* the second-order system of Appendix A (eq.
                             "Hamil1": dX = V dt, dV = (-grad V + interaction)
                             dt) by the Verlet scheme of Sec. 4.1: X_1 = X_0 +
                             dt V_0 + dt^2 F_0 / 2, X_{n+1} = 2 X_n - X_{n-1}
                             + dt^2 F_n, F_n from the RBM-1 batches of step n
                             (eq. "Hamilrand") or the full sum.  Requires
                             sigma = 0, no projection, p <= 32, and
                             rbm_verlet_set_velocity before the first step. */
} rbm_scheme;

#define RBM_FLAG_RENORM_SPHERE 1u /* X^i <- X^i/|X^i| after each step (Sec. 5.1) */
#define RBM_FLAG_GBM_NOISE 2u     /* multiplicative noise sigma X^i dB^i (the wealth
                                     model, Sec. 5.2, eq. "wealth"): the Euler-
                                     Maruyama term becomes sigma sqrt(dt) X z; with
                                     RBM_SCHEME_SPLIT the noise sub-step is the exact
                                     geometric flow X exp(-sigma^2 dt/2 + sigma
                                     sqrt(dt) z)                                    */

typedef struct {
    int64_t n;        /* particles N >= 2                                    */
    int32_t d;        /* dimension 1..3                                      */
    int32_t p;        /* batch size, 2 <= p <= min(N, 4096)                  */
    double dt;        /* time step tau > 0                                   */
    double sigma;     /* noise amplitude >= 0                                */
    uint64_t seed;    /* Philox key                                          */
    int32_t dtype;    /* rbm_dtype                                           */
    int32_t v;        /* rbm_potential                                       */
    double v_coef;    /* V coefficient                                       */
    int32_t k;        /* rbm_kernel                                          */
    double k_param;   /* kernel parameter (radius, epsilon or coefficient)   */
    uint32_t flags;   /* RBM_FLAG_*                                          */
    int32_t scheme;   /* rbm_scheme                                          */
    uint32_t replica; /* replica index r used in the Philox counter          */
} rbm_params;

/* Optional launch and scratch tuning (zero = library default). */
typedef struct {
    int32_t bucket_bits;  /* log2 of the number of permutation buckets (the
                             record path: of sub-buckets)                      */
    int32_t slot_cap;     /* slots per bucket before spilling to the overflow
                             list (path 1) or regrouping every id compactly
                             behind one more grid barrier (path 2, at most
                             and by default 2048)                              */
    int32_t sort_cap;     /* largest bucket sorted in shared memory (power of 2) */
    int32_t block;        /* threads per block of the fused step kernel      */
    int32_t direct_block; /* threads per block of the direct kernel          */
    int32_t graph_steps;  /* steps captured per CUDA graph by rbm_run        */
    int32_t path;         /* RBM step: 0 automatic (3 up to 1536 particles in
                             FP32 / 384 in FP64, 2 up to about 1.7 million,
                             beyond that 4 where it applies, else 1), 1
                             bucket-sort kernels, 2 one cooperative kernel (N
                             up to about 8 million, p <= 32), 3 one block for
                             the whole system (N <= 2048, p <= 32), 4 the
                             record path (FP32, d = 3, p <= 32, not Verlet:
                             the positions move through the steps of one call
                             as bucketed records and are written back to
                             x_dev after the call's last step); a path that
                             does not fit falls back to 1                       */
    int32_t wait_limit_us;/* bound of a grid-barrier wait in the cooperative
                             kernel (0 = 1 second); a wait that runs out
                             latches RBM_ERR_TIMEOUT                           */
    int32_t test_skip_arrival; /* test hook, 0 or 1: the next cooperative
                             step first waits at a grid barrier that block 0
                             leaves without arriving at, so the other blocks'
                             bounded waits run out (exercises RBM_ERR_TIMEOUT) */
} rbm_tuning;

/* Create a context for one particle system whose positions live at x_dev
 * (layout above).  Allocates all scratch on the device (permutation buckets,
 * the permutation, a second position buffer, the status word).  *out is set
 * on success.  Synchronous with respect to the host (allocations). */
rbm_status rbm_init(const rbm_params *prm, void *x_dev, void *cuda_stream, rbm_ctx **out);

/* One RBM-1 step m -> m+1 (Algorithm "randomdiv", eq. "firstalgorithm"),
 * in place: keys, random division, in-batch forces, -grad V, noise, update. */
rbm_status rbm_step(rbm_ctx *ctx);

/* One direct forward-Euler step m -> m+1 (the O(N^2) reference method of
 * Sec. 4.1, eq. "interactingps"), same noise as rbm_step at step m. */
rbm_status rbm_direct_step(rbm_ctx *ctx);

/* `steps` steps of `method`, launched as CUDA graphs of graph_steps steps
 * (captured on first use, replayed afterwards) plus eager remainder steps.
 * On the bucket-sort path (1) each RBM step's sort kernel also buckets the
 * ids of the next step (the random division depends on the step index
 * only), so a graph needs one bucket-scatter launch, before its first step,
 * and none when the previous call ended at the same step index. */
rbm_status rbm_run(rbm_ctx *ctx, int64_t steps, int32_t method);

/* End to end from host memory: copy N x ld positions from x_host (pinned for
 * speed, pageable accepted) to the context's device positions, take one step
 * of `method`, copy them back to x_host and wait.  Returns latched errors.
 * Up to 16 MB of pinned positions are moved by a copy kernel through the
 * mapped host address.  On the record path (path 4) larger buffers are moved
 * in eight chunks on a second stream the context creates on first use: each
 * chunk of rows is scattered as soon as it lands, and after the step each
 * contiguous range of ids is copied back as soon as its rows are placed.
 * The device positions hold the new step too on return. */
rbm_status rbm_step_host(rbm_ctx *ctx, void *x_host, int32_t method);

rbm_status rbm_get_step(const rbm_ctx *ctx, int64_t *m);
rbm_status rbm_set_step(rbm_ctx *ctx, int64_t m);

/* One Brownian path across step sizes: with refinement r the Brownian
 * increment of step m is the normalised sum of the r increments that a run
 * with step dt/r draws over the same interval,
 *     z_i = r^(-1/2) sum_{k=0}^{r-1} z_i(fine step m r + k),
 * so that sqrt(dt) z_i is that run's sqrt(dt/r) sum_k z_i(m r + k).  Runs of
 * the same system with steps dt and dt/r (refinements r q and q) are then
 * driven by the same B^i - the synchronous coupling of Sec. 3 (eq.
 * "coupling") extended to the fine-step reference the paper measures errors
 * against (Sec. 4.1) - and their difference is the time-stepping and
 * random-batch error alone, without sampling noise.  r = 1 (the default) is
 * the plain draw.  Applies to rbm_step, rbm_direct_step, rbm_run,
 * rbm_step_host (RBM-1, direct, surrogate; single and batched contexts);
 * RBM-r steps return RBM_ERR_UNSUPPORTED while r > 1.  Each step draws r
 * Box-Muller sets per particle.  1 <= r <= 65536, else RBM_ERR_INVALID.
 * Synchronous (waits for the stream; captured graphs are rebuilt). */
rbm_status rbm_set_noise_refinement(rbm_ctx *ctx, int32_t r);
rbm_status rbm_get_noise_refinement(const rbm_ctx *ctx, int32_t *r);

/* Set launch/scratch tuning; reallocates scratch.  Synchronous. */
rbm_status rbm_set_tuning(rbm_ctx *ctx, const rbm_tuning *tuning);
rbm_status rbm_get_tuning(const rbm_ctx *ctx, rbm_tuning *tuning);

/* Wait for the stream and return the latched device status. */
rbm_status rbm_sync(rbm_ctx *ctx);

/* Release the context and its scratch (waits for the stream first). */
rbm_status rbm_free(rbm_ctx *ctx);

/* Human-readable name of a status code (static storage). */
const char *rbm_status_string(int32_t status);

/* Text of the last CUDA runtime failure seen by the calling thread (the call
 * and the runtime's message), or "" if none.  Thread-local, static storage. */
const char *rbm_last_error(void);

/* ---- second-order system (RBM_SCHEME_VERLET) --------------------------- */
/* Velocities V_0 (N x ld, run dtype, device, copied) at the current step m:
 * the next step (rbm_step, rbm_direct_step, rbm_run) is the Taylor start,
 * the ones after it the two-step recurrence (the Taylor start is the step
 * whose index equals the current m modulo 2^32).  The context keeps X_{n-1}
 * in a buffer of its own.  Synchronous.  RBM_ERR_STATE when the scheme is not
 * Verlet. */
rbm_status rbm_verlet_set_velocity(rbm_ctx *ctx, const void *v_dev);

/* The Verlet buffer for checkpoint/resume: X_{n-1} (or V_0 while the Taylor
 * start is pending, *taylor_pending = 1) into prev_dev (N x ld, device);
 * set_previous restores it at the current step m.  Synchronous. */
rbm_status rbm_verlet_get_previous(rbm_ctx *ctx, void *prev_dev, int32_t *taylor_pending);
rbm_status rbm_verlet_set_previous(rbm_ctx *ctx, const void *prev_dev, int32_t taylor_pending);

/* ---- RBM-r (Sec. 2.2, Algorithm "fullyrandom") --------------------------- */
/* One step of RBM_METHOD_RBMR (rbm_run, rbm_step_host, rbm_step_profiled) is
 * K = floor(N/p) (at least 1) iterations k = m K .. m K + K - 1, in order:
 * iteration k draws p distinct ids (Philox4x32-10 blocks at counters
 * (k mod 2^32, k div 2^32, replica, 7*256 + c), words in order, id =
 * floor(w N / 2^32), repeats skipped, slots in draw order) and moves each
 * member i by X^i += dt (1/(p-1) sum_{j in C, j != i} K(X^i - X^j) - grad V)
 * + sigma sqrt(dt) z, z of slot s from the blocks (k mod 2^32, k div 2^32,
 * replica, 8*256 + 2 s + t), all forces from the positions before the
 * iteration.  The GPU runs disjoint iterations together in rounds that keep
 * every particle's iterations in order, so the result is the sequential one.
 * Requires p <= 32, the Euler scheme, additive noise, a single (not batched)
 * system.  The first RBM-r call allocates about N (16 + 9 p / p) bytes of scratch. */

/* The sets of step m (K x p uint32 ids, slot order) into sets_dev (device,
 * caller-owned, K p entries).  Does not advance m. */
rbm_status rbm_rbmr_sets(rbm_ctx *ctx, int64_t m, uint32_t *sets_dev);

/* Iterations per step and the number of rounds the last RBM-r step took
 * (0 before the first).  Synchronous. */
rbm_status rbm_rbmr_info(rbm_ctx *ctx, int64_t *iterations_per_step, int32_t *rounds_last);

/* ---- diagnostics (same conventions; used by the tests) ------------------ */

/* The random division of the current step m as the sorted id list: writes N
 * uint32 ids to perm_dev (device, caller-owned).  Does not advance m. */
rbm_status rbm_permutation(rbm_ctx *ctx, uint32_t *perm_dev);

/* Interaction force only, F^K_i (no -grad V, no noise, no update) of the
 * current step m into f_dev (N x ld, run dtype): the in-batch sum scaled by
 * 1/(|C|-1) for RBM_METHOD_RBM, the full sum scaled by 1/(N-1) for
 * RBM_METHOD_DIRECT.  Does not advance m. */
rbm_status rbm_forces(rbm_ctx *ctx, int32_t method, void *f_dev);

/* Mean-field force at nq query points q_dev (nq x ld, run dtype):
 * F(q) = 1/(N-1) sum_j K(q - X^j) over all particles, into f_dev. */
rbm_status rbm_direct_forces_at(rbm_ctx *ctx, const void *q_dev, int64_t nq, void *f_dev);

/* One step of `method` (m -> m+1; on the record path, path 4, two steps
 * m -> m+2, so that the kernels of a run's inner steps appear besides those
 * of its last step) with a CUDA event recorded on the
 * context's stream before and after each kernel it launches; waits for the
 * step and writes each kernel's duration in milliseconds to kernel_ms (up to
 * `capacity` entries), their number to *nkernels and, when `names` is given,
 * their ';'-separated names (NUL-terminated, truncated to names_len).
 * Synchronous.  Used by the benchmark to time kernels on their own stream. */
rbm_status rbm_step_profiled(rbm_ctx *ctx, int32_t method, float *kernel_ms, int32_t capacity, int32_t *nkernels,
                             char *names, int32_t names_len);

/* The latency floor of the cooperative RBM-1 step's launch shape: the mean
 * time (microseconds, 20 back-to-back launches after one warm-up, CUDA events
 * on the context's stream) of the same cooperative launch (grid, block,
 * dynamic shared memory) doing nothing: a step in the common case (no
 * bucket overflow, no general mode) waits at no grid barrier.  The
 * benchmark sets it beside the step kernel's time.  RBM_ERR_STATE when the
 * context does not use the cooperative kernel.  Synchronous. */
rbm_status rbm_latency_floor(rbm_ctx *ctx, float *us);

/* ---- learned mean-field surrogate ---------------------------------------- */
/* The paper has no surrogate.  Its mean-field limit (Sec. 1, eq.
 * "nonlinearfp") drives each particle by the force K * mu; here a
 * d -> 64 -> 64 -> d tanh network F(x) (d = 2 or 3) is trained on the direct-sum force
 * F(x) = 1/(N-1) sum_j K(x - X^j) at sampled particles and, while its held-out
 * relative error stays at or below `fallback_tol`, replaces the random-batch
 * force in the Euler-Maruyama step (-grad V and the Brownian increment as in
 * rbm_step); otherwise the RBM-1 step runs.  The choice is a device-side flag
 * set at each checkpoint; no host synchronisation is involved.
 *   network: xh = (x - mu)/s, h1 = tanh(W1 xh + b1), h2 = tanh(W2 h1 + b2),
 *            F = sF (W3 h2 + b3); weights read as bfloat16; the 64 x 64
 *            products on the tensor cores with FP32 accumulation;
 *   training: MSE on F/sF, Adam (beta 0.9, 0.999, eps 1e-8), FP32 masters,
 *            minibatches of 4096 of the 3/4 training share of the queries,
 *            in round r (0-based) of a checkpoint the rate decays
 *            geometrically from lr/2^r to lr/(100 2^r);
 *   checkpoint (every `train_every` steps, and before the first step):
 *            n_queries particle ids drawn by Philox (id q, step m, stream 2),
 *            direct forces at them, mu, s, sF fixed at the first checkpoint
 *            (unless given by rbm_surrogate_set_params),
 *            a round of iters_first (first checkpoint) or
 *            iters_per_checkpoint Adam steps, the error on the held-out
 *            quarter = ||F_net - F||_2 / ||F||_2, then further rounds of
 *            iters_per_checkpoint while that error is above fallback_tol, at
 *            most max_rounds rounds in all (the error is read back after each
 *            round: the only host synchronisation of the method);
 *   drift:   the network goes stale as the particles move, so each
 *            checkpoint after the first also measures the error of the network
 *            as it stood, on the fresh queries, before retraining: the error
 *            over the interval it just drove.  Above fallback_tol the next
 *            interval is halved (down to max(1, train_every / 16)); at that
 *            shortest interval the steps go to the RBM-1 fallback until a
 *            checkpoint measures the drift within the tolerance again; at or
 *            below half the tolerance the interval doubles back towards
 *            train_every (rbm_surrogate_drift reports the schedule).
 * Requires d = 2 or 3, FP32, the Euler scheme, additive noise, a single (not
 * batched) system.
 * Synchronous (allocates the network state). */
rbm_status rbm_surrogate_config(rbm_ctx *ctx, int32_t train_every, double fallback_tol, int64_t n_queries,
                                int32_t iters_first, int32_t iters_per_checkpoint, int32_t max_rounds, double lr);

/* One checkpoint round now (sample, direct forces, `iters` Adam steps, error). */
rbm_status rbm_surrogate_train(rbm_ctx *ctx, int32_t iters);

/* Last held-out relative error, steps taken by the network and by the RBM
 * fallback so far, whether the network is selected, and the Adam iterations
 * run so far.  Any output pointer may be NULL.  Synchronous. */
rbm_status rbm_surrogate_stats(rbm_ctx *ctx, double *last_rel_err, int64_t *n_surrogate_steps,
                               int64_t *n_fallback_steps, int32_t *active, int64_t *n_adam_steps);

/* The drift-aware schedule: the last drift error (-1 before the second
 * checkpoint), the current interval between checkpoints in steps, whether the
 * last checkpoint handed the steps to the RBM-1 fallback for drift, and how
 * many intervals it has done so.  Any output pointer may be NULL.  Host state
 * only (does not wait). */
rbm_status rbm_surrogate_drift(const rbm_ctx *ctx, double *drift_err, int32_t *interval, int32_t *forced_off,
                               int64_t *n_forced_intervals);

/* Network parameters (4224 + 129 d floats, 4482 for d = 2 and 4611 for
 * d = 3: W1[64][d], b1[64], W2[64][64], b2[64], W3[d][64], b3[d]) and
 * normalisation (d + 2 floats: mu (d values), s, sF), host buffers;
 * set_params also clears the Adam state.  Synchronous. */
rbm_status rbm_surrogate_params(rbm_ctx *ctx, float *theta_host, float *norm_host);
rbm_status rbm_surrogate_set_params(rbm_ctx *ctx, const float *theta_host, const float *norm_host);

/* Network force at nq points q_dev (nq x ld FP32 rows, device; ld = 2 for
 * d = 2, 4 for d = 3) into f_dev (same layout). */
rbm_status rbm_surrogate_forces(rbm_ctx *ctx, const void *q_dev, int64_t nq, void *f_dev);

/* Loss and its gradient (host, 4224 + 129 d floats) on nb samples: positions
 * x_dev and target forces f_target_dev (nb x ld FP32 rows, device), nb <= 65536; the
 * network's own tensor-core kernels, no update.  Synchronous. */
rbm_status rbm_surrogate_gradient(rbm_ctx *ctx, const void *x_dev, const void *f_target_dev, int64_t nb,
                                  float *grad_host, double *loss_host);

/* Checkpoint/resume of the surrogate: everything later steps and checkpoints
 * read (FP32 masters, Adam moments and step count, normalisation, selection
 * flag, last error, step counters, the checkpoint schedule) as a
 * self-describing host buffer of rbm_surrogate_state_size bytes.  Load into a
 * context configured with the same rbm_surrogate_config; together with the
 * positions and rbm_set_step the run continues bit for bit.  RBM_ERR_INVALID
 * for a short or foreign buffer.  Synchronous. */
rbm_status rbm_surrogate_state_size(const rbm_ctx *ctx, int64_t *bytes);
rbm_status rbm_surrogate_save(rbm_ctx *ctx, void *host_buf, int64_t bytes);
rbm_status rbm_surrogate_load(rbm_ctx *ctx, const void *host_buf, int64_t bytes);

/* ---- batched replicas --------------------------------------------------- */

/* A context for nrep independent systems advanced together: replica r has
 * n_host[r] particles (2 .. 2^20) occupying rows [off_r, off_r + n_host[r])
 * of the concatenated position array x_dev (off_r = sum of the earlier
 * sizes; layout, alignment and ownership as for rbm_init; base->n must be
 * the total).  All replicas share base's parameters (p <= 32, Euler scheme);
 * replica r uses replica index r in its Philox counters, so it follows the
 * same trajectory as a single system with rbm_params.replica = r.  The paper
 * has no batched form: it notes that batches can be updated in parallel once
 * the random division is known (Sec. 2.3 item 3); here whole replicas are the
 * parallel unit, all of them advanced by one kernel launch per step.
 * Accepted afterwards: rbm_step, rbm_run (RBM_METHOD_RBM), rbm_permutation
 * (replica-local ids, replica after replica), rbm_forces (RBM_METHOD_RBM),
 * rbm_step_host, rbm_get/set_step, rbm_sync, rbm_free, rbm_autotune,
 * rbm_batched_set_launch; the direct-step calls return RBM_ERR_UNSUPPORTED. */
rbm_status rbm_batched_init(const rbm_params *base, int32_t nrep, const int64_t *n_host, void *x_dev,
                            void *cuda_stream, rbm_ctx **out);

/* Launch shape of the batched step: threads per block (256, 512 or 1024) and
 * the mean bucket size of each replica's sort (64 .. 2048).  Synchronous.
 * RBM_ERR_UNSUPPORTED (shape unchanged) when the kernel for this dtype and d
 * cannot run that many threads per block (its registers do not fit). */
rbm_status rbm_batched_set_launch(rbm_ctx *ctx, int32_t threads, int32_t bucket_target);

/* Choose the launch configuration of the RBM step by timing the candidates
 * (batched: threads x bucket size; single system: bucket-sort kernels vs the
 * cooperative kernel) for trial_steps steps each on a scratch copy of the
 * positions (the state and step index are left unchanged), and apply the
 * fastest.  With table_path, a previous result for the same workload
 * signature is read from that text file instead of searching, and a new
 * result is appended to it.  A one-line report is written to `report` (up to
 * report_len bytes, NUL-terminated) when given.  Synchronous. */
rbm_status rbm_autotune(rbm_ctx *ctx, int32_t trial_steps, const char *table_path, char *report, int32_t report_len);

/* Batch size p of the context from now on (2 <= p <= min(N, 4096); batched
 * contexts p <= 32; the splitting scheme p = 2): reallocates the scratch and
 * drops captured graphs; positions and step index unchanged.  Synchronous. */
rbm_status rbm_set_batch_size(rbm_ctx *ctx, int32_t p);

/* Choose p, and a step, by accuracy.  The error of RBM-1 decays like
 * sqrt(dt / (p - 1)) (Sec. 3, the convergence theorem) while its cost per step
 * grows with p, so the batch size is chosen by the least time to reach
 * T = horizon with E(T) <= eps, E(T) the root mean square distance to the
 * direct method (eq. "errorformula"), not by step time alone:
 *   pilot    - the first pilot_n particles of the system (batched contexts:
 *              the replica whose size is closest to pilot_n, with its own
 *              replica index), from the current positions;
 *   error    - for each p in ps[0..nps) and each step dt_k = dt / 2^k,
 *              k = 0..max_halvings (dt the context's step): RBM-1 to T with
 *              noise refinement 2^(max_halvings+1-k) against the direct method
 *              at dt / 2^(max_halvings+1), so all runs share one Brownian path
 *              (rbm_set_noise_refinement);
 *   cost     - each p's step time at full size (trial_steps eager steps on a
 *              scratch copy of the state);
 *   choice   - among (p, k) with E(T) <= eps the least (T / dt_k) x step time;
 *              when none meets eps, the smallest error (*met_out = 0).
 * The chosen p is applied (rbm_set_batch_size); the chosen step is returned
 * in *dt_out (the context keeps its dt).  With table_path a previous result
 * for the same workload signature is read instead of searching, and a new
 * one appended.  Positions and step index are left unchanged.  Not for the
 * Verlet scheme (RBM_ERR_UNSUPPORTED).  Synchronous. */
rbm_status rbm_autotune_accuracy(rbm_ctx *ctx, const int32_t *ps, int32_t nps, double eps, double horizon,
                                 int32_t max_halvings, int64_t pilot_n, int32_t trial_steps, const char *table_path,
                                 int32_t *p_out, double *dt_out, int32_t *met_out, char *report, int32_t report_len);

/* ---- without allocation ------------------------------------------------ */

/* The random division of step m (the same ids, in the same order, as
 * rbm_permutation gives for a context with this n, seed and replica at step
 * m) written to perm_dev (n uint32, device, caller-owned), computed without
 * allocating memory.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory - an application whose
 * memory manager owns all of it, or a loop that must not block on or fail in
 * cudaMalloc.  It needs no context; its scratch is a fixed array of about
 * 650 KB in device memory that each GPU loading the library holds until exit.
 *   n: 2 .. 65536; larger n returns RBM_ERR_INVALID (rbm_last_error says why).
 *   cuda_stream: the work is enqueued there (cudaStream_t as void*); the call
 *   returns without waiting.
 * Each call outside stream capture looks up the array's address on the
 * current device (so a cudaDeviceReset, which reloads the module, is
 * harmless); a call made while its stream is capturing reuses the address the
 * last call on that device found, so make one call on a device before any
 * stream capture there.  All calls on a device share the array: each clears
 * what must start at zero, so calls in sequence are fine, but calls whose
 * work overlaps on the GPU race on it.  Rejected arguments (n < 2, n above
 * the maximum, m < 0, a null perm_dev) return RBM_ERR_INVALID with a reason in
 * rbm_last_error() and touch no CUDA state. */
rbm_status rbm_permutation_noalloc(int64_t n, uint64_t seed, uint32_t replica, int64_t m, uint32_t *perm_dev,
                                   void *cuda_stream);

/* Measured FP32 fused multiply-add throughput of the current device in
 * TFLOP/s (2 flop per FMA): eight independent FMA chains per thread, eight
 * 256-thread blocks per SM, scalar `fma.rn.f32` (packed = 0) or packed
 * two-lane `fma.rn.f32x2` (packed = 1); the best of five launches after one
 * warm-up, CUDA events on `cuda_stream` (a cudaStream_t; NULL = the legacy
 * default stream).  The ALU roofline of the direct O(N^2) sum.  Allocates
 * 4 bytes of device memory for the call.  RBM_ERR_INVALID for a null tflops or
 * packed other than 0 or 1.  Synchronous; needs no context. */
rbm_status rbm_fp32_fma_peak(int32_t packed, double *tflops, void *cuda_stream);

/* Number of kernel launches one step of `method` enqueues inside a run of
 * steps (for accounting; an RBM-1 run's first step adds the bucketing of its
 * ids on the bucket-sort and cooperative paths, and the scatter of the rows
 * on the record path, whose last step adds the placement of the rows by id). */
rbm_status rbm_launches_per_step(const rbm_ctx *ctx, int32_t method, int32_t *launches);

#ifdef __cplusplus
}
#endif
#endif /* RBM_H */
