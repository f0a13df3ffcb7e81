/*
 * hawkes.h -- C ABI of the GB300 (sm_103a) spatiotemporal Hawkes likelihood library.
 *
 * The library evaluates the log-likelihood of the self-exciting spatiotemporal
 * Hawkes process of Holbrook, Loeffler, Flaxman and Suchard ("Scalable Bayesian
 * inference for self-excitatory stochastic processes applied to big American
 * gunfire data"), Section 2.1, Eq. 1, and its gradient with respect to the six
 * model parameters, on one GPU:
 *
 *   lambda_n = mu0/(tau_x^2 tau_t) sum_{n'} phi2((x_n - x_n')/tau_x) phi1((t_n - t_n')/tau_t)
 *            + theta*omega/h^2 sum_{t_n' < t_n} exp(-omega (t_n - t_n')) phi2((x_n - x_n')/h)
 *   Lambda_n = mu0 (Phi((t_N - t_n)/tau_t) - Phi(-t_n/tau_t)) + theta (1 - exp(-omega (t_N - t_n)))
 *   ell      = sum_n (log lambda_n - Lambda_n)
 *
 * with d = 2 spatial dimensions, phi1/phi2 the standard normal densities on R and
 * R^2, Phi the standard normal CDF, and t_N the last event time. Two readings of
 * the paper are built in:
 *   - the trigger prefactor is theta*omega/h^2 (the paper prints theta/(omega h^d),
 *     which does not integrate to its own closed-form compensator);
 *   - the background sum includes n' = n unless HAWKES_FLAG_EXCLUDE_SELF is set.
 * The trigger indicator is strict (t_n' < t_n) on the stored times, so events with
 * equal stored times never trigger one another.
 *
 * Precision modes. HAWKES_FP64 runs every step in double precision. HAWKES_MIXED
 * stores coordinates as float32 (rounded from the uploaded doubles), computes pair
 * distances and kernel values in float32, accumulates each row in float32 over
 * 128-column tiles and folds every tile into float64; the log, the compensator and
 * all reductions are float64. All reductions run in a fixed order: the same call on
 * the same inputs returns bit-identical results. A request served through
 * hawkes_submit returns the same bits whatever it is batched with. hawkes_loglik_batch
 * returns bit-identical results to single calls in HAWKES_FP64, and in HAWKES_MIXED below
 * 12 (with the gradient) or 16 parameter vectors; larger mixed batches run a kernel that
 * shares each pair's geometry across requests, and their results agree with single calls
 * within the mixed-precision accuracy below, not bitwise.
 *
 * Mixed-precision accuracy (against float64 on the same float32-rounded inputs, measured
 * on the N = 85,000 workload): ell to about 1e-7 relative and the gradient to about 1e-7
 * of max|grad|. Scaled times and coordinates are rounded once from the exact float64
 * scales, so the float32 path carries no systematic bandwidth error; a gradient component
 * that nearly cancels (d ell / d tau_t cancels to about 1e-3 per event on that workload) has
 * an absolute error of about 1e-7 of sum_n |d ell_n / d Theta_k|, not of its own size.
 * Per-event values (hawkes_event_terms, hawkes_pi_batch) are held to about 1e-6 relative
 * for tau_x >= 1 km; background-only tiles difference coordinates pre-scaled by 1/tau_x, so
 * the error grows with the region's extent over tau_x (about 4e-6 at tau_x = 0.25 km and
 * 8e-6 at tau_x = 0.1 km on a 20 km square). HAWKES_FP64 holds them to 1e-11.
 *
 * Threading. A context may be used from several host threads; calls on one
 * context are serialised internally, except hawkes_poll/hawkes_wait, which only
 * read completed results. Every function returns a status code and never aborts.
 */
#ifndef HAWKES_H
#define HAWKES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------------- */
#define HAWKES_OK 0
#define HAWKES_E_INVAL -1     /* bad argument: NULL pointer, n < 1, non-finite value,  */
                              /* negative time, parameter out of its domain            */
#define HAWKES_E_UNSORTED -2  /* event times are not non-decreasing                    */
#define HAWKES_E_NOSET -3     /* unknown or released event-set id                      */
#define HAWKES_E_ADMISSION -4 /* the request's device footprint exceeds the budget     */
#define HAWKES_E_NOMEM -5     /* a device or pinned-host allocation failed             */
#define HAWKES_E_TIMEOUT -6   /* hawkes_wait: the result was not ready in time         */
#define HAWKES_E_PENDING -7   /* hawkes_poll: the result is not ready yet              */
#define HAWKES_E_CUDA -8      /* a CUDA runtime call failed (see hawkes_last_cuda_error) */
#define HAWKES_E_TICKET -9    /* unknown ticket, or its result was already collected   */
#define HAWKES_E_SHUTDOWN -10 /* the context is being destroyed                        */
#define HAWKES_E_DEVICE -11   /* a bounded wait inside a kernel ran out; the results of  */
                              /* the request are discarded (the context stays usable)  */

/* ---- flags (hawkes_set_flags) ----------------------------------------------------- */
#define HAWKES_FLAG_EXCLUDE_SELF 1 /* drop n' = n from the background sum of lambda_n    */
#define HAWKES_FLAG_DENSE 2        /* visit all N^2 pairs (see below)                      */
#define HAWKES_FLAG_NO_SYMMETRY 4  /* HAWKES_MIXED: evaluate every ordered pair on its own     */
/* By default a mixed-precision evaluation without HAWKES_FLAG_EXCLUDE_SELF or HAWKES_FLAG_DENSE
 * shares background terms: e_b(n, n') = e_b(n', n), so for the column tiles before a row tile's
 * own each background term is formed once and added to both events' rows; the trigger terms of
 * those tiles (nonzero only within the trigger's reach, see below) go to the later event's row
 * Every event's sums (its row's, and the shares of the tiles holding it) are then added as exact
 * fixed-point integers: 2^-F resolution with
 * F = 62 - ceil(log2 N_padded) for the background sums (about 3e-14 at N = 85,000, against a
 * background sum of at least 1, the self term) and a per-sum F from Theta for the trigger
 * moments. Integer addition commutes, so results stay bit-identical from run to run and alone or
 * batched; they differ from the row-by-row evaluation (HAWKES_FLAG_NO_SYMMETRY) by float32
 * rounding only, and the evaluation needs no partial-sum workspace (num_sums x N_padded
 * integers instead: 4.1 MB for loglik + gradient at N = 85,000). A sum that is not finite or
 * leaves the fixed-point range (possible only for inputs whose float32 pair terms overflow)
 * makes ell and the gradient NaN, with status OK. The paper's evaluation visits every ordered
 * pair (Section 2.3); this is a reorganisation of the same sum. */
/* For testing the failure path only: in loglik + gradient evaluations that merge partial sums in
 * a tree (HAWKES_FP64, the row-by-row HAWKES_MIXED evaluation, which this flag selects, and
 * grouped batches) the first work item to reach each merge node of row tile 0 publishes its
 * partial sums without marking them ready, so the bounded device wait of its sibling runs out
 * (after at most 0.5 s) and the call returns HAWKES_E_DEVICE. Nothing faults or hangs; later
 * calls without the flag are unaffected. */
#define HAWKES_FLAG_TEST_WITHHOLD_READY (1 << 30)
/* By default each row only visits the columns whose pair terms can change its sums at the
 * working precision. With the self term, the background sum holds the term n' = n = 1, so
 * lambda_n >= A = mu0 / ((2 pi)^(3/2) tau_x^2 tau_t), and columns whose terms are each below
 * 2^-P A / N are skipped (background exponent beyond (P + log2 N) ln 2 in time alone, trigger
 * exponent beyond that plus ln(C / A), C = theta omega / (2 pi h^2)): the skipped part of a row
 * stays below 2^-P of lambda_n for each kind of term. HAWKES_FP64: P = 70, 1/128 of float64's
 * rounding unit. HAWKES_MIXED: P = 40, 2^-16 of float32's rounding unit (the results move by
 * less than 1e-12 relative against visiting every pair), and never past the exponents at which
 * float32 ex2 (flushing subnormals to zero) returns exactly +0. With HAWKES_FLAG_EXCLUDE_SELF
 * (no such floor) each mode keeps every term that is not exactly zero in its precision.
 * HAWKES_FLAG_DENSE visits all pairs (in HAWKES_FP64 up to float64 exp's exact zeros). */

typedef struct hawkes_ctx hawkes_ctx;

/* Theta = (mu0, tau_x, tau_t, theta, omega, h), in the order of Section 2.1.
 * Domain: mu0, tau_x, tau_t, omega, h > 0 and finite; theta >= 0 and finite. */
typedef struct {
  double mu0, tau_x, tau_t, theta, omega, h;
} hawkes_params;

typedef enum {
  HAWKES_FP64 = 0,  /* double precision throughout                                */
  HAWKES_MIXED = 1  /* float32 pair terms, float64 row accumulation and reductions */
} hawkes_mode;

/* Create a context on CUDA device `device`. `hbm_budget_bytes` caps the device
 * memory the context may hold (event sets plus per-request workspaces); 0 means
 * 90% of the device's free memory at creation. `cuda_stream` is a cudaStream_t to
 * run on (for example PyTorch's current stream); NULL makes the context create
 * and own a non-blocking stream. The serving queue (hawkes_submit) always runs on
 * streams the context owns. Errors: E_INVAL (NULL out, bad device), E_CUDA, E_NOMEM. */
int hawkes_create(hawkes_ctx **out, int device, size_t hbm_budget_bytes, void *cuda_stream);

/* Wait for all queued work, free every device buffer and the context.
 * Pending tickets complete with E_SHUTDOWN. NULL is accepted (no-op). */
int hawkes_destroy(hawkes_ctx *ctx);

/* Set context flags (HAWKES_FLAG_*); they apply to calls made afterwards. */
int hawkes_set_flags(hawkes_ctx *ctx, int flags);

/* Copy an event set to the device (Section 2.1: events (x_n, t_n), x_n in R^2).
 * x, y (km) and t (days) are host arrays of n doubles; the caller keeps ownership
 * and may free them when the call returns. t must be non-decreasing and >= 0
 * (the compensator integrates from 0 to t_N, the last event). The library copies
 * the float64 arrays to the device and forms there, in two launches, the float32
 * copies, the tie indices and the time tables, and checks the inputs; all in
 * structure-of-arrays layout, padded to a multiple of 256 with sentinel events that
 * contribute exactly zero. The call returns when the set is ready (or rejected). The
 * set stays resident until hawkes_release_events or hawkes_destroy.
 * Errors: E_INVAL (NULL, n < 1, non-finite, t < 0), E_UNSORTED, E_ADMISSION
 * (set does not fit the budget), E_NOMEM, E_CUDA. */
int hawkes_upload_events(hawkes_ctx *ctx, const double *x, const double *y, const double *t,
                         int64_t n, int32_t *set_id_out);

/* Free a resident event set. Requests already queued on it still complete. */
int hawkes_release_events(hawkes_ctx *ctx, int32_t set_id);

/* Number of events of a resident set and the device bytes it occupies (coordinates in
 * both precisions, tie indices and work schedules). Either out pointer may be NULL. */
int hawkes_set_info(hawkes_ctx *ctx, int32_t set_id, int64_t *n_out, size_t *device_bytes_out);

/* ell(Theta) of Eq. 1 for a resident set. Blocks until the result is on the host.
 * Errors: E_INVAL, E_NOSET, E_ADMISSION, E_NOMEM, E_CUDA, E_DEVICE. If some lambda_n is
 * zero (possible only with HAWKES_FLAG_EXCLUDE_SELF) the result is -inf with status OK. */
int hawkes_loglik(hawkes_ctx *ctx, int32_t set_id, const hawkes_params *params,
                  hawkes_mode mode, double *loglik_out);

/* ell(Theta) and d ell / d Theta (six entries in Theta order) in one pass over the
 * pairs. The paper has no gradient; it is the exact derivative of Eq. 1, computed
 * from per-row moments of the same pair terms. Blocks like hawkes_loglik. */
int hawkes_loglik_grad(hawkes_ctx *ctx, int32_t set_id, const hawkes_params *params,
                       hawkes_mode mode, double *loglik_out, double grad_out[6]);

/* ---- mixture of triggering functions --------------------------------------------------
 * The paper's Discussion proposes a mixture of triggering functions for gunfire, combining a
 * very short time frame (multi-shot events) with a longer one (retaliation over days to
 * months). Read here as M components, each the triggering function of Section 2.1 with its own
 * (theta_m, omega_m, h_m):
 *   g(dx, dt) = sum_m theta_m omega_m / h_m^2 exp(-omega_m dt) phi2(dx / h_m),
 * so the compensator's trigger part is sum_m theta_m (1 - exp(-omega_m (t_N - t_n))) and M = 1
 * is the model above. The background, the flags, the exact-zero windows (taken at the longest
 * trigger reach) and the shared background work as for hawkes_loglik_grad. */
#define HAWKES_MIX_MAX 2
typedef struct {
  double mu0, tau_x, tau_t;
  double theta[HAWKES_MIX_MAX], omega[HAWKES_MIX_MAX], h[HAWKES_MIX_MAX];
} hawkes_mix_params;

/* ell of Eq. 1 with the first m (1 or 2) components of `params`, and with want_grad its gradient:
 * grad_out receives 3 + 3 m entries, (mu0, tau_x, tau_t, theta_1, omega_1, h_1[, theta_2,
 * omega_2, h_2]); it may be NULL when want_grad is 0. Domain: as hawkes_params for each
 * component (theta_m >= 0; omega_m, h_m > 0). Blocks like hawkes_loglik_grad. Errors as
 * hawkes_loglik_grad. */
int hawkes_loglik_mix(hawkes_ctx *ctx, int32_t set_id, const hawkes_mix_params *params, int m,
                      hawkes_mode mode, int want_grad, double *loglik_out, double *grad_out);

/* Asynchronous form for callers that keep results on the device: enqueue the
 * evaluation on the context's stream and return at once. `device_out` is a device
 * pointer to 7 doubles (ell, then the gradient if want_grad; the gradient entries
 * are left unchanged otherwise). The caller synchronises the stream before reading
 * it. Calls on one context share its workspace and therefore run in stream order. A device
 * wait that ran out (HAWKES_E_DEVICE for the blocking calls) leaves NaN in device_out. */
int hawkes_loglik_async(hawkes_ctx *ctx, int32_t set_id, const hawkes_params *params,
                        hawkes_mode mode, int want_grad, double *device_out);

/* K parameter vectors on one resident set in one launch (K <= 64): the batched
 * evaluation of many MCMC chains that share a data set. loglik_out has K entries;
 * grad_out (K x 6, row-major) may be NULL when want_grad is 0. Results are deterministic
 * for a given batch. In HAWKES_FP64, and in HAWKES_MIXED with K below 12 (want_grad) or
 * 16 (loglik only), each is bit-identical to the same request evaluated alone. Larger
 * HAWKES_MIXED batches run in groups of 4 or 8 requests that share each pair's geometry
 * (time differences in days, float32 sums over a work item rather than a tile), so the
 * results agree with single calls within the mixed-precision accuracy stated above, not
 * bitwise. */
int hawkes_loglik_batch(hawkes_ctx *ctx, int32_t set_id, int k, const hawkes_params *params,
                        hawkes_mode mode, int want_grad, double *loglik_out, double *grad_out);

/* Work accounting for an evaluation at Theta (host computation on the set's stored times, read
 * back from the device; no kernel launch):
 *   out[0] ordered (row, column) pairs inside the column windows the kernels cover (see
 *          HAWKES_FLAG_DENSE and the note above it), counted over real events;
 *   out[1] N^2, the pairs of Eq. 1's double sum;
 *   out[2] ordered pairs whose background term can change the sums at the mode's precision
 *          (|t_n - t_n'| below the background's reach, n' = n included);
 *   out[3] ordered pairs whose trigger term can change the sums (0 <= t_n - t_n' below the
 *          trigger's reach; pairs with equal times counted although their term is zero);
 *   out[4] pair terms the kernels evaluate: out[0] less the far pairs whose background term
 *          serves both events (see HAWKES_FLAG_NO_SYMMETRY), which are evaluated once. */
int hawkes_pair_work(hawkes_ctx *ctx, int32_t set_id, const hawkes_params *params, hawkes_mode mode,
                     int64_t out[5]);

/* Per-event terms of Eq. 2: mu_out[n] = mu(x_n, t_n) (background rate at event n)
 * and xi_out[n] = lambda_n - mu_n (the self-excitation part), so lambda_n =
 * mu_n + xi_n and pi_n = xi_n / lambda_n. Host arrays of n doubles each, owned by
 * the caller. The log-likelihood of the same pass goes to loglik_out if not NULL.
 * Accuracy in HAWKES_MIXED: mu_n to about 1e-6 relative for tau_x >= 1 km, growing as the
 * region's extent over tau_x grows (about 4e-6 at tau_x = 0.25 km and 8e-6 at 0.1 km on a
 * 20 km square); xi_n to about 1e-6 of max xi. HAWKES_FP64: 1e-11. */
int hawkes_event_terms(hawkes_ctx *ctx, int32_t set_id, const hawkes_params *params,
                       hawkes_mode mode, double *mu_out, double *xi_out, double *loglik_out);

/* Eq. 2 for k parameter vectors on one set, the posterior form of Section 3.2 (a sample
 * Theta^(1..k) gives k vectors of N probabilities): pi_out[r * n + i] = xi_i / lambda_i at
 * params[r], for events in stored (time) order. pi_out is a host array of k * n doubles and
 * loglik_out (k doubles, may be NULL) receives ell at each params[r]; both owned by the
 * caller. The call blocks; it launches up to 64 parameter vectors at a time and needs device
 * workspace for 64 * n doubles of output besides the evaluation's own. k = 0 does nothing.
 * Accuracy as hawkes_event_terms (pi_n = xi_n / lambda_n: about 1e-6 absolute in HAWKES_MIXED
 * for tau_x >= 1 km, up to about 8e-6 at tau_x = 0.1 km; 1e-11 in HAWKES_FP64).
 * Errors as hawkes_loglik; on an error the entries of pi_out not yet written are undefined. */
int hawkes_pi_batch(hawkes_ctx *ctx, int32_t set_id, int k, const hawkes_params *params,
                    hawkes_mode mode, double *pi_out, double *loglik_out);

/* ---- serving: continuous batching of requests from many chains ----------------------
 * hawkes_submit queues one request (set, Theta, gradient flag, mode) and returns a
 * ticket at once. A scheduler thread admits queued requests while their device
 * footprint fits the budget, groups them into kernel launches (up to 64
 * requests each, several launches in flight on separate streams) and completes
 * tickets as launches finish. A request's result does not depend on what it was
 * batched with. */
int hawkes_submit(hawkes_ctx *ctx, int32_t set_id, const hawkes_params *params, int want_grad,
                  hawkes_mode mode, uint64_t *ticket_out);

/* Non-blocking. done_out = 1 and the result copied (grad_out may be NULL) when the
 * request has finished; the ticket is then consumed. done_out = 0 and status
 * E_PENDING otherwise. A failed request returns its error status (and is consumed). */
int hawkes_poll(hawkes_ctx *ctx, uint64_t ticket, int *done_out, double *loglik_out,
                double grad_out[6]);

/* hawkes_poll plus the request's timing on the host's steady clock: queued_ns from submission
 * to the launch that carried it, total_ns from submission to the scheduler observing its
 * completion (either pointer may be NULL; both are written only when done_out is 1). */
int hawkes_poll_timed(hawkes_ctx *ctx, uint64_t ticket, int *done_out, double *loglik_out,
                      double grad_out[6], int64_t *queued_ns_out, int64_t *total_ns_out);

/* Block until the request finishes or `timeout_ms` elapses (E_TIMEOUT; the ticket
 * stays valid). timeout_ms < 0 waits without limit. */
int hawkes_wait(hawkes_ctx *ctx, uint64_t ticket, int timeout_ms, double *loglik_out,
                double grad_out[6]);

/* Serving counters: submitted, completed, failed, launches, requests in flight, queued,
 * and the device bytes currently held for requests. `out` has 7 entries. */
int hawkes_stats(hawkes_ctx *ctx, int64_t out[7]);

/* Kernel timing, for profiling (the paper has no counterpart; it measures whole evaluations,
 * Section 3.1). With on != 0, every evaluation enqueued on the context's own stream (blocking,
 * batch and asynchronous calls; not the serving path) records CUDA events before its pair
 * kernel, between it and the split epilogue of the mixed path, and after that; on = 0 stops.
 * The events add two or three records to each evaluation's stream work.
 * hawkes_kernel_ms waits for the most recent timed evaluation and writes, in ms, the duration
 * of its pair kernel (ms_out[0]) and of what followed it up to the end of the evaluation's
 * launches (ms_out[1]: the split epilogue in HAWKES_MIXED, about 0 otherwise). Errors:
 * E_INVAL; E_PENDING if no evaluation was timed since timing was switched on; E_CUDA. */
int hawkes_set_kernel_timing(hawkes_ctx *ctx, int on);
int hawkes_kernel_ms(hawkes_ctx *ctx, double ms_out[2]);

/* ---- evaluation without allocation -----------------------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that must not allocate
 * device memory when they evaluate, for example a program whose device memory is reserved in
 * full by another allocator, or a sampler loop in which cudaMalloc/cudaFree could stall on
 * device-wide synchronisation. It computes the same mixed-precision ell(Theta) as
 * hawkes_loglik(..., HAWKES_MIXED) without a context, from events the caller already holds
 * on the device, and calls no allocator: its temporaries live in one fixed device array of
 * the library (about 5.3 MB, reserved on every GPU that loads the library, until exit).
 *
 * x, y, t: device pointers to n float32 values each (km, km, days), t non-decreasing and
 * >= 0, coordinates finite; 1 <= n <= HAWKES_NOALLOC_MAX_EVENTS, larger n returns
 * HAWKES_E_INVAL. The event values are never read on the host: they are checked on the
 * device, and inputs that hawkes_upload_events would reject (unsorted, negative or
 * non-finite times, non-finite coordinates), or a time span too long for the float32 path at
 * this tau_t, make device_out NaN. flags: HAWKES_FLAG_EXCLUDE_SELF, HAWKES_FLAG_DENSE and
 * HAWKES_FLAG_NO_SYMMETRY (this entry point always evaluates every ordered pair on its own).
 * device_out: device pointer to one double that receives ell. cuda_stream: the stream to
 * enqueue on (NULL = the legacy default stream). The call is asynchronous: the caller
 * synchronises the stream before reading device_out.
 * The first call on each device sets up the array's device address (cudaGetSymbolAddress),
 * so make that first call before any stream capture; a device reset (cudaDeviceReset) makes
 * the next call set it up again. Every call reuses the same array, which keeps the previous
 * call's contents (each call clears what must start at zero): calls that may overlap on the
 * GPU (on different streams, or from several threads) race and must be serialised by the
 * caller. Errors: E_INVAL, E_CUDA. */
#define HAWKES_NOALLOC_MAX_EVENTS 65536
int hawkes_loglik_noalloc(const float *x, const float *y, const float *t, int64_t n,
                          const hawkes_params *params, int flags, double *device_out, void *cuda_stream);

/* Human-readable text for a status code. Never NULL. */
const char *hawkes_strerror(int status);

/* Text of the most recent CUDA error seen on this context ("" if none). */
const char *hawkes_last_cuda_error(hawkes_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* HAWKES_H */
