/*
 * gbs.h - C ABI of the GB300 library for Gaussian-boson-sampling output
 * probabilities with every input mode squeezed.
 *
 * The library evaluates
 *
 *     p(s) = |Haf(B_s)|^2 / (prod_j s_j! * prod_i cosh r_i),
 *     B    = U diag(tanh r_1, ..., tanh r_m) U^T,
 *
 * the output-probability formula of Sec. 2.3 (Eq. ProOri) written for per-mode
 * squeezing r_i; for identical r it is exactly Eq. ProOri, because
 * Haf(tanh(r) W_s) = tanh(r)^{n/2} Haf(W_s). B_s repeats row and column j of B
 * s_j times (Sec. 2.3, Eq. W_s_example); equivalently B_x(i, j) = B(x_i, x_j)
 * for the index list x of the pattern (Sec. 3.2, "Step 2: change of basis").
 *
 * Haf is computed by the 2^{n/2}-subset sum whose O(n^3 2^{n/2}) cost Sec. 2.3
 * cites (Bjorklund, Gupt, Quesada): with n = 2h and pairs {2i, 2i+1},
 *     Haf(A) = sum_{S subset of [h]} (-1)^{h-|S|} f(X A_S),
 *     f(M)   = [x^h] det(I - x M)^{-1/2},
 * X swapping the two members of each pair. One subset term is a characteristic
 * polynomial of a 2|S| x 2|S| complex matrix.
 *
 * Conventions for every call:
 *   - Return 0 on success or a negative GBS_E* code; gbs_last_error() gives a
 *     thread-local message for the last failure on the calling thread. No C++
 *     exception crosses this boundary.
 *   - Complex numbers are interleaved (re, im) doubles; matrices are row-major.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream). Work is stream-ordered on it; the call returns once the work is
 *     enqueued, unless an output pointer is host memory (then it returns after
 *     the results are in that memory).
 *   - Buffers passed in are owned by the caller and never freed or retained
 *     after the call returns. Pointer arguments documented as "host or device"
 *     are classified with cudaPointerGetAttributes.
 *   - Odd n gives Haf = 0 and p = 0 (P_n = 0 for odd n, Sec. 3.1); n = 0 gives
 *     Haf = 1 and p = prod_i sech r_i.
 */
#ifndef GBS_H
#define GBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GBS_OK 0
#define GBS_EINVAL (-1)    /* bad argument (null pointer, negative size, bad precision) */
#define GBS_ENOMEM (-2)    /* device or host allocation failed */
#define GBS_ERANGE (-3)    /* n > GBS_MAX_N, or a mode index outside [0, m) */
#define GBS_EAGAIN (-4)    /* serving queue full; retry later */
#define GBS_ETIMEDOUT (-5) /* a bounded device or host wait gave up */
#define GBS_ECUDA (-6)     /* a CUDA runtime call failed (message has the CUDA error) */
#define GBS_ENOENT (-7)    /* unknown serving ticket */
#define GBS_ECANCELED (-8) /* serving request cancelled by gbs_serve_cancel */

#define GBS_FP64 0  /* per-subset arithmetic in FP64, signed sum in double-double */
#define GBS_MIXED 1 /* power traces in FP32; their exponential series (the characteristic-
                       polynomial recurrence) in FP64 and the signed sum in double-double */

#define GBS_MAX_N 32 /* largest photon number (matrix order) accepted */

typedef struct gbs_kernel gbs_kernel; /* opaque, library-owned */
typedef struct gbs_server gbs_server; /* opaque, library-owned */

/* ------------------------------------------------------------------------ */
/* Kernel matrix                                                            */
/* ------------------------------------------------------------------------ */

/* Build the resident kernel matrix B = U diag(tanh r) U^T of an m-mode
 * interferometer (Sec. 2.3, W = U U^T, with per-mode squeezing) and the log
 * normaliser L = sum_i log cosh r_i of Eq. ProOri.
 *   U_ri  m*m complex128, interleaved, row-major, host or device.
 *   r     m doubles, host or device.
 *   m     number of modes, >= 1.
 *   out   receives a new library-owned object; free with gbs_free_kernel.
 * B (16 m^2 bytes) stays in device memory on the current device until freed.
 * Errors: GBS_EINVAL (null pointer, m < 1), GBS_ENOMEM, GBS_ECUDA. */
int gbs_build_kernel(const double* U_ri, const double* r, int m, void* stream, gbs_kernel** out);

/* Release a kernel object (waits for the device work that uses it). NULL is a no-op. */
int gbs_free_kernel(gbs_kernel* k);

/* Number of modes m and the log normaliser L = sum_i log cosh r_i (available
 * after the build's stream work completes; this call synchronises with it). */
int gbs_kernel_info(const gbs_kernel* k, int* m, double* log_norm);

/* Copy B (m*m complex128 interleaved) into dst (host or device), stream-ordered. */
int gbs_kernel_copy_B(const gbs_kernel* k, double* dst, void* stream);

/* ------------------------------------------------------------------------ */
/* Batched Hafnians and probabilities                                       */
/* ------------------------------------------------------------------------ */

/* Hafnians of a batch of symmetric complex matrices (Eq. HafMatch), by the
 * subset sum above.
 *   A_ri    concatenated matrices, complex128 interleaved, host or device;
 *           matrix b is n[b] x n[b] row-major starting at complex element
 *           offs[b]. Only the entries off the diagonal are read (no perfect
 *           matching uses V(i, i)).
 *   n,offs  host arrays of `batch` entries; 0 <= n[b] <= GBS_MAX_N.
 *   precision  GBS_FP64 or GBS_MIXED.
 *   haf_ri_out  2*batch doubles (host or device): Haf(A_b).
 *   kappa_out   batch doubles (host or device) or NULL: the cancellation ratio
 *               kappa_b = sum_S |f(X A_S)|_1 / |Haf(A_b)| (|z|_1 = |re|+|im|).
 * Errors: GBS_EINVAL, GBS_ERANGE (n[b] > GBS_MAX_N), GBS_ENOMEM, GBS_ECUDA. */
/* Ordering: the subset sum pairs positions (t, t + n/2) of each matrix by
 * default (which keeps copies of a repeated row apart); for n >= 26 this call
 * and gbs_prob_batch first try 16 orderings on a sample of subsets and run the
 * sum in the one with the smallest sampled sum |f|. The Hafnian does not depend
 * on the ordering; the cancellation, and so the rounding error, does (measured
 * on 80 matrices at n = 28 and 30: largest error 3.5e-11 with the choice,
 * 3.1e-10 in the default order). */
int gbs_hafnian_batch(const double* A_ri, const int* n, const int64_t* offs, int batch,
                      int precision, void* stream, double* haf_ri_out, double* kappa_out);

/* gbs_hafnian_batch for callers that cannot allocate memory while they run
 * (for example code inside a host callback or a memory-accounting scope, or a
 * process that reserves all device memory for other work at start-up). The
 * paper has no counterpart; this is a deployment variant of the call above.
 * Same arguments and results, except that A_ri, haf_ri_out and kappa_out must
 * be device memory (GBS_EINVAL otherwise). Its working space is one fixed
 * array of about 1.6 MB built into the library, reserved on every GPU that
 * loads it until the process exits, so the call makes no cudaMalloc, cudaFree,
 * cudaMallocHost or other allocating call. Limits: at most 1024 matrices and
 * 16384 work items per call (GBS_ERANGE beyond, with the reason in
 * gbs_last_error). The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture. All calls share the array: calls whose GPU work overlaps (on
 * different streams, or from several threads without ordering) race on it and
 * must be serialised by the caller. Matrices keep the default ordering at
 * every n (no ordering probe), so at n >= 28 an ill-conditioned matrix can
 * exceed 1e-10 relative error where gbs_hafnian_batch does not. */
int gbs_hafnian_batch_noalloc(const double* A_ri, const int* n, const int64_t* offs, int batch,
                              int precision, void* stream, double* haf_ri_out, double* kappa_out);

/* Output probabilities of a batch of patterns (Eq. ProOri).
 *   idx     concatenated 0-based mode-index lists x (host or device); pattern b
 *           is idx[offs[b] .. offs[b]+n[b]), a repeated index is a collision.
 *           Order within a list does not matter (Appendix B).
 *   n,offs  host arrays of `batch` entries; 0 <= n[b] <= GBS_MAX_N.
 *   Outputs (each host or device, each may be NULL):
 *     p_out       p(s) per pattern (underflows to 0 below ~1e-308),
 *     logp_out    log p(s) (-inf when Haf = 0),
 *     haf_ri_out  Haf(B_x), 2 doubles per pattern,
 *     err_est_out estimated relative error of Haf: c * u * kappa, u the unit
 *                 roundoff of the per-subset arithmetic and kappa the
 *                 cancellation ratio (as kappa_out of gbs_hafnian_batch):
 *                 GBS_FP64 u = 2^-53, c = n; GBS_MIXED u = 2^-24, c = min(n, 4),
 *                 fitted on the oracle (largest observed error 1.9 u kappa, at
 *                 n = 4, over workloads n = 2..32; below 0.1 u kappa from n = 24).
 * A host idx is checked on the host (GBS_ERANGE for an index >= m). A device
 * idx is checked on the device: a pattern with an out-of-range index gets NaN
 * outputs and no memory outside B is read.
 * Route: every pattern takes the subset sum of Sec. 2.3, except that with
 * GBS_FP64 a pattern whose photons are bunched into few modes (at most 16
 * distinct modes, prod_j (s_j + 1) terms costing well under the subset sum)
 * takes the repeated-row sum instead (the moment-extraction identity of Kan,
 * 2008; not in the paper). The choice is made on the device (a host idx is
 * copied there first), so it costs the host nothing and gives the same bits
 * for host and device lists; a batch reserves repeated-row partial slots for
 * at most 2^20 term chunks in all (patterns past that, in batch order, keep
 * the subset sum). On such patterns that route is also the accurate one: the subset sum
 * cancels strongly there (errors up to ~1e-8 measured at n = 24 in 8 modes,
 * flagged by err_est_out).
 * Kept plans: the host-side plan of a call (work items, per-matrix
 * descriptors, ordering-probe tables) depends only on n[], offs[], m, the
 * precision and the launch shape, never on the index lists or matrices, so
 * the library keeps it in device memory, for up to 8 such shapes and 256 MB in
 * all (least recently used evicted), and a later call of the same shape on any
 * stream (this call or gbs_hafnian_batch, host or device inputs) skips the
 * planning and its upload. gbs_clear_plans frees the kept plans.
 * Errors: GBS_EINVAL, GBS_ERANGE, GBS_ENOMEM, GBS_ECUDA. */
int gbs_prob_batch(const gbs_kernel* k, const int* idx, const int* n, const int64_t* offs,
                   int batch, int precision, void* stream, double* p_out, double* logp_out,
                   double* haf_ri_out, double* err_est_out);

/* Frees every kept plan that no call is using (see gbs_prob_batch), each after
 * its device has finished the work already issued (a device-wide synchronize).
 * The paper has no counterpart (memory management only). Returns GBS_OK, or
 * GBS_ECUDA if that synchronize reports an earlier asynchronous error. */
int gbs_clear_plans(void);

/* Instrumentation: when both are non-NULL, every later batch records `start`
 * immediately before and `stop` immediately after the kernels of its subset
 * sum (the pair terms, for n >= 26 the ordering probe and choice, and the
 * subset kernel), on the batch's stream (cudaEvent_t passed as void*), so a
 * caller can time that work alone. Pass NULL, NULL to stop. Process-wide; not
 * for concurrent use from several threads. The paper has no counterpart
 * (measurement only). */
int gbs_set_timing_events(void* start, void* stop);

/* Measurement: the FP64 (DFMA) throughput of the current device in TFLOP/s,
 * from a kernel that fills every SM with independent DFMA chains (best of
 * three timed runs after a warm-up, CUDA events on `stream`; about 50 ms).
 * The denominator of the subset sum's roofline fraction; the paper has no
 * counterpart. Errors: GBS_EINVAL, GBS_ENOMEM, GBS_ECUDA. */
int gbs_measure_fp64_peak(void* stream, double* tflops_out);

/* ------------------------------------------------------------------------ */
/* Autotuning                                                               */
/* ------------------------------------------------------------------------ */

/* Time the candidate launch shapes (subsets per warp work item, warps per
 * block) for photon number n and precision on synthetic matrices, on the
 * current device, and keep the fastest for later calls with that n. Calls
 * that find no tuned entry use a built-in default. Synchronises `stream`.
 * chosen_out (may be NULL) receives the chosen subsets-per-item. */
int gbs_autotune(int n, int precision, void* stream, int* chosen_out);

/* ------------------------------------------------------------------------ */
/* Sampling (Sec. 3)                                                        */
/* ------------------------------------------------------------------------ */

/* Step 1 of the sampler (Sec. 3.1, Eq. Eqdistribution): the total photon-number
 * distribution P_n = sum over |s| = n of p(s), for n = 0..n_max, computed on the
 * device as the power series prod_i sech r_i (1 - tanh^2 r_i z^2)^(-1/2) (the
 * negative binomial of Eq. Eqdistribution when every r_i is equal).
 *   n_max   0..2048.
 *   Pn_out  n_max + 1 doubles, host or device (caller-owned). P_n = 0 for odd n.
 * Errors: GBS_EINVAL, GBS_ERANGE, GBS_ENOMEM, GBS_ECUDA. */
int gbs_photon_number_dist(const gbs_kernel* k, int n_max, void* stream, double* Pn_out);

/* Brute-force sampler (Appendix I): p(s) of every one of the C(m+n-1, n)
 * configurations with n photons (enumerated on the device in colex order of
 * their index lists x_1 <= ... <= x_n), a fixed-order prefix sum, and for each
 * uniform u the configuration whose interval contains u * (sum of all p).
 *   n             0..GBS_MAX_N; C(m+n-1, n) must not exceed 2^26.
 *   uniforms      `draws` numbers in [0, 1), host or device.
 *   precision     GBS_FP64 or GBS_MIXED (the probability path used).
 *   patterns_out  draws * n ints, host or device: draw d's sorted mode list at
 *                 [d * n, (d + 1) * n).
 *   total_out     may be NULL; receives sum of p over all configurations
 *                 (= P_n of Eq. Eqdistribution up to rounding), host or device.
 * Errors: GBS_EINVAL, GBS_ERANGE, GBS_ENOMEM, GBS_ECUDA. */
int gbs_sample_bruteforce(const gbs_kernel* k, int n, const double* uniforms, int draws, int precision,
                          void* stream, int* patterns_out, double* total_out);

/* Theorem 1 (Sec. 3.3, Algorithm 2): marginal probabilities
 * q_n(x_1..x_k) = sum over x_{k+1..n} of |Haf(W_x)|^2 / f_n, W = U U^T, of
 * `batch` ordered prefixes of length k, for n-photon samples with identical
 * squeezing on every mode (the kernel's r must all be equal and > 0: the
 * theorem sums out the unsampled photons with the unitarity of W, which
 * B = U diag(tanh r_i) U^T lacks when the r_i differ). The sub-Hafnians of
 * the prefix's subsets that the sum reads come from the batched FP64 path;
 * the sums over s, s', A, B, mu of Theorem 1 are regrouped by the set
 * rho = [k] \ A (Per(S_{A,B}) = 0 unless A and B hold the same modes), and
 * only the sizes of rho and s inside the theorem's ranges are formed (a
 * team of lanes per rho, sized by the launch's work). Results are
 * deterministic for a given batch; the same prefix in batches of different
 * sizes can differ in the last bits (another split of its sums).
 *   x      batch * k mode indices in [0, m), prefix b at [b * k, (b + 1) * k),
 *          host or device (read before return).
 *   k      0..min(n, 20).  n  even, <= GBS_MAX_N.
 *   q_out  batch doubles, host or device. k = 0 gives 1; k = n gives
 *          |Haf(W_x)|^2 / f_n (Eq. EqDisE).
 * Errors: GBS_EINVAL (also unequal squeezing), GBS_ERANGE, GBS_ENOMEM, GBS_ECUDA. */
int gbs_marginal_batch(const gbs_kernel* k, const int* x, int kk, int batch, int n, void* stream,
                       double* q_out);

/* Algorithm 1 (Sec. 3.2): one ordered n-photon sample x_1..x_n by the chain
 * rule, x_k drawn from the m conditional weights q_n(x_1..x_{k-1}, l),
 * l = 0..m-1 (the sum of gbs_marginal_batch), by the inverse CDF in mode
 * order with the caller's uniform u_k: x_k is the first mode of positive
 * weight whose running sum of weights exceeds u_k times their total. The
 * running sums are formed on the device in a fixed order (32 contiguous runs
 * of modes joined by a fixed scan), so x_k can differ from the pick of a
 * left-to-right sum only when u_k times the total lies within rounding of a
 * running sum. Identical squeezing only. The sampled prefix's sub-Hafnians
 * stay on the device between steps (the exponential-space variant,
 * Appendix D); those of the sets that hold the new photon come from them by
 * expanding the Hafnian along its row.
 *   n         even, 0..20.
 *   uniforms  n numbers in [0, 1), HOST memory.
 *   x_out     n ints, HOST memory: the mode of each photon in draw order.
 * Errors: GBS_EINVAL, GBS_ERANGE, GBS_ENOMEM, GBS_ECUDA. */
int gbs_sample_chain(const gbs_kernel* k, int n, const double* uniforms, void* stream, int* x_out);

/* `samples` independent chain samples (gbs_sample_chain each), advanced
 * together: every step covers all samples' m candidates in the same launches,
 * and the modes are drawn on the device, so the call synchronises the stream
 * once per group of samples.
 * Sample s equals gbs_sample_chain with uniforms[s * n .. s * n + n - 1].
 *   samples   >= 0; they go in groups of at most 2^28 / 2^n (their sub-Hafnian
 *             caches, 2^n complex doubles each, stay within 4 GB).
 *   uniforms  samples * n numbers in [0, 1), sample-major, HOST memory.
 *   x_out     samples * n ints, HOST memory, sample-major.
 * Errors: GBS_EINVAL, GBS_ERANGE, GBS_ENOMEM, GBS_ECUDA. */
int gbs_sample_chain_batch(const gbs_kernel* k, int n, int samples, const double* uniforms, void* stream,
                           int* x_out);

/* One complete sample (Sec. 3, Steps 1-3): the photon number n drawn from
 * P_n of Eq. Eqdistribution restricted to n <= n_max and renormalised (inverse
 * CDF with uniforms[0]), then the n photons placed by gbs_sample_chain with
 * uniforms[1..n]. Identical squeezing only.
 *   n_max     0..20 (the chain sampler's limit); the mass above n_max is
 *             left out, so choose n_max where P_n has become negligible.
 *   uniforms  n_max + 1 numbers in [0, 1), HOST memory.
 *   n_out     HOST int: the drawn photon number (even).
 *   x_out     HOST, room for n_max ints: x_1..x_n in draw order.
 * Errors: GBS_EINVAL, GBS_ERANGE, GBS_ENOMEM, GBS_ECUDA. */
int gbs_sample(const gbs_kernel* k, int n_max, const double* uniforms, void* stream, int* n_out,
               int* x_out);

/* `samples` complete samples (gbs_sample each): every sample draws its n from
 * the truncated P_n, then the samples of each n go through
 * gbs_sample_chain_batch together. Sample s equals gbs_sample with
 * uniforms[s * (n_max + 1) .. s * (n_max + 1) + n_max].
 *   uniforms  samples * (n_max + 1) numbers in [0, 1), sample-major, HOST.
 *   n_out     samples ints, HOST: each sample's photon number.
 *   x_out     samples * n_max ints, HOST, sample-major: x_1..x_n of sample s
 *             at [s * n_max, s * n_max + n), -1 after them.
 * Errors: GBS_EINVAL, GBS_ERANGE, GBS_ENOMEM, GBS_ECUDA. */
int gbs_sample_batch(const gbs_kernel* k, int n_max, int samples, const double* uniforms, void* stream,
                     int* n_out, int* x_out);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of single-pattern probability requests      */
/* ------------------------------------------------------------------------ */

typedef struct gbs_serve_opts {
  int max_slots;          /* requests resident on the device at once (0 = 256) */
  size_t mem_budget;      /* device bytes for request state (0 = 64 MiB) */
  int queue_capacity;     /* pending requests accepted before GBS_EAGAIN (0 = 65536) */
  int subsets_per_step;   /* subset terms per request per step (0 = library choice) */
  int use_graphs;         /* 0 or 1: replay an instantiated CUDA graph per step (default);
                             -1: launch each step's copies and kernels directly */
  double wait_timeout_s;  /* bound on any internal wait (0 = 10 s) */
  int max_n;              /* largest photon number accepted (0 = GBS_MAX_N); a smaller
                             bound lets steps run more warps per SM */
  int fault_alloc_failures; /* testing: the first N admissions find the memory budget
                             used up (the request waits and is retried), 0 = none */
} gbs_serve_opts;

/* Start a server for kernel matrix k: a host thread admits requests into
 * device slots as slots and memory free up, and runs steps that advance every
 * resident request's subset sum together; partial sums stay on the device
 * between steps. Beside mem_budget the server keeps a pool of up to 256 MB
 * (less when max_slots requests of order max_n need less) for the pair sums
 * of FP64 requests of order >= 6; such a request is admitted once its pair
 * sums fit there. A request with n >= 26 is admitted once the ordering probe
 * of gbs_prob_batch has chosen its ordering (on a side stream, several
 * waiting requests per launch), so its subset sum cancels as little as in
 * the batched call. k must outlive the server. opts may be NULL. */
int gbs_serve_create(const gbs_kernel* k, const gbs_serve_opts* opts, gbs_server** out);

/* Enqueue one pattern (host index list of n entries, copied before return).
 * Non-blocking. ticket receives an id for gbs_serve_poll.
 * Errors: GBS_EAGAIN (queue full), GBS_ERANGE (n above the server's max_n, or
 * an index outside [0, m)), GBS_EINVAL. */
int gbs_serve_submit(gbs_server* s, const int* idx, int n, int precision, int64_t* ticket);

/* Returns 0 and fills p, haf_ri (2 doubles), err_est (each may be NULL) when
 * the request is done (its ticket is then released), 1 while it is pending,
 * or a negative error: GBS_ENOENT for an unknown or already-collected ticket;
 * for a request that ended without a result (its ticket is then released)
 * GBS_ECANCELED, GBS_ENOMEM (its partial sums exceed the whole memory budget),
 * GBS_ETIMEDOUT or GBS_ECUDA. */
int gbs_serve_poll(gbs_server* s, int64_t ticket, double* p, double* haf_ri, double* err_est);

/* Completion queue: collect up to max finished requests, in any order. When
 * none is finished and some are pending, waits up to timeout_s seconds (0 =
 * no wait) for one. Entry i of *count gets tickets[i] and, in each array that
 * is not NULL, p[i], haf_ri[2i..2i+1], err_est[i] and rc[i] (0, or the
 * negative code gbs_serve_poll would return for that ticket; its outputs are
 * then NaN). Collected tickets are released as by gbs_serve_poll. *count = 0
 * when the wait ran out or nothing is pending. A client serving many requests
 * collects them here instead of polling each ticket. The paper has no
 * counterpart (serving only). Errors: GBS_EINVAL. */
int gbs_serve_wait_any(gbs_server* s, double timeout_s, int max, int64_t* tickets, double* p,
                       double* haf_ri, double* err_est, int* rc, int* count);

/* Cancel a request: 0 when it was still pending (its ticket then polls
 * GBS_ECANCELED; device work already in flight for it finishes and is
 * discarded, and its slot and memory are freed after that), 1 when it had
 * already finished (poll it as usual), GBS_ENOENT for an unknown or collected
 * ticket. Host-side only: the paper has no counterpart. */
int gbs_serve_cancel(gbs_server* s, int64_t ticket);

/* Counters of a server since creation (for monitoring; the paper has no
 * counterpart). Step wall time runs from a step's launch to the host seeing
 * its completion event. */
typedef struct gbs_serve_stats_t {
  int64_t steps;          /* steps launched */
  int64_t items;          /* work items dispatched */
  int64_t subsets;        /* subset terms dispatched */
  int64_t completed;      /* requests finished on the device */
  double step_wall_s;     /* summed step wall time (launch to detected completion) */
  double step_wall_max_s; /* longest step */
  double step_device_s;   /* summed step device time (CUDA events around the step) */
  double step_device_max_s; /* longest step on the device */
  double poll_gap_max_s;  /* longest interval, while a step was in flight, between two
                             runs of the server thread's loop or completion polls
                             (large: the thread was not running) */
  double launch_max_s;    /* longest call that launches a step, of which: */
  double update_max_s;    /* longest update of a step graph's parameters */
  double submit_max_s;    /* longest submission of a step (graph launch, or the
                             direct copies and launches without graphs) */
  int64_t probed;         /* requests whose ordering the probe chose (n >= 26) */
  int64_t cancelled;      /* requests cancelled while pending */
  int64_t alloc_waits;    /* admissions that found the memory budget used up and waited */
  int64_t arena_slots;    /* partial sums the memory budget holds (a request needs one
                             per work item) */
} gbs_serve_stats_t;
int gbs_serve_stats(gbs_server* s, gbs_serve_stats_t* out);

/* Stop the server thread (after finishing resident work, bounded by the
 * timeout) and free its resources. */
int gbs_serve_destroy(gbs_server* s);

/* Thread-local message describing the last error on this thread ("" if none). */
const char* gbs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GBS_H */
