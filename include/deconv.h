/*
 * deconv.h -- C ABI of the GB300 partial-ADMM deconvolution library
 * (libdeconv.so).
 *
 * Method: "A Framework for Fast Image Deconvolution with Incomplete
 * Observations" (Simoes, Almeida, Bioucas-Dias, Chanussot, arXiv:1602.01410).
 * The library minimises, over the extended sharp image x and the unobserved
 * blurred pixels z,
 *     1/2 || [y; z] - P T~ x ||^2 + lambda * TV(x)            (Eq. (problem_xz))
 * with the partial ADMM of Eqs. (admm_aprox_1)-(admm_aprox_4): one
 * block-Gauss-Seidel pass per iteration, the FFT-diagonalised x-step
 * (Eq. (dual_x_iter_resolved_boundaries)), the over-relaxed z-step
 * (Sec. II-B, coefficient `relax`, 2 in the paper), the isotropic TV
 * vector soft-threshold (Sec. III-B) or its vectorial form over 3 channels
 * (Sec. III-C, demosaicing) and the dual update.
 *
 * Conventions shared by every entry point:
 *   - Grid: each image is the extended M x N grid of the unknown x
 *     (M = m + 2b, N = n + 2b, Sec. I-A).  Pixels are row-major; an image
 *     of C channels is stored [C][M][N]; a batch is the concatenation of
 *     its images in order (image j starts at sum_{i<j} C*M_i*N_i elements).
 *   - Kernel h: (2b+1) x (2b+1), row-major, origin at h[b][b]; the blur is a
 *     true circular convolution on the extended grid (Eq. (4)).
 *   - Element type: float or double for every real array, chosen by
 *     deconv_dims.dtype; the FP64 reductions for statistics are double.
 *   - Memory: every array argument is DEVICE memory unless the name ends in
 *     _host.  The caller owns all memory, including the plan workspace; the
 *     library never allocates or frees device memory and never frees a
 *     caller pointer.
 *   - Streams: all device work is issued on the stream given at plan
 *     creation (a cudaStream_t passed as void*; NULL = legacy default
 *     stream).  Calls are stream-ordered and asynchronous unless stated.
 *   - Errors: functions return a deconv_status and never abort.  Argument
 *     errors are found on the host before any launch.  Errors that only the
 *     device can see (non-finite values) are recorded in the workspace and
 *     returned by deconv_sync.
 *   - Threads: a plan may be used by one host thread at a time.
 */
#ifndef DECONV_H
#define DECONV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct deconv_plan_s *deconv_plan; /* opaque; destroy with deconv_plan_destroy */

typedef enum {
  DECONV_OK = 0,
  DECONV_EINVAL = 1,       /* bad argument: sizes, kernel, lambda/mu, pointer, alignment */
  DECONV_EUNSUPPORTED = 2, /* a length with a prime factor > 5, or above the largest schedule */
  DECONV_ENOMEM = 3,       /* workspace smaller than deconv_workspace_size() */
  DECONV_ECUDA = 4,        /* a CUDA runtime call failed */
  DECONV_ETIMEOUT = 5,     /* a bounded device wait expired (reserved: no kernel waits on another) */
  DECONV_ENONFINITE = 6    /* a NaN or Inf reached the iterate */
} deconv_status;

enum { DECONV_F32 = 0, DECONV_F64 = 1 };

/* Problem geometry.  rows/cols are HOST arrays of `batch` entries (the
 * extended sizes M_j, N_j); every M_j, N_j must factor into 2, 3 and 5 and
 * be >= ksize.  channels is 1, or 3 for the vectorial TV of Sec. III-C.
 * ksize = 2b+1 is odd (Sec. I-A).  kernel_per_image = 0 shares one h across
 * the batch, 1 reads batch consecutive kernels.  relax is the z
 * over-relaxation coefficient (2 in Sec. II-B; 1 gives
 * Eq. (dual_z_iter_resolved_boundaries), the form Theorem 1 covers); it must
 * lie in [1, 2]. */
typedef struct {
  int32_t batch;
  int32_t channels;
  const int32_t *rows;
  const int32_t *cols;
  int32_t ksize;
  int32_t kernel_per_image;
  int32_t dtype; /* DECONV_F32 or DECONV_F64 */
  float relax;
  /* Uneven kernel supports in one batch: NULL, or host[batch], the odd
   * support 2b_j+1 <= ksize of image j's kernel (kernel_per_image must be 1).
   * h still holds ksize x ksize taps per image, image j's kernel centred in
   * them and zero outside its support (the blur is unchanged by the zero
   * taps); b_j sets image j's boundary band for the initial fill (Sec. III-B). */
  const int32_t *ksizes;
} deconv_dims;

/* Bytes of device workspace a plan for `dims` needs (under any tuning the
 * autotuner tries).  Host only. */
deconv_status deconv_workspace_size(const deconv_dims *dims, size_t *bytes);

/* Create a plan (Sec. II-B, the precomputation of the FFT-diagonalised
 * operators).  h: device, ksize*ksize elements (times batch when
 * kernel_per_image), dtype elements; the DC gain sum(h) must be non-zero,
 * which makes the solution unique (Sec. III-B, null spaces of H and D).
 * mask: device, one byte per pixel in the batch layout (C planes per image),
 * nonzero = observed.  The boundary band of width b should be unobserved for
 * the model of Eq. (4); the library does not require it.  lambda >= 0 is the
 * TV weight, mu > 0 the ADMM penalty.  workspace: device, 256-byte aligned,
 * at least deconv_workspace_size() bytes; the plan borrows it until
 * destroyed.  stream: cudaStream_t as void*.  Synchronises the stream once
 * (it reads h back to validate the DC gain). */
deconv_status deconv_plan_create(deconv_plan *out, const deconv_dims *dims, const void *h,
                                 const uint8_t *mask, double lambda, double mu, void *workspace,
                                 size_t workspace_bytes, void *stream);

/* Run `iters` >= 0 partial-ADMM iterations.  y: device, batch layout, dtype;
 * values at unobserved pixels are ignored.  warm = 0 initialises the state
 * from y (border padding of Sec. III-B, unobserved interior pixels set to the
 * mean of the observed ones); warm = 1 continues from the plan's state (y is
 * then unused and may be NULL).  x: device output, batch layout, receives
 * x^{iters} (may be NULL when iters == 0).  stats: NULL, or device
 * [batch][iters][3] doubles receiving per iteration ||d^{i+1} - d^i||^2,
 * ||z^{i+1} - z^i||^2 and the objective of Eq. (problem_xz) at x^{i+1}
 * minimised over z; stats mode launches the iteration kernels one by one
 * instead of replaying a CUDA graph.  Asynchronous. */
deconv_status deconv_solve(deconv_plan plan, const void *y, void *x, int32_t iters, int32_t warm,
                           double *stats);

/* Variants of the iteration (Sec. II-C and III-B), applied by every later
 * deconv_solve / deconv_solve_host call of the plan.
 *   bgs_passes: block-Gauss-Seidel passes of the x- and z-steps per iteration
 *     (Eqs. (admm_aprox_1)-(admm_aprox_2) repeated with v and d fixed), 1..64.
 *     1 is the paper's Proposed-1; b for a (2b+1) x (2b+1) blur its
 *     Proposed-AD.  The statistics describe the last pass.
 *   tikh_iters, tikh_tau: a fresh solve (warm = 0) first runs tikh_iters >= 0
 *     steps of the Tikhonov initialisation of Eqs. (ini_x)-(ini_z)
 *     (x = (H^T H + tau I)^{-1} H^T [y; z], z = M_z H x, no over-relaxation,
 *     tau = tikh_tau > 0; the paper uses 100 steps and tau = 1e-3), then starts
 *     the ADMM from y~ = [y; z], x^0 = the last x, v^0 = D x^0, d^0 = 0.
 *   adapt_t: 0 keeps mu fixed; >= 1 enables the penalty adaptation of
 *     Eq. (varying_penalty) with threshold t (the paper uses 3) per image.
 * Defaults: {1, 0, 1e-3, 0}.  Returns DECONV_EINVAL for values out of range.
 * Under adaptation every iteration adds a residual-norm pass over x and d
 * (the norms of Eq. (varying_penalty) are over all pixels of an image, so
 * they are complete only after that pass) before the forward half that
 * builds r with mu^{i+1}; v is kept in the workspace.
 * deconv_grad supports the defaults only (DECONV_EUNSUPPORTED otherwise). */
typedef struct {
  int32_t bgs_passes;
  int32_t tikh_iters;
  double tikh_tau;
  double adapt_t;
} deconv_options;

deconv_status deconv_set_options(deconv_plan plan, const deconv_options *opts);

/* Tuning of the launch shapes (the paper has no counterpart: it names no
 * GPU).  row_ctas / col_ctas: CTAs a register-FFT row class / the column
 * pass aims at (rows per CTA and spectral columns per CTA follow); 0 = the
 * default (152, one per SM).  row_stage: -1 = default (the forward row half
 * stages its rows in shared memory for one-channel plans of one row class),
 * 0 = reads them through L1, 1 = stages them (one channel only).
 * fft_values: 16 gives a row or column of length L to L/16 threads (more
 * resident warps), 32 to L/32 threads (fewer transposes).
 * l2_group_mb: the images of a batch are independent problems, so the
 * captured iteration loop runs them in groups, all iterations of one group
 * before the next, each group's row-spectral intermediate (C x M x (N/2+1)
 * complex pairs per image) at most l2_group_mb MiB so that it stays in the
 * 126 MB L2 from one pass to the next (an image larger than that forms a
 * group of its own); 0 = the default, one group (every pass over the whole
 * batch), as is -1.  generic: 1 runs every image through the shared-memory
 * Stockham passes (the path of lengths without a register transform), 0 =
 * register transforms wherever they apply.  fused_rows: 0 runs the row pass
 * of a plain iteration as two kernels (inverse half, forward half); 1 runs
 * it (one BGS pass, fixed mu, no statistics) as one fused kernel that takes
 * its row blocks from a work queue in order and waits, with a bound
 * (deconv_set_wait_limit), for the x rows of the blocks above it.
 * chains: 1 runs the captured loop of a batch as one chain per kernel
 * class (the images sharing a row and a column transform length): every
 * chain iterates on a stream of its own and the chains join only at the
 * end of the loop, so that no pass waits for the other classes' tails
 * (the images are independent problems); it replaces l2_group_mb. */
typedef struct {
  int32_t row_ctas;
  int32_t col_ctas;
  int32_t row_stage;
  int32_t fft_values;     /* register row transforms: complex values per thread, 16 or 32; 0 = default (16) */
  int32_t col_fft_values; /* the same for the column transforms; 0 = default (32 for power-of-two
                             lengths, 16 for 3 * 2^k and 5 * 2^k) */
  int32_t l2_group_mb;    /* image groups of the captured loop, MiB of intermediate per group; 0 or -1 = off */
  int32_t generic;        /* 1: Stockham passes for every image; 0: register transforms where they apply */
  int32_t fused_rows;     /* 0: two row kernels; 1: the fused row pass for plain iterations */
  int32_t chains;         /* 0: every pass over all classes; 1: one independent chain per kernel class */
} deconv_tune;

/* Bound of every device-side wait, in nanoseconds (default 2e9; the paper
 * has no counterpart).  The inverse row half waits for the bulk copies of
 * its row spectra into shared memory; the fused row pass
 * (deconv_tune.fused_rows) waits for flags of earlier work items of the
 * same image.  A wait that reaches the bound makes its block set an error
 * word and return (the inverse half without its rows, a fused item without
 * its forward half), and deconv_sync then returns DECONV_ETIMEOUT (the
 * results of that call are not valid).  0 allows no waiting at all: every
 * such wait fails at once (a test of the error path).  The captured CUDA graph is rebuilt.  ns >= 0,
 * else DECONV_EINVAL. */
deconv_status deconv_set_wait_limit(deconv_plan plan, int64_t ns);

/* Re-lays out a plan for another tuning (t = NULL: the defaults).  The
 * workspace of deconv_workspace_size() holds every tuning deconv_autotune
 * tries.  The iteration state is discarded (the next solve must be fresh).
 * Synchronises the stream. */
deconv_status deconv_retune(deconv_plan plan, const deconv_tune *t);
deconv_status deconv_get_tune(deconv_plan plan, deconv_tune *t);

/* Autotuner: times trial_iters iterations (rounded up to a whole number of
 * captured 20-iteration loops) three times (after a fresh solve of y that
 * builds the CUDA graph; the plan's options apply; the fastest repetition
 * counts) under the default tuning and each candidate (row_ctas and col_ctas
 * in {152, 608}, fft_values and col_fft_values in {16, 32}, and for one
 * channel and one row class row_stage in {0, 1}); then, for a problem of
 * at most 2^20 channel-pixels, the shared-memory passes (generic = 1) on
 * the fastest of those; then, for a batch, the image-group budgets
 * l2_group_mb in {24, 48, 80} and the chains (chains = 1), and the fused
 * row pass (fused_rows = 1), each on the fastest so far.
 * Keeps the fastest (best, best_ms_per_iter: nullable host outputs)
 * and leaves the plan in it with no iteration state.  y: device, batch
 * layout.  Synchronous. */
deconv_status deconv_autotune(deconv_plan plan, const void *y, int32_t trial_iters, deconv_tune *best,
                              float *best_ms_per_iter);

/* Arbitrary sizes (Sec. II-A: any pixel may be unobserved).  For an extended
 * grid of M x N that the library does not run (a prime factor > 5), the
 * smallest supported grid M_out x N_out >= M x N (smallest area among
 * 2-3-5-smooth sides) for the given channel count, kernel size and dtype.
 * The caller embeds its image at rows 0..M-1, columns 0..N-1 of the larger
 * grid with the added rows and columns unobserved (mask 0): they become
 * part of z, estimated like the boundary band.  The added band changes where
 * the circular TV wraps, so the result is that of the enlarged problem, not
 * of an M x N circular one.  Returns M_out = M, N_out = N when M x N runs as
 * it is.  Host only. */
deconv_status deconv_fast_shape(int32_t M, int32_t N, int32_t channels, int32_t ksize, int32_t dtype,
                                int32_t *M_out, int32_t *N_out);

/* The penalty mu each image's next iteration uses (mu_host: host, batch
 * doubles).  With adaptation off, or before the first fresh solve after it
 * was switched on, every entry is the plan's mu.  Synchronises the stream.
 * Under adaptation a warm solve (warm = 1) needs a fresh solve first, or a
 * state blob saved under adaptation (DECONV_EINVAL otherwise). */
deconv_status deconv_get_mu(deconv_plan plan, double *mu_host);

/* Same as deconv_solve with warm = 0 and no statistics, but y_host and
 * x_host are HOST buffers (pinned or pageable) in the batch layout: the call
 * copies y to the device, runs, copies x back and synchronises the stream
 * before returning.  Uses the workspace as staging; nothing is allocated. */
deconv_status deconv_solve_host(deconv_plan plan, const void *y_host, void *x_host, int32_t iters);

/* Gradient of the unrolled iteration (the differentiable use of the method:
 * learning lambda or the blur kernel through a fixed number of iterations).
 * L = mean over every pixel of the batch of (x^{iters} - x_true)^2, with
 * x^{iters} from deconv_solve(y, iters, warm = 0).  Returns L and dL/dlambda
 * on the host (loss, dlambda) and dL/dh in dh (device, the layout of h).
 * Reverse-mode differentiation of Eqs. (admm_aprox_1)-(admm_aprox_4) with
 * the over-relaxed z-update: the forward pass keeps (y~, d, forward
 * spectrum) every ckpt_every iterations and stores every step of its last
 * segment; the reverse pass recomputes each other segment from its
 * checkpoint (none when ckpt_every >= iters, at the cost of a workspace
 * holding every step) and runs the adjoint iteration backwards (the
 * x-step is self-adjoint; the vector soft-threshold contributes its
 * Jacobian, zero below the threshold).  grad_ws: device, 256-byte aligned,
 * at least deconv_grad_workspace_size() bytes.  x_out: NULL or device, the
 * batch layout, receives x^{iters}.  Row and column lengths with a register
 * transform only: 2^k for 64..1024 and 3 * 2^k, 5 * 2^k for 384..2560
 * (DECONV_EUNSUPPORTED otherwise).  Synchronises the stream; leaves the plan
 * state at x^{iters}'s last recomputed segment (use warm = 0 next). */
deconv_status deconv_grad_workspace_size(deconv_plan plan, int32_t iters, int32_t ckpt_every, size_t *bytes);
deconv_status deconv_grad(deconv_plan plan, const void *y, const void *x_true, int32_t iters, int32_t ckpt_every,
                          void *grad_ws, size_t grad_ws_bytes, double *loss, double *dlambda, void *dh, void *x_out);

/* Vector-Jacobian product of the unrolled iteration (the reverse pass of
 * deconv_grad with its seed given): for any scalar loss L(x^{iters}) of the
 * caller's, with xbar = dL/dx^{iters} (device, the batch layout, dtype),
 * returns dL/dlambda (host double) and dL/dh (device, the shape of h), so
 * the solve can sit under a loss of the caller's choice (the paper's
 * parameters lambda and the blur h of Eq. (model1) learned end to end).  Same
 * workspace, checkpointing, supported sizes and options as deconv_grad;
 * x_out (nullable) receives x^{iters}.  Synchronises the stream. */
deconv_status deconv_vjp(deconv_plan plan, const void *y, const void *xbar, int32_t iters, int32_t ckpt_every,
                         void *grad_ws, size_t grad_ws_bytes, double *dlambda, void *dh, void *x_out);

/* Allocation-free solve (the paper has no counterpart; this is a service of
 * the library).  For callers that may not allocate device memory: code
 * hosted inside a framework that owns the CUDA allocator, latency-critical
 * paths where an allocation could block, or plugins in a process whose
 * device memory was reserved up front.  Runs deconv_plan_create +
 * deconv_solve(warm = 0) + deconv_sync + deconv_plan_destroy with the plan
 * workspace placed in a 32 MiB array that the library reserves statically on
 * every GPU that loads it (held until the process exits); it calls no
 * cudaMalloc, cudaFree or other allocating routine and builds no CUDA graph.
 * Arguments are those of deconv_plan_create and deconv_solve (device h,
 * mask, y, x; host dims).  Returns DECONV_ENOMEM, before any launch, when
 * deconv_workspace_size(dims) exceeds 32 MiB (for example a single FP32
 * image up to about 700 x 700).  Every call looks up the array's device
 * address in the current device's context (so it stays valid after a
 * context is recreated); it synchronises the stream, so make no call while
 * that stream is being captured.  Every call on a device shares the one array
 * (plan creation clears what must start at zero), so calls whose work
 * overlaps on the GPU (other threads or streams) race: serialise them.
 * Synchronises `stream` and returns device-side errors like deconv_sync. */
deconv_status deconv_solve_noalloc(const deconv_dims *dims, const void *h, const uint8_t *mask,
                                   const void *y, void *x, double lambda, double mu, int32_t iters,
                                   void *stream);

/* Diagnostic timing inside the captured iteration loop (no counterpart in
 * the paper).  deconv_set_profiling(plan, 1) makes the plan record a CUDA
 * event on its stream before and after every column pass and every row pass
 * of the CUDA graph it replays (the graph is re-captured; 0 turns it off).
 * After a deconv_solve that replayed the graph, deconv_graph_pass_times
 * returns, from the events of the last replay, the mean time per iteration
 * of the column passes (ms_host[0]), of the row passes (ms_host[1]) and of
 * the whole iteration (ms_host[2]) (HOST array of 3 floats; summed over
 * image groups).  The events sit between passes, where they replace the
 * overlap of a pass's launch with the tail of the one before it.
 * Synchronises the stream.  DECONV_EINVAL if no profiled graph ran. */
deconv_status deconv_set_profiling(deconv_plan plan, int32_t on);
deconv_status deconv_graph_pass_times(deconv_plan plan, float *ms_host);

/* Diagnostic timing (no counterpart in the paper): continue from the plan's
 * state for `iters` >= 1 iterations launched one kernel at a time, with a
 * CUDA event before and after every launch on the plan's stream, and return
 * in ms_host[0] / ms_host[1] the mean duration of one column pass / one row
 * pass (HOST array of 2 floats).  Requires a state (a previous
 * deconv_solve).  Synchronises the stream. */
deconv_status deconv_profile_passes(deconv_plan plan, int32_t iters, float *ms_host);

/* Checkpoint / resume of the iteration state (Sec. II-B: the state carried
 * from one iteration to the next is y~ = [y; z], the scaled dual d_x and the
 * right-hand side of the next x-step).  The state is exported as an opaque
 * device blob of deconv_state_bytes() bytes (caller-owned, 16-byte aligned)
 * holding y~, d_x, the plan's forward row spectra and, for penalty
 * adaptation (Eq. (varying_penalty)), each image's current and previous mu,
 * the d rescaling and v_x, with a flag saying whether those were live;
 * deconv_state_set restores it into a plan of the same geometry, after which
 * deconv_solve(warm = 1) continues exactly where the saved plan stood (with
 * adaptation on in the restoring plan, only from a blob saved under
 * adaptation; otherwise the warm solve returns DECONV_EINVAL).
 * deconv_state_get queues device-to-device copies on the plan's stream and
 * writes the flag from host memory (which waits for the stream's earlier
 * work); deconv_state_set synchronises the stream. */
deconv_status deconv_state_bytes(deconv_plan plan, size_t *bytes);
deconv_status deconv_state_get(deconv_plan plan, void *blob);
deconv_status deconv_state_set(deconv_plan plan, const void *blob);

/* Diagnostic (no counterpart in the paper): number of kernel launches that
 * deconv_solve(plan, y, x, iters, warm = 0, NULL) (mode 0) or
 * deconv_grad(plan, ..., iters, ckpt_every, ...) (mode 1) issues.  Host only. */
deconv_status deconv_kernel_launches(deconv_plan plan, int32_t iters, int32_t mode, int32_t ckpt_every,
                                     int64_t *count);

/* Wait for the plan's stream and report device-side errors recorded since
 * the last call, then clear them.  DECONV_ENONFINITE: a NaN or Inf reached
 * the iterate (the kernels flag it and carry on; nothing traps).
 * DECONV_ETIMEOUT is reserved for a bounded device wait: no kernel of the
 * library spins on a flag or on another block (launches are ordered by the
 * stream and programmatic dependent launch), so it is not returned now. */
deconv_status deconv_sync(deconv_plan plan);

/* Release the plan's host resources (and its cached CUDA graph).  The
 * workspace is the caller's to free. */
deconv_status deconv_plan_destroy(deconv_plan plan);

/* Diagnostic: the last CUDA runtime error seen by this thread in the
 * library ("" if none), with its name and the library source line. */
const char *deconv_last_error(void);

/* Static string for a status code. */
const char *deconv_status_string(deconv_status status);

#ifdef __cplusplus
}
#endif

#endif /* DECONV_H */
