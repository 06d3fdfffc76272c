/*
 * mra.h -- C ABI of the GB300 Synch-EM library (libmra.so).
 *
 * Synch-EM for 2-D multi-reference alignment (Janco & Bendory, "An accelerated
 * expectation-maximization algorithm for multi-reference alignment").  The
 * library runs the hot path of the method on one CUDA device: Synchronize and
 * Match, the learned rotation prior, the windowed prior-weighted EM iteration
 * and the marginal log-likelihood with its gradient.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Coefficients.  An image is stored by its steerable coefficients a_{k,q} for
 *   the angular index k = 0..K and the radial index q = 0..Q-1 (the k < 0 half
 *   is the complex conjugate for a real image, Sec. 1).  M = (K+1) Q.  A
 *   coefficient array is row-major [K+1][Q] of complex numbers stored as
 *   interleaved (re, im) pairs.  Observations y are [N][K+1][Q] complex float
 *   (8 bytes per coefficient), image-major.  Norms run over the M stored
 *   entries.
 * Rotations.  Rotating an image by phi multiplies a_{k,q} by exp(-i k phi)
 *   (Eq. fb_rotation); observations follow y_i = x o exp(-i k theta_i) + eps_i
 *   (Eq. MRA_Model_FB).  Rotations live on the grid theta = 2 pi s / L, s an
 *   integer "shift" in [0, L).
 * Window.  The EM searches the Lw offsets l0, l0+1, ..., l0+Lw-1 (mod L)
 *   around the synchronized estimate (Sec. 3.3); the paper's band [-BW/2,
 *   BW/2] is Lw = BW + 1, l0 = -BW/2.  Arrays over the window are [Lw], index i
 *   meaning offset l0 + i, the rotation theta_i = 2 pi step (l0 + i) / L.
 *   step = 1 is the grid; 0 < step < 1 is the denser-resolution window of
 *   Sec. 3.3 (the same number of rotations over a narrower range): its angles
 *   lie off the grid, it must span less than the circle ((Lw - 1) step < L,
 *   Lw <= 65536, |l0| <= 2^24) and Lw may exceed L.  The paper's example range
 *   [-pi BW/L, pi BW/L] at spacing pi BW/L^2 is Lw = 2 L + 1, l0 = -L,
 *   step = BW / (2 L).  Alignment shifts and the stopping rule stay on the grid.
 * Alignment.  Where an entry point takes shift (device int32 [N] or NULL),
 *   image j is used as y_j o exp(+2 pi i k shift[j] / L) (the alignment step
 *   before Eq. synch_initialization), folded into the kernels; y is never
 *   rewritten.  NULL means the images are used as given.
 * Memory.  Every array argument is a DEVICE pointer on the current CUDA device
 *   unless marked "host".  The caller owns every buffer; nothing is allocated
 *   inside a call.  Scratch memory is the caller's workspace (ws, ws_bytes),
 *   256-byte aligned, sized by the matching *_workspace_bytes query; its
 *   contents need no initialisation and are not preserved between calls.
 *   Observations y must be 16-byte aligned.
 * Streams.  stream is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Calls are asynchronous on that stream except where noted;
 *   outputs are valid once the stream has reached the call.
 * Errors.  Every entry point returns an mra_status.  Arguments are checked on
 *   the host before any launch; on error nothing is launched and outputs are
 *   untouched.  A device-side failure (a bounded wait that ran out) is
 *   recorded in the workspace status word and returned by the next call that
 *   synchronizes (mra_em_run, mra_ws_status).
 */
#ifndef MRA_H
#define MRA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MRA_API __attribute__((visibility("default")))

typedef enum {
  MRA_OK = 0,
  MRA_EINVAL = -1,     /* bad dimensions, NULL or misaligned pointer, a window the limits exclude, ... */
  MRA_ENOMEM = -2,     /* a host-side allocation inside the library failed */
  MRA_ECUDA = -3,      /* a CUDA runtime call failed (launch, copy, graph) */
  MRA_ETIMEOUT = -4,   /* a bounded device-side wait ran out; the kernel returned early */
  MRA_ENUMERIC = -5,   /* non-finite value where a finite one is required */
  MRA_EWORKSPACE = -6  /* ws_bytes smaller than the workspace query */
} mra_status;

/* Problem size.  sigma2 is the noise variance per stored complex entry
 * (E|eps|^2 = sigma2, Eq. MRA_Model_FB); beta = 1/sigma2.
 * Limits: N >= 1, K >= 0, Q >= 1, (K+1)*Q even, L >= 1, sigma2 > 0. */
typedef struct {
  int32_t N, K, Q, L;
  double sigma2;
} mra_dims;

/* Parameters of Algorithm Synch-EM (inputs L, rho_bar, BW, gamma, Gamma_a, tol, T). */
typedef struct {
  int32_t Lw;                /* window size, 1 <= Lw <= L on the grid (see Window above for step < 1) */
  int32_t l0;                /* first window offset (|l0| <= 2^30; taken mod L on the grid) */
  double gamma;              /* prior weight gamma >= 0 of p(rho) ~ exp(-gamma KL(rho_bar, rho)) */
  const double* log_rho_bar; /* device [Lw] log rho_bar on the window (-inf allowed); may be NULL if gamma == 0 */
  const double* gamma_a_inv; /* device [(K+1)*Q] diagonal of Gamma_a^{-1} (>= 0), or NULL for a flat image prior */
  int32_t update_rho;        /* 1: rho_{t+1} = (W + gamma rho_bar)/sum; 0: rho kept fixed */
  double tol;                /* mra_em_run stops after the iteration whose step is < tol; <= 0 never stops early */
  int32_t max_iters;         /* mra_em_run: at most this many iterations (T) */
  int32_t check_every;       /* mra_em_run: iterations per CUDA-graph launch between host checks (>= 1) */
  float* sweep_ms;           /* mra_em_run: host [max_iters] device time (ms) of each iteration's sweep over y,
                                from CUDA events recorded around the sweep kernel; NULL = not timed.  When set,
                                the run synchronizes after every graph launch. */
  double step;               /* spacing of the window's rotations in grid units, 0 < step <= 1 (0 is read as 1,
                                the grid): theta_i = 2 pi step (l0 + i) / L (Sec. 3.3, denser resolution) */
} mra_em_params;

MRA_API const char* mra_status_string(int status);

/* Number of streaming multiprocessors and the persistent-grid size the EM
 * sweep uses on the current device (host outputs).  Useful for sizing; a runtime
 * query with no counterpart in the paper. */
MRA_API int mra_device_info(int32_t* num_sms, int32_t* sweep_grid);

/* ------------------------------------------------------------------ EM */

/* Workspace bytes for mra_em_step, mra_em_run and mra_loglik_grad (sizing of the
 * caller-owned scratch; no counterpart in the paper). */
MRA_API size_t mra_em_workspace_bytes(const mra_dims* dims, int32_t Lw);

/* One iteration of Algorithm Synch-EM (E-step with Eq. weights_2d_em on the
 * window, normalisation, W_t, the a-update of Eq. coefficients_update and the
 * prior-weighted rho update), plus the stopping quantity.
 *   y          [N][K+1][Q] complex float observations
 *   shift      [N] int32 alignment shifts or NULL
 *   x_in       [K+1][Q] complex double a_t
 *   log_rho_in [Lw] double log rho_t on the window (-inf allowed, not all -inf)
 *   x_out      [K+1][Q] complex double a_{t+1}  (may alias x_in)
 *   log_rho_out[Lw] double log rho_{t+1}        (may alias log_rho_in)
 *   loglik_out [1] double: sum_j log sum_l rho_t[l] (pi sigma2)^{-M} exp(-||a_t o e^{-i k theta_l} - y_j||^2/sigma2)
 *   step_out   [1] double: min over all L grid rotations of ||a_{t+1} - e^{-2 pi i k l/L} a_t||^2
 *   w_out      [N][Lw] float posterior weights w_t^{l,j}, or NULL
 * Any of loglik_out, step_out may be NULL. */
MRA_API int mra_em_step(const mra_dims* dims, const mra_em_params* prm, const float* y, const int32_t* shift,
                        const double* x_in, const double* log_rho_in, double* x_out, double* log_rho_out,
                        double* loglik_out, double* step_out, float* w_out, void* ws, size_t ws_bytes,
                        void* stream);

/* Algorithm Synch-EM's loop: up to prm->max_iters iterations from (x_inout,
 * log_rho_inout), stopping after the first iteration whose step is < prm->tol.
 * The iterations run as CUDA-graph launches of prm->check_every iterations;
 * a device flag skips the remaining work of a launch once converged.  This
 * call synchronizes the stream between launches when tol > 0 and at the end.
 *   x_inout        [K+1][Q] complex double: a_0 in, final a out
 *   log_rho_inout  [Lw] double: log rho_0 in, final log rho out
 *   iters_out      host int32: iterations performed
 *   stats_out      [max_iters][2] double (loglik at a_t, step), or NULL
 *   x_traj_out     [max_iters][K+1][Q] complex double a_{t+1} per iteration, or NULL */
MRA_API int mra_em_run(const mra_dims* dims, const mra_em_params* prm, const float* y, const int32_t* shift,
                       double* x_inout, double* log_rho_inout, int32_t* iters_out, double* stats_out,
                       double* x_traj_out, void* ws, size_t ws_bytes, void* stream);

/* y as a BF16 hi/lo split (a storage format for the streamed observations, no
 * counterpart in the paper; the paper's method is unchanged).  Each pair of complex values (re0, im0, re1, im1)
 * of y occupies one 16-byte group: bf16 hi of the four values, then bf16 lo of
 * their residuals, hi = rn_bf16(v), lo = rn_bf16(v - hi); the kernels read
 * v = hi + lo, which FP32 holds exactly (relative error of the split <= 2^-16).
 * Same 8 bytes per complex value as complex64, same [N][K+1][Q] order.
 *   y        device [count] complex64, 16-byte aligned
 *   count    complex values, even (N (K+1) Q)
 *   y_hl_out device [count / 2] 16-byte groups, 16-byte aligned */
MRA_API int mra_y_split_bf16(const float* y, int64_t count, void* y_hl_out, void* stream);

/* Algorithm Synch-EM as mra_em_step / mra_em_run, with y in the BF16 hi/lo split (other
 * arguments as there).  Products and sums stay FP32 as in the complex64 path; the cross-image
 * reductions are FP64.  The batch sweep reads this format (the chunked sweep too,
 * where the autotuner or MRA_SWEEP=chunk chooses it); a window whose distance table
 * does not fit in shared memory next to the batch sweep's ring is read from global
 * memory.  MRA_EINVAL where no such sweep can take the shape (Q a multiple of 8 and
 * (K+1) Q / 4 <= 512 are required). */
MRA_API int mra_em_step_hl(const mra_dims* dims, const mra_em_params* prm, const void* y_hl, const int32_t* shift,
                           const double* x_in, const double* log_rho_in, double* x_out, double* log_rho_out,
                           double* loglik_out, double* step_out, float* w_out, void* ws, size_t ws_bytes,
                           void* stream);
MRA_API int mra_em_run_hl(const mra_dims* dims, const mra_em_params* prm, const void* y_hl, const int32_t* shift,
                          double* x_inout, double* log_rho_inout, int32_t* iters_out, double* stats_out,
                          double* x_traj_out, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ autotuner and batched runs
 * Neither has a counterpart in the paper, which treats one problem at a time. */

/* (No counterpart in the paper.)  Times every EM sweep that can take the problem
 * (the lean warp sweep and the paired-warp sweep, two warps per image, for grid windows of at
 * most 32 mirror units that are not the whole circle; the split sweep with its tcgen05 window transform for windows of 65 to 1024 rotations
 * and K+1 <= 48 (the default on the whole circle); the warp-per-image sweep; the batch sweep at
 * 16, 12, 8 or 4 images per batch and
 * 2 or 3 ring stages; the
 * chunked two-read sweep at 128, 64, 32 or 16 images per chunk and 1 or 2 CTAs per
 * SM) for one sweep over y from the state (x, log_rho), and caches the fastest for
 * this device and shape (a candidate later in this list replaces an earlier one only when it
 * is at least 1% faster) (K, Q, L, Lw, l0, step, y_format).  Later EM calls on that
 * shape use the cached choice unless the MRA_SWEEP* environment variables fix one.
 * Synchronizes the stream.
 *   y_format   0: y complex64; 1: the BF16 hi/lo split of mra_y_split_bf16
 *   choice_out host int32[3]: kind (1 warp, 2 batch, 3 chunked, 4 lean warp, 5 split,
 *              6 paired warps, 0 none applies),
 *              images per batch or chunk, ring stages or CTAs per SM; or NULL
 * The workspace is the one of mra_em_workspace_bytes; its contents are clobbered. */
MRA_API int mra_em_autotune(const mra_dims* dims, const mra_em_params* prm, const void* y, int32_t y_format,
                            const int32_t* shift, const double* x, const double* log_rho, int32_t* choice_out,
                            void* ws, size_t ws_bytes, void* stream);

/* One independent problem of a batched run (all pointers device, as in mra_em_run;
 * prm.max_iters iterations, prm.tol stops an instance early, prm.check_every and
 * prm.sweep_ms are not used). */
typedef struct {
  mra_dims dims;
  mra_em_params prm;
  const void* y;           /* [N][K+1][Q] complex64, or the BF16 hi/lo split */
  int32_t y_format;        /* 0 complex64, 1 BF16 hi/lo split */
  const int32_t* shift;    /* [N] or NULL */
  double* x_inout;         /* [K+1][Q] complex double: a_0 in, final a out */
  double* log_rho_inout;   /* [Lw] */
  double* stats_out;       /* [max_iters][2] (loglik, step) or NULL */
} mra_instance;

/* Workspace for mra_em_run_batched: the instances' EM workspaces, 256-byte aligned, in order,
 * then the persistent kernel's instance table and counters (sizing; no counterpart in the paper). */
MRA_API size_t mra_em_batched_workspace_bytes(const mra_instance* inst, int32_t n);

/* Algorithm Synch-EM's loop for n independent problems of uneven N, K and window
 * in ONE graph launch.  Where every instance has rows of 16 coefficients, complex64 y and a window
 * the lean warp sweep (or the warp sweep's any-window instance) takes, the graph holds the
 * instances' setups, ONE persistent cooperative kernel for all their iterations, and the exports:
 * one CTA per SM takes (instance, CTA slot) sweep items from a queue, then the instances'
 * reductions and updates, with a bounded grid barrier between the phases (a wait that runs out
 * ends the run with MRA_ETIMEOUT); each instance runs the arithmetic of its own launches of the same
 * sweep.
 * Otherwise (or with the environment variable MRA_BATCHED=graph) each instance's setup,
 * iterations and export are captured as a branch of the graph.  The graph is launched once and
 * synchronized.
 *   tune        1: run mra_em_autotune first for every shape not yet in the cache
 *   iters_out   host int32[n] iterations performed per instance, or NULL
 *   exec_ms_out host float: device time of the graph launch (CUDA events), or NULL
 * A repeated call with tune = 0 and the same instance array contents, workspace and
 * device launches the graph instantiated by the earlier call (a few are kept).
 * Returns the first failing status; instance results are valid only on MRA_OK. */
MRA_API int mra_em_run_batched(const mra_instance* inst, int32_t n, int32_t tune, int32_t* iters_out,
                               float* exec_ms_out, void* ws, size_t ws_bytes, void* stream);

/* Marginal log-likelihood over the window (Sec. 2.2, the likelihood of the observation model) and its
 * gradient (Fisher identity),
 *   l(x, kappa, eta) = sum_j log sum_l rho_l (pi sigma2)^{-M} exp(-||x o e^{-i k theta_l} - y_j||^2 / sigma2),
 *   log rho_l = kappa cos(theta_l) + eta_l - log sum_win exp(kappa cos theta + eta),
 *   theta_l = 2 pi step (l0+l)/L (step as in mra_em_params; 0 is read as 1).
 * The posterior is recomputed in one pass over y (never stored).
 *   x       [K+1][Q] complex double
 *   logits  [Lw] double eta (window logits)
 *   loglik_out [1] double
 *   dx_out  [K+1][Q] complex double dl/dRe x + i dl/dIm x = (2/sigma2)(sum_j sum_l w_jl e^{+i k theta_l} y_j - N x), or NULL
 *   dlogits_out [Lw] double dl/deta_l = W_l - N rho_l, or NULL
 *   dkappa_out  [1] double sum_l (W_l - N rho_l) cos theta_l, or NULL */
MRA_API int mra_loglik_grad(const mra_dims* dims, int32_t Lw, int32_t l0, double step, const float* y,
                            const int32_t* shift, const double* x, const double* logits, double kappa,
                            double* loglik_out, double* dx_out, double* dlogits_out, double* dkappa_out, void* ws,
                            size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ synchronization */

/* Workspace bytes for mra_sync and its parts (sizing; no counterpart in the paper). */
MRA_API size_t mra_sync_workspace_bytes(const mra_dims* dims, int32_t P);

/* Relative rotations of the first P images, Eq. (relative_angle_2d_dist):
 * rel[i][j] = argmin_s sum_{k,q} |y_i - e^{2 pi i k s/L} y_j|^2 for i < j
 * (smallest s on ties), rel[j][i] = (L - rel[i][j]) mod L, rel[i][i] = 0.
 *   rel_out [P][P] int32.  1 <= P <= N. */
MRA_API int mra_sync_pairwise(const mra_dims* dims, const float* y, int32_t P, int32_t* rel_out, void* stream);

/* Projected power method on H_ij = exp(-2 pi i rel[i][j] / L) (Eq. cost_synchronization):
 * z = 1, n_power steps z <- Hz/||Hz||, n_ppm steps z <- phase(Hz) with
 * phase(0) = 1, global phase fixed so that phi[0] = 0, then
 * phi[i] = floor(arg z_i L / (2 pi) + 1/2) mod L.
 *   rel [P][P] int32 in, phi_out [P] int32.  1 <= P <= 1024. */
MRA_API int mra_sync_ppm(int32_t L, int32_t P, const int32_t* rel, int32_t n_power, int32_t n_ppm, int32_t* phi_out,
                         void* stream);

/* Matching step of Algorithm Synchronize and Match: image i takes phi[n*],
 * n* = argmin_{n < P, n != i} ||y_i - y_n||^2 (smallest n on ties), scored as
 * ||y_n||^2 - 2 <y_i, y_n>.  For P <= 256 the inner products are one tcgen05 GEMM of all images with
 * the P references (each FP32 value split into three BF16 pieces, six piece products, FP32
 * accumulation) with the arg-min fused into its epilogue; a bounded wait that runs out sets the sync
 * workspace's status word (mra_ws_status(ws)) to MRA_ETIMEOUT.  Larger P use an FP32 CUDA-core tile kernel.
 *   phi [P] int32 in, shift_out [N] int32. */
MRA_API int mra_sync_match(const mra_dims* dims, const float* y, int32_t P, const int32_t* phi, int32_t* shift_out,
                           void* ws, size_t ws_bytes, void* stream);

/* Algorithm Synchronize and Match: pairwise + PPM on the first P images, then
 * matching for all N.  shift_out [N] int32. */
MRA_API int mra_sync(const mra_dims* dims, const float* y, int32_t P, int32_t n_power, int32_t n_ppm,
                     int32_t* shift_out, void* ws, size_t ws_bytes, void* stream);

/* Align and average, Eq. (synch_initialization): x_out = (1/N) sum_i y_i o e^{+2 pi i k shift_i/L}.
 *   x_out [K+1][Q] complex double.  Uses the EM workspace (mra_em_workspace_bytes with Lw = 1). */
MRA_API int mra_align_mean(const mra_dims* dims, const float* y, const int32_t* shift, double* x_out, void* ws,
                           size_t ws_bytes, void* stream);

/* Template matching (Sec. 2.1.1): every image against one reference,
 *   shift_out[j] = argmin_s sum_{k,q} |ref_kq - e^{2 pi i k s/L} y_jkq|^2   (grid index; smallest s among ties),
 * the relative rotation of Eq. (relative_angle_2d_dist) with the reference as the first image: aligning
 * y_j by shift_out[j] (as with the shifts of mra_sync) brings it to the reference's orientation.
 * O(N L M).  Robust only at high SNR (the paper's point), and the basis of App. B.
 *   ref [K+1][Q] complex float, 16-byte aligned (for example an observation, or a known signal);
 *   shift_out [N] int32.  No workspace. */
MRA_API int mra_template_match(const mra_dims* dims, const float* y, const float* ref, int32_t* shift_out,
                               void* stream);

/* ------------------------------------------------------------------ Fourier-Bessel front end (App. A) */

/* From n x n pixel images to the steerable coefficients a_{k,q}, k = 0..K, q = 1..Q, as the least-squares
 * solution over the sampled Fourier-Bessel basis
 *   u^{k,q}(r, theta) = N_{k,q} J_|k|(R_{|k|,q} r / c) e^{i k theta} for r <= c = (n - 1)/2, 0 beyond,
 *   R_{k,q} the q-th positive zero of J_k, N_{k,q} = 1 / (c sqrt(pi) |J_{k+1}(R_{k,q})|),
 * with a_{-k,q} = conj(a_{k,q}) (real images).  Pixel (row iy, column ix) sits at x = ix - c, y = iy - c,
 * theta = atan2(y, x); rotating an image by phi multiplies a_{k,q} by e^{-i k phi} (Eq. fb_rotation).
 * Limits: 3 <= n <= 1024, (K+1) Q even, and the sampling criterion R_{K,Q} <= pi n / 2 (checked as
 * Q + K/2 + 1/4 <= n/2).
 *
 * mra_fb_setup (once per n, K, Q; synchronizes the stream): computes the zeros, the design matrix, its
 * Gram matrix and inverse (FP64) and writes the projection P [n*n][K+1][Q] complex float: the coefficients
 * of an image are sum over pixels of image[pixel] * P[pixel].
 *   P_out      device, 16-byte aligned, n*n*(K+1)*Q complex float
 *   zeros_out  device [(K+1)][Q] double R_{k,q}, or NULL
 *   ws         workspace of mra_fb_setup_workspace_bytes(n, K, Q) bytes (about 16 n^2 (Q + 2KQ) bytes)
 * Returns MRA_ENUMERIC if a zero was not found or the inverse did not converge. */
MRA_API size_t mra_fb_setup_workspace_bytes(int32_t n, int32_t K, int32_t Q);
MRA_API int mra_fb_setup(int32_t n, int32_t K, int32_t Q, float* P_out, double* zeros_out, void* ws, size_t ws_bytes,
                         void* stream);

/* App. A, the Fourier-Bessel expansion of pixel images, applied to every image: the projection P of
 * mra_fb_setup is first packed into the operand of the library's tensor-core GEMM (P^T in 256-column
 * by 32-pixel tiles, each value split into three BF16 pieces that sum to it within 2^-24), once per P:
 *   mra_fb_operand_bytes(n, K, Q): size of that operand (0 for dimensions mra_fb_setup rejects);
 *   mra_fb_pack: op_out (device, 256-byte aligned) from P (device, as written by mra_fb_setup).
 * mra_fb_project: y_out [N][K+1][Q] complex float = images [N][n][n] float times P, one tcgen05 GEMM
 * over all images: the images are split into the same three pieces as they are read, six of the nine
 * piece products accumulate in FP32 (relative error ~1e-6, as FP32); fast != 0 keeps three of them
 * (relative error ~1e-5).  y_out has the layout every EM and synchronization entry point reads.
 * images and y_out 16-byte aligned, op 256-byte aligned.  A bounded wait that runs out leaves y_out
 * incomplete and sets the operand's status word to MRA_ETIMEOUT (read and cleared by
 * mra_ws_status(op, stream)). */
MRA_API size_t mra_fb_operand_bytes(int32_t n, int32_t K, int32_t Q);
MRA_API int mra_fb_pack(int32_t n, int32_t K, int32_t Q, const float* P, void* op_out, void* stream);
MRA_API int mra_fb_project(int32_t N, int32_t n, int32_t K, int32_t Q, const float* images, const void* op,
                           float* y_out, int32_t fast, void* stream);

/* Steerable PCA of coefficients (App. A: a data-driven radial basis per angular index k that keeps
 * steerability).  For every k the uncentred second moment C_k = (1/N) sum_i a_ik a_ik^H over the Q
 * radial entries (FP32 products summed in FP64 per chunk of 2,048 images, the chunks added in order), its
 * eigenvectors on the host (FP64 Jacobi), kept where the
 * eigenvalue exceeds sigma2 (1 + sqrt(Q/N))^2 (dims->sigma2 is the coefficients' noise variance).  Each
 * kept eigenvector's largest-magnitude entry is real positive; eigenvalues descend.  The reduced
 * coefficients b_ik = U_k^H a_ik have shape [K2+1][Q2]: K2 the largest k that keeps a component, Q2 the
 * largest count (plus one if (K2+1) Q2 would be odd); entries beyond a k's count are zero.  Rotations
 * still multiply b_ik by e^{-i k theta} and white noise stays white with the same variance.
 *
 * mra_spca_fit (synchronizes the stream): y [N][K+1][Q] complex float (device);
 *   basis_out device [K+1][Q][Q] complex float (column c of block k = the c-th eigenvector of C_k, zero
 *   beyond the kept count); eig_out host [K+1][Q] double or NULL; counts_out host [K+1] int32 or NULL;
 *   K2_out, Q2_out host; ws of mra_spca_workspace_bytes(dims) bytes.
 * mra_spca_project: y_out [N][K2+1][Q2] complex float = the reduced coefficients of y. */
MRA_API size_t mra_spca_workspace_bytes(const mra_dims* dims);
MRA_API int mra_spca_fit(const mra_dims* dims, const float* y, float* basis_out, double* eig_out, int32_t* counts_out,
                         int32_t* K2_out, int32_t* Q2_out, void* ws, size_t ws_bytes, void* stream);
MRA_API int mra_spca_project(const mra_dims* dims, const float* y, int32_t K2, int32_t Q2, const float* basis,
                             float* y_out, void* stream);

/* The eigenvectors of the steerable PCA step of App. A:
 * eigen-decomposition of a Hermitian n x n matrix (HOST pointers, column-major complex double, n <= 512):
 * w [n] descending, V [n][n] eigenvectors as columns, each with its largest-magnitude entry real positive.
 * FP64 cyclic Jacobi on the real symmetric embedding.  Used by mra_spca_fit; no GPU needed. */
MRA_API int mra_hermitian_eig(int32_t n, const double* A, double* w, double* V);

/* ------------------------------------------------------------------ rotation prior */

/* One trial of Algorithm 1 (learning the post-synchronization rotation distribution):
 * c = argmin_s ||xbar o e^{-2 pi i k s/L} - x_true||^2 with xbar = align_mean(y, shift_est),
 * r_j = (shift_true[j] - shift_est[j] + c) mod L, hist_inout[r_j] += 1.
 * r_j is the EM window offset of image j after alignment.
 *   x_true [K+1][Q] complex double, hist_inout [L] int32 (accumulated), center_out [1] int32 or NULL.
 * Uses the EM workspace (mra_em_workspace_bytes with Lw = 1). */
MRA_API int mra_prior_hist(const mra_dims* dims, const float* y, const int32_t* shift_true, const int32_t* shift_est,
                           const double* x_true, int32_t* hist_inout, int32_t* center_out, void* ws, size_t ws_bytes,
                           void* stream);

/* rho_bar from pooled residual counts (Algorithm 1, averaged over trials), on the window of
 * positions u_i = step (l0 + i) grid units (step as in mra_em_params; 0 is read as 1).
 *   kind 0: log_prior_out[i] = log(rho_bar[b_i] / sum over the window), b_i = floor(u_i + 1/2) mod L,
 *           the grid bin nearest to u_i ((l0+i) mod L on the grid)   (the learned histogram)
 *   kind 1: von Mises fit, kappa solving I1(kappa)/I0(kappa) = sum_s rho_bar[s] cos(2 pi s/L)
 *           (0 if that mean is <= 0), log_prior_out[i] = kappa cos(2 pi u_i / L) - log Z
 *   counts [L] int32, log_prior_out [Lw] double, kappa_out [1] double or NULL. */
MRA_API int mra_fit_prior(int32_t L, int32_t Lw, int32_t l0, double step, const int32_t* counts, int32_t kind,
                          double* log_prior_out, double* kappa_out, void* stream);

/* Relative error up to rotation (Sec. 2.2): min over continuous theta of
 * ||R_theta x_hat - x||/||x|| with the k > 0 rows counted twice (the k < 0 half).
 *   x_hat, x [K+1][Q] complex double; err_out [1] double. */
MRA_API int mra_relerr(int32_t K, int32_t Q, const double* x_hat, const double* x, double* err_out, void* stream);

/* mra_em_step for callers that cannot allocate device memory (no counterpart
 * in the paper).  Some callers cannot hand the library a workspace: code that
 * runs where another component owns all device memory and offers no extra
 * buffer, or code that must not call cudaMalloc/cudaFree because those calls
 * can synchronize the device.  This entry point takes the same arguments as
 * mra_em_step without ws/ws_bytes and computes the same results; its scratch
 * is one fixed array of 8 MiB that the library places in device memory when it
 * is loaded, on every device that loads it, until the process exits.  Nothing
 * is allocated by the call.
 *   - Problems whose EM workspace (mra_em_workspace_bytes) exceeds 8 MiB are
 *     rejected with MRA_EWORKSPACE.
 *   - The first call on a device looks up the array's device address (once per
 *     device, with that device current); make that first call before any CUDA
 *     stream capture.
 *   - All calls share the one array and it keeps the previous call's contents;
 *     the call initialises everything it reads.  Calls that overlap on the GPU
 *     (for example on two streams) race on the array: serialise them.
 *   - The array's address is looked up in the current context on every call,
 *     so calls after cudaDeviceReset get the array of the new context (its
 *     contents start over).
 *   - A bounded wait that runs out inside the step is recorded in the array's
 *     status word, which only mra_em_step_noalloc_status reads; the next call
 *     of this entry point resets it, so query it after each step whose outputs
 *     must be trusted. */
MRA_API int mra_em_step_noalloc(const mra_dims* dims, const mra_em_params* prm, const float* y, const int32_t* shift,
                                const double* x_in, const double* log_rho_in, double* x_out, double* log_rho_out,
                                double* loglik_out, double* step_out, float* w_out, void* stream);

/* Status of the last mra_em_step_noalloc on the current device (no counterpart
 * in the paper): synchronizes the stream, returns the fixed scratch's device
 * status word (MRA_OK, or MRA_ETIMEOUT when a bounded wait ran out and the
 * step's outputs are incomplete) and clears it.  MRA_ECUDA if the scratch's
 * address cannot be looked up. */
MRA_API int mra_em_step_noalloc_status(void* stream);

/* Synchronize the stream and return the workspace's device status word
 * (MRA_OK or MRA_ETIMEOUT), then clear it (failure detection; no counterpart in the paper). */
MRA_API int mra_ws_status(void* ws, void* stream);

/* Self-test of the device-side failure detection (no counterpart in the paper).
 * Launches one thread that waits on an mbarrier nothing arrives on, bounded by
 * limit_us microseconds (the same bounded wait every streaming kernel uses, whose
 * limit there is 2 s); when it gives up it writes MRA_ETIMEOUT, else MRA_OK.  The
 * wait ends by itself: no fault, the context stays usable.
 *   limit_us   1 .. 2,000,000
 *   status_out device int32[1], written by the kernel */
MRA_API int mra_selftest_wait_timeout(int32_t limit_us, int32_t* status_out, void* stream);

/* Self-test of the grid barrier that separates the iterations of a persistent batched run (no
 * counterpart in the paper).  One CTA per SM is launched cooperatively and meets at one grid
 * barrier that CTA 0 never reaches; every waiting CTA gives up after limit_us microseconds (the
 * batched run's limit is 2 s) and writes MRA_ETIMEOUT to scratch[2].  The waits end by themselves:
 * no fault, the context stays usable.
 *   limit_us   1 .. 2,000,000
 *   scratch    device int32[4], 16-byte aligned: cleared by the call, then the barrier's two words
 *              and the status (MRA_OK or MRA_ETIMEOUT) */
MRA_API int mra_selftest_grid_barrier(int32_t limit_us, int32_t* scratch, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MRA_H */
