/*
 * GSVD-MUSIC sound source localization on GB300 (sm_103a): C ABI.
 *
 * The method is the one of Lin et al., "An Efficient GPU-based Implementation
 * for Noise Robust Sound Source Localization" (arXiv 2504.03373), Sec. III-A:
 *   correlation (eq. 2-3) -> whitening by the preset noise correlation K and
 *   the singular value decomposition of K^{-1} R (eq. 4, Sec. III-B) -> noise
 *   subspace E_n (Sec. III-A) -> MUSIC spectrum (eq. 5) -> sum over bins
 *   (eq. 6) -> peak search (Sec. III-A, last paragraph).
 *
 * Conventions for every call below
 *  - Complex numbers are interleaved (re, im) float pairs ("c64"); a complex
 *    array of n elements is 2n floats.  All matrices are row-major.
 *  - Pointers are DEVICE pointers unless a call says otherwise.  The caller
 *    owns every buffer it passes; the library never frees caller memory.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Every
 *    call is asynchronous on that stream; outputs are valid once the stream
 *    has been synchronised.  Argument errors are returned synchronously;
 *    numeric failures are written to the per-item `status` arrays on the
 *    device and OR-ed into the context's sticky device flags
 *    (ssl_device_flags).  No call traps or aborts the device.
 *  - A context is bound to one device and must not be used from two host
 *    threads at once.  Its calls may go to different streams: the calls
 *    that use the context's workspace (ssl_gsvd, ssl_gevd, ssl_music_spectrum,
 *    ssl_localize*, ssl_gsvd_f64) are ordered after one another on the
 *    device by the library (each waits for the previous one's work, on
 *    whatever stream it ran), except inside a stream capture, where the
 *    caller orders the captured work.
 *  - Limits: 1 <= M <= SSL_MAX_M, 1 <= Ns < M, T >= 1, B >= 1, D >= 1,
 *    n_az * n_el == D <= SSL_MAX_D.
 */
#ifndef SSL_GSVD_MUSIC_H
#define SSL_GSVD_MUSIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ssl_status;

#define SSL_OK 0
#define SSL_E_INVALID_ARG 1    /* bad pointer, size or enum; nothing launched */
#define SSL_E_NOT_PD 2         /* K(w) not positive definite (Cholesky pivot <= 0) */
#define SSL_E_NO_CONVERGENCE 3 /* Jacobi reached max_sweeps with rotations still applied */
#define SSL_E_NONFINITE 4      /* NaN/Inf met in an input matrix */
#define SSL_E_OOM 5            /* device allocation failed */
#define SSL_E_ADMISSION 6      /* serving: request refused by the memory budget */
#define SSL_E_TIMEOUT 7        /* a bounded device wait gave up */
#define SSL_E_CUDA 8           /* a CUDA runtime call failed; see ssl_last_error */
#define SSL_E_UNSUPPORTED 9    /* valid request this library does not implement */
#define SSL_E_CAPACITY 10      /* request larger than a fixed, preallocated capacity */

/* Sticky device flags (bit mask), see ssl_device_flags. */
#define SSL_FLAG_NOT_PD (1u << 0)
#define SSL_FLAG_NO_CONVERGENCE (1u << 1)
#define SSL_FLAG_NONFINITE (1u << 2)
#define SSL_FLAG_TIMEOUT (1u << 3)
#define SSL_FLAG_BOUNDS (1u << 4) /* bounds-checked debug build only: an index check
                                   * failed and its access was skipped */

/* Denominator of eq. 5. */
#define SSL_FORM_ABS 0 /* sum_{i>Ns} |h^H e_i|   (as printed in eq. 5) */
#define SSL_FORM_SQ 1  /* sum_{i>Ns} |h^H e_i|^2 (basis-invariant MUSIC form) */

/* Arithmetic of the spectrum contraction h^H E_n. */
#define SSL_PREC_FP32 0 /* FP32 FMA on the SIMT cores */
#define SSL_PREC_TF32 1 /* tcgen05 kind::tf32 tensor cores, FP32 accumulation in TMEM */
#define SSL_PREC_BF16 2 /* tcgen05 kind::f16 with bf16 operands, FP32 accumulation in TMEM */
#define SSL_PREC_TF32X3 3 /* 3xTF32 on tcgen05 kind::tf32: each FP32 operand split into
                           * TF32 high and low parts, three products per step (FP32 class);
                           * stateless calls (ssl_music_spectrum, ssl_localize) only */

/* Arithmetic of the Jacobi rotation angles and convergence test. */
#define SSL_ANGLES_F64 0 /* FP64 decision and tan(theta) (default) */
#define SSL_ANGLES_F32 1 /* FP32 throughout */

#define SSL_MAX_M 64
#define SSL_MAX_D 8192
#define SSL_MAX_NS 16

typedef struct ssl_ctx ssl_ctx;
typedef struct ssl_steering ssl_steering;

/* Controls of the decomposition of eq. 4 (ssl_gsvd and every call that runs
 * it).  method SSL_SVD_JACOBI (default): one-sided Jacobi on A^H; a pair of
 * columns (g_p, g_q) is rotated only while
 *     |g_p^H g_q| > rel_tol * |g_p| |g_q|          (relative test) and
 *     |g_p^H g_q| > abs_tol * max_c |g_c|^2        (absolute test),
 * the absolute test being the Jacobi counterpart of Sec. III-B's tolerance
 * derived from the global maximum of the matrix.  It applies only to pairs
 * whose larger squared norm max(|g_p|^2, |g_q|^2) is at most
 * sqrt(abs_tol) * max_c |g_c|^2 (pairs of small columns); a pair with a
 * larger column is held to the relative test alone, so the absolute test
 * never leaves a large singular vector mixed with a small one (the residual
 * it allows moves singular vectors by |g_p^H g_q| / (|g_p|^2 - |g_q|^2)).
 * The iteration ends once a
 * sweep's worth of consecutive rounds rotates nothing, or after max_sweeps.
 * method SSL_SVD_BIDIAG: the paper's route (Sec. III-B, SVD1-SVD6 of Alg. 1):
 * Householder bidiagonalisation, phase transform, implicit-shift QR with
 * deflation below abs_tol (else 2^-23) times the largest column sum
 * |d_i| + |e_{i-1}| of the real bidiagonal (SVD2's global maximum), sort,
 * back-transformation; FP32 throughout (rel_tol and angles unused;
 * max_sweeps * 64 bounds the QR iterations; statistics report QR iterations
 * and Givens rotations). */
#define SSL_SVD_JACOBI 0
#define SSL_SVD_BIDIAG 1
/* method SSL_SVD_SPLIT: the noise subspace without its individual vectors,
 * for the SQ form of eq. 5, which depends on E_n only through the projector
 * E_n E_n^H = I - E_s E_s^H.  One-sided Jacobi on A's columns restricted to
 * pairs of one of the Ns pivot columns (the largest) with one other column,
 * plus the pivot pairs; a rotation keeps the larger column in the pivot.  Same
 * tests, tolerances and angle arithmetic as SSL_SVD_JACOBI.  At convergence
 * the pivots are sigma_s E_s; E's first Ns columns are E_s (sorted), the
 * remaining M - Ns columns an orthonormal basis of the complement (the
 * trailing columns of the Householder Q of E_s, not singular vectors), and
 * sigma's entries past Ns the norms of the other columns of A V sorted
 * descending (their squares sum to sum_{i>Ns} sigma_i^2, they are not the
 * individual singular values).  A matrix still rotating after
 * min(8, max_sweeps) sweeps of M - Ns rounds, or one whose pivot-partner
 * couplings after the preconditioning show that the rounds would not finish
 * (sigma_{Ns+1} close to sigma_Ns), is solved again by SSL_SVD_BIDIAG (its
 * status, sigma, E and stats are then that route's); every matrix with
 * Ns > 8 or 3 Ns > M takes SSL_SVD_JACOBI.  Needs Ns:
 * split_ns in ssl_gsvd, ssl_gsvd_kinv and ssl_gsvd_noalloc, cfg.Ns in the
 * calls that take a config, which refuse it with the ABS form
 * (SSL_E_UNSUPPORTED: that form needs the individual noise vectors). */
#define SSL_SVD_SPLIT 2
typedef struct ssl_jacobi_opts {
  int max_sweeps; /* <= 0: 30 */
  float rel_tol;  /* <= 0: M * 2^-24 */
  float abs_tol;  /* <= 0: no absolute test (full relative accuracy) */
  int angles;     /* SSL_ANGLES_F64 or SSL_ANGLES_F32 */
  int method;     /* SSL_SVD_JACOBI (0), SSL_SVD_BIDIAG or SSL_SVD_SPLIT */
  int split_ns;   /* SSL_SVD_SPLIT in the calls without a config: Ns (1..M-1) */
} ssl_jacobi_opts;

/* ------------------------------------------------------------------------
 * Context
 * --------------------------------------------------------------------- */

/* Create a context on CUDA device `device`.  *out receives the handle.
 * Allocates a small device flag word; the workspace grows on demand. */
ssl_status ssl_create(ssl_ctx** out, int device);

/* Destroy a context (synchronises the device first).  NULL is a no-op. */
ssl_status ssl_destroy(ssl_ctx* ctx);

/* Copy the last error message of `ctx` (NUL-terminated, truncated to len). */
ssl_status ssl_last_error(const ssl_ctx* ctx, char* buf, size_t len);

/* Synchronise `stream`, then read and clear the sticky device flags
 * (SSL_FLAG_* bits raised by any kernel of this context since the last
 * read).  *flags is a host pointer. */
ssl_status ssl_device_flags(ssl_ctx* ctx, void* stream, uint32_t* flags);

/* Limit, in ns, of each bounded wait inside the context's tensor-core
 * spectrum kernels (the hand-offs between their copy, MMA and epilogue
 * roles); 0 restores the default of 0.25 s.  A wait that runs out makes the
 * kernel stop its pipeline, wait (with the default limit) for the copies and
 * MMAs it has in flight, release its tensor memory and return; the launch
 * then raises SSL_FLAG_TIMEOUT and its spectrum is incomplete.  No paper
 * counterpart: it lets a caller with a tighter deadline, or a test, make the
 * waits give up sooner.  Applies to calls issued after it. */
ssl_status ssl_set_wait_limit(ssl_ctx* ctx, uint64_t ns);

/* Test hook for the failure path above: with on != 0, the context's
 * tensor-core spectrum launches (ssl_music_spectrum, ssl_localize) issue no
 * operand load at all, so their MMA role waits for data that never arrives
 * until the wait limit runs out; the launch then stops cleanly and raises
 * SSL_FLAG_TIMEOUT, and its spectrum is not computed.  on = 0 restores
 * normal operation.  No paper counterpart. */
ssl_status ssl_set_test_stall(ssl_ctx* ctx, int on);

/* ------------------------------------------------------------------------
 * Stateless steps of the hot path
 * --------------------------------------------------------------------- */

/* Correlation, eq. 2-3 (AddCorrelation + NormalizeCorrelation), read
 * block-wise: for each block k and bin w,
 *     R[k][w] = (1/T) sum_{f<T} x_f x_f^H,   x_f = X[k][f][w][0..M-1].
 * X: c64 [nblk][T][B][M].  R: c64 [nblk][B][M][M] (full Hermitian matrix).
 * Also used for K from noise-only frames (nblk = 1, T = number of frames). */
ssl_status ssl_correlate(ssl_ctx* ctx, const float* X, int nblk, int T, int B, int M,
                         float* R, void* stream);

/* Inverse of the preset noise correlation (eq. 4, Sec. III-B), computed in
 * FP64 through the Cholesky factorisation K = L L^H, K^{-1} = L^{-H} L^{-1}.
 * K: c64 [B][M][M] Hermitian (lower triangle is read).  Kinv: c64 [B][M][M].
 * status: int32 [B], 0 or SSL_E_NOT_PD / SSL_E_NONFINITE (Kinv zeroed). */
ssl_status ssl_noise_inverse(ssl_ctx* ctx, const float* K, int B, int M, float* Kinv,
                             int32_t* status, void* stream);

/* Generalised SVD of eq. 4: A = K^{-1} R = E Lambda E_r^H per (block, bin),
 * by one-sided Jacobi on A^H with FP32 data (angles per opts->angles).
 * K (c64 [B][M][M], shared by all blocks) is inverted with
 * ssl_noise_inverse into the context workspace.
 * R: c64 [nblk][B][M][M].  opts: NULL for the defaults.
 * sigma: f32 [nblk][B][M], descending.
 * E: c64 [nblk][B][M][M]; column i of E[k][w] is the left singular vector
 *    e_{i+1} (so E_n is columns Ns..M-1).
 * status: int32 [nblk][B] or NULL (0, SSL_E_NO_CONVERGENCE, SSL_E_NONFINITE). */
ssl_status ssl_gsvd(ssl_ctx* ctx, const float* R, const float* K, int nblk, int B, int M,
                    const ssl_jacobi_opts* opts, float* sigma, float* E, int32_t* status,
                    void* stream);

/* As ssl_gsvd, with K^{-1} (c64 [B][M][M]) supplied by the caller.
 * stats: optional int32 [nblk][B][2] receiving, per (block, bin), the number
 * of column pairs tested (inner products g_p^H g_q formed between two of
 * the M columns; a full sweep tests M (M - 1) / 2) and of rotations applied
 * (NULL to skip).  SSL_SVD_BIDIAG: implicit-QR iterations and rotations;
 * SSL_SVD_SPLIT: pivot-partner rounds after the batched test and rotations,
 * or SSL_SVD_BIDIAG's pair for a matrix handed to that route. */
ssl_status ssl_gsvd_kinv(ssl_ctx* ctx, const float* R, const float* Kinv, int nblk, int B, int M,
                         const ssl_jacobi_opts* opts, float* sigma, float* E, int32_t* status,
                         int32_t* stats, void* stream);

/* SEVD-MUSIC's decomposition (Sec. II, Sec. IV-B: MUSIC without a noise
 * correlation, the K = I case of eq. 4): R = E Lambda E^H per (block, bin),
 * R Hermitian PSD, by the same one-sided Jacobi with the identity for
 * K^{-1}.  R: c64 [nblk][B][M][M].  lambda: f32 [nblk][B][M] eigenvalues,
 * descending.  E: c64 [nblk][B][M][M], column i = eigenvector i.  status as
 * ssl_gsvd.  The paper has no separate SEVD kernel; this is eq. 4 with K = I. */
ssl_status ssl_sevd(ssl_ctx* ctx, const float* R, int nblk, int B, int M,
                    const ssl_jacobi_opts* opts, float* lambda, float* E, int32_t* status,
                    void* stream);

/* GEVD-MUSIC's decomposition (the generalised eigenproblem of the pair
 * (R, K) that Sec. II contrasts with the GSVD): R e = lambda K e.  K = L L^H
 * (FP64 Cholesky), W = L^{-1}; the Hermitian PSD matrix W R W^H is
 * decomposed by one-sided Jacobi (FP32 data) and E = W^H Y.  lambda: f32
 * [nblk][B][M], descending; E: c64 [nblk][B][M][M], columns K-orthonormal
 * (E^H K E = I).  Under R = s a a^H + sigma^2 K the columns Ns..M-1 are
 * exactly orthogonal to a.  K: c64 [B][M][M].  status as ssl_gsvd.  Uses the
 * context workspace (2 B M^2 + 2 nblk B M^2 complex values). */
ssl_status ssl_gevd(ssl_ctx* ctx, const float* R, const float* K, int nblk, int B, int M,
                    const ssl_jacobi_opts* opts, float* lambda, float* E, int32_t* status,
                    void* stream);

/* Allocation-free form of ssl_gsvd for callers that may not allocate device
 * memory: real-time audio threads whose per-block deadline cannot absorb a
 * cudaMalloc (which may synchronise the device), and host frameworks that own
 * the device memory budget and forbid library-side allocations.  The paper
 * has no counterpart; it is an interface addition of this library.
 * Same arguments and results as ssl_gsvd, without a context.  The scratch
 * (K^{-1} and one status word per bin) lives in a fixed 8 MiB array compiled
 * into the library (2^20 complex values) that every GPU loading the library
 * keeps until the process exits; requests with
 * B * M * M + ceil(B / 2) > 2^20 return SSL_E_CAPACITY before launching
 * anything.  The call runs on the current device; its first call on a device
 * looks up the array's device address (a one-time host-side step), so make
 * that first call before any stream capture.  All calls share the array and
 * it keeps the last call's contents (nothing needs to start at zero); calls
 * that overlap on the GPU, e.g. on two streams, race on it.
 * status (int32 [nblk][B]) is required here: with no context there is no
 * sticky flag word, so it is the only error channel.  A bin whose K is not
 * positive definite (or holds NaN/Inf) gets SSL_E_NOT_PD (SSL_E_NONFINITE)
 * in every block, with K^{-1} = 0 behind it (sigma = 0).
 * Returns SSL_OK, SSL_E_INVALID_ARG, SSL_E_CAPACITY or SSL_E_CUDA. */
ssl_status ssl_gsvd_noalloc(const float* R, const float* K, int nblk, int B, int M,
                            const ssl_jacobi_opts* opts, float* sigma, float* E,
                            int32_t* status, void* stream);

/* Steering table (H of eq. 5): copies H (c64 [B][D][M], device or host
 * pointer) into a library-owned object holding the FP32 table, the squared
 * norms |h^H h| and the tensor-core operand images (built on first use). */
ssl_status ssl_steering_create(ssl_ctx* ctx, const float* H, int B, int D, int M,
                               ssl_steering** out);
ssl_status ssl_steering_destroy(ssl_steering* st);

/* Analytic steering (the steering vectors h of eq. 5 in closed form for a
 * free field and far-field sources): h_m(d, w) = exp(+j 2 pi f_w (u_d . p_m) / c)
 * for microphone positions pos (f32 [M][3], metres), direction unit vectors
 * dirs (f32 [D][3]) and bin frequencies freqs (f32 [B], Hz), speed of sound
 * c (m/s).  Host or device pointers, copied (synchronous).  The object holds
 * only the geometry (a few KB): with the TF32 and BF16 tensor-core spectra the kernel
 * generates each steering tile where it is consumed (phase reduced to
 * [-1/2, 1/2] turns in FP32, hardware sine/cosine, about 2^-21 absolute,
 * below the operand rounding) and takes |h|^2 = M; the paths that read a
 * table (FP32 SIMT, 3xTF32, FP64, mixed plans, streams) build the c64 table
 * from the geometry on first use (phases in FP64).  The paper's H is a
 * measured table (Sec. V); this is the free-field model of it.  Returns
 * SSL_E_INVALID_ARG for non-finite inputs or c <= 0. */
ssl_status ssl_steering_create_analytic(ssl_ctx* ctx, const float* pos, const float* dirs,
                                        const float* freqs, float c, int B, int D, int M,
                                        ssl_steering** out);

/* Neighbour lists of a direction set that is not a grid, for the peak search
 * (Sec. III-A, last step; the paper's measured transfer functions cover 2522
 * directions over the sphere, Sec. V, which form no n_el x n_az grid).
 * Compressed rows: the neighbours of direction d are
 * nbr_idx[nbr_ptr[d] .. nbr_ptr[d + 1] - 1].  nbr_ptr: int32 [D + 1],
 * nbr_idx: int32 [n_edges]; host or device pointers, copied (synchronous).
 * The lists must start at 0, not decrease, end at n_edges and hold indices
 * in [0, D) (else SSL_E_INVALID_ARG, nothing attached); an entry equal to d
 * is ignored.  They replace any lists attached before.  A steering object
 * with lists serves ssl_peaks_nbr and ssl_localize with cfg->n_el == 0. */
ssl_status ssl_steering_set_neighbours(ssl_steering* st, const int32_t* nbr_ptr,
                                       const int32_t* nbr_idx, int n_edges);

/* Search range of the peak search (Sec. III-A, last step: peaks are searched
 * in the directional range theta_min .. theta_max): in_range is D bytes (host
 * or device, copied; synchronous), nonzero for the directions inside the
 * range; NULL removes the range (every direction).  Only directions inside
 * the range are reported as peaks; the peak test of such a direction still
 * compares it with all of its neighbours.  Applies to every call that uses
 * this steering object for the peak search (ssl_peaks_nbr, the localization
 * calls, sessions, streams, plans); ssl_peaks, which takes no steering
 * object, searches the whole grid. */
ssl_status ssl_steering_set_search_range(ssl_steering* st, const uint8_t* in_range);

/* MUSIC spectrum, eq. 5, and its sum over bins, eq. 6:
 *   P[k][w][d] = |h^H h| / sum_{i=Ns}^{M-1} |h^H e_i|      (form ABS)
 *              = |h^H h| / sum_{i=Ns}^{M-1} |h^H e_i|^2    (form SQ)
 *   Pbar[k][d] = sum_w P[k][w][d]   (fixed bin order, deterministic)
 * with h = H[w][d], e_i = column i of E[k][w].  A zero denominator is
 * clamped to FLT_MIN.  E: c64 [nblk][B][M][M].  P: f32 [nblk][B][D] or NULL.
 * Pbar: f32 [nblk][D]. */
ssl_status ssl_music_spectrum(ssl_ctx* ctx, const float* E, int nblk, int B, int M, int Ns,
                              const ssl_steering* st, int form, int precision, float* P,
                              float* Pbar, void* stream);

/* Peak search (Sec. III-A): on an n_el x n_az grid (d = e * n_az + a),
 * d is a peak iff for each of its 8 neighbours n (azimuth wraps, elevation
 * rows outside the grid are dropped) Pbar[d] > Pbar[n], or they are equal
 * and d < n.  The Ns largest peaks (ties to the lower index) are returned;
 * missing ones as idx -1, val 0.  Pbar: f32 [nblk][D].  idx: int32
 * [nblk][Ns].  val: f32 [nblk][Ns]. */
ssl_status ssl_peaks(ssl_ctx* ctx, const float* Pbar, int nblk, int n_az, int n_el, int Ns,
                     int32_t* idx, float* val, void* stream);

/* Peak search (Sec. III-A) over the direction set of `st`, whose neighbour
 * lists (ssl_steering_set_neighbours) take the place of the grid: d is a peak
 * iff for each listed neighbour n != d, Pbar[d] > Pbar[n], or they are equal
 * and d < n.  The Ns largest peaks (ties to the lower index), missing ones as
 * idx -1, val 0.  Pbar: f32 [nblk][D].  idx: int32 [nblk][Ns].  val: f32
 * [nblk][Ns].  SSL_E_INVALID_ARG if st has no neighbour lists. */
ssl_status ssl_peaks_nbr(ssl_ctx* ctx, const float* Pbar, int nblk, const ssl_steering* st,
                         int Ns, int32_t* idx, float* val, void* stream);

/* ------------------------------------------------------------------------
 * The whole hot path
 * --------------------------------------------------------------------- */

typedef struct ssl_config {
  int M;          /* microphones (1..SSL_MAX_M) */
  int T;          /* frames per block */
  int B;          /* frequency bins */
  int Ns;         /* sources (signal-subspace size) */
  int n_az;       /* direction grid: azimuth columns */
  int n_el;       /* direction grid: elevation rows; D = n_az * n_el.  In
                   * every call that takes an ssl_config (localization,
                   * sessions, streams, plans), n_el = 0 selects a direction
                   * set of D = n_az directions whose peak search uses the
                   * steering object's neighbour lists
                   * (ssl_steering_set_neighbours; required then) */
  int form;       /* SSL_FORM_* */
  int precision;  /* SSL_PREC_* */
  ssl_jacobi_opts jacobi;
} ssl_config;

/* Localize nblk independent blocks: correlation -> K^{-1} (FP64 Cholesky) ->
 * whitening + Jacobi SVD -> E_n -> spectrum -> bin sum -> peaks.
 * X: c64 [nblk][T][B][M]; K: c64 [B][M][M]; both may be DEVICE or HOST
 * pointers (host data is copied in on `stream`).  peak_idx: int32
 * [nblk][Ns], peak_val: f32 [nblk][Ns], Pbar: f32 [nblk][D] or NULL; each
 * may be a device or a host pointer (host outputs are copied back on
 * `stream`; synchronise it before reading them). */
ssl_status ssl_localize(ssl_ctx* ctx, const float* X, int nblk, const float* K,
                        const ssl_steering* st, const ssl_config* cfg, int32_t* peak_idx,
                        float* peak_val, float* Pbar, void* stream);

/* As ssl_localize with K^{-1} (c64 [B][M][M], device or host; e.g. from
 * ssl_noise_inverse, computed once per preset K) in place of K: a caller that
 * localizes many batches against one noise correlation skips the FP64
 * Cholesky of K (eq. 4, Sec. III-B) in every call.  Same results as
 * ssl_localize given the K^{-1} that ssl_noise_inverse returns for K. */
ssl_status ssl_localize_kinv(ssl_ctx* ctx, const float* X, int nblk, const float* Kinv,
                             const ssl_steering* st, const ssl_config* cfg, int32_t* peak_idx,
                             float* peak_val, float* Pbar, void* stream);

/* ------------------------------------------------------------------------
 * The FP64 path: the same method with every sum, product and decision in
 * double precision (the FP32 frames, noise correlation and steering table
 * widened).  It is the accuracy reference on the GPU, against which the FP32
 * path's error separates from the method's; it is slower (FP64 issues at a
 * small fraction of the FP32 rate on this part).
 * --------------------------------------------------------------------- */

/* eq. 4 in FP64: K^{-1} (FP64 Cholesky of the c64 K [B][M][M], kept in FP64)
 * times R (complex double [nblk][B][M][M]), and the SVD of that product by
 * one-sided Jacobi on complex doubles: a pair rotates while
 * |g_p^H g_q| > rel_tol |g_p| |g_q| (rel_tol <= 0: M 2^-53) and, for pairs of
 * small columns (larger squared norm at most sqrt(abs_tol) max |g|^2), while
 * |g_p^H g_q| > abs_tol max_c |g_c|^2; the iteration ends after a sweep
 * without a rotation or after max_sweeps (SSL_E_NO_CONVERGENCE).  opts->angles
 * is ignored; opts->method must be SSL_SVD_JACOBI (else SSL_E_UNSUPPORTED).
 * sigma: double [nblk][B][M] descending; E: complex double [nblk][B][M][M]
 * (columns = left singular vectors); status: int32 [nblk][B] or NULL; stats:
 * int32 [nblk][B][2] (pairs tested, rotations) or NULL.  Device pointers. */
ssl_status ssl_gsvd_f64(ssl_ctx* ctx, const double* R, const float* K, int nblk, int B, int M,
                        const ssl_jacobi_opts* opts, double* sigma, double* E, int32_t* status,
                        int32_t* stats, void* stream);

/* The whole hot path in FP64: correlation (FP64 sums) -> K^{-1} (FP64
 * Cholesky) -> whitening and one-sided Jacobi SVD (ssl_gsvd_f64's controls
 * from cfg->jacobi) -> E_n -> spectrum (FP64 SIMT) -> bin sum -> peaks.
 * X: c64 [nblk][T][B][M]; K: c64 [B][M][M]; st as for ssl_localize
 * (cfg->n_el == 0: its neighbour lists).  cfg->precision is ignored.
 * peak_idx: int32 [nblk][Ns]; peak_val: double [nblk][Ns]; Pbar: double
 * [nblk][D] or NULL.  DEVICE pointers only (SSL_E_INVALID_ARG otherwise). */
ssl_status ssl_localize_f64(ssl_ctx* ctx, const float* X, int nblk, const float* K,
                            const ssl_steering* st, const ssl_config* cfg, int32_t* peak_idx,
                            double* peak_val, double* Pbar, void* stream);

/* ------------------------------------------------------------------------
 * Sessions and serving (continuous batching of many arrays' blocks)
 *
 * The paper processes one array's blocks at fixed intervals (Sec. VI); these
 * calls serve many arrays at once.  A session holds one array's K^{-1}
 * (computed once, FP64 Cholesky), a caller-owned steering object and a ring
 * of device slots for its blocks in flight.  The server batches every queued
 * block of every session into one launch per stage per shape class, each
 * block with its own array's K^{-1} and steering, and keeps up to two
 * batches on the GPU: blocks submitted while a batch runs join the next one.
 * All server calls are driven from one host thread.
 * --------------------------------------------------------------------- */

typedef struct ssl_server ssl_server;
typedef struct ssl_session ssl_session;
typedef uint64_t ssl_ticket;

typedef struct ssl_array_desc {
  ssl_config cfg;  /* shape and method options of this array */
  int queue_depth; /* device slots for blocks in flight (>= 1) */
} ssl_array_desc;

typedef struct ssl_result {
  int32_t done;                    /* 1 once the fields below are valid */
  int32_t status;                  /* SSL_OK or the block's largest per-bin SSL_E_* */
  int32_t peak_idx[SSL_MAX_NS];    /* first cfg.Ns entries used, as ssl_peaks */
  float peak_val[SSL_MAX_NS];
  uint64_t t_arrival_ns;           /* as submitted */
  uint64_t t_done_ns;              /* server clock (ssl_now_ns) at retirement */
} ssl_result;

typedef struct ssl_stats {
  uint64_t blocks_done, batches, sessions, sessions_refused, blocks_refused, blocks_pending;
  size_t hbm_budget, hbm_used; /* admission budget and the sessions' footprint */
  size_t hbm_work;             /* batch working memory (outside the budget) */
  double busy_ms;              /* wall time with at least one batch on the GPU */
  double latency_p50_ms, latency_p99_ms, latency_max_ms; /* t_done - t_arrival */
} ssl_stats;

/* Steady host clock in ns, the time base of t_arrival / t_done. */
ssl_status ssl_now_ns(uint64_t* out);

/* Server on ctx's device with an admission budget (bytes of session state)
 * and a maximum number of blocks per batch. */
ssl_status ssl_server_create(ssl_ctx* ctx, size_t hbm_budget_bytes, int max_batch,
                             ssl_server** out);
/* Synchronises, frees every session of the server and the server. */
ssl_status ssl_server_destroy(ssl_server* srv);

/* New session.  K: c64 [B][M][M] (device or host); st must outlive the
 * session and match cfg's B, D, M.  Returns SSL_E_INVALID_ARG for a shape,
 * form, precision or Jacobi option that the stateless calls reject,
 * SSL_E_ADMISSION if the session's footprint (K^{-1} + queue_depth input
 * slots) exceeds the remaining budget, SSL_E_NOT_PD / SSL_E_NONFINITE if
 * some K(w) cannot be factored.  Synchronous (K^{-1} is ready on return, and
 * so is the steering object's tensor-core image for cfg.precision, so that no
 * server step has to build one); a device K is read only after all work on
 * the device has finished, so it may come from any stream. */
ssl_status ssl_session_create(ssl_server* srv, const ssl_array_desc* desc, const float* K,
                              const ssl_steering* st, ssl_session** out);
/* Frees a session, also while some of its blocks are in flight (a client
 * that went away): its queued blocks are dropped, and batches on the GPU that
 * hold some of its blocks are waited for and retired (their other blocks'
 * results go to their sessions as usual); this session's results, retired or
 * not yet polled, are discarded.  Other sessions are unaffected.  Returns
 * SSL_E_CUDA (and keeps the session) if waiting for a batch fails. */
ssl_status ssl_session_destroy(ssl_session* sess);

/* Saved session state (checkpoint / resume of a server's sessions; the paper
 * has no counterpart).  The state is the array config, the queue depth and
 * K^{-1} (c64 [B][M][M]) behind a small versioned header, in host memory of
 * ssl_session_state_size bytes; blocks in flight and unpolled results are not
 * part of it, and the steering object stays the caller's.  ssl_session_save
 * is synchronous (SSL_E_INVALID_ARG if len is too small).
 * ssl_session_restore creates a session on srv from such a state and a
 * steering object that matches its config, without repeating the Cholesky of
 * K: same admission and errors as ssl_session_create, and SSL_E_INVALID_ARG
 * for a state that is not one (wrong header, size or non-finite K^{-1}).  A
 * restored session serves blocks exactly as the saved one did. */
ssl_status ssl_session_state_size(const ssl_session* sess, size_t* bytes);
ssl_status ssl_session_save(const ssl_session* sess, void* buf, size_t len);
ssl_status ssl_session_restore(ssl_server* srv, const void* buf, size_t len,
                               const ssl_steering* st, ssl_session** out);

/* Queue one block X (c64 [T][B][M], host or device) with its arrival time.
 * The copy into the session's slot runs on the server's own copy stream and
 * is not ordered after any stream of the caller: X must be complete when the
 * call is made (host data, or device data whose producer has been
 * synchronised; else use ssl_session_submit_after).  The copy is
 * asynchronous: device memory and pinned host memory must stay valid and
 * unchanged until the block is retired (pageable host memory is copied
 * before the call returns).  Returns SSL_E_ADMISSION while all of the
 * session's slots are in flight. */
ssl_status ssl_session_submit(ssl_session* sess, const float* X, uint64_t t_arrival_ns,
                              ssl_ticket* out);
/* As ssl_session_submit, with the copy ordered after the work already issued
 * to `stream` (a cudaStream_t, NULL = the legacy default stream): for a device
 * X still being produced on that stream. */
ssl_status ssl_session_submit_after(ssl_session* sess, const float* X, uint64_t t_arrival_ns,
                                    void* stream, ssl_ticket* out);
/* Non-blocking: out->done = 0 until the ticket's block has been retired; a
 * retired result is returned once and then forgotten. */
ssl_status ssl_session_poll(ssl_session* sess, ssl_ticket t, ssl_result* out);
/* Drives ssl_server_run_step until the ticket is retired or timeout_ns passes
 * (SSL_E_TIMEOUT). */
ssl_status ssl_session_wait(ssl_session* sess, ssl_ticket t, uint64_t timeout_ns,
                            ssl_result* out);

/* One serving step: retire finished batches, then launch one batch of all
 * queued blocks (up to max_batch) if a batch slot is free.  *launched and
 * *retired (may be NULL) receive the block counts. */
ssl_status ssl_server_run_step(ssl_server* srv, int* launched, int* retired);
ssl_status ssl_server_stats(ssl_server* srv, ssl_stats* out);
/* Clears the latency record and the counters (not the sessions). */
ssl_status ssl_server_reset_stats(ssl_server* srv);

/* ---- Streams: per-frame processing with a sliding window -----------------
 * The sliding form of eq. 3 (Sec. III-A sums the correlation over the past
 * frames; Sec. VI names processing at shorter intervals): a stream keeps the
 * last cfg->T frames of one array on the device and, for every hop new
 * frames, recomputes R over that window and runs eq. 4-6 and the peak
 * search.  The decomposition continues from the previous window's E (the
 * Jacobi rotations restart from V0 = E_prev, whitening by E_prev^H K^{-1}),
 * which needs a fraction of the rotations of a cold start; results agree
 * with the block path on the same window within its tolerance.  Until T
 * frames have arrived the missing frames count as zero (R is then scaled by
 * the frames present over T, which changes neither E nor the peaks). */
typedef struct ssl_stream ssl_stream;

/* cfg: M, T (window frames), B, Ns, grid, form, precision, Jacobi options.
 * hop: frames per push, 1..T.  K: c64 [B][M][M], host or device, copied;
 * its inverse is taken once (SSL_E_NOT_PD if K is not positive definite).
 * st: steering table [B][D][M], kept by reference.  Synchronous. */
ssl_status ssl_stream_create(ssl_ctx* ctx, const ssl_config* cfg, int hop, const float* K,
                             const ssl_steering* st, ssl_stream** out);
/* X: c64 [hop][B][M], host or device (copied on `stream` before the call's
 * kernels).  Outputs (host or device): peak_idx int32 [Ns], peak_val f32
 * [Ns], Pbar f32 [D] or NULL, stats int32 [B][2] (pairs tested, rotations
 * per bin; device memory) or NULL.  Asynchronous on `stream`; pushes of one
 * stream must be issued on one CUDA stream. */
ssl_status ssl_stream_push(ssl_stream* s, const float* X, int32_t* peak_idx, float* peak_val,
                           float* Pbar, int32_t* stats, void* stream);
ssl_status ssl_stream_destroy(ssl_stream* s);

/* ---- Mixed batches: many arrays of different sizes in one pass ----------
 * The per-array steps of Sec. III-A (eq. 2-6 and the peak search) for n
 * arrays whose M, T, B, Ns and direction grids differ, run as one launch per
 * stage over all (array, bin) pairs: correlation, whitening + Jacobi SVD (a
 * persistent kernel that packs one 64-class, two 32-class or four 16-class
 * matrices into each CTA), spectrum, bin sum, peaks.  The paper has no
 * counterpart: it runs one array.  A plan fixes the arrays and buffers once;
 * each ssl_plan_run recomputes every array's result from the current
 * contents of its X buffer.  */
typedef struct ssl_plan ssl_plan;

typedef struct ssl_batch_item {
  ssl_config cfg;              /* M, T, B, Ns, n_az, n_el per array; form,
                                * precision and jacobi must agree across the plan */
  const float* X;              /* device c64 [T][B][M]: one block, caller-owned */
  const float* Kinv;           /* device c64 [B][M][M]: K^{-1} (ssl_noise_inverse) */
  const ssl_steering* steering;/* [B][D][M] table of this array */
  int32_t* peak_idx;           /* device int32 [Ns] */
  float* peak_val;             /* device f32 [Ns] */
  int32_t* status;             /* device int32 [1] (largest bin status) or NULL */
  float* Pbar;                 /* device f32 [D] or NULL */
} ssl_batch_item;

#define SSL_PLAN_GRAPH 1u    /* capture the stages in a CUDA graph at creation */
#define SSL_PLAN_AUTOTUNE 2u /* time the Jacobi size classes per M on the device */

typedef struct ssl_plan_info {
  int n_items;
  int n_bins;          /* (array, bin) pairs */
  int gsvd_units;      /* CTA work units of the Jacobi kernel */
  int gsvd_grid;       /* its persistent grid */
  int launches;        /* kernels per run */
  int graph;           /* 1 if runs replay a CUDA graph */
  int class_of_m[SSL_MAX_M + 1]; /* Jacobi size class (16/32/64) per M, 0 = unused */
  double autotune_ms;  /* time spent timing candidates at creation */
} ssl_plan_info;

/* Builds a plan over n items (all pointers device memory that stays valid
 * for the plan's lifetime).  flags: SSL_PLAN_*.  With SSL_PLAN_AUTOTUNE the
 * X buffers must hold representative data at creation: each M's matrices
 * are solved once per candidate size class and the fastest class is kept
 * (classes differ in the order of the Jacobi rotations, not in accuracy).
 * The plan allocates its own scratch (R, E, spectra); creation synchronises
 * the device.  Returns SSL_E_INVALID_ARG (mismatched or invalid items),
 * SSL_E_OOM, SSL_E_CUDA. */
ssl_status ssl_plan_create(ssl_ctx* ctx, int n, const ssl_batch_item* items, unsigned flags,
                           ssl_plan** out);
/* One pass over all arrays, asynchronous on `stream`.  Runs of one plan share
 * its scratch: issue them on one CUDA stream (or order them yourself). */
ssl_status ssl_plan_run(ssl_plan* plan, void* stream);
ssl_status ssl_plan_get_info(const ssl_plan* plan, ssl_plan_info* out);
ssl_status ssl_plan_destroy(ssl_plan* plan);

#ifdef __cplusplus
}
#endif

#endif /* SSL_GSVD_MUSIC_H */
