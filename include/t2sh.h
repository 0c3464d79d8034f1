/*
 * t2sh.h -- C ABI of the GB300 (sm_103a) T2 Shuffling PICS solver.
 *
 * The library solves, independently for every decoupled readout slice (Sec. II.A:
 * after the inverse FFT along the fully sampled readout the 3D problem splits into 2D
 * (ky, kz) problems), the T2 Shuffling reconstruction of Eq. 5:
 *
 *     argmin_alpha  1/2 || y - P F S Phi alpha ||_2^2  +  lambda sum_n || R_n(alpha) ||_*
 *
 * with FISTA (Sec. II.A, Sec. III.B).  The normal operator is applied through the
 * space-time kernel Psi(n) = Phi^T P(n) Phi (Sec. IV.B) and the LLR prox is the
 * singular-value soft threshold of non-overlapping b x b x K blocks of the randomly
 * circular-shifted coefficient images (Eq. 4, Sec. IV.C).  The SVT of each block is
 * formed from its K x K Gram matrix (float32 accumulation) and a cyclic Jacobi
 * eigendecomposition, in float32 unless T2SH_EIG_FP64 is set.
 *
 * Conventions shared by every entry point
 *   - Complex arrays are interleaved single precision (re, im), C order, last index
 *     fastest.  Shapes below name their dimensions; S = nslices, C = ncoils,
 *     M = nmaps, T = nechoes, K = nbasis.
 *   - F is the centred, unitary 2D DFT over (ny, nz): k-space arrays hold DC at
 *     (ny/2, nz/2), image arrays hold the image centre at (ny/2, nz/2).
 *   - Array arguments are DEVICE pointers owned by the caller, unless the plan was
 *     created with T2SH_HOST_IO, in which case the k-space, map, mask, basis and
 *     result arguments of t2sh_plan / t2sh_solve are HOST pointers (pinned memory
 *     recommended) and the library copies them through its own device buffers.
 *     Device pointers must be 16-byte aligned.
 *   - Work is enqueued on the plan's stream and is asynchronous unless stated.
 *   - Errors are reported by status code only; nothing is thrown across the ABI.
 *     t2sh_last_error() returns a message for the last failing call of the calling
 *     thread.  A plan is not thread-safe: use one plan per host thread and stream.
 *     Different plans may be made and used from different host threads at the same
 *     time (the library's shared state, its memory pool and launch caches, is locked).
 */
#ifndef T2SH_H
#define T2SH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  T2SH_OK = 0,
  T2SH_EINVAL = 1,       /* bad argument or unsupported dimension                      */
  T2SH_ENOMEM = 2,       /* device allocation failed or the workspace cap was exceeded */
  T2SH_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed                */
  T2SH_EUNSUPPORTED = 4, /* valid request that this build does not implement          */
  T2SH_ETIMEOUT = 5,     /* a bounded device wait ran out                              */
  T2SH_EBUSY = 6         /* the plan is in use                                         */
} t2sh_status;

/*
 * t2sh_dims.precision.  T2SH_FP32: every step in single precision.  T2SH_MIXED_BF16: the
 * column pass of the normal operator (DFT along ky, the space-time kernel Psi of Sec. IV.B,
 * inverse DFT) runs its DFTs as GEMMs on the tensor cores with operands split into BF16
 * hi/lo pairs and FP32 accumulation (about 16 significant bits per product); the stated
 * accuracy of this path is a per-slice NRMSE <= 1e-3 of the solve.  Shapes the tensor-core
 * kernel does not cover (ny not 16 R1 with R1 in {3,4,6,8,10,12,15,16}, nz % 4 != 0 or
 * nbasis > 4) use the FP32 column pass.  The paper has no mixed-precision variant.
 */
enum { T2SH_FP32 = 0, T2SH_MIXED_BF16 = 1 };

/* kform argument: layout of k-space data */
enum {
  T2SH_KSPACE_TE = 0,  /* zero-filled per-echo data      [S][C][T][ny][nz] complex */
  T2SH_KSPACE_PROJ = 1 /* projected data Phi^T P y       [S][C][K][ny][nz] complex */
};

/* t2sh_dims.flags */
#define T2SH_NO_SHIFT 0x1u /* LLR without random shifts (fixed block grid)            */
#define T2SH_HOST_IO 0x2u  /* array arguments of plan/solve are host pointers         */
#define T2SH_EIG_FP64 0x4u /* LLR Gram eigendecomposition in float64 (default float32) */
#define T2SH_FUSED_ROWS 0x8u /* t2sh_solve: one kernel per iteration for the row adjoint,
                                gradient step, LLR, momentum and row forward of each 8-row
                                LLR band (M = 1, K <= 4, block 8, nz in {48..192}); off by
                                default: measured slower than the separate kernels        */

typedef struct {
  int32_t ny, nz;          /* slice matrix (phase encodes y, z); both even, products of
                              2, 3, 5 and 13 (Table I: 260 x 240), 8 <= ny, nz <= 512     */
  int32_t ncoils;          /* C >= 1 (virtual coils after compression, Sec. III.A)       */
  int32_t nmaps;           /* M in {1, 2}: soft-SENSE map sets (Sec. II.A)               */
  int32_t nechoes;         /* T >= K: echo train length                                  */
  int32_t nbasis;          /* K in [1, 8]: subspace size (Eq. 3)                         */
  int32_t nslices;         /* S >= 1: decoupled readout slices solved together           */
  int32_t block;           /* LLR block edge b in [1, 16] (blocks b x b, Eq. 4)          */
  float lambda;            /* LLR weight lambda >= 0 (Eq. 4)                             */
  int32_t iters;           /* FISTA iterations >= 0                                      */
  uint64_t seed;           /* seed of the random LLR shifts                              */
  float step;              /* > 0: FISTA step mu; <= 0: the plan computes mu = 1/L with
                              L = max_n lambda_max Psi(n) * max_p lambda_max S(p)^H S(p) */
  int32_t precision;       /* T2SH_FP32 or T2SH_MIXED_BF16 (other values: T2SH_EINVAL)  */
  uint32_t flags;          /* T2SH_NO_SHIFT | T2SH_HOST_IO | T2SH_EIG_FP64 | T2SH_FUSED_ROWS */
} t2sh_dims;

typedef struct t2sh_plan_s* t2sh_plan_t;

/*
 * t2sh_plan -- validate dims, allocate the plan's device workspace and precompute
 * what every iteration shares (Sec. IV.B, Sec. IV.C "basis and space-time kernel
 * caching"):
 *   - Psi(n) = Phi^T P(n) Phi for every k-space point (real symmetric, upper triangle
 *     stored, Sec. IV.B), built from mask and phi;
 *   - the coil maps with the FFT centring sign (-1)^(y+z) folded in (Sec. IV.A);
 *   - the LLR shift table of all iterations (t2sh_shifts);
 *   - the step mu (dims.step, or 1/L as described above).
 *
 *   phi   [T][K]            float32, real temporal basis Phi (Eq. 3)
 *   mask  [T][ny][nz]       uint8 one-zero sampling pattern per echo (centred k-space)
 *   maps  [S][C][M][ny][nz] complex coil sensitivities S_{c,m} per slice
 *   stream                  cudaStream_t the plan enqueues on (NULL: default stream)
 *   out                     receives the plan handle; NULL on failure
 *
 * The inputs are copied; the caller may free them when t2sh_plan returns (it
 * synchronises the stream once to read back mu).  Errors: EINVAL (dims, NULL
 * pointers), ENOMEM (allocation), ECUDA.
 */
t2sh_status t2sh_plan(const t2sh_dims* dims, const float* phi, const uint8_t* mask,
                      const void* maps, void* stream, t2sh_plan_t* out);

/* Release every device buffer of the plan (after synchronising its stream).  Plan
 * buffers come from a library-owned, stream-ordered memory pool of the current device
 * that keeps released memory for the next plan (no fresh page mapping per plan); the
 * pool's unused memory goes back to the device with t2sh_release_cached. */
t2sh_status t2sh_destroy(t2sh_plan_t plan);

/* t2sh_release_cached -- return the pool's unused memory on the current device to the
 * device (memory of live plans stays).  Errors: ECUDA. */
t2sh_status t2sh_release_cached(void);

/*
 * t2sh_forward -- y = A x = P F S Phi x (Eq. 5 forward model; Eq. 1 per echo).
 *   x [S][M][K][ny][nz] complex (device)
 *   y kform == T2SH_KSPACE_TE:   [S][C][T][ny][nz] zero-filled per-echo k-space
 *     kform == T2SH_KSPACE_PROJ: [S][C][K][ny][nz] = Phi^T P A x = Psi (F S x)
 * Device pointers only.  Errors: EINVAL.
 */
t2sh_status t2sh_forward(t2sh_plan_t plan, const void* x, void* y, int32_t kform);

/*
 * t2sh_adjoint -- x = A^H y = S^H F^H Phi^T P y (the data term of the FISTA
 * gradient, Sec. II.A).  y as in t2sh_forward (a TE-form y is masked by P first);
 * x [S][M][K][ny][nz].  Device pointers only.
 */
t2sh_status t2sh_adjoint(t2sh_plan_t plan, const void* y, int32_t kform, void* x);

/*
 * t2sh_normal_op -- y = A^H A x = S^H F^H Psi F S x (Sec. IV.B, Algorithm 1).
 *   x, y [S][M][K][ny][nz] complex (device); x == y is allowed.
 */
t2sh_status t2sh_normal_op(t2sh_plan_t plan, const void* x, void* y);

/*
 * t2sh_llr_prox -- in place, x <- LLR prox of x with threshold tau (Eq. 4, Sec. IV.C):
 * for every map set m and block (i, j) covering rows (sy + i b + r) mod ny and
 * columns (sz + j b + c) mod nz (the last block per axis partial when b does not
 * divide the size), the (pixels x K) matrix X becomes U max(Sigma - tau, 0) V^H.
 *   x [S][M][K][ny][nz] complex (device); tau >= 0; 0 <= sy, sz < block.
 */
t2sh_status t2sh_llr_prox(t2sh_plan_t plan, void* x, float tau, int32_t sy, int32_t sz);

/*
 * t2sh_solve -- dims.iters FISTA iterations on Eq. 5 (Sec. II.A, Sec. III.B):
 *   x_0 = z_0 = 0, t_0 = 1;  g = z_k - mu (A^H A z_k - A^H y);
 *   x_{k+1} = LLR prox of g, threshold mu*lambda, shift of iteration k;
 *   t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2;  z_{k+1} = x_{k+1} + (t_k - 1)/t_{k+1} (x_{k+1} - x_k).
 *   kspace     per kform (see above); a TE-form input is masked and projected first
 *   alpha_out  [S][M][K][ny][nz] complex: x_iters
 *   residual_out  NULL, or host double[iters]: ||x_{k+1} - x_k||_2 / ||x_{k+1}||_2 over
 *              all slices; when non-NULL the call synchronises the stream.
 * With T2SH_HOST_IO, kspace and alpha_out are host pointers and the call returns
 * after alpha_out is written.
 */
t2sh_status t2sh_solve(t2sh_plan_t plan, const void* kspace, int32_t kform, void* alpha_out,
                       double* residual_out);

/*
 * t2sh_solve_admm -- the same problem (Eq. 5, Sec. II.A) solved by ADMM in scaled form
 * instead of FISTA, with the splitting alpha = v (the LLR term on v) and conjugate-gradient
 * alpha-updates.  From alpha = v = u = 0, for each of dims.iters iterations k:
 *   alpha <- cg_iters CG iterations on (A^H A + rho I) alpha = A^H y + rho (v - u), started
 *            at the previous alpha (per-slice float64 dot products);
 *   v     <- LLR prox of alpha + u with threshold lambda / rho and shift k (the FISTA
 *            shift sequence);
 *   u     <- u + alpha - v.
 * alpha_out receives v [S][M][K][ny][nz].  rho > 0 (finite), 0 <= cg_iters <= 1000.
 * residual_out (nullable, dims.iters doubles): ||v_{k+1} - v_k|| / ||v_{k+1}|| per
 * iteration.  The paper itself uses FISTA; this is the alternative solver loop.  Allocates
 * three more vectors in the plan on its first call.  Leaves no resumable state.
 */
t2sh_status t2sh_solve_admm(t2sh_plan_t plan, const void* kspace, int32_t kform, void* alpha_out, float rho,
                            int32_t cg_iters, double* residual_out);

/*
 * t2sh_objective -- the data term of Eq. 5 at x for every slice,
 *   f_s(x) = 1/2 || P F S Phi x_s - y_s ||^2 over the acquired samples,
 * returned in two parts, f_s = h_s + c_s:
 *   out[2 s]      h_s = 1/2 <x_s, A^H A x_s> - Re <x_s, A^H y_s>   (the part that depends on x)
 *   out[2 s + 1]  c_s = 1/2 sum_{c,t,n} P_t(n) |y_{s,c,t}(n)|^2 for T-form k-space; NaN for
 *                 projected k-space, which does not determine it.
 *   kspace, kform  as for t2sh_solve (host pointers with T2SH_HOST_IO)
 *   x              [S][M][K][ny][nz] complex (host with T2SH_HOST_IO)
 *   out            host double[2 S]
 * Inner products accumulate in float64 across threads.  One normal operator, one
 * A^H y and the reductions; the plan's gradient and intermediate buffers are scratch,
 * the solver state is not touched, so it may be called between t2sh_solve_iterate
 * calls.  Synchronises the stream.  Errors: EINVAL, ENOMEM (first call allocates the
 * accumulators), ECUDA.
 */
t2sh_status t2sh_objective(t2sh_plan_t plan, const void* kspace, int32_t kform, const void* x, double* out);

/*
 * t2sh_postprocess -- TE images from reconstructed coefficients (the "Process TE" step of
 * Sec. III.C and the Reconstruction paragraph of Sec. V): for each requested echo
 * te_index[i] (rows of the plan's basis Phi, 0-based) and each slice,
 *   x_m(t) = sum_k Phi[t][k] alpha[m][k]          back-projection with the basis (Eq. 3)
 *   x_c(t) = sum_m S_{c,m} x_m(t)                  virtual-coil images
 *   homodyne detection along z (the slice direction, partial Fourier fraction pf in
 *   (1/2, 1]): centred unitary DFT along z, acquired lines d in [-w, nz/2) with
 *   w = ceil(pf nz) - nz/2 (computed in double from the float pf), weighting 0 / 1 / 2
 *   outside / inside / beyond the two-sided band |d| <= w, phase from the band alone,
 *   result Re(IFFT(H k) exp(-i phase))
 *   out = sqrt(sum_c homodyne(x_c(t))^2)           root sum of squares
 * alpha: device [S][M][K][ny][nz] complex64; out: device [S][nte][ny][nz] float32 (caller
 * owned).  1 <= nte <= 8.  Asynchronous on the plan's stream.  Plans made with
 * T2SH_HOST_IO return T2SH_EUNSUPPORTED.  (The paper's 3D wavelet denoising that comes
 * before this step is t2sh_wavelet_denoise.)
 */
t2sh_status t2sh_postprocess(t2sh_plan_t plan, const void* alpha, const int32_t* te_index, int32_t nte, float pf,
                             void* out);

/*
 * t2sh_wavelet_denoise -- the wavelet soft-threshold that follows the solve (Sec. II.C
 * after Eq. 5; the single 3D wavelet soft-thresholding of the re-joined volume in Process
 * TE, Sec. III.C), in place on alpha: device [S][M][K][ny][nz] complex64, 16-byte
 * aligned, where the plan's S slices are the whole volume along the readout x.  For every
 * basis-coefficient image (m, k), the orthonormal 3D Haar pyramid over (x, y, z) with
 * `levels` levels (each transforms the previous approximation), every detail coefficient
 * c replaced by c max(1 - tau / |c|, 0), the coarsest approximation kept, then the
 * inverse pyramid.  The paper names neither the wavelet nor the threshold: the Haar
 * wavelet and the caller's tau are this library's reading.  Requires 1 <= levels <= 16,
 * tau finite >= 0, and S, ny, nz multiples of 2^levels (T2SH_EINVAL otherwise).
 * Asynchronous on the plan's stream; T2SH_HOST_IO plans return T2SH_EUNSUPPORTED.
 */
t2sh_status t2sh_wavelet_denoise(t2sh_plan_t plan, void* alpha, float tau, int32_t levels);

/*
 * Pre-processing (Sec. III.A): from the acquisition as a sparse array of fully sampled
 * readout lines to the projected k-space and masks the solve takes.  Line j (of nlines)
 * holds the channels [nchan][nx] of phase encode (ky[j], kz[j]) at echo t[j]; every axis
 * has its DC sample at index n/2.  The index arrays are host memory (read during the
 * call); line data and results are device memory.  Both calls are plan-free; their
 * scratch is allocated and freed in stream order on `stream`.
 */
typedef struct {
  int32_t nlines, nchan, nx, ny, nz, nechoes;
  const int32_t* t;   /* host [nlines], 0 <= t < nechoes  */
  const int32_t* ky;  /* host [nlines], 0 <= ky < ny      */
  const int32_t* kz;  /* host [nlines], 0 <= kz < nz      */
} t2sh_sparse;

/*
 * t2sh_coil_compression -- Re-sort and Average plus Coil Compression: the central
 * window^3 k-space block of every channel, each (ky, kz) averaged over the echoes that
 * sampled it, as calibration rows X [points][nchan]; W [nchan][ncomp] = eigenvectors of
 * X^H X (right singular vectors of X) by decreasing eigenvalue, each column turned so that
 * its entry of largest magnitude (first such) is real positive (SVD compression, Zhang et
 * al. 2013).  lines: device [nlines][nchan][nx] complex64; w_out: device [nchan][ncomp]
 * complex64.  nchan <= 32, 1 <= ncomp <= nchan, 1 <= window <= min(nx, ny, nz).
 * Synchronises the stream (to report a non-converged eigensolve as T2SH_ECUDA).
 */
t2sh_status t2sh_coil_compression(const t2sh_sparse* sp, const void* lines, int32_t window, int32_t ncomp,
                                  void* w_out, void* stream);

/*
 * t2sh_preprocess -- Coil compression applied (y_v = y W), the readout slices decoupled
 * by the centred unitary 1D inverse DFT along x (Sec. III.B), Re-Sort and Project Data and
 * Compute Mask: ytil[x][c][k][ky][kz] = sum over lines j at (ky, kz) of phi[t_j][k]
 * yhat_j[c][x] (lines repeating (t, ky, kz) add), mask[t][ky][kz] = 1 where sampled.
 * ytil_out: device [nx][ncomp][nbasis][ny][nz] complex64 = the projected k-space of nx
 * slices as t2sh_solve takes it (kform T2SH_KSPACE_PROJ); mask_out: device [nechoes][ny][nz].
 * phi: device [nechoes][nbasis] float.  nx even, a product of 2, 3, 5 and 13.
 * Asynchronous on `stream`.
 */
t2sh_status t2sh_preprocess(const t2sh_sparse* sp, const void* lines, const void* w, int32_t ncomp, const float* phi,
                            int32_t nbasis, void* ytil_out, uint8_t* mask_out, void* stream);

/*
 * Resumable solve, for schedulers that interleave several scans (t2sh_solve is
 * t2sh_solve_begin + t2sh_solve_iterate(dims.iters) + t2sh_solve_end):
 *   t2sh_solve_begin    forms A^H y from the k-space (as t2sh_solve) and resets the FISTA
 *                       state: x = z = 0, t = 1, iteration counter 0; the convergence
 *                       monitor is recorded.
 *   t2sh_solve_iterate  runs the next min(n, dims.iters - done) iterations; *done (nullable)
 *                       receives the number of iterations completed so far.  The state
 *                       (x, z, t_k, counter) stays on the device between calls.
 *   t2sh_solve_end      copies x into alpha_out (host pointer with T2SH_HOST_IO, then the
 *                       call synchronises) and, if residual_out is non-NULL, the monitor of
 *                       the completed iterations (synchronises).
 * Errors: EINVAL if begin was not called.
 */
t2sh_status t2sh_solve_begin(t2sh_plan_t plan, const void* kspace, int32_t kform);
t2sh_status t2sh_solve_iterate(t2sh_plan_t plan, int32_t n, int32_t* done);
t2sh_status t2sh_solve_end(t2sh_plan_t plan, void* alpha_out, double* residual_out);

/*
 * t2sh_solve_batch -- solve n plans at once (scans of different sizes and coil counts:
 * the batched multi-scan form, the paper's many slices per machine of Sec. IV.E).  Each
 * plan's normal operator runs on a stream forked from `stream`; all iterations of all
 * plans are captured into one CUDA graph, which is launched once, so the scans' kernels
 * overlap on the GPU.  The LLR step of each iteration is one launch over a work list of
 * (scan, slice, map set, band) units of every plan still iterating, when the plans share
 * the LLR variant (all K <= 4 or all K > 4, the same T2SH_EIG_FP64) and none uses
 * T2SH_FUSED_ROWS; otherwise each plan launches its own on its stream.  kspace[i] /
 * kform[i] / alpha_out[i] as for t2sh_solve (device pointers; plans with T2SH_HOST_IO are
 * rejected).  A plan may appear once.  Synchronous: returns when every alpha_out is
 * written.  Results equal the plans' single solves bit for bit.
 */
t2sh_status t2sh_solve_batch(t2sh_plan_t* plans, int32_t n, const void* const* kspace, const int32_t* kform,
                             void* const* alpha_out, void* stream);

/*
 * t2sh_batch_schedule -- process-wide choice for t2sh_solve_batch: 0 (default) the LLR
 * work list described there, 1 one LLR launch per plan on its own stream (for
 * comparison).  Affects solves that start after the call.  The paper has no counterpart.
 */
t2sh_status t2sh_batch_schedule(int32_t per_scan_llr);

/*
 * t2sh_autotune -- choose, for the plan's problem shape, the column-pass variant
 * (0: tiles of 8 columns moved by TMA, 4: tiles of 4 by TMA, 1: tiles of 8 by cp.async,
 * 2: tiles of 4 by cp.async; a T2SH_MIXED_BF16 plan keeps its tensor-core column pass,
 * variant 3) and
 * separate versus fused row kernels, by timing probe_iters
 * iterations (default 3 when <= 0) of each candidate on the plan's buffers; the choice
 * is remembered per shape (and appended to the file named by the environment variable
 * T2SH_TUNE_CACHE, read back by later processes).  With probe_iters >= 0 a shape that is
 * already known is not timed again; probe_iters < 0 forces a new measurement.  Clobbers
 * the plan's FISTA state: call it before t2sh_solve_begin.  Synchronises the stream.
 * col_variant_out / fused_out (nullable) receive the choice.
 */
t2sh_status t2sh_autotune(t2sh_plan_t plan, int32_t probe_iters, int32_t* col_variant_out, int32_t* fused_out);

/*
 * t2sh_configure -- pin the plan's kernel choices instead of tuning them: col_variant as
 * for t2sh_autotune (0, 1, 2, 4, or 3 for the tensor-core mixed-precision column pass; shapes
 * a variant does not cover fall back to the FP32 kernels), fused_rows != 0 for the fused
 * band kernel where it applies.  Not during a solve.
 */
t2sh_status t2sh_configure(t2sh_plan_t plan, int32_t col_variant, int32_t fused_rows);

/*
 * t2sh_sync -- synchronise the plan's stream and report failures of its asynchronous
 * work: T2SH_ETIMEOUT if a bounded device wait (a TMA tile copy that did not complete
 * within 2 s) made a kernel give up since the last call (the flag is then cleared),
 * T2SH_ECUDA for a CUDA error.
 */
t2sh_status t2sh_sync(t2sh_plan_t plan);

/*
 * t2sh_wait_selftest -- exercises the bounded-wait failure path without a fault: a kernel
 * on the plan's stream waits, through the same bounded wait the tile kernels use, on a
 * barrier that nothing completes, gives up after limit_ns (1 .. 1e9 ns) and records the
 * timeout; the next t2sh_sync returns T2SH_ETIMEOUT and clears it, and the plan stays
 * usable.  The paper has no counterpart.
 */
t2sh_status t2sh_wait_selftest(t2sh_plan_t plan, uint64_t limit_ns);

/* The step mu the plan uses (host float). */
t2sh_status t2sh_get_step(t2sh_plan_t plan, float* step);

/*
 * t2sh_shifts -- host only: the LLR shift pair of every iteration, out[2*it] = sy,
 * out[2*it+1] = sz, from output it+1 of SplitMix64(seed) (Steele, Lea, Flood 2014):
 * sy = (low 32 bits) mod block, sz = (high 32 bits) mod block.  The paper only says
 * the shift is random and smaller than the patch (Sec. IV.C); this is the library's
 * generator.  out must hold 2*iters int32.
 */
t2sh_status t2sh_shifts(uint64_t seed, int32_t iters, int32_t block, int32_t* out);

/* Host only: device bytes a plan with these dims allocates (for admission control). */
t2sh_status t2sh_workspace_bytes(const t2sh_dims* dims, size_t* bytes);

/*
 * Kernel timing.  While enabled, the plan records a CUDA event pair on its stream
 * around every kernel it launches and counts the launches, per kernel class:
 *   0 row pass forward  (S.z then DFT along z)           1 row pass adjoint (IDFT_z, S^H, coil sum)
 *   2 column pass       (DFT_y, Psi, IDFT_y or variants)  3 LLR prox / FISTA update
 *   4 (reserved: plan-time kernels run inside t2sh_plan, before timing can be enabled)
 *   5 projection of per-echo k-space
 *   6 fused band kernel of t2sh_solve (row adjoint + gradient + LLR + momentum + row forward)
 *   7 conjugate-gradient vector kernels of t2sh_solve_admm
 *   8 TE-image post-processing (t2sh_postprocess)
 * t2sh_timing_enable(plan, 1) clears the counters and starts recording; (plan, 0) stops.
 * t2sh_timing_read synchronises the stream and returns the launch count and the summed
 * event-to-event milliseconds of one class since the last enable.  Recording adds two
 * event records per launch; leave it off when not measuring.
 */
t2sh_status t2sh_timing_enable(t2sh_plan_t plan, int32_t enable);
t2sh_status t2sh_timing_read(t2sh_plan_t plan, int32_t kernel_class, int64_t* launches, double* ms);

/*
 * t2sh_normal_op_noalloc -- y = A^H A x like t2sh_normal_op, for callers that cannot
 * allocate device memory (code running where cudaMalloc is not permitted, or an
 * application that owns all device memory and forbids libraries to allocate).  It takes
 * no plan and allocates nothing: the twiddle tables, Psi, the sign-folded maps and the
 * per-coil intermediate live in one static device array of t2sh_noalloc_scratch_bytes()
 * bytes (64 MiB) that every GPU loading the library holds until the process exits.
 * The paper has no counterpart of this entry point.
 *   dims  as for t2sh_plan (nslices, ny, nz, ncoils, nmaps, nbasis, nechoes used;
 *         T2SH_HOST_IO not allowed)
 *   phi [T][K] float32, mask [T][ny][nz] uint8, maps [S][C][M][ny][nz] complex,
 *   x, y [S][M][K][ny][nz] complex (x == y allowed): all device pointers
 *   stream  cudaStream_t to enqueue on (NULL: default stream)
 * Sizes whose scratch (twiddles + Psi + maps + S*C*K*ny*nz complex, each rounded up to
 * 256 bytes) exceeds the array are rejected with T2SH_EINVAL and a message.  The first
 * call on a device resolves the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  Every call reuses
 * the same array and overwrites what the previous call left there, so calls that
 * overlap on the GPU (different streams, or threads without ordering) race: serialise
 * them.  Asynchronous on the stream: the status says only that the work was queued.
 * Like the planned operator, the kernels bound every wait on a tile copy or tensor-core
 * operation (2 s); a wait that runs out sets a flag in the array, which stays set across
 * later calls until t2sh_noalloc_sync reads and clears it.  Call t2sh_noalloc_sync before
 * trusting y.
 */
t2sh_status t2sh_normal_op_noalloc(const t2sh_dims* dims, const float* phi, const uint8_t* mask,
                                   const void* maps, const void* x, void* y, void* stream);

/* Size in bytes of the static scratch array behind t2sh_normal_op_noalloc. */
size_t t2sh_noalloc_scratch_bytes(void);

/*
 * t2sh_noalloc_sync -- synchronise `stream` (cudaStream_t, NULL: default stream) and
 * report whether a bounded device wait of t2sh_normal_op_noalloc ran out on the current
 * device since the last t2sh_noalloc_sync: T2SH_ETIMEOUT if it did (the flag is then
 * cleared, and the y of the call that timed out is not valid), T2SH_ECUDA for a CUDA
 * error, else T2SH_OK.  Allocates nothing.  The paper has no counterpart.
 */
t2sh_status t2sh_noalloc_sync(void* stream);

/*
 * t2sh_noalloc_wait_selftest -- exercises that failure path without a fault: one kernel
 * on `stream` waits, through the bounded wait the tile kernels use, on a barrier that
 * nothing completes, gives up after limit_ns (1 .. 1e9 ns) and sets the flag of the
 * static array; the next t2sh_noalloc_sync returns T2SH_ETIMEOUT.  The paper has no
 * counterpart.
 */
t2sh_status t2sh_noalloc_wait_selftest(uint64_t limit_ns, void* stream);

/* Message of the last failing call on this thread ("" if none).  Never NULL. */
const char* t2sh_last_error(void);

/* ABI version: 100 * major + minor. */
int32_t t2sh_version(void);

#ifdef __cplusplus
}
#endif
#endif /* T2SH_H */
