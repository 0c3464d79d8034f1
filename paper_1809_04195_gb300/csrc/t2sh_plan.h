// Internal structures shared by the host runtime (t2sh_api.cu) and the kernel
// translation units.  Not part of the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace t2sh {

constexpr int kThreads = 256;                    // threads of the prep and LLR CTAs
constexpr int kFftThreads = 512;                 // threads of the row / column FFT CTAs
constexpr int kStage = 16;                       // complex values a thread stages per FFT pass
constexpr int kMaxLineElems = kStage * kFftThreads;  // complex elements one CTA transforms at once
constexpr int kMaxPass = 8;
constexpr int kMaxK = 8;
constexpr int kMaxM = 2;
constexpr int kMaxBlock = 16;
constexpr int kMaxPostTe = 8;                    // echoes one t2sh_postprocess call synthesises
constexpr int kMaxChan = 32;                     // receive channels of the coil-compression step

// Radix plan of a length-n FFT: pass q has radix radix[q] and ns[q] = prod of the
// radices of passes 0..q-1 (Stockham autosort).
struct FftPlan {
  int n;
  int npass;
  int radix[kMaxPass];
  int ns[kMaxPass];
};

inline bool plan_has13(const FftPlan& p) {
  for (int q = 0; q < p.npass; ++q)
    if (p.radix[q] == 13) return true;
  return false;
}

// Geometry of one batch of slices, passed by value to every kernel.
struct Geom {
  int S, C, M, K, T;   // slices, coils, map sets, basis size, echoes
  int ny, nz;          // slice matrix
  int P;               // K (K + 1) / 2: stored entries of Psi(n)
  float gsign;         // (-1)^(ny/2 + nz/2): global sign of the centred DFT
  float inv_sqrt_n;    // 1 / sqrt(ny nz)
  int colvar;          // normal-operator column pass: 0 TMA tiles of 8 columns, 1 cp.async
                       // tiles of 8, 2 cp.async tiles of 4 (size-specialised kernels),
                       // 3 tensor-core DFT-as-GEMM in split BF16 (mixed precision),
                       // 4 TMA tiles of 4 columns (two CTAs per SM)
  int* err;            // nullable device flag: set to 1 when a bounded wait ran out
};

// Column-pass (ky direction) modes.
enum ColMode : int {
  COL_NORMAL = 0,    // DFT_y, Psi (pre-scaled by 1/N), IDFT_y                 (normal operator)
  COL_ADJ_DATA = 1,  // multiply by gsign (-1)^(ky+kz) / sqrt(N), IDFT_y          (A^H y)
  COL_FWD_PROJ = 2,  // DFT_y, multiply by gsign (-1)^(ky+kz) / sqrt(N), Psi * N  (Phi^T P A x)
  COL_FWD_TE = 3     // DFT_y, multiply by gsign (-1)^(ky+kz) / sqrt(N), P_t Phi  (A x, per echo)
};

// Row-pass (kz direction) modes.
enum RowMode : int {
  ROW_FWD = 0,  // t[c][k] = DFT_z( sum_m S'_{c,m} x_{m,k} )
  ROW_ADJ = 1   // out[m][k] = sum_c conj(S'_{c,m}) IDFT_z( t[c][k] )
};

struct FistaArgs {
  float mu;      // step
  float tau;     // mu * lambda
  float beta;    // (t_k - 1) / t_{k+1}
  int sy, sz;    // LLR shift of this iteration
  int b;         // block edge
  int eig64;     // 1: eigendecomposition in float64, 0: float32
  int skip_adj;  // fused band kernel: z_k = 0, so A^H A z_k = 0 (first iteration)
  int skip_fwd;  // fused band kernel: no next iteration, skip DFT_z(S z_{k+1})
  double* res;   // nullable: accumulates {sum |x_{k+1} - x_k|^2, sum |x_{k+1}|^2}
};

// ------------------------------ launchers -----------------------------------------
// All return the cudaGetLastError() of their launch.
cudaError_t launch_maps_prep(const Geom& g, const float2* maps_in, float2* maps_out, unsigned* lam_s_bits,
                             cudaStream_t st);
cudaError_t launch_psi_build(const Geom& g, const float* phi, const uint8_t* mask, float* psi,
                             unsigned* lam_psi_bits, cudaStream_t st);
cudaError_t launch_project(const Geom& g, const float* phi, const uint8_t* mask, const float2* y_te,
                           float2* y_proj, cudaStream_t st);
cudaError_t launch_row(const Geom& g, RowMode mode, const FftPlan& pz, const float2* tw_z, const float2* maps,
                       const float2* x, float2* t, float2* out, cudaStream_t st);
cudaError_t launch_col(const Geom& g, ColMode mode, const FftPlan& py, const float2* tw_y, const float* psi,
                       const float* phi, const uint8_t* mask, const float2* tin, float2* tout, cudaStream_t st);
// TE images: back-projection at echoes te[0..nte), coil images, homodyne along z with
// band half-width w, root sum of squares -> out [S][nte][ny][nz] float
size_t post_smem_bytes(const Geom& g, int nte);
cudaError_t launch_post(const Geom& g, const FftPlan& pz, const float2* tw_z, const float2* maps, const float* phi,
                        const float2* alpha, const int* te, int nte, int w, float* out, cudaStream_t st);
// pre-processing from sparse readout lines (k_preproc.cu)
cudaError_t launch_calib(const float2* lines, int ctot, int nx, const int* order, const int* seg_off, const int* wseg,
                         int nwseg, int win, float2* X, cudaStream_t st);
cudaError_t launch_gram_eig(const float2* X, long long npts, int ctot, int ncomp, double* G, float2* W, int* err,
                            cudaStream_t st);
cudaError_t launch_compress_readout(const float2* lines, const float2* W, int nlines, int ctot, int ncomp,
                                    const FftPlan& px, const float2* tw_x, float2* yh, cudaStream_t st);
cudaError_t launch_project_lines(const float2* yh, int ncomp, int nx, const int* order, const int* tj,
                                 const int* seg_off, const int* seg_y, const int* seg_z, int nseg, const float* phi,
                                 int K, int ny, int nz, float2* ytil, cudaStream_t st);
cudaError_t launch_mark_mask(const int* t, const int* ky, const int* kz, int n, int ny, int nz, uint8_t* mask,
                             cudaStream_t st);
// ADMM v-update: w = alpha + u, v = LLR prox of w (threshold a.tau, shift a.sy/a.sz), u <- w - v
cudaError_t launch_llr_admm(const Geom& g, const FistaArgs& a, const float2* alpha, float2* v, float2* u,
                            cudaStream_t st);
// conjugate-gradient vector kernels of the ADMM alpha-update (per-slice float64 accumulators)
cudaError_t launch_cg_init(const Geom& g, const float2* x, const float2* w, const float2* aty, const float2* v,
                           const float2* u, float rho, float2* r, float2* p, double* rr, cudaStream_t st);
cudaError_t launch_cg_dot(const Geom& g, const float2* p, const float2* w, float rho, double* pq, cudaStream_t st);
// out[s] += sum of P_t(n) |y|^2 over T-form k-space y [S][C][T][ny][nz]
cudaError_t launch_masked_energy(const Geom& g, const uint8_t* mask, const float2* y, double* out, cudaStream_t st);
cudaError_t launch_cg_step(const Geom& g, float2* x, float2* r, const float2* p, const float2* w, float rho,
                           const double* rr, const double* pq, double* rr_new, cudaStream_t st);
cudaError_t launch_cg_dir(const Geom& g, const float2* r, float2* p, const double* rr, const double* rr_new,
                          double* pq, double* rr_next, cudaStream_t st);
cudaError_t launch_llr(const Geom& g, const FistaArgs& a, float2* x, float2* z, const float2* grad,
                       const float2* aty, cudaStream_t st);

// One scan's part of a work-list LLR launch (the FISTA step of several scans in one grid):
// its geometry, this iteration's arguments and buffers, and its first CTA in the launch.
struct LlrJob {
  Geom g;
  FistaArgs a;
  float2* x;
  float2* z;
  const float2* grad;
  const float2* aty;
  int unit0;
};
int llr_units(const Geom& g, int b);  // CTAs of one scan's LLR launch
size_t llr_smem_bytes(const Geom& g, int b);
// jobs: device array in increasing unit0; units = total CTAs; kc8: some scan has K > 4;
// smem: the largest llr_smem_bytes of the jobs
cudaError_t launch_llr_list(const LlrJob* jobs, int njobs, int units, bool kc8, bool eig64, size_t smem,
                            cudaStream_t st);

// size-specialised passes (k_fft_fast.cu); cudaErrorNotSupported when the shape has none
cudaError_t launch_row_fast(const Geom& g, RowMode mode, const float2* tw_z, const float2* maps, const float2* x,
                            float2* t, float2* out, cudaStream_t st);
cudaError_t launch_col_normal_fast(const Geom& g, const float2* tw_y, const float* psi, float2* t, cudaStream_t st);
// cuTensorMapEncodeTiled, resolved once through the runtime (nullptr if unavailable)
using TmaEncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
TmaEncodeFn tma_encode_fn();
cudaError_t launch_wait_selftest(int* err, unsigned long long limit_ns, cudaStream_t st);
cudaError_t launch_col_normal_pr(const Geom& g, const float2* tw_y, const float* psi, float2* t, cudaStream_t st);
cudaError_t launch_col_normal_tc(const Geom& g, const float2* tw_y, const float* psi, float2* t, cudaStream_t st);
cudaError_t launch_col_normal_tma(const Geom& g, const float2* tw_y, const float* psi, float2* t, cudaStream_t st);
// A^H y column pass on TMA tiles (K <= 4, nz % 8 == 0, ny = 16 R1 <= 256; tin may equal tout)
cudaError_t launch_col_adj_tma(const Geom& g, const float2* tw_y, const float2* tin, float2* tout, cudaStream_t st);

// fused row work of one FISTA iteration (k_fused.cu)
bool band_fused_supported(const Geom& g, int block);
cudaError_t launch_band_fused(const Geom& g, const FistaArgs& a, const float2* tw_z, const float2* maps, float2* t,
                              float2* x, float2* z, const float2* aty, cudaStream_t st);

// Per-device launch set-up shared by the launchers (a process may drive several GPUs):
// a kernel's dynamic shared-memory limit is raised once per (kernel, device), and the
// SM count and a kernel's resident CTAs per SM are cached per device.  All act on the
// current device.
cudaError_t smem_optin(const void* kernel, int bytes);
cudaError_t sm_count(int* n);
cudaError_t ctas_per_sm(const void* kernel, int threads, size_t smem, int* per);

// wavelet soft-threshold of the coefficient volume alpha [S][M][K][ny][nz] in place (k_wavelet.cu):
// `levels`-level orthonormal 3D Haar pyramid over (slice, y, z), details soft-thresholded by tau
cudaError_t launch_wavelet_denoise(const Geom& g, float2* alpha, float tau, int levels, cudaStream_t st);

int row_rows_per_cta(const Geom& g);
int col_cols_per_cta(const Geom& g);

}  // namespace t2sh
