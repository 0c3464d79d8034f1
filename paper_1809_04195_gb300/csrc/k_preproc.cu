// Pre-processing in front of the per-slice solve (Sec. III.A), from a sparse array of
// fully sampled readout lines: line j holds the channels [Ctot][Nx] of phase encode
// (ky_j, kz_j) at echo t_j.  The host sorts the lines by (ky, kz) into segments (one per
// sampled phase encode); every kernel below works on that table.
//
//   coil compression: the central win^3 window averaged over the echoes of each (ky, kz)
//     (k_calib), its channel Gram matrix G = X^H X (k_gram), eigenvectors of G by a
//     float64 cyclic Jacobi in one CTA, decreasing eigenvalue, canonical phase (k_eig):
//     W [Ctot][C];
//   decoupling: y_v = y W per line, then the centred unitary inverse DFT along x
//     (k_compress_readout): yhat [n][C][Nx];
//   re-sort and project: ytil[x][c][k][ky][kz] = sum_{j in segment} Phi[t_j][k] yhat[j][c][x]
//     (k_project_lines) and the masks mask[t_j][ky_j][kz_j] = 1 (k_mark_mask).
#include "t2sh_device.cuh"

namespace t2sh {

namespace {

constexpr int kPpThreads = 256;

// calibration rows X[p][c], p = (segment in the window, kx in the window)
__global__ void __launch_bounds__(kPpThreads) k_calib(const float2* __restrict__ lines, int ctot, int nx,
                                                    const int* __restrict__ order, const int* __restrict__ seg_off,
                                                    const int* __restrict__ wseg, int nwseg, int win,
                                                    float2* __restrict__ X) {
  const int x0 = nx / 2 - win / 2;
  const long long total = (long long)nwseg * win * ctot;
  for (long long e = blockIdx.x * (long long)kPpThreads + threadIdx.x; e < total; e += (long long)gridDim.x * kPpThreads) {
    const int c = (int)(e % ctot);
    const long long p = e / ctot;
    const int xw = (int)(p % win), si = (int)(p / win);
    const int sg = wseg[si];
    const int j0 = seg_off[sg], j1 = seg_off[sg + 1];
    float2 acc = make_float2(0.f, 0.f);
    for (int j = j0; j < j1; ++j) {
      const float2 v = lines[((long long)order[j] * ctot + c) * nx + x0 + xw];
      acc.x += v.x;
      acc.y += v.y;
    }
    const float inv = 1.f / (float)(j1 - j0);
    X[p * ctot + c] = make_float2(acc.x * inv, acc.y * inv);
  }
}

// G[c1][c2] += sum_p conj(X[p][c1]) X[p][c2] over this CTA's chunk of rows (float64 atomics)
__global__ void __launch_bounds__(kPpThreads) k_gram(const float2* __restrict__ X, long long npts, int ctot,
                                                   int chunk, double* G) {
  const long long p0 = (long long)blockIdx.x * chunk;
  const long long p1 = p0 + chunk < npts ? p0 + chunk : npts;
  for (int pr = threadIdx.x; pr < ctot * ctot; pr += kPpThreads) {
    const int c1 = pr / ctot, c2 = pr - c1 * ctot;
    float re = 0.f, im = 0.f;
    for (long long p = p0; p < p1; ++p) {
      const float2 a = X[p * ctot + c1], b = X[p * ctot + c2];
      re += a.x * b.x + a.y * b.y;
      im += a.x * b.y - a.y * b.x;
    }
    atomicAdd(&G[2 * pr], (double)re);
    atomicAdd(&G[2 * pr + 1], (double)im);
  }
}

// Eigenvectors of the Hermitian G (interleaved re/im, ctot <= kMaxChan) by cyclic Jacobi
// in float64 on one thread, sorted by decreasing eigenvalue, each column rotated so that
// its entry of largest magnitude (first such index) is real positive; W [ctot][ncomp].
__global__ void k_eig(const double* G, int ctot, int ncomp, float2* W, int* err) {
  __shared__ double ar[kMaxChan][kMaxChan], ai[kMaxChan][kMaxChan], vr[kMaxChan][kMaxChan], vi[kMaxChan][kMaxChan];
  __shared__ int ord[kMaxChan];
  if (threadIdx.x != 0) return;
  const int n = ctot;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      ar[i][j] = G[2 * (i * n + j)];
      ai[i][j] = G[2 * (i * n + j) + 1];
      vr[i][j] = i == j ? 1.0 : 0.0;
      vi[i][j] = 0.0;
    }
  // symmetrise (the float partial sums are Hermitian only to rounding)
  for (int i = 0; i < n; ++i) {
    ai[i][i] = 0.0;
    for (int j = i + 1; j < n; ++j) {
      const double r = 0.5 * (ar[i][j] + ar[j][i]), m = 0.5 * (ai[i][j] - ai[j][i]);
      ar[i][j] = r; ar[j][i] = r; ai[i][j] = m; ai[j][i] = -m;
    }
  }
  bool converged = false;
  for (int sweep = 0; sweep < 60 && !converged; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int p = 0; p < n; ++p) {
      diag += ar[p][p] * ar[p][p];
      for (int q = p + 1; q < n; ++q) off += ar[p][q] * ar[p][q] + ai[p][q] * ai[p][q];
    }
    if (!(off > 1e-30 * diag)) {
      converged = true;
      break;
    }
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double xr = ar[p][q], xi = ai[p][q];
        const double r2 = xr * xr + xi * xi;
        if (!(r2 > 0.0)) continue;
        const double r = sqrt(r2), dr = xr / r, di = -xi / r;  // column q *= d = conj(a_pq)/|a_pq|
        for (int k = 0; k < n; ++k) {
          if (k == q) continue;
          const double yr = ar[k][q] * dr - ai[k][q] * di, yi = ar[k][q] * di + ai[k][q] * dr;
          ar[k][q] = yr; ai[k][q] = yi; ar[q][k] = yr; ai[q][k] = -yi;
        }
        for (int k = 0; k < n; ++k) {
          const double yr = vr[k][q] * dr - vi[k][q] * di, yi = vr[k][q] * di + vi[k][q] * dr;
          vr[k][q] = yr; vi[k][q] = yi;
        }
        const double theta = (ar[q][q] - ar[p][p]) / (2.0 * r);
        double t = 1.0 / (fabs(theta) + sqrt(theta * theta + 1.0));
        if (theta < 0.0) t = -t;
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        ar[p][p] -= t * r;
        ar[q][q] += t * r;
        ar[p][q] = 0.0; ar[q][p] = 0.0; ai[p][q] = 0.0; ai[q][p] = 0.0;
        for (int k = 0; k < n; ++k) {
          if (k == p || k == q) continue;
          const double pr_ = ar[k][p], pi_ = ai[k][p], qr_ = ar[k][q], qi_ = ai[k][q];
          const double npr = c * pr_ - s * qr_, npi = c * pi_ - s * qi_;
          const double nqr = s * pr_ + c * qr_, nqi = s * pi_ + c * qi_;
          ar[k][p] = npr; ai[k][p] = npi; ar[p][k] = npr; ai[p][k] = -npi;
          ar[k][q] = nqr; ai[k][q] = nqi; ar[q][k] = nqr; ai[q][k] = -nqi;
        }
        for (int k = 0; k < n; ++k) {
          const double pr_ = vr[k][p], pi_ = vi[k][p], qr_ = vr[k][q], qi_ = vi[k][q];
          vr[k][p] = c * pr_ - s * qr_; vi[k][p] = c * pi_ - s * qi_;
          vr[k][q] = s * pr_ + c * qr_; vi[k][q] = s * pi_ + c * qi_;
        }
      }
  }
  if (!converged && err) atomicExch(err, 1);
  // order by decreasing eigenvalue (stable selection)
  for (int i = 0; i < n; ++i) ord[i] = i;
  for (int i = 0; i < n; ++i) {
    int best = i;
    for (int j = i + 1; j < n; ++j)
      if (ar[ord[j]][ord[j]] > ar[ord[best]][ord[best]]) best = j;
    const int tmp = ord[i]; ord[i] = ord[best]; ord[best] = tmp;
  }
  for (int c = 0; c < ncomp; ++c) {
    const int col = ord[c];
    int im = 0;
    double mm = -1.0;
    for (int k = 0; k < n; ++k) {
      const double m2 = vr[k][col] * vr[k][col] + vi[k][col] * vi[k][col];
      if (m2 > mm) { mm = m2; im = k; }
    }
    const double a = sqrt(mm);
    const double pr_ = a > 0.0 ? vr[im][col] / a : 1.0, pi_ = a > 0.0 ? -vi[im][col] / a : 0.0;  // conj phase
    for (int k = 0; k < n; ++k)
      W[k * ncomp + c] = make_float2((float)(vr[k][col] * pr_ - vi[k][col] * pi_),
                                     (float)(vr[k][col] * pi_ + vi[k][col] * pr_));
  }
}

// y_v = y W for line blockIdx.x, then the centred unitary inverse DFT along x:
// x[n] = s (-1)^n / sqrt(Nx) * IDFT((-1)^k X[k])[n], s = (-1)^(Nx/2).
template <bool R13>
__global__ void __launch_bounds__(kPpThreads) k_compress_readout(const float2* __restrict__ lines,
                                                               const float2* __restrict__ W, int ctot, int ncomp,
                                                               int nx, FftPlan px, const float2* __restrict__ tw_g,
                                                               int cb, float2* __restrict__ yh) {
  extern __shared__ float2 smem[];
  const int ld = nx + 1;
  float2* tw = smem;
  float2* ws = tw + ((nx + 1) & ~1);         // [ctot][ncomp]
  float2* buf = ws + ctot * ncomp;           // [cb][ld]
  const long long j = blockIdx.x;
  for (int i = threadIdx.x; i < nx; i += kPpThreads) tw[i] = tw_g[i];
  for (int i = threadIdx.x; i < ctot * ncomp; i += kPpThreads) ws[i] = W[i];
  const float scale = ((nx / 2) & 1 ? -1.f : 1.f) * rsqrtf((float)nx);
  for (int c0 = 0; c0 < ncomp; c0 += cb) {
    const int nc = min(cb, ncomp - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < nc * nx; e += kPpThreads) {
      const int cl = e / nx, x = e - cl * nx;
      float2 v = make_float2(0.f, 0.f);
      for (int c = 0; c < ctot; ++c) cfma(v, lines[(j * ctot + c) * nx + x], ws[c * ncomp + c0 + cl]);
      buf[cl * ld + x] = (x & 1) ? make_float2(-v.x, -v.y) : v;
    }
    __syncthreads();
    fft_lines<true, R13>(buf, ld, nc, px, tw);
    for (int e = threadIdx.x; e < nc * nx; e += kPpThreads) {
      const int cl = e / nx, x = e - cl * nx;
      const float sg = (x & 1) ? -scale : scale;
      const float2 v = buf[cl * ld + x];
      yh[(j * ncomp + c0 + cl) * nx + x] = make_float2(sg * v.x, sg * v.y);
    }
  }
}

// ytil[x][c][k][ky][kz] = sum_{j in segment} Phi[t_j][k] yhat[j][c][x]
__global__ void __launch_bounds__(kPpThreads) k_project_lines(const float2* __restrict__ yh, int ncomp, int nx,
                                                            const int* __restrict__ order, const int* __restrict__ tj,
                                                            const int* __restrict__ seg_off, const int* __restrict__ seg_y,
                                                            const int* __restrict__ seg_z, int nseg,
                                                            const float* __restrict__ phi, int K, int ny, int nz,
                                                            float2* __restrict__ ytil) {
  const long long total = (long long)nseg * ncomp * nx;
  const long long N = (long long)ny * nz;
  for (long long e = blockIdx.x * (long long)kPpThreads + threadIdx.x; e < total; e += (long long)gridDim.x * kPpThreads) {
    const int x = (int)(e % nx);
    const long long r = e / nx;
    const int c = (int)(r % ncomp), sg = (int)(r / ncomp);
    float2 acc[kMaxK];
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) acc[k] = make_float2(0.f, 0.f);
    for (int q = seg_off[sg]; q < seg_off[sg + 1]; ++q) {
      const float2 v = yh[((long long)order[q] * ncomp + c) * nx + x];
      const float* ph = phi + (long long)tj[q] * K;
#pragma unroll
      for (int k = 0; k < kMaxK; ++k)
        if (k < K) {
          acc[k].x = fmaf(ph[k], v.x, acc[k].x);
          acc[k].y = fmaf(ph[k], v.y, acc[k].y);
        }
    }
    const long long pix = (long long)seg_y[sg] * nz + seg_z[sg];
    float2* o = ytil + ((long long)x * ncomp + c) * K * N + pix;
#pragma unroll
    for (int k = 0; k < kMaxK; ++k)
      if (k < K) o[k * N] = acc[k];
  }
}

__global__ void k_mark_mask(const int* __restrict__ t, const int* __restrict__ ky, const int* __restrict__ kz, int n,
                            int ny, int nz, uint8_t* mask) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) mask[((long long)t[j] * ny + ky[j]) * nz + kz[j]] = 1;
}

int grid_for(long long total) {
  const long long b = (total + kPpThreads - 1) / kPpThreads;
  return (int)(b < 65535LL * 16 ? (b > 0 ? b : 1) : 65535LL * 16);
}

}  // namespace

cudaError_t launch_calib(const float2* lines, int ctot, int nx, const int* order, const int* seg_off, const int* wseg,
                         int nwseg, int win, float2* X, cudaStream_t st) {
  const long long total = (long long)nwseg * win * ctot;
  if (total == 0) return cudaSuccess;
  k_calib<<<grid_for(total), kPpThreads, 0, st>>>(lines, ctot, nx, order, seg_off, wseg, nwseg, win, X);
  return cudaGetLastError();
}

cudaError_t launch_gram_eig(const float2* X, long long npts, int ctot, int ncomp, double* G, float2* W, int* err,
                            cudaStream_t st) {
  if (ctot > kMaxChan) return cudaErrorInvalidValue;
  const int chunk = 256;
  const long long nb = (npts + chunk - 1) / chunk;
  cudaError_t e = cudaMemsetAsync(G, 0, sizeof(double) * 2 * ctot * ctot, st);
  if (e != cudaSuccess) return e;
  if (nb > 0) k_gram<<<(unsigned)nb, kPpThreads, 0, st>>>(X, npts, ctot, chunk, G);
  k_eig<<<1, 32, 0, st>>>(G, ctot, ncomp, W, err);
  return cudaGetLastError();
}

cudaError_t launch_compress_readout(const float2* lines, const float2* W, int nlines, int ctot, int ncomp,
                                    const FftPlan& px, const float2* tw_x, float2* yh, cudaStream_t st) {
  const int nx = px.n;
  int cb = (kStage * kPpThreads) / nx;
  if (cb < 1) return cudaErrorInvalidValue;
  if (cb > ncomp) cb = ncomp;
  const size_t sm = sizeof(float2) * (((nx + 1) & ~1) + (size_t)ctot * ncomp + (size_t)cb * (nx + 1));
  if (sm > 200 * 1024) return cudaErrorInvalidValue;
  if (plan_has13(px)) {
    {
      const cudaError_t e = smem_optin((const void*)k_compress_readout<true>, 200 * 1024);
      if (e != cudaSuccess) return e;
    }
    k_compress_readout<true><<<nlines, kPpThreads, sm, st>>>(lines, W, ctot, ncomp, nx, px, tw_x, cb, yh);
  } else {
    {
      const cudaError_t e = smem_optin((const void*)k_compress_readout<false>, 200 * 1024);
      if (e != cudaSuccess) return e;
    }
    k_compress_readout<false><<<nlines, kPpThreads, sm, st>>>(lines, W, ctot, ncomp, nx, px, tw_x, cb, yh);
  }
  return cudaGetLastError();
}

cudaError_t launch_project_lines(const float2* yh, int ncomp, int nx, const int* order, const int* tj,
                                 const int* seg_off, const int* seg_y, const int* seg_z, int nseg, const float* phi,
                                 int K, int ny, int nz, float2* ytil, cudaStream_t st) {
  const long long total = (long long)nseg * ncomp * nx;
  if (total == 0) return cudaSuccess;
  k_project_lines<<<grid_for(total), kPpThreads, 0, st>>>(yh, ncomp, nx, order, tj, seg_off, seg_y, seg_z, nseg, phi,
                                                          K, ny, nz, ytil);
  return cudaGetLastError();
}

cudaError_t launch_mark_mask(const int* t, const int* ky, const int* kz, int n, int ny, int nz, uint8_t* mask,
                             cudaStream_t st) {
  k_mark_mask<<<(n + 255) / 256, 256, 0, st>>>(t, ky, kz, n, ny, nz, mask);
  return cudaGetLastError();
}

}  // namespace t2sh
