// Column pass of the normal operator (DFT_y, Psi, IDFT_y) for line lengths N = P R1 that
// are not 16 R1, with P threads per line (the paper's 260 = 20 x 13).  Cooley-Tukey with
// the input index n = j + P q (j < P, q < R1):
//   forward:  thread j: DFT_R1 over q of x[j + P q] -> Y[j][k1] (exchange [j][k1], stride R1);
//             thread k1 < R1: twiddle w_N^(j k1), DFT_P over j -> X[k1 + R1 k2], natural order;
//   Psi at every (ky, column) across the K basis lines;
//   inverse:  thread k1 < R1: IDFT_P over k2 of X[k1 + R1 k2] -> Z[k1][j] (stride P + 1);
//             thread j: twiddle w_N^(-k1 j), IDFT_R1 over k1 -> x[j + P q], straight to memory.
// Persistent CTAs of W x 4 x P threads over (slice, coil, W-column tile) tiles; the tile and
// its Psi block are staged by cp.async, the next tile's copies issued as soon as the staging
// area is free.  (The TMA column kernels copy a 260-row column as two tensor-map boxes;
// this kernel serves the cp.async column variants at this length.)
// R1 odd (the stage-A exchange stride), K <= 4, nz % W == 0.
#include <algorithm>

// packed two-lane complex additions in the butterflies: measured 2.6 % faster here
#define T2SH_PACKED_ADD 1
#include "t2sh_device.cuh"

namespace t2sh {

namespace {

template <int P, int R1, int W>
struct ColPR {
  static constexpr int N = P * R1;
  static constexpr int SI = P + 1;  // inverse exchange stride (odd for P even)
  static constexpr int LS0 = (N > R1 * SI ? N : R1 * SI) + 1;
  static constexpr int LS = LS0 | 1;  // line stride, odd
  static constexpr int PS = N * W + W;
  static constexpr int THREADS = W * 4 * P;
  static constexpr size_t smem(int np) {
    return sizeof(float2) * (((size_t)N + 1) / 2 * 2 + 4 * W * (size_t)LS + 4 * (size_t)PS) +
           sizeof(float) * (size_t)np * N * W;
  }
  static_assert(R1 % 2 == 1, "stage-A exchange stride must be odd");
};

template <int P, int R1, int W>
__global__ void __launch_bounds__(W * 4 * P, 2) k_col_pr(Geom g, const float2* __restrict__ tw_g,
                                                     const float* __restrict__ psi, float2* t, int ntz, int ntiles) {
  using CP = ColPR<P, R1, W>;
  constexpr int N = CP::N, LS = CP::LS, PS = CP::PS, SI = CP::SI;
  extern __shared__ float2 smem[];
  const int nz = g.nz, NN = N * nz, K = g.K, NP = g.P;
  const int w = threadIdx.x % W, k = (threadIdx.x / W) & 3, j = threadIdx.x / (4 * W);
  float2* tw = smem;
  float2* ex = tw + (N + 1) / 2 * 2;                         // [k][w][LS]
  float2* st = ex + 4 * W * LS;                              // [k][y][W] (+ pad per k)
  float* ps = reinterpret_cast<float*>(st + 4 * PS);         // [p][y][W]
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];

  auto issue_t = [&](int tile) {
    const int sc = tile / ntz, z0 = (tile - sc * ntz) * W;
    const float2* tb = t + (long long)sc * K * NN + z0;
    const int n16 = K * N * (W / 2);
    for (int e = threadIdx.x; e < n16; e += blockDim.x) {
      const int w2 = (e % (W / 2)) * 2;
      const int row = e / (W / 2);
      const int kk = row / N, y = row - kk * N;
      cp_async16(st + kk * PS + y * W + w2, tb + (long long)kk * NN + (long long)y * nz + w2);
    }
  };
  auto issue_psi = [&](int tile) {
    const int sc = tile / ntz, z0 = (tile - sc * ntz) * W;
    const int n16 = NP * N * (W / 4);
    for (int e = threadIdx.x; e < n16; e += blockDim.x) {
      const int w4 = (e % (W / 4)) * 4;
      const int row = e / (W / 4);
      const int pp = row / N, y = row - pp * N;
      cp_async16(ps + (pp * N + y) * W + w4, psi + (long long)pp * NN + (long long)y * nz + z0 + w4);
    }
  };
  int tile = blockIdx.x;
  if (tile < ntiles) {
    issue_t(tile);
    issue_psi(tile);
  }
  cp_async_commit();
  float2* exl = ex + (k * W + w) * LS;
  const bool live = k < K;
  for (; tile < ntiles; tile += gridDim.x) {
    const int nxt = tile + gridDim.x;
    const int sc = tile / ntz, z0 = (tile - sc * ntz) * W;
    cp_async_wait<0>();
    __syncthreads();
    // forward stage A: DFT_R1 of x[j + P q] -> [j][k1]
    if (live) {
      const float2* sp = st + k * PS + w;
      float2 a[R1];
#pragma unroll
      for (int q = 0; q < R1; ++q) a[q] = sp[(j + P * q) * W];
      dft_r<R1, false>(a);
#pragma unroll
      for (int q = 0; q < R1; ++q) exl[j * R1 + q] = a[q];
    }
    __syncthreads();
    if (nxt < ntiles) issue_t(nxt);
    cp_async_commit();
    // forward stage B: twiddle, DFT_P -> X[k1 + R1 k2] in natural order
    if (live && j < R1) {
      float2 b[P];
#pragma unroll
      for (int q = 0; q < P; ++q) b[q] = exl[j + R1 * q];
#pragma unroll
      for (int q = 1; q < P; ++q) b[q] = twiddle_mul<false>(b[q], tw[q * j]);
      dft_r<P, false>(b);
#pragma unroll
      for (int q = 0; q < P; ++q) exl[j + R1 * q] = b[q];
    }
    __syncthreads();
    // space-time kernel
    for (int pg = threadIdx.x; pg < N * (W / 4); pg += blockDim.x) {
      const int ky = pg % N, c0 = (pg / N) * 4;
      float2 v[4][4], u[4][4];
#pragma unroll
      for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          v[l][c] = (l < K) ? ex[(l * W + c0 + c) * LS + ky] : make_float2(0.f, 0.f);
          u[l][c] = make_float2(0.f, 0.f);
        }
      int pp = 0;
#pragma unroll
      for (int a_ = 0; a_ < 4; ++a_)
#pragma unroll
        for (int b_ = a_; b_ < 4; ++b_)
          if (b_ < K) {
            const float4 q4 = *reinterpret_cast<const float4*>(ps + (pp * N + ky) * W + c0);
            const float pv[4] = {q4.x, q4.y, q4.z, q4.w};
            ++pp;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              u[a_][c].x = fmaf(pv[c], v[b_][c].x, u[a_][c].x);
              u[a_][c].y = fmaf(pv[c], v[b_][c].y, u[a_][c].y);
              if (b_ != a_) {
                u[b_][c].x = fmaf(pv[c], v[a_][c].x, u[b_][c].x);
                u[b_][c].y = fmaf(pv[c], v[a_][c].y, u[b_][c].y);
              }
            }
          }
#pragma unroll
      for (int l = 0; l < 4; ++l)
        if (l < K)
#pragma unroll
          for (int c = 0; c < 4; ++c) ex[(l * W + c0 + c) * LS + ky] = u[l][c];
    }
    __syncthreads();
    if (nxt < ntiles) issue_psi(nxt);
    cp_async_commit();
    // inverse stage A': IDFT_P over k2 of X[k1 + R1 k2] -> Z[k1][j] (stride SI)
    float2 b[P];
    if (live && j < R1) {
#pragma unroll
      for (int q = 0; q < P; ++q) b[q] = exl[j + R1 * q];
      dft_r<P, true>(b);
    }
    __syncthreads();
    if (live && j < R1) {
#pragma unroll
      for (int q = 0; q < P; ++q) exl[j * SI + q] = b[q];
    }
    __syncthreads();
    // inverse stage B': twiddle, IDFT_R1 over k1 -> x[j + P q], to global memory
    if (live) {
      float2 a[R1];
#pragma unroll
      for (int q = 0; q < R1; ++q) a[q] = twiddle_mul<true>(exl[q * SI + j], tw[q * j]);
      dft_r<R1, true>(a);
      float2* ob = t + ((long long)sc * K + k) * NN + z0 + w;
#pragma unroll
      for (int q = 0; q < R1; ++q) ob[(long long)(j + P * q) * nz] = a[q];
    }
  }
  cp_async_wait<0>();
}

template <int P, int R1, int W>
cudaError_t col_pr_go(const Geom& g, const float2* tw, const float* psi, float2* t, cudaStream_t st) {
  using CP = ColPR<P, R1, W>;
  int nsm = 0, per = 0;
  const void* kern = (const void*)k_col_pr<P, R1, W>;
  cudaError_t e = smem_optin(kern, (int)CP::smem(10));
  if (e == cudaSuccess) e = sm_count(&nsm);
  if (e == cudaSuccess) e = ctas_per_sm(kern, CP::THREADS, CP::smem(10), &per);
  if (e != cudaSuccess) return e;
  const int ntz = g.nz / W;
  const long long ntiles = (long long)g.S * g.C * ntz;
  if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (ntiles == 0) return cudaSuccess;
  const int grid = (int)std::min<long long>(ntiles, (long long)nsm * per);
  k_col_pr<P, R1, W><<<grid, CP::THREADS, CP::smem(g.P), st>>>(g, tw, psi, t, ntz, (int)ntiles);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_col_normal_pr(const Geom& g, const float2* tw_y, const float* psi, float2* t, cudaStream_t st) {
  if (g.K > 4 || g.nz % 4 != 0) return cudaErrorNotSupported;
  switch (g.ny) {
    case 260: return col_pr_go<20, 13, 4>(g, tw_y, psi, t, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace t2sh
