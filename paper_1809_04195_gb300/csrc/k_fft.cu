// Row (kz, contiguous) and column (ky, strided) passes of the normal operator
// S^H F^H Psi F S (Sec. IV.B, Algorithm 1) and of the forward / adjoint operators.
//
// Row pass: one CTA per (slice, group of rows).  It loops over the coils inside, as
// Algorithm 1 puts the coil loop outermost, so the image rows it needs (x in the
// forward direction, the accumulated output in the adjoint direction) stay in
// registers across all coils; only the per-coil intermediate t[c][k] goes to memory.
// Column pass: one CTA per (slice, coil, group of columns).  It performs the forward
// column DFT, applies the K x K space-time kernel point by point and the inverse
// column DFT without writing the k-space intermediate back in between (the
// "transpose shortcut" of Sec. IV.B: Psi does not care about the data order).
#include <algorithm>

#include "t2sh_device.cuh"

namespace t2sh {

// pixels one thread owns in the row pass (acc / x registers: PMAX * MC * KC complex)
template <int KC, int MC>
struct RowCaps {
  static constexpr int PMAX = (KC * MC <= 4) ? 4 : (KC * MC <= 8 ? 2 : 1);
};

template <int MODE, int KC, int MC, bool R13>
__global__ void __launch_bounds__(kFftThreads) k_row(Geom g, FftPlan pz, const float2* __restrict__ tw_g,
                                                   const float2* __restrict__ maps, const float2* __restrict__ x,
                                                   float2* __restrict__ t, float2* __restrict__ out, int RB) {
  constexpr int PMAX = RowCaps<KC, MC>::PMAX;
  extern __shared__ float2 smem[];
  const int nz = g.nz, N = g.ny * g.nz, K = g.K, M = g.M;
  const int ld = nz + 1;
  const int s = blockIdx.y;
  const int y0 = blockIdx.x * RB;
  const int rb = min(RB, g.ny - y0);
  const int npix = rb * nz;
  // shared memory: twiddles | FFT lines (x2 for the adjoint's double buffer) | maps rows x2
  float2* tw = smem;
  float2* lines0 = smem + ((nz + 1) & ~1);
  const int line_elems = (K * RB * ld + 1) & ~1;  // even: keeps the maps area 16-byte aligned
  float2* lines1 = (MODE == ROW_ADJ) ? lines0 + line_elems : lines0;
  float2* maps0 = lines1 + line_elems;
  const int map_elems = M * RB * nz;
  float2* maps1 = maps0 + map_elems;
  for (int i = threadIdx.x; i < nz; i += blockDim.x) tw[i] = tw_g[i];

  // asynchronous copy of coil c's inputs: maps rows (and, adjoint, the t rows)
  auto issue = [&](int c, float2* lbuf, float2* mbuf) {
    const float2* mp = maps + ((long long)(s * g.C + c) * M) * N + (long long)y0 * nz;
    const int nm2 = (M * npix) >> 1;
    for (int e2 = threadIdx.x; e2 < nm2; e2 += kFftThreads) {
      const int e = 2 * e2;
      const int m = e / npix, rem = e - m * npix;
      cp_async16(mbuf + e, mp + (long long)m * N + rem);
    }
    if (MODE == ROW_ADJ) {
      const float2* tc = t + ((long long)(s * g.C + c) * K) * N + (long long)y0 * nz;
      const int nel = K * npix;
      for (int e = threadIdx.x; e < nel; e += kFftThreads) {
        const int k = e / npix, rem = e - k * npix;
        const int r = rem / nz, zz = rem - r * nz;
        cp_async8(lbuf + (k * rb + r) * ld + zz, tc + (long long)k * N + rem);
      }
    }
  };
  issue(0, lines0, maps0);
  cp_async_commit();

  int pr[PMAX], pzz[PMAX];
#pragma unroll
  for (int u = 0; u < PMAX; ++u) {
    const int p = threadIdx.x + u * kFftThreads;
    pr[u] = (p < npix) ? p / nz : -1;
    pzz[u] = (p < npix) ? p - (p / nz) * nz : 0;
  }
  float2 reg[PMAX][MC][KC];  // ROW_FWD: x values; ROW_ADJ: accumulators
#pragma unroll
  for (int u = 0; u < PMAX; ++u)
#pragma unroll
    for (int m = 0; m < MC; ++m)
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        reg[u][m][k] = make_float2(0.f, 0.f);
        if (MODE == ROW_FWD && pr[u] >= 0 && m < M && k < K)
          reg[u][m][k] = x[((long long)(s * M + m) * K + k) * N + (long long)(y0 + pr[u]) * nz + pzz[u]];
      }

  const int nelem2 = (K * npix) >> 1;  // float4 pairs of the K rb x nz tile (nz even)
  for (int c = 0; c < g.C; ++c) {
    const int cur = c & 1;
    float2* lbuf = cur ? lines1 : lines0;
    float2* mbuf = cur ? maps1 : maps0;
    if (c + 1 < g.C) issue(c + 1, cur ? lines0 : lines1, cur ? maps0 : maps1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    if (MODE == ROW_FWD) {
      float2* tc = t + ((long long)(s * g.C + c) * K) * N + (long long)y0 * nz;
#pragma unroll
      for (int u = 0; u < PMAX; ++u) {
        if (pr[u] >= 0) {
          float2 sv[MC];
#pragma unroll
          for (int m = 0; m < MC; ++m)
            sv[m] = (m < M) ? mbuf[m * npix + pr[u] * nz + pzz[u]] : make_float2(0.f, 0.f);
#pragma unroll
          for (int k = 0; k < KC; ++k) {
            if (k < K) {
              float2 v = make_float2(0.f, 0.f);
#pragma unroll
              for (int m = 0; m < MC; ++m) cfma(v, sv[m], reg[u][m][k]);
              lbuf[(k * rb + pr[u]) * ld + pzz[u]] = v;
            }
          }
        }
      }
      __syncthreads();
      fft_lines<false, R13>(lbuf, ld, K * rb, pz, tw);
      for (int e = threadIdx.x; e < nelem2; e += kFftThreads) {
        const int e0 = 2 * e;
        const int k = e0 / npix;
        const int rem = e0 - k * npix;
        const int r = rem / nz, zz = rem - r * nz;
        const float2 a = lbuf[(k * rb + r) * ld + zz];
        const float2 b = lbuf[(k * rb + r) * ld + zz + 1];
        *reinterpret_cast<float4*>(tc + (long long)k * N + rem) = make_float4(a.x, a.y, b.x, b.y);
      }
      __syncthreads();
    } else {
      fft_lines<true, R13>(lbuf, ld, K * rb, pz, tw);
#pragma unroll
      for (int u = 0; u < PMAX; ++u) {
        if (pr[u] >= 0) {
#pragma unroll
          for (int m = 0; m < MC; ++m) {
            if (m < M) {
              const float2 sv = mbuf[m * npix + pr[u] * nz + pzz[u]];
#pragma unroll
              for (int k = 0; k < KC; ++k)
                if (k < K) cfmac(reg[u][m][k], sv, lbuf[(k * rb + pr[u]) * ld + pzz[u]]);
            }
          }
        }
      }
      __syncthreads();
    }
  }
  if (MODE == ROW_ADJ) {
#pragma unroll
    for (int u = 0; u < PMAX; ++u)
      if (pr[u] >= 0)
#pragma unroll
        for (int m = 0; m < MC; ++m)
#pragma unroll
          for (int k = 0; k < KC; ++k)
            if (m < M && k < K)
              out[((long long)(s * M + m) * K + k) * N + (long long)(y0 + pr[u]) * nz + pzz[u]] = reg[u][m][k];
  }
}

// Normal-operator column pass, persistent and double buffered: each CTA walks the
// (slice, coil, column tile) list; the next tile streams into shared memory with
// cp.async while the current one is transformed (DFT_y, Psi, IDFT_y) and written back.
template <int KC, bool R13>
__global__ void __launch_bounds__(kFftThreads, 1) k_col_normal(Geom g, FftPlan py, const float2* __restrict__ tw_g,
                                                             const float* __restrict__ psi, float2* t, int W,
                                                             int ntz, int ntiles) {
  extern __shared__ float2 smem[];
  const int ny = g.ny, nz = g.nz, N = ny * nz, K = g.K;
  const int ld = ny + 1;
  float2* tw = smem;
  float2* bufs = smem + ((ny + 1) & ~1);
  const int tile_elems = K * W * ld;
  for (int i = threadIdx.x; i < ny; i += blockDim.x) tw[i] = tw_g[i];

  auto issue = [&](int tile, float2* buf) {
    const int sc = tile / ntz, zt = tile - sc * ntz;
    const int z0 = zt * W, wc = min(W, nz - z0);
    const float2* tb = t + (long long)sc * K * N + z0;
    const int nel = K * ny * wc;
    for (int e = threadIdx.x; e < nel; e += kFftThreads) {
      const int w = e % wc;
      const int rest = e / wc;
      const int y = rest % ny, k = rest / ny;
      cp_async8(buf + (k * wc + w) * ld + y, tb + (long long)k * N + (long long)y * nz + w);
    }
  };
  int tile = blockIdx.x;
  if (tile < ntiles) issue(tile, bufs);
  cp_async_commit();
  int cur = 0;
  for (; tile < ntiles; tile += gridDim.x) {
    const int next = tile + gridDim.x;
    float2* buf = bufs + cur * tile_elems;
    if (next < ntiles) issue(next, bufs + (cur ^ 1) * tile_elems);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const int sc = tile / ntz, zt = tile - sc * ntz;
    const int z0 = zt * W, wc = min(W, nz - z0);
    fft_lines<false, R13>(buf, ld, K * wc, py, tw);
    const int npt = ny * wc;
    for (int q = threadIdx.x; q < npt; q += kFftThreads) {
      const int w = q % wc, y = q / wc;
      const long long n = (long long)y * nz + z0 + w;
      float2 v[KC], u[KC];
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        v[k] = (k < K) ? buf[(k * wc + w) * ld + y] : make_float2(0.f, 0.f);
        u[k] = make_float2(0.f, 0.f);
      }
      int p = 0;
#pragma unroll
      for (int k = 0; k < KC; ++k)
#pragma unroll
        for (int l = k; l < KC; ++l)
          if (l < K) {
            const float ps = __ldg(psi + (long long)p * N + n);
            ++p;
            u[k].x = fmaf(ps, v[l].x, u[k].x);
            u[k].y = fmaf(ps, v[l].y, u[k].y);
            if (l != k) {
              u[l].x = fmaf(ps, v[k].x, u[l].x);
              u[l].y = fmaf(ps, v[k].y, u[l].y);
            }
          }
#pragma unroll
      for (int k = 0; k < KC; ++k)
        if (k < K) buf[(k * wc + w) * ld + y] = u[k];
    }
    __syncthreads();
    fft_lines<true, R13>(buf, ld, K * wc, py, tw);
    float2* ob = t + (long long)sc * K * N + z0;
    const int nel = K * ny * wc;
    for (int e = threadIdx.x; e < nel; e += kFftThreads) {
      const int w = e % wc;
      const int rest = e / wc;
      const int y = rest % ny, k = rest / ny;
      ob[(long long)k * N + (long long)y * nz + w] = buf[(k * wc + w) * ld + y];
    }
    __syncthreads();
    cur ^= 1;
  }
  cp_async_wait<0>();
}

// Column pass.  tin/tout are [S][C][K][ny][nz] (may alias); FWD_TE writes yout
// [S][C][T][ny][nz] and FWD_PROJ writes yout [S][C][K][ny][nz].
template <int MODE, int KC, bool R13>
__global__ void __launch_bounds__(kFftThreads) k_col(Geom g, FftPlan py, const float2* __restrict__ tw_g,
                                                const float* __restrict__ psi, const float* __restrict__ phi,
                                                const uint8_t* __restrict__ mask, const float2* tin, float2* tout,
                                                int W) {
  extern __shared__ float2 smem[];
  const int ny = g.ny, nz = g.nz, N = ny * nz, K = g.K;
  float2* tw = smem;
  float2* buf = smem + ((ny + 1) & ~1);
  const int ld = ny + 1;
  const int s = blockIdx.z, c = blockIdx.y;
  const int z0 = blockIdx.x * W;
  const int wc = min(W, nz - z0);
  for (int i = threadIdx.x; i < ny; i += blockDim.x) tw[i] = tw_g[i];
  const float2* tb = tin + ((long long)(s * g.C + c) * K) * N + z0;
  const int nel = K * ny * wc;
  for (int e = threadIdx.x; e < nel; e += kFftThreads) {
    const int w = e % wc;
    const int rest = e / wc;
    const int y = rest % ny, k = rest / ny;
    float2 v = tb[(long long)k * N + (long long)y * nz + w];
    if (MODE == COL_ADJ_DATA) v = cscale(v, g.gsign * g.inv_sqrt_n * parity_sign(y + z0 + w));
    buf[(k * wc + w) * ld + y] = v;
  }
  __syncthreads();
  if (MODE == COL_ADJ_DATA) {
    fft_lines<true, R13>(buf, ld, K * wc, py, tw);
  } else {
    fft_lines<false, R13>(buf, ld, K * wc, py, tw);
    const int npt = ny * wc;
    if (MODE == COL_NORMAL || MODE == COL_FWD_PROJ) {
      const float pscale = (MODE == COL_FWD_PROJ) ? (float)N : 1.0f;
      for (int q = threadIdx.x; q < npt; q += kFftThreads) {
        const int w = q % wc, y = q / wc;
        const long long n = (long long)y * nz + z0 + w;
        float2 v[KC], u[KC];
        const float sg = (MODE == COL_FWD_PROJ) ? g.gsign * g.inv_sqrt_n * parity_sign(y + z0 + w) : 1.0f;
#pragma unroll
        for (int k = 0; k < KC; ++k) {
          v[k] = (k < K) ? cscale(buf[(k * wc + w) * ld + y], sg) : make_float2(0.f, 0.f);
          u[k] = make_float2(0.f, 0.f);
        }
        int p = 0;
#pragma unroll
        for (int k = 0; k < KC; ++k)
#pragma unroll
          for (int l = k; l < KC; ++l)
            if (l < K) {
              const float ps = __ldg(psi + (long long)p * N + n) * pscale;
              ++p;
              u[k].x = fmaf(ps, v[l].x, u[k].x);
              u[k].y = fmaf(ps, v[l].y, u[k].y);
              if (l != k) {
                u[l].x = fmaf(ps, v[k].x, u[l].x);
                u[l].y = fmaf(ps, v[k].y, u[l].y);
              }
            }
        if (MODE == COL_NORMAL) {
#pragma unroll
          for (int k = 0; k < KC; ++k)
            if (k < K) buf[(k * wc + w) * ld + y] = u[k];
        } else {
          float2* yb = tout + ((long long)(s * g.C + c) * K) * N + n;
#pragma unroll
          for (int k = 0; k < KC; ++k)
            if (k < K) yb[(long long)k * N] = u[k];
        }
      }
      __syncthreads();
      if (MODE == COL_FWD_PROJ) return;
      fft_lines<true, R13>(buf, ld, K * wc, py, tw);
    } else {  // COL_FWD_TE
      for (int q = threadIdx.x; q < npt; q += kFftThreads) {
        const int w = q % wc, y = q / wc;
        const long long n = (long long)y * nz + z0 + w;
        const float sg = g.gsign * g.inv_sqrt_n * parity_sign(y + z0 + w);
        float2 v[KC];
#pragma unroll
        for (int k = 0; k < KC; ++k) v[k] = (k < K) ? cscale(buf[(k * wc + w) * ld + y], sg) : make_float2(0.f, 0.f);
        float2* yb = tout + ((long long)(s * g.C + c) * g.T) * N + n;
        for (int tt = 0; tt < g.T; ++tt) {
          float2 a = make_float2(0.f, 0.f);
          if (mask[(long long)tt * N + n]) {
#pragma unroll
            for (int k = 0; k < KC; ++k)
              if (k < K) {
                const float ph = __ldg(phi + tt * K + k);
                a.x = fmaf(ph, v[k].x, a.x);
                a.y = fmaf(ph, v[k].y, a.y);
              }
          }
          yb[(long long)tt * N] = a;
        }
      }
      return;
    }
  }
  // store the columns back (COL_NORMAL, COL_ADJ_DATA)
  float2* ob = tout + ((long long)(s * g.C + c) * K) * N + z0;
  for (int e = threadIdx.x; e < nel; e += kFftThreads) {
    const int w = e % wc;
    const int rest = e / wc;
    const int y = rest % ny, k = rest / ny;
    ob[(long long)k * N + (long long)y * nz + w] = buf[(k * wc + w) * ld + y];
  }
}

int row_rows_per_cta(const Geom& g) {
  const int kc = g.K <= 4 ? 4 : 8;
  const int pmax = (kc * g.M <= 4) ? 4 : (kc * g.M <= 8 ? 2 : 1);
  int rb = 8;
  while (rb > 1 && (rb * g.nz > pmax * kFftThreads || g.K * rb * g.nz > kMaxLineElems)) --rb;
  return rb;
}

int col_cols_per_cta(const Geom& g) {
  int w = 8;
  while (w > 1 && g.K * w * g.ny > kMaxLineElems) --w;
  return w;
}

template <int MODE, int KC, int MC, bool R13>
static cudaError_t row_go13(const Geom& g, const FftPlan& pz, const float2* tw, const float2* maps, const float2* x,
                            float2* t, float2* out, cudaStream_t st) {
  const int RB = row_rows_per_cta(g);
  const size_t lines = (((size_t)g.K * RB * (g.nz + 1) + 1) & ~(size_t)1) * (MODE == ROW_ADJ ? 2 : 1);
  const size_t sm = sizeof(float2) * (((g.nz + 1) & ~1) + lines + 2 * (size_t)g.M * RB * g.nz);
  {
    const cudaError_t e = smem_optin((const void*)k_row<MODE, KC, MC, R13>, 200 * 1024);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((g.ny + RB - 1) / RB, g.S);
  k_row<MODE, KC, MC, R13><<<grid, kFftThreads, sm, st>>>(g, pz, tw, maps, x, t, out, RB);
  return cudaGetLastError();
}

template <int MODE, int KC, int MC>
static cudaError_t row_go(const Geom& g, const FftPlan& pz, const float2* tw, const float2* maps, const float2* x,
                          float2* t, float2* out, cudaStream_t st) {
  return plan_has13(pz) ? row_go13<MODE, KC, MC, true>(g, pz, tw, maps, x, t, out, st)
                        : row_go13<MODE, KC, MC, false>(g, pz, tw, maps, x, t, out, st);
}

cudaError_t launch_row(const Geom& g, RowMode mode, const FftPlan& pz, const float2* tw_z, const float2* maps,
                       const float2* x, float2* t, float2* out, cudaStream_t st) {
  const cudaError_t ef = launch_row_fast(g, mode, tw_z, maps, x, t, out, st);
  if (ef != cudaErrorNotSupported) return ef;
  const bool k4 = g.K <= 4, m1 = g.M == 1;
  if (mode == ROW_FWD) {
    if (k4 && m1) return row_go<ROW_FWD, 4, 1>(g, pz, tw_z, maps, x, t, out, st);
    if (k4) return row_go<ROW_FWD, 4, 2>(g, pz, tw_z, maps, x, t, out, st);
    if (m1) return row_go<ROW_FWD, 8, 1>(g, pz, tw_z, maps, x, t, out, st);
    return row_go<ROW_FWD, 8, 2>(g, pz, tw_z, maps, x, t, out, st);
  }
  if (k4 && m1) return row_go<ROW_ADJ, 4, 1>(g, pz, tw_z, maps, x, t, out, st);
  if (k4) return row_go<ROW_ADJ, 4, 2>(g, pz, tw_z, maps, x, t, out, st);
  if (m1) return row_go<ROW_ADJ, 8, 1>(g, pz, tw_z, maps, x, t, out, st);
  return row_go<ROW_ADJ, 8, 2>(g, pz, tw_z, maps, x, t, out, st);
}

template <int MODE, int KC, bool R13>
static cudaError_t col_go13(const Geom& g, const FftPlan& py, const float2* tw, const float* psi, const float* phi,
                            const uint8_t* mask, const float2* tin, float2* tout, cudaStream_t st) {
  const int W = col_cols_per_cta(g);
  const size_t sm = sizeof(float2) * (((g.ny + 1) & ~1) + (size_t)g.K * W * (g.ny + 1));
  {
    const cudaError_t e = smem_optin((const void*)k_col<MODE, KC, R13>, 200 * 1024);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((g.nz + W - 1) / W, g.C, g.S);
  k_col<MODE, KC, R13><<<grid, kFftThreads, sm, st>>>(g, py, tw, psi, phi, mask, tin, tout, W);
  return cudaGetLastError();
}

template <int MODE, int KC>
static cudaError_t col_go(const Geom& g, const FftPlan& py, const float2* tw, const float* psi, const float* phi,
                          const uint8_t* mask, const float2* tin, float2* tout, cudaStream_t st) {
  return plan_has13(py) ? col_go13<MODE, KC, true>(g, py, tw, psi, phi, mask, tin, tout, st)
                        : col_go13<MODE, KC, false>(g, py, tw, psi, phi, mask, tin, tout, st);
}

template <int KC, bool R13>
static cudaError_t col_normal_go13(const Geom& g, const FftPlan& py, const float2* tw, const float* psi, float2* t,
                                   cudaStream_t st) {
  const int W = col_cols_per_cta(g);
  const size_t sm = sizeof(float2) * (((g.ny + 1) & ~1) + 2 * (size_t)g.K * W * (g.ny + 1));
  int grid_per_sm = 0, nsm = 0;
  {
    const void* kern = (const void*)k_col_normal<KC, R13>;
    cudaError_t e = smem_optin(kern, 200 * 1024);
    if (e == cudaSuccess) e = sm_count(&nsm);
    if (e == cudaSuccess) e = ctas_per_sm(kern, kFftThreads, sm, &grid_per_sm);
    if (e != cudaSuccess) return e;
  }
  const int ntz = (g.nz + W - 1) / W;
  const long long ntiles = (long long)g.S * g.C * ntz;
  if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  const int grid = (int)std::min<long long>(ntiles, (long long)nsm * grid_per_sm);
  k_col_normal<KC, R13><<<grid, kFftThreads, sm, st>>>(g, py, tw, psi, t, W, ntz, (int)ntiles);
  return cudaGetLastError();
}

template <int KC>
static cudaError_t col_normal_go(const Geom& g, const FftPlan& py, const float2* tw, const float* psi, float2* t,
                                 cudaStream_t st) {
  return plan_has13(py) ? col_normal_go13<KC, true>(g, py, tw, psi, t, st)
                        : col_normal_go13<KC, false>(g, py, tw, psi, t, st);
}

cudaError_t launch_col(const Geom& g, ColMode mode, const FftPlan& py, const float2* tw_y, const float* psi,
                       const float* phi, const uint8_t* mask, const float2* tin, float2* tout, cudaStream_t st) {
  const bool k4 = g.K <= 4;
  switch (mode) {
    case COL_NORMAL:
      if (tin != tout) return cudaErrorInvalidValue;  // the normal-operator pass works in place
      if (g.colvar == 3) {
        const cudaError_t ec = launch_col_normal_tc(g, tw_y, psi, tout, st);
        if (ec != cudaErrorNotSupported) return ec;
      }
      if (g.colvar == 0 || g.colvar == 3 || g.colvar == 4) {
        const cudaError_t et = launch_col_normal_tma(g, tw_y, psi, tout, st);
        if (et != cudaErrorNotSupported) return et;
      }
      {
        const cudaError_t ef = launch_col_normal_fast(g, tw_y, psi, tout, st);
        if (ef != cudaErrorNotSupported) return ef;
        const cudaError_t ep = launch_col_normal_pr(g, tw_y, psi, tout, st);
        if (ep != cudaErrorNotSupported) return ep;
      }
      return k4 ? col_normal_go<4>(g, py, tw_y, psi, tout, st) : col_normal_go<8>(g, py, tw_y, psi, tout, st);
    case COL_ADJ_DATA: {
      const cudaError_t et = launch_col_adj_tma(g, tw_y, tin, tout, st);
      if (et != cudaErrorNotSupported) return et;
    }
      return k4 ? col_go<COL_ADJ_DATA, 4>(g, py, tw_y, psi, phi, mask, tin, tout, st)
                : col_go<COL_ADJ_DATA, 8>(g, py, tw_y, psi, phi, mask, tin, tout, st);
    case COL_FWD_PROJ:
      return k4 ? col_go<COL_FWD_PROJ, 4>(g, py, tw_y, psi, phi, mask, tin, tout, st)
                : col_go<COL_FWD_PROJ, 8>(g, py, tw_y, psi, phi, mask, tin, tout, st);
    case COL_FWD_TE:
      return k4 ? col_go<COL_FWD_TE, 4>(g, py, tw_y, psi, phi, mask, tin, tout, st)
                : col_go<COL_FWD_TE, 8>(g, py, tw_y, psi, phi, mask, tin, tout, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace t2sh
