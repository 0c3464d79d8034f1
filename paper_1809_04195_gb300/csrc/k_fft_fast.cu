// Size-specialised row and column passes for line lengths N = 16 * R1 (R1 in
// {3, 4, 6, 8, 10, 12, 15, 16}: 48 ... 256, all slice sizes of the knee workloads).
//
// A line of N points is transformed by 16 threads in two register stages with one
// shared-memory exchange, every index a compile-time constant:
//   forward  [R1, 16]: thread j < 16 holds x[j + 16 r] (r < R1), DFT_R1; exchange;
//                      thread j' < R1 holds Y[j' + R1 r] (r < 16), twiddle w^(r j'), DFT_16
//                      -> X[j' + R1 k] (k < 16).
//   inverse  [16, R1]: thread j' < R1 holds X[j' + R1 r], IDFT_16; exchange;
//                      thread j < 16 holds Y[j + 16 r], twiddle w^(-r j), IDFT_R1
//                      -> x[j + 16 k] (k < R1).
// The row pass (kz) keeps each line in one half-warp, so global loads of a row are
// 128-byte runs; the column pass (ky) puts the 8 columns of a tile on adjacent lanes.
// The column pass and the row pass's map rows stream into shared memory with cp.async while
// the previous tile or coil is transformed; the adjoint row pass reads its t rows straight
// from global memory into registers (a half-warp reads 16 consecutive values).
#include <algorithm>

// packed two-lane complex additions in the butterflies: measured 3 % faster for the
// forward and 10 % faster for the adjoint row pass on the knee scan
#define T2SH_PACKED_ADD 1
#include "t2sh_device.cuh"

namespace t2sh {

template <int R1>
using Ex = ExLayout<R1>;

// ------------------------------------------------------------------------------------
// Row pass.  CTA = (slice, band of RB rows), 16 x 4 x RB threads, thread
// (j, line = k * RB + r).  K <= 4, M <= 2.  With one map set and N < 240 the bands are
// two rows (128 threads) and the kernel is held to 64 registers (forward, eight CTAs per
// SM) or 96 (adjoint, five): many small CTAs keep the SM issuing while others wait at
// their per-coil barriers (forward 1.47 -> 1.18 ms on the knee scan against bands of 8
// rows).  N >= 240 and two map sets keep bands of 4 rows without a block bound, except
// two map sets at N = 240 (Table I), which run two-row bands at 96 registers for the forward
// (five CTAs per SM; at 64 registers it spills: 2.17 ms) and 128 for the adjoint (four):
// forward 1.44 -> 1.39 ms, adjoint 1.58 -> 1.48 ms.  The
// adjoint reads t straight into registers instead of staging it by cp.async (knee
// 1.51 -> 1.31 ms, Table I shape 2.30 -> 1.52 ms): the staging cost more instructions
// than the latency it hid.  On two-row bands the next coil's values are loaded one coil
// ahead (1.31 -> 1.28 ms).
// ------------------------------------------------------------------------------------
// Padded strides (float2) of the row pass's exchange lines (LX) and staged map rows (MS).
// The packed second stage reads R1 consecutive items from each of several lines per
// half-warp; a stride congruent to R1 modulo 16 lays those windows side by side across
// the banks.  MS stays even so that the 16-byte cp.async copies remain aligned.
template <int N>
struct RowPad {
  static constexpr int R1 = N / 16;
  static constexpr int LINE = ExLayout<R1>::LINE;
  static constexpr int even_r1 = (R1 % 2 == 0) ? R1 : R1 + 1;
  static constexpr int LX = (R1 < 16) ? LINE + ((R1 - LINE % 16) % 16 + 16) % 16 : LINE;
  static constexpr int MS = (R1 < 16) ? N + ((even_r1 - N % 16) % 16 + 16) % 16 : N;
  static_assert(MS % 2 == 0 && LX >= LINE && MS >= N, "row pass strides");
};

template <int N, int MC, int MODE>
struct RowFastRB {
  // two-row bands, occupancy-bounded kernel
  static constexpr bool small = (MC == 1 && N < 240) || (MC == 2 && N == 240);
  static constexpr int value = small ? 2 : 4;
  static constexpr int min_blocks = MC == 2 ? (MODE == ROW_FWD ? 5 : 4) : (MODE == ROW_FWD ? 8 : 5);
};

template <int N, int MODE, int MC, int kRowRB = RowFastRB<N, MC, MODE>::value>
__device__ __forceinline__ void row_fast_body(const Geom& g, const float2* __restrict__ tw_g,
                                              const float2* __restrict__ maps, const float2* __restrict__ x,
                                              float2* __restrict__ t, float2* __restrict__ out) {
  constexpr int R1 = N / 16;
  constexpr int LINE = RowPad<N>::LX;
  constexpr int MS = RowPad<N>::MS;
  constexpr int SF = Ex<R1>::SF;
  extern __shared__ float2 smem[];
  const int NN = g.ny * N, K = g.K, M = g.M;
  const int s = blockIdx.y, y0 = blockIdx.x * kRowRB;
  const int rb = min(kRowRB, g.ny - y0);
  constexpr int NL = 4 * kRowRB;  // lines per CTA
  const int j = threadIdx.x & 15;
  const int L = threadIdx.x >> 4;  // line: k * RB + r
  const int k = L / kRowRB, r = L - k * kRowRB;
  const bool live = (k < K) && (r < rb);
  // shared memory: twiddles | exchange [NL][LINE] | maps stage x2 [MC][RB][MS]
  float2* tw = smem;
  float2* ex = tw + N;
  float2* mst = ex + NL * LINE;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];

  // 16-byte copies of the coil's map rows walked over
  // (plane, row < RB, column pair) with compile-time divisors; rows past a partial band's
  // end are skipped
  auto issue = [&](int c, int buf) {
    constexpr int H = N / 2;  // 16-byte copies per row
    const float2* mp = maps + ((long long)(s * g.C + c) * M) * NN + (long long)y0 * N;
    float2* md = mst + buf * MC * kRowRB * MS;
    for (int e2 = threadIdx.x; e2 < M * kRowRB * H; e2 += blockDim.x) {
      const int line = e2 / H, col = 2 * (e2 - line * H);
      const int m = line / kRowRB, row = line - m * kRowRB;
      if (row < rb) cp_async16(md + line * MS + col, mp + (long long)m * NN + row * N + col);
    }
  };
  issue(0, 0);
  cp_async_commit();

  float2 xr[MC][R1];   // ROW_FWD: x at z = j + 16 q
  float2 acc[MC][16];  // ROW_ADJ: accumulated output at z = j + R1 q (j < R1)
#pragma unroll
  for (int m = 0; m < MC; ++m) {
#pragma unroll
    for (int q = 0; q < R1; ++q) {
      xr[m][q] = make_float2(0.f, 0.f);
      if (MODE == ROW_FWD && live && m < M)
        xr[m][q] = x[((long long)(s * M + m) * K + k) * NN + (long long)(y0 + r) * N + j + 16 * q];
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[m][q] = make_float2(0.f, 0.f);
  }
  float2* exl = ex + L * LINE;
  // Stage B has R1 < 16 work items per line: they are packed onto consecutive threads
  // (item (Lb, jb) on thread Lb * R1 + jb) so that whole warps idle instead of 16 - R1
  // lanes of every line's half-warp.
  constexpr bool kPack = R1 < 16;
  const int Lb = kPack ? (int)threadIdx.x / R1 : L;
  const int jb = kPack ? (int)threadIdx.x - Lb * R1 : j;
  const int kb = Lb / kRowRB, rbb = Lb - kb * kRowRB;
  const bool liveb = (kPack ? ((int)threadIdx.x < NL * R1) : (j < R1)) && kb < K && rbb < rb;
  const float2* exb = ex + Lb * LINE;

  // adjoint on two-row bands: the next coil's t values are requested one coil ahead, into
  // registers (the four-row kernel has no registers to spare for them)
  constexpr bool kPrefetchT = MODE == ROW_ADJ && RowFastRB<N, MC, MODE>::small;
  float2 tn[kPrefetchT ? R1 : 1];
  if constexpr (kPrefetchT) {
    const float2* trow = t + ((long long)(s * g.C) * K + k) * NN + (long long)(y0 + r) * N;
#pragma unroll
    for (int q = 0; q < R1; ++q) tn[q] = live ? trow[j + 16 * q] : make_float2(0.f, 0.f);
  }
  for (int c = 0; c < g.C; ++c) {
    const int buf = c & 1;
    if (c + 1 < g.C) issue(c + 1, buf ^ 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const float2* mrow = mst + buf * MC * kRowRB * MS + r * MS;
    float2 a[R1];
    if (MODE == ROW_FWD) {
#pragma unroll
      for (int q = 0; q < R1; ++q) {
        float2 v = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < MC; ++m)
          if (m < M) cfma(v, mrow[m * kRowRB * MS + j + 16 * q], xr[m][q]);
        a[q] = v;
      }
      dft_r<R1, false>(a);
    } else {
      // t straight from global memory: a half-warp reads 16 consecutive values per q
      if constexpr (kPrefetchT) {
#pragma unroll
        for (int q = 0; q < R1; ++q) a[q] = tn[q];
        if (c + 1 < g.C) {
          const float2* trow = t + ((long long)(s * g.C + c + 1) * K + k) * NN + (long long)(y0 + r) * N;
#pragma unroll
          for (int q = 0; q < R1; ++q) tn[q] = live ? trow[j + 16 * q] : make_float2(0.f, 0.f);
        }
      } else {
        const float2* trow = t + ((long long)(s * g.C + c) * K + k) * NN + (long long)(y0 + r) * N;
#pragma unroll
        for (int q = 0; q < R1; ++q) a[q] = live ? trow[j + 16 * q] : make_float2(0.f, 0.f);
      }
      dft_r<R1, true>(a);
    }
#pragma unroll
    for (int q = 0; q < R1; ++q) exl[j * SF + q] = a[q];
    __syncthreads();
    if (liveb) {
      float2 b[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) b[q] = exb[q * SF + jb];
#pragma unroll
      for (int q = 1; q < 16; ++q) b[q] = (MODE == ROW_FWD) ? twiddle_mul<false>(b[q], tw[q * jb]) : twiddle_mul<true>(b[q], tw[q * jb]);
      if (MODE == ROW_FWD) {
        dft16<false>(b);
        float2* tp = t + ((long long)(s * g.C + c) * K + kb) * NN + (long long)(y0 + rbb) * N + jb;
#pragma unroll
        for (int q = 0; q < 16; ++q) tp[R1 * q] = b[q];
      } else {
        dft16<true>(b);
        const float2* mrowb = mst + buf * MC * kRowRB * MS + rbb * MS;
#pragma unroll
        for (int m = 0; m < MC; ++m)
          if (m < M) {
#pragma unroll
            for (int q = 0; q < 16; ++q) cfmac(acc[m][q], mrowb[m * kRowRB * MS + jb + R1 * q], b[q]);
          }
      }
    }
    __syncthreads();
  }
  cp_async_wait<0>();
  if (MODE == ROW_ADJ && liveb) {
#pragma unroll
    for (int m = 0; m < MC; ++m)
      if (m < M) {
        float2* op = out + ((long long)(s * M + m) * K + kb) * NN + (long long)(y0 + rbb) * N + jb;
#pragma unroll
        for (int q = 0; q < 16; ++q) op[R1 * q] = acc[m][q];
      }
  }
}

template <int N, int MODE, int MC>
__global__ void __launch_bounds__(64 * RowFastRB<N, MC, MODE>::value, RowFastRB<N, MC, MODE>::min_blocks)
    k_row_fast(Geom g, const float2* __restrict__ tw_g, const float2* __restrict__ maps,
               const float2* __restrict__ x, float2* __restrict__ t, float2* __restrict__ out) {
  row_fast_body<N, MODE, MC>(g, tw_g, maps, x, t, out);
}

template <int N, int MODE, int MC>
__global__ void __launch_bounds__(64 * RowFastRB<N, MC, MODE>::value)
    k_row_fast_wide(Geom g, const float2* __restrict__ tw_g, const float2* __restrict__ maps,
                    const float2* __restrict__ x, float2* __restrict__ t, float2* __restrict__ out) {
  row_fast_body<N, MODE, MC>(g, tw_g, maps, x, t, out);
}

// ------------------------------------------------------------------------------------
// Column pass of the normal operator (DFT_y, Psi, IDFT_y), persistent over
// (slice, coil, W-column tile) tiles, W x 4 x 16 threads, thread (w, k, j).
// The tile's columns are staged in shared memory by cp.async, refilled for the next
// tile as soon as the forward stage A has consumed them; the tile's block of Psi
// (P x N x W floats) is staged the same way right after the Psi step.  With W = 4 a
// CTA uses about 106 KB, so two CTAs share an SM.  Requires nz % W == 0, K <= 4.
// ------------------------------------------------------------------------------------
template <int N, int W>
struct ColFast {
  static constexpr int R1 = N / 16;
  static constexpr int LS = N + 1;         // exchange line stride (odd)
  static constexpr int PS = N * W + W;     // staging plane stride (pad W: basis lines on other banks)
  static constexpr int THREADS = W * 64;
  static constexpr size_t smem(int P) {
    return sizeof(float2) * ((size_t)N + 4 * W * (size_t)LS + 4 * (size_t)PS) + sizeof(float) * (size_t)P * N * W;
  }
};

template <int N, int W>
__global__ void __launch_bounds__(W * 64) k_col_fast(Geom g, const float2* __restrict__ tw_g,
                                                    const float* __restrict__ psi, float2* t, int ntz, int ntiles) {
  using CF = ColFast<N, W>;
  constexpr int R1 = CF::R1, LS = CF::LS, PS = CF::PS;
  extern __shared__ float2 smem[];
  const int nz = g.nz, NN = N * nz, K = g.K, P = g.P;
  const int w = threadIdx.x % W, k = (threadIdx.x / W) & 3, j = threadIdx.x / (4 * W);
  float2* tw = smem;
  float2* ex = tw + N;                                      // [k][w][LS]
  float2* st = ex + 4 * W * LS;                             // [k][y][W] (+ pad per k)
  float* ps = reinterpret_cast<float*>(st + 4 * PS);         // [p][y][W]
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];

  auto issue_t = [&](int tile) {
    const int sc = tile / ntz, z0 = (tile - sc * ntz) * W;
    const float2* tb = t + (long long)sc * K * NN + z0;
    const int n16 = K * N * (W / 2);  // 16-byte copies
    for (int e = threadIdx.x; e < n16; e += blockDim.x) {
      const int w2 = (e % (W / 2)) * 2;
      const int row = e / (W / 2);  // k * N + y
      const int kk = row / N, y = row - kk * N;
      cp_async16(st + kk * PS + y * W + w2, tb + (long long)kk * NN + (long long)y * nz + w2);
    }
  };
  auto issue_psi = [&](int tile) {
    const int sc = tile / ntz, z0 = (tile - sc * ntz) * W;
    const int n16 = P * N * (W / 4);  // 16-byte copies of 4 floats
    for (int e = threadIdx.x; e < n16; e += blockDim.x) {
      const int w4 = (e % (W / 4)) * 4;
      const int row = e / (W / 4);  // p * N + y
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
    // forward stage A: x[j + 16 q] of column w, basis line k
    if (live) {
      const float2* sp = st + k * PS + w;
      float2 a[R1];
#pragma unroll
      for (int q = 0; q < R1; ++q) a[q] = sp[(j + 16 * q) * W];
      dft_r<R1, false>(a);
#pragma unroll
      for (int q = 0; q < R1; ++q) exl[j * R1 + q] = a[q];
    }
    __syncthreads();
    if (nxt < ntiles) issue_t(nxt);  // the staging area is free again
    cp_async_commit();
    // forward stage B: X[j + R1 q]
    if (live && j < R1) {
      float2 b[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) b[q] = exl[j + R1 * q];
#pragma unroll
      for (int q = 1; q < 16; ++q) b[q] = twiddle_mul<false>(b[q], tw[q * j]);
      dft16<false>(b);
#pragma unroll
      for (int q = 0; q < 16; ++q) exl[j + R1 * q] = b[q];
    }
    __syncthreads();
    // space-time kernel: u_k = sum_l Psi_kl v_l; a thread takes 4 adjacent points of row ky
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
    if (nxt < ntiles) issue_psi(nxt);  // the Psi block is free again
    cp_async_commit();
    // inverse stage A': IDFT_16 of X[j + R1 q]
    float2 b[16];
    if (live && j < R1) {
#pragma unroll
      for (int q = 0; q < 16; ++q) b[q] = exl[j + R1 * q];
      dft16<true>(b);
    }
    __syncthreads();
    if (live && j < R1) {
#pragma unroll
      for (int q = 0; q < 16; ++q) exl[j * 16 + q] = b[q];
    }
    __syncthreads();
    // inverse stage B': y = j + 16 q, written straight back to global memory
    if (live) {
      float2 a[R1];
#pragma unroll
      for (int q = 0; q < R1; ++q) a[q] = twiddle_mul<true>(exl[j + 16 * q], tw[q * j]);
      dft_r<R1, true>(a);
      float2* ob = t + ((long long)sc * K + k) * NN + z0 + w;
#pragma unroll
      for (int q = 0; q < R1; ++q) ob[(long long)(j + 16 * q) * nz] = a[q];
    }
  }
  cp_async_wait<0>();
}

// ------------------------------------------------------------------------------------
// launchers: return cudaErrorNotSupported when the shape has no specialised kernel
// ------------------------------------------------------------------------------------
constexpr int kColW = 8;  // columns per tile of the column pass
template <int N, int MODE, int MC>
static size_t row_fast_smem() {
  constexpr int R1 = N / 16, RB = RowFastRB<N, MC, MODE>::value, NL = 4 * RB;
  constexpr int MS = RowPad<N>::MS;
  return sizeof(float2) * ((size_t)N + NL * RowPad<N>::LX + 2 * (size_t)MC * RB * MS +
                           0);
}

template <int N, int MODE, int MC>
static cudaError_t row_fast_go(const Geom& g, const float2* tw, const float2* maps, const float2* x, float2* t,
                               float2* out, cudaStream_t st) {
  using RF = RowFastRB<N, MC, MODE>;
  constexpr int RB = RF::value;
  const size_t sm = row_fast_smem<N, MODE, MC>();
  auto kern = [] {
    if constexpr (RF::small) return k_row_fast<N, MODE, MC>;
    else return k_row_fast_wide<N, MODE, MC>;
  }();
  {
    const cudaError_t e = smem_optin((const void*)kern, (int)sm);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((g.ny + RB - 1) / RB, g.S);
  kern<<<grid, 64 * RB, sm, st>>>(g, tw, maps, x, t, out);
  return cudaGetLastError();
}

template <int N>
static cudaError_t row_fast_n(const Geom& g, RowMode mode, const float2* tw, const float2* maps, const float2* x,
                              float2* t, float2* out, cudaStream_t st) {
  if (mode == ROW_FWD)
    return g.M == 1 ? row_fast_go<N, ROW_FWD, 1>(g, tw, maps, x, t, out, st)
                    : row_fast_go<N, ROW_FWD, 2>(g, tw, maps, x, t, out, st);
  return g.M == 1 ? row_fast_go<N, ROW_ADJ, 1>(g, tw, maps, x, t, out, st)
                  : row_fast_go<N, ROW_ADJ, 2>(g, tw, maps, x, t, out, st);
}

cudaError_t launch_row_fast(const Geom& g, RowMode mode, const float2* tw_z, const float2* maps, const float2* x,
                            float2* t, float2* out, cudaStream_t st) {
  if (g.K > 4 || g.M > 2) return cudaErrorNotSupported;
  switch (g.nz) {
    case 48: return row_fast_n<48>(g, mode, tw_z, maps, x, t, out, st);
    case 64: return row_fast_n<64>(g, mode, tw_z, maps, x, t, out, st);
    case 96: return row_fast_n<96>(g, mode, tw_z, maps, x, t, out, st);
    case 128: return row_fast_n<128>(g, mode, tw_z, maps, x, t, out, st);
    case 160: return row_fast_n<160>(g, mode, tw_z, maps, x, t, out, st);
    case 192: return row_fast_n<192>(g, mode, tw_z, maps, x, t, out, st);
    case 240: return row_fast_n<240>(g, mode, tw_z, maps, x, t, out, st);
    case 256: return row_fast_n<256>(g, mode, tw_z, maps, x, t, out, st);
    default: return cudaErrorNotSupported;
  }
}

template <int N, int W>
static cudaError_t col_fast_go(const Geom& g, const float2* tw, const float* psi, float2* t, cudaStream_t st) {
  using CF = ColFast<N, W>;
  const size_t sm = CF::smem(g.P);
  int nsm = 0, per = 0;
  {
    const void* kern = (const void*)k_col_fast<N, W>;
    cudaError_t e = smem_optin(kern, (int)CF::smem(10));
    if (e == cudaSuccess) e = sm_count(&nsm);
    if (e == cudaSuccess) e = ctas_per_sm(kern, CF::THREADS, CF::smem(10), &per);
    if (e != cudaSuccess) return e;
  }
  const int ntz = g.nz / W;
  const long long ntiles = (long long)g.S * g.C * ntz;
  if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  const int grid = (int)std::min<long long>(ntiles, (long long)nsm * per);
  k_col_fast<N, W><<<grid, CF::THREADS, sm, st>>>(g, tw, psi, t, ntz, (int)ntiles);
  return cudaGetLastError();
}

template <int W>
static cudaError_t col_fast_w(const Geom& g, const float2* tw_y, const float* psi, float2* t, cudaStream_t st) {
  if (g.K > 4 || g.nz % W != 0) return cudaErrorNotSupported;
  switch (g.ny) {
    case 48: return col_fast_go<48, W>(g, tw_y, psi, t, st);
    case 64: return col_fast_go<64, W>(g, tw_y, psi, t, st);
    case 96: return col_fast_go<96, W>(g, tw_y, psi, t, st);
    case 128: return col_fast_go<128, W>(g, tw_y, psi, t, st);
    case 160: return col_fast_go<160, W>(g, tw_y, psi, t, st);
    case 192: return col_fast_go<192, W>(g, tw_y, psi, t, st);
    case 240: return col_fast_go<240, W>(g, tw_y, psi, t, st);
    case 256: return col_fast_go<256, W>(g, tw_y, psi, t, st);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t launch_col_normal_fast(const Geom& g, const float2* tw_y, const float* psi, float2* t, cudaStream_t st) {
  return g.colvar == 2 ? col_fast_w<4>(g, tw_y, psi, t, st) : col_fast_w<kColW>(g, tw_y, psi, t, st);
}

}  // namespace t2sh
