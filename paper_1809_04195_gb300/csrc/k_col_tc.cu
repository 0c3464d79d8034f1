// Mixed-precision column pass of the normal operator on the tensor cores: the DFT along
// ky, the space-time kernel Psi, the inverse DFT along ky (the column part of
// F^H Psi F, Sec. IV.B), with each length-N DFT (N = 16 R1) computed as two batched
// small-DFT GEMMs on tcgen05 (Cooley-Tukey with N1 = R1, N2 = 16):
//
//   stage 1:  Y[l, n2, k1] = sum_n1 W_R1^(n1 k1) x_l[16 n1 + n2]        (GEMM, K = R1)
//   twiddle:  Y'           = W_N^(n2 k1) Y                              (CUDA cores)
//   stage 2:  X_l[k1 + R1 k2] = sum_n2 W_16^(n2 k2) Y'[l, n2, k1]       (GEMM, K = 16)
//
// A complex GEMM is a real one on interleaved (re, im) pairs: the DFT matrix becomes the
// 2R x 2R real matrix [[c, -s], [s, c]] per entry.  Operands are split BF16 pairs
// (x = x_hi + x_lo, W = W_hi + W_lo) and D = W_hi x_hi + W_hi x_lo + W_lo x_hi is
// accumulated in FP32 in tensor memory, about 16 significant bits per product.
//
// One CTA (256 threads, two per SM) owns a tile of 4 columns z of one (slice, coil) and
// all K <= 4 basis images, i.e. L = 4 K lines of length N.  The tile arrives by a 3D
// tensor-map copy (TMA) into shared memory; then forward stages 1 and 2, Psi applied in
// shared memory at every (ky, z) across the K basis values, inverse stages 1 and 2
// (conjugate matrices and twiddles), and the result goes from TMEM straight to global
// memory.  The next tile's copy is issued as soon as the inverse stage-1 operand has
// been built from the current one, so it overlaps the inverse GEMMs and epilogues.  Thread 0 issues the MMAs; completion arrives on an mbarrier whose waits are
// bounded by the global timer.  Each CTA allocates 128 TMEM columns and at least 80 KB of
// shared memory, so at most two such CTAs share an SM and TMEM is never oversubscribed.
#include <cuda.h>

#include <algorithm>

#include "t2sh_device.cuh"

namespace t2sh {

namespace {

constexpr int kTcThreads = 256;
constexpr int kTcW = 4;           // z columns per tile
constexpr int kTcTmemCols = 128;  // stage-1 accumulators at column 0, stage-2 at 64

template <int R1>
struct ColTc {
  static constexpr int N = 16 * R1;
  static constexpr int KD1 = (2 * R1 <= 16) ? 16 : 32;  // stage-1 K extent (reals), padded
  static constexpr int ND1 = KD1;                       // stage-1 N extent (2 R1, padded)
  static constexpr int LBO1 = 128, SBO1 = KD1 / 8 * 128;
  // stage-2 operand: core matrices along K 192 B apart (not 128) so that the scattered
  // 4-byte writes of the stage-1 epilogue hit 32 different banks
  static constexpr int LBO2 = 192, SBO2 = 768;
  static constexpr int kMatB1 = ND1 * KD1 * 2;  // bytes of one stage-1 matrix
  static constexpr int kMatB2 = 32 * 32 * 2;
  static constexpr size_t kA = 32 * SBO2;       // bytes of one operand buffer (256 rows)
  // shared-memory map (bytes)
  static constexpr size_t up(size_t b) { return (b + 1023) / 1024 * 1024; }
  static constexpr size_t off_b1 = up((size_t)N * 8);        // after the twiddles
  static constexpr size_t off_b2 = off_b1 + 4 * kMatB1;      // fwd hi, fwd lo, inv hi, inv lo
  static constexpr size_t off_ahi = up(off_b2 + 4 * kMatB2);
  static constexpr size_t off_alo = off_ahi + kA;
  static constexpr size_t off_x = off_alo + kA;               // t tile [k][y][4] (TMA box)
  static constexpr size_t off_bar = off_x + (size_t)4 * N * kTcW * 8;
  static constexpr size_t bytes = off_bar + 64;
  static constexpr size_t smem = bytes < 80 * 1024 ? 80 * 1024 : bytes;
  static_assert(bytes <= 110 * 1024, "two CTAs per SM");
  static_assert(3 * 192 + 128 <= SBO2, "stage-2 core matrices of one row group must not overlap");
};

// byte offset of element (row, k) in a K-major, unswizzled operand
__device__ __forceinline__ unsigned kmaj_off(int row, int k, int lbo, int sbo) {
  return (unsigned)((row >> 3) * sbo + (k >> 3) * lbo + (row & 7) * 16 + (k & 7) * 2);
}

// real expansion of the R-point DFT matrix, entry (n = 2 k1 + eo, k = 2 n1 + ei), split
// into hi/lo BF16 and stored K-major: w = exp(-+2 pi i k1 n1 / R) taken from the length-N
// twiddle table at index stride * ((k1 n1) mod R)
template <int R, int ND, int KD, bool INV>
__device__ void build_dft_matrix(const float2* tw, int stride, unsigned char* hi, unsigned char* lo) {
  constexpr int sbo = KD / 8 * 128;
  for (int e = threadIdx.x; e < ND * KD; e += blockDim.x) {
    const int n = e / KD, k = e % KD;
    const int k1 = n >> 1, eo = n & 1, n1 = k >> 1, ei = k & 1;
    float v = 0.f;
    if (k1 < R && n1 < R) {
      const float2 w = tw[stride * ((k1 * n1) % R)];
      const float c = w.x, s = INV ? -w.y : w.y;
      v = eo == 0 ? (ei == 0 ? c : -s) : (ei == 0 ? s : c);
    }
    const unsigned h = pack_bf16x2(v, 0.f) & 0xFFFFu;
    const unsigned l = pack_bf16x2(v - __uint_as_float(h << 16), 0.f) & 0xFFFFu;
    const unsigned off = kmaj_off(n, k, 128, sbo);
    *reinterpret_cast<unsigned short*>(hi + off) = (unsigned short)h;
    *reinterpret_cast<unsigned short*>(lo + off) = (unsigned short)l;
  }
}

// issue D = A_hi B_hi + A_lo B_hi + A_hi B_lo over `mblocks` 128-row blocks (one thread)
template <int KD, int ND, int LBOA, int SBOA>
__device__ __forceinline__ void issue_stage(unsigned tcol, const unsigned char* ahi, const unsigned char* alo,
                                            const unsigned char* bhi, const unsigned char* blo, int mblocks,
                                            unsigned long long* bar) {
  constexpr int sbob = KD / 8 * 128;
  constexpr unsigned idesc = umma_idesc_bf16(128, ND);
  tc_fence_after();
  for (int b = 0; b < mblocks; ++b) {
#pragma unroll
    for (int ks = 0; ks < KD / 16; ++ks) {
      const size_t ao = (size_t)b * 16 * SBOA + ks * 2 * LBOA;
      const unsigned long long dah = umma_smem_desc(ahi + ao, LBOA, SBOA), dal = umma_smem_desc(alo + ao, LBOA, SBOA);
      const unsigned long long dbh = umma_smem_desc(bhi + ks * 256, 128, sbob);
      const unsigned long long dbl = umma_smem_desc(blo + ks * 256, 128, sbob);
      const unsigned d = tcol + b * ND;
      umma_bf16(d, dah, dbh, idesc, ks > 0 ? 1u : 0u);
      umma_bf16(d, dal, dbh, idesc, 1u);
      umma_bf16(d, dah, dbl, idesc, 1u);
    }
  }
  umma_commit(bar);
}

template <int R1>
struct TcSmem {
  float2* tw;
  unsigned char *b1, *b2, *ahi, *alo;
  float2* xs;  // [k][y][4]
  unsigned long long* bar;  // [0] MMA completion, [1] t tile arrival
};

// One length-N transform of the tile's 4 K lines (direction INV) from xs: stage-1 GEMM,
// twiddle, stage-2 GEMM; the result goes back to xs (forward) or to global memory
// (inverse, dst = the tile's first column of basis 0).  `pre_issue` runs on thread 0
// after the stage-1 operand is in place (xs is free from then on in the inverse).
// Returns false if an MMA wait ran out.
template <int R1, bool INV, typename PreIssue>
__device__ __forceinline__ bool tc_transform(const TcSmem<R1>& sm, unsigned tbase, unsigned& ph, int K, float2* dst,
                                             long long NN, int nz, PreIssue pre_issue) {
  using CT = ColTc<R1>;
  constexpr int N = CT::N, KD1 = CT::KD1, ND1 = CT::ND1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3, eb = warp >> 2;
  const unsigned lane_addr = (unsigned)(q * 32) << 16;
  const int M1 = 64 * K, M2 = 4 * K * R1;
  const int mb1 = (M1 + 127) / 128, mb2 = (M2 + 127) / 128;
  // ---- stage-1 operand: row m = (k, n2, zz) holds x[16 n1 + n2], n1 < R1
  if (tid < M1) {
    const int k = tid >> 6, n2 = (tid >> 2) & 15, zz = tid & 3;
    const float2* src = sm.xs + (k * N + n2) * kTcW + zz;
#pragma unroll
    for (int c = 0; c < KD1 / 8; ++c) {
      float2 v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] = (4 * c + i < R1) ? src[(4 * c + i) * 16 * kTcW] : make_float2(0.f, 0.f);
      uint4 h, l;
      split_bf16(v[0], h.x, l.x);
      split_bf16(v[1], h.y, l.y);
      split_bf16(v[2], h.z, l.z);
      split_bf16(v[3], h.w, l.w);
      const unsigned off = kmaj_off(tid, 8 * c, CT::LBO1, CT::SBO1);
      *reinterpret_cast<uint4*>(sm.ahi + off) = h;
      *reinterpret_cast<uint4*>(sm.alo + off) = l;
    }
  }
  fence_proxy_async_smem();
  __syncthreads();
  if (tid == 0) {
    pre_issue();
    issue_stage<KD1, ND1, CT::LBO1, CT::SBO1>(tbase, sm.ahi, sm.alo, sm.b1 + (INV ? 2 : 0) * CT::kMatB1,
                                              sm.b1 + (INV ? 3 : 1) * CT::kMatB1, mb1, &sm.bar[0]);
  }
  if (__syncthreads_or(!mbar_wait_bounded(&sm.bar[0], ph))) return false;
  ph ^= 1;
  tc_fence_after();
  // ---- stage-1 result, twiddle, stage-2 operand: row m' = (k, k1, zz), column n2
  if (eb < mb1) {
    float d[ND1];
    if constexpr (ND1 == 16)
      tmem_ld16(tbase + lane_addr + eb * ND1, d);
    else
      tmem_ld32(tbase + lane_addr + eb * ND1, d);
    const int m = eb * 128 + q * 32 + lane;
    if (m < M1) {
      const int k = m >> 6, n2 = (m >> 2) & 15, zz = m & 3;
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) {
        float2 y = make_float2(d[2 * k1], d[2 * k1 + 1]);
        if (k1 > 0) y = twiddle_mul<INV>(y, sm.tw[n2 * k1]);
        unsigned h, l;
        split_bf16(y, h, l);
        const unsigned off = kmaj_off((k * R1 + k1) * kTcW + zz, 2 * n2, CT::LBO2, CT::SBO2);
        *reinterpret_cast<unsigned*>(sm.ahi + off) = h;
        *reinterpret_cast<unsigned*>(sm.alo + off) = l;
      }
    }
  }
  tc_fence_before();
  fence_proxy_async_smem();
  __syncthreads();
  if (tid == 0)
    issue_stage<32, 32, CT::LBO2, CT::SBO2>(tbase + 64, sm.ahi, sm.alo, sm.b2 + (INV ? 2 : 0) * CT::kMatB2,
                                            sm.b2 + (INV ? 3 : 1) * CT::kMatB2, mb2, &sm.bar[0]);
  if (__syncthreads_or(!mbar_wait_bounded(&sm.bar[0], ph))) return false;
  ph ^= 1;
  tc_fence_after();
  // ---- stage-2 result X[k1 + R1 k2]
  if (eb < mb2) {
    float d[32];
    tmem_ld32(tbase + 64 + lane_addr + eb * 32, d);
    const int m = eb * 128 + q * 32 + lane;
    if (m < M2) {
      const int zz = m & 3, kk = (m >> 2) / R1, k1 = (m >> 2) - kk * R1;
      if (INV) {
        float2* o = dst + kk * NN + (long long)k1 * nz + zz;
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) o[(long long)(R1 * k2) * nz] = make_float2(d[2 * k2], d[2 * k2 + 1]);
      } else {
        float2* o = sm.xs + (kk * N + k1) * kTcW + zz;
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) o[R1 * k2 * kTcW] = make_float2(d[2 * k2], d[2 * k2 + 1]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  return true;
}

template <int R1>
__global__ void __launch_bounds__(kTcThreads, 2)
    k_col_tc(Geom g, const __grid_constant__ CUtensorMap tm_t, const float2* __restrict__ tw_g,
             const float* __restrict__ psi, float2* t, int ntz, int ntiles) {
  using CT = ColTc<R1>;
  constexpr int N = CT::N, KD1 = CT::KD1, ND1 = CT::ND1;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TcSmem<R1> sm;
  sm.tw = reinterpret_cast<float2*>(smem_raw);
  sm.b1 = smem_raw + CT::off_b1;
  sm.b2 = smem_raw + CT::off_b2;
  sm.ahi = smem_raw + CT::off_ahi;
  sm.alo = smem_raw + CT::off_alo;
  sm.xs = reinterpret_cast<float2*>(smem_raw + CT::off_x);
  sm.bar = reinterpret_cast<unsigned long long*>(smem_raw + CT::off_bar);
  unsigned* tslot = reinterpret_cast<unsigned*>(smem_raw + CT::off_bar + 16);

  const int tid = threadIdx.x, warp = tid >> 5;
  const int K = g.K, nz = g.nz;
  const long long NN = (long long)N * nz;
  const unsigned bytes_t = (unsigned)(K * N * kTcW * 8);

  if (warp == 0) tmem_alloc(tslot, kTcTmemCols);
  if (tid == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    fence_mbar_init();
  }
  for (int i = tid; i < N; i += kTcThreads) sm.tw[i] = tw_g[i];
  __syncthreads();
  if (tid == 0 && blockIdx.x < ntiles) {  // first tile
    const int sc = blockIdx.x / ntz, z0 = (blockIdx.x - sc * ntz) * kTcW;
    mbar_expect_tx(&sm.bar[1], bytes_t);
    tma_load_3d(sm.xs, &tm_t, &sm.bar[1], z0, 0, sc * K);
  }
  build_dft_matrix<R1, ND1, KD1, false>(sm.tw, 16, sm.b1, sm.b1 + CT::kMatB1);
  build_dft_matrix<R1, ND1, KD1, true>(sm.tw, 16, sm.b1 + 2 * CT::kMatB1, sm.b1 + 3 * CT::kMatB1);
  build_dft_matrix<16, 32, 32, false>(sm.tw, R1, sm.b2, sm.b2 + CT::kMatB2);
  build_dft_matrix<16, 32, 32, true>(sm.tw, R1, sm.b2 + 2 * CT::kMatB2, sm.b2 + 3 * CT::kMatB2);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tbase = *tslot;
  unsigned ph = 0, pt = 0;
  int failed = 0;  // 1: a tile-copy wait ran out, 2: an MMA wait ran out
  bool t_pending = blockIdx.x < ntiles;

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int nxt = tile + gridDim.x;
    const int sc = tile / ntz, z0 = (tile - sc * ntz) * kTcW;
    if (__syncthreads_or(!mbar_wait_bounded(&sm.bar[1], pt))) {
      failed = 1;
      break;
    }
    pt ^= 1;
    t_pending = false;
    if (!tc_transform<R1, false>(sm, tbase, ph, K, nullptr, NN, nz, [] {})) {
      failed = 2;
      break;
    }
    // ---- space-time kernel at (ky, z0 .. z0 + 3) across the K basis values
    for (int ky = tid; ky < N; ky += kTcThreads) {
      float2 v[4][4], u[4][4];
#pragma unroll
      for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          v[l][c] = (l < K) ? sm.xs[(l * N + ky) * kTcW + c] : make_float2(0.f, 0.f);
          u[l][c] = make_float2(0.f, 0.f);
        }
      int pp = 0;
#pragma unroll
      for (int a_ = 0; a_ < 4; ++a_)
#pragma unroll
        for (int b_ = a_; b_ < 4; ++b_)
          if (b_ < K) {
            const float4 q4 = __ldg(reinterpret_cast<const float4*>(psi + (long long)pp * NN + (long long)ky * nz + z0));
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
          for (int c = 0; c < 4; ++c) sm.xs[(l * N + ky) * kTcW + c] = u[l][c];
    }
    __syncthreads();
    // inverse; once its stage-1 operand is built, xs takes the next tile's t block
    float2* dst = t + (long long)sc * K * NN + z0;
    auto prefetch = [&] {
      if (nxt < ntiles) {
        const int sn = nxt / ntz, zn = (nxt - sn * ntz) * kTcW;
        fence_proxy_async_smem();
        mbar_expect_tx(&sm.bar[1], bytes_t);
        tma_load_3d(sm.xs, &tm_t, &sm.bar[1], zn, 0, sn * K);
      }
    };
    t_pending = nxt < ntiles;
    if (!tc_transform<R1, true>(sm, tbase, ph, K, dst, NN, nz, prefetch)) {
      failed = 2;
      break;
    }
  }
  if (failed && tid == 0) {  // record, then give the MMAs and copies in flight one more bounded wait
    if (g.err) atomicExch(g.err, 1);
    if (failed == 2) mbar_wait_bounded(&sm.bar[0], ph);
    if (t_pending) mbar_wait_bounded(&sm.bar[1], pt);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, kTcTmemCols);
  }
}

template <int R1>
cudaError_t col_tc_go(const Geom& g, const float2* tw, const float* psi, float2* t, cudaStream_t st) {
  using CT = ColTc<R1>;
  TmaEncodeFn enc = tma_encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap tm_t;
  const cuuint64_t dt[3] = {(cuuint64_t)g.nz, (cuuint64_t)CT::N, (cuuint64_t)g.S * g.C * g.K};
  const cuuint64_t st_t[2] = {(cuuint64_t)g.nz * 8, (cuuint64_t)CT::N * g.nz * 8};
  const cuuint32_t bt[3] = {(cuuint32_t)kTcW, (cuuint32_t)CT::N, (cuuint32_t)g.K};
  const cuuint32_t es[3] = {1, 1, 1};
  if (enc(&tm_t, CU_TENSOR_MAP_DATA_TYPE_INT64, 3, t, dt, st_t, bt, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorNotSupported;
  int nsm = 0;
  {
    cudaError_t e = smem_optin((const void*)k_col_tc<R1>, (int)CT::smem);
    if (e == cudaSuccess) e = sm_count(&nsm);
    if (e != cudaSuccess) return e;
  }
  const int ntz = g.nz / kTcW;
  const long long ntiles = (long long)g.S * g.C * ntz;
  if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (ntiles == 0) return cudaSuccess;
  const int grid = (int)std::min<long long>(ntiles, 2LL * nsm);
  k_col_tc<R1><<<grid, kTcThreads, CT::smem, st>>>(g, tm_t, tw, psi, t, ntz, (int)ntiles);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_col_normal_tc(const Geom& g, const float2* tw_y, const float* psi, float2* t, cudaStream_t st) {
  if (g.K > 4 || g.nz % kTcW != 0) return cudaErrorNotSupported;
  switch (g.ny) {
    case 48: return col_tc_go<3>(g, tw_y, psi, t, st);
    case 64: return col_tc_go<4>(g, tw_y, psi, t, st);
    case 96: return col_tc_go<6>(g, tw_y, psi, t, st);
    case 128: return col_tc_go<8>(g, tw_y, psi, t, st);
    case 160: return col_tc_go<10>(g, tw_y, psi, t, st);
    case 192: return col_tc_go<12>(g, tw_y, psi, t, st);
    case 240: return col_tc_go<15>(g, tw_y, psi, t, st);
    case 256: return col_tc_go<16>(g, tw_y, psi, t, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace t2sh
