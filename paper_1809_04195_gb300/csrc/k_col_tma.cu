// Column pass of the normal operator (DFT_y, Psi, IDFT_y) with its tiles moved by the
// Tensor Memory Accelerator.  Persistent CTAs walk the (slice, coil, 8-column tile)
// list; for each tile one thread issues two tensor-map box copies that complete on
// mbarriers: the K x ny x 8 block of the intermediate t and the (Psi entries) x ny x 8
// block of Psi.  The next tile's t block is requested as soon as the forward stage A has read the
// current one.  Once Psi is applied, its block serves as the destination of the inverse
// stage's transposed lines, so that stage needs no barrier between its reads of the
// exchange lines and its writes; the next tile's Psi block is requested right after that
// tile's first wait, which every thread reaches only after reading the scratch.  Five
// block-wide barriers per tile.  Results go straight from registers to global memory.
//
// Transform layout (N = P R1 with P = 16, or P = 20 for the 260-point lines of Table I):
// thread (w, j < P) of basis line k holds column w's x[j + P q]; forward [R1, P] and
// inverse [P, R1] two-stage transforms as in the size-specialised kernels.  A half-warp
// spans the W columns x 16 / W consecutive j of one basis line, the exchange lines are
// padded to a stride = 16 / W (mod 16) float2 and the in-line layouts use odd strides, so
// the 16 lanes of a half-warp address 16 different 8-byte bank pairs in every stage.  A column longer
// than a tensor-map box (256 rows) is copied as two halves by a 4D map whose two middle
// dimensions split y, landing in the same [k][y][w] layout.  Requires nz % W == 0, K <= 4,
// ny = N <= 256 or N = 260.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "t2sh_device.cuh"

namespace t2sh {

template <int N, int W>
struct ColTma {
  static constexpr int P = N % 16 == 0 ? 16 : 20;  // stage-A threads per line = stage-B radix
  static constexpr int R1 = N / P;
  static_assert(P * R1 == N, "N = 16 R1 or 20 R1");
  static constexpr int SF = (R1 % 2) ? R1 : R1 + 1;  // forward in-line stride (odd)
  static constexpr int SI = P + 1;                   // inverse in-line stride (odd)
  static constexpr int LINE = (P * SF > R1 * SI) ? P * SF : R1 * SI;
  static constexpr int THREADS = 4 * W * P;
  static constexpr int MINB = 8 / W;     // CTAs per SM the shared memory allows
  static constexpr bool Y4D = N > 256;  // y split over two box dimensions
  // a half-warp holds W columns x JPH = 16 / W consecutive j; the exchange line stride
  // LS = JPH (mod 16) with SF = 1 (mod 16) spreads its accesses over all banks
  static constexpr int JPH = 16 / W;
  static constexpr int LS = LINE + ((16 + JPH - LINE % 16) % 16);
  static constexpr size_t off_ex = ((size_t)N * 8 + 127) / 128 * 128;                       // bytes
  static constexpr size_t off_t = (off_ex + (size_t)4 * W * LS * 8 + 127) / 128 * 128;
  static constexpr size_t off_psi = off_t + (size_t)4 * N * W * 8;
  // the Psi block also holds the inverse stage's transposed lines once Psi is applied
  static constexpr size_t ex_bytes = (size_t)4 * W * LS * 8;
  // np = K (K + 1) / 2 stored entries of Psi per point
  __host__ __device__ static size_t psi_region(int np) {
    const size_t pb = ((size_t)np * N * W * 4 + 127) / 128 * 128;
    return pb > ex_bytes ? pb : (ex_bytes + 127) / 128 * 128;
  }
  __host__ __device__ static size_t smem(int np) { return off_psi + psi_region(np) + 64; }
};

// the tile's rows row0 .. row0 + box - 1 of columns z0 .. z0 + W - 1 (3D map, or 4D with y
// split in halves)
template <bool Y4D>
__device__ __forceinline__ void tma_tile(void* dst, const CUtensorMap* m, unsigned long long* bar, int z0, int row0) {
  if constexpr (Y4D)
    tma_load_4d(dst, m, bar, z0, 0, 0, row0);
  else
    tma_load_3d(dst, m, bar, z0, 0, row0);
}

template <int N, int W>
__global__ void __launch_bounds__(ColTma<N, W>::THREADS, ColTma<N, W>::MINB) k_col_tma(Geom g, const __grid_constant__ CUtensorMap tm_t,
                                                   const __grid_constant__ CUtensorMap tm_psi,
                                                   const float2* __restrict__ tw_g, float2* t, int ntz, int ntiles) {
  using CT = ColTma<N, W>;
  constexpr int P1 = CT::P, R1 = CT::R1, SF = CT::SF, SI = CT::SI, LS = CT::LS;
  constexpr int WL = W == 8 ? 3 : 2;  // log2 W
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* ex = reinterpret_cast<float2*>(smem_raw + CT::off_ex);   // [k][w][LS]
  float2* st = reinterpret_cast<float2*>(smem_raw + CT::off_t);    // [k][y][W] (TMA box)
  float* ps = reinterpret_cast<float*>(smem_raw + CT::off_psi);    // [p][y][W] (TMA box)
  const int nz = g.nz, NN = N * nz, K = g.K, P = g.P;
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem_raw + CT::off_psi + CT::psi_region(P));
  constexpr int JPH = CT::JPH;
  const int w = threadIdx.x & (W - 1), jl = (threadIdx.x >> WL) & (JPH - 1), k = (threadIdx.x >> 4) & 3,
            j = JPH * (threadIdx.x >> 6) + jl;
  const bool live = k < K;
  const unsigned bytes_t = (unsigned)(K * N * W * 8), bytes_p = (unsigned)(P * N * W * 4);
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
  __syncthreads();
  int tile = blockIdx.x;
  if (threadIdx.x == 0 && tile < ntiles) {
    const int sc = tile / ntz, z0 = (tile - sc * ntz) * W;
    mbar_expect_tx(&bars[0], bytes_t);
    tma_tile<CT::Y4D>(st, &tm_t, &bars[0], z0, sc * K);
    mbar_expect_tx(&bars[1], bytes_p);
    tma_tile<CT::Y4D>(ps, &tm_psi, &bars[1], z0, 0);
  }
  unsigned ph_t = 0, ph_p = 0;
  float2* exl = ex + (k * W + w) * LS;
  float2* oxl = reinterpret_cast<float2*>(ps) + (k * W + w) * LS;  // inverse lines, in the Psi block
  bool psi_issued = true;  // the first tile's Psi block was requested above
  for (; tile < ntiles; tile += gridDim.x) {
    const int nxt = tile + gridDim.x;
    const int sc = tile / ntz, z0 = (tile - sc * ntz) * W;
    bool ok = mbar_wait_bounded(&bars[0], ph_t);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {  // record, then give copies in flight one more bounded wait
        if (g.err) atomicExch(g.err, 1);
        mbar_wait_bounded(&bars[0], ph_t);
        if (psi_issued) mbar_wait_bounded(&bars[1], ph_p);
      }
      return;
    }
    ph_t ^= 1;
    // every thread has left the previous tile's last stage, which read the Psi block as
    // scratch: this tile's Psi block may land there now
    if (threadIdx.x == 0 && !psi_issued) {
      fence_proxy_async_smem();
      mbar_expect_tx(&bars[1], bytes_p);
      tma_tile<CT::Y4D>(ps, &tm_psi, &bars[1], z0, 0);
    }
    psi_issued = true;
    // forward stage A: DFT_R1 of x[j + P q]
    if (live) {
      const float2* sp = st + (k * N) * W + w;
      float2 a[R1];
#pragma unroll
      for (int q = 0; q < R1; ++q) a[q] = sp[(j + P1 * q) * W];
      dft_r<R1, false>(a);
#pragma unroll
      for (int q = 0; q < R1; ++q) exl[j * SF + q] = a[q];
    }
    __syncthreads();
    if (threadIdx.x == 0 && nxt < ntiles) {  // the t block is consumed: fetch the next one
      const int sn = nxt / ntz, zn = (nxt - sn * ntz) * W;
      fence_proxy_async_smem();
      mbar_expect_tx(&bars[0], bytes_t);
      tma_tile<CT::Y4D>(st, &tm_t, &bars[0], zn, sn * K);
    }
    // forward stage B: twiddle, DFT_P -> X[j + R1 q] at [q][j]
    if (live && j < R1) {
      float2 b[P1];
#pragma unroll
      for (int q = 0; q < P1; ++q) b[q] = exl[q * SF + j];
#pragma unroll
      for (int q = 1; q < P1; ++q) b[q] = twiddle_mul<false>(b[q], tw[q * j]);
      dft_r<P1, false>(b);
#pragma unroll
      for (int q = 0; q < P1; ++q) exl[q * SF + j] = b[q];
    }
    ok = mbar_wait_bounded(&bars[1], ph_p);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        if (g.err) atomicExch(g.err, 1);
        mbar_wait_bounded(&bars[1], ph_p);
        if (nxt < ntiles) mbar_wait_bounded(&bars[0], ph_t);
      }
      return;
    }
    ph_p ^= 1;
    // space-time kernel at the points (ky, c0 .. c0 + 3) of the tile
    for (int pg = threadIdx.x; pg < (W / 4) * N; pg += blockDim.x) {
      const int c0 = (W == 8) ? (pg & 1) * 4 : 0, ky = (W == 8) ? pg >> 1 : pg;
      const int pos = (ky / R1) * SF + (ky % R1);
      float2 v[4][4], u[4][4];
#pragma unroll
      for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          v[l][c] = (l < K) ? ex[(l * W + c0 + c) * LS + pos] : make_float2(0.f, 0.f);
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
          for (int c = 0; c < 4; ++c) ex[(l * W + c0 + c) * LS + pos] = u[l][c];
    }
    __syncthreads();
    psi_issued = false;  // the Psi block is consumed; the next tile's lands after its first wait
    // inverse stage A': IDFT_P of X[j + R1 q], result to [j][r1] (stride P + 1) in the Psi
    // block, so no thread's write can overtake another's read of the exchange lines
    if (live && j < R1) {
      float2 b[P1];
#pragma unroll
      for (int q = 0; q < P1; ++q) b[q] = exl[q * SF + j];
      dft_r<P1, true>(b);
#pragma unroll
      for (int q = 0; q < P1; ++q) oxl[j * SI + q] = b[q];
    }
    __syncthreads();
    // inverse stage B': twiddle, IDFT_R1 -> y = j + P q, straight to global memory (the next
    // tile's first wait, a block-wide barrier, orders these reads before anything overwrites
    // the exchange lines or the Psi block)
    if (live) {
      float2 a[R1];
#pragma unroll
      for (int q = 0; q < R1; ++q) a[q] = twiddle_mul<true>(oxl[q * SI + j], tw[q * j]);
      dft_r<R1, true>(a);
      float2* ob = t + ((long long)sc * K + k) * NN + z0 + w;
#pragma unroll
      for (int q = 0; q < R1; ++q) ob[(long long)(j + P1 * q) * nz] = a[q];
    }
  }
}

// A^H y column pass (COL_ADJ_DATA): x[y] = IDFT_y of the projected k-space column scaled by
// gsign (-1)^(ky + kz) / sqrt(ny nz), from tin to tout.  Same tiles, copies and inverse
// stages as the normal pass, without the forward transform and Psi: thread (line, j < R1)
// takes X[j + R1 q] (q < P) straight from the tile into registers, IDFT_P, transposed
// lines to the scratch block, then IDFT_R1 to global memory.  Two block-wide barriers per
// tile; the next tile's copy is requested as soon as the current one has been read.
template <int N, int W>
__global__ void __launch_bounds__(ColTma<N, W>::THREADS, ColTma<N, W>::MINB) k_col_tma_adj(Geom g, const __grid_constant__ CUtensorMap tm_in,
                                                          const float2* __restrict__ tw_g, float2* tout, int ntz,
                                                          int ntiles) {
  using CT = ColTma<N, W>;
  constexpr int P1 = CT::P, R1 = CT::R1, SI = CT::SI, LS = CT::LS;
  constexpr int WL = W == 8 ? 3 : 2;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* st = reinterpret_cast<float2*>(smem_raw + CT::off_t);                // [k][y][W] (TMA box)
  float2* ox = reinterpret_cast<float2*>(smem_raw + CT::off_psi);              // [k][w][LS] inverse lines
  const int nz = g.nz, NN = N * nz, K = g.K;
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem_raw + CT::off_psi + CT::psi_region(g.P));
  constexpr int JPH = CT::JPH;
  const int w = threadIdx.x & (W - 1), jl = (threadIdx.x >> WL) & (JPH - 1), k = (threadIdx.x >> 4) & 3,
            j = JPH * (threadIdx.x >> 6) + jl;
  const bool live = k < K;
  const unsigned bytes_t = (unsigned)(K * N * W * 8);
  const float scale = g.gsign * g.inv_sqrt_n;
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
  __syncthreads();
  int tile = blockIdx.x;
  if (threadIdx.x == 0 && tile < ntiles) {
    const int sc = tile / ntz, z0 = (tile - sc * ntz) * W;
    mbar_expect_tx(&bars[0], bytes_t);
    tma_tile<CT::Y4D>(st, &tm_in, &bars[0], z0, sc * K);
  }
  unsigned ph_t = 0;
  float2* oxl = ox + (k * W + w) * LS;
  for (; tile < ntiles; tile += gridDim.x) {
    const int nxt = tile + gridDim.x;
    const int sc = tile / ntz, z0 = (tile - sc * ntz) * W;
    const bool ok = mbar_wait_bounded(&bars[0], ph_t);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {  // record, then give the copy in flight one more bounded wait
        if (g.err) atomicExch(g.err, 1);
        mbar_wait_bounded(&bars[0], ph_t);
      }
      return;
    }
    ph_t ^= 1;
    // IDFT_P over q of the scaled X[j + R1 q], result to [j][r1] (stride P + 1)
    if (live && j < R1) {
      float2 b[P1];
      const float2* sp = st + (k * N + j) * W + w;
#pragma unroll
      for (int q = 0; q < P1; ++q) b[q] = cscale(sp[R1 * q * W], scale * parity_sign(j + R1 * q + z0 + w));
      dft_r<P1, true>(b);
#pragma unroll
      for (int q = 0; q < P1; ++q) oxl[j * SI + q] = b[q];
    }
    __syncthreads();
    if (threadIdx.x == 0 && nxt < ntiles) {  // the tile is read: fetch the next one
      const int sn = nxt / ntz, zn = (nxt - sn * ntz) * W;
      fence_proxy_async_smem();
      mbar_expect_tx(&bars[0], bytes_t);
      tma_tile<CT::Y4D>(st, &tm_in, &bars[0], zn, sn * K);
    }
    // twiddle, IDFT_R1 -> y = j + P q (the next tile's first wait orders these reads
    // before the scratch is written again)
    if (live) {
      float2 a[R1];
#pragma unroll
      for (int q = 0; q < R1; ++q) a[q] = twiddle_mul<true>(oxl[q * SI + j], tw[q * j]);
      dft_r<R1, true>(a);
      float2* ob = tout + ((long long)sc * K + k) * NN + z0 + w;
#pragma unroll
      for (int q = 0; q < R1; ++q) ob[(long long)(j + P1 * q) * nz] = a[q];
    }
  }
}

// Self-test of the bounded-wait path: one thread waits on an mbarrier that nothing
// completes, with a limit of limit_ns, and records the timeout in the error flag exactly
// as the tile kernels do.  Nothing is in flight, so the kernel simply returns.
__global__ void k_wait_selftest(int* err, unsigned long long limit_ns) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, limit_ns) && err) atomicExch(err, 1);
}

cudaError_t launch_wait_selftest(int* err, unsigned long long limit_ns, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(err, limit_ns);
  return cudaGetLastError();
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda)
TmaEncodeFn tma_encode_fn() {
  static TmaEncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<TmaEncodeFn>(p);
    cudaGetLastError();
  });
  return fn;
}

namespace {
// Tensor map of a [rows][N][nz] array of esize-byte elements with W x N x box_rows boxes;
// for N > 256 the y dimension is split into two halves of N / 2 (4D map, same box layout)
template <int N, int W>
bool encode_columns(TmaEncodeFn enc, CUtensorMap* m, CUtensorMapDataType type, const void* base, int nz,
                    long long rows, int esize, int box_rows) {
  const cuuint32_t es[4] = {1, 1, 1, 1};
  if constexpr (N > 256) {
    static_assert(N % 2 == 0 && N / 2 <= 256, "two boxes per column");
    const cuuint64_t d[4] = {(cuuint64_t)nz, (cuuint64_t)(N / 2), 2, (cuuint64_t)rows};
    const cuuint64_t s[3] = {(cuuint64_t)nz * esize, (cuuint64_t)(N / 2) * nz * esize, (cuuint64_t)N * nz * esize};
    const cuuint32_t b[4] = {(cuuint32_t)W, (cuuint32_t)(N / 2), 2, (cuuint32_t)box_rows};
    return enc(m, type, 4, const_cast<void*>(base), d, s, b, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  } else {
    const cuuint64_t d[3] = {(cuuint64_t)nz, (cuuint64_t)N, (cuuint64_t)rows};
    const cuuint64_t s[2] = {(cuuint64_t)nz * esize, (cuuint64_t)N * nz * esize};
    const cuuint32_t b[3] = {(cuuint32_t)W, (cuuint32_t)N, (cuuint32_t)box_rows};
    return enc(m, type, 3, const_cast<void*>(base), d, s, b, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
}

template <int N, int W>
cudaError_t col_tma_go(const Geom& g, const float2* tw, const float* psi, float2* t, cudaStream_t st) {
  using CT = ColTma<N, W>;
  TmaEncodeFn enc = tma_encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap tm_t, tm_psi;
  if (!encode_columns<N, W>(enc, &tm_t, CU_TENSOR_MAP_DATA_TYPE_INT64, t, g.nz, (long long)g.S * g.C * g.K, 8, g.K) ||
      !encode_columns<N, W>(enc, &tm_psi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, psi, g.nz, g.P, 4, g.P))
    return cudaErrorNotSupported;
  const size_t sm = CT::smem(g.P);
  int nsm = 0;
  {
    cudaError_t e = smem_optin((const void*)k_col_tma<N, W>, (int)CT::smem(10));
    if (e == cudaSuccess) e = sm_count(&nsm);
    if (e != cudaSuccess) return e;
  }
  const int ntz = g.nz / W;
  const long long ntiles = (long long)g.S * g.C * ntz;
  if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  const int grid = (int)std::min<long long>(ntiles, (long long)nsm * CT::MINB);
  k_col_tma<N, W><<<grid, CT::THREADS, sm, st>>>(g, tm_t, tm_psi, tw, t, ntz, (int)ntiles);
  return cudaGetLastError();
}

template <int W>
cudaError_t col_tma_w(const Geom& g, const float2* tw_y, const float* psi, float2* t, cudaStream_t st) {
  if (g.K > 4 || g.nz % W != 0) return cudaErrorNotSupported;
  switch (g.ny) {
    case 48: return col_tma_go<48, W>(g, tw_y, psi, t, st);
    case 64: return col_tma_go<64, W>(g, tw_y, psi, t, st);
    case 96: return col_tma_go<96, W>(g, tw_y, psi, t, st);
    case 128: return col_tma_go<128, W>(g, tw_y, psi, t, st);
    case 160: return col_tma_go<160, W>(g, tw_y, psi, t, st);
    case 192: return col_tma_go<192, W>(g, tw_y, psi, t, st);
    case 240: return col_tma_go<240, W>(g, tw_y, psi, t, st);
    case 256: return col_tma_go<256, W>(g, tw_y, psi, t, st);
    case 260: return col_tma_go<260, W>(g, tw_y, psi, t, st);
    default: return cudaErrorNotSupported;
  }
}
template <int N, int W>
cudaError_t col_tma_adj_go(const Geom& g, const float2* tw, const float2* tin, float2* tout, cudaStream_t st) {
  using CT = ColTma<N, W>;
  TmaEncodeFn enc = tma_encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap tm_in;
  if (!encode_columns<N, W>(enc, &tm_in, CU_TENSOR_MAP_DATA_TYPE_INT64, tin, g.nz, (long long)g.S * g.C * g.K, 8, g.K))
    return cudaErrorNotSupported;
  const size_t sm = CT::smem(g.P);
  int nsm = 0;
  {
    cudaError_t e = smem_optin((const void*)k_col_tma_adj<N, W>, (int)CT::smem(10));
    if (e == cudaSuccess) e = sm_count(&nsm);
    if (e != cudaSuccess) return e;
  }
  const int ntz = g.nz / W;
  const long long ntiles = (long long)g.S * g.C * ntz;
  if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (ntiles == 0) return cudaSuccess;
  const int grid = (int)std::min<long long>(ntiles, (long long)nsm * CT::MINB);
  k_col_tma_adj<N, W><<<grid, CT::THREADS, sm, st>>>(g, tm_in, tw, tout, ntz, (int)ntiles);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_col_adj_tma(const Geom& g, const float2* tw_y, const float2* tin, float2* tout, cudaStream_t st) {
  constexpr int W = 8;
  if (g.K > 4 || g.nz % W != 0) return cudaErrorNotSupported;  // in place is fine: a tile is read whole before it is written
  switch (g.ny) {
    case 48: return col_tma_adj_go<48, W>(g, tw_y, tin, tout, st);
    case 64: return col_tma_adj_go<64, W>(g, tw_y, tin, tout, st);
    case 96: return col_tma_adj_go<96, W>(g, tw_y, tin, tout, st);
    case 128: return col_tma_adj_go<128, W>(g, tw_y, tin, tout, st);
    case 160: return col_tma_adj_go<160, W>(g, tw_y, tin, tout, st);
    case 192: return col_tma_adj_go<192, W>(g, tw_y, tin, tout, st);
    case 240: return col_tma_adj_go<240, W>(g, tw_y, tin, tout, st);
    case 256: return col_tma_adj_go<256, W>(g, tw_y, tin, tout, st);
    case 260: return col_tma_adj_go<260, W>(g, tw_y, tin, tout, st);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t launch_col_normal_tma(const Geom& g, const float2* tw_y, const float* psi, float2* t, cudaStream_t st) {
  return g.colvar == 4 ? col_tma_w<4>(g, tw_y, psi, t, st) : col_tma_w<8>(g, tw_y, psi, t, st);
}

}  // namespace t2sh
