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
// all K <= 4 basis images, i.e. L = 4 K lines of length N.  Per tile: forward stage 1
// (rows l x n2 of the A operand, read from global memory), forward stage 2, Psi applied
// in shared memory at every (ky, z) across the K basis values, inverse stages 1 and 2
// (conjugate matrices and twiddles), and the result goes from TMEM straight to global
// memory.  Thread 0 issues the MMAs; completion arrives on an mbarrier whose waits are
// bounded by the global timer.  Each CTA allocates 128 TMEM columns and at least 80 KB of
// shared memory, so at most two such CTAs share an SM and TMEM is never oversubscribed.
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
  static constexpr int SBO1 = KD1 / 8 * 128;            // bytes between 8-row groups, stage 1
  static constexpr int SBO2 = 32 / 8 * 128;             // stage 2 (K = 32 reals)
  static constexpr int kRows = 256;                     // A rows (>= 64 K and >= 4 K R1 rounded)
  static constexpr int kMatB1 = ND1 * KD1 * 2;          // bytes of one stage-1 matrix
  static constexpr int kMatB2 = 32 * 32 * 2;
  // shared-memory map (bytes)
  static constexpr size_t off_b1 = ((size_t)N * 8 + 1023) / 1024 * 1024;  // after twiddles
  static constexpr size_t off_b2 = off_b1 + 4 * kMatB1;                   // fwd hi, fwd lo, inv hi, inv lo
  static constexpr size_t off_ahi = off_b2 + 4 * kMatB2;
  static constexpr size_t off_alo = off_ahi + (size_t)kRows * 64;
  static constexpr size_t off_x = off_alo + (size_t)kRows * 64;
  static constexpr size_t off_bar = off_x + (size_t)4 * N * kTcW * 8;
  static constexpr size_t bytes = off_bar + 64;
  static constexpr size_t smem = bytes < 80 * 1024 ? 80 * 1024 : bytes;
  static_assert(bytes <= 110 * 1024, "two CTAs per SM");
};

// byte offset of element (row, k) in a K-major, unswizzled operand with 8-row groups sbo apart
__device__ __forceinline__ unsigned kmaj_off(int row, int k, int sbo) {
  return (unsigned)((row >> 3) * sbo + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
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
    const unsigned off = kmaj_off(n, k, sbo);
    *reinterpret_cast<unsigned short*>(hi + off) = (unsigned short)h;
    *reinterpret_cast<unsigned short*>(lo + off) = (unsigned short)l;
  }
}

// issue D = A_hi B_hi + A_lo B_hi + A_hi B_lo over `mblocks` 128-row blocks (thread 0)
template <int KD, int ND>
__device__ __forceinline__ void issue_stage(unsigned tcol, const unsigned char* ahi, const unsigned char* alo,
                                            const unsigned char* bhi, const unsigned char* blo, int mblocks,
                                            unsigned long long* bar) {
  constexpr int sbo = KD / 8 * 128;
  constexpr unsigned idesc = umma_idesc_bf16(128, ND);
  tc_fence_after();
  for (int b = 0; b < mblocks; ++b) {
#pragma unroll
    for (int ks = 0; ks < KD / 16; ++ks) {
      const size_t ao = (size_t)b * 16 * sbo + ks * 256;
      const unsigned long long dah = umma_smem_desc(ahi + ao, 128, sbo), dal = umma_smem_desc(alo + ao, 128, sbo);
      const unsigned long long dbh = umma_smem_desc(bhi + ks * 256, 128, sbo);
      const unsigned long long dbl = umma_smem_desc(blo + ks * 256, 128, sbo);
      const unsigned d = tcol + b * ND;
      umma_bf16(d, dah, dbh, idesc, ks > 0 ? 1u : 0u);
      umma_bf16(d, dal, dbh, idesc, 1u);
      umma_bf16(d, dah, dbl, idesc, 1u);
    }
  }
  umma_commit(bar);
}

template <int R1>
__global__ void __launch_bounds__(kTcThreads, 2)
    k_col_tc(Geom g, const float2* __restrict__ tw_g, const float* __restrict__ psi, float2* t, int ntz, int ntiles) {
  using CT = ColTc<R1>;
  constexpr int N = CT::N, KD1 = CT::KD1, ND1 = CT::ND1;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  unsigned char* b1 = smem_raw + CT::off_b1;
  unsigned char* b2 = smem_raw + CT::off_b2;
  unsigned char* ahi = smem_raw + CT::off_ahi;
  unsigned char* alo = smem_raw + CT::off_alo;
  float2* xs = reinterpret_cast<float2*>(smem_raw + CT::off_x);  // [k][y][4]
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + CT::off_bar);
  unsigned* tslot = reinterpret_cast<unsigned*>(smem_raw + CT::off_bar + 8);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = g.K, nz = g.nz, P = g.P;
  const long long NN = (long long)N * nz;
  const int M1 = 64 * K, M2 = 4 * K * R1;
  const int mb1 = (M1 + 127) / 128, mb2 = (M2 + 127) / 128;

  if (warp == 0) tmem_alloc(tslot, kTcTmemCols);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  for (int i = tid; i < N; i += kTcThreads) tw[i] = tw_g[i];
  __syncthreads();
  build_dft_matrix<R1, ND1, KD1, false>(tw, 16, b1, b1 + CT::kMatB1);
  build_dft_matrix<R1, ND1, KD1, true>(tw, 16, b1 + 2 * CT::kMatB1, b1 + 3 * CT::kMatB1);
  build_dft_matrix<16, 32, 32, false>(tw, R1, b2, b2 + CT::kMatB2);
  build_dft_matrix<16, 32, 32, true>(tw, R1, b2 + 2 * CT::kMatB2, b2 + 3 * CT::kMatB2);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tbase = *tslot;
  unsigned ph = 0;
  bool failed = false;

  // thread -> TMEM lane mapping of the epilogues: warp quarter q reads lanes 32 q .. 32 q + 31
  const int q = warp & 3, eb = warp >> 2;  // eb: 128-row block handled by this warp
  const unsigned lane_addr = (unsigned)(q * 32) << 16;

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int sc = tile / ntz, z0 = (tile - sc * ntz) * kTcW;
    float2* tg = t + (long long)sc * K * NN + z0;
#pragma unroll 1
    for (int dir = 0; dir < 2; ++dir) {  // 0: forward DFT_y, 1: inverse
      const bool inv = dir == 1;
      // ---- stage-1 operand: row m = (k, n2, zz) holds x[16 n1 + n2], n1 < R1
      if (tid < M1) {
        const int k = tid >> 6, n2 = (tid >> 2) & 15, zz = tid & 3;
        float2 v[16];
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) {
          v[n1] = make_float2(0.f, 0.f);
          if (n1 < R1) {
            const int y = 16 * n1 + n2;
            v[n1] = inv ? xs[(k * N + y) * kTcW + zz] : tg[k * NN + (long long)y * nz + zz];
          }
        }
#pragma unroll
        for (int c = 0; c < KD1 / 8; ++c) {
          uint4 h, l;
          split_bf16(v[4 * c + 0], h.x, l.x);
          split_bf16(v[4 * c + 1], h.y, l.y);
          split_bf16(v[4 * c + 2], h.z, l.z);
          split_bf16(v[4 * c + 3], h.w, l.w);
          const unsigned off = kmaj_off(tid, 8 * c, CT::SBO1);
          *reinterpret_cast<uint4*>(ahi + off) = h;
          *reinterpret_cast<uint4*>(alo + off) = l;
        }
      }
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0)
        issue_stage<KD1, ND1>(tbase, ahi, alo, b1 + (inv ? 2 : 0) * CT::kMatB1, b1 + (inv ? 3 : 1) * CT::kMatB1, mb1,
                              bar);
      if (__syncthreads_or(!mbar_wait_bounded(bar, ph))) {
        failed = true;
        break;
      }
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
            if (k1 > 0 && n2 > 0) y = inv ? twiddle_mul<true>(y, tw[n2 * k1]) : twiddle_mul<false>(y, tw[n2 * k1]);
            unsigned h, l;
            split_bf16(y, h, l);
            const int r = (k * R1 + k1) * kTcW + zz;
            const unsigned off = kmaj_off(r, 2 * n2, CT::SBO2);
            *reinterpret_cast<unsigned*>(ahi + off) = h;
            *reinterpret_cast<unsigned*>(alo + off) = l;
          }
        }
      }
      tc_fence_before();
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0)
        issue_stage<32, 32>(tbase + 64, ahi, alo, b2 + (inv ? 2 : 0) * CT::kMatB2, b2 + (inv ? 3 : 1) * CT::kMatB2, mb2,
                            bar);
      if (__syncthreads_or(!mbar_wait_bounded(bar, ph))) {
        failed = true;
        break;
      }
      ph ^= 1;
      tc_fence_after();
      // ---- stage-2 result X[k1 + R1 k2]: to shared memory (forward) or global memory (inverse)
      if (eb < mb2) {
        float d[32];
        tmem_ld32(tbase + 64 + lane_addr + eb * 32, d);
        const int m = eb * 128 + q * 32 + lane;
        if (m < M2) {
          const int zz = m & 3, kk = (m >> 2) / R1, k1 = (m >> 2) - kk * R1;
#pragma unroll
          for (int k2 = 0; k2 < 16; ++k2) {
            const int y = k1 + R1 * k2;
            const float2 v = make_float2(d[2 * k2], d[2 * k2 + 1]);
            if (inv)
              tg[kk * NN + (long long)y * nz + zz] = v;
            else
              xs[(kk * N + y) * kTcW + zz] = v;
          }
        }
      }
      tc_fence_before();
      __syncthreads();
      if (!inv) {
        // ---- space-time kernel at (ky, z0 .. z0 + 3) across the K basis values
        for (int ky = tid; ky < N; ky += kTcThreads) {
          float2 v[4][4], u[4][4];
#pragma unroll
          for (int l = 0; l < 4; ++l)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              v[l][c] = (l < K) ? xs[(l * N + ky) * kTcW + c] : make_float2(0.f, 0.f);
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
              for (int c = 0; c < 4; ++c) xs[(l * N + ky) * kTcW + c] = u[l][c];
        }
        (void)P;
        __syncthreads();
      }
    }
    if (failed) break;
  }
  if (failed && tid == 0) {  // record, then give the MMAs in flight one more bounded wait
    if (g.err) atomicExch(g.err, 1);
    mbar_wait_bounded(bar, ph);
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
  static int nsm = 0;
  if (!nsm) {
    cudaError_t e = cudaFuncSetAttribute(k_col_tc<R1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CT::smem);
    if (e != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  }
  const int ntz = g.nz / kTcW;
  const long long ntiles = (long long)g.S * g.C * ntz;
  if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (ntiles == 0) return cudaSuccess;
  const int grid = (int)std::min<long long>(ntiles, 2LL * nsm);
  k_col_tc<R1><<<grid, kTcThreads, CT::smem, st>>>(g, tw, psi, t, ntz, (int)ntiles);
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
