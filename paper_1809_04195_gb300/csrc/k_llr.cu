// Locally-low-rank prox (Eq. 4, Sec. II.B) in one pass over the coefficient images,
// as Sec. IV.C describes: the random circular shift is folded into the gather
// indices (no shifted copy), each block is thresholded on chip and written back.
//
// Work unit = (slice, map set, band of b shifted rows); the blocks of different map sets
// are independent.  Per unit: gather the band into shared memory; per block (b x b
// pixels x K) a warp forms the K x K Gram matrix G = X^H X with shuffle reductions; one
// thread per block eigendecomposes G = V diag(lambda) V^H (cyclic Jacobi, float32 by
// default, float64 on request), sigma_i = sqrt(lambda_i), and forms
// W = V diag(max(1 - tau/sigma_i, 0)) V^H, so that X W = U max(Sigma - tau, 0) V^H
// (since X V = U Sigma); then X' = X W is written back.  The FISTA variant fuses the
// gradient step before the prox and the momentum update after it (Sec. II.A); the ADMM
// variant thresholds alpha + u and writes v and the scaled dual u + alpha - v.
//
// One unit per CTA.  (A persistent schedule with two band buffers, one warp
// thresholding unit i while the others gather unit i+1, measured slower at the knee
// shape: its two CTAs per SM hide less memory latency than three single-buffer CTAs.)
#include <algorithm>

#include "t2sh_device.cuh"

namespace t2sh {

enum { LLR_PROX = 0, LLR_FISTA = 1, LLR_ADMM = 2 };

namespace {

struct LlrUnit {
  int s, m0, band, rb;
};

// Row stride (complex values) of the band in shared memory: nz rounded up to 8 (mod 16),
// so that rows r and r + 1 start in opposite halves of the 32 banks and the Gram phase's
// reads of four rows x 8 columns per warp take the minimum two wavefronts.
__host__ __device__ constexpr int llr_ld(int nz) { return nz + (24 - nz % 16) % 16; }

// Per-block strides of the Gram matrices (floats) and threshold weights (complex): one
// more than KC * KC, so that the blocks a warp touches at once (the eigen-step threads,
// and the eight blocks under a warp's 64 pixels in the apply step) fall in different banks.
template <int KC> constexpr int kGramStride = KC * KC + 1;
template <int KC> constexpr int kWStride = KC * KC + 1;

__device__ __forceinline__ LlrUnit llr_unit(const Geom& g, int b, int unit) {
  const int nbands = (g.ny + b - 1) / b;
  LlrUnit un;
  un.band = unit % nbands;
  const int sm = unit / nbands;
  un.m0 = sm % g.M;
  un.s = sm / g.M;
  un.rb = min(b, g.ny - un.band * b);
  return un;
}

// Rows of the band as stored in gs are walked by P = nth / H groups of H = nz / 2 threads,
// one pixel pair (a float4) per thread and row, so that the column-dependent quantities
// of a thread are formed once and a row step is an add and a conditional subtract
// (nz <= 512 keeps H <= 256 and P >= 1).  y of band row r is the shifted image row.
struct LlrCols {
  int tid, H, P, lp, c2;  // thread in the phase, pixel pairs per row, rows per pass, first row, pair
  bool active;
};
__device__ __forceinline__ LlrCols llr_cols(int nz, int t0, int nth) {
  LlrCols c;
  c.tid = (int)threadIdx.x - t0;
  c.H = nz >> 1;
  c.P = nth / c.H;
  c.lp = c.tid / c.H;
  c.c2 = c.tid - c.lp * c.H;
  c.active = c.tid >= 0 && c.lp < c.P;
  return c;
}
__device__ __forceinline__ int llr_row0(const Geom& g, const FistaArgs& a, const LlrUnit& un) {
  const int y = a.sy % g.ny + un.band * a.b;  // a shift may exceed a small image: reduce it first
  return y >= g.ny ? y - g.ny : y;
}

// 1. gather the band into gs [K][rb][llr_ld(nz)] (gradient step fused for FISTA), threads
// t0 .. t0 + nth - 1 of the CTA
template <int MODE>
__device__ __forceinline__ void llr_gather(const Geom& g, const FistaArgs& a, const LlrUnit& un, float2* gs,
                                           const float2* x, const float2* z, const float2* __restrict__ grad,
                                           const float2* __restrict__ aty, const float2* u, int t0, int nth) {
  const int ny = g.ny, nz = g.nz, N = ny * nz, K = g.K, rb = un.rb;
  const LlrCols c = llr_cols(nz, t0, nth);
  if (!c.active) return;
  const int y0 = llr_row0(g, a, un);
  const long long base = ((long long)un.s * g.M + un.m0) * K * (long long)N + 2 * c.c2;
  int k = 0, r = c.lp;
  while (r >= rb) {
    r -= rb;
    ++k;
  }
#pragma unroll 4
  for (int l = c.lp; l < K * rb; l += c.P) {
    int y = y0 + r;
    y -= y >= ny ? ny : 0;
    const long long gi = base + (long long)k * N + (long long)y * nz;
    float4 v;
    // global-space loads (ld.global.cg): the compiler may then batch them across iterations
    // ahead of the shared-memory stores, which generic loads could alias
    if (MODE == LLR_ADMM) {
      const float4 av = __ldcg(reinterpret_cast<const float4*>(x + gi));
      const float4 uv = __ldcg(reinterpret_cast<const float4*>(u + gi));
      v = make_float4(av.x + uv.x, av.y + uv.y, av.z + uv.z, av.w + uv.w);
    } else if (MODE == LLR_FISTA) {
      const float4 zv = __ldcg(reinterpret_cast<const float4*>(z + gi));
      const float4 gv = __ldcg(reinterpret_cast<const float4*>(grad + gi));
      const float4 av = __ldcg(reinterpret_cast<const float4*>(aty + gi));
      v = make_float4(zv.x - a.mu * (gv.x - av.x), zv.y - a.mu * (gv.y - av.y), zv.z - a.mu * (gv.z - av.z),
                      zv.w - a.mu * (gv.w - av.w));
    } else {
      v = __ldcg(reinterpret_cast<const float4*>(x + gi));
    }
    *reinterpret_cast<float4*>(gs + (long long)l * llr_ld(nz) + 2 * c.c2) = v;
    r += c.P;
    while (r >= rb) {
      r -= rb;
      ++k;
    }
  }
}

// 2. Gram matrices of the band's blocks, one warp per block, warps w0 .. w0 + nw - 1
template <int KC>
__device__ __forceinline__ void llr_gram(const Geom& g, const FistaArgs& a, const LlrUnit& un, const float2* gs,
                                         float* gram, int w0, int nw) {
  const int nz = g.nz, K = g.K, b = a.b, rb = un.rb;
  const int nbz = (nz + b - 1) / b;
  const int warp = (int)(threadIdx.x >> 5) - w0, lane = threadIdx.x & 31;
  for (int blk = warp; blk < nbz; blk += nw) {
    const int j = blk;
    const int cb = min(b, nz - j * b);
    float gr[KC][KC];  // upper: re at [k][l] (k <= l), im at [l][k] (l > k)
#pragma unroll
    for (int k = 0; k < KC; ++k)
#pragma unroll
      for (int l = 0; l < KC; ++l) gr[k][l] = 0.f;
    // lane (r0, cc) takes column cc of rows r0, r0 + RP, ... of the block
    const int RP = 32 / cb, r0 = lane / cb, cc = lane - r0 * cb;
    int zz = a.sz % nz + j * b + cc;  // j b + cc < nz, so zz < 2 nz
    zz -= zz >= nz ? nz : 0;
    for (int r = r0 < RP ? r0 : rb; r < rb; r += RP) {
      float2 xv[KC];
#pragma unroll
      for (int k = 0; k < KC; ++k) xv[k] = (k < K) ? gs[(k * rb + r) * llr_ld(nz) + zz] : make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < KC; ++k)
#pragma unroll
        for (int l = k; l < KC; ++l) {
          // conj(x_k) x_l
          gr[k][l] = fmaf(xv[k].x, xv[l].x, fmaf(xv[k].y, xv[l].y, gr[k][l]));
          if (l > k) gr[l][k] = fmaf(xv[k].x, xv[l].y, fmaf(-xv[k].y, xv[l].x, gr[l][k]));
        }
    }
#pragma unroll
    for (int k = 0; k < KC; ++k)
#pragma unroll
      for (int l = 0; l < KC; ++l)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gr[k][l] += __shfl_xor_sync(0xffffffffu, gr[k][l], o);
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < KC; ++k)
#pragma unroll
        for (int l = 0; l < KC; ++l) gram[blk * kGramStride<KC> + k * KC + l] = gr[k][l];
    }
  }
}

// 3. threshold weights, one thread per block, threads t0 .. t0 + nth - 1
template <int KC, typename ET>
__device__ __forceinline__ void llr_eigen(const float* gram, float tau, float2* wm, int nblk, int t0, int nth) {
  for (int blk = (int)threadIdx.x - t0; blk < nblk; blk += nth)
    svt_weights<ET, KC>(gram + blk * kGramStride<KC>, tau, wm + (size_t)blk * kWStride<KC>);
}

// 4. X' = X W, then the FISTA momentum or the ADMM dual; write back.  The optional
// convergence monitor sums |change|^2 and |new|^2 in float32 per thread.
template <int KC, int MODE>
__device__ __forceinline__ void llr_apply(const Geom& g, const FistaArgs& a, const LlrUnit& un, const float2* gs,
                                          const float2* wm, float2* x, float2* z, float2* u, bool want_res, float& d2,
                                          float& x2) {
  const int ny = g.ny, nz = g.nz, N = ny * nz, K = g.K, b = a.b, rb = un.rb;
  const LlrCols c = llr_cols(nz, 0, blockDim.x);
  if (!c.active) return;
  // the two pixels of this thread's pair and the blocks they fall in (the band's columns
  // are shifted by sz: block j holds the columns (sz + j b + 0 .. b - 1) mod nz)
  const int zz = 2 * c.c2;
  int d0 = zz - a.sz % nz;
  d0 += d0 < 0 ? nz : 0;
  const int d1 = d0 + 1 == nz ? 0 : d0 + 1;
  const float2* w0 = wm + (size_t)(d0 / b) * kWStride<KC>;
  const float2* w1 = wm + (size_t)(d1 / b) * kWStride<KC>;
  const int y0 = llr_row0(g, a, un);
  const long long gb0 = ((long long)(un.s * g.M + un.m0) * K) * N + zz;
  for (int r = c.lp; r < rb; r += c.P) {
    int y = y0 + r;
    y -= y >= ny ? ny : 0;
    float4 xv[KC];  // (pixel zz, pixel zz + 1) of each basis image
#pragma unroll
    for (int k = 0; k < KC; ++k)
      xv[k] = (k < K) ? *reinterpret_cast<const float4*>(gs + (k * rb + r) * llr_ld(nz) + zz)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
    const long long gb = gb0 + (long long)y * nz;
    float4 xp[KC];  // x_k of the pair in every basis image, requested before any store of the row
    if (MODE == LLR_FISTA) {
#pragma unroll
      for (int k = 0; k < KC; ++k)
        xp[k] = (k < K) ? *reinterpret_cast<const float4*>(x + gb + (long long)k * N) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      if (k < K) {
        float2 o0 = make_float2(0.f, 0.f), o1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < KC; ++l) {
          cfma(o0, make_float2(xv[l].x, xv[l].y), w0[l * KC + k]);
          cfma(o1, make_float2(xv[l].z, xv[l].w), w1[l * KC + k]);
        }
        const float4 o = make_float4(o0.x, o0.y, o1.x, o1.y);
        const float4 xk = xv[k];
        const long long gi = gb + (long long)k * N;
        if (MODE == LLR_ADMM) {
          if (want_res) {
            const float4 zo = *reinterpret_cast<const float4*>(z + gi);
            const float dx0 = o.x - zo.x, dy0 = o.y - zo.y, dx1 = o.z - zo.z, dy1 = o.w - zo.w;
            d2 = fmaf(dx0, dx0, fmaf(dy0, dy0, fmaf(dx1, dx1, fmaf(dy1, dy1, d2))));
            x2 = fmaf(o.x, o.x, fmaf(o.y, o.y, fmaf(o.z, o.z, fmaf(o.w, o.w, x2))));
          }
          *reinterpret_cast<float4*>(z + gi) = o;
          *reinterpret_cast<float4*>(u + gi) = make_float4(xk.x - o.x, xk.y - o.y, xk.z - o.z, xk.w - o.w);
          continue;
        }
        if (MODE == LLR_FISTA) {
          const float4 xo = xp[k];
          const float4 dx = make_float4(o.x - xo.x, o.y - xo.y, o.z - xo.z, o.w - xo.w);
          *reinterpret_cast<float4*>(z + gi) =
              make_float4(o.x + a.beta * dx.x, o.y + a.beta * dx.y, o.z + a.beta * dx.z, o.w + a.beta * dx.w);
          if (want_res) {
            d2 = fmaf(dx.x, dx.x, fmaf(dx.y, dx.y, fmaf(dx.z, dx.z, fmaf(dx.w, dx.w, d2))));
            x2 = fmaf(o.x, o.x, fmaf(o.y, o.y, fmaf(o.z, o.z, fmaf(o.w, o.w, x2))));
          }
        }
        *reinterpret_cast<float4*>(x + gi) = o;
      }
    }
  }
}

// float32 per-thread sums of the monitor, float64 across threads (the float64 pipe is a
// small fraction of float32 on GB300)
__device__ __forceinline__ void llr_res_flush(double* res, float d2, float x2) {
  double dd = d2, xx = x2;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dd += __shfl_xor_sync(0xffffffffu, dd, o);
    xx += __shfl_xor_sync(0xffffffffu, xx, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(res, dd);
    atomicAdd(res + 1, xx);
  }
}

template <int KC>
__host__ __device__ constexpr size_t llr_unit_bytes(int K, int b, int nz) {
  return sizeof(float2) * ((size_t)K * b * llr_ld(nz) + (size_t)((nz + b - 1) / b) * kWStride<KC>) +
         sizeof(float) * (size_t)((nz + b - 1) / b) * kGramStride<KC>;
}

// The K <= 4 float32 variant is held to 80 registers (three CTAs per SM) or, where four
// CTAs' shared memory fits on an SM, to 64 registers (four per SM; a few values spill to
// L1), so that the single-thread eigen-steps of one band overlap the memory phases of the
// others: 0.735 -> 0.649 ms on the knee scan with four.  The FISTA momentum's loads of x_k
// for a pixel pair are issued for all K images before the row's first store (the compiler
// may not move a load of x above a store through z, which could alias it): 0.573 -> 0.528
// ms on the knee scan.  Where a band is so large that only two CTAs fit (the 12-row bands
// of Table I's 260 x 240 slices), the CTAs have 512 threads at 64 registers, so the memory
// phases keep as many loads in flight.
// MODE LLR_PROX: x <- prox(x).  LLR_FISTA: x_{k+1} <- prox(z - mu (grad - aty)),
// z <- x_{k+1} + beta (x_{k+1} - x_k).  LLR_ADMM: w = x + u (x = alpha), z <- v = prox(w),
// u <- w - v.
// One CTA's work: unit = (slice s, map set m0, band) decoded by llr_unit.
template <int KC, int MODE, typename ET, int NT>
__device__ __forceinline__ void llr_band(const Geom& g, const FistaArgs& a, int unit, float2* x, float2* z,
                                         const float2* __restrict__ grad, const float2* __restrict__ aty, float2* u) {
  extern __shared__ float2 smem[];
  const LlrUnit un = llr_unit(g, a.b, unit);
  const int nbz = (g.nz + a.b - 1) / a.b;
  float2* gs = smem;                                         // [K][rb][llr_ld(nz)]
  float2* wm = gs + (size_t)g.K * un.rb * llr_ld(g.nz);      // [nbz][kWStride]: KC x KC weights
  float* gram = reinterpret_cast<float*>(wm + (size_t)nbz * kWStride<KC>);  // [nbz][kGramStride]
  llr_gather<MODE>(g, a, un, gs, x, z, grad, aty, u, 0, NT);
  __syncthreads();
  llr_gram<KC>(g, a, un, gs, gram, 0, NT / 32);
  __syncthreads();
  llr_eigen<KC, ET>(gram, a.tau, wm, nbz, 0, NT);
  __syncthreads();
  const bool want_res = (MODE == LLR_FISTA || MODE == LLR_ADMM) && a.res != nullptr;
  float d2 = 0.f, x2 = 0.f;
  llr_apply<KC, MODE>(g, a, un, gs, wm, x, z, u, want_res, d2, x2);
  if (want_res) llr_res_flush(a.res, d2, x2);
}

template <int KC, int MODE, typename ET, int MINB, int NT = kThreads>
__global__ void __launch_bounds__(NT, MINB)
    k_llr(Geom g, FistaArgs a, float2* x, float2* z, const float2* __restrict__ grad,
          const float2* __restrict__ aty, float2* u) {
  const int nbands = (g.ny + a.b - 1) / a.b;
  llr_band<KC, MODE, ET, NT>(g, a, (blockIdx.y * g.M + blockIdx.z) * nbands + blockIdx.x, x, z, grad, aty, u);
}

// Work-list form for batched solves: one launch runs the FISTA LLR step of several scans;
// CTA i belongs to the last job whose first unit is <= i (jobs in increasing unit0).
template <int KC, typename ET, int MINB, int NT = kThreads>
__global__ void __launch_bounds__(NT, MINB) k_llr_list(const LlrJob* __restrict__ jobs, int njobs) {
  int j = 0;
  while (j + 1 < njobs && jobs[j + 1].unit0 <= (int)blockIdx.x) ++j;
  const Geom g = jobs[j].g;
  const FistaArgs a = jobs[j].a;
  llr_band<KC, LLR_FISTA, ET, NT>(g, a, (int)blockIdx.x - jobs[j].unit0, jobs[j].x, jobs[j].z, jobs[j].grad,
                                  jobs[j].aty, nullptr);
}

template <int KC, int MODE, typename ET, int MINB, int NT = kThreads>
cudaError_t llr_launch(const Geom& g, const FistaArgs& a, size_t sm, float2* x, float2* z, const float2* grad,
                       const float2* aty, float2* u, cudaStream_t st) {
  {
    const cudaError_t e = smem_optin((const void*)k_llr<KC, MODE, ET, MINB, NT>, 200 * 1024);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((g.ny + a.b - 1) / a.b, g.S, g.M);
  k_llr<KC, MODE, ET, MINB, NT><<<grid, NT, sm, st>>>(g, a, x, z, grad, aty, u);
  return cudaGetLastError();
}

// CTAs per SM whose shared memory (plus the 1 KB each reserves) fits in 228 KB
constexpr bool llr_fits(size_t sm, int n) { return (size_t)n * (sm + 1024) <= (size_t)228 * 1024; }

template <int KC, int MODE, typename ET>
cudaError_t llr_go(const Geom& g, const FistaArgs& a, float2* x, float2* z, const float2* grad, const float2* aty,
                   float2* u, cudaStream_t st) {
  const size_t sm = llr_unit_bytes<KC>(g.K, a.b, g.nz);
  if constexpr (KC == 4 && sizeof(ET) == 4) {
    if (llr_fits(sm, 4)) return llr_launch<KC, MODE, ET, 4>(g, a, sm, x, z, grad, aty, u, st);
    if (llr_fits(sm, 3)) return llr_launch<KC, MODE, ET, 3>(g, a, sm, x, z, grad, aty, u, st);
    return llr_launch<KC, MODE, ET, 2, 2 * kThreads>(g, a, sm, x, z, grad, aty, u, st);
  } else {
    return llr_launch<KC, MODE, ET, 1>(g, a, sm, x, z, grad, aty, u, st);
  }
}

template <int MODE>
cudaError_t llr_mode(const Geom& g, const FistaArgs& a, float2* x, float2* z, const float2* grad, const float2* aty,
                     float2* u, cudaStream_t st) {
  if (a.eig64)
    return g.K <= 4 ? llr_go<4, MODE, double>(g, a, x, z, grad, aty, u, st)
                    : llr_go<8, MODE, double>(g, a, x, z, grad, aty, u, st);
  return g.K <= 4 ? llr_go<4, MODE, float>(g, a, x, z, grad, aty, u, st)
                  : llr_go<8, MODE, float>(g, a, x, z, grad, aty, u, st);
}

}  // namespace

cudaError_t launch_llr(const Geom& g, const FistaArgs& a, float2* x, float2* z, const float2* grad,
                       const float2* aty, cudaStream_t st) {
  return z != nullptr ? llr_mode<LLR_FISTA>(g, a, x, z, grad, aty, nullptr, st)
                      : llr_mode<LLR_PROX>(g, a, x, nullptr, nullptr, nullptr, nullptr, st);
}

cudaError_t launch_llr_admm(const Geom& g, const FistaArgs& a, const float2* alpha, float2* v, float2* u,
                            cudaStream_t st) {
  return llr_mode<LLR_ADMM>(g, a, const_cast<float2*>(alpha), v, nullptr, nullptr, u, st);
}

int llr_units(const Geom& g, int b) { return ((g.ny + b - 1) / b) * g.S * g.M; }

cudaError_t launch_llr_list(const LlrJob* jobs, int njobs, int units, bool kc8, bool eig64, size_t smem,
                            cudaStream_t st) {
  if (njobs <= 0 || units <= 0) return cudaSuccess;
  auto go = [&](auto kern, int nt) -> cudaError_t {
    const cudaError_t e = smem_optin((const void*)kern, 200 * 1024);
    if (e != cudaSuccess) return e;
    kern<<<units, nt, smem, st>>>(jobs, njobs);
    return cudaGetLastError();
  };
  // the same register bounds and CTA sizes as the per-scan launches (llr_go)
  if (eig64) return kc8 ? go(k_llr_list<8, double, 1>, kThreads) : go(k_llr_list<4, double, 1>, kThreads);
  if (kc8) return go(k_llr_list<8, float, 1>, kThreads);
  if (llr_fits(smem, 4)) return go(k_llr_list<4, float, 4>, kThreads);
  if (llr_fits(smem, 3)) return go(k_llr_list<4, float, 3>, kThreads);
  return go(k_llr_list<4, float, 2, 2 * kThreads>, 2 * kThreads);
}

size_t llr_smem_bytes(const Geom& g, int b) {
  return g.K <= 4 ? llr_unit_bytes<4>(g.K, b, g.nz) : llr_unit_bytes<8>(g.K, b, g.nz);
}

}  // namespace t2sh
