// Locally-low-rank prox (Eq. 4, Sec. II.B) in one pass over the coefficient images,
// as Sec. IV.C describes: the random circular shift is folded into the gather
// indices (no shifted copy), each block is thresholded on chip and written back.
//
// One CTA per (slice, band of b shifted rows).  Per block (b x b pixels x K, per map
// set) a warp forms the K x K Gram matrix G = X^H X with shuffle reductions; one
// thread per block then eigendecomposes G = V diag(lambda) V^H (cyclic Jacobi, float32
// by default, float64 on request), sigma_i = sqrt(lambda_i), and forms
// W = V diag(max(1 - tau/sigma_i, 0)) V^H,
// so that X W = U max(Sigma - tau, 0) V^H (since X V = U Sigma).  The FISTA variant
// fuses the gradient step before the prox and the momentum update after it (Sec. II.A);
// the ADMM variant thresholds alpha + u and writes v and the scaled dual u + alpha - v.
#include "t2sh_device.cuh"

namespace t2sh {

enum { LLR_PROX = 0, LLR_FISTA = 1, LLR_ADMM = 2 };

// The K <= 4 float32 variant is held to 80 registers so that three CTAs share an SM and
// the single-thread eigen-steps of one band overlap the memory phases of the others.
// MODE LLR_PROX: x <- prox(x).  LLR_FISTA: x_{k+1} <- prox(z - mu (grad - aty)),
// z <- x_{k+1} + beta (x_{k+1} - x_k).  LLR_ADMM: w = x + u (x = alpha), z <- v = prox(w),
// u <- w - v.
template <int KC, int MODE, typename ET>
__global__ void __launch_bounds__(kThreads, (KC == 4 && sizeof(ET) == 4) ? 3 : 1)
    k_llr(Geom g, FistaArgs a, float2* x, float2* z, const float2* __restrict__ grad,
          const float2* __restrict__ aty, float2* u) {
  constexpr bool FISTA = MODE == LLR_FISTA;
  extern __shared__ float2 smem[];
  // one CTA per (band, slice, map set): the blocks of different map sets are independent
  const int ny = g.ny, nz = g.nz, N = ny * nz, K = g.K, b = a.b;
  const int M = 1, MS = g.M, m0 = blockIdx.z;  // map sets staged by this CTA, total, this one
  const int s = blockIdx.y, band = blockIdx.x;
  const int rb = min(b, ny - band * b);
  const int nbz = (nz + b - 1) / b;
  const int nblk = M * nbz;
  float2* gs = smem;                                   // [M][K][rb][nz]
  float2* wm = gs + (size_t)M * K * rb * nz;           // [nblk][KC][KC]
  float* gram = reinterpret_cast<float*>(wm + (size_t)nblk * KC * KC);  // [nblk][KC*KC]

  // 1. gather the band (gradient step fused for FISTA), two pixels per float4
  const int nel2 = (M * K * rb * nz) >> 1;
#pragma unroll 4
  for (int e2 = threadIdx.x; e2 < nel2; e2 += kThreads) {
    const int e = 2 * e2;
    const int zz = e % nz;
    int rest = e / nz;
    const int r = rest % rb;
    rest /= rb;  // m * K + k
    const int y = (a.sy + band * b + r) % ny;
    const long long gi = (((long long)s * MS + m0) * K + rest) * N + (long long)y * nz + zz;
    float4 v;
    if (MODE == LLR_ADMM) {
      const float4 av = *reinterpret_cast<const float4*>(x + gi);
      const float4 uv = *reinterpret_cast<const float4*>(u + gi);
      v = make_float4(av.x + uv.x, av.y + uv.y, av.z + uv.z, av.w + uv.w);
    } else if (FISTA) {
      const float4 zv = *reinterpret_cast<const float4*>(z + gi);
      const float4 gv = *reinterpret_cast<const float4*>(grad + gi);
      const float4 av = *reinterpret_cast<const float4*>(aty + gi);
      v = make_float4(zv.x - a.mu * (gv.x - av.x), zv.y - a.mu * (gv.y - av.y), zv.z - a.mu * (gv.z - av.z),
                      zv.w - a.mu * (gv.w - av.w));
    } else {
      v = *reinterpret_cast<const float4*>(x + gi);
    }
    gs[e] = make_float2(v.x, v.y);
    gs[e + 1] = make_float2(v.z, v.w);
  }
  __syncthreads();

  // 2. Gram matrices, one warp per block
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int blk = warp; blk < nblk; blk += kThreads / 32) {
    const int m = blk / nbz, j = blk - m * nbz;
    const int cb = min(b, nz - j * b);
    float gr[KC][KC];  // upper: re at [k][l] (k <= l), im at [l][k] (l > k)
#pragma unroll
    for (int k = 0; k < KC; ++k)
#pragma unroll
      for (int l = 0; l < KC; ++l) gr[k][l] = 0.f;
    for (int p = lane; p < rb * cb; p += 32) {
      const int r = p / cb, cc = p - r * cb;
      const int zz = (a.sz + j * b + cc) % nz;
      float2 xv[KC];
#pragma unroll
      for (int k = 0; k < KC; ++k) xv[k] = (k < K) ? gs[((m * K + k) * rb + r) * nz + zz] : make_float2(0.f, 0.f);
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
        for (int l = 0; l < KC; ++l) gram[blk * KC * KC + k * KC + l] = gr[k][l];
    }
  }
  __syncthreads();

  // 3. eigendecomposition and threshold weights, one thread per block
  for (int blk = threadIdx.x; blk < nblk; blk += kThreads)
    svt_weights<ET, KC>(gram + blk * KC * KC, a.tau, wm + (size_t)blk * KC * KC);
  __syncthreads();

  // 4. X' = X W, then FISTA momentum; write back.  The optional convergence monitor sums
  // |x_{k+1} - x_k|^2 and |x_{k+1}|^2 in float32 per thread (float64 only for the
  // cross-thread reduction: the float64 pipe is a small fraction of float32 on GB300).
  const bool want_res = (FISTA || MODE == LLR_ADMM) && a.res != nullptr;
  float d2 = 0.f, x2 = 0.f;
  const int npx = M * rb * nz;
  for (int e = threadIdx.x; e < npx; e += kThreads) {
    const int zz = e % nz;
    const int rest = e / nz;
    const int r = rest % rb, m = rest / rb;
    const int y = (a.sy + band * b + r) % ny;
    const int j = (((zz - a.sz) % nz + nz) % nz) / b;
    const float2* w = wm + (size_t)(m * nbz + j) * KC * KC;
    float2 xv[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) xv[k] = (k < K) ? gs[((m * K + k) * rb + r) * nz + zz] : make_float2(0.f, 0.f);
    const long long gb = ((long long)(s * MS + m0 + m) * K) * N + (long long)y * nz + zz;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      if (k < K) {
        float2 o = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < KC; ++l) cfma(o, xv[l], w[l * KC + k]);
        const long long gi = gb + (long long)k * N;
        if (MODE == LLR_ADMM) {
          if (want_res) {
            const float2 dv = csub(o, z[gi]);
            d2 = fmaf(dv.x, dv.x, fmaf(dv.y, dv.y, d2));
            x2 = fmaf(o.x, o.x, fmaf(o.y, o.y, x2));
          }
          z[gi] = o;
          u[gi] = csub(xv[k], o);
          continue;
        }
        if (FISTA) {
          const float2 xo = x[gi];
          const float2 dx = csub(o, xo);
          z[gi] = make_float2(o.x + a.beta * dx.x, o.y + a.beta * dx.y);
          if (want_res) {
            d2 = fmaf(dx.x, dx.x, fmaf(dx.y, dx.y, d2));
            x2 = fmaf(o.x, o.x, fmaf(o.y, o.y, x2));
          }
        }
        x[gi] = o;
      }
    }
  }
  if (want_res) {
    double dd = d2, xx = x2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dd += __shfl_xor_sync(0xffffffffu, dd, o);
      xx += __shfl_xor_sync(0xffffffffu, xx, o);
    }
    if (lane == 0) {
      atomicAdd(a.res, dd);
      atomicAdd(a.res + 1, xx);
    }
  }
}

template <int KC, int MODE, typename ET>
static cudaError_t llr_go(const Geom& g, const FistaArgs& a, float2* x, float2* z, const float2* grad,
                          const float2* aty, float2* u, cudaStream_t st) {
  const int nbz = (g.nz + a.b - 1) / a.b;
  const int nblk = nbz;  // per map set
  const size_t sm = sizeof(float2) * ((size_t)g.K * a.b * g.nz + (size_t)nblk * KC * KC) +
                    sizeof(float) * (size_t)nblk * KC * KC;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_llr<KC, MODE, ET>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((g.ny + a.b - 1) / a.b, g.S, g.M);
  k_llr<KC, MODE, ET><<<grid, kThreads, sm, st>>>(g, a, x, z, grad, aty, u);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t llr_mode(const Geom& g, const FistaArgs& a, float2* x, float2* z, const float2* grad,
                            const float2* aty, float2* u, cudaStream_t st) {
  if (a.eig64)
    return g.K <= 4 ? llr_go<4, MODE, double>(g, a, x, z, grad, aty, u, st)
                    : llr_go<8, MODE, double>(g, a, x, z, grad, aty, u, st);
  return g.K <= 4 ? llr_go<4, MODE, float>(g, a, x, z, grad, aty, u, st)
                  : llr_go<8, MODE, float>(g, a, x, z, grad, aty, u, st);
}

cudaError_t launch_llr(const Geom& g, const FistaArgs& a, float2* x, float2* z, const float2* grad,
                       const float2* aty, cudaStream_t st) {
  return z != nullptr ? llr_mode<LLR_FISTA>(g, a, x, z, grad, aty, nullptr, st)
                      : llr_mode<LLR_PROX>(g, a, x, nullptr, nullptr, nullptr, nullptr, st);
}

cudaError_t launch_llr_admm(const Geom& g, const FistaArgs& a, const float2* alpha, float2* v, float2* u,
                            cudaStream_t st) {
  return llr_mode<LLR_ADMM>(g, a, const_cast<float2*>(alpha), v, nullptr, nullptr, u, st);
}

size_t llr_smem_bytes(const Geom& g, int b) {
  const int kc = g.K <= 4 ? 4 : 8;
  const int nblk = (g.nz + b - 1) / b;  // one map set per CTA
  return sizeof(float2) * ((size_t)g.K * b * g.nz + (size_t)nblk * kc * kc) + sizeof(float) * (size_t)nblk * kc * kc;
}

}  // namespace t2sh
