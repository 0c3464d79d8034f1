// Conjugate-gradient vector kernels for the ADMM alpha-update
// (A^H A + rho I) alpha = A^H y + rho (v - u), one independent system per slice.
//
// Every vector is [S][M][K][ny][nz] complex64; slice s owns a contiguous run of
// L = M K ny nz values, and every scalar of the iteration is per slice.  The kernels
// stream float4 (two complex values) per load; a thread sums its few terms in float32,
// the CTA reduces in float64 with warp shuffles and adds its partial into the slice's
// float64 accumulator with one atomic.  The step a = <r,r> / <p,q> and the direction
// weight b = <r_new,r_new> / <r,r> are formed on the device from those accumulators
// (a zero denominator gives a zero quotient), so an iteration needs no host round trip.
#include <algorithm>

#include "t2sh_device.cuh"

namespace t2sh {

namespace {

constexpr int kCgThreads = 256;
constexpr int kCgPerThread = 2;  // float4 loads per thread per vector

__device__ __forceinline__ void block_add(double v, double* out) {
  __shared__ double part[kCgThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) part[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < kCgThreads / 32 ? part[lane] : 0.0;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) atomicAdd(out, v);
  }
}

__device__ __forceinline__ float4 ld4(const float2* p, long long i) { return *reinterpret_cast<const float4*>(p + i); }
__device__ __forceinline__ void st4(float2* p, long long i, float4 v) { *reinterpret_cast<float4*>(p + i) = v; }
__device__ __forceinline__ float dot4(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }

// Every kernel first issues all of its loads (kCgPerThread float4 per vector), then
// computes and stores, so that each thread keeps its loads in flight together.  The
// per-slice quotient (a float64 division) is formed once per CTA and broadcast.
__device__ __forceinline__ float cta_quotient(const double* num, const double* den, int s) {
  __shared__ float q;
  if (threadIdx.x == 0) {
    const double d = den[s];
    q = d != 0.0 ? (float)(num[s] / d) : 0.f;
  }
  __syncthreads();
  return q;
}
#define CG_INDEX(i) (2 * ((long long)(blockIdx.x * kCgPerThread + (i)) * kCgThreads + threadIdx.x))

// r = aty + rho (v - u) - w - rho x  (w = A^H A x);  p = r;  rr[s] += |r|^2
__global__ void __launch_bounds__(kCgThreads) k_cg_init(long long L, const float2* __restrict__ x,
                                                       const float2* __restrict__ w, const float2* __restrict__ aty,
                                                       const float2* __restrict__ v, const float2* __restrict__ u,
                                                       float rho, float2* __restrict__ r, float2* __restrict__ p,
                                                       double* rr) {
  const long long base = (long long)blockIdx.y * L;
  float4 xa[kCgPerThread], wa[kCgPerThread], ya[kCgPerThread], va[kCgPerThread], ua[kCgPerThread];
#pragma unroll
  for (int i = 0; i < kCgPerThread; ++i) {
    const long long e = CG_INDEX(i);
    if (e < L) {
      xa[i] = ld4(x, base + e); wa[i] = ld4(w, base + e); ya[i] = ld4(aty, base + e);
      va[i] = ld4(v, base + e); ua[i] = ld4(u, base + e);
    }
  }
  float acc = 0.f;
#pragma unroll
  for (int i = 0; i < kCgPerThread; ++i) {
    const long long e = CG_INDEX(i);
    if (e < L) {
      float4 ra;
      ra.x = ya[i].x + rho * (va[i].x - ua[i].x) - wa[i].x - rho * xa[i].x;
      ra.y = ya[i].y + rho * (va[i].y - ua[i].y) - wa[i].y - rho * xa[i].y;
      ra.z = ya[i].z + rho * (va[i].z - ua[i].z) - wa[i].z - rho * xa[i].z;
      ra.w = ya[i].w + rho * (va[i].w - ua[i].w) - wa[i].w - rho * xa[i].w;
      st4(r, base + e, ra);
      st4(p, base + e, ra);
      acc += dot4(ra, ra);
    }
  }
  block_add((double)acc, rr + blockIdx.y);
}

// pq[s] += Re <p, w + rho p>  (w = A^H A p)
__global__ void __launch_bounds__(kCgThreads) k_cg_dot(long long L, const float2* __restrict__ p,
                                                      const float2* __restrict__ w, float rho, double* pq) {
  const long long base = (long long)blockIdx.y * L;
  float4 pa[kCgPerThread], wa[kCgPerThread];
#pragma unroll
  for (int i = 0; i < kCgPerThread; ++i) {
    const long long e = CG_INDEX(i);
    if (e < L) {
      pa[i] = ld4(p, base + e);
      wa[i] = ld4(w, base + e);
    }
  }
  float acc = 0.f;
#pragma unroll
  for (int i = 0; i < kCgPerThread; ++i)
    if (CG_INDEX(i) < L)
      acc += pa[i].x * (wa[i].x + rho * pa[i].x) + pa[i].y * (wa[i].y + rho * pa[i].y) +
             pa[i].z * (wa[i].z + rho * pa[i].z) + pa[i].w * (wa[i].w + rho * pa[i].w);
  block_add((double)acc, pq + blockIdx.y);
}

// a = rr / pq;  x += a p;  r -= a (w + rho p);  rr_new[s] += |r|^2
__global__ void __launch_bounds__(kCgThreads) k_cg_step(long long L, float2* __restrict__ x, float2* __restrict__ r,
                                                       const float2* __restrict__ p, const float2* __restrict__ w,
                                                       float rho, const double* rr, const double* pq,
                                                       double* rr_new) {
  const int s = blockIdx.y;
  const long long base = (long long)s * L;
  float4 pa[kCgPerThread], wa[kCgPerThread], xa[kCgPerThread], ra[kCgPerThread];
#pragma unroll
  for (int i = 0; i < kCgPerThread; ++i) {
    const long long e = CG_INDEX(i);
    if (e < L) {
      pa[i] = ld4(p, base + e); wa[i] = ld4(w, base + e);
      xa[i] = ld4(x, base + e); ra[i] = ld4(r, base + e);
    }
  }
  const float a = cta_quotient(rr, pq, s);
  float acc = 0.f;
#pragma unroll
  for (int i = 0; i < kCgPerThread; ++i) {
    const long long e = CG_INDEX(i);
    if (e < L) {
      xa[i].x = fmaf(a, pa[i].x, xa[i].x);
      xa[i].y = fmaf(a, pa[i].y, xa[i].y);
      xa[i].z = fmaf(a, pa[i].z, xa[i].z);
      xa[i].w = fmaf(a, pa[i].w, xa[i].w);
      ra[i].x -= a * (wa[i].x + rho * pa[i].x);
      ra[i].y -= a * (wa[i].y + rho * pa[i].y);
      ra[i].z -= a * (wa[i].z + rho * pa[i].z);
      ra[i].w -= a * (wa[i].w + rho * pa[i].w);
      st4(x, base + e, xa[i]);
      st4(r, base + e, ra[i]);
      acc += dot4(ra[i], ra[i]);
    }
  }
  block_add((double)acc, rr_new + s);
}

// b = rr_new / rr;  p = r + b p.  The first CTA of each slice also clears the
// accumulators the next iteration adds into (pq and the next rr_new slot).
__global__ void __launch_bounds__(kCgThreads) k_cg_dir(long long L, const float2* __restrict__ r,
                                                      float2* __restrict__ p, const double* rr, const double* rr_new,
                                                      double* pq, double* rr_next) {
  const int s = blockIdx.y;
  const long long base = (long long)s * L;
  float4 ra[kCgPerThread], pa[kCgPerThread];
#pragma unroll
  for (int i = 0; i < kCgPerThread; ++i) {
    const long long e = CG_INDEX(i);
    if (e < L) {
      ra[i] = ld4(r, base + e);
      pa[i] = ld4(p, base + e);
    }
  }
  const float b = cta_quotient(rr_new, rr, s);
#pragma unroll
  for (int i = 0; i < kCgPerThread; ++i) {
    const long long e = CG_INDEX(i);
    if (e < L) {
      pa[i].x = fmaf(b, pa[i].x, ra[i].x);
      pa[i].y = fmaf(b, pa[i].y, ra[i].y);
      pa[i].z = fmaf(b, pa[i].z, ra[i].z);
      pa[i].w = fmaf(b, pa[i].w, ra[i].w);
      st4(p, base + e, pa[i]);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    pq[s] = 0.0;
    rr_next[s] = 0.0;
  }
}
#undef CG_INDEX

// out[s] += sum_{c,t,n} P_t(n) |y_{s,c,t}(n)|^2 of T-form k-space y [S][C][T][N] (float64
// per thread: a diagnostic reduction, not on the iteration path)
__global__ void __launch_bounds__(kCgThreads) k_masked_energy(long long N, int C, int T, const uint8_t* __restrict__ mask,
                                                             const float2* __restrict__ y, double* out) {
  const int s = blockIdx.y;
  const long long L = (long long)C * T * N;
  const float2* ys = y + (long long)s * L;
  double acc = 0.0;
  for (long long n = (long long)blockIdx.x * kCgThreads + threadIdx.x; n < N; n += (long long)gridDim.x * kCgThreads)
    for (int t = 0; t < T; ++t)
      if (mask[(long long)t * N + n])
        for (int c = 0; c < C; ++c) {
          const float2 v = ys[((long long)c * T + t) * N + n];
          acc += (double)v.x * v.x + (double)v.y * v.y;
        }
  block_add(acc, out + s);
}

dim3 cg_grid(const Geom& g, long long L) {
  const long long per_cta = 2LL * kCgThreads * kCgPerThread;
  return dim3((unsigned)((L + per_cta - 1) / per_cta), (unsigned)g.S);
}

}  // namespace

// L = M K ny nz complex values per slice (even: ny, nz are even)
cudaError_t launch_cg_init(const Geom& g, const float2* x, const float2* w, const float2* aty, const float2* v,
                           const float2* u, float rho, float2* r, float2* p, double* rr, cudaStream_t st) {
  const long long L = (long long)g.M * g.K * g.ny * g.nz;
  k_cg_init<<<cg_grid(g, L), kCgThreads, 0, st>>>(L, x, w, aty, v, u, rho, r, p, rr);
  return cudaGetLastError();
}

cudaError_t launch_cg_dot(const Geom& g, const float2* p, const float2* w, float rho, double* pq, cudaStream_t st) {
  const long long L = (long long)g.M * g.K * g.ny * g.nz;
  k_cg_dot<<<cg_grid(g, L), kCgThreads, 0, st>>>(L, p, w, rho, pq);
  return cudaGetLastError();
}

cudaError_t launch_cg_step(const Geom& g, float2* x, float2* r, const float2* p, const float2* w, float rho,
                           const double* rr, const double* pq, double* rr_new, cudaStream_t st) {
  const long long L = (long long)g.M * g.K * g.ny * g.nz;
  k_cg_step<<<cg_grid(g, L), kCgThreads, 0, st>>>(L, x, r, p, w, rho, rr, pq, rr_new);
  return cudaGetLastError();
}

cudaError_t launch_masked_energy(const Geom& g, const uint8_t* mask, const float2* y, double* out, cudaStream_t st) {
  const long long N = (long long)g.ny * g.nz;
  const unsigned gx = (unsigned)std::min<long long>((N + kCgThreads - 1) / kCgThreads, 64);
  k_masked_energy<<<dim3(gx, (unsigned)g.S), kCgThreads, 0, st>>>(N, g.C, g.T, mask, y, out);
  return cudaGetLastError();
}

cudaError_t launch_cg_dir(const Geom& g, const float2* r, float2* p, const double* rr, const double* rr_new,
                          double* pq, double* rr_next, cudaStream_t st) {
  const long long L = (long long)g.M * g.K * g.ny * g.nz;
  k_cg_dir<<<cg_grid(g, L), kCgThreads, 0, st>>>(L, r, p, rr, rr_new, pq, rr_next);
  return cudaGetLastError();
}

}  // namespace t2sh
