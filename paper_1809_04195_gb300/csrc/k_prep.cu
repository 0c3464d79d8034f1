// Plan-time kernels: coil-map preparation, the space-time kernel Psi (Sec. IV.B) and
// the projection of per-echo k-space onto the basis (re-sort and project, Sec. III.A).
#include "t2sh_device.cuh"

namespace t2sh {

// S'_{c,m}(y, z) = (-1)^(y+z) S_{c,m}(y, z): the image-side half of the FFT centring
// (FFTmod, Sec. IV.A) folded into the maps once.  Also the per-pixel largest
// eigenvalue of S(p)^H S(p) (C x M), max-reduced over all pixels into *lam_bits
// (float bits; non-negative floats order like their bit patterns).
__global__ void __launch_bounds__(kThreads) k_maps_prep(Geom g, const float2* in, float2* out,
                                                      unsigned* lam_bits) {
  const int N = g.ny * g.nz;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // over S * N pixels
  float lam = 0.0f;
  if (idx < (long long)g.S * N) {
    const int s = (int)(idx / N);
    const int n = (int)(idx - (long long)s * N);
    const int y = n / g.nz, z = n - y * g.nz;
    const float sg = parity_sign(y + z);
    double a = 0.0, d = 0.0, br = 0.0, bi = 0.0;
    for (int c = 0; c < g.C; ++c) {
      const long long base = ((long long)(s * g.C + c) * g.M) * N + n;
      const float2 s0 = in[base];
      out[base] = cscale(s0, sg);
      a += (double)s0.x * s0.x + (double)s0.y * s0.y;
      if (g.M > 1) {
        const float2 s1 = in[base + N];
        out[base + N] = cscale(s1, sg);
        d += (double)s1.x * s1.x + (double)s1.y * s1.y;
        br += (double)s0.x * s1.x + (double)s0.y * s1.y;  // conj(s0) s1
        bi += (double)s0.x * s1.y - (double)s0.y * s1.x;
      }
    }
    double l = a;
    if (g.M > 1) {
      const double h = 0.5 * (a - d);
      l = 0.5 * (a + d) + sqrt(h * h + br * br + bi * bi);
    }
    lam = (float)l;
  }
  // warp max then one atomic per warp
  for (int o = 16; o > 0; o >>= 1) lam = fmaxf(lam, __shfl_xor_sync(0xffffffffu, lam, o));
  if ((threadIdx.x & 31) == 0 && lam > 0.0f) atomicMax(lam_bits, __float_as_uint(lam));
}

// Psi(n)_{kl} = sum_t Phi_{tk} P_t(n) Phi_{tl} in float64, stored as float32 upper
// triangle (p = 0.. for k <= l, row by row) scaled by 1/N so the unnormalised
// DFT pair needs no other scaling, SoA [P][ny][nz].  Also lambda_max(Psi(n)) max-reduced.
template <int KC>
__global__ void __launch_bounds__(kThreads) k_psi_build(Geom g, const float* __restrict__ phi,
                                                      const uint8_t* __restrict__ mask, float* __restrict__ psi,
                                                      unsigned* lam_bits) {
  extern __shared__ float sphi[];  // [T][K]
  for (int i = threadIdx.x; i < g.T * g.K; i += blockDim.x) sphi[i] = phi[i];
  __syncthreads();
  const int N = g.ny * g.nz;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  float lam = 0.0f;
  if (n < N) {
    double acc[KC][KC];
#pragma unroll
    for (int k = 0; k < KC; ++k)
#pragma unroll
      for (int l = 0; l < KC; ++l) acc[k][l] = 0.0;
    for (int t = 0; t < g.T; ++t) {
      if (mask[(long long)t * N + n]) {
        const float* ph = sphi + t * g.K;
#pragma unroll
        for (int k = 0; k < KC; ++k)
#pragma unroll
          for (int l = k; l < KC; ++l)
            if (l < g.K) acc[k][l] += (double)ph[k] * (double)ph[l];
      }
    }
    const double inv_n = 1.0 / (double)N;
    int p = 0;
#pragma unroll
    for (int k = 0; k < KC; ++k)
#pragma unroll
      for (int l = k; l < KC; ++l)
        if (l < g.K) {
          psi[(long long)p * N + n] = (float)(acc[k][l] * inv_n);
          ++p;
        }
    double ar[KC][KC], ai[KC][KC], vr[KC][KC], vi[KC][KC];
#pragma unroll
    for (int k = 0; k < KC; ++k)
#pragma unroll
      for (int l = 0; l < KC; ++l) {
        const bool in = (k < g.K && l < g.K);
        ar[k][l] = in ? (k <= l ? acc[k][l] : acc[l][k]) : 0.0;
        ai[k][l] = 0.0;
      }
    herm_jacobi<double, KC>(ar, ai, vr, vi, 12);
    double m = 0.0;
#pragma unroll
    for (int k = 0; k < KC; ++k) m = fmax(m, ar[k][k]);
    lam = (float)m;
  }
  for (int o = 16; o > 0; o >>= 1) lam = fmaxf(lam, __shfl_xor_sync(0xffffffffu, lam, o));
  if ((threadIdx.x & 31) == 0 && lam > 0.0f) atomicMax(lam_bits, __float_as_uint(lam));
}

// ytil[s][c][k][n] = sum_t Phi_{tk} P_t(n) y[s][c][t][n]
template <int KC>
__global__ void __launch_bounds__(kThreads) k_project(Geom g, const float* __restrict__ phi,
                                                    const uint8_t* __restrict__ mask,
                                                    const float2* __restrict__ y, float2* __restrict__ out) {
  extern __shared__ float sphi[];
  for (int i = threadIdx.x; i < g.T * g.K; i += blockDim.x) sphi[i] = phi[i];
  __syncthreads();
  const int N = g.ny * g.nz;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int sc = blockIdx.y;  // s * C + c
  if (n >= N) return;
  float2 acc[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) acc[k] = make_float2(0.f, 0.f);
  const float2* yb = y + (long long)sc * g.T * N + n;
  for (int t = 0; t < g.T; ++t) {
    if (mask[(long long)t * N + n]) {
      const float2 v = yb[(long long)t * N];
      const float* ph = sphi + t * g.K;
#pragma unroll
      for (int k = 0; k < KC; ++k)
        if (k < g.K) {
          acc[k].x = fmaf(ph[k], v.x, acc[k].x);
          acc[k].y = fmaf(ph[k], v.y, acc[k].y);
        }
    }
  }
  float2* ob = out + (long long)sc * g.K * N + n;
#pragma unroll
  for (int k = 0; k < KC; ++k)
    if (k < g.K) ob[(long long)k * N] = acc[k];
}

cudaError_t launch_maps_prep(const Geom& g, const float2* maps_in, float2* maps_out, unsigned* lam_bits,
                             cudaStream_t st) {
  const long long tot = (long long)g.S * g.ny * g.nz;
  const unsigned grid = (unsigned)((tot + kThreads - 1) / kThreads);
  k_maps_prep<<<grid, kThreads, 0, st>>>(g, maps_in, maps_out, lam_bits);
  return cudaGetLastError();
}

cudaError_t launch_psi_build(const Geom& g, const float* phi, const uint8_t* mask, float* psi,
                             unsigned* lam_bits, cudaStream_t st) {
  const int N = g.ny * g.nz;
  const unsigned grid = (unsigned)((N + kThreads - 1) / kThreads);
  const size_t sm = sizeof(float) * g.T * g.K;
  if (g.K <= 4) k_psi_build<4><<<grid, kThreads, sm, st>>>(g, phi, mask, psi, lam_bits);
  else k_psi_build<8><<<grid, kThreads, sm, st>>>(g, phi, mask, psi, lam_bits);
  return cudaGetLastError();
}

cudaError_t launch_project(const Geom& g, const float* phi, const uint8_t* mask, const float2* y_te,
                           float2* y_proj, cudaStream_t st) {
  const int N = g.ny * g.nz;
  dim3 grid((N + kThreads - 1) / kThreads, g.S * g.C);
  const size_t sm = sizeof(float) * g.T * g.K;
  if (g.K <= 4) k_project<4><<<grid, kThreads, sm, st>>>(g, phi, mask, y_te, y_proj);
  else k_project<8><<<grid, kThreads, sm, st>>>(g, phi, mask, y_te, y_proj);
  return cudaGetLastError();
}

}  // namespace t2sh
