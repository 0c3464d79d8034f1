// TE images from the reconstructed coefficients (post-processing, Sec. III.C and Sec. V):
// back-projection with the basis at chosen echoes, virtual-coil images, homodyne
// detection along z (the slice direction, partial Fourier), root sum of squares.
//
// One CTA per (slice, band of kPostRB rows).  For each requested echo t the CTA forms
// x_m(t) = sum_k Phi[t][k] alpha[m][k] for its rows in shared memory, then for every coil
// the coil line x' = sum_m S'_{c,m} x_m(t) with the plan's sign-folded maps
// S' = S (-1)^(y+z), its plain DFT along z (the (-1)^z factor puts DC at index Nz/2, so
// index k is frequency d = k - Nz/2), the homodyne weighting H(d) (0, 1 or 2) and the
// band mask B(d) = 1_{|d| <= w}, two inverse DFTs h' and l', and accumulates
// (Re(h' conj(l')) / |l'| / Nz)^2.  The remaining row sign (-1)^y and the output-side
// (-1)^z multiply h' and l' alike and cancel in h' conj(l').  Output: sqrt of the
// accumulated squares, float [S][nte][ny][nz].
#include "t2sh_device.cuh"

namespace t2sh {

namespace {

constexpr int kPostThreads = 256;
constexpr int kPostRB = 4;

struct PostArgs {
  int te[kMaxPostTe];
  int nte;
  int w;  // half-width of the two-sided band
};

template <int MC, bool R13>
__global__ void __launch_bounds__(kPostThreads) k_post(Geom g, FftPlan pz, const float2* __restrict__ tw_g,
                                                     const float2* __restrict__ maps, const float* __restrict__ phi,
                                                     const float2* __restrict__ alpha, PostArgs pa,
                                                     float* __restrict__ out) {
  extern __shared__ float2 smem[];
  const int ny = g.ny, nz = g.nz, K = g.K, M = g.M, C = g.C;
  const long long N = (long long)ny * nz;
  const int s = blockIdx.y, y0 = blockIdx.x * kPostRB;
  const int rb = min(kPostRB, ny - y0);
  const int ld = nz + 1;
  const int c0 = nz / 2;
  float2* tw = smem;                                             // [nz]
  float2* xm = tw + ((nz + 1) & ~1);                             // [MC][RB][nz]
  float2* lines = xm + (size_t)MC * kPostRB * nz;                // [2 RB][ld]: h lines then band lines
  float* acc = reinterpret_cast<float*>(lines + 2 * kPostRB * ld + 1);  // [nte][RB][nz]
  for (int i = threadIdx.x; i < nz; i += kPostThreads) tw[i] = tw_g[i];
  for (int i = threadIdx.x; i < pa.nte * kPostRB * nz; i += kPostThreads) acc[i] = 0.f;
  const int npt = rb * nz;
  for (int ti = 0; ti < pa.nte; ++ti) {
    const float* ph = phi + (size_t)pa.te[ti] * K;
    __syncthreads();
    // x_m(t) for the band's rows
    for (int e = threadIdx.x; e < M * npt; e += kPostThreads) {
      const int m = e / npt, q = e - m * npt, r = q / nz, z = q - r * nz;
      const float2* ap = alpha + ((long long)(s * M + m) * K) * N + (long long)(y0 + r) * nz + z;
      float2 v = make_float2(0.f, 0.f);
      for (int k = 0; k < K; ++k) {
        const float2 a = ap[(long long)k * N];
        v.x = fmaf(ph[k], a.x, v.x);
        v.y = fmaf(ph[k], a.y, v.y);
      }
      xm[(m * kPostRB + r) * nz + z] = v;
    }
    for (int c = 0; c < C; ++c) {
      __syncthreads();
      for (int q = threadIdx.x; q < npt; q += kPostThreads) {
        const int r = q / nz, z = q - r * nz;
        float2 v = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < MC; ++m)
          if (m < M) cfma(v, maps[((long long)(s * C + c) * M + m) * N + (long long)(y0 + r) * nz + z],
                          xm[(m * kPostRB + r) * nz + z]);
        lines[r * ld + z] = v;
      }
      __syncthreads();
      fft_lines<false, R13>(lines, ld, rb, pz, tw);
      for (int q = threadIdx.x; q < npt; q += kPostThreads) {
        const int r = q / nz, k = q - r * nz, d = k - c0;
        const float2 v = lines[r * ld + k];
        const float hw = d < -pa.w ? 0.f : (d <= pa.w ? 1.f : 2.f);
        lines[(kPostRB + r) * ld + k] = (d >= -pa.w && d <= pa.w) ? v : make_float2(0.f, 0.f);
        lines[r * ld + k] = make_float2(hw * v.x, hw * v.y);
      }
      __syncthreads();
      fft_lines<true, R13>(lines, ld, kPostRB + rb, pz, tw);  // h lines 0..rb-1, band lines RB..RB+rb-1
      const float inv_n = 1.f / (float)nz;
      for (int q = threadIdx.x; q < npt; q += kPostThreads) {
        const int r = q / nz, z = q - r * nz;
        const float2 h = lines[r * ld + z], l = lines[(kPostRB + r) * ld + z];
        const float l2 = l.x * l.x + l.y * l.y;
        const float o = (l2 > 0.f ? (h.x * l.x + h.y * l.y) * rsqrtf(l2) : h.x) * inv_n;
        acc[(ti * kPostRB + r) * nz + z] += o * o;
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < pa.nte * npt; e += kPostThreads) {
    const int ti = e / npt, q = e - ti * npt, r = q / nz, z = q - r * nz;
    out[((long long)s * pa.nte + ti) * N + (long long)(y0 + r) * nz + z] = sqrtf(acc[(ti * kPostRB + r) * nz + z]);
  }
}

template <int MC, bool R13>
cudaError_t post_go(const Geom& g, const FftPlan& pz, const float2* tw_z, const float2* maps, const float* phi,
                    const float2* alpha, const PostArgs& pa, float* out, dim3 grid, size_t sm, cudaStream_t st) {
  {
    const cudaError_t e = smem_optin((const void*)k_post<MC, R13>, 200 * 1024);
    if (e != cudaSuccess) return e;
  }
  k_post<MC, R13><<<grid, kPostThreads, sm, st>>>(g, pz, tw_z, maps, phi, alpha, pa, out);
  return cudaGetLastError();
}

}  // namespace

size_t post_smem_bytes(const Geom& g, int nte) {
  const int mc = g.M <= 1 ? 1 : 2;
  return sizeof(float2) * (((g.nz + 1) & ~1) + (size_t)mc * kPostRB * g.nz + 2 * kPostRB * (size_t)(g.nz + 1) + 1) +
         sizeof(float) * (size_t)nte * kPostRB * g.nz;
}

cudaError_t launch_post(const Geom& g, const FftPlan& pz, const float2* tw_z, const float2* maps, const float* phi,
                        const float2* alpha, const int* te, int nte, int w, float* out, cudaStream_t st) {
  if (nte < 1 || nte > kMaxPostTe || g.M > 2) return cudaErrorInvalidValue;
  PostArgs pa{};
  for (int i = 0; i < nte; ++i) pa.te[i] = te[i];
  pa.nte = nte;
  pa.w = w;
  const size_t sm = post_smem_bytes(g, nte);
  dim3 grid((g.ny + kPostRB - 1) / kPostRB, g.S);
  const bool r13 = plan_has13(pz);
  if (g.M == 1) {
    if (r13) return post_go<1, true>(g, pz, tw_z, maps, phi, alpha, pa, out, grid, sm, st);
    return post_go<1, false>(g, pz, tw_z, maps, phi, alpha, pa, out, grid, sm, st);
  }
  if (r13) return post_go<2, true>(g, pz, tw_z, maps, phi, alpha, pa, out, grid, sm, st);
  return post_go<2, false>(g, pz, tw_z, maps, phi, alpha, pa, out, grid, sm, st);
}

}  // namespace t2sh
