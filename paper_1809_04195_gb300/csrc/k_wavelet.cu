// Wavelet soft-threshold of the re-joined coefficient volume (Sec. II.C after Eq. 5, and
// Process TE of Sec. III.C): an orthonormal 3D Haar pyramid over (x = readout slice, y, z)
// of every basis-coefficient image, a complex soft threshold of every detail coefficient,
// and the inverse pyramid.
//
// In place, interleaved layout: level l (lattice stride s = 2^(l-1)) transforms every
// 2 x 2 x 2 cube of lattice points (2 s i + s dx, 2 s j + s dy, 2 s k + s dz) and stores the
// coefficient with low/high pattern (ex, ey, ez) at the cube point (dx, dy, dz) = (ex, ey, ez):
// the approximation lands on the cube origin, the next level's lattice.  Details are
// thresholded as they are formed; the coarsest level's inverse runs in the same pass and
// the finer inverses follow level by level.  The 2-point Haar pair (a + b, a - b) / sqrt(2)
// is its own inverse, so the inverse passes apply the same butterflies.  One thread per
// cube; at level 1 the z pairs are 16-byte loads of consecutive threads (coalesced).
#include <algorithm>

#include "t2sh_device.cuh"

namespace t2sh {

namespace {

enum { WV_FWD = 0, WV_FWD_INV = 1, WV_INV = 2 };

__device__ __forceinline__ void haar_pair(float2& a, float2& b) {
  constexpr float r = 0.70710678118654752f;  // 1 / sqrt(2)
  const float2 s = make_float2((a.x + b.x) * r, (a.y + b.y) * r);
  const float2 d = make_float2((a.x - b.x) * r, (a.y - b.y) * r);
  a = s;
  b = d;
}

// c max(1 - tau / |c|, 0)
__device__ __forceinline__ float2 soft_threshold(float2 c, float tau) {
  const float m = sqrtf(c.x * c.x + c.y * c.y);
  if (!(m > tau)) return make_float2(0.f, 0.f);
  const float f = 1.f - tau / m;
  return make_float2(c.x * f, c.y * f);
}

// the separable 3D pair transform: every z pair, then every y pair, then every x pair
__device__ __forceinline__ void haar_cube(float2 (&v)[2][2][2]) {
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) haar_pair(v[a][b][0], v[a][b][1]);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) haar_pair(v[a][0][b], v[a][1][b]);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) haar_pair(v[0][a][b], v[1][a][b]);
}

// a [S][MK][ny][nz]; level stride s; the volume sizes are multiples of 2 s
template <int MODE>
__global__ void k_haar(float2* a, int S, int MK, int ny, int nz, int s, float tau) {
  const int cx = S / (2 * s), cy = ny / (2 * s), cz = nz / (2 * s);
  const long long ncube = (long long)cx * MK * cy * cz;
  const long long sx = (long long)MK * ny * nz;  // stride of x
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncube;
       q += (long long)gridDim.x * blockDim.x) {
    long long r = q;
    const int l = (int)(r % cz);
    r /= cz;
    const int j = (int)(r % cy);
    r /= cy;
    const int mk = (int)(r % MK);
    const int i = (int)(r / MK);
    float2* base = a + (long long)(2 * s * i) * sx + (long long)mk * ny * nz + (long long)(2 * s * j) * nz + 2 * s * l;
    const long long ox = (long long)s * sx, oy = (long long)s * nz;
    float2 v[2][2][2];
#pragma unroll
    for (int dx = 0; dx < 2; ++dx)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const float2* p = base + dx * ox + dy * oy;
        if (s == 1) {
          const float4 w = *reinterpret_cast<const float4*>(p);
          v[dx][dy][0] = make_float2(w.x, w.y);
          v[dx][dy][1] = make_float2(w.z, w.w);
        } else {
          v[dx][dy][0] = p[0];
          v[dx][dy][1] = p[s];
        }
      }
    if (MODE != WV_INV) {
      haar_cube(v);
#pragma unroll
      for (int e = 1; e < 8; ++e) {
        float2& c = v[e >> 2][(e >> 1) & 1][e & 1];
        c = soft_threshold(c, tau);
      }
    }
    if (MODE != WV_FWD) haar_cube(v);
#pragma unroll
    for (int dx = 0; dx < 2; ++dx)
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        float2* p = base + dx * ox + dy * oy;
        if (s == 1) {
          *reinterpret_cast<float4*>(p) = make_float4(v[dx][dy][0].x, v[dx][dy][0].y, v[dx][dy][1].x, v[dx][dy][1].y);
        } else {
          p[0] = v[dx][dy][0];
          p[s] = v[dx][dy][1];
        }
      }
  }
}

template <int MODE>
cudaError_t haar_go(float2* a, int S, int MK, int ny, int nz, int s, float tau, cudaStream_t st) {
  const long long ncube = (long long)(S / (2 * s)) * MK * (ny / (2 * s)) * (nz / (2 * s));
  if (ncube == 0) return cudaSuccess;
  int nsm = 0;
  const cudaError_t e = sm_count(&nsm);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<long long>((ncube + 255) / 256, 8LL * nsm);
  k_haar<MODE><<<grid, 256, 0, st>>>(a, S, MK, ny, nz, s, tau);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_wavelet_denoise(const Geom& g, float2* alpha, float tau, int levels, cudaStream_t st) {
  const int MK = g.M * g.K;
  cudaError_t e = cudaSuccess;
  for (int l = 1; l < levels && e == cudaSuccess; ++l)
    e = haar_go<WV_FWD>(alpha, g.S, MK, g.ny, g.nz, 1 << (l - 1), tau, st);
  if (e == cudaSuccess) e = haar_go<WV_FWD_INV>(alpha, g.S, MK, g.ny, g.nz, 1 << (levels - 1), tau, st);
  for (int l = levels - 1; l >= 1 && e == cudaSuccess; --l)
    e = haar_go<WV_INV>(alpha, g.S, MK, g.ny, g.nz, 1 << (l - 1), tau, st);
  return e;
}

}  // namespace t2sh
