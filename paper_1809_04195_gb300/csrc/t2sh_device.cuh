// Device building blocks of the T2 Shuffling solver: complex arithmetic, the
// register radix butterflies and an in-place shared-memory Stockham FFT over a batch
// of lines, and a Jacobi eigensolver for the small Hermitian Gram matrices of the LLR
// prox.  Included by the kernel translation units only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "t2sh_plan.h"

namespace t2sh {

// A translation unit that defines T2SH_PACKED_ADD before including this header gets the
// complex additions and subtractions of every butterfly as packed two-lane float32
// instructions (one instruction per complex value).  The arithmetic is the same per
// component; whether it pays depends on the kernel (measured faster for the row passes,
// slower for the TMA column pass), so it is chosen per translation unit.  The two forms
// live in different inline namespaces, so their definitions never collide.
#if defined(T2SH_PACKED_ADD)
inline namespace packed_add {
#else
inline namespace scalar_add {
#endif

// ---------------------------------------------------------------------------------
// complex float helpers (interleaved float2)
// ---------------------------------------------------------------------------------
#if defined(T2SH_PACKED_ADD)
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
#else
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
#endif
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
// a += b * c
__device__ __forceinline__ void cfma(float2& a, float2 b, float2 c) {
  a.x = fmaf(b.x, c.x, fmaf(-b.y, c.y, a.x));
  a.y = fmaf(b.x, c.y, fmaf(b.y, c.x, a.y));
}
// a += conj(b) * c
__device__ __forceinline__ void cfmac(float2& a, float2 b, float2 c) {
  a.x = fmaf(b.x, c.x, fmaf(b.y, c.y, a.x));
  a.y = fmaf(b.x, c.y, fmaf(-b.y, c.x, a.y));
}
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot_i(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
template <bool INV>
__device__ __forceinline__ float2 twiddle_mul(float2 a, float2 w) {  // w = exp(-2 pi i m / N)
  return INV ? cmulc(w, a) : cmul(a, w);
}

// ---------------------------------------------------------------------------------
// Radix-R DFTs in registers, X_k = sum_n x_n exp(-+2 pi i n k / R) (sign + for INV).
// Constants are exact trigonometric values written out.
// ---------------------------------------------------------------------------------
template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft3(float2* v) {
  const float c = -0.5f, s = 0.86602540378443865f;  // cos(2pi/3), sin(2pi/3)
  float2 t1 = cadd(v[1], v[2]);
  float2 t2 = make_float2(fmaf(c, t1.x, v[0].x), fmaf(c, t1.y, v[0].y));
  float2 t3 = cscale(csub(v[1], v[2]), s);  // s (x1 - x2)
  v[0] = cadd(v[0], t1);
  float2 r = rot_i<INV>(t3);  // -+ i s (x1 - x2)
  v[1] = cadd(t2, r);
  v[2] = csub(t2, r);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2* v) {
  float2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
  float2 c = cadd(v[1], v[3]), d = rot_i<INV>(csub(v[1], v[3]));
  v[0] = cadd(a, c);
  v[2] = csub(a, c);
  v[1] = cadd(b, d);
  v[3] = csub(b, d);
}

template <bool INV>
__device__ __forceinline__ void dft5(float2* v) {
  const float c1 = 0.30901699437494742f, c2 = -0.80901699437494742f;  // cos(2pi/5), cos(4pi/5)
  const float s1 = 0.95105651629515357f, s2 = 0.58778525229247313f;   // sin(2pi/5), sin(4pi/5)
  float2 u1 = cadd(v[1], v[4]), u2 = cadd(v[2], v[3]);
  float2 w1 = csub(v[1], v[4]), w2 = csub(v[2], v[3]);
  float2 x0 = v[0];
  float2 a1 = make_float2(x0.x + c1 * u1.x + c2 * u2.x, x0.y + c1 * u1.y + c2 * u2.y);
  float2 a2 = make_float2(x0.x + c2 * u1.x + c1 * u2.x, x0.y + c2 * u1.y + c1 * u2.y);
  float2 b1 = make_float2(s1 * w1.x + s2 * w2.x, s1 * w1.y + s2 * w2.y);
  float2 b2 = make_float2(s2 * w1.x - s1 * w2.x, s2 * w1.y - s1 * w2.y);
  float2 r1 = rot_i<INV>(b1), r2 = rot_i<INV>(b2);
  v[0] = cadd(x0, cadd(u1, u2));
  v[1] = cadd(a1, r1);
  v[4] = csub(a1, r1);
  v[2] = cadd(a2, r2);
  v[3] = csub(a2, r2);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  const float h = 0.70710678118654752f;
  float2 e[4] = {v[0], v[2], v[4], v[6]};
  float2 o[4] = {v[1], v[3], v[5], v[7]};
  dft4<INV>(e);
  dft4<INV>(o);
  // w8^k, k = 0..3: 1, (1 -+ i)/sqrt2, -+i, (-1 -+ i)/sqrt2
  float2 o1 = INV ? make_float2(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
                  : make_float2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
  float2 o2 = rot_i<INV>(o[2]);
  float2 o3 = INV ? make_float2(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
                  : make_float2(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
  v[0] = cadd(e[0], o[0]);
  v[4] = csub(e[0], o[0]);
  v[1] = cadd(e[1], o1);
  v[5] = csub(e[1], o1);
  v[2] = cadd(e[2], o2);
  v[6] = csub(e[2], o2);
  v[3] = cadd(e[3], o3);
  v[7] = csub(e[3], o3);
}

// 16 = 4 x 4 Cooley-Tukey: DFT_4 over n1 of x[4 n1 + n2] for each n2, twiddles
// w16^(n2 k1), DFT_4 over n2 -> X[k1 + 4 k2].  w16^4 = -+i is a swap; the others are
// constant complex multiplies (cos and sin of m pi / 8 written out).
template <bool INV>
__device__ __forceinline__ float2 cmul_cs(float2 v, float c, float s) {  // v * (c -+ i s)
  const float si = INV ? s : -s;
  return make_float2(v.x * c - v.y * si, v.x * si + v.y * c);
}
template <bool INV>
__device__ __forceinline__ void dft16(float2* v) {
  constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
  float2 a[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) a[n2][n1] = v[4 * n1 + n2];
    dft4<INV>(a[n2]);
  }
  // a[n2][k1] *= w16^(n2 k1), w16^m = cos(m pi / 8) -+ i sin(m pi / 8)
  a[1][1] = cmul_cs<INV>(a[1][1], c1, s1);   // m = 1
  a[1][2] = cmul_cs<INV>(a[1][2], h, h);     // m = 2
  a[1][3] = cmul_cs<INV>(a[1][3], s1, c1);   // m = 3
  a[2][1] = cmul_cs<INV>(a[2][1], h, h);     // m = 2
  a[2][2] = rot_i<INV>(a[2][2]);             // m = 4
  a[2][3] = cmul_cs<INV>(a[2][3], -h, h);    // m = 6
  a[3][1] = cmul_cs<INV>(a[3][1], s1, c1);   // m = 3
  a[3][2] = cmul_cs<INV>(a[3][2], -h, h);    // m = 6
  a[3][3] = cmul_cs<INV>(a[3][3], -c1, -s1); // m = 9
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 b[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
    dft4<INV>(b);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = b[k2];
  }
}

// 13-point DFT through the pair symmetry of the kernel: with u_n = x_n + x_(13-n) and
// w_n = x_n - x_(13-n) (n = 1..6), X_k = x_0 + sum_n cos(2 pi n k / 13) u_n -+ i sum_n
// sin(2 pi n k / 13) w_n and X_(13-k) the same with the other sign (k = 1..6).  The
// cosines and sines of 2 pi m / 13 are written out; the index n k mod 13 folds onto
// m <= 6 at compile time.
template <bool INV>
__device__ __forceinline__ void dft13(float2* v) {
  constexpr float C[7] = {1.0f, 0.88545602565320991f, 0.56806474673115592f, 0.12053668025532301f,
                          -0.35460488704253545f, -0.74851074817110119f, -0.97094181742605201f};
  constexpr float S[7] = {0.0f, 0.46472317204376851f, 0.82298386589365635f, 0.99270887409805397f,
                          0.93501624268541483f, 0.66312265824079519f, 0.23931566428755768f};
  float2 u[6], w[6];
#pragma unroll
  for (int n = 1; n <= 6; ++n) {
    u[n - 1] = cadd(v[n], v[13 - n]);
    w[n - 1] = csub(v[n], v[13 - n]);
  }
  const float2 x0 = v[0];
  float2 sum = x0;
#pragma unroll
  for (int n = 0; n < 6; ++n) sum = cadd(sum, u[n]);
  v[0] = sum;
#pragma unroll
  for (int k = 1; k <= 6; ++k) {
    float2 a = x0, b = make_float2(0.f, 0.f);
#pragma unroll
    for (int n = 1; n <= 6; ++n) {
      const int m = (n * k) % 13;
      const float cc = m <= 6 ? C[m] : C[13 - m];
      const float ss = m <= 6 ? S[m] : -S[13 - m];
      a.x = fmaf(cc, u[n - 1].x, a.x);
      a.y = fmaf(cc, u[n - 1].y, a.y);
      b.x = fmaf(ss, w[n - 1].x, b.x);
      b.y = fmaf(ss, w[n - 1].y, b.y);
    }
    // forward: X_k = a - i b, X_(13-k) = a + i b; inverse the other way round
    const float2 mib = make_float2(b.y, -b.x), pib = make_float2(-b.y, b.x);
    v[k] = cadd(a, INV ? pib : mib);
    v[13 - k] = cadd(a, INV ? mib : pib);
  }
}

// Good-Thomas (prime factor) DFT of length A*B with gcd(A, B) = 1: with input map
// n = (B n1 + A n2) mod AB and output map k = (B eA k1 + A eB k2) mod AB, where
// eA = B^-1 mod A and eB = A^-1 mod B, the length-AB DFT is a 2D A x B DFT with no
// twiddle factors.  Every index is a compile-time constant.
constexpr int inv_mod(int a, int m) {
  for (int x = 1; x < m; ++x)
    if ((a * x) % m == 1) return x;
  return 1;
}
template <int R, bool INV>
__device__ __forceinline__ void dft_r(float2* v);

template <int A, int B, bool INV>
__device__ __forceinline__ void dft_pfa(float2* v) {
  constexpr int N = A * B;
  constexpr int eA = inv_mod(B % A, A), eB = inv_mod(A % B, B);
  float2 c[B][A];
#pragma unroll
  for (int n2 = 0; n2 < B; ++n2) {
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) c[n2][n1] = v[(B * n1 + A * n2) % N];
    dft_r<A, INV>(c[n2]);
  }
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) {
    float2 d[B];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) d[n2] = c[n2][k1];
    dft_r<B, INV>(d);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) v[(B * eA * k1 + A * eB * k2) % N] = d[k2];
  }
}

template <int R, bool INV>
__device__ __forceinline__ void dft_r(float2* v) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) dft2<INV>(v[0], v[1]);
  else if constexpr (R == 3) dft3<INV>(v);
  else if constexpr (R == 4) dft4<INV>(v);
  else if constexpr (R == 5) dft5<INV>(v);
  else if constexpr (R == 6) dft_pfa<2, 3, INV>(v);
  else if constexpr (R == 8) dft8<INV>(v);
  else if constexpr (R == 10) dft_pfa<2, 5, INV>(v);
  else if constexpr (R == 12) dft_pfa<4, 3, INV>(v);
  else if constexpr (R == 13) dft13<INV>(v);
  else if constexpr (R == 15) dft_pfa<3, 5, INV>(v);
  else if constexpr (R == 16) dft16<INV>(v);
  else if constexpr (R == 20) dft_pfa<4, 5, INV>(v);
  else static_assert(R == 2, "unsupported radix");
}

// ---------------------------------------------------------------------------------
// In-place Stockham autosort FFT of `nbatch` lines of length p.n held in shared
// memory (line b at buf[b * ld], unit stride), natural order in and out, unnormalised.
// Each pass first pulls every butterfly's inputs into registers, synchronises, then
// writes its outputs, so one buffer suffices.  Consecutive threads take consecutive
// lines of the same butterfly: with ld odd the accesses are bank-conflict free and
// the twiddle read is a broadcast.  Requires nbatch * p.n <= kStage * blockDim.x.
//   tw[m] = exp(-2 pi i m / n), m < n (shared memory copy).
// ---------------------------------------------------------------------------------
constexpr int kStageRegs = 20;    // >= ceil(kStage / R) * R for the radices 2, 3, 4, 5, 8, 16
constexpr int kStageRegs13 = 26;  // with radix 13 (2 x 13): only plans that contain a radix-13 pass
constexpr int kStageBf = 8;     // >= ceil(kStage / R) for every radix used

template <int R, bool INV, int NV>
__device__ __forceinline__ void stockham_pass(float2* buf, int ld, int nbatch, int n, int ns, const float2* tw,
                                              float2 (&v)[NV], int (&dst)[kStageBf]) {
  constexpr int UMAX = (kStage + R - 1) / R;
  static_assert(UMAX * R <= NV && UMAX <= kStageBf, "staging registers");
  const int nbf = n / R;
  const int total = nbf * nbatch;
  const int tstride = n / (ns * R);
  const int nthr = blockDim.x;
#pragma unroll
  for (int u = 0; u < UMAX; ++u) {
    const int idx = threadIdx.x + u * nthr;
    dst[u] = -1;
    if (idx < total) {
      const int j = idx / nbatch;
      const int b = idx - j * nbatch;
      const float2* src = buf + b * ld + j;
#pragma unroll
      for (int r = 0; r < R; ++r) v[u * R + r] = src[r * nbf];
      const int jm = j % ns;
      if (ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[u * R + r] = twiddle_mul<INV>(v[u * R + r], tw[r * jm * tstride]);
      }
      dft_r<R, INV>(v + u * R);
      dst[u] = b * ld + (j - jm) * R + jm;
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < UMAX; ++u) {
    if (dst[u] >= 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) buf[dst[u] + r * ns] = v[u * R + r];
    }
  }
  __syncthreads();
}

// R13: the plan may contain a radix-13 pass (wider staging; a separate instantiation so
// that plans without one keep the smaller register footprint)
template <bool INV, bool R13 = false>
__device__ __forceinline__ void fft_lines(float2* buf, int ld, int nbatch, const FftPlan& p, const float2* tw) {
  constexpr int NV = R13 ? kStageRegs13 : kStageRegs;
  float2 v[NV];
  int dst[kStageBf];
  for (int q = 0; q < p.npass; ++q) {
    const int ns = p.ns[q];
    switch (p.radix[q]) {
      case 16: stockham_pass<16, INV, NV>(buf, ld, nbatch, p.n, ns, tw, v, dst); break;
      case 8: stockham_pass<8, INV, NV>(buf, ld, nbatch, p.n, ns, tw, v, dst); break;
      case 4: stockham_pass<4, INV, NV>(buf, ld, nbatch, p.n, ns, tw, v, dst); break;
      case 2: stockham_pass<2, INV, NV>(buf, ld, nbatch, p.n, ns, tw, v, dst); break;
      case 3: stockham_pass<3, INV, NV>(buf, ld, nbatch, p.n, ns, tw, v, dst); break;
      case 5: stockham_pass<5, INV, NV>(buf, ld, nbatch, p.n, ns, tw, v, dst); break;
      case 13:
        if constexpr (R13) stockham_pass<13, INV, NV>(buf, ld, nbatch, p.n, ns, tw, v, dst);
        break;
      default: break;
    }
  }
}

// ---------------------------------------------------------------------------------
// Cyclic Jacobi eigensolver for a Hermitian K x K matrix, real type T.  On entry
// (ar, ai) hold the full matrix; on exit the diagonal of ar holds the eigenvalues and
// (vr, vi) the eigenvectors as columns.  Each rotation first makes a_pq real with a
// diagonal phase, then applies the real Jacobi rotation with tan(theta) the smaller
// root of t^2 + 2 t theta - 1 = 0, theta = (a_qq - a_pp) / (2 a_pq).  Sweeps stop
// when the off-diagonal mass is below (eps^2) of the diagonal mass.
// ---------------------------------------------------------------------------------
template <typename T> struct JacobiTol;
// rel2: stop when off-diagonal^2 < rel2 * diagonal^2; pivot2: skip a rotation whose
// |a_pq|^2 is at most this (float32: below the normal range, where rsqrt is not exact)
template <> struct JacobiTol<double> { static constexpr double rel2 = 1e-30, pivot2 = 0.0; };
template <> struct JacobiTol<float> { static constexpr float rel2 = 1e-13f, pivot2 = 1e-36f; };

// Reciprocal square root and reciprocal for the rotation parameters.  Any unitary
// rotation that zeroes the pivot serves Jacobi, and the LLR step re-orthonormalises the
// eigenvectors and recomputes the eigenvalues afterwards, so the float32 variant takes
// the hardware approximations; float64 stays exact.
__device__ __forceinline__ float jac_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double jac_rsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float jac_rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double jac_rcp(double x) { return 1.0 / x; }

template <typename T, int K>
__device__ __forceinline__ void herm_jacobi(T (&ar)[K][K], T (&ai)[K][K], T (&vr)[K][K], T (&vi)[K][K],
                                            int max_sweeps) {
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int j = 0; j < K; ++j) {
      vr[i][j] = (i == j) ? T(1) : T(0);
      vi[i][j] = T(0);
    }
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    T off = 0, diag = 0;
#pragma unroll
    for (int p = 0; p < K; ++p) {
      diag += ar[p][p] * ar[p][p];
#pragma unroll
      for (int q = p + 1; q < K; ++q) off += ar[p][q] * ar[p][q] + ai[p][q] * ai[p][q];
    }
    if (!(off > JacobiTol<T>::rel2 * diag)) break;
#pragma unroll
    for (int p = 0; p < K - 1; ++p) {
#pragma unroll
      for (int q = p + 1; q < K; ++q) {
        const T xr = ar[p][q], xi = ai[p][q];
        const T r2 = xr * xr + xi * xi;
        if (r2 > JacobiTol<T>::pivot2) {
          const T ir = jac_rsqrt(r2), r = r2 * ir;
          // phase: column q *= d, row q *= conj(d), d = conj(a_pq) / |a_pq|
          const T dr = xr * ir, di = -xi * ir;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            if (k != q) {
              const T yr = ar[k][q] * dr - ai[k][q] * di;
              const T yi = ar[k][q] * di + ai[k][q] * dr;
              ar[k][q] = yr; ai[k][q] = yi;
              ar[q][k] = yr; ai[q][k] = -yi;
            }
          }
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const T yr = vr[k][q] * dr - vi[k][q] * di;
            const T yi = vr[k][q] * di + vi[k][q] * dr;
            vr[k][q] = yr; vi[k][q] = yi;
          }
          // a_pq is now the real r: real rotation on rows/columns p, q
          const T theta = (ar[q][q] - ar[p][p]) * (T(0.5) * ir);
          const T at = fabs(theta);
          T t;
          if (at > T(1e18)) {  // theta^2 would overflow float32: t = 1 / (2 |theta|) to first order
            t = T(0.5) / at;
          } else {
            const T u = at * at + T(1);
            t = jac_rcp(at + u * jac_rsqrt(u));
          }
          if (theta < T(0)) t = -t;
          const T c = jac_rsqrt(t * t + T(1));
          const T s = t * c;
          ar[p][p] -= t * r;
          ar[q][q] += t * r;
          ar[p][q] = T(0); ar[q][p] = T(0);
          ai[p][q] = T(0); ai[q][p] = T(0);
#pragma unroll
          for (int k = 0; k < K; ++k) {
            if (k != p && k != q) {
              const T akp_r = ar[k][p], akp_i = ai[k][p];
              const T akq_r = ar[k][q], akq_i = ai[k][q];
              const T nkp_r = c * akp_r - s * akq_r, nkp_i = c * akp_i - s * akq_i;
              const T nkq_r = s * akp_r + c * akq_r, nkq_i = s * akp_i + c * akq_i;
              ar[k][p] = nkp_r; ai[k][p] = nkp_i; ar[p][k] = nkp_r; ai[p][k] = -nkp_i;
              ar[k][q] = nkq_r; ai[k][q] = nkq_i; ar[q][k] = nkq_r; ai[q][k] = -nkq_i;
            }
          }
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const T vkp_r = vr[k][p], vkp_i = vi[k][p];
            const T vkq_r = vr[k][q], vkq_i = vi[k][q];
            vr[k][p] = c * vkp_r - s * vkq_r; vi[k][p] = c * vkp_i - s * vkq_i;
            vr[k][q] = s * vkp_r + c * vkq_r; vi[k][q] = s * vkp_i + c * vkq_i;
          }
        }
      }
    }
  }
}

// Round-robin (tournament) ordering of the K (K - 1) / 2 index pairs of an even K into
// K - 1 rounds of K / 2 disjoint pairs: in round r, i < K - 1 meets j = (r - i) mod (K - 1),
// and the i with j = i meets K - 1.
__host__ __device__ constexpr int jac_pair(int K, int r, int m, bool second) {
  int cnt = 0;
  for (int i = 0; i < K - 1; ++i) {
    const int j = ((r - i) % (K - 1) + (K - 1)) % (K - 1);
    int a = i, b = j;
    if (i == j) b = K - 1;
    else if (i > j) continue;
    if (cnt == m) return second ? b : a;
    ++cnt;
  }
  return 0;
}

// The same Jacobi method with each sweep taken as K - 1 rounds of K / 2 disjoint pivots
// (the parallel ordering): a round's rotations act on disjoint rows and columns, so they
// commute and their parameters all come from the matrix before the round.  One thread
// then works on K / 2 independent rotations at a time instead of one dependent chain.
// Same interface and stopping rule as herm_jacobi; K even.
template <typename T, int K>
__device__ __forceinline__ void herm_jacobi_rounds(T (&ar)[K][K], T (&ai)[K][K], T (&vr)[K][K], T (&vi)[K][K],
                                                   int max_sweeps) {
  static_assert(K % 2 == 0, "the round-robin ordering needs an even size");
  constexpr int H = K / 2;
#pragma unroll
  for (int i = 0; i < K; ++i)
#pragma unroll
    for (int j = 0; j < K; ++j) {
      vr[i][j] = (i == j) ? T(1) : T(0);
      vi[i][j] = T(0);
    }
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    T off = 0, diag = 0;
#pragma unroll
    for (int p = 0; p < K; ++p) {
      diag += ar[p][p] * ar[p][p];
#pragma unroll
      for (int q = p + 1; q < K; ++q) off += ar[p][q] * ar[p][q] + ai[p][q] * ai[p][q];
    }
    if (!(off > JacobiTol<T>::rel2 * diag)) break;
#pragma unroll
    for (int rd = 0; rd < K - 1; ++rd) {
      // parameters of the round's rotations, all from the matrix before the round
      T dr[H], di[H], rr[H], tt[H], cc[H], ss[H];
      bool on[H];
#pragma unroll
      for (int m = 0; m < H; ++m) {
        const int p = jac_pair(K, rd, m, false), q = jac_pair(K, rd, m, true);
        const T xr = ar[p][q], xi = ai[p][q];
        const T r2 = xr * xr + xi * xi;
        on[m] = r2 > JacobiTol<T>::pivot2;
        const T ir = on[m] ? jac_rsqrt(r2) : T(0);
        rr[m] = r2 * ir;
        dr[m] = on[m] ? xr * ir : T(1);  // phase d = conj(a_pq) / |a_pq|
        di[m] = -xi * ir;
        const T theta = (ar[q][q] - ar[p][p]) * (T(0.5) * ir);
        const T at = fabs(theta);
        T t;
        if (at > T(1e18)) {
          t = T(0.5) / at;
        } else {
          const T u = at * at + T(1);
          t = jac_rcp(at + u * jac_rsqrt(u));
        }
        if (theta < T(0)) t = -t;
        if (!on[m]) t = T(0);
        tt[m] = t;
        cc[m] = jac_rsqrt(t * t + T(1));
        ss[m] = t * cc[m];
      }
      // phases: column q *= d, row q *= conj(d); V column q *= d
#pragma unroll
      for (int m = 0; m < H; ++m) {
        const int q = jac_pair(K, rd, m, true);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if (k != q) {
            const T yr = ar[k][q] * dr[m] - ai[k][q] * di[m];
            const T yi = ar[k][q] * di[m] + ai[k][q] * dr[m];
            ar[k][q] = yr; ai[k][q] = yi;
            ar[q][k] = yr; ai[q][k] = -yi;
          }
          const T wr = vr[k][q] * dr[m] - vi[k][q] * di[m];
          const T wi = vr[k][q] * di[m] + vi[k][q] * dr[m];
          vr[k][q] = wr; vi[k][q] = wi;
        }
      }
      // real rotations on the now real pivots
#pragma unroll
      for (int m = 0; m < H; ++m) {
        const int p = jac_pair(K, rd, m, false), q = jac_pair(K, rd, m, true);
        const T c = cc[m], sn = ss[m];
        ar[p][p] -= tt[m] * rr[m];
        ar[q][q] += tt[m] * rr[m];
        ar[p][q] = T(0); ar[q][p] = T(0);
        ai[p][q] = T(0); ai[q][p] = T(0);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          if (k != p && k != q) {
            const T akp_r = ar[k][p], akp_i = ai[k][p];
            const T akq_r = ar[k][q], akq_i = ai[k][q];
            const T nkp_r = c * akp_r - sn * akq_r, nkp_i = c * akp_i - sn * akq_i;
            const T nkq_r = sn * akp_r + c * akq_r, nkq_i = sn * akp_i + c * akq_i;
            ar[k][p] = nkp_r; ai[k][p] = nkp_i; ar[p][k] = nkp_r; ai[p][k] = -nkp_i;
            ar[k][q] = nkq_r; ai[k][q] = nkq_i; ar[q][k] = nkq_r; ai[q][k] = -nkq_i;
          }
          const T vkp_r = vr[k][p], vkp_i = vi[k][p];
          const T vkq_r = vr[k][q], vkq_i = vi[k][q];
          vr[k][p] = c * vkp_r - sn * vkq_r; vi[k][p] = c * vkp_i - sn * vkq_i;
          vr[k][q] = sn * vkp_r + c * vkq_r; vi[k][q] = sn * vkp_i + c * vkq_i;
        }
      }
    }
  }
}
static_assert(jac_pair(4, 0, 0, false) == 0 && jac_pair(4, 0, 0, true) == 3 && jac_pair(4, 0, 1, false) == 1 &&
                  jac_pair(4, 0, 1, true) == 2 && jac_pair(4, 1, 0, true) == 1 && jac_pair(4, 1, 1, false) == 2 &&
                  jac_pair(4, 2, 0, true) == 2 && jac_pair(4, 2, 1, true) == 3,
              "round-robin pairs of 4");

// ---------------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async, completion per commit group).
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------------
// Singular-value soft threshold of one LLR block through its K x K Gram matrix:
// G = X^H X = V diag(lambda) V^H, sigma_i = sqrt(lambda_i), and the block's threshold
// weights W = V diag(max(1 - tau / sigma_i, 0)) V^H, so that X W = U max(Sigma - tau, 0) V^H
// (X V = U Sigma).  gram holds G as KC*KC floats: real part at [k][l] for k <= l, imaginary
// part of G_kl at [l][k] for l > k.  W_lk is written to w[l * KC + k].
// ---------------------------------------------------------------------------------
template <typename ET, int KC>
__device__ __forceinline__ void svt_weights(const float* gp, float tau, float2* w) {
  ET ar[KC][KC], ai[KC][KC], vr[KC][KC], vi[KC][KC];
#pragma unroll
  for (int k = 0; k < KC; ++k)
#pragma unroll
    for (int l = 0; l < KC; ++l) {
      if (k == l) { ar[k][l] = gp[k * KC + k]; ai[k][l] = ET(0); }
      else if (k < l) { ar[k][l] = gp[k * KC + l]; ai[k][l] = gp[l * KC + k]; }
      else { ar[k][l] = gp[l * KC + k]; ai[k][l] = -gp[k * KC + l]; }
    }
  // Five sweeps converge a 4 x 4 Hermitian matrix to working precision.
  herm_jacobi_rounds<ET, KC>(ar, ai, vr, vi, 5);
  // Rotations accumulated in float32 drift V away from orthonormal, and FISTA's
  // momentum amplifies the resulting error in W; so re-orthonormalise V (modified
  // Gram-Schmidt) and take each eigenvalue as the Rayleigh quotient v^H G v on the
  // original Gram matrix.
#pragma unroll
  for (int i = 0; i < KC; ++i) {
#pragma unroll
    for (int j = 0; j < i; ++j) {
      ET pr = ET(0), pi = ET(0);  // v_j^H v_i
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        pr += vr[k][j] * vr[k][i] + vi[k][j] * vi[k][i];
        pi += vr[k][j] * vi[k][i] - vi[k][j] * vr[k][i];
      }
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        const ET nr = vr[k][i] - (pr * vr[k][j] - pi * vi[k][j]);
        const ET ni = vi[k][i] - (pr * vi[k][j] + pi * vr[k][j]);
        vr[k][i] = nr;
        vi[k][i] = ni;
      }
    }
    ET nn = ET(0);
#pragma unroll
    for (int k = 0; k < KC; ++k) nn += vr[k][i] * vr[k][i] + vi[k][i] * vi[k][i];
    const ET inv = nn > ET(0) ? ET(1) / sqrt(nn) : ET(0);
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      vr[k][i] *= inv;
      vi[k][i] *= inv;
    }
  }
  ET f[KC];
#pragma unroll
  for (int i = 0; i < KC; ++i) {
    ET lam = ET(0);
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      ET gvr = ET(0), gvi = ET(0);  // (G v_i)_k
#pragma unroll
      for (int l = 0; l < KC; ++l) {
        ET gr_, gi_;
        if (k == l) { gr_ = gp[k * KC + k]; gi_ = ET(0); }
        else if (k < l) { gr_ = gp[k * KC + l]; gi_ = gp[l * KC + k]; }
        else { gr_ = gp[l * KC + k]; gi_ = -gp[k * KC + l]; }
        gvr += gr_ * vr[l][i] - gi_ * vi[l][i];
        gvi += gr_ * vi[l][i] + gi_ * vr[l][i];
      }
      lam += vr[k][i] * gvr + vi[k][i] * gvi;
    }
    const ET sig = sqrt(lam > ET(0) ? lam : ET(0));
    f[i] = (sig > (ET)tau) ? ET(1) - (ET)tau / sig : ET(0);
  }
#pragma unroll
  for (int l = 0; l < KC; ++l)
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      // W_lk = sum_i V_li f_i conj(V_ki)
      ET wr = ET(0), wi = ET(0);
#pragma unroll
      for (int i = 0; i < KC; ++i) {
        wr += f[i] * (vr[l][i] * vr[k][i] + vi[l][i] * vi[k][i]);
        wi += f[i] * (vi[l][i] * vr[k][i] - vr[l][i] * vi[k][i]);
      }
      w[l * KC + k] = make_float2((float)wr, (float)wi);
    }
}

// Exchange layouts of the two-stage line transforms (N = 16 R1): odd row strides keep
// half-warp accesses free of bank conflicts.
template <int R1>
struct ExLayout {
  static constexpr int SF = (R1 % 2) ? R1 : R1 + 1;  // forward: [j < 16][r1 < R1]
  static constexpr int SI = 17;                        // inverse: [j' < R1][r1 < 16]
  static constexpr int LINE = (16 * SF > R1 * SI) ? 16 * SF : R1 * SI;
};

// ---------------------------------------------------------------------------------
// Tensor-memory-access (TMA) bulk copies completing on shared-memory mbarriers.
// Every wait is bounded by the global timer: after kWaitNs the caller gets `false`,
// records an error and leaves the kernel instead of spinning forever.
// ---------------------------------------------------------------------------------
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, unsigned long long* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const void* tmap, unsigned long long* bar, int x, int y, int z,
                                            int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z), "r"(w)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
// wait for phase `phase` of the barrier; false if it has not completed within limit_ns
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned phase,
                                                  unsigned long long limit_ns = kWaitNs) {
  if (mbar_try_wait(bar, phase)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, phase))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}

// ---------------------------------------------------------------------------------
// Fifth-generation tensor cores (tcgen05): TMEM allocation, BF16 MMA from shared memory
// with FP32 accumulation in TMEM, completion through an mbarrier, TMEM -> register loads.
//
// Operand layout in shared memory: K-major without swizzle, i.e. 8-row x 16-byte core
// matrices stored as 128 contiguous bytes (row r at byte 16 r); core matrices adjacent
// along K are `lbo` bytes apart, 8-row groups along M (or N) are `sbo` bytes apart.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long umma_smem_desc(const void* p, unsigned lbo, unsigned sbo) {
  unsigned long long d = (unsigned long long)((smem_u32(p) >> 4) & 0x3FFFu);
  d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;  // descriptor version of the fifth-generation tensor cores; no swizzle
  return d;
}
// instruction descriptor: D FP32, A and B BF16, both K-major, M x N
__host__ __device__ constexpr unsigned umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}
__device__ __forceinline__ void tmem_alloc(unsigned* slot, unsigned ncols) {  // whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {  // whole warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// D (TMEM) = A B^T (+ D if acc): A M x 16, B N x 16 (K-major), one thread issues
__device__ __forceinline__ void umma_bf16(unsigned d_tmem, unsigned long long adesc, unsigned long long bdesc,
                                          unsigned idesc, unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
// arrive on `bar` once every MMA this thread issued before has completed
__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 16 / 32 consecutive FP32 columns of this thread's TMEM lane (lane = warp quarter base +
// lane id); the load and its wait are one statement so no use can be scheduled between
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32]) {
  unsigned r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
// round-to-nearest BF16 pair: `lo_elem` in the low 16 bits, `hi_elem` in the high
__device__ __forceinline__ unsigned pack_bf16x2(float lo_elem, float hi_elem) {
  unsigned d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi_elem), "f"(lo_elem));
  return d;
}
// complex value as two BF16 pairs (re, im): hi = bf16(v), lo = bf16(v - hi), so that
// hi + lo carries about 16 significant bits
__device__ __forceinline__ void split_bf16(float2 v, unsigned& hi, unsigned& lo) {
  hi = pack_bf16x2(v.x, v.y);
  lo = pack_bf16x2(v.x - __uint_as_float(hi << 16), v.y - __uint_as_float(hi & 0xFFFF0000u));
}

// sign (-1)^(a) as float
__device__ __forceinline__ float parity_sign(int a) { return (a & 1) ? -1.0f : 1.0f; }

}  // inline namespace
}  // namespace t2sh
