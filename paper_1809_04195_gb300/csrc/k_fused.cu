// One FISTA iteration's row work in a single kernel: one CTA per (slice, LLR band of
// 8 circularly shifted rows).  For its band it
//   A. accumulates A^H A z = sum_c S_c^H IDFT_z(t_c) over all coils (t_c already went
//      through the column pass DFT_y, Psi, IDFT_y), as the adjoint half of Algorithm 1;
//   B. takes the gradient step g = z - mu (A^H A z - A^H y), applies the singular-value
//      soft threshold to every 8 x 8 x K block of the band (the single-pass LLR of
//      Sec. IV.C: the random shift is folded into the row and column indices), and the
//      FISTA momentum z' = x' + beta (x' - x);
//   C. starts the next normal-operator application: t_c = DFT_z(S_c z') for all coils.
// The image rows of the band never leave the SM between A and C; only the per-coil
// k-space intermediate t and the FISTA vectors touch HBM.  M = 1, K <= 4, b = 8 and
// row lengths N = 16 R1 <= 192 (other shapes take the separate kernels).
#include "t2sh_device.cuh"

namespace t2sh {

constexpr int kBandRows = 8;

template <int N, typename ET>
__global__ void __launch_bounds__(512, 1) k_band_fused(Geom g, FistaArgs a, const float2* __restrict__ tw_g,
                                                      const float2* __restrict__ maps, float2* t, float2* x,
                                                      float2* z, const float2* __restrict__ aty) {
  constexpr int R1 = N / 16, SF = ExLayout<R1>::SF, LINE = ExLayout<R1>::LINE;
  constexpr int RB = kBandRows, NL = 4 * RB, NBZ = N / 8;
  extern __shared__ float2 smem[];
  __shared__ int rowoff[RB];
  const int ny = g.ny, NN = ny * N, K = g.K, C = g.C;
  const int s = blockIdx.y, band = blockIdx.x;
  const int rb = min(RB, ny - band * RB);
  const int j = threadIdx.x & 15, L = threadIdx.x >> 4, k = L >> 3, r = L & 7;
  const bool live = (k < K) && (r < rb);
  float2* tw = smem;
  float2* ex = tw + N;             // exchange [NL][LINE]; in phase B: Gram + threshold weights
  float2* mst = ex + NL * LINE;    // maps rows, double buffered [2][RB][N]
  float2* tst = mst + 2 * RB * N;  // t rows, double buffered [2][NL][N]; in phase B: G | Z
  float2* G = tst;                 // gradient-step image of the band [K][RB][N]
  float2* Z = tst + NL * N;        // z_{k+1} of the band [K][RB][N]
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
  if (threadIdx.x < RB) rowoff[threadIdx.x] = ((a.sy + band * RB + (int)threadIdx.x) % ny) * N;
  __syncthreads();
  const long long slice = (long long)s * K * NN;

  auto issue = [&](int c, int buf, bool with_t) {
    const float2* mp = maps + (long long)(s * C + c) * NN;
    float2* md = mst + buf * RB * N;
    for (int e2 = threadIdx.x; e2 < rb * N / 2; e2 += blockDim.x) {
      const int e = 2 * e2, rr = e / N, zz = e - rr * N;
      cp_async16(md + e, mp + rowoff[rr] + zz);
    }
    if (with_t) {
      const float2* tp = t + (long long)(s * C + c) * K * NN;
      float2* td = tst + buf * NL * N;
      for (int e2 = threadIdx.x; e2 < K * rb * N / 2; e2 += blockDim.x) {
        const int e = 2 * e2, kk = e / (rb * N), rem = e - kk * rb * N, rr = rem / N, zz = rem - rr * N;
        cp_async16(td + (kk * RB + rr) * N + zz, tp + (long long)kk * NN + rowoff[rr] + zz);
      }
    }
  };

  // ---------------- A: adjoint rows, accumulated over the coils -----------------------
  float2 acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = make_float2(0.f, 0.f);
  float2* exl = ex + L * LINE;
  if (!a.skip_adj) {
    issue(0, 0, true);
    cp_async_commit();
    for (int c = 0; c < C; ++c) {
      const int buf = c & 1;
      if (c + 1 < C) issue(c + 1, buf ^ 1, true);
      cp_async_commit();
      cp_async_wait<1>();
      __syncthreads();
      float2 av[R1];
      const float2* trow = tst + buf * NL * N + L * N;
#pragma unroll
      for (int q = 0; q < R1; ++q) av[q] = trow[j + 16 * q];
      dft_r<R1, true>(av);
#pragma unroll
      for (int q = 0; q < R1; ++q) exl[j * SF + q] = av[q];
      __syncthreads();
      if (j < R1 && live) {
        float2 b[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) b[q] = exl[q * SF + j];
#pragma unroll
        for (int q = 1; q < 16; ++q) b[q] = twiddle_mul<true>(b[q], tw[q * j]);
        dft16<true>(b);
        const float2* mrow = mst + buf * RB * N + r * N;
#pragma unroll
        for (int q = 0; q < 16; ++q) cfmac(acc[q], mrow[j + R1 * q], b[q]);
      }
      __syncthreads();
    }
    cp_async_wait<0>();
    __syncthreads();
  }

  // ---------------- B: gradient step, LLR soft threshold, momentum ---------------------
  if (j < R1 && live) {
    const long long gb = slice + (long long)k * NN + rowoff[r];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int zz = j + R1 * q;
      const float2 zv = z[gb + zz], av = aty[gb + zz];
      G[(k * RB + r) * N + zz] = make_float2(zv.x - a.mu * (acc[q].x - av.x), zv.y - a.mu * (acc[q].y - av.y));
    }
  }
  __syncthreads();
  float* gram = reinterpret_cast<float*>(ex);  // [NBZ][16]
  float2* wts = ex + NBZ * 8;                  // [NBZ][16]
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int blk = warp; blk < NBZ; blk += 16) {
      float gr[4][4];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) gr[p][q] = 0.f;
      for (int p = lane; p < rb * 8; p += 32) {
        const int rr = p >> 3;
        int zz = a.sz + blk * 8 + (p & 7);
        if (zz >= N) zz -= N;
        float2 xv[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) xv[l] = (l < K) ? G[(l * RB + rr) * N + zz] : make_float2(0.f, 0.f);
#pragma unroll
        for (int p_ = 0; p_ < 4; ++p_)
#pragma unroll
          for (int q_ = p_; q_ < 4; ++q_) {
            gr[p_][q_] = fmaf(xv[p_].x, xv[q_].x, fmaf(xv[p_].y, xv[q_].y, gr[p_][q_]));
            if (q_ > p_) gr[q_][p_] = fmaf(xv[p_].x, xv[q_].y, fmaf(-xv[p_].y, xv[q_].x, gr[q_][p_]));
          }
      }
#pragma unroll
      for (int p_ = 0; p_ < 4; ++p_)
#pragma unroll
        for (int q_ = 0; q_ < 4; ++q_)
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) gr[p_][q_] += __shfl_xor_sync(0xffffffffu, gr[p_][q_], o);
      if (lane == 0) {
#pragma unroll
        for (int p_ = 0; p_ < 4; ++p_)
#pragma unroll
          for (int q_ = 0; q_ < 4; ++q_) gram[blk * 16 + p_ * 4 + q_] = gr[p_][q_];
      }
    }
  }
  __syncthreads();
  for (int blk = threadIdx.x; blk < NBZ; blk += blockDim.x) svt_weights<ET, 4>(gram + blk * 16, a.tau, wts + blk * 16);
  __syncthreads();
  {
    const bool want_res = a.res != nullptr;
    float d2 = 0.f, x2 = 0.f;
    const int npx = K * rb * N;
    for (int e = threadIdx.x; e < npx; e += blockDim.x) {
      const int zz = e % N, rest = e / N, rr = rest % rb, kk = rest / rb;
      int zs = zz - a.sz;
      if (zs < 0) zs += N;
      const float2* w = wts + (zs >> 3) * 16;
      float2 o = make_float2(0.f, 0.f);
#pragma unroll
      for (int l = 0; l < 4; ++l)
        if (l < K) cfma(o, G[(l * RB + rr) * N + zz], w[l * 4 + kk]);
      const long long gi = slice + (long long)kk * NN + rowoff[rr] + zz;
      const float2 xo = x[gi];
      const float2 dx = csub(o, xo);
      const float2 zn = make_float2(o.x + a.beta * dx.x, o.y + a.beta * dx.y);
      x[gi] = o;
      z[gi] = zn;
      Z[(kk * RB + rr) * N + zz] = zn;
      if (want_res) {
        d2 = fmaf(dx.x, dx.x, fmaf(dx.y, dx.y, d2));
        x2 = fmaf(o.x, o.x, fmaf(o.y, o.y, x2));
      }
    }
    if (want_res) {
      double dd = d2, xx = x2;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        dd += __shfl_xor_sync(0xffffffffu, dd, o);
        xx += __shfl_xor_sync(0xffffffffu, xx, o);
      }
      if ((threadIdx.x & 31) == 0) {
        atomicAdd(a.res, dd);
        atomicAdd(a.res + 1, xx);
      }
    }
  }
  __syncthreads();
  if (a.skip_fwd) return;

  // ---------------- C: forward rows of z_{k+1} for every coil ---------------------------
  float2 xr[R1];
#pragma unroll
  for (int q = 0; q < R1; ++q) xr[q] = live ? Z[(k * RB + r) * N + j + 16 * q] : make_float2(0.f, 0.f);
  issue(0, 0, false);
  cp_async_commit();
  for (int c = 0; c < C; ++c) {
    const int buf = c & 1;
    if (c + 1 < C) issue(c + 1, buf ^ 1, false);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const float2* mrow = mst + buf * RB * N + r * N;
    float2 av[R1];
#pragma unroll
    for (int q = 0; q < R1; ++q) av[q] = cmul(mrow[j + 16 * q], xr[q]);
    dft_r<R1, false>(av);
#pragma unroll
    for (int q = 0; q < R1; ++q) exl[j * SF + q] = av[q];
    __syncthreads();
    if (j < R1 && live) {
      float2 b[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) b[q] = exl[q * SF + j];
#pragma unroll
      for (int q = 1; q < 16; ++q) b[q] = twiddle_mul<false>(b[q], tw[q * j]);
      dft16<false>(b);
      float2* tp = t + ((long long)(s * C + c) * K + k) * NN + rowoff[r] + j;
#pragma unroll
      for (int q = 0; q < 16; ++q) tp[R1 * q] = b[q];
    }
    __syncthreads();
  }
  cp_async_wait<0>();
}

template <int N>
static size_t band_smem() {
  constexpr int R1 = N / 16;
  return sizeof(float2) * ((size_t)N + 4 * kBandRows * ExLayout<R1>::LINE + 2 * (size_t)kBandRows * N +
                           2 * 4 * (size_t)kBandRows * N);
}

template <int N, typename ET>
static cudaError_t band_go(const Geom& g, const FistaArgs& a, const float2* tw, const float2* maps, float2* t,
                           float2* x, float2* z, const float2* aty, cudaStream_t st) {
  const size_t sm = band_smem<N>();
  {
    const cudaError_t e = smem_optin((const void*)k_band_fused<N, ET>, (int)sm);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((g.ny + kBandRows - 1) / kBandRows, g.S);
  k_band_fused<N, ET><<<grid, 512, sm, st>>>(g, a, tw, maps, t, x, z, aty);
  return cudaGetLastError();
}

bool band_fused_supported(const Geom& g, int block) {
  if (g.M != 1 || g.K > 4 || block != kBandRows) return false;
  switch (g.nz) {
    case 48: case 64: case 96: case 128: case 160: case 192: return true;
    default: return false;
  }
}

cudaError_t launch_band_fused(const Geom& g, const FistaArgs& a, const float2* tw_z, const float2* maps, float2* t,
                              float2* x, float2* z, const float2* aty, cudaStream_t st) {
  if (!band_fused_supported(g, a.b)) return cudaErrorNotSupported;
#define T2SH_BAND(NV)                                                             \
  case NV:                                                                        \
    return a.eig64 ? band_go<NV, double>(g, a, tw_z, maps, t, x, z, aty, st)      \
                   : band_go<NV, float>(g, a, tw_z, maps, t, x, z, aty, st);
  switch (g.nz) {
    T2SH_BAND(48)
    T2SH_BAND(64)
    T2SH_BAND(96)
    T2SH_BAND(128)
    T2SH_BAND(160)
    T2SH_BAND(192)
    default: return cudaErrorNotSupported;
  }
#undef T2SH_BAND
}

}  // namespace t2sh
