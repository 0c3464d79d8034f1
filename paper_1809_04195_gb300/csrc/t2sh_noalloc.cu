// t2sh_normal_op_noalloc: the normal operator y = A^H A x for callers that cannot
// allocate device memory, for example code that runs where cudaMalloc is not allowed
// (inside a host callback or a stream-ordered region the caller does not own), or an
// embedding application that hands out all device memory itself and forbids libraries
// from allocating more.  It needs no plan: every intermediate (twiddle tables, the
// space-time kernel Psi, the sign-folded coil maps and the per-coil k-space
// intermediate) lives in one fixed-size device array defined in this file, which every
// GPU that loads the library holds until the process exits.  A bounded device wait that
// runs out is recorded in the array and reported by t2sh_noalloc_sync.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/t2sh.h"
#include "t2sh_plan.h"

namespace t2sh {
t2sh_status check_dims(const t2sh_dims* d);
bool fft_plan_for(int n, FftPlan& p);
void set_last_error(const char* msg);
}  // namespace t2sh

using namespace t2sh;

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 128;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// Layout of the first 256 bytes of the array, the same for every problem size:
//   int at byte 0        the bounded-wait flag: set by a kernel whose wait ran out, kept
//                        until t2sh_noalloc_sync reads and clears it
//   unsigned at 32..63   the eigenvalue reductions of the plan-time kernels, cleared by
//                        every call
// The per-call data (twiddles, Psi, maps, intermediate) follow from byte 256.
constexpr size_t kFlagOff = 0;
constexpr size_t kRedOff = 32;
constexpr size_t kHeader = 256;

// Device address of the array on the current device.  The first call on a device resolves
// it (cudaGetSymbolAddress, with that device current); later calls read the cached value.
t2sh_status scratch_base(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    set_last_error("t2sh_normal_op_noalloc: cudaGetDevice failed");
    return T2SH_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      set_last_error("t2sh_normal_op_noalloc: cudaGetSymbolAddress of the scratch array failed");
      return T2SH_ECUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  return T2SH_OK;
}

// exp(-2 pi i m / n) for m < n, in double, rounded to float
__global__ void k_twiddle_table(float2* out, int n) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < n) {
    double s, c;
    sincospi(-2.0 * (double)m / (double)n, &s, &c);
    out[m] = make_float2((float)c, (float)s);
  }
}

t2sh_status fail(t2sh_status st, const char* msg) {
  set_last_error(msg);
  return st;
}

}  // namespace

extern "C" size_t t2sh_noalloc_scratch_bytes(void) { return kScratchBytes; }

extern "C" t2sh_status t2sh_normal_op_noalloc(const t2sh_dims* dims, const float* phi, const uint8_t* mask,
                                              const void* maps, const void* x, void* y, void* stream) {
  t2sh_status s = check_dims(dims);
  if (s != T2SH_OK) return s;
  if (!phi || !mask || !maps || !x || !y) return fail(T2SH_EINVAL, "t2sh_normal_op_noalloc: NULL argument");
  if (dims->flags & T2SH_HOST_IO)
    return fail(T2SH_EINVAL, "t2sh_normal_op_noalloc: takes device pointers only (T2SH_HOST_IO not allowed)");
  const t2sh_dims& d = *dims;
  const size_t N = (size_t)d.ny * d.nz;
  const int P = d.nbasis * (d.nbasis + 1) / 2;
  const size_t off_twy = kHeader;
  const size_t off_twz = off_twy + up256(sizeof(float2) * d.ny);
  const size_t off_psi = off_twz + up256(sizeof(float2) * d.nz);
  const size_t off_maps = off_psi + up256(sizeof(float) * P * N);
  const size_t off_t = off_maps + up256(sizeof(float2) * (size_t)d.nslices * d.ncoils * d.nmaps * N);
  const size_t need = off_t + up256(sizeof(float2) * (size_t)d.nslices * d.ncoils * d.nbasis * N);
  if (need > kScratchBytes) {
    static thread_local char msg[192];
    snprintf(msg, sizeof(msg),
             "t2sh_normal_op_noalloc: needs %zu bytes of scratch, the static array holds %zu (64 MiB)", need,
             kScratchBytes);
    return fail(T2SH_EINVAL, msg);
  }
  FftPlan py{}, pz{};
  if (!fft_plan_for(d.ny, py) || !fft_plan_for(d.nz, pz))
    return fail(T2SH_EINVAL, "t2sh_normal_op_noalloc: no radix plan for ny, nz");

  unsigned char* base = nullptr;
  s = scratch_base(&base);
  if (s != T2SH_OK) return s;
  float2* tw_y = reinterpret_cast<float2*>(base + off_twy);
  float2* tw_z = reinterpret_cast<float2*>(base + off_twz);
  unsigned* red = reinterpret_cast<unsigned*>(base + kRedOff);
  float* psi = reinterpret_cast<float*>(base + off_psi);
  float2* maps_s = reinterpret_cast<float2*>(base + off_maps);
  float2* t = reinterpret_cast<float2*>(base + off_t);

  Geom g{};
  g.S = d.nslices; g.C = d.ncoils; g.M = d.nmaps; g.K = d.nbasis; g.T = d.nechoes;
  g.ny = d.ny; g.nz = d.nz; g.P = P;
  g.gsign = (((d.ny / 2) + (d.nz / 2)) & 1) ? -1.f : 1.f;
  g.inv_sqrt_n = (float)(1.0 / sqrt((double)N));
  g.colvar = d.precision == T2SH_MIXED_BF16 ? 3 : 0;
  g.err = reinterpret_cast<int*>(base + kFlagOff);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  cudaError_t e = cudaSuccess;
  k_twiddle_table<<<(d.ny + 255) / 256, 256, 0, st>>>(tw_y, d.ny);
  k_twiddle_table<<<(d.nz + 255) / 256, 256, 0, st>>>(tw_z, d.nz);
  e = cudaGetLastError();
  // the eigenvalue reductions of the plan-time kernels start from zero on every call; the
  // bounded-wait flag is left alone so that t2sh_noalloc_sync still sees an earlier timeout
  if (e == cudaSuccess) e = cudaMemsetAsync(red, 0, kHeader - kRedOff, st);
  if (e == cudaSuccess) e = launch_maps_prep(g, static_cast<const float2*>(maps), maps_s, red, st);
  if (e == cudaSuccess) e = launch_psi_build(g, phi, mask, psi, red + 1, st);
  if (e == cudaSuccess) e = launch_row(g, ROW_FWD, pz, tw_z, maps_s, static_cast<const float2*>(x), t, nullptr, st);
  if (e == cudaSuccess) e = launch_col(g, COL_NORMAL, py, tw_y, psi, nullptr, nullptr, t, t, st);
  if (e == cudaSuccess) e = launch_row(g, ROW_ADJ, pz, tw_z, maps_s, nullptr, t, static_cast<float2*>(y), st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(T2SH_ECUDA, cudaGetErrorString(e));
  }
  return T2SH_OK;
}

extern "C" t2sh_status t2sh_noalloc_sync(void* stream) {
  unsigned char* base = nullptr;
  t2sh_status s = scratch_base(&base);
  if (s != T2SH_OK) return s;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  int flag = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&flag, base + kFlagOff, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && flag) e = cudaMemset(base + kFlagOff, 0, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(T2SH_ECUDA, cudaGetErrorString(e));
  }
  if (flag)
    return fail(T2SH_ETIMEOUT,
                "t2sh_normal_op_noalloc: a bounded device wait ran out (a tile copy or tensor-core operation did not "
                "complete in time); the result of that call is not valid");
  return T2SH_OK;
}

extern "C" t2sh_status t2sh_noalloc_wait_selftest(uint64_t limit_ns, void* stream) {
  if (limit_ns < 1 || limit_ns > 1000000000ull)
    return fail(T2SH_EINVAL, "t2sh_noalloc_wait_selftest: limit_ns must be in [1, 1e9]");
  unsigned char* base = nullptr;
  t2sh_status s = scratch_base(&base);
  if (s != T2SH_OK) return s;
  cudaError_t e = launch_wait_selftest(reinterpret_cast<int*>(base + kFlagOff), (unsigned long long)limit_ns,
                                       static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(T2SH_ECUDA, cudaGetErrorString(e));
  }
  return T2SH_OK;
}
