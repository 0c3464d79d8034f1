// Host runtime behind the C ABI of include/t2sh.h: argument validation, the plan's
// device workspace, plan-time precomputation (Psi, sign-folded maps, step, shift
// table) and the FISTA driver that enqueues the kernels of each iteration.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <atomic>
#include <tuple>
#include <vector>

#include "../../include/t2sh.h"
#include "t2sh_plan.h"

namespace t2sh {
size_t llr_smem_bytes(const Geom& g, int b);
}

using namespace t2sh;

namespace {

thread_local std::string g_err;

void set_err(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

#define T2SH_CK(call)                                                                \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      set_err("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return T2SH_ECUDA;                                                             \
    }                                                                                \
  } while (0)

#define T2SH_REQ(cond, ...)        \
  do {                             \
    if (!(cond)) {                 \
      set_err(__VA_ARGS__);        \
      return T2SH_EINVAL;          \
    }                              \
  } while (0)

// Stream-ordered pool for every plan buffer and the host-IO k-space stage, one per device,
// keeping its memory (release threshold at the maximum) so that plans made one after
// another reuse it instead of mapping fresh pages; t2sh_release_cached returns it.
cudaMemPool_t stage_pool() {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  uint64_t keep = ~0ull;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  pools[dev] = pool;
  return pool;
}

std::mutex g_launch_mu;
std::map<std::pair<const void*, int>, int> g_optin;            // (kernel, device) -> bytes
std::map<int, int> g_nsm;                                       // device -> SMs
std::map<std::tuple<const void*, int, int, size_t>, int> g_per; // (kernel, device, threads, smem) -> CTAs
}  // namespace

namespace t2sh {

cudaError_t smem_optin(const void* kernel, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_launch_mu);
  auto it = g_optin.find({kernel, dev});
  if (it != g_optin.end() && it->second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) g_optin[{kernel, dev}] = bytes;
  return e;
}

cudaError_t sm_count(int* n) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_launch_mu);
  auto it = g_nsm.find(dev);
  if (it != g_nsm.end()) {
    *n = it->second;
    return cudaSuccess;
  }
  e = cudaDeviceGetAttribute(n, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) g_nsm[dev] = *n;
  return e;
}

cudaError_t ctas_per_sm(const void* kernel, int threads, size_t smem, int* per) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_launch_mu);
  const auto key = std::make_tuple(kernel, dev, threads, smem);
  auto it = g_per.find(key);
  if (it != g_per.end()) {
    *per = it->second;
    return cudaSuccess;
  }
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, kernel, threads, smem);
  if (e != cudaSuccess) return e;
  if (*per < 1) *per = 1;
  g_per[key] = *per;
  return cudaSuccess;
}
}  // namespace t2sh

namespace {

// SplitMix64 (Steele, Lea & Flood 2014): output number i+1 of the stream from `seed`.
uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t zz = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  zz = (zz ^ (zz >> 30)) * 0xBF58476D1CE4E5B9ull;
  zz = (zz ^ (zz >> 27)) * 0x94D049BB133111EBull;
  return zz ^ (zz >> 31);
}

// sizes the FFT passes cover: products of 2, 3, 5 and 13 (the paper's 260 = 4 * 5 * 13)
bool smooth_ok(int n) {
  for (int p : {2, 3, 5, 13})
    while (n % p == 0) n /= p;
  return n == 1;
}

// Radix plan: as many radix-16 passes as divide n, then 8, 4, 2, 5, 3, 13.
bool make_fft_plan(int n, FftPlan& p) {
  p.n = n;
  p.npass = 0;
  int m = n, ns = 1;
  auto add = [&](int r) {
    if (p.npass >= kMaxPass) return false;
    p.radix[p.npass] = r;
    p.ns[p.npass] = ns;
    ns *= r;
    m /= r;
    ++p.npass;
    return true;
  };
  while (m % 16 == 0)
    if (!add(16)) return false;
  for (int r : {8, 4, 2, 5, 3, 13})
    while (m % r == 0)
      if (!add(r)) return false;
  return m == 1;
}

size_t cbytes(long long n) { return (size_t)n * sizeof(float2); }

struct Footprint {
  size_t maps, psi, phi, mask, vec, t, tw, shifts, red;
  size_t total() const { return maps + psi + phi + mask + 4 * vec + t + tw + shifts + red; }
};

Footprint footprint(const t2sh_dims& d) {
  const long long N = (long long)d.ny * d.nz;
  const int P = d.nbasis * (d.nbasis + 1) / 2;
  Footprint f;
  f.maps = cbytes((long long)d.nslices * d.ncoils * d.nmaps * N);
  f.psi = sizeof(float) * P * N;
  f.phi = sizeof(float) * d.nechoes * d.nbasis;
  f.mask = (size_t)d.nechoes * N;
  f.vec = cbytes((long long)d.nslices * d.nmaps * d.nbasis * N);
  f.t = cbytes((long long)d.nslices * d.ncoils * d.nbasis * N);
  f.tw = cbytes(d.ny + d.nz);
  f.shifts = 0;
  f.red = sizeof(double) * 2 * (size_t)(d.iters > 0 ? d.iters : 1) + 64;
  return f;
}

t2sh_status validate(const t2sh_dims* d) {
  T2SH_REQ(d != nullptr, "dims is NULL");
  T2SH_REQ(d->ny >= 8 && d->nz >= 8 && d->ny <= 512 && d->nz <= 512, "ny, nz must be in [8, 512] (got %d, %d)",
           d->ny, d->nz);
  T2SH_REQ(d->ny % 2 == 0 && d->nz % 2 == 0, "ny, nz must be even (centred FFT)");
  T2SH_REQ(smooth_ok(d->ny) && smooth_ok(d->nz), "ny, nz must be products of 2, 3, 5 and 13");
  T2SH_REQ(d->ncoils >= 1 && d->ncoils <= 1024, "ncoils out of range");
  T2SH_REQ(d->nmaps >= 1 && d->nmaps <= kMaxM, "nmaps must be 1 or 2");
  T2SH_REQ(d->nbasis >= 1 && d->nbasis <= kMaxK, "nbasis must be in [1, 8]");
  T2SH_REQ(d->nechoes >= d->nbasis && d->nechoes <= 4096, "nechoes must be in [nbasis, 4096]");
  T2SH_REQ(d->nslices >= 1 && d->nslices <= 65535, "nslices must be in [1, 65535]");
  T2SH_REQ(d->block >= 1 && d->block <= kMaxBlock, "block must be in [1, 16]");
  T2SH_REQ(d->iters >= 0, "iters must be >= 0");
  T2SH_REQ(std::isfinite(d->lambda) && d->lambda >= 0.f, "lambda must be finite and >= 0");
  T2SH_REQ(std::isfinite(d->step), "step must be finite");
  T2SH_REQ(d->precision == T2SH_FP32 || d->precision == T2SH_MIXED_BF16, "precision must be T2SH_FP32 or T2SH_MIXED_BF16");
  T2SH_REQ((d->flags & ~(T2SH_NO_SHIFT | T2SH_HOST_IO | T2SH_EIG_FP64 | T2SH_FUSED_ROWS)) == 0,
           "unknown flag bits");
  Geom g{};
  g.M = d->nmaps; g.K = d->nbasis; g.nz = d->nz;
  if (llr_smem_bytes(g, d->block) > 200 * 1024) {
    set_err("LLR band of %d x %d x %d x %d does not fit shared memory", d->nmaps, d->nbasis, d->block, d->nz);
    return T2SH_EUNSUPPORTED;
  }
  return T2SH_OK;
}

}  // namespace

// Shared with the allocation-free entry point (t2sh_noalloc.cu).
namespace t2sh {
t2sh_status check_dims(const t2sh_dims* d) { return validate(d); }
bool fft_plan_for(int n, FftPlan& p) { return make_fft_plan(n, p); }
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace t2sh

struct t2sh_plan_s {
  t2sh_dims d{};
  cudaStream_t st = nullptr;
  bool host_io = false;
  Geom g{};
  FftPlan py{}, pz{};
  float2* tw_y = nullptr;
  float2* tw_z = nullptr;
  float* phi = nullptr;
  uint8_t* mask = nullptr;
  float* psi = nullptr;
  float2* maps = nullptr;
  float2* x = nullptr;
  float2* z = nullptr;
  float2* aty = nullptr;
  float2* grad = nullptr;
  float2* t = nullptr;
  double* res = nullptr;
  unsigned* red = nullptr;
  void* stage = nullptr;  // host-IO staging of k-space input (from stage_pool(), stream-ordered)
  cudaStream_t cs = nullptr;           // copy stream of the pipelined host-IO solve
  std::vector<cudaEvent_t> cev;        // its events
  size_t stage_bytes = 0;
  std::vector<int32_t> shifts;
  float mu = 1.f;
  std::vector<std::pair<void*, bool>> allocs;  // (pointer, from the stage pool)
  // resumable FISTA state (t2sh_solve_begin / _iterate / _end)
  bool begun = false;
  int iter_done = 0;
  double tk = 1.0;
  bool record_res = false;
  bool fused_rows = false;  // tunable: fused band kernel for the row work
  // kernel timing (t2sh_timing_*)
  static constexpr int kClasses = 9;
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
  size_t ev_next = 0;
  int64_t launches[kClasses] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  // ADMM state (allocated on the first t2sh_solve_admm): scaled dual u, CG residual and
  // direction, per-slice float64 accumulators rr[3][S] and pq[S]
  float2* u = nullptr;
  float2* cg_r = nullptr;
  float2* cg_p = nullptr;
  double* cg_red = nullptr;
  // data-term diagnostic (t2sh_objective, allocated on its first call): per-slice float64
  // accumulators [3][S] and, for host-buffer plans, a device copy of the evaluated x
  double* obj = nullptr;
  float2* ov = nullptr;

  // Plan buffers come from the stage pool in the plan stream's order (plain cudaMalloc if
  // the pool is unavailable).  A pool allocation that fails is retried once after the
  // pool's unused memory has been returned.
  template <typename T>
  t2sh_status alloc(T** p, size_t bytes) {
    void* q = nullptr;
    const size_t b = bytes ? bytes : 16;
    cudaMemPool_t pool = stage_pool();
    cudaError_t e = pool ? cudaMallocFromPoolAsync(&q, b, pool, st) : cudaMalloc(&q, b);
    if (e != cudaSuccess && pool) {
      cudaGetLastError();
      cudaStreamSynchronize(st);
      cudaMemPoolTrimTo(pool, 0);
      e = cudaMallocFromPoolAsync(&q, b, pool, st);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_err("allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
      return T2SH_ENOMEM;
    }
    allocs.emplace_back(q, pool != nullptr);
    *p = static_cast<T*>(q);
    return T2SH_OK;
  }
  ~t2sh_plan_s() {
    if (cs) cudaStreamSynchronize(cs);
    cudaStreamSynchronize(st);
    for (cudaEvent_t e : cev) cudaEventDestroy(e);
    if (cs) cudaStreamDestroy(cs);
    bool pooled = false;
    for (auto& a : allocs) {
      if (a.second) {
        cudaFreeAsync(a.first, st);
        pooled = true;
      } else {
        cudaFree(a.first);
      }
    }
    if (pooled) cudaStreamSynchronize(st);
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
  }
  cudaEvent_t next_event() {
    if (ev_next == ev_pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      ev_pool.push_back(e);
    }
    return ev_pool[ev_next++];
  }
};

namespace {
// Brackets one kernel launch with events when the plan records timings.
struct KTimer {
  t2sh_plan_s* p;
  int cls;
  cudaEvent_t a = nullptr;
  KTimer(t2sh_plan_s* p_, int c) : p(p_), cls(c) {
    p->launches[cls]++;
    if (p->timing) {
      a = p->next_event();
      if (a) cudaEventRecord(a, p->st);
    }
  }
  ~KTimer() {
    if (p->timing && a) {
      cudaEvent_t b = p->next_event();
      if (b) {
        cudaEventRecord(b, p->st);
        p->ev_used.push_back({cls, {a, b}});
      }
    }
  }
};
enum { KC_ROW_FWD = 0, KC_ROW_ADJ = 1, KC_COL = 2, KC_LLR = 3, KC_PLAN = 4, KC_PROJ = 5, KC_BAND = 6, KC_CG = 7, KC_POST = 8 };
}  // namespace

namespace {

t2sh_status normal_op(t2sh_plan_t p, const float2* x, float2* y) {
  { KTimer k(p, KC_ROW_FWD); T2SH_CK(launch_row(p->g, ROW_FWD, p->pz, p->tw_z, p->maps, x, p->t, nullptr, p->st)); }
  { KTimer k(p, KC_COL); T2SH_CK(launch_col(p->g, COL_NORMAL, p->py, p->tw_y, p->psi, p->phi, p->mask, p->t, p->t, p->st)); }
  { KTimer k(p, KC_ROW_ADJ); T2SH_CK(launch_row(p->g, ROW_ADJ, p->pz, p->tw_z, p->maps, nullptr, p->t, y, p->st)); }
  return T2SH_OK;
}

// A^H y for device k-space in either form, result in x.
t2sh_status adjoint_data(t2sh_plan_t p, const void* y, int32_t kform, float2* x) {
  const float2* proj = static_cast<const float2*>(y);
  if (kform == T2SH_KSPACE_TE) {
    KTimer k(p, KC_PROJ);
    T2SH_CK(launch_project(p->g, p->phi, p->mask, static_cast<const float2*>(y), p->t, p->st));
    proj = p->t;
  }
  { KTimer k(p, KC_COL); T2SH_CK(launch_col(p->g, COL_ADJ_DATA, p->py, p->tw_y, p->psi, p->phi, p->mask, proj, p->t, p->st)); }
  { KTimer k(p, KC_ROW_ADJ); T2SH_CK(launch_row(p->g, ROW_ADJ, p->pz, p->tw_z, p->maps, nullptr, p->t, x, p->st)); }
  return T2SH_OK;
}

size_t kspace_bytes(const t2sh_dims& d, int32_t kform) {
  const long long N = (long long)d.ny * d.nz;
  return cbytes((long long)d.nslices * d.ncoils * (kform == T2SH_KSPACE_TE ? d.nechoes : d.nbasis) * N);
}

}  // namespace

extern "C" {

int32_t t2sh_version(void) { return 100; }

const char* t2sh_last_error(void) { return g_err.c_str(); }

t2sh_status t2sh_shifts(uint64_t seed, int32_t iters, int32_t block, int32_t* out) {
  T2SH_REQ(out != nullptr || iters == 0, "out is NULL");
  T2SH_REQ(iters >= 0 && block >= 1, "iters >= 0 and block >= 1 required");
  for (int32_t i = 0; i < iters; ++i) {
    const uint64_t h = splitmix64_at(seed, (uint64_t)i);
    out[2 * i] = (int32_t)((h & 0xFFFFFFFFull) % (uint64_t)block);
    out[2 * i + 1] = (int32_t)((h >> 32) % (uint64_t)block);
  }
  return T2SH_OK;
}

t2sh_status t2sh_workspace_bytes(const t2sh_dims* dims, size_t* bytes) {
  t2sh_status s = validate(dims);
  if (s != T2SH_OK) return s;
  T2SH_REQ(bytes != nullptr, "bytes is NULL");
  *bytes = footprint(*dims).total();
  return T2SH_OK;
}

t2sh_status t2sh_plan(const t2sh_dims* dims, const float* phi, const uint8_t* mask, const void* maps, void* stream,
                      t2sh_plan_t* out) {
  if (out) *out = nullptr;
  t2sh_status s = validate(dims);
  if (s != T2SH_OK) return s;
  T2SH_REQ(out && phi && mask && maps, "NULL argument");
  t2sh_plan_s* p = new (std::nothrow) t2sh_plan_s();
  if (!p) {
    set_err("host allocation failed");
    return T2SH_ENOMEM;
  }
  p->d = *dims;
  p->st = static_cast<cudaStream_t>(stream);
  p->host_io = (dims->flags & T2SH_HOST_IO) != 0;
  const t2sh_dims& d = p->d;
  Geom& g = p->g;
  g.S = d.nslices; g.C = d.ncoils; g.M = d.nmaps; g.K = d.nbasis; g.T = d.nechoes;
  g.ny = d.ny; g.nz = d.nz; g.P = d.nbasis * (d.nbasis + 1) / 2;
  g.gsign = (((d.ny / 2) + (d.nz / 2)) & 1) ? -1.f : 1.f;
  g.inv_sqrt_n = (float)(1.0 / std::sqrt((double)d.ny * d.nz));
  g.colvar = d.precision == T2SH_MIXED_BF16 ? 3 : 0;
  p->fused_rows = (d.flags & T2SH_FUSED_ROWS) != 0;
  if (!make_fft_plan(d.ny, p->py) || !make_fft_plan(d.nz, p->pz)) {
    delete p;
    set_err("no radix plan for ny=%d nz=%d", d.ny, d.nz);
    return T2SH_EINVAL;
  }
  const Footprint f = footprint(d);
#define ALLOC(ptr, bytes)                   \
  do {                                      \
    t2sh_status a_ = p->alloc(&(ptr), (bytes)); \
    if (a_ != T2SH_OK) {                    \
      delete p;                             \
      return a_;                            \
    }                                       \
  } while (0)
  ALLOC(p->maps, f.maps);
  ALLOC(p->psi, f.psi);
  ALLOC(p->phi, f.phi);
  ALLOC(p->mask, f.mask);
  ALLOC(p->x, f.vec);
  ALLOC(p->z, f.vec);
  ALLOC(p->aty, f.vec);
  ALLOC(p->grad, f.vec);
  ALLOC(p->t, f.t);
  ALLOC(p->tw_y, cbytes(d.ny));
  ALLOC(p->tw_z, cbytes(d.nz));
  ALLOC(p->res, sizeof(double) * 2 * (size_t)(d.iters > 0 ? d.iters : 1));
  ALLOC(p->red, 64);
#undef ALLOC
  g.err = reinterpret_cast<int*>(p->red + 8);
  // twiddles exp(-2 pi i m / n), computed in double
  std::vector<float2> tw(std::max(d.ny, d.nz));
  auto fill_tw = [&](int n) {
    for (int m = 0; m < n; ++m) {
      const double a = -2.0 * M_PI * (double)m / (double)n;
      tw[m] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
  };
#define FAIL_CK(call)                                                                                 \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      set_err("%s failed: %s", #call, cudaGetErrorString(e_));                                      \
      delete p;                                                                                     \
      return T2SH_ECUDA;                                                                            \
    }                                                                                               \
  } while (0)
  fill_tw(d.ny);
  FAIL_CK(cudaMemcpyAsync(p->tw_y, tw.data(), cbytes(d.ny), cudaMemcpyHostToDevice, p->st));
  FAIL_CK(cudaStreamSynchronize(p->st));
  fill_tw(d.nz);
  FAIL_CK(cudaMemcpyAsync(p->tw_z, tw.data(), cbytes(d.nz), cudaMemcpyHostToDevice, p->st));
  const cudaMemcpyKind kind = p->host_io ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  FAIL_CK(cudaMemcpyAsync(p->phi, phi, f.phi, kind, p->st));
  FAIL_CK(cudaMemcpyAsync(p->mask, mask, f.mask, kind, p->st));
  const float2* maps_src = static_cast<const float2*>(maps);
  if (p->host_io) {
    FAIL_CK(cudaMemcpyAsync(p->maps, maps, f.maps, kind, p->st));
    maps_src = p->maps;
  }
  FAIL_CK(cudaMemsetAsync(p->red, 0, 64, p->st));
  FAIL_CK(launch_maps_prep(g, maps_src, p->maps, p->red, p->st));
  FAIL_CK(launch_psi_build(g, p->phi, p->mask, p->psi, p->red + 1, p->st));
  unsigned bits[2];
  FAIL_CK(cudaMemcpyAsync(bits, p->red, sizeof(bits), cudaMemcpyDeviceToHost, p->st));
  FAIL_CK(cudaStreamSynchronize(p->st));
#undef FAIL_CK
  float lam_s, lam_psi;
  std::memcpy(&lam_s, &bits[0], 4);
  std::memcpy(&lam_psi, &bits[1], 4);
  const double L = (double)lam_s * (double)lam_psi;
  p->mu = d.step > 0.f ? d.step : (L > 0.0 ? (float)(1.0 / L) : 1.f);
  p->shifts.assign(2 * (size_t)d.iters, 0);
  if (!(d.flags & T2SH_NO_SHIFT)) t2sh_shifts(d.seed, d.iters, d.block, p->shifts.data());
  *out = p;
  return T2SH_OK;
}

t2sh_status t2sh_destroy(t2sh_plan_t p) {
  if (!p) return T2SH_OK;
  cudaStreamSynchronize(p->st);
  if (p->stage) {
    cudaFreeAsync(p->stage, p->st);
    cudaStreamSynchronize(p->st);
  }
  delete p;
  return T2SH_OK;
}

t2sh_status t2sh_release_cached(void) {
  cudaMemPool_t pool = stage_pool();
  if (!pool) return T2SH_OK;
  T2SH_CK(cudaMemPoolTrimTo(pool, 0));
  return T2SH_OK;
}

t2sh_status t2sh_timing_enable(t2sh_plan_t p, int32_t enable) {
  T2SH_REQ(p, "NULL plan");
  if (enable) {
    T2SH_CK(cudaStreamSynchronize(p->st));
    p->ev_used.clear();
    p->ev_next = 0;
    for (int i = 0; i < t2sh_plan_s::kClasses; ++i) p->launches[i] = 0;
  }
  p->timing = enable != 0;
  return T2SH_OK;
}

t2sh_status t2sh_timing_read(t2sh_plan_t p, int32_t cls, int64_t* launches, double* ms) {
  T2SH_REQ(p && launches && ms, "NULL argument");
  T2SH_REQ(cls >= 0 && cls < t2sh_plan_s::kClasses, "bad kernel class %d", cls);
  T2SH_CK(cudaStreamSynchronize(p->st));
  double tot = 0.0;
  for (auto& u : p->ev_used) {
    if (u.first != cls) continue;
    float m = 0.f;
    T2SH_CK(cudaEventElapsedTime(&m, u.second.first, u.second.second));
    tot += m;
  }
  *launches = p->launches[cls];
  *ms = tot;
  return T2SH_OK;
}

t2sh_status t2sh_configure(t2sh_plan_t p, int32_t col_variant, int32_t fused_rows) {
  T2SH_REQ(p, "NULL plan");
  T2SH_REQ(col_variant >= 0 && col_variant <= 4, "col_variant must be in [0, 4]");
  T2SH_REQ(!p->begun || p->iter_done == p->d.iters, "configure must not interrupt a solve in progress");
  p->g.colvar = col_variant;
  p->fused_rows = fused_rows != 0;
  return T2SH_OK;
}

t2sh_status t2sh_sync(t2sh_plan_t p) {
  T2SH_REQ(p, "NULL plan");
  T2SH_CK(cudaStreamSynchronize(p->st));
  int flag = 0;
  T2SH_CK(cudaMemcpy(&flag, p->g.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    T2SH_CK(cudaMemset(p->g.err, 0, sizeof(int)));
    set_err("a bounded device wait ran out (a copy or tensor-core operation did not complete in time)");
    return T2SH_ETIMEOUT;
  }
  return T2SH_OK;
}

t2sh_status t2sh_wait_selftest(t2sh_plan_t p, uint64_t limit_ns) {
  T2SH_REQ(p, "NULL plan");
  T2SH_REQ(limit_ns >= 1 && limit_ns <= 1000000000ull, "limit_ns must be in [1, 1e9]");
  T2SH_CK(launch_wait_selftest(p->g.err, (unsigned long long)limit_ns, p->st));
  return T2SH_OK;
}

t2sh_status t2sh_get_step(t2sh_plan_t p, float* step) {
  T2SH_REQ(p && step, "NULL argument");
  *step = p->mu;
  return T2SH_OK;
}

t2sh_status t2sh_forward(t2sh_plan_t p, const void* x, void* y, int32_t kform) {
  T2SH_REQ(p && x && y, "NULL argument");
  T2SH_REQ(kform == T2SH_KSPACE_TE || kform == T2SH_KSPACE_PROJ, "bad kform %d", kform);
  { KTimer k(p, KC_ROW_FWD); T2SH_CK(launch_row(p->g, ROW_FWD, p->pz, p->tw_z, p->maps, static_cast<const float2*>(x), p->t, nullptr, p->st)); }
  { KTimer k(p, KC_COL); T2SH_CK(launch_col(p->g, kform == T2SH_KSPACE_TE ? COL_FWD_TE : COL_FWD_PROJ, p->py, p->tw_y, p->psi, p->phi,
                     p->mask, p->t, static_cast<float2*>(y), p->st)); }
  return T2SH_OK;
}

t2sh_status t2sh_adjoint(t2sh_plan_t p, const void* y, int32_t kform, void* x) {
  T2SH_REQ(p && x && y, "NULL argument");
  T2SH_REQ(kform == T2SH_KSPACE_TE || kform == T2SH_KSPACE_PROJ, "bad kform %d", kform);
  return adjoint_data(p, y, kform, static_cast<float2*>(x));
}

t2sh_status t2sh_normal_op(t2sh_plan_t p, const void* x, void* y) {
  T2SH_REQ(p && x && y, "NULL argument");
  return normal_op(p, static_cast<const float2*>(x), static_cast<float2*>(y));
}

t2sh_status t2sh_llr_prox(t2sh_plan_t p, void* x, float tau, int32_t sy, int32_t sz) {
  T2SH_REQ(p && x, "NULL argument");
  T2SH_REQ(std::isfinite(tau) && tau >= 0.f, "tau must be finite and >= 0");
  T2SH_REQ(sy >= 0 && sz >= 0 && sy < p->d.block && sz < p->d.block, "shift must be in [0, block)");
  FistaArgs a{};
  a.mu = 0.f; a.tau = tau; a.beta = 0.f; a.sy = sy; a.sz = sz; a.b = p->d.block; a.res = nullptr;
  a.eig64 = (p->d.flags & T2SH_EIG_FP64) ? 1 : 0;
  KTimer k(p, KC_LLR);
  T2SH_CK(launch_llr(p->g, a, static_cast<float2*>(x), nullptr, nullptr, nullptr, p->st));
  return T2SH_OK;
}

}  // extern "C"

namespace {

// The host-IO stage of at least kb bytes, allocated in stream order on the plan's stream
// from the stage pool (the default pool if that is unavailable).
t2sh_status ensure_stage(t2sh_plan_t p, size_t kb) {
  if (p->stage_bytes >= kb) return T2SH_OK;
  if (p->stage) cudaFreeAsync(p->stage, p->st);
  p->stage = nullptr;
  p->stage_bytes = 0;
  cudaMemPool_t pool = stage_pool();
  const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p->stage, kb, pool, p->st) : cudaMallocAsync(&p->stage, kb, p->st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    p->stage = nullptr;
    set_err("allocation of %zu bytes for the k-space stage failed", kb);
    return T2SH_ENOMEM;
  }
  p->stage_bytes = kb;
  return T2SH_OK;
}

// A^H y from the k-space (staged through the plan with T2SH_HOST_IO) and a fresh FISTA state.
t2sh_status begin_impl(t2sh_plan_t p, const void* kspace, int32_t kform, bool record_res) {
  T2SH_REQ(p && kspace, "NULL argument");
  T2SH_REQ(kform == T2SH_KSPACE_TE || kform == T2SH_KSPACE_PROJ, "bad kform %d", kform);
  const t2sh_dims& d = p->d;
  const size_t vec = footprint(d).vec;
  const void* ky = kspace;
  if (p->host_io) {
    const size_t kb = kspace_bytes(d, kform);
    t2sh_status se = ensure_stage(p, kb);
    if (se != T2SH_OK) return se;
    T2SH_CK(cudaMemcpyAsync(p->stage, kspace, kb, cudaMemcpyHostToDevice, p->st));
    ky = p->stage;
  }
  t2sh_status s = adjoint_data(p, ky, kform, p->aty);
  if (s != T2SH_OK) return s;
  T2SH_CK(cudaMemsetAsync(p->x, 0, vec, p->st));
  T2SH_CK(cudaMemsetAsync(p->z, 0, vec, p->st));
  if (record_res && d.iters > 0) T2SH_CK(cudaMemsetAsync(p->res, 0, sizeof(double) * 2 * (size_t)d.iters, p->st));
  p->begun = true;
  p->iter_done = 0;
  p->tk = 1.0;
  p->record_res = record_res;
  return T2SH_OK;
}

// FISTA arguments of iteration `it` of plan p when t_k = tk before it; *tn gets t_{k+1}.
FistaArgs fista_args(t2sh_plan_t p, int it, double tk, double* tn) {
  const t2sh_dims& d = p->d;
  *tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * tk * tk));
  FistaArgs a{};
  a.mu = p->mu;
  a.tau = p->mu * d.lambda;
  a.beta = (float)((tk - 1.0) / *tn);
  a.sy = p->shifts[2 * it];
  a.sz = p->shifts[2 * it + 1];
  a.b = d.block;
  a.eig64 = (d.flags & T2SH_EIG_FP64) ? 1 : 0;
  a.skip_adj = (it == 0);
  a.skip_fwd = (it == d.iters - 1);
  a.res = p->record_res ? p->res + 2 * it : nullptr;
  return a;
}

// One FISTA iteration (index p->iter_done) of Eq. 5.
t2sh_status iteration(t2sh_plan_t p) {
  const t2sh_dims& d = p->d;
  const size_t vec = cbytes((long long)p->g.S * p->g.M * p->g.K * p->g.ny * p->g.nz);  // slices in view
  const int it = p->iter_done;
  double tn = 0.0;
  const FistaArgs a = fista_args(p, it, p->tk, &tn);
  if (p->fused_rows && band_fused_supported(p->g, d.block)) {
    // column pass of the normal operator, then the band kernel: A^H A z, gradient,
    // LLR, momentum and DFT_z(S z_{k+1}) for the next iteration (z_0 = 0: no A^H A z_0)
    if (it > 0) {
      KTimer k(p, KC_COL);
      T2SH_CK(launch_col(p->g, COL_NORMAL, p->py, p->tw_y, p->psi, p->phi, p->mask, p->t, p->t, p->st));
    }
    KTimer k(p, KC_BAND);
    T2SH_CK(launch_band_fused(p->g, a, p->tw_z, p->maps, p->t, p->x, p->z, p->aty, p->st));
  } else {
    if (it == 0) {
      T2SH_CK(cudaMemsetAsync(p->grad, 0, vec, p->st));  // z_0 = 0
    } else {
      t2sh_status s = normal_op(p, p->z, p->grad);
      if (s != T2SH_OK) return s;
    }
    KTimer k(p, KC_LLR);
    T2SH_CK(launch_llr(p->g, a, p->x, p->z, p->grad, p->aty, p->st));
  }
  p->tk = tn;
  p->iter_done = it + 1;
  return T2SH_OK;
}

t2sh_status iterate_impl(t2sh_plan_t p, int n) {
  T2SH_REQ(p, "NULL plan");
  T2SH_REQ(p->begun, "t2sh_solve_begin has not been called on this plan");
  T2SH_REQ(n >= 0, "n must be >= 0");
  for (int i = 0; i < n && p->iter_done < p->d.iters; ++i) {
    t2sh_status s = iteration(p);
    if (s != T2SH_OK) return s;
  }
  return T2SH_OK;
}

// 0: batched solves launch the LLR step of all scans as one work list when they qualify;
// 1: one LLR launch per scan on the scan's own stream (t2sh_batch_schedule)
std::atomic<int> g_batch_per_scan_llr{0};

// The FISTA iterations of several begun plans as one work list per stage: every iteration
// runs each active plan's normal operator on that plan's stream (plans[i]->st), then one
// LLR launch on `origin` covers the bands of every active plan, from a per-iteration job
// table prepared in device memory before the caller begins stream capture.  Only for
// plans that all take the FISTA LLR of the same register variant (K <= 4 or not, float32
// or float64 eigen-step) and no fused row kernel; see batch_list_eligible.
struct BatchList {
  std::vector<LlrJob> jobs;      // all iterations, in order
  std::vector<int> off, count;   // per iteration: first job, number of jobs
  std::vector<int> units;        // per iteration: CTAs
  std::vector<double> tk_end;    // per plan: t_k after its last iteration
  size_t smem = 0;
  bool kc8 = false, eig64 = false;
  LlrJob* dev = nullptr;
};

bool batch_list_eligible(t2sh_plan_t* plans, int n) {
  for (int i = 0; i < n; ++i) {
    const t2sh_plan_t p = plans[i];
    if (p->fused_rows && band_fused_supported(p->g, p->d.block)) return false;
    if ((p->g.K > 4) != (plans[0]->g.K > 4)) return false;
    if (((p->d.flags ^ plans[0]->d.flags) & T2SH_EIG_FP64) != 0) return false;
  }
  return true;
}

void batch_list_prepare(t2sh_plan_t* plans, int n, BatchList& bl) {
  int maxit = 0;
  for (int i = 0; i < n; ++i) maxit = std::max(maxit, plans[i]->d.iters);
  std::vector<double> tk(n);
  for (int i = 0; i < n; ++i) tk[i] = plans[i]->tk;
  bl.kc8 = plans[0]->g.K > 4;
  bl.eig64 = (plans[0]->d.flags & T2SH_EIG_FP64) != 0;
  for (int it = 0; it < maxit; ++it) {
    bl.off.push_back((int)bl.jobs.size());
    int units = 0;
    for (int i = 0; i < n; ++i) {
      const t2sh_plan_t p = plans[i];
      if (it >= p->d.iters) continue;
      double tn = 0.0;
      LlrJob j{};
      j.g = p->g;
      j.a = fista_args(p, it, tk[i], &tn);
      j.x = p->x;
      j.z = p->z;
      j.grad = p->grad;
      j.aty = p->aty;
      j.unit0 = units;
      units += llr_units(p->g, p->d.block);
      bl.smem = std::max(bl.smem, llr_smem_bytes(p->g, p->d.block));
      bl.jobs.push_back(j);
      tk[i] = tn;
    }
    bl.count.push_back((int)bl.jobs.size() - bl.off.back());
    bl.units.push_back(units);
  }
  bl.tk_end = tk;
}

// Enqueue (for capture) every iteration of the work-list batch.
t2sh_status batch_list_iterate(t2sh_plan_t* plans, int n, const BatchList& bl, cudaStream_t origin,
                               std::vector<cudaEvent_t>& ev) {
  const int maxit = (int)bl.off.size();
  for (int it = 0; it < maxit; ++it) {
    T2SH_CK(cudaEventRecord(ev[n + 1], origin));
    for (int i = 0; i < n; ++i) {
      const t2sh_plan_t p = plans[i];
      if (it >= p->d.iters) continue;
      T2SH_CK(cudaStreamWaitEvent(p->st, ev[n + 1], 0));
      if (it == 0) {
        T2SH_CK(cudaMemsetAsync(p->grad, 0, footprint(p->d).vec, p->st));  // z_0 = 0
      } else {
        const t2sh_status s = normal_op(p, p->z, p->grad);
        if (s != T2SH_OK) return s;
      }
      T2SH_CK(cudaEventRecord(ev[i], p->st));
      T2SH_CK(cudaStreamWaitEvent(origin, ev[i], 0));
    }
    for (int i = 0; i < n; ++i)
      if (it < plans[i]->d.iters) {
        plans[i]->launches[KC_LLR]++;  // one launch, counted once
        break;
      }
    T2SH_CK(launch_llr_list(bl.dev + bl.off[it], bl.count[it], bl.units[it], bl.kc8, bl.eig64, bl.smem, origin));
  }
  for (int i = 0; i < n; ++i) {
    plans[i]->tk = bl.tk_end[i];
    plans[i]->iter_done = plans[i]->d.iters;
  }
  return T2SH_OK;
}

t2sh_status end_impl(t2sh_plan_t p, void* alpha_out, double* residual_out, const float2* src = nullptr) {
  T2SH_REQ(p && alpha_out, "NULL argument");
  T2SH_REQ(p->begun, "t2sh_solve_begin has not been called on this plan");
  const t2sh_dims& d = p->d;
  const size_t vec = footprint(d).vec;
  T2SH_CK(cudaMemcpyAsync(alpha_out, src ? src : p->x, vec,
                          p->host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, p->st));
  if (residual_out && p->iter_done > 0) {
    T2SH_REQ(p->record_res, "the monitor was not recorded for this solve");
    std::vector<double> r(2 * (size_t)p->iter_done);
    T2SH_CK(cudaMemcpyAsync(r.data(), p->res, sizeof(double) * r.size(), cudaMemcpyDeviceToHost, p->st));
    T2SH_CK(cudaStreamSynchronize(p->st));
    for (int it = 0; it < p->iter_done; ++it)
      residual_out[it] = r[2 * it + 1] > 0.0 ? std::sqrt(r[2 * it] / r[2 * it + 1]) : 0.0;
  } else if (p->host_io) {
    T2SH_CK(cudaStreamSynchronize(p->st));
  }
  return T2SH_OK;
}

// The plan's per-slice buffers seen as the slices [s0, s0 + n) only; restores the full view.
struct SliceView {
  t2sh_plan_t p;
  Geom g;
  float2 *x, *z, *aty, *grad, *maps;
  SliceView(t2sh_plan_t p_, int s0, int n) : p(p_), g(p_->g), x(p_->x), z(p_->z), aty(p_->aty), grad(p_->grad), maps(p_->maps) {
    const long long N = (long long)g.ny * g.nz;
    const long long vs = (long long)g.M * g.K * N, ms = (long long)g.C * g.M * N;
    p->g.S = n;
    p->x += s0 * vs; p->z += s0 * vs; p->aty += s0 * vs; p->grad += s0 * vs; p->maps += s0 * ms;
  }
  ~SliceView() {
    p->g = g; p->x = x; p->z = z; p->aty = aty; p->grad = grad; p->maps = maps;
  }
};

constexpr int kHostChunks = 2;

// One-shot solve through host buffers (T2SH_HOST_IO).  Slices are independent and every
// slice runs the same shift and momentum sequence, so the scan is solved in two chunks of
// slices: a small first one (an eighth) whose copy alone is waited for, and the rest, whose
// k-space crosses on a copy stream while the first chunk is solved.  Each chunk's result
// is copied back on the copy stream (the first one's while the second is solved).
t2sh_status solve_host_pipelined(t2sh_plan_t p, const void* kspace, int32_t kform, void* alpha_out,
                                 double* residual_out) {
  T2SH_REQ(p && kspace && alpha_out, "NULL argument");
  T2SH_REQ(kform == T2SH_KSPACE_TE || kform == T2SH_KSPACE_PROJ, "bad kform %d", kform);
  const t2sh_dims& d = p->d;
  const int S = d.nslices;
  const int first = std::max(1, S / 8);
  const int bounds[kHostChunks + 1] = {0, first, S};
  const int nch = kHostChunks;
  const size_t kb = kspace_bytes(d, kform), kbs = kb / S;
  const size_t vslice = footprint(d).vec / S;
  {
    t2sh_status se = ensure_stage(p, kb);
    if (se != T2SH_OK) return se;
  }
  if (!p->cs) T2SH_CK(cudaStreamCreateWithFlags(&p->cs, cudaStreamNonBlocking));
  while ((int)p->cev.size() < 2 * kHostChunks + 2) {
    cudaEvent_t e;
    T2SH_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    p->cev.push_back(e);
  }
  cudaEvent_t* ev_in = p->cev.data();
  cudaEvent_t* ev_out = ev_in + kHostChunks;
  cudaEvent_t ev_start = p->cev[2 * kHostChunks], ev_done = p->cev[2 * kHostChunks + 1];
  // the copies must not overwrite the stage under work already queued on the plan's stream
  T2SH_CK(cudaEventRecord(ev_start, p->st));
  T2SH_CK(cudaStreamWaitEvent(p->cs, ev_start, 0));
  char* stage = static_cast<char*>(p->stage);
  const char* src = static_cast<const char*>(kspace);
  for (int c = 0; c < nch; ++c) {
    const int s0 = bounds[c], n = bounds[c + 1] - s0;
    T2SH_CK(cudaMemcpyAsync(stage + s0 * kbs, src + s0 * kbs, n * kbs, cudaMemcpyHostToDevice, p->cs));
    T2SH_CK(cudaEventRecord(ev_in[c], p->cs));
  }
  const bool rec = residual_out != nullptr;
  if (rec && d.iters > 0) T2SH_CK(cudaMemsetAsync(p->res, 0, sizeof(double) * 2 * (size_t)d.iters, p->st));
  char* out = static_cast<char*>(alpha_out);
  for (int c = 0; c < nch; ++c) {
    const int s0 = bounds[c], n = bounds[c + 1] - s0;
    T2SH_CK(cudaStreamWaitEvent(p->st, ev_in[c], 0));
    {
      SliceView view(p, s0, n);
      t2sh_status s = adjoint_data(p, stage + s0 * kbs, kform, p->aty);
      if (s != T2SH_OK) return s;
      T2SH_CK(cudaMemsetAsync(p->x, 0, n * vslice, p->st));
      T2SH_CK(cudaMemsetAsync(p->z, 0, n * vslice, p->st));
      p->begun = true;
      p->iter_done = 0;
      p->tk = 1.0;
      p->record_res = rec;
      s = iterate_impl(p, d.iters);
      if (s != T2SH_OK) return s;
      T2SH_CK(cudaEventRecord(ev_out[c], p->st));
      T2SH_CK(cudaStreamWaitEvent(p->cs, ev_out[c], 0));
      T2SH_CK(cudaMemcpyAsync(out + s0 * vslice, p->x, n * vslice, cudaMemcpyDeviceToHost, p->cs));
    }
  }
  T2SH_CK(cudaEventRecord(ev_done, p->cs));
  T2SH_CK(cudaStreamWaitEvent(p->st, ev_done, 0));
  if (rec && d.iters > 0) {
    std::vector<double> r(2 * (size_t)d.iters);
    T2SH_CK(cudaMemcpyAsync(r.data(), p->res, sizeof(double) * r.size(), cudaMemcpyDeviceToHost, p->st));
    T2SH_CK(cudaStreamSynchronize(p->st));
    for (int it = 0; it < d.iters; ++it) residual_out[it] = r[2 * it + 1] > 0.0 ? std::sqrt(r[2 * it] / r[2 * it + 1]) : 0.0;
  } else {
    T2SH_CK(cudaStreamSynchronize(p->st));
  }
  return T2SH_OK;
}

}  // namespace

extern "C" {

t2sh_status t2sh_solve(t2sh_plan_t p, const void* kspace, int32_t kform, void* alpha_out, double* residual_out) {
  T2SH_REQ(p && kspace && alpha_out, "NULL argument");
  if (p->host_io && p->d.nslices > 1) return solve_host_pipelined(p, kspace, kform, alpha_out, residual_out);
  t2sh_status s = begin_impl(p, kspace, kform, residual_out != nullptr);
  if (s == T2SH_OK) s = iterate_impl(p, p->d.iters);
  if (s == T2SH_OK) s = end_impl(p, alpha_out, residual_out);
  return s;
}

// ADMM (scaled form) for Eq. 5 with conjugate-gradient alpha-updates; the iteration the
// oracle's admm() states step by step.  alpha lives in p->x, v in p->z, u in p->u.
t2sh_status t2sh_solve_admm(t2sh_plan_t p, const void* kspace, int32_t kform, void* alpha_out, float rho,
                            int32_t cg_iters, double* residual_out) {
  T2SH_REQ(p && kspace && alpha_out, "NULL argument");
  T2SH_REQ(std::isfinite(rho) && rho > 0.f, "rho must be finite and > 0");
  T2SH_REQ(cg_iters >= 0 && cg_iters <= 1000, "cg_iters must be in [0, 1000]");
  const t2sh_dims& d = p->d;
  const Geom& g = p->g;
  const size_t vec = footprint(d).vec;
  if (!p->u) {
    t2sh_status a = p->alloc(&p->u, vec);
    if (a == T2SH_OK) a = p->alloc(&p->cg_r, vec);
    if (a == T2SH_OK) a = p->alloc(&p->cg_p, vec);
    if (a == T2SH_OK) a = p->alloc(&p->cg_red, sizeof(double) * 4 * (size_t)d.nslices);
    if (a != T2SH_OK) return a;
  }
  t2sh_status s = begin_impl(p, kspace, kform, residual_out != nullptr);
  if (s != T2SH_OK) return s;
  T2SH_CK(cudaMemsetAsync(p->u, 0, vec, p->st));
  double* rr[3] = {p->cg_red, p->cg_red + d.nslices, p->cg_red + 2 * (size_t)d.nslices};
  double* pq = p->cg_red + 3 * (size_t)d.nslices;
  for (int it = 0; it < d.iters; ++it) {
    if (cg_iters > 0) {
      // alpha-update: cg_iters CG steps on (A^H A + rho I) alpha = A^H y + rho (v - u) from alpha
      T2SH_CK(cudaMemsetAsync(p->cg_red, 0, sizeof(double) * 4 * (size_t)d.nslices, p->st));
      if (it == 0) {
        T2SH_CK(cudaMemsetAsync(p->grad, 0, vec, p->st));  // alpha_0 = 0
      } else {
        s = normal_op(p, p->x, p->grad);
        if (s != T2SH_OK) return s;
      }
      {
        KTimer k(p, KC_CG);
        T2SH_CK(launch_cg_init(g, p->x, p->grad, p->aty, p->z, p->u, rho, p->cg_r, p->cg_p, rr[0], p->st));
      }
      for (int i = 0; i < cg_iters; ++i) {
        s = normal_op(p, p->cg_p, p->grad);
        if (s != T2SH_OK) return s;
        KTimer k(p, KC_CG);
        T2SH_CK(launch_cg_dot(g, p->cg_p, p->grad, rho, pq, p->st));
        T2SH_CK(launch_cg_step(g, p->x, p->cg_r, p->cg_p, p->grad, rho, rr[i % 3], pq, rr[(i + 1) % 3], p->st));
        T2SH_CK(launch_cg_dir(g, p->cg_r, p->cg_p, rr[i % 3], rr[(i + 1) % 3], pq, rr[(i + 2) % 3], p->st));
      }
    }
    // v-update (LLR prox of alpha + u, threshold lambda / rho, this iteration's shift) and dual update
    FistaArgs a{};
    a.tau = d.lambda / rho;
    a.sy = p->shifts[2 * it];
    a.sz = p->shifts[2 * it + 1];
    a.b = d.block;
    a.eig64 = (d.flags & T2SH_EIG_FP64) ? 1 : 0;
    a.res = p->record_res ? p->res + 2 * it : nullptr;
    KTimer k(p, KC_LLR);
    T2SH_CK(launch_llr_admm(g, a, p->x, p->z, p->u, p->st));
  }
  p->iter_done = d.iters;
  s = end_impl(p, alpha_out, residual_out, p->z);
  p->begun = false;  // the FISTA state was not kept: no t2sh_solve_iterate on top of this
  return s;
}

t2sh_status t2sh_postprocess(t2sh_plan_t p, const void* alpha, const int32_t* te_index, int32_t nte, float pf,
                             void* out) {
  T2SH_REQ(p && alpha && te_index && out, "NULL argument");
  const t2sh_dims& d = p->d;
  if (p->host_io) {
    set_err("t2sh_postprocess takes device pointers (the plan has T2SH_HOST_IO)");
    return T2SH_EUNSUPPORTED;
  }
  T2SH_REQ(nte >= 1 && nte <= kMaxPostTe, "nte must be in [1, %d]", kMaxPostTe);
  for (int i = 0; i < nte; ++i)
    T2SH_REQ(te_index[i] >= 0 && te_index[i] < d.nechoes, "te_index[%d] = %d is not an echo of the basis", i, te_index[i]);
  T2SH_REQ(std::isfinite(pf) && pf > 0.5f && pf <= 1.f, "pf must be in (0.5, 1]");
  if (post_smem_bytes(p->g, nte) > 200 * 1024) {
    set_err("post-processing band of %d echoes x nz = %d does not fit shared memory", nte, d.nz);
    return T2SH_EUNSUPPORTED;
  }
  // band half-width, decided in double from the float fraction
  const int w = (int)std::ceil((double)pf * (double)d.nz) - d.nz / 2;
  int te[kMaxPostTe];
  for (int i = 0; i < nte; ++i) te[i] = te_index[i];
  KTimer k(p, KC_POST);
  T2SH_CK(launch_post(p->g, p->pz, p->tw_z, p->maps, p->phi, static_cast<const float2*>(alpha), te, nte, w,
                      static_cast<float*>(out), p->st));
  return T2SH_OK;
}

t2sh_status t2sh_wavelet_denoise(t2sh_plan_t p, void* alpha, float tau, int32_t levels) {
  T2SH_REQ(p && alpha, "NULL argument");
  const t2sh_dims& d = p->d;
  if (p->host_io) {
    set_err("t2sh_wavelet_denoise takes device pointers (the plan has T2SH_HOST_IO)");
    return T2SH_EUNSUPPORTED;
  }
  T2SH_REQ(((uintptr_t)alpha & 15) == 0, "alpha must be 16-byte aligned");
  T2SH_REQ(levels >= 1 && levels <= 16, "levels must be in [1, 16]");
  T2SH_REQ(std::isfinite(tau) && tau >= 0.f, "tau must be finite and >= 0");
  const int f = 1 << levels;
  T2SH_REQ(d.nslices % f == 0 && d.ny % f == 0 && d.nz % f == 0,
           "nslices = %d, ny = %d and nz = %d must be multiples of 2^levels = %d", d.nslices, d.ny, d.nz, f);
  KTimer k(p, KC_POST);
  T2SH_CK(launch_wavelet_denoise(p->g, static_cast<float2*>(alpha), tau, levels, p->st));
  return T2SH_OK;
}

t2sh_status t2sh_solve_begin(t2sh_plan_t p, const void* kspace, int32_t kform) {
  return begin_impl(p, kspace, kform, true);
}

t2sh_status t2sh_solve_iterate(t2sh_plan_t p, int32_t n, int32_t* done) {
  t2sh_status s = iterate_impl(p, n);
  if (s == T2SH_OK && done) *done = p->iter_done;
  return s;
}

t2sh_status t2sh_solve_end(t2sh_plan_t p, void* alpha_out, double* residual_out) {
  return end_impl(p, alpha_out, residual_out);
}

// ---------------------------------------------------------------------------------
// Batched solve: several plans (scans of different sizes) on forked streams, every
// iteration of every plan captured into one CUDA graph and launched once.
// ---------------------------------------------------------------------------------
t2sh_status t2sh_solve_batch(t2sh_plan_t* plans, int32_t n, const void* const* kspace, const int32_t* kform,
                             void* const* alpha_out, void* stream) {
  T2SH_REQ(plans && kspace && kform && alpha_out && n >= 1 && n <= 64, "bad batch arguments");
  for (int i = 0; i < n; ++i) {
    T2SH_REQ(plans[i] && kspace[i] && alpha_out[i], "NULL entry %d in the batch", i);
    T2SH_REQ(!plans[i]->host_io, "batched solves take device pointers (plan %d has T2SH_HOST_IO)", i);
    for (int j = 0; j < i; ++j) T2SH_REQ(plans[i] != plans[j], "plan %d appears twice in the batch", i);
  }
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  std::vector<cudaStream_t> fs(n, nullptr);
  std::vector<cudaStream_t> saved(n);
  std::vector<bool> timing(n);
  std::vector<cudaEvent_t> ev(n + 2, nullptr);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  t2sh_status st = T2SH_OK;
  cudaStream_t origin = nullptr;
  BatchList bl;
  const bool use_list = batch_list_eligible(plans, n) && !g_batch_per_scan_llr;
#define B_CK(call)                                                                   \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      set_err("%s failed: %s", #call, cudaGetErrorString(e_));                       \
      st = T2SH_ECUDA;                                                               \
      goto done;                                                                     \
    }                                                                                \
  } while (0)
  for (auto& e : ev) B_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  B_CK(cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking));
  for (int i = 0; i < n; ++i) B_CK(cudaStreamCreateWithFlags(&fs[i], cudaStreamNonBlocking));
  // fork from the caller's stream, begin every solve (A^H y) on its own stream
  B_CK(cudaEventRecord(ev[n], cs));
  for (int i = 0; i < n; ++i) {
    saved[i] = plans[i]->st;
    timing[i] = plans[i]->timing;
    plans[i]->st = fs[i];
    plans[i]->timing = false;
    B_CK(cudaStreamWaitEvent(fs[i], ev[n], 0));
    st = begin_impl(plans[i], kspace[i], kform[i], false);
    if (st != T2SH_OK) goto done;
    B_CK(cudaEventRecord(ev[i], fs[i]));
    B_CK(cudaStreamWaitEvent(origin, ev[i], 0));
  }
  if (use_list) {  // the per-iteration LLR job tables, in device memory before the capture
    batch_list_prepare(plans, n, bl);
    if (!bl.jobs.empty()) {
      B_CK(cudaMalloc(&bl.dev, sizeof(LlrJob) * bl.jobs.size()));
      B_CK(cudaMemcpy(bl.dev, bl.jobs.data(), sizeof(LlrJob) * bl.jobs.size(), cudaMemcpyHostToDevice));
    }
  }
  // capture all iterations of all plans
  B_CK(cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed));
  if (use_list) {
    st = batch_list_iterate(plans, n, bl, origin, ev);
    if (st != T2SH_OK) {
      cudaStreamEndCapture(origin, &graph);
      goto done;
    }
  } else {
    B_CK(cudaEventRecord(ev[n + 1], origin));
    for (int i = 0; i < n; ++i) {
      B_CK(cudaStreamWaitEvent(fs[i], ev[n + 1], 0));
      st = iterate_impl(plans[i], plans[i]->d.iters);
      if (st != T2SH_OK) {
        cudaStreamEndCapture(origin, &graph);
        goto done;
      }
      B_CK(cudaEventRecord(ev[i], fs[i]));
      B_CK(cudaStreamWaitEvent(origin, ev[i], 0));
    }
  }
  B_CK(cudaStreamEndCapture(origin, &graph));
  B_CK(cudaGraphInstantiate(&exec, graph, 0));
  B_CK(cudaGraphLaunch(exec, origin));
  B_CK(cudaEventRecord(ev[n + 1], origin));
  for (int i = 0; i < n; ++i) {
    B_CK(cudaStreamWaitEvent(fs[i], ev[n + 1], 0));
    st = end_impl(plans[i], alpha_out[i], nullptr);
    if (st != T2SH_OK) goto done;
    B_CK(cudaEventRecord(ev[i], fs[i]));
    B_CK(cudaStreamWaitEvent(cs, ev[i], 0));
  }
  B_CK(cudaStreamSynchronize(cs));
done:
#undef B_CK
  for (int i = 0; i < n; ++i)
    if (fs[i]) {
      cudaStreamSynchronize(fs[i]);
      plans[i]->st = saved[i];
      plans[i]->timing = timing[i];
    }
  if (origin) cudaStreamSynchronize(origin);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (bl.dev) cudaFree(bl.dev);
  for (auto& f : fs)
    if (f) cudaStreamDestroy(f);
  if (origin) cudaStreamDestroy(origin);
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  return st;
}

t2sh_status t2sh_batch_schedule(int32_t per_scan_llr) {
  T2SH_REQ(per_scan_llr == 0 || per_scan_llr == 1, "per_scan_llr must be 0 or 1");
  g_batch_per_scan_llr = per_scan_llr;
  return T2SH_OK;
}

t2sh_status t2sh_objective(t2sh_plan_t p, const void* kspace, int32_t kform, const void* x, double* out) {
  T2SH_REQ(p && kspace && x && out, "NULL argument");
  T2SH_REQ(kform == T2SH_KSPACE_TE || kform == T2SH_KSPACE_PROJ, "bad kform %d", kform);
  const t2sh_dims& d = p->d;
  const int S = d.nslices;
  const size_t vec = footprint(d).vec;
  if (!p->obj) {
    t2sh_status a = p->alloc(&p->obj, sizeof(double) * 3 * (size_t)S);
    if (a != T2SH_OK) return a;
  }
  const void* ky = kspace;
  const float2* xd = static_cast<const float2*>(x);
  if (p->host_io) {
    const size_t kb = kspace_bytes(d, kform);
    t2sh_status se = ensure_stage(p, kb);
    if (se != T2SH_OK) return se;
    if (!p->ov) {
      t2sh_status a = p->alloc(&p->ov, vec);
      if (a != T2SH_OK) return a;
    }
    T2SH_CK(cudaMemcpyAsync(p->stage, kspace, kb, cudaMemcpyHostToDevice, p->st));
    T2SH_CK(cudaMemcpyAsync(p->ov, x, vec, cudaMemcpyHostToDevice, p->st));
    ky = p->stage;
    xd = p->ov;
  }
  double* xx = p->obj;          // <x, A^H A x>
  double* xa = p->obj + S;      // Re <x, A^H y>
  double* yy = p->obj + 2 * S;  // ||P y||^2
  T2SH_CK(cudaMemsetAsync(p->obj, 0, sizeof(double) * 3 * (size_t)S, p->st));
  // the gradient buffer is scratch between iterations: A^H A x, then A^H y
  t2sh_status s = normal_op(p, xd, p->grad);
  if (s != T2SH_OK) return s;
  T2SH_CK(launch_cg_dot(p->g, xd, p->grad, 0.f, xx, p->st));
  s = adjoint_data(p, ky, kform, p->grad);
  if (s != T2SH_OK) return s;
  T2SH_CK(launch_cg_dot(p->g, xd, p->grad, 0.f, xa, p->st));
  if (kform == T2SH_KSPACE_TE)
    T2SH_CK(launch_masked_energy(p->g, p->mask, static_cast<const float2*>(ky), yy, p->st));
  std::vector<double> h(3 * (size_t)S);
  T2SH_CK(cudaMemcpyAsync(h.data(), p->obj, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, p->st));
  T2SH_CK(cudaStreamSynchronize(p->st));
  for (int i = 0; i < S; ++i) {
    out[2 * i] = 0.5 * h[i] - h[S + i];
    out[2 * i + 1] = kform == T2SH_KSPACE_TE ? 0.5 * h[2 * S + i] : std::nan("");
  }
  return T2SH_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Autotuner: per problem shape, time the column-pass tile width (8 or 4 columns) and
// the separate or fused row kernels on the plan's own buffers; cache the choice in
// memory and, when T2SH_TUNE_CACHE names a file, in that file (one line per shape).
// ---------------------------------------------------------------------------------
namespace {
std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune;  // shape -> (colw, fused)
bool g_tune_loaded = false;

std::string tune_key(const t2sh_dims& d) {
  char b[128];
  snprintf(b, sizeof(b), "%d %d %d %d %d %d %d", d.ny, d.nz, d.ncoils, d.nbasis, d.nmaps, d.block, d.precision);
  return b;
}

void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* f = std::getenv("T2SH_TUNE_CACHE");
  if (!f) return;
  FILE* fp = std::fopen(f, "r");
  if (!fp) return;
  int a[9];
  while (std::fscanf(fp, "%d %d %d %d %d %d %d %d %d", &a[0], &a[1], &a[2], &a[3], &a[4], &a[5], &a[6], &a[7],
                     &a[8]) == 9) {
    char b[128];
    snprintf(b, sizeof(b), "%d %d %d %d %d %d %d", a[0], a[1], a[2], a[3], a[4], a[5], a[6]);
    if (a[7] >= 0 && a[7] <= 4) g_tune[b] = {a[7], a[8]};
  }
  std::fclose(fp);
}

void tune_store(const std::string& key, int colw, int fused) {
  const char* f = std::getenv("T2SH_TUNE_CACHE");
  if (!f) return;
  FILE* fp = std::fopen(f, "a");
  if (!fp) return;
  std::fprintf(fp, "%s %d %d\n", key.c_str(), colw, fused);
  std::fclose(fp);
}
}  // namespace

extern "C" t2sh_status t2sh_autotune(t2sh_plan_t p, int32_t probe_iters, int32_t* colw_out, int32_t* fused_out) {
  T2SH_REQ(p, "NULL plan");
  T2SH_REQ(!p->begun || p->iter_done == p->d.iters, "autotune must not interrupt a solve in progress");
  const t2sh_dims& d = p->d;
  const std::string key = tune_key(d);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load();
    auto it = g_tune.find(key);
    if (it != g_tune.end() && probe_iters >= 0) {
      p->g.colvar = it->second.first;
      p->fused_rows = it->second.second != 0;
      if (colw_out) *colw_out = p->g.colvar;
      if (fused_out) *fused_out = p->fused_rows ? 1 : 0;
      return T2SH_OK;
    }
  }
  const int probe = probe_iters > 0 ? probe_iters : 3;
  const int iters_keep = d.iters;
  T2SH_REQ(iters_keep >= 2, "autotune needs a plan with at least 2 iterations");
  const size_t vec = footprint(d).vec;
  T2SH_CK(cudaMemsetAsync(p->x, 0, vec, p->st));
  T2SH_CK(cudaMemsetAsync(p->z, 0, vec, p->st));
  T2SH_CK(cudaMemsetAsync(p->aty, 0, vec, p->st));
  T2SH_CK(cudaMemsetAsync(p->t, 0, footprint(d).t, p->st));
  cudaEvent_t e0, e1;
  T2SH_CK(cudaEventCreate(&e0));
  T2SH_CK(cudaEventCreate(&e1));
  const bool timing = p->timing;
  p->timing = false;
  float best = 1e30f;
  int bw = 0, bf = 0;
  t2sh_status st = T2SH_OK;
  // the mixed-precision column pass is the precision's choice, not a tuning candidate
  const std::vector<int> cols = d.precision == T2SH_MIXED_BF16 ? std::vector<int>{3} : std::vector<int>{0, 4, 1, 2};
  for (int colw : cols) {
    for (int fused = 0; fused <= (band_fused_supported(p->g, d.block) ? 1 : 0); ++fused) {
      p->g.colvar = colw;
      p->fused_rows = fused != 0;
      p->begun = true;
      p->record_res = false;
      float ms = 0.f;
      for (int rep = 0; rep < 2 && st == T2SH_OK; ++rep) {  // first repetition warms up
        p->iter_done = 1;
        p->tk = 1.0;
        if (cudaEventRecord(e0, p->st) != cudaSuccess) st = T2SH_ECUDA;
        for (int i = 0; i < probe && st == T2SH_OK; ++i) {
          p->iter_done = 1 + (i % (iters_keep - 1));
          st = iteration(p);
        }
        if (st == T2SH_OK && cudaEventRecord(e1, p->st) != cudaSuccess) st = T2SH_ECUDA;
        if (st == T2SH_OK && cudaEventSynchronize(e1) != cudaSuccess) st = T2SH_ECUDA;
        if (st == T2SH_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = T2SH_ECUDA;
      }
      if (st != T2SH_OK) break;
      if (ms < best) {
        best = ms;
        bw = colw;
        bf = fused;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p->timing = timing;
  p->begun = false;
  p->iter_done = 0;
  if (st != T2SH_OK) {
    if (g_err.empty()) set_err("autotune: a CUDA call failed");
    return st;
  }
  p->g.colvar = bw;
  p->fused_rows = bf != 0;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = {bw, bf};
    tune_store(key, bw, bf);
  }
  if (colw_out) *colw_out = bw;
  if (fused_out) *fused_out = bf;
  return T2SH_OK;
}
