// Host side of the pre-processing entry points (t2sh_coil_compression, t2sh_preprocess):
// argument checks, the (ky, kz) segment table of the sparse lines, stream-ordered scratch.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "../../include/t2sh.h"
#include "t2sh_plan.h"

namespace t2sh {
bool fft_plan_for(int n, FftPlan& p);
void set_last_error(const char* msg);
}  // namespace t2sh

using namespace t2sh;

namespace {

t2sh_status fail(t2sh_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

#define PP_CK(call)                                                   \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) return fail(T2SH_ECUDA, cudaGetErrorString(e_)); \
  } while (0)

t2sh_status check_sparse(const t2sh_sparse* sp) {
  if (!sp || !sp->t || !sp->ky || !sp->kz) return fail(T2SH_EINVAL, "sparse description or index array is NULL");
  if (sp->nlines < 1 || sp->nchan < 1 || sp->nx < 2 || sp->ny < 1 || sp->nz < 1 || sp->nechoes < 1)
    return fail(T2SH_EINVAL, "nlines, nchan, nx, ny, nz, nechoes must be positive (nx >= 2)");
  if (sp->nchan > kMaxChan) return fail(T2SH_EINVAL, "nchan must be <= 32");
  if ((long long)sp->nechoes * sp->ny * sp->nz > (1LL << 31)) return fail(T2SH_EINVAL, "mask too large");
  for (int j = 0; j < sp->nlines; ++j)
    if (sp->t[j] < 0 || sp->t[j] >= sp->nechoes || sp->ky[j] < 0 || sp->ky[j] >= sp->ny || sp->kz[j] < 0 ||
        sp->kz[j] >= sp->nz)
      return fail(T2SH_EINVAL, "a line's (t, ky, kz) index is out of range");
  return T2SH_OK;
}

struct Segments {
  std::vector<int> order, t_sorted, off, y, z;
};

// lines sorted (stably) by phase encode; one segment per distinct (ky, kz)
void build_segments(const t2sh_sparse* sp, Segments& s) {
  const int n = sp->nlines;
  s.order.resize(n);
  std::iota(s.order.begin(), s.order.end(), 0);
  std::stable_sort(s.order.begin(), s.order.end(), [&](int a, int b) {
    return (long long)sp->ky[a] * sp->nz + sp->kz[a] < (long long)sp->ky[b] * sp->nz + sp->kz[b];
  });
  s.t_sorted.resize(n);
  for (int q = 0; q < n; ++q) {
    const int j = s.order[q];
    s.t_sorted[q] = sp->t[j];
    if (q == 0 || sp->ky[j] != sp->ky[s.order[q - 1]] || sp->kz[j] != sp->kz[s.order[q - 1]]) {
      s.off.push_back(q);
      s.y.push_back(sp->ky[j]);
      s.z.push_back(sp->kz[j]);
    }
  }
  s.off.push_back(n);
}

// stream-ordered device copies of host tables; freed with release()
struct Scratch {
  cudaStream_t st;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t s) : st(s) {}
  template <typename T>
  cudaError_t alloc(T** p, size_t n) {
    void* q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, n ? n * sizeof(T) : 16, st);
    if (e == cudaSuccess) {
      ptrs.push_back(q);
      *p = static_cast<T*>(q);
    }
    return e;
  }
  template <typename T>
  cudaError_t upload(T** p, const std::vector<T>& v) {
    cudaError_t e = alloc(p, v.size());
    if (e == cudaSuccess && !v.empty()) e = cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    return e;
  }
  ~Scratch() {
    for (void* q : ptrs) cudaFreeAsync(q, st);
  }
};

bool fft_size_ok(int n) {
  if (n % 2) return false;
  for (int p : {2, 3, 5, 13})
    while (n % p == 0) n /= p;
  return n == 1;
}

}  // namespace

extern "C" {

t2sh_status t2sh_coil_compression(const t2sh_sparse* sp, const void* lines, int32_t window, int32_t ncomp,
                                  void* w_out, void* stream) {
  t2sh_status s = check_sparse(sp);
  if (s != T2SH_OK) return s;
  if (!lines || !w_out) return fail(T2SH_EINVAL, "NULL argument");
  if (ncomp < 1 || ncomp > sp->nchan) return fail(T2SH_EINVAL, "ncomp must be in [1, nchan]");
  if (window < 1 || window > sp->nx || window > sp->ny || window > sp->nz)
    return fail(T2SH_EINVAL, "window must be in [1, min(nx, ny, nz)]");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Segments sg;
  build_segments(sp, sg);
  const int y0 = sp->ny / 2 - window / 2, z0 = sp->nz / 2 - window / 2;
  std::vector<int> wseg;
  for (size_t i = 0; i + 1 < sg.off.size(); ++i)
    if (sg.y[i] >= y0 && sg.y[i] < y0 + window && sg.z[i] >= z0 && sg.z[i] < z0 + window) wseg.push_back((int)i);
  if (wseg.empty()) return fail(T2SH_EINVAL, "no line falls in the calibration window");
  {
    Scratch sc(st);
    int *order = nullptr, *off = nullptr, *wsg = nullptr, *err = nullptr;
    float2* X = nullptr;
    double* G = nullptr;
    const long long npts = (long long)wseg.size() * window;
    PP_CK(sc.upload(&order, sg.order));
    PP_CK(sc.upload(&off, sg.off));
    PP_CK(sc.upload(&wsg, wseg));
    PP_CK(sc.alloc(&X, (size_t)npts * sp->nchan));
    PP_CK(sc.alloc(&G, 2 * (size_t)sp->nchan * sp->nchan));
    PP_CK(sc.alloc(&err, 1));
    PP_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    PP_CK(launch_calib(static_cast<const float2*>(lines), sp->nchan, sp->nx, order, off, wsg, (int)wseg.size(), window,
                       X, st));
    PP_CK(launch_gram_eig(X, npts, sp->nchan, ncomp, G, static_cast<float2*>(w_out), err, st));
    int herr = 0;
    PP_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    PP_CK(cudaStreamSynchronize(st));
    if (herr) return fail(T2SH_ECUDA, "the channel eigendecomposition did not converge");
  }
  return T2SH_OK;
}

t2sh_status t2sh_preprocess(const t2sh_sparse* sp, const void* lines, const void* w, int32_t ncomp, const float* phi,
                            int32_t nbasis, void* ytil_out, uint8_t* mask_out, void* stream) {
  t2sh_status s = check_sparse(sp);
  if (s != T2SH_OK) return s;
  if (!lines || !w || !phi || !ytil_out || !mask_out) return fail(T2SH_EINVAL, "NULL argument");
  if (ncomp < 1 || ncomp > sp->nchan) return fail(T2SH_EINVAL, "ncomp must be in [1, nchan]");
  if (nbasis < 1 || nbasis > kMaxK || nbasis > sp->nechoes) return fail(T2SH_EINVAL, "nbasis must be in [1, min(8, nechoes)]");
  if (!fft_size_ok(sp->nx) || sp->nx > 8192) return fail(T2SH_EINVAL, "nx must be even, a product of 2, 3, 5 and 13, <= 8192");
  FftPlan px{};
  if (!fft_plan_for(sp->nx, px)) return fail(T2SH_EINVAL, "no radix plan for nx");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Segments sg;
  build_segments(sp, sg);
  const int nseg = (int)sg.off.size() - 1;
  std::vector<float2> tw(sp->nx);
  for (int m = 0; m < sp->nx; ++m) {
    const double a = -2.0 * 3.14159265358979323846 * m / sp->nx;
    tw[m] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  {
    Scratch sc(st);
    int *order = nullptr, *ts = nullptr, *off = nullptr, *sy = nullptr, *sz = nullptr, *tl = nullptr, *kyl = nullptr,
        *kzl = nullptr;
    float2 *yh = nullptr, *twd = nullptr;
    PP_CK(sc.upload(&order, sg.order));
    PP_CK(sc.upload(&ts, sg.t_sorted));
    PP_CK(sc.upload(&off, sg.off));
    PP_CK(sc.upload(&sy, sg.y));
    PP_CK(sc.upload(&sz, sg.z));
    PP_CK(sc.upload(&tl, std::vector<int>(sp->t, sp->t + sp->nlines)));
    PP_CK(sc.upload(&kyl, std::vector<int>(sp->ky, sp->ky + sp->nlines)));
    PP_CK(sc.upload(&kzl, std::vector<int>(sp->kz, sp->kz + sp->nlines)));
    PP_CK(sc.upload(&twd, tw));
    PP_CK(sc.alloc(&yh, (size_t)sp->nlines * ncomp * sp->nx));
    const size_t ybytes = sizeof(float2) * (size_t)sp->nx * ncomp * nbasis * sp->ny * sp->nz;
    PP_CK(cudaMemsetAsync(ytil_out, 0, ybytes, st));
    PP_CK(cudaMemsetAsync(mask_out, 0, (size_t)sp->nechoes * sp->ny * sp->nz, st));
    PP_CK(launch_compress_readout(static_cast<const float2*>(lines), static_cast<const float2*>(w), sp->nlines,
                                  sp->nchan, ncomp, px, twd, yh, st));
    PP_CK(launch_project_lines(yh, ncomp, sp->nx, order, ts, off, sy, sz, nseg, phi, nbasis, sp->ny, sp->nz,
                               static_cast<float2*>(ytil_out), st));
    PP_CK(launch_mark_mask(tl, kyl, kzl, sp->nlines, sp->ny, sp->nz, mask_out, st));
  }
  return T2SH_OK;
}

}  // extern "C"
