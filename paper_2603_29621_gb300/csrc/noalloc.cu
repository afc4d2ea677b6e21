// mfns_smooth_noalloc: the smoothing step of mfns_smooth for callers that must not
// allocate device memory at call time, with its two scratch vectors (Chebyshev
// direction and operator product) held in a fixed file-scope device array.
#include <mutex>
#include <string>

#include "capi_types.hpp"
#include "vec.hpp"

namespace {

constexpr int64_t kMaxEntries = int64_t(1) << 20;  // per scratch vector (FP64 or FP32 entries)
constexpr int kMaxDevices = 64;

// 2 vectors x 2^20 doubles = 16 MiB, resident on every GPU that loads the library until exit.
static __device__ __align__(256) double g_smooth_scratch[2 * kMaxEntries];

// Device address of g_smooth_scratch per device (host code must not use the symbol itself).
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// Once per device, with that device current.
void* scratch_address(int device) {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[device]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_smooth_scratch);
    if (e != cudaSuccess) throw mfns::Error(mfns::kErrCuda, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[device] = ptr;
  }
  return g_scratch_addr[device];
}

// The smoothing recurrence of mfns_smooth, with caller-supplied scratch d (direction) and t (A x).
template <typename T>
void smooth_with_scratch(mfns::Problem& p, int level, int prec, const T* b, T* x, bool x_is_zero, T* d, T* t,
                         cudaStream_t s) {
  using namespace mfns;
  OpLevel& lv = *p.levels[level];
  const int64_t n = lv.n_dofs;
  const T* dinv = lv.dinv[prec].as<T>();
  const double lmax = lv.lmax, lmin = lmax / 20.0;
  const int degree = p.smoother_degree;
  if (p.smoother == 1) {
    const T omega = (T)(2.0 / (lmin + lmax));
    for (int it = 0; it < degree; ++it) {
      if (it == 0 && x_is_zero) {
        vcheby0<T>(x, d, b, dinv, omega, n, s);
      } else {
        oplevel_vmult(lv, prec, x, t, s);
        vcheby<T>(x, d, b, t, dinv, T(0), omega, n, s);
      }
    }
    return;
  }
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  double rho_old = 1.0 / sigma;
  if (x_is_zero) {
    vcheby0<T>(x, d, b, dinv, (T)(1.0 / theta), n, s);
  } else {
    oplevel_vmult(lv, prec, x, t, s);
    vcheby<T>(x, d, b, t, dinv, T(0), (T)(1.0 / theta), n, s);
  }
  for (int j = 1; j < degree; ++j) {
    oplevel_vmult(lv, prec, x, t, s);
    const double rho = 1.0 / (2.0 * sigma - rho_old);
    vcheby<T>(x, d, b, t, dinv, (T)(rho * rho_old), (T)(2.0 * rho / delta), n, s);
    rho_old = rho;
  }
}

}  // namespace

extern "C" int mfns_smooth_noalloc(mfns_problem* p, int level, int precision, const void* b, void* x, int64_t n_in,
                                   int x_is_zero, void* stream) {
  using namespace mfns;
  try {
    (void)cudaGetLastError();  // a pending error of another component of the process is not ours
    if (!p || level < 0 || level >= (int)p->p->levels.size() || !b || !x || (precision != 0 && precision != 1))
      return capi_fail(kErrArg, "bad arguments");
    if (p->p->ls) return capi_fail(kErrUnsupported, "single-level smoothing is not exposed for local smoothing");
    if (p->p->smoother == 2) return capi_fail(kErrUnsupported, "the no-allocation smoother is point-Jacobi based");
    const int64_t n = p->p->levels[level]->n_dofs;
    if (n_in != n)
      return capi_fail(kErrArg, ("b/x has " + std::to_string(n_in) + " entries, expected " + std::to_string(n)).c_str());
    if (n > kMaxEntries)
      return capi_fail(kErrArg, ("mfns_smooth_noalloc: level has " + std::to_string(n) +
                                 " entries, the fixed scratch holds at most 1048576 per vector").c_str());
    const int dev = p->ctx->device;
    if (dev < 0 || dev >= kMaxDevices) return capi_fail(kErrArg, "device ordinal out of range");
    MFNS_CUDA(cudaSetDevice(dev));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* base = static_cast<char*>(scratch_address(dev));
    const size_t es = precision == 0 ? 8 : 4;
    void* d = base;
    void* t = base + (size_t)kMaxEntries * 8;  // second half of the array
    // the direction vector is read (times zero) before it is first written: clear it
    MFNS_CUDA(cudaMemsetAsync(d, 0, (size_t)n * es, s));
    if (precision == 0)
      smooth_with_scratch<double>(*p->p, level, 0, (const double*)b, (double*)x, x_is_zero != 0, (double*)d,
                                  (double*)t, s);
    else
      smooth_with_scratch<float>(*p->p, level, 1, (const float*)b, (float*)x, x_is_zero != 0, (float*)d, (float*)t,
                                 s);
  } catch (const Error& e) {
    return capi_fail(e.code, e.what());
  } catch (const std::exception& e) {
    return capi_fail(kErrArg, e.what());
  }
  return MFNS_OK;
}
