// Runtime dispatch of the operator kernels and the host-side 1D tables.
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>

#include "mesh.hpp"
#include "op_kernel.cuh"
#include "op_launch.hpp"
#include "common.hpp"

namespace mfns {

constexpr int kOpWarpsDefault = 4;

#define MFNS_DECL(DIM, K, OP)                                                                                  \
  extern template void op_launch<DIM, K, OP, double>(const OpLaunch&, const double*, double*, bool, cudaStream_t, \
                                                     int, int, int64_t, const OpEpilogue*);                      \
  extern template void op_launch<DIM, K, OP, float>(const OpLaunch&, const float*, float*, bool, cudaStream_t, int, \
                                                    int, int64_t, const OpEpilogue*);                            \
  extern template void op_launch_multi<DIM, K, OP, double>(const OpLaunch&, int, const MultiColour&, cudaStream_t); \
  extern template void op_launch_multi<DIM, K, OP, float>(const OpLaunch&, int, const MultiColour&, cudaStream_t);

MFNS_DECL(3, 1, OP_STAB_NS) MFNS_DECL(3, 2, OP_STAB_NS) MFNS_DECL(3, 3, OP_STAB_NS)
MFNS_DECL(2, 1, OP_STAB_NS) MFNS_DECL(2, 2, OP_STAB_NS) MFNS_DECL(2, 3, OP_STAB_NS) MFNS_DECL(2, 4, OP_STAB_NS)
MFNS_DECL(3, 2, OP_STOKES) MFNS_DECL(3, 3, OP_STOKES) MFNS_DECL(3, 4, OP_STOKES)
MFNS_DECL(2, 2, OP_STOKES) MFNS_DECL(2, 3, OP_STOKES) MFNS_DECL(2, 4, OP_STOKES)
MFNS_DECL(3, 1, OP_STOKES_A) MFNS_DECL(3, 2, OP_STOKES_A) MFNS_DECL(3, 3, OP_STOKES_A) MFNS_DECL(3, 4, OP_STOKES_A)
MFNS_DECL(2, 1, OP_STOKES_A) MFNS_DECL(2, 2, OP_STOKES_A) MFNS_DECL(2, 3, OP_STOKES_A) MFNS_DECL(2, 4, OP_STOKES_A)
MFNS_DECL(2, 1, OP_PMASS) MFNS_DECL(2, 2, OP_PMASS) MFNS_DECL(2, 3, OP_PMASS)
MFNS_DECL(3, 1, OP_PMASS) MFNS_DECL(3, 2, OP_PMASS) MFNS_DECL(3, 3, OP_PMASS)
MFNS_DECL(2, 2, OP_VMASS) MFNS_DECL(2, 3, OP_VMASS) MFNS_DECL(2, 4, OP_VMASS)
MFNS_DECL(3, 2, OP_VMASS) MFNS_DECL(3, 3, OP_VMASS) MFNS_DECL(3, 4, OP_VMASS)

#define MFNS_DECL_DEFER(K, OP)                                                                                  \
  extern template void op_launch_deferred<3, K, OP, double>(const OpLaunch&, const double*, double*, cudaStream_t); \
  extern template void op_launch_deferred<3, K, OP, float>(const OpLaunch&, const float*, float*, cudaStream_t);
MFNS_DECL_DEFER(1, OP_STAB_NS) MFNS_DECL_DEFER(2, OP_STAB_NS) MFNS_DECL_DEFER(3, OP_STAB_NS)
MFNS_DECL_DEFER(1, OP_STOKES_A) MFNS_DECL_DEFER(2, OP_STOKES_A) MFNS_DECL_DEFER(3, OP_STOKES_A)
MFNS_DECL_DEFER(4, OP_STOKES_A)
MFNS_DECL_DEFER(1, OP_PMASS) MFNS_DECL_DEFER(2, OP_PMASS) MFNS_DECL_DEFER(3, OP_PMASS)
#undef MFNS_DECL_DEFER

bool op_supported(int dim, int k, int op) {
  if (dim != 2 && dim != 3) return false;
  switch (op) {
    case OP_STAB_NS: return k >= 1 && k <= (dim == 3 ? 3 : 4);
    case OP_STOKES: return k >= 2 && k <= 4;
    case OP_STOKES_A: return k >= 1 && k <= 4;
    case OP_PMASS: return k >= 1 && k <= 3;
    case OP_VMASS: return k >= 2 && k <= 4;  // the Taylor--Hood velocity degrees
  }
  return false;
}

template <typename T>
static void dispatch(const OpLaunch& L, const T* s, T* d, bool diag, cudaStream_t st, int fq_mode = -1,
                     int ncols = 1, int64_t col_stride = 0, const OpEpilogue* epi = nullptr) {
#define MFNS_CASE(DIM, K, OP)                   \
  if (L.dim == DIM && L.k == K && L.op == OP) \
    return op_launch<DIM, K, OP, T>(L, s, d, diag, st, fq_mode, ncols, col_stride, epi);
  MFNS_CASE(3, 1, OP_STAB_NS) MFNS_CASE(3, 2, OP_STAB_NS) MFNS_CASE(3, 3, OP_STAB_NS)
  MFNS_CASE(2, 1, OP_STAB_NS) MFNS_CASE(2, 2, OP_STAB_NS) MFNS_CASE(2, 3, OP_STAB_NS) MFNS_CASE(2, 4, OP_STAB_NS)
  MFNS_CASE(3, 2, OP_STOKES) MFNS_CASE(3, 3, OP_STOKES) MFNS_CASE(3, 4, OP_STOKES)
  MFNS_CASE(2, 2, OP_STOKES) MFNS_CASE(2, 3, OP_STOKES) MFNS_CASE(2, 4, OP_STOKES)
  MFNS_CASE(3, 1, OP_STOKES_A) MFNS_CASE(3, 2, OP_STOKES_A) MFNS_CASE(3, 3, OP_STOKES_A) MFNS_CASE(3, 4, OP_STOKES_A)
  MFNS_CASE(2, 1, OP_STOKES_A) MFNS_CASE(2, 2, OP_STOKES_A) MFNS_CASE(2, 3, OP_STOKES_A) MFNS_CASE(2, 4, OP_STOKES_A)
  MFNS_CASE(2, 1, OP_PMASS) MFNS_CASE(2, 2, OP_PMASS) MFNS_CASE(2, 3, OP_PMASS)
  MFNS_CASE(3, 1, OP_PMASS) MFNS_CASE(3, 2, OP_PMASS) MFNS_CASE(3, 3, OP_PMASS)
  MFNS_CASE(2, 2, OP_VMASS) MFNS_CASE(2, 3, OP_VMASS) MFNS_CASE(2, 4, OP_VMASS)
  MFNS_CASE(3, 2, OP_VMASS) MFNS_CASE(3, 3, OP_VMASS) MFNS_CASE(3, 4, OP_VMASS)
#undef MFNS_CASE
  throw Error(kErrUnsupported, "unsupported (dim, degree, operator) combination");
}

void KernelTimer::record_pair_begin(cudaStream_t s) {
  if (used + 2 > ev.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      MFNS_CUDA(cudaEventCreate(&e));
      ev.push_back(e);
    }
  }
  MFNS_CUDA(cudaEventRecord(ev[used], s));
}
void KernelTimer::record_pair_end(cudaStream_t s) {
  MFNS_CUDA(cudaEventRecord(ev[used + 1], s));
  used += 2;
}
double KernelTimer::read_ms(int64_t* launches) {
  double total = 0.0;
  for (size_t i = 0; i + 1 < used; i += 2) {
    MFNS_CUDA(cudaEventSynchronize(ev[i + 1]));
    float ms = 0.f;
    MFNS_CUDA(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
    total += ms;
  }
  if (launches) *launches = (int64_t)(used / 2);
  used = 0;
  op_check_wait_flag();  // the timed launches completed; none of their waits may have run out
  return total;
}
KernelTimer::~KernelTimer() {
  for (cudaEvent_t e : ev) cudaEventDestroy(e);
}

int64_t frozen_point_values_per_cell(int dim, int k) {
  // one cell's block [point][quad][lane][4 values] (FrozenPoint in op_apply.cuh)
  const int q = k + 1;
  const int64_t lanes = dim == 3 ? q * q : q;
  const int nfq = dim + dim * dim + dim + 1;
  return lanes * q * ((nfq + 3) / 4) * 4;
}

void op_precompute_frozen(const OpLaunch& L, int prec, cudaStream_t s) {
  if (L.op != OP_STAB_NS || !L.fq[prec]) return;
  if (prec == 0)
    dispatch<double>(L, nullptr, nullptr, false, s, 2);
  else
    dispatch<float>(L, nullptr, nullptr, false, s, 2);
}

void op_residual(const OpLaunch& L, int prec, void* dst, cudaStream_t s) {
  if (L.op != OP_STAB_NS) throw Error(kErrArg, "residual: not a stabilised NS operator");
  if (prec == 0)
    dispatch<double>(L, nullptr, static_cast<double*>(dst), false, s, 3);
  else
    dispatch<float>(L, nullptr, static_cast<float*>(dst), false, s, 3);
}

int* op_wait_flag() {
  static std::mutex mu;
  static std::map<int, int*> flags;
  int dev = 0;
  MFNS_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  auto it = flags.find(dev);
  if (it != flags.end()) return it->second;
  int* p = nullptr;
  MFNS_CUDA(cudaMalloc(&p, sizeof(int)));
  MFNS_CUDA(cudaMemset(p, 0, sizeof(int)));
  flags[dev] = p;
  return p;
}

void op_check_wait_flag() {
  int* p = op_wait_flag();
  int h = 0;
  MFNS_CUDA(cudaMemcpy(&h, p, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    MFNS_CUDA(cudaMemset(p, 0, sizeof(int)));
    throw Error(kErrTimeout, "a cell kernel's wait for its staged frozen block ran out (results invalid)");
  }
}

int autotune_warps(OpLaunch& L, int prec, void* src, void* dst, int64_t n, cudaStream_t s) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int, bool>, int> cache;
  const auto key = std::make_tuple(L.dim, L.k, L.op, prec, L.structured);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return L.warps[prec] = it->second;
  }
  (void)n;
  cudaEvent_t e0, e1;
  MFNS_CUDA(cudaEventCreate(&e0));
  MFNS_CUDA(cudaEventCreate(&e1));
  KernelTimer* saved = L.timer;
  L.timer = nullptr;
  int best = kOpWarpsDefault;
  float best_ms = 1e30f;
  for (int w : {1, 2, 4}) {
    L.warps[prec] = w;
    op_apply(L, prec, src, dst, false, s);  // warm-up
    MFNS_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < 3; ++r) op_apply(L, prec, src, dst, false, s);
    MFNS_CUDA(cudaEventRecord(e1, s));
    MFNS_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    MFNS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_ms * 0.98f) {  // prefer the earlier (smaller) block size unless clearly slower
      best_ms = ms;
      best = w;
    }
  }
  L.timer = saved;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  op_check_wait_flag();
  L.warps[prec] = best;
  std::lock_guard<std::mutex> lock(mu);
  cache[key] = best;
  return best;
}

void op_apply(const OpLaunch& L, int prec, const void* src, void* dst, bool diag, cudaStream_t s) {
  if (prec == 0)
    dispatch<double>(L, static_cast<const double*>(src), static_cast<double*>(dst), diag, s);
  else
    dispatch<float>(L, static_cast<const float*>(src), static_cast<float*>(dst), diag, s);
}

void op_apply_multi(const OpLaunch& L, int prec, int color, const MultiColour& mc, cudaStream_t s) {
#define MFNS_CASE(DIM, K, OP)                                           \
  if (L.dim == DIM && L.k == K && L.op == OP) {                         \
    if (prec == 0) return op_launch_multi<DIM, K, OP, double>(L, color, mc, s); \
    return op_launch_multi<DIM, K, OP, float>(L, color, mc, s);         \
  }
  MFNS_CASE(3, 1, OP_STAB_NS) MFNS_CASE(3, 2, OP_STAB_NS) MFNS_CASE(3, 3, OP_STAB_NS)
  MFNS_CASE(2, 1, OP_STAB_NS) MFNS_CASE(2, 2, OP_STAB_NS) MFNS_CASE(2, 3, OP_STAB_NS) MFNS_CASE(2, 4, OP_STAB_NS)
  MFNS_CASE(3, 1, OP_STOKES_A) MFNS_CASE(3, 2, OP_STOKES_A) MFNS_CASE(3, 3, OP_STOKES_A) MFNS_CASE(3, 4, OP_STOKES_A)
  MFNS_CASE(2, 1, OP_STOKES_A) MFNS_CASE(2, 2, OP_STOKES_A) MFNS_CASE(2, 3, OP_STOKES_A) MFNS_CASE(2, 4, OP_STOKES_A)
  MFNS_CASE(2, 1, OP_PMASS) MFNS_CASE(2, 2, OP_PMASS) MFNS_CASE(2, 3, OP_PMASS)
  MFNS_CASE(3, 1, OP_PMASS) MFNS_CASE(3, 2, OP_PMASS) MFNS_CASE(3, 3, OP_PMASS)
#undef MFNS_CASE
  throw Error(kErrUnsupported, "multi-problem launch: unsupported (dim, degree, operator)");
}

// dst = 0, then lets the colour launches that follow start early.  16-byte stores when dst is
// 16-byte aligned; element stores otherwise (the library's own callers pass sub-vectors, e.g. the
// stages of a space-time vector, that are only element-aligned).
template <typename T>
__global__ void k_clear_then_release(T* y, int64_t n) {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((reinterpret_cast<uintptr_t>(y) & 15u) == 0) {
    constexpr int V = 16 / sizeof(T);
    const int64_t nv = n / V;
    for (int64_t i = i0; i < nv; i += stride) reinterpret_cast<float4*>(y)[i] = make_float4(0, 0, 0, 0);
    for (int64_t i = nv * V + i0; i < n; i += stride) y[i] = T(0);
  } else {
    for (int64_t i = i0; i < n; i += stride) y[i] = T(0);
  }
}

// dst = src on the rows marked in keep (bit i % 32 of word i / 32), 0 elsewhere, then lets the
// colour launches that follow start early.  16-byte accesses when both vectors are 16-byte aligned
// (the 16 / sizeof(T) entries of one access share a mask word), element accesses otherwise.
template <typename T>
__global__ void k_clear_keep_then_release(T* y, const T* x, const uint32_t* __restrict__ keep, int64_t n) {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  auto bit = [&](int64_t i) { return (keep[i >> 5] >> (i & 31)) & 1u; };
  int64_t done = 0;
  if (((reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(x)) & 15u) == 0) {
    constexpr int V = 16 / sizeof(T);
    const int64_t nv = n / V;
    for (int64_t i = i0; i < nv; i += stride) {
      const uint32_t b = (keep[(i * V) >> 5] >> ((i * V) & 31)) & ((1u << V) - 1u);
      float4 v = make_float4(0, 0, 0, 0);
      if (b) {
        v = reinterpret_cast<const float4*>(x)[i];
        T* e = reinterpret_cast<T*>(&v);
#pragma unroll
        for (int j = 0; j < V; ++j)
          if (!((b >> j) & 1u)) e[j] = T(0);
      }
      reinterpret_cast<float4*>(y)[i] = v;
    }
    done = nv * V;
  }
  for (int64_t i = done + i0; i < n; i += stride) y[i] = bit(i) ? x[i] : T(0);
}

struct ColourOffsets {
  int64_t off[8];
};

// a + b rounded as the L2's FP32 reduction rounds it (subnormal inputs and result flushed to
// zero), so that a gathered sum equals the colour-ordered reductions bit for bit; the FP64
// reduction does not flush
__device__ __forceinline__ float add_as_reduction(float a, float b) {
  float r;
  asm("add.rn.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ double add_as_reduction(double a, double b) { return a + b; }

// dst = A src on a uniform 3D level (NU components per node, the first NVEL velocity) from the
// per-cell contributions of a deferred product: every node adds its cells' contributions in colour
// order, starting from zero -- the additions, in the same order, that the colour launches'
// reductions make onto a cleared vector -- and the identity rows (velocity of boundary nodes) get
// src + 0 (src plus the zeros the colours add there).  Node (i0, i1, i2) of the (k n + 1)^3 lattice
// lies in one cell along a direction where i_d is not a multiple of k, else in the cells i_d / k - 1
// and i_d / k that exist; the colour of a cell is the parity of its coordinates.
template <typename T, int NU, int NVEL>
__global__ void k_gather_cells(T* __restrict__ dst, const T* __restrict__ src, const T* __restrict__ defer, int n,
                               int K, ColourOffsets co) {
  const int64_t M = (int64_t)K * n + 1, nn = M * M * M;
  const int nb1 = K + 1, nbc = nb1 * nb1 * nb1;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i[3] = {g % M, (g / M) % M, g / (M * M)};
    T acc[NU];
#pragma unroll
    for (int f = 0; f < NU; ++f) acc[f] = T(0);
    for (int c = 0; c < 8; ++c) {
      int64_t cd[3];
      int loc[3];
      bool ok = true;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int64_t b = (c >> d) & 1;
        const int64_t q = i[d] / K, r = i[d] - q * K;
        int64_t cell;
        if (r != 0) {
          cell = q;
          ok = ok && (cell & 1) == b;
        } else if ((q & 1) == b) {
          cell = q;
          ok = ok && q < n;
        } else {
          cell = q - 1;
          ok = ok && q >= 1;
        }
        cd[d] = cell;
        loc[d] = (int)(i[d] - (int64_t)K * cell);
      }
      if (!ok) continue;
      // the cell's position in the colour-major enumeration of the cell kernels
      const int64_t m0 = (n - (c & 1) + 1) / 2, m1 = (n - ((c >> 1) & 1) + 1) / 2;
      const int64_t pos = co.off[c] + (cd[0] >> 1) + m0 * ((cd[1] >> 1) + m1 * (cd[2] >> 1));
      const int slot = (loc[2] * nb1 + loc[1]) * nb1 + loc[0];
      const T* v = defer + ((size_t)pos * nbc + slot) * NU;
#pragma unroll
      for (int f = 0; f < NU; ++f) acc[f] = add_as_reduction(acc[f], v[f]);
    }
    const bool bnd = i[0] == 0 || i[0] == M - 1 || i[1] == 0 || i[1] == M - 1 || i[2] == 0 || i[2] == M - 1;
#pragma unroll
    for (int f = 0; f < NU; ++f)
      dst[g * NU + f] = (f < NVEL && bnd) ? add_as_reduction(src[g * NU + f], T(0)) : acc[f];
  }
}

void op_apply_deferred(const OpLaunch& L, int prec, const void* src, void* dst, void* defer, cudaStream_t s) {
  if (L.dim != 3 || (L.op != OP_STAB_NS && L.op != OP_STOKES_A && L.op != OP_PMASS) || !L.structured)
    throw Error(kErrArg, "deferred products: uniform 3D stabilised, vector-Laplacian or pressure-mass levels");
#define MFNS_CASE(K, OP)                                                                                      \
  if (L.k == K && L.op == OP) {                                                                               \
    if (prec == 0)                                                                                            \
      op_launch_deferred<3, K, OP, double>(L, static_cast<const double*>(src), static_cast<double*>(defer), s); \
    else                                                                                                      \
      op_launch_deferred<3, K, OP, float>(L, static_cast<const float*>(src), static_cast<float*>(defer), s);    \
  } else
  MFNS_CASE(1, OP_STAB_NS) MFNS_CASE(2, OP_STAB_NS) MFNS_CASE(3, OP_STAB_NS)
  MFNS_CASE(1, OP_STOKES_A) MFNS_CASE(2, OP_STOKES_A) MFNS_CASE(3, OP_STOKES_A) MFNS_CASE(4, OP_STOKES_A)
  MFNS_CASE(1, OP_PMASS) MFNS_CASE(2, OP_PMASS) MFNS_CASE(3, OP_PMASS)
  throw Error(kErrUnsupported, "deferred products: degree");
#undef MFNS_CASE
  ColourOffsets co{};
  int64_t off = 0;
  for (int c = 0; c < 8; ++c) {
    int64_t nc = 1;
    for (int d = 0; d < 3; ++d) nc *= (L.n - ((c >> d) & 1) + 1) / 2;
    co.off[c] = off;
    off += nc;
  }
  const int64_t M = (int64_t)L.k * L.n + 1, nn = M * M * M;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nn + 255) / 256, 152 * 16));
  auto go = [&](auto tag, auto nu_tag, auto nvel_tag) {
    using T = decltype(tag);
    constexpr int NU = decltype(nu_tag)::value, NVEL = decltype(nvel_tag)::value;
    k_gather_cells<T, NU, NVEL><<<grid, 256, 0, s>>>(static_cast<T*>(dst), static_cast<const T*>(src),
                                                     static_cast<const T*>(defer), L.n, L.k, co);
  };
  using I0 = std::integral_constant<int, 0>;
  using I1 = std::integral_constant<int, 1>;
  using I3 = std::integral_constant<int, 3>;
  using I4 = std::integral_constant<int, 4>;
  if (L.op == OP_STAB_NS) {
    if (prec == 0) go(double(), I4(), I3());
    else go(float(), I4(), I3());
  } else if (L.op == OP_STOKES_A) {
    if (prec == 0) go(double(), I3(), I3());
    else go(float(), I3(), I3());
  } else {  // pressure mass: one field, no identity rows
    if (prec == 0) go(double(), I1(), I0());
    else go(float(), I1(), I0());
  }
  MFNS_CUDA(cudaGetLastError());
}

void op_apply_cleared(const OpLaunch& L, int prec, const void* src, void* dst, int64_t n, cudaStream_t s,
                      const uint32_t* keep) {
  const int64_t nbytes = n * (prec == 0 ? 8 : 4);
  const unsigned grid = (unsigned)std::min<int64_t>((nbytes / 16 + 255) / 256 + 1, 152 * 8);
  if (keep && prec == 0)
    k_clear_keep_then_release<double><<<grid, 256, 0, s>>>(static_cast<double*>(dst),
                                                            static_cast<const double*>(src), keep, n);
  else if (keep)
    k_clear_keep_then_release<float><<<grid, 256, 0, s>>>(static_cast<float*>(dst), static_cast<const float*>(src),
                                                           keep, n);
  else if (prec == 0)
    k_clear_then_release<double><<<grid, 256, 0, s>>>(static_cast<double*>(dst), n);
  else
    k_clear_then_release<float><<<grid, 256, 0, s>>>(static_cast<float*>(dst), n);
  MFNS_CUDA(cudaGetLastError());
  OpEpilogue e;
  e.after_clear = true;
  if (prec == 0)
    dispatch<double>(L, static_cast<const double*>(src), static_cast<double*>(dst), false, s, -1, 1, 0, &e);
  else
    dispatch<float>(L, static_cast<const float*>(src), static_cast<float*>(dst), false, s, -1, 1, 0, &e);
}

void op_apply_epi(const OpLaunch& L, int prec, const void* src, void* dst, const OpEpilogue& epi, cudaStream_t s) {
  if (prec == 0)
    dispatch<double>(L, static_cast<const double*>(src), static_cast<double*>(dst), false, s, -1, 1, 0, &epi);
  else
    dispatch<float>(L, static_cast<const float*>(src), static_cast<float*>(dst), false, s, -1, 1, 0, &epi);
}

void op_apply_cols(const OpLaunch& L, int prec, const void* src, void* dst, int ncols, int64_t col_stride,
                   cudaStream_t s) {
  if (prec == 0)
    dispatch<double>(L, static_cast<const double*>(src), static_cast<double*>(dst), false, s, -1, ncols, col_stride);
  else
    dispatch<float>(L, static_cast<const float*>(src), static_cast<float*>(dst), false, s, -1, ncols, col_stride);
}

// Collocation derivative on the Gauss points: D[i][j] = l_j'(x_i), Lagrange basis on the Gauss points.
void fill_tables(OpLaunch& L) {
  const int q = L.op == OP_PMASS ? L.k + 1 : L.k + 1;
  L.Q = q;
  L.N = L.k + 1;
  L.NP = L.op == OP_STOKES ? L.k : L.k + 1;
  std::vector<double> xg, wg;
  gauss_rule(q, xg, wg);
  std::vector<double> xn = gll_nodes(L.k);
  L.S.assign(q * L.N, 0.0);
  for (int i = 0; i < q; ++i)
    for (int a = 0; a < L.N; ++a) L.S[i * L.N + a] = lagrange(xn, a, xg[i]);
  L.Sp.assign(q * L.NP, 0.0);
  if (L.op == OP_STOKES) {
    std::vector<double> xp = gll_nodes(L.k - 1);
    for (int i = 0; i < q; ++i)
      for (int a = 0; a < L.NP; ++a) L.Sp[i * L.NP + a] = lagrange(xp, a, xg[i]);
  }
  L.D.assign(q * q, 0.0);
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) L.D[i * q + j] = lagrange_deriv(xg, j, xg[i]);
  L.D2.assign(q * q, 0.0);
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) {
      double s = 0;
      for (int r = 0; r < q; ++r) s += L.D[i * q + r] * L.D[r * q + j];
      L.D2[i * q + j] = s;
    }
  L.W = wg;
  auto halves = [](int k, std::vector<double>& P) {
    std::vector<double> x = gll_nodes(k);
    int n = k + 1;
    P.assign(2 * n * n, 0.0);
    for (int h = 0; h < 2; ++h)
      for (int s = 0; s < n; ++s)
        for (int m = 0; m < n; ++m) P[(h * n + s) * n + m] = lagrange(x, m, 0.5 * (h + x[s]));
  };
  halves(L.k, L.P);
  if (L.op == OP_STOKES) halves(L.k - 1, L.Pp);
  else L.Pp.assign(2 * L.NP * L.NP, 0.0);
}

}  // namespace mfns
