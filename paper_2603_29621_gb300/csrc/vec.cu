// Vector kernels (see vec.hpp).
#include "common.hpp"
#include "vec.hpp"

namespace mfns {

namespace {
constexpr int kThreads = 256;
inline unsigned grid_for(int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g > 0 ? g : 1);
}
#define GRID_STRIDE(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

template <typename T> __global__ void k_zero(T* x, int64_t n) { GRID_STRIDE(i, n) x[i] = T(0); }
template <typename T> __global__ void k_copy(T* y, const T* x, int64_t n) { GRID_STRIDE(i, n) y[i] = x[i]; }
template <typename T> __global__ void k_axpy(T* y, T a, const T* x, int64_t n) { GRID_STRIDE(i, n) y[i] += a * x[i]; }
template <typename T> __global__ void k_axpby(T* y, T a, const T* x, T b, int64_t n) {
  GRID_STRIDE(i, n) y[i] = a * x[i] + b * y[i];
}
template <typename T> __global__ void k_sub(T* r, const T* b, const T* ax, int64_t n) { GRID_STRIDE(i, n) r[i] = b[i] - ax[i]; }
template <typename T> __global__ void k_scale(T* y, T a, int64_t n) { GRID_STRIDE(i, n) y[i] *= a; }
__global__ void k_d2f(float* y, const double* x, int64_t n) { GRID_STRIDE(i, n) y[i] = (float)x[i]; }
__global__ void k_unit_cols(double* X, int64_t n, int64_t j0, int64_t nb) {
  GRID_STRIDE(t, n * nb) {
    const int64_t j = t / n, i = t - j * n;
    X[t] = i == j0 + j ? 1.0 : 0.0;
  }
}
template <typename T>
__global__ void k_cheby_idx(const T* x, T* xout, T* d, const T* b, const T* dinv, T c1, T c2, const int32_t* idx,
                            int64_t m) {
  GRID_STRIDE(t, m) {
    const int32_t i = idx[t];
    // identity row: (A x)_i = x_i; c1 = 0 (a first step) does not read d, which may be unset
    const T di = (c1 != T(0) ? c1 * d[i] : T(0)) + c2 * dinv[i] * (b[i] - x[i]);
    d[i] = di;
    xout[i] = x[i] + di;
  }
}
template <typename T>
__global__ void k_sub_idx(T* r, const T* b, const T* x, const int32_t* idx, int64_t m) {
  GRID_STRIDE(t, m) {
    const int32_t i = idx[t];
    r[i] = b[i] - x[i];
  }
}
template <typename T>
__global__ void k_copy_idx_cols(T* Y, const T* X, const int32_t* idx, int64_t m, int64_t n, int64_t nb) {
  GRID_STRIDE(t, m * nb) {
    const int64_t j = t / m, i = idx[t - j * m];
    Y[j * n + i] = X[j * n + i];
  }
}
__global__ void k_lincomb3(double* y, double a, const double* x1, double b, const double* x2, double c,
                           const double* x3, int64_t n) {
  GRID_STRIDE(i, n) {
    double v = a * x1[i];
    if (x2) v += b * x2[i];
    if (x3) v += c * x3[i];
    y[i] = v;
  }
}
// max over nodes of the squared Euclidean norm of the first `dim` entries of each node's record;
// the maximum is order independent, and non-negative doubles order like their bit patterns
__global__ void k_max_node_norm2(unsigned long long* out, const double* x, int64_t nodes, int stride, int dim) {
  double m = 0.0;
  GRID_STRIDE(i, nodes) {
    double s = 0.0;
    for (int d = 0; d < dim; ++d) {
      const double v = x[i * stride + d];
      s += v * v;
    }
    m = fmax(m, s);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}
__global__ void k_f2d(double* y, const float* x, int64_t n) { GRID_STRIDE(i, n) y[i] = (double)x[i]; }
template <typename T> __global__ void k_copy_idx(T* y, const T* x, const int32_t* idx, int64_t n) {
  GRID_STRIDE(i, n) y[idx[i]] = x[idx[i]];
}
template <typename T> __global__ void k_set_idx(T* y, T v, const int32_t* idx, int64_t n) { GRID_STRIDE(i, n) y[idx[i]] = v; }
template <typename T>
__global__ void k_condense(T* y, const int32_t* mdof, const int32_t* ptr, const int32_t* sdof, const T* w, int64_t n) {
  GRID_STRIDE(i, n) {
    T acc = T(0);
    for (int32_t j = ptr[i]; j < ptr[i + 1]; ++j) acc += w[j] * y[sdof[j]];
    y[mdof[i]] += acc;
  }
}
template <typename T>
__global__ void k_copy_map(T* y, const int32_t* ymap, const T* x, const int32_t* xmap, int64_t n, int nc) {
  GRID_STRIDE(t, n * nc) {
    const int64_t i = t / nc, c = t - i * nc;
    y[(int64_t)ymap[i] * nc + c] = x[(int64_t)xmap[i] * nc + c];
  }
}
template <typename T>
__global__ void k_distribute(T* x, const int32_t* dof, const int32_t* ptr, const int32_t* src, const T* w, int64_t n) {
  GRID_STRIDE(i, n) {
    T s = 0;
    for (int32_t j = ptr[i]; j < ptr[i + 1]; ++j) s += w[j] * x[src[j]];
    x[dof[i]] = s;
  }
}
template <typename T>
__global__ void k_cheby(T* x, T* d, const T* b, const T* ax, const T* dinv, T c1, T c2, int64_t n) {
  GRID_STRIDE(i, n) {
    const T di = (c1 != T(0) ? c1 * d[i] : T(0)) + c2 * dinv[i] * (b[i] - ax[i]);  // c1 = 0: d not read
    d[i] = di;
    x[i] += di;
  }
}
template <typename T> __global__ void k_cheby_pre(T* x, T* d, const T* z, T c1, T c2, int64_t n) {
  GRID_STRIDE(i, n) {
    const T di = (c1 != T(0) ? c1 * d[i] : T(0)) + c2 * z[i];
    d[i] = di;
    x[i] += di;
  }
}
template <typename T> __global__ void k_cheby0(T* x, T* d, const T* b, const T* dinv, T c2, int64_t n) {
  GRID_STRIDE(i, n) {
    const T di = c2 * dinv[i] * b[i];
    d[i] = di;
    x[i] = di;
  }
}
template <typename T> __global__ void k_mul(T* y, const T* dinv, const T* x, int64_t n) { GRID_STRIDE(i, n) y[i] = dinv[i] * x[i]; }
template <typename T> __global__ void k_recip(T* y, const T* x, int64_t n) { GRID_STRIDE(i, n) y[i] = T(1) / x[i]; }
template <typename T> __global__ void k_gemv(T* y, const T* M, const T* x, int64_t n) {
  // one warp per row, fixed summation order
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0;
  for (int64_t j = lane; j < n; j += 32) s += (double)M[row * n + j] * (double)x[j];
  for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = (T)s;
}

// block reduction of kRedThreads doubles
__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = kRedThreads / 2; o; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void k_multidot_part(double* part, const double* const* V, const double* w, int m, int64_t n) {
  __shared__ double sh[kRedThreads];
  for (int k = 0; k < m; ++k) {
    double s = 0;
    const double* v = V[k];
    for (int64_t i = blockIdx.x * (int64_t)kRedThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRedThreads)
      s += v[i] * w[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[k * gridDim.x + blockIdx.x] = s;
  }
}
__global__ void k_final(double* out, const double* part, int m, int nb) {
  __shared__ double sh[kRedThreads];
  for (int k = 0; k < m; ++k) {
    double s = 0;
    for (int i = threadIdx.x; i < nb; i += kRedThreads) s += part[k * nb + i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) out[k] = s;
  }
}
template <typename T> __global__ void k_dot_part(double* part, const T* a, const T* b, int64_t n) {
  __shared__ double sh[kRedThreads];
  double s = 0;
  for (int64_t i = blockIdx.x * (int64_t)kRedThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRedThreads)
    s += (double)a[i] * (double)b[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}
template <typename T> __global__ void k_sum_idx_part(double* part, const T* x, const int32_t* idx, int64_t n) {
  __shared__ double sh[kRedThreads];
  double s = 0;
  for (int64_t i = blockIdx.x * (int64_t)kRedThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRedThreads)
    s += (double)x[idx[i]];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}
template <typename T> __global__ void k_sub_mean_idx(T* x, const int32_t* idx, int64_t n, const double* sum) {
  const T mean = (T)(*sum / (double)n);
  GRID_STRIDE(i, n) x[idx[i]] -= mean;
}
__global__ void k_multi_axpy(double* w, const double* const* V, const double* h, int m, int64_t n) {
  GRID_STRIDE(i, n) {
    double s = w[i];
    for (int k = 0; k < m; ++k) s -= h[k] * V[k][i];
    w[i] = s;
  }
}
__global__ void k_multi_axpy_add(double* x, const double* const* Z, const double* y, int m, int64_t n) {
  GRID_STRIDE(i, n) {
    double s = x[i];
    for (int k = 0; k < m; ++k) s += y[k] * Z[k][i];
    x[i] = s;
  }
}
template <typename T>
__global__ void k_cg_xr(T* x, T* r, const T* p, const T* q, const double* num, const double* den, int64_t n) {
  const double d = *den;
  const T alpha = (T)(d != 0.0 ? *num / d : 0.0);
  GRID_STRIDE(i, n) {
    x[i] += alpha * p[i];
    r[i] -= alpha * q[i];
  }
}
template <typename T>
__global__ void k_cg_p(T* p, const T* z, const double* num, const double* den, int64_t n) {
  const double d = *den;
  const T beta = (T)(d != 0.0 ? *num / d : 0.0);
  GRID_STRIDE(i, n) p[i] = z[i] + beta * p[i];
}
}  // namespace

#define LAUNCH(kern, n, s, ...)                                    \
  do {                                                             \
    if ((n) > 0) kern<<<grid_for(n), kThreads, 0, s>>>(__VA_ARGS__); \
    MFNS_CUDA(cudaGetLastError());                                 \
  } while (0)

template <typename T> void vzero(T* x, int64_t n, cudaStream_t s) { LAUNCH(k_zero<T>, n, s, x, n); }
template <typename T> void vcopy(T* y, const T* x, int64_t n, cudaStream_t s) { LAUNCH(k_copy<T>, n, s, y, x, n); }
template <typename T> void vaxpy(T* y, T a, const T* x, int64_t n, cudaStream_t s) { LAUNCH(k_axpy<T>, n, s, y, a, x, n); }
template <typename T> void vaxpby(T* y, T a, const T* x, T b, int64_t n, cudaStream_t s) {
  LAUNCH(k_axpby<T>, n, s, y, a, x, b, n);
}
template <typename T> void vsub(T* r, const T* b, const T* ax, int64_t n, cudaStream_t s) { LAUNCH(k_sub<T>, n, s, r, b, ax, n); }
template <typename T> void vscale(T* y, T a, int64_t n, cudaStream_t s) { LAUNCH(k_scale<T>, n, s, y, a, n); }
void vcast_d2f(float* y, const double* x, int64_t n, cudaStream_t s) { LAUNCH(k_d2f, n, s, y, x, n); }
void vunit_cols(double* X, int64_t n, int64_t j0, int64_t nb, cudaStream_t s) {
  LAUNCH(k_unit_cols, n * nb, s, X, n, j0, nb);
}
template <typename T>
void vcopy_idx_cols(T* Y, const T* X, const int32_t* idx, int64_t m, int64_t n, int64_t nb, cudaStream_t s) {
  LAUNCH(k_copy_idx_cols<T>, m * nb, s, Y, X, idx, m, n, nb);
}
template <typename T>
void vcheby_idx(const T* x, T* xout, T* d, const T* b, const T* dinv, T c1, T c2, const int32_t* idx, int64_t m,
                cudaStream_t s) {
  LAUNCH(k_cheby_idx<T>, m, s, x, xout, d, b, dinv, c1, c2, idx, m);
}
template <typename T>
void vsub_idx(T* r, const T* b, const T* x, const int32_t* idx, int64_t m, cudaStream_t s) {
  LAUNCH(k_sub_idx<T>, m, s, r, b, x, idx, m);
}
template void vcheby_idx<double>(const double*, double*, double*, const double*, const double*, double, double,
                                 const int32_t*, int64_t, cudaStream_t);
template void vcheby_idx<float>(const float*, float*, float*, const float*, const float*, float, float,
                                const int32_t*, int64_t, cudaStream_t);
template void vsub_idx<double>(double*, const double*, const double*, const int32_t*, int64_t, cudaStream_t);
template void vsub_idx<float>(float*, const float*, const float*, const int32_t*, int64_t, cudaStream_t);
template void vcopy_idx_cols<double>(double*, const double*, const int32_t*, int64_t, int64_t, int64_t, cudaStream_t);
template void vcopy_idx_cols<float>(float*, const float*, const int32_t*, int64_t, int64_t, int64_t, cudaStream_t);
void vlincomb3(double* y, double a, const double* x1, double b, const double* x2, double c, const double* x3,
               int64_t n, cudaStream_t s) {
  LAUNCH(k_lincomb3, n, s, y, a, x1, b, x2, c, x3, n);
}
void max_node_norm2(unsigned long long* out, const double* x, int64_t nodes, int stride, int dim, cudaStream_t s) {
  MFNS_CUDA(cudaMemsetAsync(out, 0, sizeof(unsigned long long), s));
  LAUNCH(k_max_node_norm2, nodes, s, out, x, nodes, stride, dim);
}
void vcast_f2d(double* y, const float* x, int64_t n, cudaStream_t s) { LAUNCH(k_f2d, n, s, y, x, n); }
template <typename T> void vcopy_idx(T* y, const T* x, const int32_t* idx, int64_t n, cudaStream_t s) {
  LAUNCH(k_copy_idx<T>, n, s, y, x, idx, n);
}
template <typename T> void vset_idx(T* y, T v, const int32_t* idx, int64_t n, cudaStream_t s) {
  LAUNCH(k_set_idx<T>, n, s, y, v, idx, n);
}
template <typename T>
void vcondense(T* y, const int32_t* mdof, const int32_t* ptr, const int32_t* sdof, const T* w, int64_t n, cudaStream_t s) {
  LAUNCH(k_condense<T>, n, s, y, mdof, ptr, sdof, w, n);
}
template <typename T>
void vcopy_map(T* y, const int32_t* ymap, const T* x, const int32_t* xmap, int64_t n, int nc, cudaStream_t s) {
  LAUNCH(k_copy_map<T>, n * nc, s, y, ymap, x, xmap, n, nc);
}
template <typename T>
void vdistribute(T* x, const int32_t* dof, const int32_t* ptr, const int32_t* src, const T* w, int64_t n, cudaStream_t s) {
  LAUNCH(k_distribute<T>, n, s, x, dof, ptr, src, w, n);
}
template <typename T>
void vcheby(T* x, T* d, const T* b, const T* ax, const T* dinv, T c1, T c2, int64_t n, cudaStream_t s) {
  LAUNCH(k_cheby<T>, n, s, x, d, b, ax, dinv, c1, c2, n);
}
template <typename T>
void vcheby_pre(T* x, T* d, const T* z, T c1, T c2, int64_t n, cudaStream_t s) {
  LAUNCH(k_cheby_pre<T>, n, s, x, d, z, c1, c2, n);
}
template void vcheby_pre<double>(double*, double*, const double*, double, double, int64_t, cudaStream_t);
template void vcheby_pre<float>(float*, float*, const float*, float, float, int64_t, cudaStream_t);
template <typename T> void vcheby0(T* x, T* d, const T* b, const T* dinv, T c2, int64_t n, cudaStream_t s) {
  LAUNCH(k_cheby0<T>, n, s, x, d, b, dinv, c2, n);
}
template <typename T> void vmul(T* y, const T* dinv, const T* x, int64_t n, cudaStream_t s) { LAUNCH(k_mul<T>, n, s, y, dinv, x, n); }
template <typename T> void vrecip(T* y, const T* x, int64_t n, cudaStream_t s) { LAUNCH(k_recip<T>, n, s, y, x, n); }
template <typename T> void vgemv(T* y, const T* M, const T* x, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  const unsigned grid = (unsigned)((n * 32 + 255) / 256);
  k_gemv<T><<<grid, 256, 0, s>>>(y, M, x, n);
  MFNS_CUDA(cudaGetLastError());
}

void multidot(double* out, const double* const* V, const double* w, int m, int64_t n, double* part,
              const double** Vdev, cudaStream_t s) {
  (void)V;
  k_multidot_part<<<kRedBlocks, kRedThreads, 0, s>>>(part, Vdev, w, m, n);
  MFNS_CUDA(cudaGetLastError());
  k_final<<<1, kRedThreads, 0, s>>>(out, part, m, kRedBlocks);
  MFNS_CUDA(cudaGetLastError());
}
template <typename T> void dot(double* out, const T* a, const T* b, int64_t n, double* part, cudaStream_t s) {
  k_dot_part<T><<<kRedBlocks, kRedThreads, 0, s>>>(part, a, b, n);
  MFNS_CUDA(cudaGetLastError());
  k_final<<<1, kRedThreads, 0, s>>>(out, part, 1, kRedBlocks);
  MFNS_CUDA(cudaGetLastError());
}
void multi_axpy(double* w, const double* const* Vdev, const double* h, int m, int64_t n, cudaStream_t s) {
  LAUNCH(k_multi_axpy, n, s, w, Vdev, h, m, n);
}
void multi_axpy_add(double* x, const double* const* Zdev, const double* y, int m, int64_t n, cudaStream_t s) {
  LAUNCH(k_multi_axpy_add, n, s, x, Zdev, y, m, n);
}
template <typename T> void sum_idx(double* out, const T* x, const int32_t* idx, int64_t n, double* part, cudaStream_t s) {
  k_sum_idx_part<T><<<kRedBlocks, kRedThreads, 0, s>>>(part, x, idx, n);
  MFNS_CUDA(cudaGetLastError());
  k_final<<<1, kRedThreads, 0, s>>>(out, part, 1, kRedBlocks);
  MFNS_CUDA(cudaGetLastError());
}
template <typename T> void sub_mean_idx(T* x, const int32_t* idx, int64_t n, const double* sum, cudaStream_t s) {
  LAUNCH(k_sub_mean_idx<T>, n, s, x, idx, n, sum);
}

template <typename T>
void cg_step_xr(T* x, T* r, const T* p, const T* q, const double* num, const double* den, int64_t n, cudaStream_t s) {
  LAUNCH(k_cg_xr<T>, n, s, x, r, p, q, num, den, n);
}
template <typename T>
void cg_step_p(T* p, const T* z, const double* num, const double* den, int64_t n, cudaStream_t s) {
  LAUNCH(k_cg_p<T>, n, s, p, z, num, den, n);
}

#define INST(T)                                                                                     \
  template void vzero<T>(T*, int64_t, cudaStream_t);                                                \
  template void vcopy<T>(T*, const T*, int64_t, cudaStream_t);                                      \
  template void vaxpy<T>(T*, T, const T*, int64_t, cudaStream_t);                                   \
  template void vaxpby<T>(T*, T, const T*, T, int64_t, cudaStream_t);                               \
  template void vsub<T>(T*, const T*, const T*, int64_t, cudaStream_t);                             \
  template void vscale<T>(T*, T, int64_t, cudaStream_t);                                            \
  template void vcopy_idx<T>(T*, const T*, const int32_t*, int64_t, cudaStream_t);                  \
  template void vset_idx<T>(T*, T, const int32_t*, int64_t, cudaStream_t);                          \
  template void vcopy_map<T>(T*, const int32_t*, const T*, const int32_t*, int64_t, int, cudaStream_t); \
  template void vcondense<T>(T*, const int32_t*, const int32_t*, const int32_t*, const T*, int64_t, cudaStream_t); \
  template void vdistribute<T>(T*, const int32_t*, const int32_t*, const int32_t*, const T*, int64_t, cudaStream_t); \
  template void vcheby<T>(T*, T*, const T*, const T*, const T*, T, T, int64_t, cudaStream_t);       \
  template void vcheby0<T>(T*, T*, const T*, const T*, T, int64_t, cudaStream_t);                   \
  template void vmul<T>(T*, const T*, const T*, int64_t, cudaStream_t);                             \
  template void vrecip<T>(T*, const T*, int64_t, cudaStream_t);                                     \
  template void vgemv<T>(T*, const T*, const T*, int64_t, cudaStream_t);                            \
  template void dot<T>(double*, const T*, const T*, int64_t, double*, cudaStream_t);                \
  template void sum_idx<T>(double*, const T*, const int32_t*, int64_t, double*, cudaStream_t);      \
  template void sub_mean_idx<T>(T*, const int32_t*, int64_t, const double*, cudaStream_t);        \
  template void cg_step_xr<T>(T*, T*, const T*, const T*, const double*, const double*, int64_t, cudaStream_t); \
  template void cg_step_p<T>(T*, const T*, const double*, const double*, int64_t, cudaStream_t);
INST(float)
INST(double)

}  // namespace mfns
