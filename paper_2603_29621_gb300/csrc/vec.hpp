// Vector kernels used by the smoothers, transfers and Krylov solvers.
// Reductions are deterministic: a fixed grid writes per-block partial sums that
// a single block adds in a fixed order.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace mfns {

constexpr int kRedBlocks = 304;   // 2 x 152 SMs; fixed for determinism
constexpr int kRedThreads = 256;
constexpr int kMaxDots = 32;      // vectors per multi-dot

template <typename T> void vzero(T* x, int64_t n, cudaStream_t s);
template <typename T> void vcopy(T* y, const T* x, int64_t n, cudaStream_t s);
template <typename T> void vaxpy(T* y, T a, const T* x, int64_t n, cudaStream_t s);          // y += a x
template <typename T> void vaxpby(T* y, T a, const T* x, T b, int64_t n, cudaStream_t s);   // y = a x + b y
template <typename T> void vsub(T* r, const T* b, const T* ax, int64_t n, cudaStream_t s);   // r = b - ax
template <typename T> void vscale(T* y, T a, int64_t n, cudaStream_t s);
void vcast_d2f(float* y, const double* x, int64_t n, cudaStream_t s);
// X (n x nb, column-major) = columns j0 .. j0+nb-1 of the identity
void vunit_cols(double* X, int64_t n, int64_t j0, int64_t nb, cudaStream_t s);
// constrained (identity) rows of a fused smoothing step / residual
template <typename T>
void vcheby_idx(const T* x, T* xout, T* d, const T* b, const T* dinv, T c1, T c2, const int32_t* idx, int64_t m,
                cudaStream_t s);
template <typename T>
void vsub_idx(T* r, const T* b, const T* x, const int32_t* idx, int64_t m, cudaStream_t s);
// Y[:, j][idx] = X[:, j][idx] for the nb columns of length n
template <typename T>
void vcopy_idx_cols(T* Y, const T* X, const int32_t* idx, int64_t m, int64_t n, int64_t nb, cudaStream_t s);
// y = a x1 + b x2 + c x3 (x2, x3 may be null: their terms are left out)
void vlincomb3(double* y, double a, const double* x1, double b, const double* x2, double c, const double* x3,
               int64_t n, cudaStream_t s);
// *out (device) = bit pattern of max over nodes i of sum_{d < dim} x[i * stride + d]^2
void max_node_norm2(unsigned long long* out, const double* x, int64_t nodes, int stride, int dim, cudaStream_t s);
void vcast_f2d(double* y, const float* x, int64_t n, cudaStream_t s);
// y[idx[i]] = x[idx[i]]
template <typename T> void vcopy_idx(T* y, const T* x, const int32_t* idx, int64_t n, cudaStream_t s);
// y[idx[i]] = v
template <typename T> void vset_idx(T* y, T v, const int32_t* idx, int64_t n, cudaStream_t s);
// transpose of a constraint distribution: y[mdof[i]] += sum_{j in ptr[i]..ptr[i+1]} w[j] y[sdof[j]]
// (every mdof distinct and never an sdof)
template <typename T>
void vcondense(T* y, const int32_t* mdof, const int32_t* ptr, const int32_t* sdof, const T* w, int64_t n,
               cudaStream_t s);
// node-interleaved blocks of nc entries: y[ymap[i] * nc + c] = x[xmap[i] * nc + c], i < n, c < nc
template <typename T>
void vcopy_map(T* y, const int32_t* ymap, const T* x, const int32_t* xmap, int64_t n, int nc, cudaStream_t s);
// hanging entries: x[dof[i]] = sum_{j in ptr[i]..ptr[i+1]} w[j] x[src[j]]
template <typename T>
void vdistribute(T* x, const int32_t* dof, const int32_t* ptr, const int32_t* src, const T* w, int64_t n,
                 cudaStream_t s);
// Chebyshev step (Saad, Alg. 12.1 on D^-1 A): d = c1 d + c2 dinv (b - ax); x += d
template <typename T>
void vcheby(T* x, T* d, const T* b, const T* ax, const T* dinv, T c1, T c2, int64_t n, cudaStream_t s);
// Chebyshev step around a general preconditioner, z = P^{-1} (b - A x): d = c1 d + c2 z (c1 = 0: d
// not read); x += d
template <typename T>
void vcheby_pre(T* x, T* d, const T* z, T c1, T c2, int64_t n, cudaStream_t s);
// first step from a zero iterate: d = c2 dinv b; x = d
template <typename T> void vcheby0(T* x, T* d, const T* b, const T* dinv, T c2, int64_t n, cudaStream_t s);
// y = dinv * x (pointwise)
template <typename T> void vmul(T* y, const T* dinv, const T* x, int64_t n, cudaStream_t s);
// y = 1 / x
template <typename T> void vrecip(T* y, const T* x, int64_t n, cudaStream_t s);
// dense gemv y = M x (row-major n x n)
template <typename T> void vgemv(T* y, const T* M, const T* x, int64_t n, cudaStream_t s);

// Deterministic reductions into device scratch `part` (kRedBlocks * kMaxDots doubles) and
// the final result `out` (device, double): out[k] = sum_i V_k[i] w[i], k < m.
void multidot(double* out, const double* const* V, const double* w, int m, int64_t n, double* part,
              const double** Vdev, cudaStream_t s);
template <typename T> void dot(double* out, const T* a, const T* b, int64_t n, double* part, cudaStream_t s);
// w -= sum_k h[k] V_k (h on device)
void multi_axpy(double* w, const double* const* Vdev, const double* h, int m, int64_t n, cudaStream_t s);
// x += sum_k y[k] Z_k (y on device)
void multi_axpy_add(double* x, const double* const* Zdev, const double* y, int m, int64_t n, cudaStream_t s);
// sum of x over idx (device double result)
template <typename T> void sum_idx(double* out, const T* x, const int32_t* idx, int64_t n, double* part, cudaStream_t s);
// x[idx] -= (*mean_sum) / n
template <typename T> void sub_mean_idx(T* x, const int32_t* idx, int64_t n, const double* sum, cudaStream_t s);

// CG steps with device-resident scalars (no host round trip, capturable into CUDA graphs):
// alpha = num/den (0 when den == 0): x += alpha p, r -= alpha q
template <typename T>
void cg_step_xr(T* x, T* r, const T* p, const T* q, const double* num, const double* den, int64_t n, cudaStream_t s);
// beta = num/den (0 when den == 0): p = z + beta p
template <typename T>
void cg_step_p(T* p, const T* z, const double* num, const double* den, int64_t n, cudaStream_t s);

}  // namespace mfns
