// Separable transfers between uniform meshes (Eq. 4 on tensor-product grids), nested
// (n -> n/2) or non-nested (odd n -> (n+1)/2, Section 2) h-steps and p-steps.
//
// On a uniform mesh the Q_k space is the tensor product of 1D spaces, and the
// interpolation P of Eq. 4 (coarse FE function evaluated at the fine nodes) is
// the tensor product of one 1D matrix P1 per direction: h-steps (n -> 2n cells,
// same degree) and p-steps (same cells, degree k-1 -> k) alike.  Restriction
// (P^T) and prolongation are therefore applied as one 1D stencil pass per
// direction over the global node grid: no cell loop, no colouring, coalesced
// neighbour reads along every axis.  Constrained (Dirichlet) velocity entries are
// masked exactly as in the cell-based transfer: P ignores the coarse ones and
// gives zero on the fine ones, so the restriction reads fine boundary velocity
// entries as zero and the prolongation never adds into them.
#include "problem.hpp"
#include "vec.hpp"

namespace mfns {

namespace {

// One 1D pass along `axis` of a grid (Mx, My, Mz) -> (Mx', My', Mz') with only the axis
// extent changing.  out[node'] (+)= sum_j w_j in[node along axis = idx_j].
// Masks: mask_in zeroes velocity components of input nodes on the boundary of the input
// grid (first pass only); skip_out leaves velocity components of output boundary nodes
// untouched (last pass of the prolongation only).  ADD: out += result, else out = result.
template <typename T, int NC, bool ADD>
__global__ void k_pass(const T* __restrict__ in, T* __restrict__ out, int axis, int64_t ix, int64_t iy, int64_t iz,
                       int64_t mo, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                       const T* __restrict__ w, int nvel, int mask_in, int skip_out) {
  int64_t ext_in[3] = {ix, iy, iz};
  int64_t ext_out[3] = {ix, iy, iz};
  ext_out[axis] = mo;
  const int64_t total = ext_out[0] * ext_out[1] * ext_out[2];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t c[3] = {t % ext_out[0], (t / ext_out[0]) % ext_out[1], t / (ext_out[0] * ext_out[1])};
    const int64_t o = c[axis];
    T acc[NC];
#pragma unroll
    for (int f = 0; f < NC; ++f) acc[f] = 0;
    bool in_bnd_other = false;
    if (mask_in) {
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (d != axis && ext_in[d] > 1) in_bnd_other |= c[d] == 0 || c[d] == ext_in[d] - 1;
    }
    for (int32_t j = ptr[o]; j < ptr[o + 1]; ++j) {
      int64_t ci[3] = {c[0], c[1], c[2]};
      ci[axis] = idx[j];
      const T* src = in + ((ci[2] * ext_in[1] + ci[1]) * ext_in[0] + ci[0]) * NC;
      const bool bnd = mask_in && (in_bnd_other || ci[axis] == 0 || ci[axis] == ext_in[axis] - 1);
      const T wj = w[j];
#pragma unroll
      for (int f = 0; f < NC; ++f) acc[f] += (bnd && f < nvel) ? T(0) : wj * src[f];
    }
    T* dst = out + t * NC;
    bool skip = false;
    if (skip_out) {
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (ext_out[d] > 1) skip |= c[d] == 0 || c[d] == ext_out[d] - 1;
    }
#pragma unroll
    for (int f = 0; f < NC; ++f) {
      if (ADD) {
        if (!(skip && f < nvel)) dst[f] += acc[f];
      } else {
        dst[f] = acc[f];
      }
    }
  }
}

template <typename T, int NC>
void pass(const T* in, T* out, int axis, const int64_t ext[3], int64_t mo, const DevBuf& ptr, const DevBuf& idx,
          const DevBuf& w, int nvel, bool mask_in, bool skip_out, bool add, cudaStream_t s) {
  int64_t eo[3] = {ext[0], ext[1], ext[2]};
  eo[axis] = mo;
  const int64_t total = eo[0] * eo[1] * eo[2];
  const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16);
  if (add)
    k_pass<T, NC, true><<<grid, 256, 0, s>>>(in, out, axis, ext[0], ext[1], ext[2], mo, ptr.as<int32_t>(),
                                             idx.as<int32_t>(), w.as<T>(), nvel, mask_in, skip_out);
  else
    k_pass<T, NC, false><<<grid, 256, 0, s>>>(in, out, axis, ext[0], ext[1], ext[2], mo, ptr.as<int32_t>(),
                                              idx.as<int32_t>(), w.as<T>(), nvel, mask_in, skip_out);
  MFNS_CUDA(cudaGetLastError());
}

// CSR of a 1D matrix given as dense rows (drop exact zeros)
void to_csr(const std::vector<double>& M, int64_t rows, int64_t cols, std::vector<int32_t>& ptr,
            std::vector<int32_t>& idx, std::vector<double>& w) {
  ptr.assign(1, 0);
  idx.clear();
  w.clear();
  for (int64_t r = 0; r < rows; ++r) {
    for (int64_t c = 0; c < cols; ++c) {
      const double v = M[r * cols + c];
      if (std::fabs(v) > 1e-15) {
        idx.push_back((int32_t)c);
        w.push_back(v);
      }
    }
    ptr.push_back((int32_t)idx.size());
  }
}

}  // namespace

bool build_separable(SepTransfer& t, const OpLevel& fine, const OpLevel& coarse, Budget* bud) {
  if (!fine.forest.uniform() || !coarse.forest.uniform() || !fine.L.structured || !coarse.L.structured) return false;
  const int nf = fine.forest.n, nc = coarse.forest.n, kf = fine.k, kc = coarse.k;
  const bool h = kf == kc && nc == (nf + 1) / 2 && nc < nf;  // nested (even nf) or non-nested (odd nf)
  const bool p = nf == nc && kf > kc;
  if (!h && !p) return false;
  t.dim = fine.dim;
  t.ncomp = fine.NU;
  t.nvel = fine.op == OP_PMASS ? 0 : fine.dim;
  t.Mf = (int64_t)kf * nf + 1;
  t.Mc = (int64_t)kc * nc + 1;
  // dense 1D interpolation P1 (Mf x Mc): coarse basis at every fine node
  std::vector<double> xf = gll_nodes(kf), xc = gll_nodes(kc);
  std::vector<double> P1(t.Mf * t.Mc, 0.0);
  for (int64_t g = 0; g < t.Mf; ++g) {
    int64_t cf = g / kf, s = g % kf;
    if (cf == nf) { cf = nf - 1; s = kf; }
    int64_t cc = cf;
    double xi = xf[s];
    if (h && nf == 2 * nc) {  // nested: child half of the parent cell
      cc = cf / 2;
      xi = 0.5 * ((cf % 2) + xf[s]);
    } else if (h) {           // non-nested: locate the fine node in the coarse mesh
      const double X = (double(cf) + xf[s]) * double(nc) / double(nf);
      cc = std::min<int64_t>((int64_t)std::floor(X), nc - 1);
      xi = X - double(cc);
    }
    for (int m = 0; m <= kc; ++m) P1[g * t.Mc + (int64_t)kc * cc + m] = lagrange(xc, m, xi);
  }
  std::vector<double> P1T(t.Mc * t.Mf);
  for (int64_t g = 0; g < t.Mf; ++g)
    for (int64_t c = 0; c < t.Mc; ++c) P1T[c * t.Mf + g] = P1[g * t.Mc + c];
  std::vector<int32_t> ptr, idx;
  std::vector<double> w;
  to_csr(P1, t.Mf, t.Mc, ptr, idx, w);
  t.p_ptr = upload(bud, ptr);
  t.p_idx = upload(bud, idx);
  t.p_w[0] = upload(bud, w);
  t.p_w[1] = upload(bud, std::vector<float>(w.begin(), w.end()));
  to_csr(P1T, t.Mc, t.Mf, ptr, idx, w);
  t.r_ptr = upload(bud, ptr);
  t.r_idx = upload(bud, idx);
  t.r_w[0] = upload(bud, w);
  t.r_w[1] = upload(bud, std::vector<float>(w.begin(), w.end()));
  // dense 1D interpolation I1 (Mc x Mf): fine basis at every coarse node (used to carry a fine
  // FE function, e.g. a Newton state, down the hierarchy)
  std::vector<double> I1(t.Mc * t.Mf, 0.0);
  for (int64_t g = 0; g < t.Mc; ++g) {
    int64_t cc = g / kc, s = g % kc;
    if (cc == nc) { cc = nc - 1; s = kc; }
    const double X = (double(cc) + xc[s]) * double(nf) / double(nc);  // position in fine cells
    const int64_t cf = std::min<int64_t>((int64_t)std::floor(X), nf - 1);
    const double xi = X - double(cf);
    for (int m = 0; m <= kf; ++m) I1[g * t.Mf + (int64_t)kf * cf + m] = lagrange(xf, m, xi);
  }
  to_csr(I1, t.Mc, t.Mf, ptr, idx, w);
  t.i_ptr = upload(bud, ptr);
  t.i_idx = upload(bud, idx);
  t.i_w = upload(bud, w);
  // intermediate grids: after the first pass and after the second (3D)
  const int64_t a = t.dim == 3 ? t.Mc * t.Mf * t.Mf : t.Mc * t.Mf;
  const int64_t b = t.dim == 3 ? t.Mc * t.Mc * t.Mf : 0;
  for (int prec = 0; prec < 2; ++prec) {
    t.tmp1[prec].alloc(bud, std::max<int64_t>(a, 1) * t.ncomp * esize(prec));
    t.tmp2[prec].alloc(bud, std::max<int64_t>(b, 1) * t.ncomp * esize(prec));
  }
  return true;
}

template <typename T, int NC>
static void sep_restrict_t(const SepTransfer& t, int prec, const T* fine, T* coarse, cudaStream_t s) {
  const int64_t Mf = t.Mf, Mc = t.Mc;
  T* t1 = t.tmp1[prec].as<T>();
  T* t2 = t.tmp2[prec].as<T>();
  if (t.dim == 3) {
    const int64_t e0[3] = {Mf, Mf, Mf}, e1[3] = {Mc, Mf, Mf}, e2[3] = {Mc, Mc, Mf};
    pass<T, NC>(fine, t1, 0, e0, Mc, t.r_ptr, t.r_idx, t.r_w[prec], t.nvel, true, false, false, s);
    pass<T, NC>(t1, t2, 1, e1, Mc, t.r_ptr, t.r_idx, t.r_w[prec], t.nvel, false, false, false, s);
    pass<T, NC>(t2, coarse, 2, e2, Mc, t.r_ptr, t.r_idx, t.r_w[prec], t.nvel, false, false, false, s);
  } else {
    const int64_t e0[3] = {Mf, Mf, 1}, e1[3] = {Mc, Mf, 1};
    pass<T, NC>(fine, t1, 0, e0, Mc, t.r_ptr, t.r_idx, t.r_w[prec], t.nvel, true, false, false, s);
    pass<T, NC>(t1, coarse, 1, e1, Mc, t.r_ptr, t.r_idx, t.r_w[prec], t.nvel, false, false, false, s);
  }
}

template <typename T, int NC>
static void sep_prolongate_t(const SepTransfer& t, int prec, const T* coarse, T* fine, cudaStream_t s) {
  const int64_t Mf = t.Mf, Mc = t.Mc;
  T* t1 = t.tmp1[prec].as<T>();
  T* t2 = t.tmp2[prec].as<T>();
  if (t.dim == 3) {
    const int64_t e0[3] = {Mc, Mc, Mc}, e1[3] = {Mc, Mc, Mf}, e2[3] = {Mc, Mf, Mf};
    pass<T, NC>(coarse, t2, 2, e0, Mf, t.p_ptr, t.p_idx, t.p_w[prec], t.nvel, true, false, false, s);
    pass<T, NC>(t2, t1, 1, e1, Mf, t.p_ptr, t.p_idx, t.p_w[prec], t.nvel, false, false, false, s);
    pass<T, NC>(t1, fine, 0, e2, Mf, t.p_ptr, t.p_idx, t.p_w[prec], t.nvel, false, true, true, s);
  } else {
    const int64_t e0[3] = {Mc, Mc, 1}, e1[3] = {Mc, Mf, 1};
    pass<T, NC>(coarse, t1, 1, e0, Mf, t.p_ptr, t.p_idx, t.p_w[prec], t.nvel, true, false, false, s);
    pass<T, NC>(t1, fine, 0, e1, Mf, t.p_ptr, t.p_idx, t.p_w[prec], t.nvel, false, true, true, s);
  }
}

template <typename T>
static void sep_dispatch(const SepTransfer& t, int prec, const T* in, T* out, bool restrict_, cudaStream_t s) {
  switch (t.ncomp) {
#define C(NC)                                                   \
  case NC:                                                      \
    if (restrict_) sep_restrict_t<T, NC>(t, prec, in, out, s);  \
    else sep_prolongate_t<T, NC>(t, prec, in, out, s);          \
    return;
    C(1) C(2) C(3) C(4)
#undef C
  }
  throw Error(kErrUnsupported, "separable transfer: unsupported component count");
}

template <int NC>
static void sep_interpolate_t(const SepTransfer& t, const double* fine, double* coarse, cudaStream_t s) {
  const int64_t Mf = t.Mf, Mc = t.Mc;
  double* t1 = t.tmp1[0].as<double>();
  double* t2 = t.tmp2[0].as<double>();
  if (t.dim == 3) {
    const int64_t e0[3] = {Mf, Mf, Mf}, e1[3] = {Mc, Mf, Mf}, e2[3] = {Mc, Mc, Mf};
    pass<double, NC>(fine, t1, 0, e0, Mc, t.i_ptr, t.i_idx, t.i_w, 0, false, false, false, s);
    pass<double, NC>(t1, t2, 1, e1, Mc, t.i_ptr, t.i_idx, t.i_w, 0, false, false, false, s);
    pass<double, NC>(t2, coarse, 2, e2, Mc, t.i_ptr, t.i_idx, t.i_w, 0, false, false, false, s);
  } else {
    const int64_t e0[3] = {Mf, Mf, 1}, e1[3] = {Mc, Mf, 1};
    pass<double, NC>(fine, t1, 0, e0, Mc, t.i_ptr, t.i_idx, t.i_w, 0, false, false, false, s);
    pass<double, NC>(t1, coarse, 1, e1, Mc, t.i_ptr, t.i_idx, t.i_w, 0, false, false, false, s);
  }
}

void sep_interpolate(const SepTransfer& t, const double* fine, double* coarse, cudaStream_t s) {
  switch (t.ncomp) {
    case 1: return sep_interpolate_t<1>(t, fine, coarse, s);
    case 2: return sep_interpolate_t<2>(t, fine, coarse, s);
    case 3: return sep_interpolate_t<3>(t, fine, coarse, s);
    case 4: return sep_interpolate_t<4>(t, fine, coarse, s);
  }
  throw Error(kErrUnsupported, "separable interpolation: unsupported component count");
}

void sep_restrict(const SepTransfer& t, int prec, const void* fine, void* coarse, cudaStream_t s) {
  if (prec == 0) sep_dispatch<double>(t, 0, (const double*)fine, (double*)coarse, true, s);
  else sep_dispatch<float>(t, 1, (const float*)fine, (float*)coarse, true, s);
}

void sep_prolongate_add(const SepTransfer& t, int prec, const void* coarse, void* fine, cudaStream_t s) {
  if (prec == 0) sep_dispatch<double>(t, 0, (const double*)coarse, (double*)fine, false, s);
  else sep_dispatch<float>(t, 1, (const float*)coarse, (float*)fine, false, s);
}

}  // namespace mfns
