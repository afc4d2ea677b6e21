// Section 3's blended smoother on hp levels: additive Schwarz blocks on the combined h+p faces and
// point Jacobi on the entries in no block, P^{-1} r = sum_B R_B^T A_BB^{-1} R_B r + J r (J = 1 / A_ii
// outside every block, 0 inside).  The blocks' matrices are probed with the level's operator; their
// inverses are formed on the host.
#include <algorithm>
#include <vector>

#include "hp_space.hpp"
#include "problem.hpp"
#include "spacetime.hpp"
#include "vec.hpp"

namespace mfns {

namespace {

// one block per thread block: gather r on the block, times the block's inverse (stored column by
// column: the threads of a warp, one row each, read consecutive words), into zloc
template <typename T>
__global__ void k_block_solve(const T* __restrict__ r, T* __restrict__ zloc, const int64_t* __restrict__ b_ptr,
                              const int32_t* __restrict__ b_idx, const int64_t* __restrict__ k_ptr,
                              const T* __restrict__ kinv) {
  extern __shared__ unsigned char smem[];
  T* rl = reinterpret_cast<T*>(smem);
  const int64_t p = blockIdx.x;
  const int64_t b0 = b_ptr[p];
  const int m = (int)(b_ptr[p + 1] - b0);
  for (int t = threadIdx.x; t < m; t += blockDim.x) rl[t] = r[b_idx[b0 + t]];
  __syncthreads();
  const T* Kp = kinv + k_ptr[p];
  for (int row = threadIdx.x; row < m; row += blockDim.x) {
    T v = 0;
    for (int j = 0; j < m; ++j) v += Kp[(int64_t)j * m + row] * rl[j];
    zloc[b0 + row] = v;
  }
}

// z[i] = J_i r_i + the block results holding i, in a fixed order
template <typename T>
__global__ void k_block_gather(T* __restrict__ z, const T* __restrict__ r, const T* __restrict__ zloc,
                               const int64_t* __restrict__ e_ptr, const int64_t* __restrict__ e_base,
                               const T* __restrict__ jdinv, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T v = jdinv[i] * r[i];
    for (int64_t o = e_ptr[i]; o < e_ptr[i + 1]; ++o) v += zloc[e_base[o]];
    z[i] = v;
  }
}

template <typename T>
void apply_t(const OpLevel& lv, int prec, const T* r, T* z, cudaStream_t s) {
  const HpData::Asm& A = *lv.hp->asm_;
  const size_t smem = (size_t)A.max_block * sizeof(T);
  k_block_solve<T><<<(unsigned)A.n_block, 128, smem, s>>>(r, A.zloc[prec].as<T>(), A.b_ptr.as<int64_t>(),
                                                           A.b_idx.as<int32_t>(), A.k_ptr.as<int64_t>(),
                                                           A.kinv[prec].as<T>());
  const int64_t n = lv.n_dofs;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
  k_block_gather<T><<<grid, 256, 0, s>>>(z, r, A.zloc[prec].as<T>(), A.e_ptr.as<int64_t>(), A.e_base.as<int64_t>(),
                                         A.jdinv[prec].as<T>(), n);
  MFNS_CUDA(cudaGetLastError());
}

}  // namespace

void build_hp_asm(OpLevel& lv, Budget* bud, cudaStream_t s) {
  if (!lv.hp || lv.op != OP_STOKES_A) return;
  const HpSpace& sp = lv.hp->space;
  const int ncomp = lv.NU;
  const std::vector<std::vector<int32_t>> blocks = hp_asm_blocks(lv.forest, sp, ncomp);
  if (blocks.empty()) return;
  const int64_t n = lv.n_dofs;
  const size_t nc = sp.cell_ptr.size() - 1;
  // cells reaching a node: those holding it, and those holding a constrained node of which it is a
  // master (an operator entry couples two entries only through a cell reaching both)
  std::vector<std::vector<int32_t>> held(sp.n_nodes), hang_of(sp.n_nodes);
  for (size_t c = 0; c < nc; ++c)
    for (int64_t j = sp.cell_ptr[c]; j < sp.cell_ptr[c + 1]; ++j) held[sp.cell_nodes[j]].push_back((int32_t)c);
  for (size_t i = 0; i < sp.hang_node.size(); ++i)
    for (int32_t j = sp.hang_ptr[i]; j < sp.hang_ptr[i + 1]; ++j) hang_of[sp.hang_master[j]].push_back(sp.hang_node[i]);
  std::vector<std::vector<int32_t>> reach(blocks.size());
  for (size_t b = 0; b < blocks.size(); ++b) {
    std::vector<int32_t>& R = reach[b];
    for (int32_t e : blocks[b]) {
      const int32_t g = e / ncomp;
      R.insert(R.end(), held[g].begin(), held[g].end());
      for (int32_t h : hang_of[g]) R.insert(R.end(), held[h].begin(), held[h].end());
    }
    std::sort(R.begin(), R.end());
    R.erase(std::unique(R.begin(), R.end()), R.end());
  }
  std::vector<std::vector<int32_t>> cell_colours(nc);
  std::vector<int32_t> colour(blocks.size());
  int ncol = 0;
  for (size_t b = 0; b < blocks.size(); ++b) {
    std::vector<char> used(ncol + 1, 0);
    for (int32_t c : reach[b])
      for (int32_t col : cell_colours[c]) used[col] = 1;
    int col = 0;
    while (used[col]) ++col;
    colour[b] = col;
    ncol = std::max(ncol, col + 1);
    for (int32_t c : reach[b]) cell_colours[c].push_back(col);
  }
  // probe: for every colour and local index, the unit entries of that index in the colour's blocks
  std::vector<std::vector<double>> Abb(blocks.size());
  for (size_t b = 0; b < blocks.size(); ++b) Abb[b].assign(blocks[b].size() * blocks[b].size(), 0.0);
  DevBuf X, Y;
  X.alloc(bud, (size_t)n * 8);
  Y.alloc(bud, (size_t)n * 8);
  std::vector<double> Xh(n), Yh(n);
  for (int col = 0; col < ncol; ++col) {
    size_t len = 0;
    for (size_t b = 0; b < blocks.size(); ++b)
      if (colour[b] == col) len = std::max(len, blocks[b].size());
    for (size_t m = 0; m < len; ++m) {
      std::fill(Xh.begin(), Xh.end(), 0.0);
      for (size_t b = 0; b < blocks.size(); ++b)
        if (colour[b] == col && m < blocks[b].size()) Xh[blocks[b][m]] = 1.0;
      MFNS_CUDA(cudaMemcpyAsync(X.get(), Xh.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s));
      hp_vmult(lv, 0, X.get(), Y.get(), s);
      MFNS_CUDA(cudaMemcpyAsync(Yh.data(), Y.get(), (size_t)n * 8, cudaMemcpyDeviceToHost, s));
      MFNS_CUDA(cudaStreamSynchronize(s));
      for (size_t b = 0; b < blocks.size(); ++b) {
        if (colour[b] != col || m >= blocks[b].size()) continue;
        const size_t mb = blocks[b].size();
        for (size_t a = 0; a < mb; ++a) Abb[b][a * mb + m] = Yh[blocks[b][a]];
      }
    }
  }
  auto A = std::make_unique<HpData::Asm>();
  std::vector<int64_t> b_ptr(1, 0), k_ptr(1, 0);
  std::vector<int32_t> b_idx;
  std::vector<double> kinv;
  for (size_t b = 0; b < blocks.size(); ++b) {
    std::vector<double> K = Abb[b];
    if (!invert_dense_rel(K, (int64_t)blocks[b].size(), 1e-14)) throw Error(kErrArg, "singular Schwarz block");
    b_idx.insert(b_idx.end(), blocks[b].begin(), blocks[b].end());
    b_ptr.push_back((int64_t)b_idx.size());
    const int64_t mb = (int64_t)blocks[b].size();
    for (int64_t j = 0; j < mb; ++j)  // column by column
      for (int64_t i = 0; i < mb; ++i) kinv.push_back(K[(size_t)i * mb + j]);
    k_ptr.push_back((int64_t)kinv.size());
    A->max_block = std::max<int64_t>(A->max_block, (int64_t)blocks[b].size());
  }
  if (A->max_block * 8 > 48 * 1024) throw Error(kErrUnsupported, "Schwarz block too large");
  std::vector<int64_t> e_ptr(n + 1, 0);
  for (int32_t i : b_idx) e_ptr[i + 1]++;
  for (int64_t i = 0; i < n; ++i) e_ptr[i + 1] += e_ptr[i];
  std::vector<int64_t> e_base(e_ptr[n]);
  {
    std::vector<int64_t> fill(e_ptr.begin(), e_ptr.end() - 1);
    for (int64_t j = 0; j < (int64_t)b_idx.size(); ++j) e_base[fill[b_idx[j]]++] = j;
  }
  std::vector<double> jd(n);
  MFNS_CUDA(cudaMemcpyAsync(jd.data(), lv.dinv[0].get(), (size_t)n * 8, cudaMemcpyDeviceToHost, s));
  MFNS_CUDA(cudaStreamSynchronize(s));
  for (int32_t i : b_idx) jd[i] = 0.0;
  A->n_block = (int64_t)blocks.size();
  A->b_ptr = upload(bud, b_ptr);
  A->b_idx = upload(bud, b_idx);
  A->k_ptr = upload(bud, k_ptr);
  A->kinv[0] = upload(bud, kinv);
  A->kinv[1] = upload(bud, std::vector<float>(kinv.begin(), kinv.end()));
  A->e_ptr = upload(bud, e_ptr);
  A->e_base = upload(bud, e_base);
  A->jdinv[0] = upload(bud, jd);
  A->jdinv[1] = upload(bud, std::vector<float>(jd.begin(), jd.end()));
  A->zloc[0].alloc(bud, (size_t)b_idx.size() * 8);
  A->zloc[1].alloc(bud, (size_t)b_idx.size() * 4);
  lv.hp->asm_ = std::move(A);
}

void hp_asm_apply(const OpLevel& lv, int prec, const void* r, void* z, cudaStream_t s) {
  if (!lv.hp || !lv.hp->asm_) throw Error(kErrArg, "no Schwarz blocks on this level");
  if (prec == 0)
    apply_t<double>(lv, 0, (const double*)r, (double*)z, s);
  else
    apply_t<float>(lv, 1, (const float*)r, (float*)z, s);
}

}  // namespace mfns
