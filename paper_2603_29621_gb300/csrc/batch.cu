// Multi-problem operator application: the descriptor table of one launch per colour over the
// cells of several problems (structured levels sharing dimension, degree, operator, precision and
// frozen-data mode).  Each problem's blocks follow the previous problem's; every block reads its
// problem's fields (vectors, mesh size, physics) from the table, so the arithmetic per cell is the
// one of a single-problem launch and results are bitwise those of separate applications.
#include "op_kernel.cuh"
#include "problem.hpp"
#include "vec.hpp"

namespace mfns {

struct MultiOp {
  int prec = 1;
  const OpLaunch* L0 = nullptr;
  std::vector<const OpLevel*> lv;
  std::vector<const void*> src;
  std::vector<void*> dst;
  std::vector<MultiColour> col;
  DevBuf probs, pid;
};

void multi_op_destroy(MultiOp* m) { delete m; }

static int64_t colour_cells(const OpLaunch& L, int c) {
  int64_t nc = 1;
  for (int d = 0; d < L.dim; ++d) nc *= (L.n - ((c >> d) & 1) + 1) / 2;
  return nc;
}

template <typename T>
static void fill(MultiOp& m, Budget* bud) {
  const OpLaunch& L0 = *m.L0;
  const int nmem = (int)m.lv.size();
  const int ncol = L0.n_colors;
  const int warps = L0.warps[m.prec] > 0 ? L0.warps[m.prec] : 4;
  const int tpc = L0.dim == 3 ? L0.Q * L0.Q : L0.Q;  // lanes per cell
  const int64_t cells_per_block = (int64_t)warps * (32 / tpc);
  std::vector<ProbArgs<T>> pa((size_t)ncol * nmem);
  std::vector<int32_t> pid;
  std::vector<int64_t> pid_off(ncol + 1, 0);
  std::vector<int64_t> offset(nmem, 0);  // colour offsets (cells of earlier colours) per member
  for (int c = 0; c < ncol; ++c) {
    int64_t first = 0;
    for (int i = 0; i < nmem; ++i) {
      const OpLaunch& L = m.lv[i]->L;
      ProbArgs<T>& a = pa[(size_t)c * nmem + i];
      a.src = static_cast<const T*>(m.src[i]);
      a.dst = static_cast<T*>(m.dst[i]);
      a.frozen = static_cast<const T*>(L.frozen[m.prec]);
      a.gexp = static_cast<const T*>(L.gexp[m.prec]);
      a.fq = static_cast<T*>(L.fq[m.prec]);
      a.color_offset = offset[i];
      a.p_offset = L.p_offset;
      a.first_block = first;
      a.n = L.n;
      a.h = (T)L.h;
      a.nu = (T)L.nu;
      const double dt_inv = L.dt > 0 ? 1.0 / L.dt : 0.0;
      a.dt_inv = (T)dt_inv;
      a.cm = (T)(L.alpha * dt_inv);
      a.div_sign = (T)L.div_sign;
      for (int b = 0; b < 7; ++b) a.cf[b] = (L.terms >> b) & 1 ? T(1) : T(0);
      const int64_t ncell = colour_cells(L, c);
      const int64_t nb = (ncell + cells_per_block - 1) / cells_per_block;
      for (int64_t k = 0; k < nb; ++k) pid.push_back(i);
      first += nb;
      offset[i] += ncell;
    }
    pid_off[c + 1] = (int64_t)pid.size();
  }
  if (pid.size() >= (size_t)1 << 31) throw Error(kErrUnsupported, "multi-problem launch: too many blocks");
  m.probs = upload(bud, pa);
  m.pid = upload(bud, pid);
  m.col.resize(ncol);
  for (int c = 0; c < ncol; ++c) {
    m.col[c].probs = m.probs.as<ProbArgs<T>>() + (size_t)c * nmem;
    m.col[c].block_pid = m.pid.as<int32_t>() + pid_off[c];
    m.col[c].nblocks = (unsigned)(pid_off[c + 1] - pid_off[c]);
  }
}

MultiOp* multi_op_create(const std::vector<const OpLevel*>& lv, const std::vector<const void*>& src,
                         const std::vector<void*>& dst, int prec, Budget* bud) {
  if (lv.empty() || lv.size() != src.size() || lv.size() != dst.size()) throw Error(kErrArg, "multi-op: members");
  const OpLaunch& L0 = lv[0]->L;
  for (const OpLevel* l : lv) {
    const OpLaunch& L = l->L;
    if (!L.structured || L.dim != L0.dim || L.k != L0.k || L.op != L0.op || L.n_colors != L0.n_colors ||
        (L.fq[prec] != nullptr) != (L0.fq[prec] != nullptr) || L.warps[prec] != L0.warps[prec])
      throw Error(kErrArg, "multi-op: members differ in kind, degree, layout or block size");
  }
  auto m = std::make_unique<MultiOp>();
  m->prec = prec;
  m->L0 = &L0;
  m->lv = lv;
  m->src = src;
  m->dst = dst;
  if (prec == 0)
    fill<double>(*m, bud);
  else
    fill<float>(*m, bud);
  return m.release();
}

// dst_i = A_i src_i for every member (constrained rows dst = src), one launch per colour.
void multi_vmult(const MultiOp& m, cudaStream_t s) {
  const size_t es = m.prec == 0 ? 8 : 4;
  for (size_t i = 0; i < m.lv.size(); ++i) MFNS_CUDA(cudaMemsetAsync(m.dst[i], 0, m.lv[i]->n_dofs * es, s));
  for (int c = 0; c < (int)m.col.size(); ++c) op_apply_multi(*m.L0, m.prec, c, m.col[c], s);
  for (size_t i = 0; i < m.lv.size(); ++i) {
    const OpLevel& lv = *m.lv[i];
    const int64_t nc = (int64_t)lv.constrained_host.size();
    if (m.prec == 0)
      vcopy_idx<double>((double*)m.dst[i], (const double*)m.src[i], lv.constrained.as<int32_t>(), nc, s);
    else
      vcopy_idx<float>((float*)m.dst[i], (const float*)m.src[i], lv.constrained.as<int32_t>(), nc, s);
  }
}

}  // namespace mfns
