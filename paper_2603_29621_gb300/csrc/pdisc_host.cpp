// Host tables of the Q_k / P^disc_{k-1} pair on uniform meshes (see pdisc.hpp).
#include <algorithm>
#include <cmath>

#include "mesh.hpp"
#include "pdisc.hpp"

namespace mfns {

std::vector<std::array<int, 3>> pdisc_exponents(int dim, int kp) {
  std::vector<std::array<int, 3>> out;
  for (int tot = 0; tot <= kp; ++tot) {
    if (dim == 2) {
      for (int a = tot; a >= 0; --a) out.push_back({a, tot - a, 0});
    } else {
      for (int a = tot; a >= 0; --a)
        for (int b = tot - a; b >= 0; --b) out.push_back({a, b, tot - a - b});
    }
  }
  return out;
}

std::vector<double> pdisc_cell_B(int dim, int k, double h) {
  const std::vector<std::array<int, 3>> ex = pdisc_exponents(dim, k - 1);
  const int npc = (int)ex.size(), np1 = k + 1;
  int nb = 1;
  for (int d = 0; d < dim; ++d) nb *= np1;
  const std::vector<double> t = gll_nodes(k);
  std::vector<double> xg, wg;
  gauss_rule(k + 2, xg, wg);  // exact: degree <= (k - 1) + k per direction
  // 1D integrals on [0, 1]: V[e][i] = int (x - 1/2)^e L_i(x), D[e][i] = int (x - 1/2)^e L_i'(x)
  std::vector<double> V(k * np1, 0.0), D(k * np1, 0.0);
  for (int e = 0; e < k; ++e)
    for (int i = 0; i < np1; ++i)
      for (size_t g = 0; g < xg.size(); ++g) {
        const double m = std::pow(xg[g] - 0.5, e);
        V[e * np1 + i] += wg[g] * m * lagrange(t, i, xg[g]);
        D[e * np1 + i] += wg[g] * m * lagrange_deriv(t, i, xg[g]);
      }
  // dx = h^dim dxi, d/dx_d = (1/h) d/dxi_d
  const double scale = -std::pow(h, dim - 1);
  std::vector<double> B((size_t)npc * nb * dim, 0.0);
  for (int a = 0; a < npc; ++a)
    for (int b = 0; b < nb; ++b) {
      const int bi[3] = {b % np1, (b / np1) % np1, dim == 3 ? b / (np1 * np1) : 0};
      for (int d = 0; d < dim; ++d) {
        double v = scale;
        for (int e = 0; e < dim; ++e) v *= (e == d ? D : V)[ex[a][e] * np1 + bi[e]];
        B[((size_t)a * nb + b) * dim + d] = v;
      }
    }
  return B;
}

std::vector<double> pdisc_child_embedding(int dim, int kp, int child) {
  const std::vector<std::array<int, 3>> ex = pdisc_exponents(dim, kp);
  const int npc = (int)ex.size();
  auto binom = [](int n, int j) {
    double v = 1.0;
    for (int i = 1; i <= j; ++i) v = v * (n - j + i) / i;
    return v;
  };
  std::vector<double> E((size_t)npc * npc, 0.0);
  for (int b = 0; b < npc; ++b)    // fine monomial
    for (int a = 0; a < npc; ++a) {  // coarse monomial
      double v = 1.0;
      for (int e = 0; e < dim && v != 0.0; ++e) {
        if (ex[b][e] > ex[a][e]) {
          v = 0.0;
          break;
        }
        const double delta = ((child >> e) & 1) ? 0.25 : -0.25;
        const int j = ex[b][e];
        v *= binom(ex[a][e], j) * std::pow(delta, ex[a][e] - j) * std::pow(0.5, j);
      }
      E[(size_t)b * npc + a] = v;
    }
  return E;
}

std::vector<double> pdisc_degree_embedding(int dim, int kpf, int kpc) {
  const int nf = (int)pdisc_exponents(dim, kpf).size(), nc = (int)pdisc_exponents(dim, kpc).size();
  std::vector<double> E((size_t)nf * nc, 0.0);
  for (int a = 0; a < std::min(nf, nc); ++a) E[(size_t)a * nc + a] = 1.0;
  return E;
}

std::vector<std::vector<int32_t>> pdisc_cell_patches(int dim, int n, int k) {
  const int64_t M = (int64_t)k * n + 1;
  const int64_t n_nodes = dim == 3 ? M * M * M : M * M;
  const int64_t n_main = n_nodes * dim;
  const int npc = (int)pdisc_exponents(dim, k - 1).size();
  const int nz = dim == 3 ? n : 1;
  std::vector<std::vector<int32_t>> out;
  for (int cz = 0; cz < nz; ++cz)
    for (int cy = 0; cy < n; ++cy)
      for (int cx = 0; cx < n; ++cx) {
        const int64_t cell = cx + (int64_t)n * (cy + (int64_t)n * cz);
        std::vector<int32_t> p;
        for (int bz = 0; bz <= (dim == 3 ? k : 0); ++bz)
          for (int by = 0; by <= k; ++by)
            for (int bx = 0; bx <= k; ++bx) {
              const int64_t ix = (int64_t)k * cx + bx, iy = (int64_t)k * cy + by, iz = (int64_t)k * cz + bz;
              const bool bnd = ix == 0 || ix == M - 1 || iy == 0 || iy == M - 1 ||
                               (dim == 3 && (iz == 0 || iz == M - 1));
              if (bnd) continue;
              const int64_t g = ix + M * (iy + M * iz);
              for (int c = 0; c < dim; ++c) p.push_back((int32_t)(g * dim + c));
            }
        for (int a = 0; a < npc; ++a) p.push_back((int32_t)(n_main + cell * npc + a));
        std::sort(p.begin(), p.end());
        out.push_back(std::move(p));
      }
  return out;
}

}  // namespace mfns
