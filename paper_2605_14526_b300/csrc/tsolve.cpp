// Host construction of the level-scheduled partitioned-inverse solves. See
// tsolve.h.
#include "tsolve.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace pdf {

namespace {

// rows x cols column-major dense block of the node's columns of L
struct Dense {
  int rows = 0, cols = 0;
  std::vector<double> a;
  double& at(int i, int j) { return a[(size_t)j * rows + i]; }
  double at(int i, int j) const { return a[(size_t)j * rows + i]; }
};

// Linv = L_ss^-1 and M = L_below Linv from the dense block column
// D = [L_ss; L_below] (column-major), written as packed row-major and
// column-major copies of [Linv; M].
void node_inverse(const Dense& D, int nc, int nb, double* prow, double* pcol, bool parallel) {
  const int rows = nc + nb;
  // Linv column by column: forward substitution L_ss x = e_j (column-oriented)
  std::vector<double> Li((size_t)nc * nc, 0.0);   // column-major, lower
#pragma omp parallel for schedule(dynamic, 4) if (parallel)
  for (int j = 0; j < nc; ++j) {
    double* x = &Li[(size_t)j * nc];
    x[j] = 1.0;
    for (int k = j; k < nc; ++k) {
      const double xk = x[k] / D.at(k, k);
      x[k] = xk;
      if (xk == 0.0) continue;
      for (int i = k + 1; i < nc; ++i) x[i] -= D.at(i, k) * xk;
    }
  }
  // M[:, k] = sum_{i >= k} L_below[:, i] Linv[i, k]
  std::vector<double> M((size_t)nb * nc, 0.0);    // column-major
#pragma omp parallel for schedule(dynamic, 4) if (parallel)
  for (int k = 0; k < nc; ++k) {
    double* m = &M[(size_t)k * nb];
    for (int i = k; i < nc; ++i) {
      const double l = Li[(size_t)k * nc + i];
      if (l == 0.0) continue;
      const double* col = &D.a[(size_t)i * rows + nc];
      for (int r = 0; r < nb; ++r) m[r] += col[r] * l;
    }
  }
  // packed copies
  int64_t o = 0;
  for (int r = 0; r < nc; ++r)
    for (int k = 0; k <= r; ++k) prow[o++] = Li[(size_t)k * nc + r];
  for (int r = 0; r < nb; ++r)
    for (int k = 0; k < nc; ++k) prow[o++] = M[(size_t)k * nb + r];
  o = 0;
  for (int k = 0; k < nc; ++k) {
    for (int r = k; r < nc; ++r) pcol[o++] = Li[(size_t)k * nc + r];
    for (int r = 0; r < nb; ++r) pcol[o++] = M[(size_t)k * nb + r];
  }
}

}  // namespace

void build_tsolve(const Factor& f, TSolve& t) {
  const auto t0 = std::chrono::steady_clock::now();
  t = TSolve();
  const int n = f.n;
  t.n = n;
  const int ns = (int)f.sup_start.size() - 1;
  // supernode tree
  std::vector<int> sp(ns, -1), nch(ns, 0);
  for (int s = 0; s < ns; ++s) {
    const int p = f.parent[f.sup_start[s + 1] - 1];
    if (p >= 0) {
      sp[s] = f.col2sup[p];
      nch[sp[s]]++;
    }
  }
  // nodes: chains of supernodes (post-ordered, so a chain is contiguous)
  std::vector<int> nstart, node_of(ns);
  for (int s = 0; s < ns; ++s) {
    const bool merge = s > 0 && sp[s - 1] == s && nch[s] == 1 &&
                       f.sup_start[s + 1] - f.sup_start[nstart.back()] <= kNodeMaxCols;
    if (!merge) nstart.push_back(s);
    node_of[s] = (int)nstart.size() - 1;
  }
  const int nn = (int)nstart.size();
  nstart.push_back(ns);
  t.n_node = nn;
  t.c0.resize(nn);
  t.nc.resize(nn);
  t.nb.resize(nn);
  t.height.assign(nn, 0);
  std::vector<int> npar(nn, -1);
  t.boff.assign(nn + 1, 0);
  std::vector<std::vector<int>> blw(nn);
  for (int u = 0; u < nn; ++u) {
    const int s0 = nstart[u], s1 = nstart[u + 1];
    const int c0 = f.sup_start[s0], c1 = f.sup_start[s1];
    t.c0[u] = c0;
    t.nc[u] = c1 - c0;
    std::vector<int>& b = blw[u];
    for (int s = s0; s < s1; ++s)
      for (int64_t p = f.rowptr[s]; p < f.rowptr[s + 1]; ++p)
        if (f.rows[p] >= c1) b.push_back(f.rows[p]);
    std::sort(b.begin(), b.end());
    b.erase(std::unique(b.begin(), b.end()), b.end());
    t.nb[u] = (int)b.size();
    const int p = sp[s1 - 1];
    npar[u] = p < 0 ? -1 : node_of[p];
  }
  for (int u = 0; u < nn; ++u) {   // children precede parents (post-order)
    if (npar[u] >= 0) t.height[npar[u]] = std::max(t.height[npar[u]], t.height[u] + 1);
    t.boff[u + 1] = t.boff[u] + t.nb[u];
  }
  t.u_rows = t.boff[nn];
  t.below.resize(t.u_rows);
  for (int u = 0; u < nn; ++u) std::copy(blw[u].begin(), blw[u].end(), t.below.begin() + t.boff[u]);
  std::vector<std::vector<int>>().swap(blw);
  // partitioned inverses
  t.poff.assign(nn + 1, 0);
  for (int u = 0; u < nn; ++u)
    t.poff[u + 1] = t.poff[u] + (int64_t)t.nc[u] * (t.nc[u] + 1) / 2 + (int64_t)t.nb[u] * t.nc[u];
  t.entries = t.poff[nn];
  t.prow.assign(t.entries, 0.0);
  t.pcol.assign(t.entries, 0.0);
  auto one_node = [&](int u, bool parallel, std::vector<int>& pos) {
    const int c0 = t.c0[u], nc = t.nc[u], nb = t.nb[u];
    Dense D;
    D.rows = nc + nb;
    D.cols = nc;
    D.a.assign((size_t)D.rows * nc, 0.0);
    for (int i = 0; i < nb; ++i) pos[t.below[t.boff[u] + i]] = nc + i;
    for (int s = nstart[u]; s < nstart[u + 1]; ++s) {
      const int64_t nr = f.rowptr[s + 1] - f.rowptr[s];
      const int* rw = &f.rows[f.rowptr[s]];
      for (int c = f.sup_start[s]; c < f.sup_start[s + 1]; ++c) {
        const double* col = &f.val[f.valptr[s] + (int64_t)(c - f.sup_start[s]) * nr];
        for (int64_t r = c - f.sup_start[s]; r < nr; ++r) {
          const int row = rw[r];
          const int o = row < c0 + nc ? row - c0 : pos[row];
          D.at(o, c - c0) = col[r];
        }
      }
    }
    node_inverse(D, nc, nb, &t.prow[t.poff[u]], &t.pcol[t.poff[u]], parallel);
  };
  // large nodes one at a time with their columns in parallel, then the small
  // ones in parallel over nodes
  constexpr int kBig = 192;
  {
    std::vector<int> pos(n, -1);
    for (int u = 0; u < nn; ++u)
      if (t.nc[u] >= kBig) one_node(u, true, pos);
  }
#pragma omp parallel
  {
    std::vector<int> pos(n, -1);
#pragma omp for schedule(dynamic, 8)
    for (int u = 0; u < nn; ++u)
      if (t.nc[u] < kBig) one_node(u, false, pos);
  }
  // gather lists: position o of node s receives U rows of its children
  t.goff.assign(nn + 1, 0);
  for (int u = 0; u < nn; ++u) t.goff[u + 1] = t.goff[u] + t.nc[u] + t.nb[u];
  std::vector<std::vector<int>> kids(nn);
  for (int u = 0; u < nn; ++u)
    if (npar[u] >= 0) kids[npar[u]].push_back(u);
  std::vector<int> cnt(t.goff[nn] + 1, 0);
  std::vector<int64_t> src_pos;   // (global position index, U row) pairs, as two arrays
  std::vector<int> src_row;
  {
    std::vector<int> pos(n, -1);
    for (int u = 0; u < nn; ++u) {
      const int c0 = t.c0[u], nc = t.nc[u];
      for (int i = 0; i < t.nb[u]; ++i) pos[t.below[t.boff[u] + i]] = nc + i;
      for (int c : kids[u])
        for (int j = 0; j < t.nb[c]; ++j) {
          const int row = t.below[t.boff[c] + j];
          const int o = row < c0 + nc ? row - c0 : pos[row];
          src_pos.push_back(t.goff[u] + o);
          src_row.push_back((int)(t.boff[c] + j));
          cnt[t.goff[u] + o + 1]++;
        }
    }
  }
  t.gptr.assign(t.goff[nn] + 1, 0);
  for (int64_t i = 0; i < t.goff[nn]; ++i) t.gptr[i + 1] = t.gptr[i] + cnt[i + 1];
  t.gsrc.assign(src_row.size(), 0);
  {
    std::vector<int> fill(t.gptr.begin(), t.gptr.end() - 1);
    for (size_t i = 0; i < src_row.size(); ++i) t.gsrc[fill[src_pos[i]]++] = src_row[i];   // children in order
  }
  // schedule per height
  int H = 0;
  for (int u = 0; u < nn; ++u) H = std::max(H, t.height[u]);
  t.n_level = nn ? H + 1 : 0;
  t.lev_f.assign(t.n_level + 1, 0);
  t.lev_b.assign(t.n_level + 1, 0);
  t.lev_wf.assign(t.n_level + 1, 0);
  t.lev_wb.assign(t.n_level + 1, 0);
  for (int h = 0; h < t.n_level; ++h) {
    for (int u = 0; u < nn; ++u) {
      if (t.height[u] != h) continue;
      const int nc = t.nc[u], rows = nc + t.nb[u];
      // forward: a node of at most 32 columns is one warp item per 32 rows
      // (each item forms r_s from the gathers itself); up to kLaneNodeCols
      // columns a lane per row in units of 8 x 32 rows; larger nodes a warp
      // per row in units of 32 rows
      if (nc <= kWarpNodeCols) {
        for (int r0 = 0; r0 < rows; r0 += 32) t.wnode_f.insert(t.wnode_f.end(), {u, r0});
      } else if (nc <= kLaneNodeCols) {
        for (int r0 = 0; r0 < rows; r0 += 256) t.unit_f.insert(t.unit_f.end(), {u, r0, std::min(256, rows - r0), 1});
      } else {
        for (int r0 = 0; r0 < rows; r0 += kUnitRows)
          t.unit_f.insert(t.unit_f.end(), {u, r0, std::min(kUnitRows, rows - r0), 0});
      }
      // backward: a small node with a short right-hand side is one warp's
      // (a lane per column); otherwise a warp per column in units of enough
      // columns that staging the right-hand side once pays off, while it
      // fits the staging vector, else 8 columns with chunked staging
      if (nc <= kWarpNodeCols && rows <= kWarpNodeRows) {
        t.wnode_b.push_back(u);
      } else {
        const int uc = rows <= kStageRows ? std::max(kUnitCols, kUnitEntries / rows) : kUnitCols;
        for (int k0 = 0; k0 < nc; k0 += uc) t.unit_b.insert(t.unit_b.end(), {u, k0, std::min(uc, nc - k0), 0});
      }
    }
    t.lev_f[h + 1] = (int)t.unit_f.size() / 4;
    t.lev_b[h + 1] = (int)t.unit_b.size() / 4;
    t.lev_wf[h + 1] = (int)t.wnode_f.size() / 2;
    t.lev_wb[h + 1] = (int)t.wnode_b.size();
  }
  t.build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

void tsolve_host(const TSolve& t, const double* b, double* x) {
  const int n = t.n;
  std::vector<double> y((size_t)3 * n, 0.0), U((size_t)3 * t.u_rows, 0.0);
  auto node_fwd = [&](int u) {
    const int c0 = t.c0[u], nc = t.nc[u], nb = t.nb[u];
    std::vector<double> r((size_t)3 * nc), g((size_t)3 * (nc + nb), 0.0);
    for (int o = 0; o < nc + nb; ++o)
      for (int p = t.gptr[t.goff[u] + o]; p < t.gptr[t.goff[u] + o + 1]; ++p)
        for (int a = 0; a < 3; ++a) g[3 * o + a] += U[3 * (size_t)t.gsrc[p] + a];
    for (int k = 0; k < nc; ++k)
      for (int a = 0; a < 3; ++a) r[3 * k + a] = b[3 * (size_t)(c0 + k) + a] - g[3 * k + a];
    const double* P = &t.prow[t.poff[u]];
    int64_t off = 0;
    for (int o = 0; o < nc + nb; ++o) {
      const int len = o < nc ? o + 1 : nc;
      double acc[3] = {0.0, 0.0, 0.0};
      for (int k = 0; k < len; ++k)
        for (int a = 0; a < 3; ++a) acc[a] += P[off + k] * r[3 * k + a];
      off += len;
      for (int a = 0; a < 3; ++a) {
        if (o < nc) y[3 * (size_t)(c0 + o) + a] = acc[a];
        else U[3 * (size_t)(t.boff[u] + o - nc) + a] = acc[a] + g[3 * o + a];
      }
    }
  };
  auto node_bwd = [&](int u) {
    const int c0 = t.c0[u], nc = t.nc[u], nb = t.nb[u];
    std::vector<double> z((size_t)3 * (nc + nb));
    for (int r = 0; r < nc; ++r)
      for (int a = 0; a < 3; ++a) z[3 * r + a] = y[3 * (size_t)(c0 + r) + a];
    for (int r = 0; r < nb; ++r)
      for (int a = 0; a < 3; ++a) z[3 * (nc + r) + a] = -x[3 * (size_t)t.below[t.boff[u] + r] + a];
    const double* P = &t.pcol[t.poff[u]];
    int64_t off = 0;
    for (int k = 0; k < nc; ++k) {
      const int len = nc - k + nb;
      double acc[3] = {0.0, 0.0, 0.0};
      for (int i = 0; i < len; ++i)
        for (int a = 0; a < 3; ++a) acc[a] += P[off + i] * z[3 * (k + i) + a];
      off += len;
      for (int a = 0; a < 3; ++a) x[3 * (size_t)(c0 + k) + a] = acc[a];
    }
  };
  std::vector<std::vector<int>> by_h(t.n_level);
  for (int u = 0; u < t.n_node; ++u) by_h[t.height[u]].push_back(u);
  for (int h = 0; h < t.n_level; ++h)
    for (int u : by_h[h]) node_fwd(u);
  for (int h = t.n_level - 1; h >= 0; --h)
    for (int u : by_h[h]) node_bwd(u);
}

}  // namespace pdf
