// Host-side FP64 factorization of the scalar PD operator. See factor.h.
#include "factor.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace pdf {

// ---------------------------------------------------------------- ordering

namespace {

struct NDState {
  const std::vector<int64_t>* ptr;
  const std::vector<int>* idx;
  const double* xyz;
  int leaf;
  std::vector<int> stamp, side;
  int next_stamp = 1;
  std::vector<int> out;
};

void nd_rec(NDState& st, std::vector<int> verts) {
  const int m = (int)verts.size();
  if (m == 0) return;
  if (m <= st.leaf) {
    st.out.insert(st.out.end(), verts.begin(), verts.end());
    return;
  }
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int v : verts)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], st.xyz[3 * v + a]);
      hi[a] = std::max(hi[a], st.xyz[3 * v + a]);
    }
  int ax = 0;
  for (int a = 1; a < 3; ++a)
    if (hi[a] - lo[a] > hi[ax] - lo[ax]) ax = a;
  std::stable_sort(verts.begin(), verts.end(),
                   [&](int a, int b) { return st.xyz[3 * a + ax] < st.xyz[3 * b + ax]; });
  // split at a change of coordinate near the median so that a grid is cut
  // between two vertex planes (the left plane becomes the separator)
  int mid = m / 2;
  const double tol = 1e-9 * std::max(1.0, hi[ax] - lo[ax]);
  int cut = mid;
  while (cut > 0 && st.xyz[3 * verts[cut] + ax] - st.xyz[3 * verts[cut - 1] + ax] <= tol) --cut;
  if (cut == 0) {
    cut = mid;
    while (cut < m && st.xyz[3 * verts[cut] + ax] - st.xyz[3 * verts[cut - 1] + ax] <= tol) ++cut;
    if (cut >= m) cut = mid;  // all coordinates equal: plain index split
  }
  const int s = st.next_stamp++;
  for (int i = 0; i < m; ++i) {
    st.stamp[verts[i]] = s;
    st.side[verts[i]] = i < cut ? 0 : 1;
  }
  std::vector<int> left, right, sep;
  for (int i = 0; i < cut; ++i) {
    int v = verts[i];
    bool touches = false;
    for (int64_t p = (*st.ptr)[v]; p < (*st.ptr)[v + 1]; ++p) {
      int u = (*st.idx)[p];
      if (st.stamp[u] == s && st.side[u] == 1) {
        touches = true;
        break;
      }
    }
    (touches ? sep : left).push_back(v);
  }
  right.assign(verts.begin() + cut, verts.end());
  nd_rec(st, std::move(left));
  nd_rec(st, std::move(right));
  st.out.insert(st.out.end(), sep.begin(), sep.end());
}

}  // namespace

std::vector<int> nested_dissection(int n, const std::vector<int64_t>& ptr, const std::vector<int>& idx,
                                   const double* xyz, int leaf) {
  NDState st;
  st.ptr = &ptr;
  st.idx = &idx;
  st.xyz = xyz;
  st.leaf = std::max(leaf, 1);
  st.stamp.assign(n, 0);
  st.side.assign(n, 0);
  std::vector<int> all(n);
  std::iota(all.begin(), all.end(), 0);
  nd_rec(st, all);
  return st.out;
}

// ---------------------------------------------------------------- symbolic

void symbolic(Factor& f, const SymCSR& A, std::vector<int> perm) {
  const int n = A.n;
  f.n = n;
  std::vector<int> iperm(n);
  for (int k = 0; k < n; ++k) iperm[perm[k]] = k;

  // elimination tree (Liu, with path compression)
  std::vector<int> parent(n, -1), anc(n, -1);
  for (int k = 0; k < n; ++k) {
    int orig = perm[k];
    for (int64_t p = A.ptr[orig]; p < A.ptr[orig + 1]; ++p) {
      int i = iperm[A.idx[p]];
      if (i >= k) continue;
      int r = i;
      while (anc[r] != -1 && anc[r] != k) {
        int t = anc[r];
        anc[r] = k;
        r = t;
      }
      if (anc[r] == -1) {
        anc[r] = k;
        parent[r] = k;
      }
    }
  }
  // post-order (children visited in increasing order)
  std::vector<int> head(n, -1), next(n, -1);
  for (int k = n - 1; k >= 0; --k)
    if (parent[k] >= 0) {
      next[k] = head[parent[k]];
      head[parent[k]] = k;
    }
  std::vector<int> post;
  post.reserve(n);
  std::vector<int> stack;
  for (int r = 0; r < n; ++r) {
    if (parent[r] != -1) continue;
    stack.push_back(r);
    while (!stack.empty()) {
      int v = stack.back();
      if (head[v] != -1) {
        int c = head[v];
        head[v] = next[c];
        stack.push_back(c);
      } else {
        stack.pop_back();
        post.push_back(v);
      }
    }
  }
  std::vector<int> ipost(n);
  for (int k = 0; k < n; ++k) ipost[post[k]] = k;
  f.perm.resize(n);
  f.iperm.resize(n);
  f.parent.assign(n, -1);
  for (int k = 0; k < n; ++k) {
    f.perm[k] = perm[post[k]];
    f.iperm[f.perm[k]] = k;
    int p = parent[post[k]];
    f.parent[k] = p < 0 ? -1 : ipost[p];
  }
  f.first_desc.resize(n);
  for (int k = 0; k < n; ++k) f.first_desc[k] = k;
  for (int k = 0; k < n; ++k)
    if (f.parent[k] >= 0) f.first_desc[f.parent[k]] = std::min(f.first_desc[f.parent[k]], f.first_desc[k]);
  f.depth.assign(n, 0);
  for (int k = n - 1; k >= 0; --k)
    if (f.parent[k] >= 0) f.depth[k] = f.depth[f.parent[k]] + 1;

  // column counts by row-subtree traversal: L_ik != 0 iff k on a path from
  // some j (A_ij != 0, j < i) up towards i
  std::vector<int> colcount(n, 1), mark(n, -1);
  for (int i = 0; i < n; ++i) {
    mark[i] = i;
    int orig = f.perm[i];
    for (int64_t p = A.ptr[orig]; p < A.ptr[orig + 1]; ++p) {
      int j = f.iperm[A.idx[p]];
      if (j >= i) continue;
      for (int k = j; mark[k] != i; k = f.parent[k]) {
        mark[k] = i;
        colcount[k]++;
      }
    }
  }
  // fundamental supernodes
  std::vector<int> nchild(n, 0);
  for (int k = 0; k < n; ++k)
    if (f.parent[k] >= 0) nchild[f.parent[k]]++;
  f.sup_start.clear();
  f.col2sup.assign(n, 0);
  for (int k = 0; k < n; ++k) {
    bool merge = k > 0 && f.parent[k - 1] == k && colcount[k - 1] == colcount[k] + 1 && nchild[k] == 1 &&
                 (k - f.sup_start.back()) < 256;
    if (!merge) f.sup_start.push_back(k);
    f.col2sup[k] = (int)f.sup_start.size() - 1;
  }
  const int ns = (int)f.sup_start.size();
  f.sup_start.push_back(n);
  // supernode row structure = structure of its first column
  f.rowptr.assign(ns + 1, 0);
  for (int s = 0; s < ns; ++s) f.rowptr[s + 1] = f.rowptr[s] + colcount[f.sup_start[s]];
  f.rows.assign(f.rowptr[ns], 0);
  std::vector<int64_t> fill(ns);
  for (int s = 0; s < ns; ++s) {
    fill[s] = f.rowptr[s];
    for (int c = f.sup_start[s]; c < f.sup_start[s + 1]; ++c) f.rows[fill[s]++] = c;
  }
  std::fill(mark.begin(), mark.end(), -1);
  for (int i = 0; i < n; ++i) {
    mark[i] = i;
    int orig = f.perm[i];
    for (int64_t p = A.ptr[orig]; p < A.ptr[orig + 1]; ++p) {
      int j = f.iperm[A.idx[p]];
      if (j >= i) continue;
      for (int k = j; mark[k] != i; k = f.parent[k]) {
        mark[k] = i;
        int s = f.col2sup[k];
        if (k == f.sup_start[s] && i >= f.sup_start[s + 1]) f.rows[fill[s]++] = i;
      }
    }
  }
  f.valptr.assign(ns + 1, 0);
  f.nnz_L = 0;
  f.flops = 0;
  for (int s = 0; s < ns; ++s) {
    std::sort(f.rows.begin() + f.rowptr[s], f.rows.begin() + f.rowptr[s + 1]);
    int64_t nr = f.rowptr[s + 1] - f.rowptr[s];
    int64_t nc = f.sup_start[s + 1] - f.sup_start[s];
    f.valptr[s + 1] = f.valptr[s] + nr * nc;
    f.nnz_L += nr * nc - nc * (nc - 1) / 2;
    for (int64_t c = 0; c < nc; ++c) {
      double below = (double)(nr - c - 1);
      f.flops += below * below + below;
    }
  }
}

// ---------------------------------------------------------------- numeric

int64_t numeric(Factor& f, const SymCSR& A) {
  const int n = f.n;
  const int ns = (int)f.sup_start.size() - 1;
  f.val.assign(f.valptr[ns], 0.0);
  std::vector<int> map(n, -1);
  // scatter the lower triangle of P A P^T
  for (int s = 0; s < ns; ++s) {
    const int64_t nr = f.rowptr[s + 1] - f.rowptr[s];
    for (int64_t r = 0; r < nr; ++r) map[f.rows[f.rowptr[s] + r]] = (int)r;
    for (int c = f.sup_start[s]; c < f.sup_start[s + 1]; ++c) {
      int orig = f.perm[c];
      double* col = &f.val[f.valptr[s] + (int64_t)(c - f.sup_start[s]) * nr];
      for (int64_t p = A.ptr[orig]; p < A.ptr[orig + 1]; ++p) {
        int i = f.iperm[A.idx[p]];
        if (i < c) continue;
        col[map[i]] += A.val[p];
      }
    }
  }
#ifdef _OPENMP
  const int nth = omp_get_max_threads();
#else
  const int nth = 1;
#endif
  std::vector<std::vector<double>> Cbuf(nth);
  std::vector<std::vector<int>> maps(nth, std::vector<int>(n, -1));
  std::vector<int> grp;
  for (int s = 0; s < ns; ++s) {
    const int c0 = f.sup_start[s];
    const int nc = f.sup_start[s + 1] - c0;
    const int64_t nr = f.rowptr[s + 1] - f.rowptr[s];
    double* B = &f.val[f.valptr[s]];
    // dense Cholesky of the nr x nc panel (left-looking over its columns;
    // the rows of a tall panel are split over threads)
    const bool par_panel = (double)nr * nc * nc > 4e6;
    for (int j = 0; j < nc; ++j) {
      double* cj = B + (int64_t)j * nr;
      // the diagonal entry first (it needs only rows j of earlier columns)
      for (int k = 0; k < j; ++k) cj[j] -= B[(int64_t)k * nr + j] * B[(int64_t)k * nr + j];
      const double d = cj[j];
      if (!(d > 0.0) || !std::isfinite(d)) return 1 + c0 + j;
      const double r = std::sqrt(d);
      cj[j] = r;
      const double inv = 1.0 / r;
      const int64_t rows = nr - j - 1;
      constexpr int64_t kChunk = 256;
      const int64_t nchunk = (rows + kChunk - 1) / kChunk;
#pragma omp parallel for schedule(static) if (par_panel && nchunk > 1)
      for (int64_t ch = 0; ch < nchunk; ++ch) {
        const int64_t i0 = j + 1 + ch * kChunk, i1 = std::min<int64_t>(nr, i0 + kChunk);
        for (int k = 0; k < j; ++k) {
          const double* ck = B + (int64_t)k * nr;
          const double a = ck[j];
          for (int64_t i = i0; i < i1; ++i) cj[i] -= ck[i] * a;
        }
        for (int64_t i = i0; i < i1; ++i) cj[i] *= inv;
      }
    }
    // push the Schur update of the below rows onto the ancestor supernodes:
    // one group of rows per ancestor supernode K; the groups write disjoint
    // columns (those of K), so they run in parallel, each thread with its own
    // product buffer and row map
    const int nb = (int)(nr - nc);
    if (nb <= 0) continue;
    const int* R = &f.rows[f.rowptr[s] + nc];
    grp.clear();
    for (int a0 = 0; a0 < nb;) {
      const int K = f.col2sup[R[a0]];
      int a1 = a0;
      while (a1 < nb && f.col2sup[R[a1]] == K) ++a1;
      grp.push_back(a0);
      a0 = a1;
    }
    grp.push_back(nb);
    const int ng = (int)grp.size() - 1;
#pragma omp parallel if ((double)nb * nb * nc > 2e6 && ng > 1)
    {
#ifdef _OPENMP
      const int th = omp_get_thread_num();
#else
      const int th = 0;
#endif
      std::vector<double>& C = Cbuf[th];
      std::vector<int>& map = maps[th];
#pragma omp for schedule(dynamic, 1)
      for (int gi = 0; gi < ng; ++gi) {
        const int a0 = grp[gi], a1 = grp[gi + 1];
        const int K = f.col2sup[R[a0]];
        const int g = a1 - a0;
        const int64_t h = nb - a0;  // rows a0..nb-1
        C.assign((size_t)h * g, 0.0);
        // C[r, c] = sum_k B[nc+a0+r, k] * B[nc+a0+c, k]
        for (int c = 0; c < g; ++c) {
          double* Cc = &C[(size_t)c * h];
          for (int k = 0; k < nc; ++k) {
            const double* bk = B + (int64_t)k * nr + nc + a0;
            const double coef = bk[c];
            if (coef == 0.0) continue;
            for (int64_t r = c; r < h; ++r) Cc[r] += bk[r] * coef;
          }
        }
        const int64_t nrK = f.rowptr[K + 1] - f.rowptr[K];
        for (int64_t r = 0; r < nrK; ++r) map[f.rows[f.rowptr[K] + r]] = (int)r;
        double* BK = &f.val[f.valptr[K]];
        for (int c = 0; c < g; ++c) {
          double* colK = BK + (int64_t)(R[a0 + c] - f.sup_start[K]) * nrK;
          const double* Cc = &C[(size_t)c * h];
          for (int64_t r = c; r < h; ++r) colK[map[R[a0 + r]]] -= Cc[r];
        }
      }
    }
  }
  return 0;
}

// ------------------------------------------------------------ inverse factor

int64_t inverse_factor_nnz(const Factor& f) {
  int64_t nnz = 0;
  for (int k = 0; k < f.n; ++k) nnz += (int64_t)f.depth[k] + 1;
  return nnz;
}

void inverse_factor(const Factor& f, std::vector<int64_t>& s_rowptr, std::vector<double>& s_val,
                    std::vector<int64_t>& st_ptr, std::vector<int>& st_idx, std::vector<double>& st_val) {
  const int n = f.n;
  s_rowptr.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) s_rowptr[i + 1] = s_rowptr[i] + (i - f.first_desc[i] + 1);
  st_ptr.assign(n + 1, 0);
  for (int j = 0; j < n; ++j) st_ptr[j + 1] = st_ptr[j] + f.depth[j] + 1;
  const int64_t nnz = st_ptr[n];
  s_val.assign(s_rowptr[n], 0.0);
  st_idx.assign(nnz, 0);
  st_val.assign(nnz, 0.0);
  // column j of L^-1: forward substitution restricted to the path j -> root
#pragma omp parallel
  {
    std::vector<double> x(n, 0.0);
#pragma omp for schedule(dynamic, 16)
    for (int j = 0; j < n; ++j) {
      x[j] = 1.0;
      int64_t out = st_ptr[j];
      for (int k = j; k >= 0; k = f.parent[k]) {
        const int s = f.col2sup[k];
        const int c = k - f.sup_start[s];
        const int64_t nr = f.rowptr[s + 1] - f.rowptr[s];
        const double* col = &f.val[f.valptr[s] + (int64_t)c * nr];
        const int* rw = &f.rows[f.rowptr[s]];
        const double xk = x[k] / col[c];
        x[k] = 0.0;
        for (int64_t r = c + 1; r < nr; ++r) x[rw[r]] -= col[r] * xk;
        st_idx[out] = k;
        st_val[out] = xk;
        s_val[s_rowptr[k] + (j - f.first_desc[k])] = xk;
        ++out;
      }
    }
  }
}

void solve_host(const Factor& f, const double* b, double* x) {
  const int n = f.n;
  const int ns = (int)f.sup_start.size() - 1;
  std::vector<double> y(n);
  for (int k = 0; k < n; ++k) y[k] = b[f.perm[k]];
  for (int s = 0; s < ns; ++s) {
    const int64_t nr = f.rowptr[s + 1] - f.rowptr[s];
    const int* rw = &f.rows[f.rowptr[s]];
    for (int c = 0; c < f.sup_start[s + 1] - f.sup_start[s]; ++c) {
      const double* col = &f.val[f.valptr[s] + (int64_t)c * nr];
      const int k = f.sup_start[s] + c;
      y[k] /= col[c];
      for (int64_t r = c + 1; r < nr; ++r) y[rw[r]] -= col[r] * y[k];
    }
  }
  for (int s = ns - 1; s >= 0; --s) {
    const int64_t nr = f.rowptr[s + 1] - f.rowptr[s];
    const int* rw = &f.rows[f.rowptr[s]];
    for (int c = f.sup_start[s + 1] - f.sup_start[s] - 1; c >= 0; --c) {
      const double* col = &f.val[f.valptr[s] + (int64_t)c * nr];
      const int k = f.sup_start[s] + c;
      double acc = y[k];
      for (int64_t r = c + 1; r < nr; ++r) acc -= col[r] * y[rw[r]];
      y[k] = acc / col[c];
    }
  }
  for (int k = 0; k < n; ++k) x[f.perm[k]] = y[k];
}

}  // namespace pdf
