// Host-only driver of the library's factorization for CPU tests: factor a
// symmetric matrix, solve with the supernodal factor, and apply
// A^-1 = S^T S through the skyline rows of S and the CSR of S^T exactly as
// the GPU kernels traverse them.
#include <cstdint>
#include <vector>

#include "../../paper_2605_14526_b300/csrc/factor.h"

extern "C" int factor_check(int n, const int64_t* ptr, const int* idx, const double* val, const double* xyz,
                            const double* b, double* x_solve, double* x_sts, int64_t* stats) {
  pdf::SymCSR A;
  A.n = n;
  A.ptr.assign(ptr, ptr + n + 1);
  A.idx.assign(idx, idx + ptr[n]);
  A.val.assign(val, val + ptr[n]);
  pdf::Factor f;
  std::vector<int> perm = pdf::nested_dissection(n, A.ptr, A.idx, xyz, 8);
  // perm must be a permutation
  std::vector<int> seen(n, 0);
  for (int v : perm) {
    if (v < 0 || v >= n || seen[v]) return -1;
    seen[v] = 1;
  }
  if ((int)perm.size() != n) return -2;
  pdf::symbolic(f, A, perm);
  if (pdf::numeric(f, A)) return -3;
  pdf::solve_host(f, b, x_solve);
  std::vector<int64_t> srp, stp;
  std::vector<double> sv, stv;
  std::vector<int> sti;
  pdf::inverse_factor(f, srp, sv, stp, sti, stv);
  std::vector<double> bp(n), y(n, 0.0);
  for (int k = 0; k < n; ++k) bp[k] = b[f.perm[k]];
  for (int i = 0; i < n; ++i)
    for (int j = f.first_desc[i]; j <= i; ++j) y[i] += sv[srp[i] + (j - f.first_desc[i])] * bp[j];
  for (int j = 0; j < n; ++j) {
    double acc = 0.0;
    for (int64_t p = stp[j]; p < stp[j + 1]; ++p) acc += stv[p] * y[sti[p]];
    x_sts[f.perm[j]] = acc;
  }
  stats[0] = f.nnz_L;
  stats[1] = stp[n];
  stats[2] = (int64_t)f.sup_start.size() - 1;
  return 0;
}

// Mode T on the host: the partitioned-inverse sweeps (tsolve.h) on 3
// right-hand sides b [n][3] (original order) -> x [n][3]; stats: nodes,
// levels, stored entries of one copy, nnz(L), rows of U, and a structural
// check code (0 = every node's gather sources are its children's U rows,
// every column is owned by exactly one node, heights increase to the root).
#include "../../paper_2605_14526_b300/csrc/tsolve.h"

extern "C" int tsolve_check(int n, const int64_t* ptr, const int* idx, const double* val, const double* xyz,
                            int leaf, const double* b, double* x, int64_t* stats) {
  pdf::SymCSR A;
  A.n = n;
  A.ptr.assign(ptr, ptr + n + 1);
  A.idx.assign(idx, idx + ptr[n]);
  A.val.assign(val, val + ptr[n]);
  pdf::Factor f;
  std::vector<int> perm = pdf::nested_dissection(n, A.ptr, A.idx, xyz, leaf);
  pdf::symbolic(f, A, perm);
  if (pdf::numeric(f, A)) return -3;
  pdf::TSolve t;
  pdf::build_tsolve(f, t);
  // structure: columns owned once, contiguous
  std::vector<int> owner(n, -1);
  for (int u = 0; u < t.n_node; ++u)
    for (int c = t.c0[u]; c < t.c0[u] + t.nc[u]; ++c) {
      if (owner[c] != -1) return -10;
      owner[c] = u;
    }
  for (int c = 0; c < n; ++c)
    if (owner[c] == -1) return -11;
  // below rows lie past the node and belong to nodes of larger height
  for (int u = 0; u < t.n_node; ++u)
    for (int64_t i = t.boff[u]; i < t.boff[u + 1]; ++i) {
      const int r = t.below[i];
      if (r < t.c0[u] + t.nc[u] || t.height[owner[r]] <= t.height[u]) return -12;
    }
  // every U row feeds exactly one position of exactly one node
  std::vector<int> fed(t.u_rows, 0);
  for (int s : t.gsrc) {
    if (s < 0 || s >= t.u_rows) return -13;
    fed[s]++;
  }
  for (int u = 0; u < t.n_node; ++u)
    for (int64_t i = t.boff[u]; i < t.boff[u + 1]; ++i)
      if (fed[i] != 1) return -14;
  std::vector<double> bp((size_t)3 * n), xp((size_t)3 * n);
  for (int k = 0; k < n; ++k)
    for (int a = 0; a < 3; ++a) bp[3 * (size_t)k + a] = b[3 * (size_t)f.perm[k] + a];
  pdf::tsolve_host(t, bp.data(), xp.data());
  for (int k = 0; k < n; ++k)
    for (int a = 0; a < 3; ++a) x[3 * (size_t)f.perm[k] + a] = xp[3 * (size_t)k + a];
  stats[0] = t.n_node;
  stats[1] = t.n_level;
  stats[2] = t.entries;
  stats[3] = f.nnz_L;
  stats[4] = t.u_rows;
  return 0;
}
