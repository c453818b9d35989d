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
