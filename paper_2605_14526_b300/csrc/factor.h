// Host-side FP64 factorization of the scalar PD operator (Sec. 4.5).
//
// A = L_A (x) I_3 decouples per axis, so one scalar SPD matrix is factored and
// applied to three right-hand sides. The ordering is a geometric nested
// dissection of the mesh graph (recursive median plane cuts along the longest
// axis of the rest shape; the paper uses METIS nested dissection), post-ordered
// so that every elimination subtree is a contiguous index range. The numeric
// factorization is a supernodal left-to-right Cholesky P A P^T = L L^T
// (the paper's L D L^T with D folded into L), and the inverse factor
// S = L^-1 P gives A^-1 = S^T S (eq. Ainv_STS).
#pragma once
#include <cstdint>
#include <vector>

namespace pdf {

struct SymCSR {            // symmetric sparse matrix, full pattern, CSR
  int n = 0;
  std::vector<int64_t> ptr;
  std::vector<int> idx;
  std::vector<double> val;
};

struct Factor {
  int n = 0;
  std::vector<int> perm;       // perm[k]  = original index eliminated k-th
  std::vector<int> iperm;      // iperm[i] = elimination position of original i
  std::vector<int> parent;     // elimination tree (positions), -1 at roots
  std::vector<int> first_desc; // first descendant: subtree(k) = [first_desc[k], k]
  std::vector<int> depth;      // number of proper ancestors
  // supernodes: columns [sup_start[s], sup_start[s+1])
  std::vector<int> sup_start, col2sup;
  std::vector<int64_t> rowptr; // row structure of supernode s: rows[rowptr[s] .. rowptr[s+1])
  std::vector<int> rows;       // (positions; the first ncols rows are the supernode's own columns)
  std::vector<int64_t> valptr; // dense column-major block of supernode s
  std::vector<double> val;
  int64_t nnz_L = 0;
  double flops = 0;
};

// Geometric nested dissection of the graph (ptr, idx) with vertex coordinates
// xyz[3*i]; returns perm (elimination order). Leaves of <= leaf vertices.
std::vector<int> nested_dissection(int n, const std::vector<int64_t>& ptr, const std::vector<int>& idx,
                                   const double* xyz, int leaf);

// Symbolic analysis for the given ordering (post-orders it in place).
void symbolic(Factor& f, const SymCSR& A, std::vector<int> perm);

// Numeric supernodal Cholesky; returns 0, or 1 + position of a non-positive pivot.
int64_t numeric(Factor& f, const SymCSR& A);

// Inverse factor S = L^-1 (positions). Skyline rows: row i holds columns
// [first_desc[i], i] densely at s_val[s_rowptr[i] + (j - first_desc[i])].
// Transposed CSR: row j of S^T (= column j of S) lists its non-zeros at the
// ancestors i of j (st_idx = i, increasing) with st_val.
int64_t inverse_factor_nnz(const Factor& f);
void inverse_factor(const Factor& f, std::vector<int64_t>& s_rowptr, std::vector<double>& s_val,
                    std::vector<int64_t>& st_ptr, std::vector<int>& st_idx, std::vector<double>& st_val);

// Reference solve with the factor (host, for self-checks): x = A^-1 b.
void solve_host(const Factor& f, const double* b, double* x);

}  // namespace pdf
