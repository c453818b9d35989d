// Host construction of the level-scheduled triangular solves with the factor
// (solve mode T): A^-1 b = P^T L^-T L^-1 P b on the supernodal Cholesky factor
// of factor.h, for meshes whose inverse factor S = L^-1 P (eq. Ainv_STS) is
// too dense to store or stream.
//
// The factor's columns are grouped into nodes: maximal chains of supernodes
// in which every member but the lowest is the only child of the next, capped
// at kNodeMaxCols columns. Under the post-ordered nested dissection a node is
// a separator plane (or a piece of one) or a leaf block, and the node tree is
// the separator tree. A node s owns the contiguous columns [c0, c0 + nc) and
// the rows below(s) (positions past its columns where its columns have
// entries, nb of them). Each node's block column of L is replaced by its
// partitioned inverse (Alvarado, Pothen and Schreiber 1993):
//
//   Linv_s = (L_ss)^-1          (nc x nc, lower triangular)
//   M_s    = L_{below,s} Linv_s (nb x nc, dense)
//
// so that one node of the forward solve L y = P b is one dense product,
//   r_s = b_s - sum_{children c} U_c|cols(s)
//   y_s = Linv_s r_s,   U_s = M_s r_s + sum_{children c} U_c|below(s)
// (U_t = L_{below(t), subtree(t)} y_subtree(t), the update a subtree passes
// up), and one node of the backward solve L^T x = y is one dense product,
//   x_s = Linv_s^T y_s - M_s^T x_below(s).
// Nodes of equal height in the node tree are independent in both sweeps, so
// a sweep is one pass per height (the forward from the leaves up, the
// backward from the root down) with one team barrier between heights.
// [Linv_s; M_s] is stored twice, row-major (packed: row o < nc holds
// Linv_s[o, 0..o], row nc + j holds M_s[j, 0..nc-1]) and column-major (column
// k holds Linv_s[k..nc-1, k], then M_s[0..nb-1, k]), so that both sweeps read
// contiguous runs whichever of the two index directions a lane walks.
#pragma once
#include <cstdint>
#include <vector>

#include "factor.h"

namespace pdf {

constexpr int kNodeMaxCols = 1024;   // columns per node (the forward stages r_s, nc x 3 FP64, in shared memory)
constexpr int kStageRows = 1024;     // rows of the device's shared staging vector (backward right-hand side)
constexpr int kWarpNodeCols = 32;    // nodes of at most this many columns are done by one warp
constexpr int kLaneNodeCols = 256;   // forward: larger nodes up to this many, a lane per row (no reductions)
constexpr int kWarpNodeRows = 160;   // backward: a small node with at most this many rows is one warp's
constexpr int kUnitRows = 32;        // least forward rows of a block-mode node per work unit
constexpr int kUnitCols = 8;         // backward columns per work unit when the right-hand side is staged in chunks
constexpr int kUnitEntries = 16384;  // target stored entries per work unit (staging is paid once per unit)

struct TSolve {
  int n = 0;                       // free vertices (positions)
  int n_node = 0, n_level = 0;
  std::vector<int> c0, nc, nb;     // per node: first column, columns, rows below
  std::vector<int> height;         // per node (leaves 0)
  std::vector<int64_t> boff;       // [n_node + 1]: offset of the node's below rows in `below` and in U
  std::vector<int> below;          // below rows of every node, ascending per node
  std::vector<int64_t> poff;       // [n_node + 1]: offset of the node's entries in prow and in pcol
  std::vector<double> prow, pcol;  // [Linv; M] row-major packed / column-major packed
  std::vector<int64_t> goff;       // [n_node + 1]: offset of the node's positions 0 .. nc + nb - 1 in gptr
  std::vector<int> gptr;           // [goff[n_node] + 1]: gather lists per (node, position) into gsrc
  std::vector<int> gsrc;           // U rows of the children that feed a position
  // schedule per height: block forward units {node, row0, rows, lane}
  // (lane = 1: a lane per row, nodes of at most kLaneNodeCols columns),
  // block backward units {node, col0, cols, 0}, warp forward items
  // {node, row0} (32 rows of a node of at most kWarpNodeCols columns), warp
  // backward nodes (at most kWarpNodeCols columns and kWarpNodeRows rows)
  std::vector<int> lev_f, lev_b, lev_wf, lev_wb;   // [n_level + 1] ranges into the lists below
  std::vector<int> unit_f, unit_b;                  // 4 ints per unit
  std::vector<int> wnode_f;                         // 2 ints per item
  std::vector<int> wnode_b;
  int64_t entries = 0;             // stored entries of one copy ([Linv; M] over all nodes)
  int64_t u_rows = 0;              // rows of the update buffer U (sum of nb)
  double build_seconds = 0;
};

// Nodes, partitioned inverses, gather lists and the per-height schedule.
void build_tsolve(const Factor& f, TSolve& t);

// x = L^-T L^-1 b in elimination order (3 right-hand sides, [n][3]), by the
// same per-height sweeps, gathers and node products as the device (host
// self-check and CPU tests; the summation order within a dot differs).
void tsolve_host(const TSolve& t, const double* b, double* x);

}  // namespace pdf
