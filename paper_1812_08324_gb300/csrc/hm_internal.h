// Internal types shared by the host planner, the kernels and the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "levy_hmat.h"

namespace hm {

// ---------------------------------------------------------------- host plan

// A cluster: a contiguous range of Morton positions with its integer cell
// bounding box [lo, hi) (App. "Construction and Storage": X_I = {x_i}_{i in I}).
struct Cluster {
  int begin, end;
  int lo[2], hi[2];
  int level, parent;
  int nchild;
  int child[4];
};

enum BlockType { BT_H = 0, BT_LR = 1, BT_DENSE = 2 };

// A node of the block tree (t, s): H (subdivided), low rank or dense.
// H children are stored at child0 + i * ncc + j for row child i, column child j.
struct Block {
  int t, s;
  int type;
  int level;
  int child0, nrc, ncc;
  int id;  // index into the low-rank or dense tables
};

struct Plan {
  int dim = 1;
  int n[2] = {1, 1};
  int N = 0;
  double h = 0;
  int leaf = 64;
  double eta = 1.0;
  std::vector<int> perm;   // Morton position -> natural index
  std::vector<int> iperm;  // natural index -> Morton position
  std::vector<int> coord;  // Morton position -> (i0, i1), 2 ints each
  std::vector<Cluster> cl; // cl[0] = root
  std::vector<Block> bl;   // bl[0] = root block (root, root)
  std::vector<int> lr_block;     // LR id -> block id
  std::vector<int> dense_block;  // dense id -> block id
  std::vector<int> leaves;       // leaf cluster ids in Morton order
  int depth = 0;
};

int make_plan(const hm_problem& p, const hm_opts& o, Plan& plan, std::string& err);
// HM_SOLVE_SUBST or HM_SOLVE_HINV for these options (HM_SOLVE_AUTO resolved).
int solve_mode(const hm_problem& p, const hm_opts& o);
// Relative truncation of the hierarchical inverses' blocks.
double hinv_tolerance(const hm_opts& o);

// ---------------------------------------------------------------- device tables

// Row-independent constants of the discrete generator.
struct GenConst {
  double h;
  double a, b0, b1, c;
  double lam_w;   // sum' w_j nu(y_j) over the window
  double tail;    // T: mass of nu outside the window
  double kappa;   // coefficient of the central second difference (per axis)
  double diag;    // c - 2 d a/h^2 - 2 d kappa - lam_w - T
  double stencil_p[2], stencil_m[2];  // kappa + a/h^2 +- b_d/(2h)
};

// What a kernel needs to evaluate G between two Morton positions.
struct EntryCtx {
  int dim, n0, n1;
  const int2* coord;      // Morton position -> (i0, i1)
  const double* tab;      // w(j) nu(|j| h) for |j0| < n0, |j1| < n1, index j1 * n0 + j0
  const GenConst* gc;     // device copy
  // variable order (nullptr otherwise), per Morton row p: jump factor B_p,
  // exponent E_p, stencil kappa_p, diagonal; nw = window half-width in steps
  const double* rowB = nullptr;
  const double* rowE = nullptr;
  const double* rowK = nullptr;
  const double* rowD = nullptr;
  int nw = 0;
};

struct LRDesc {    // low-rank block U V', U: m x kcap, V: n x kcap, column-major
  int r0, m, c0, n, kcap;
  int pad;
  int64_t uoff, voff;
};

struct DenseDesc { // dense block, row-major m x n with row stride ld (ld >= n, ld % 4 == 0)
  int r0, m, c0, n, ld, pad;
  int64_t off;
};

// Far-field partial task of the H-matvec: V[c_lo:c_lo+len, :]' x[c0+c_lo : ...]
struct VTask {
  int lr, c_lo, len, out;  // out = index of the partial-result row
};

// Row chunk of the H-matvec: rows [r0, r0+nrow) with the lists of blocks
// covering them: items [item_begin, item_end) of the item array.
struct RowChunk {
  int r0, nrow;
  int dense_begin, dense_end;   // into dense item list (dense ids)
  int lr_begin, lr_end;         // into lr item list (lr ids)
};

}  // namespace hm
