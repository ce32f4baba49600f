// Host-side expansion of the H-LU factorisation and of the H-triangular
// solves into scheduled operation lists (App. "LU Decomposition").
#pragma once

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "hlu_ops.h"
#include "hm_internal.h"

namespace hm {

// A strided matrix view on device memory plus the row range of its owning
// buffer, for dependency tracking.
struct View {
  double* p = nullptr;
  int rows = 0, cols = 0;
  int64_t rs = 0, cs = 0;
  int buf = -1;
  int br0 = 0, br1 = 0;   // rows of the buffer touched
  bool tr = false;        // rows of the view are columns of the buffer

  View sub(int r0, int c0, int nr, int nc) const {
    View v = *this;
    v.p = p + r0 * rs + c0 * cs;
    v.rows = nr;
    v.cols = nc;
    if (!tr) { v.br0 = br0 + r0; v.br1 = v.br0 + nr; }
    return v;
  }
  View T() const {
    View v = *this;
    v.rows = cols;
    v.cols = rows;
    v.rs = cs;
    v.cs = rs;
    v.tr = !tr;
    return v;
  }
};

// Device arena: chunked bump allocation, freed as a whole.  In dry-run mode
// (fake = true) it hands out addresses from a fake range without touching the
// device, so that schedules can be planned and checked on a host without a GPU.
struct Arena {
  std::vector<void*> chunks;
  std::vector<std::pair<uintptr_t, uintptr_t>> ranges;  // [begin, end) of every chunk
  double* cur = nullptr;
  int64_t left = 0;
  int64_t total = 0;
  int status = 0;
  bool fake = false;
  uintptr_t fake_next = uintptr_t(1) << 40;
  int64_t fake_limit = -1;    // dry runs: bytes after which alloc fails (-1: no limit)
  double* alloc(int64_t n);   // doubles, 32-byte aligned
  void release();
};

// Check that every operand of every operation lies inside one of `ranges`
// (byte intervals).  Returns the number of violations.
int64_t check_spans(const std::vector<Wave>& waves,
                    const std::vector<std::pair<uintptr_t, uintptr_t>>& ranges, std::string& first,
                    const std::vector<RowSrc>* srcs = nullptr);

// Final layout of the factors consumed by the solves.
struct FactorLayout {
  std::vector<double*> linv, uinv;       // per diagonal dense block (dense id), m x m row-major
  std::vector<int64_t> linv_ld;
  std::vector<View> dense;               // per dense block (current storage)
  std::vector<double*> lr_u, lr_v;       // per LR block: U (m x kf), V (n x kf) column-major
  int kf = 0;
  int* d_rank = nullptr;                 // per LR block rank (device)
  // Solve blocks: a cut of the cluster tree (clusters of at most
  // SOLVE_BLOCK rows, twice that for 1D problems of >= 32768 unknowns).  Each keeps the exact inverses of its diagonal factor
  // blocks L_BB and U_BB (dense, row-major), and every factor block that
  // couples two solve blocks is stored scaled by the inverse of its row
  // block: P = L_BB^{-1} L_BA (dense blocks, S x n) or L_BB^{-1} U_q (rows of a
  // low-rank block's U inside B, S x kf), likewise with U_BB^{-1}.
  struct Scaled {
    bool lower;    // L part (row block after the columns) or U part
    bool lowrank;  // low-rank block q (x = V_q' y) or dense block (x = y[cols])
    int id;        // dense id or LR id
    int sb;        // solve block of the rows
    double* M;     // S x ncols row-major
    int ncols;
    int row_lo, row_hi;  // rows of M that can be nonzero (the inverse is triangular)
  };
  std::vector<int> sb_cluster;           // cluster of each solve block (Morton order)
  std::vector<double*> sb_linv, sb_uinv; // S x S row-major
  std::vector<Scaled> scaled;
};

#ifndef HM_SOLVE_BLOCK
#define HM_SOLVE_BLOCK 1024  // largest solve block (build-time tuning parameter)
#endif
constexpr int SOLVE_BLOCK = HM_SOLVE_BLOCK;

// A slice of the H-LU schedule in emission order: the ops with ids
// [first, first + graph.size()), grouped by their (global) dependency wave,
// with their producers (global op ids).  Ops only depend on ops of earlier
// ids, so slices run one after another in emission order.
struct HluChunk {
  int first = 0;
  std::vector<int> wave_idx;  // global wave of waves[i]
  std::vector<Wave> waves;    // op ids are global
  OpGraph graph;              // producers of op first + i, global ids
};

struct HluBuild {
  std::vector<Wave> waves;
  OpGraph graph;
  FactorLayout F;
  int64_t ops = 0;
  double gemm_fma[3] = {0.0, 0.0, 0.0};  // GEMM FMAs: H-LU, solve-block inverses, scaled couplings
  std::string err;
  // Streaming: with a sink, every chunk_ops ops emitted are handed to it as a
  // chunk (called on the planning thread), and the rest when planning ends;
  // `waves` then ends up empty.
  std::function<void(HluChunk&&)> sink;
  int64_t chunk_ops = 0;
};

// Expand H-LU of M = alpha I + theta G for the block tree of `P`.
//  dense_pool/ld: H's dense leaves (DenseDesc order), lr: H's low-rank blocks,
//  d_rank_f: device array (nlr) that will hold the factor ranks.
int plan_hlu(const Plan& P, const std::vector<DenseDesc>& dd, const double* d_dense,
             const std::vector<LRDesc>& ld, const double* d_U, const double* d_V, int kf,
             double theta, double lu_tol, int* d_rank_f, Arena& arena, HluBuild& out, double alpha = 1.0,
             int sb_rows_opt = 0, bool solve_blocks = true, Arena* tmp_arena = nullptr);
// sb_rows_opt: rows of the largest solve block (0: SOLVE_BLOCK, twice that for
// 1D problems of >= 32768 unknowns); solve_blocks = false skips the solve
// blocks' inverses and scaled couplings (only the substitution solve reads them);
// tmp_arena (if given) takes the pooled temporaries, which no operation after
// the schedule reads: the caller may release it once the schedule has run.

// Expand z = U^{-1} L^{-1} b (forward then backward H-triangular
// substitution, leaf by leaf over the scaled factors) into phases of row and
// partial-product tasks on Morton-order device vectors; replayed per solve.
struct SolveVectors {
  const double* b;
  double* y;     // forward result
  double* z;     // backward result
  double* acc1;  // forward partial rows
  double* acc2;  // backward partial rows
};
// rank: the factor ranks of the low-rank blocks (nullptr: the storage width kf).
int plan_solve(const Plan& P, const std::vector<DenseDesc>& dd, const std::vector<LRDesc>& ld,
               const FactorLayout& F, const std::vector<int>* rank, const SolveVectors& v, Arena& arena,
               std::vector<Wave>& waves, std::vector<RowSrc>& srcs, OpGraph& graph);

}  // namespace hm
