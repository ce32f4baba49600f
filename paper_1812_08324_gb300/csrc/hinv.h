// Hierarchical inverses of the H-LU triangular factors (1D problems).
//
// The triangular solves L y = b, U z = y of App. "LU Decomposition" are a
// chain of dependent leaf steps.  For the binary cluster tree of a 1D grid
// the inverses of the factors are themselves hierarchical with small ranks:
// for a cluster tau with children a (first) and b,
//     L_tau^{-1} = [ X_a  0 ; -X_b L_ba X_a   X_b ],
//     U_tau^{-1} = [ Y_a  -Y_a U_ab Y_b ;  0   Y_b ],
// and the off-diagonal blocks W_tau = -X_b L_ba X_a (-Y_a U_ab Y_b) have
// numerical ranks of a few tens at 1e-12.  They are formed bottom-up, level
// by level, from products with the factors and the already formed lower
// levels only (randomised two-sided sketch: Y = W Omega, Z = W^T Psi,
// W ~ Y (Psi^T Y)^+ Z^T with a column-pivoted QR of the small core as the
// truncated pseudo-inverse; Nakatsukasa, "Fast and stable randomized low-rank
// matrix approximation", 2020).  Applying them is then a fully parallel,
// bandwidth-bound product per factor instead of a substitution chain.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "hm_internal.h"

namespace hm {

struct FactorLayout;

constexpr int HINV_S = 48;      // range-sketch columns
constexpr int HINV_SP = 64;     // co-range-sketch columns
constexpr int HINV_KCAP = 40;   // rank cap of an inverse block (ranks that reach it are flagged)
constexpr int HINV_MAXS = 64;   // widest multi-vector of the construction
constexpr int HINV_RCH = 32;    // rows per row chunk of the construction
constexpr int HINV_ACH = 64;    // rows per row chunk of the per-step products (two per lane)
constexpr int HINV_AWARPS = 4;  // warps per row chunk of the per-step products
constexpr int HINV_TCH = 256;   // rows per chunk of the per-step V'x products
constexpr int HINV_MCH = 128;   // rows per chunk of the construction's reductions

// storage of the per-step inverses: FP64; FP32 or BF16 (mixed precision);
// DF = FP64-accurate pairs of floats (hi + lo) applied in double-float arithmetic
enum HinvPrec { HINV_F64 = 0, HINV_F32 = 1, HINV_BF16 = 2, HINV_DF = 3 };
constexpr int HINV_MAX_ANC = 24;  // deepest 1D cluster tree the per-step kernels stage

// ---- per-step application of one triangular inverse (device tables)
struct HinvLeaf {     // inverse of a diagonal leaf block: its triangle, column-major, column stride ld
  int r0, m, ld;
  int64_t off;              // into the leaf pool (elements)
};
struct HinvNode {     // inverse block P Q^T of an internal cluster
  int tgt0, tgt_n, src0, src_n;
  int pld, qld;             // column strides (multiples of 8) of P (tgt_n x KCAP) and Q (src_n x KCAP)
  int tch_begin, tch_end;   // its chunks of the per-step V'x products
  int64_t poff, qoff;       // column-major P and Q in the pools
};
// A run of columns multiplied into the rows of one row chunk: of a leaf
// triangle (vector: the input b) or of an inverse block's P (vector: t).
struct HinvSeg {
  int64_t off;              // pool element of column 0 at the chunk's first row
  int64_t voff;             // vector entry of column 0 (into b or into tvec)
  int ld, n;                // column stride, columns
  int kind;                 // 0: leaf triangle, 1: P
  int a_hi;                 // rows [0, 32) of the chunk read columns [0, a_hi)
  int b_lo;                 // rows [32, 64) read columns [b_lo, n) (the rest is zero)
  int pad;
};
struct HinvRChunk {   // HINV_ACH rows and their segments (host-balanced over the warps)
  int row0, nr;
  int seg_begin, seg_end;
};
struct HinvApply {
  int lower;                // 1: L^{-1} (leaf rows read j <= i), 0: U^{-1} (j >= i)
  int prec;                 // HinvPrec of the pools
  int nleaf, nnode, ntch, nrch;
  const HinvNode* nodes;
  const int4* tch;          // (node, first source row offset, partial slot, -) per product chunk,
                            // heaviest first; slots run in chunk order per node
  const HinvRChunk* rch;    // row chunks, heaviest first
  const HinvSeg* segs;      // their segments
  const void* leaf_pool;
  const void* p_pool;
  const void* q_pool;
  const int* rank;          // per node
  void* tpart;              // per product chunk: KCAP partial sums   (in the accumulator type of prec:
  void* tvec;               // per node: KCAP coefficients             FP64 double, pairs float2, else float)
  unsigned* tcount;         // per node: finished chunks (reset by the last one)
};
// One triangular inverse applied to a Morton-order vector: y = X b, or, with
// sub given, y = scale (X b) - sub (y may then alias sub, not b).
struct HinvJob {
  HinvApply A;
  const double* b;
  double* y;
  const double* sub;
  double scale;
};

// Launchers (hinv_apply.cu).  Single: two launches; batch: two launches for all jobs.
int launch_hinv_apply(const HinvApply& A, const double* b, double* y, cudaStream_t st);
struct HinvBatch {
  HinvJob* jobs = nullptr;
  int* off[2] = {nullptr, nullptr};  // per job its first CTA of the two launches; off[k][count] = total
  int total[2] = {0, 0};
  int count = 0;
  int prec = -1;  // the jobs' common HinvPrec, -1 if they differ
};
int launch_hinv_batch(const HinvBatch& B, cudaStream_t st);

// ---- the inverses of one factorisation
struct HinvTriangle {
  HinvApply A{};            // in the chosen storage precision
  HinvApply A64{};          // FP64 pools of the construction (released when A converts them)
  std::vector<HinvLeaf> h_leaves;
  std::vector<HinvNode> h_nodes;
  std::vector<int> h_rank;
};
struct HinvData {
  int prec = HINV_F64;
  double tol = 0.0;
  HinvTriangle tri[2];      // 0: L^{-1}, 1: U^{-1}
  std::vector<void*> allocs;
  int64_t bytes = 0;        // device bytes held
  int64_t step_bytes = 0;   // bytes one application of both inverses reads
  int max_rank = 0, capped = 0;
  double build_ms = 0.0;
  double* d_y = nullptr;    // intermediate vector (N)
  void release();
};

// Form the inverses of the factors of one or more factorisations (1D plans
// only; the ranks of each factor's blocks on the device in d_rank_f).  The
// construction steps of all of them (in groups of at most 2^19 stacked rows)
// run in one launch per kernel and step; each out receives the same inverses,
// bit for bit, as when built alone.  build_ms is the time of the whole call;
// d_err collects device errors.  Synchronises the stream.
struct HinvBuildJob {
  const Plan* P;
  const std::vector<DenseDesc>* dd;
  const FactorLayout* F;
  const int* d_rank_f;
  int prec;
  double tol;
  HinvData* out;
};
int hinv_build_batch(const std::vector<HinvBuildJob>& jobs, int* d_err, cudaStream_t st, std::string& err);

// z = U^{-1} L^{-1} b (Morton order; z may alias b).
int hinv_solve(const HinvData& D, const double* b, double* z, cudaStream_t st);

}  // namespace hm
