// Operation records of the H-LU schedule and their batched executors.
//
// The H-LU factorisation (App. "LU Decomposition") is expanded on the host
// into a list of small dense operations on device buffers; a dependency
// analysis on row segments groups independent operations into waves, and
// each wave runs as one batched launch per operation kind.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace hm {

// C = beta C + alpha A B on strided views: X(i, j) = X[i * rs + j * cs].
struct GemmOp {
  const double* A;
  const double* B;
  double* C;
  int m, n, k;
  int pad;
  int64_t ars, acs, brs, bcs, crs, ccs;
  double alpha, beta;
};

// Unpivoted LU of an m x m block (m <= LU_BASE), writing the inverses of its
// unit-lower and upper factors (full m x m storage, zeros in the other triangle).
struct LuOp {
  double* A;
  double* Li;
  double* Ui;
  int64_t lda, ldl, ldu;
  int m;
  int pad;
};

// Truncation core of a low-rank sum X = A B' (A: m x K, B: n x K) from the
// Gram matrices GA = A'A, GB = B'B (K x K, row-major): writes TA, TB (K x kf,
// row-major) with X ~= (A TA)(B TB)', and the rank.
struct TruncOp {
  const double* GA;
  const double* GB;
  double* TA;
  double* TB;
  int* rank;
  int K, kf;
  double tol;
};

// dst = beta dst + alpha src on strided m x n views (src == nullptr: the
// constant alpha; beta == 0 does not read dst).
struct CopyOp {
  const double* src;
  double* dst;
  int m, n;
  int64_t srs, scs, drs, dcs;
  double alpha, beta;
};

// dst[i] = sum_{p < nparts} parts[p * stride + i], i < count.
struct ReduceOp {
  const double* parts;
  double* dst;
  int64_t stride, count;
  int nparts;
  int pad;
};

constexpr int LU_BASE = 32;    // leaf LU base-case size (one CTA)
constexpr int TRUNC_MAXK = 96;   // 3 K x K FP64 matrices fit in 227 KB of shared memory

struct Wave {
  std::vector<GemmOp> gemm;
  std::vector<LuOp> lu;
  std::vector<TruncOp> trunc;
  std::vector<CopyOp> copy;
  std::vector<ReduceOp> reduce;
};

// Device-resident copy of a schedule, executed wave by wave.
struct DevSchedule {
  int nwaves = 0;
  // per wave: [begin, end) into the flat per-kind arrays, 5 kinds
  std::vector<int> begin, end;  // size 5 * nwaves each
  std::vector<int> tile_begin;  // per wave: first tile of its GEMMs in the flat tile prefix
  GemmOp* gemm = nullptr;
  LuOp* lu = nullptr;
  TruncOp* trunc = nullptr;
  CopyOp* copy = nullptr;
  ReduceOp* reduce = nullptr;
  int* gemm_tile_prefix = nullptr;  // per GEMM op: first tile (global prefix)
  std::vector<int> h_gemm_tiles_total;  // per wave: tiles
};

int upload_schedule(const std::vector<Wave>& waves, DevSchedule& S, std::vector<void*>& allocs);
int run_schedule(const DevSchedule& S, int* d_err, cudaStream_t st);

int gemm_tiles(int m, int n);

}  // namespace hm
