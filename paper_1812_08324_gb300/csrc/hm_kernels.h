// Launcher declarations of the device kernels (one translation unit each).
#pragma once

#include <cuda_runtime.h>

#include "hm_internal.h"

namespace hm {

void count_launches(int n);  // process-wide launch statistics

// Parameters of nu and of the discretisation, passed by value to kernels.
struct NuParams {
  int dim, kernel, nw, n0, n1;
  double h, s, eps, lam, trunc, LW, r;
  double cds;   // c_{d,s}
  double expo;  // d + 2 s
};

constexpr int MV_CHUNK = 32;   // rows per H-matvec row chunk
constexpr int VT_CHUNK = 256;  // columns per far-field V' x task
constexpr int ACA_MAXK = 128;  // largest rank cap of an ACA block

int launch_constants(const NuParams& q, double* d_tab, double* d_scratch, cudaStream_t st);
int launch_finalize_constants(const NuParams& q, double a, const double* b, double c,
                              const double* d_scratch, GenConst* d_gc, cudaStream_t st);
int launch_near_fill(const EntryCtx& E, const DenseDesc* d_dd, int ndense, double* pool,
                     cudaStream_t st);
// Split form of the H-matvec: jump entries of the dense leaves and a plain
// FP64 -> float-pair split of an array.
int launch_near_fill_jump(const EntryCtx& E, const DenseDesc* d_dd, int ndense, float2* pool, cudaStream_t st);
int launch_split(const double* src, float2* dst, int64_t n, cudaStream_t st);
// copy segments (source offset, target offset, count: 3 int64 per segment, device) of src to dst
int launch_copy_segments(const int64_t* d_jobs, int njobs, const double* src, double* dst, cudaStream_t st);
int launch_entries(const EntryCtx& E, const int* iperm, int N, int64_t count, const int* rows,
                   const int* cols, double* out, int* err, cudaStream_t st);
int launch_to_dense(const DenseDesc* d_dd, int ndense, const double* pool, const LRDesc* d_ld,
                    int nlr, const int* rank, const double* U, const double* V, const int* perm,
                    int N, double* out, cudaStream_t st);

int launch_aca(const EntryCtx& E, const LRDesc* d_ld, int nlr, int max_m, double* U, double* V,
               int* rank, int* capped, double tol, cudaStream_t st);

// H-matvec pieces (Morton-order vectors).
struct MatvecPlan {
  int nlr, ndense, nvt, nchunk;
  const LRDesc* ld;
  const DenseDesc* dd;
  const int* rank;
  const double* U;
  const double* V;
  const double* D;
  const VTask* vt;
  const int* vt_range;     // per LR: [begin, end) of its tasks (2 ints each)
  const RowChunk* chunks;
  const int* dense_items;
  const int* lr_items;
  double* partial;         // nvt x ACA_MAXK scratch
  double* tvec;            // nlr x ACA_MAXK scratch
  int kmax;                // largest rank cap (<= ACA_MAXK)
  // Split form (constant-order problems on a box; null otherwise): G = S + J
  // with S the stencil and the diagonal (applied in FP64 from the constants)
  // and J the jump entries (dense leaves with the diagonal and the stencil
  // removed, and the low-rank blocks) stored as float pairs (hi + lo) and
  // multiplied in double-float arithmetic.
  const float2* Ddf;       // like D: jump entries, zero on the diagonal
  const float2* Udf;
  const float2* Vdf;
  float2* tdf;             // nlr x ACA_MAXK: tvec as float pairs
  const int4* nb;          // per Morton row: neighbours (-axis0, +axis0, -axis1, +axis1), -1 if none
  const GenConst* gc;      // diag and stencil coefficients
};

// y = alpha x + beta (H x) + gamma (w1 + w2) (+ w3 * 1 if w3 != nullptr)
int launch_matvec(const MatvecPlan& P, double alpha, double beta, const double* x, double gamma,
                  const double* w1, const double* w2, const double* w3, double* y, cudaStream_t st);

// One H-matvec of a batch: y = alpha x + beta (H x) + gamma (w1 + w2) (+ w3).
struct MvJob {
  MatvecPlan P;
  double alpha, beta, gamma;
  const double* x;
  const double* w1;
  const double* w2;
  const double* w3;
  double* y;
};
// Device job table of a batch and, per launch kind (V'x tasks, reductions,
// row chunks), the first block of every job (count + 1 entries) and the total.
// Jobs without V'x tasks contribute no blocks to the first two launches.
struct MvBatch {
  const MvJob* jobs;
  const int* off[3];
  int total[3];
  int count;
};
int launch_matvec_batch(const MvBatch& B, cudaStream_t st);

// Fixed scratch of hm_matvec_noalloc: capacity in doubles and device address
// (looked up on first use per device).
size_t noalloc_capacity();
int noalloc_scratch(double** out);

int launch_gather(const int* perm, int N, const double* src, double* dst, cudaStream_t st);
int launch_scatter(const int* perm, int N, const double* src, double* dst, cudaStream_t st);

}  // namespace hm
