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
// GemmOp::shape flag: FP64 arithmetic instead of double-float (HM_GEMM_FP64=1)
constexpr int GEMM_FP64 = 4;

struct GemmOp {
  const double* A;
  const double* B;
  double* C;
  int m, n, k;
  int shape;         // output tile: 0 = 32 x 32, 1 = 64 x 16, 2 = 16 x 64 (gemm_shape), 3 = 64 x 64, | GEMM_FP64
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
  int pad;       // flags: LU_DF
};
// LuOp::pad flag: double-float base LU instead of FP64 (HM_LU_DF=1)
constexpr int LU_DF = 1;

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

// dst(i, j) = beta dst(i, j) + alpha sum_{p < nparts} parts[p * stride + i * n + j]
// for i < m, j < n (dst strided; beta == 0 does not read dst).
struct ReduceOp {
  const double* parts;
  double* dst;
  int64_t stride, drs, dcs;
  int m, n;
  int nparts;
  int pad;
  double alpha, beta;
};

// One source of a row task: dense row-major block (x = a vector segment of
// ncols entries) or low-rank factor rows (column-major, x = the sum of nparts
// partial products of kf entries each, laid out back to back).
struct RowSrc {
  const double* M;   // element (r, c) of the task's rows: M[r * rs + c * cs], r relative to the task
  int64_t rs, cs;
  const double* x;
  int ncols;
  int nparts;        // 0: dense source; > 0: low-rank source
  double sign;
  // shared-memory staging of the task, set by plan_rows_staging:
  int pre_off;       // offset of the copied rows of M (-1: read from global memory)
  int dyn_off;       // offset of the gathered x; -(start + 1) when x is read from global memory
};

// out[r] = base[r] + sum over sources, rows r0 .. r0 + nr - 1 (nr <= 32);
// base == nullptr means 0.
struct RowsOp {
  double* out;
  const double* base;
  int r0, nr;
  int src_begin, src_end;
  int dyn_base, dyn_total;  // gathered base rows start at dyn_base; dyn_total doubles in all
};

// Executor modes: 0 runs H-LU schedules (one CTA per SM, 225 KB shared
// memory, truncation cores up to TRUNC_MAXK); 3 runs H-LU schedules whose
// truncation cores stay within TRUNC_MAXK_2CTA with two CTAs per SM (101 KB
// each: twice the warps to hide the latency of the small tasks); the solve
// modes trade shared-memory staging for CTAs per SM: mode 1 (latency: one
// solve) two CTAs per SM, mode 2 (throughput: batched solves) four.  Staging
// of a row task (doubles): copied matrix rows, gathered inputs; and the
// copied V rows of a partial-product task.
constexpr int EXEC_MODES = 4;
constexpr int SOLVE_MODE_LATENCY = 1, SOLVE_MODE_THROUGHPUT = 2, FACTOR_MODE_2CTA = 3;
constexpr int TRUNC_MAXK_2CTA = 64;
__host__ __device__ constexpr int mode_ctas(int m) { return m == 0 ? 1 : (m == 2 ? 4 : 2); }
__host__ __device__ constexpr bool mode_factor(int m) { return m == 0 || m == FACTOR_MODE_2CTA; }
__host__ __device__ constexpr int mode_prefetch(int m) { return m == 1 ? 6144 : 3072; }
__host__ __device__ constexpr int mode_dyn(int m) { return m == 1 ? 5120 : 2560; }
__host__ __device__ constexpr int mode_vpart(int m) { return m == 1 ? 8192 : 4096; }
constexpr int ROWS_MAX_SRC = 64;

// Lays out the staging of one row task: the rows of M of each source go to
// shared memory while they fit (low-rank rows padded to ncols + 1 against bank
// conflicts), and so do the source vectors and the base rows.
void plan_rows_staging(RowsOp& op, RowSrc* src, int mode);

// part[l] = sum_{r < len} V[r + l * ldv] y[r], l < kf.
struct VPartOp {
  const double* V;
  const double* y;
  double* part;
  int64_t ldv;
  int len, kf;
};

constexpr int LU_BASE = 32;    // leaf LU base-case size (one CTA)
constexpr int LU_SEG = 32;     // rows per dependency-tracking segment of the factor blocks
constexpr int TRUNC_MAXK = 96;   // 3 K x K FP64 matrices fit in 227 KB of shared memory

// Operations of one wave (a topological level), with their global op ids.
struct Wave {
  std::vector<GemmOp> gemm;
  std::vector<LuOp> lu;
  std::vector<TruncOp> trunc;
  std::vector<CopyOp> copy;
  std::vector<ReduceOp> reduce;
  std::vector<RowsOp> rows;
  std::vector<VPartOp> vpart;
  std::vector<int> gemm_id, lu_id, trunc_id, copy_id, reduce_id, rows_id, vpart_id;
  void add(const GemmOp& o, int id) { gemm.push_back(o); gemm_id.push_back(id); }
  void add(const LuOp& o, int id) { lu.push_back(o); lu_id.push_back(id); }
  void add(const TruncOp& o, int id) { trunc.push_back(o); trunc_id.push_back(id); }
  void add(const CopyOp& o, int id) { copy.push_back(o); copy_id.push_back(id); }
  void add(const ReduceOp& o, int id) { reduce.push_back(o); reduce_id.push_back(id); }
  void add(const RowsOp& o, int id) { rows.push_back(o); rows_id.push_back(id); }
  void add(const VPartOp& o, int id) { vpart.push_back(o); vpart_id.push_back(id); }
  size_t size() const {
    return gemm.size() + lu.size() + trunc.size() + copy.size() + reduce.size() + rows.size() + vpart.size();
  }
};

// Producer ops of every op (by op id): an op may start once all its
// producers have finished (read-after-write, write-after-read, write-after-write).
struct OpGraph {
  std::vector<int> off = std::vector<int>(1, 0);  // producers of op i: flat[off[i] .. off[i+1])
  std::vector<int> flat;
  std::vector<int> prio;  // per op: urgency, lower first among the tasks of a wave
  int add_op(const std::vector<int>& d, int p = 0) { return add_op(d.data(), d.data() + d.size(), p); }
  int add_op(const int* b, const int* e, int p = 0) {
    flat.insert(flat.end(), b, e);
    off.push_back((int)flat.size());
    prio.push_back(p);
    return (int)off.size() - 2;
  }
  int size() const { return (int)off.size() - 1; }
  const int* begin(int i) const { return flat.data() + off[i]; }
  const int* end(int i) const { return flat.data() + off[i + 1]; }
  int prio_of(int i) const { return i < (int)prio.size() ? prio[i] : 0; }
  void release() {
    std::vector<int>(1, 0).swap(off);
    std::vector<int>().swap(flat);
    std::vector<int>().swap(prio);
  }
};

// A unit of work for one CTA of the persistent executor: kind, index of the
// operation in its per-kind array, the part (tile / chunk) of it, and the op id.
enum TaskKind { TK_GEMM = 0, TK_LU = 1, TK_TRUNC = 2, TK_COPY = 3, TK_REDUCE = 4, TK_ROWS = 5, TK_VPART = 6 };
struct Task {
  int kind, op, sub, nsub, id;
};

struct OpInfo {
  int ntasks, dep_begin, dep_end, pad;
};

// Device-resident schedule.  Tasks are listed wave by wave; CTA c takes the
// tasks of each wave whose position is c modulo the grid, in wave order, and
// starts a task once the completion counters of its op's producers are full.
struct DevSchedule {
  int nwaves = 0;
  int nops = 0;
  int64_t ntasks = 0;
  GemmOp* gemm = nullptr;
  LuOp* lu = nullptr;
  TruncOp* trunc = nullptr;
  CopyOp* copy = nullptr;
  ReduceOp* reduce = nullptr;
  RowsOp* rows = nullptr;
  VPartOp* vpart = nullptr;
  RowSrc* srcs = nullptr;
  Task* tasks = nullptr;
  int* wave_begin = nullptr;
  OpInfo* ops = nullptr;
  int2* deps = nullptr;      // dependency edges: (producer op, its task count)
  int* counters = nullptr;   // per op: finished tasks
  std::vector<Task> host_tasks;  // the task list in hand-out order (for tracing)
  int mode = 0;                  // executor mode (0 / FACTOR_MODE_2CTA: H-LU; SOLVE_MODE_LATENCY / _THROUGHPUT)
  unsigned long long wait_ns = 4000000000ull;  // limit of one dependency wait (ns; set at upload)
};

// One schedule among several uploaded side by side (independent problems):
// its waves, producer graph and row-task sources.
struct SchedPart {
  const std::vector<Wave>* waves;
  const OpGraph* graph;
  const std::vector<RowSrc>* srcs;
};
// Uploads the parts as one schedule: op ids shift by the ops of the parts
// before, wave k of every part joins wave k, row tasks' sources shift
// likewise; restage: re-plan row-task staging for `mode`.  copy_stream: copy
// with cudaMemcpyAsync on that (non-blocking) stream, so that an executor
// running meanwhile is not waited for; the call returns once the copies are done.
int upload_schedules(const std::vector<SchedPart>& parts, DevSchedule& S, std::vector<void*>& allocs, int mode,
                     bool restage, cudaStream_t copy_stream = nullptr);

// mode: executor mode of a solve schedule (ignored when the schedule holds H-LU operations).
int upload_schedule(const std::vector<Wave>& waves, const OpGraph& g, DevSchedule& S,
                    std::vector<void*>& allocs, const std::vector<RowSrc>* srcs = nullptr,
                    int mode = SOLVE_MODE_LATENCY);

// Run a schedule in one persistent cooperative launch (one CTA per SM).  Every
// wait is bounded in time: on expiry the kernel sets DEVERR_TIMEOUT in *d_err
// and returns instead of hanging.
// Kernel attributes and grid size of the executor for S (done once per kind;
// also done by run_schedule, but must precede any stream capture).
int prepare_executor(const DevSchedule& S);

constexpr int TRACE_STRIDE = 8;  // trace words per task
int run_schedule(const DevSchedule& S, int* d_err, cudaStream_t st,
                 unsigned long long* trace = nullptr);

int gemm_shape(int m, int n);  // tile shape of an m x n output
int gemm_tiles(int m, int n);  // tasks of an m x n output

}  // namespace hm
