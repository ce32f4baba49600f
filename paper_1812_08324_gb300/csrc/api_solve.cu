// C ABI: H-LU factorisation (hm_factor), H-triangular solves (hm_solve) and
// Crank-Nicolson steps with refinement (cn_step, cn_solve).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <tuple>
#include <mutex>
#include <thread>

#include "api_common.h"
#include "hinv.h"
#include "hlu_plan.h"
#include "hm_device.cuh"

using namespace hm;

namespace { bool g_batch_graphed = false; }

struct hm_factors {
  const hm_matrix* H = nullptr;
  double theta = 0.0;
  double alpha = 1.0;  // factors of alpha I + theta G
  int kf = 0;
  Arena arena;
  Arena tmp;                   // the H-LU's pooled temporaries, released once it has run
  std::vector<void*> allocs;
  DevSchedule solve;
  FactorLayout F;
  int* d_rank = nullptr;
  double* d_y = nullptr;      // solve input b (Morton order)
  double* d_sv = nullptr;     // forward result y, backward result z, two accumulators: 4 x N
  double* d_vec = nullptr;    // cn work vectors: 6 x N
  double* d_norm = nullptr;   // [|s|^2, |rhs|^2]
  int64_t lu_bytes = 0;
  int64_t fact_ops = 0;
  int fact_waves = 0, solve_waves = 0;
  std::vector<int> h_rank;
  int capped = 0;
  double fact_ms = 0.0;
  double fact_fma = 0.0;
  hm_batch* batch1 = nullptr;  // cn_solve's persistent one-problem batch (created on first use)
  // host copy of the solve schedule, for merging into batched solves
  std::vector<Wave> sw;
  std::vector<RowSrc> srcs;
  OpGraph sg;
  int solve_mode = HM_SOLVE_SUBST;
  HinvData* hinv = nullptr;    // hierarchical inverses of the factors (HM_SOLVE_HINV)
};

namespace hm {
namespace {

__global__ void axpy_kernel(int N, double a, const double* x, double* y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) y[i] += a * x[i];
}

__global__ void copy_vec_kernel(int N, const double* x, double* y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) y[i] = x[i];
}

// out[0] = |a|^2, out[1] = |b|^2 (one CTA, deterministic order)
__global__ void norms_kernel(int N, const double* a, const double* b, double* out) {
  __shared__ double sc[32];
  double sa = 0.0, sb = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    sa += a[i] * a[i];
    sb += b[i] * b[i];
  }
  sa = block_sum(sa, sc);
  sb = block_sum(sb, sc);
  if (threadIdx.x == 0) { out[0] = sa; out[1] = sb; }
}

int vgrid(int N) { return std::min((N + 255) / 256, 152 * 8); }

// Tracing (HM_PHASE_TRACE=1): run a schedule once recording every op's
// finish time and print the span, the time per op kind along the waves, and
// the ops that finished last.
void trace_schedule(const char* what, const std::vector<Wave>& waves, const OpGraph& graph,
                    const DevSchedule& S, int* d_err, cudaStream_t st) {
  const size_t nt = std::max<size_t>(S.host_tasks.size(), 1);
  unsigned long long* d_tr = nullptr;
  if (cudaMalloc(&d_tr, sizeof(unsigned long long) * TRACE_STRIDE * nt) != cudaSuccess) return;
  cudaMemsetAsync(d_tr, 0, sizeof(unsigned long long) * TRACE_STRIDE * nt, st);
  cudaStreamSynchronize(st);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  run_schedule(S, d_err, st, d_tr);
  cudaEventRecord(e1, st);
  cudaStreamSynchronize(st);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  std::vector<unsigned long long> tr(TRACE_STRIDE * nt);
  cudaMemcpy(tr.data(), d_tr, sizeof(unsigned long long) * TRACE_STRIDE * nt, cudaMemcpyDeviceToHost);
  cudaFree(d_tr);
  // op -> wave
  std::vector<int> wave_of(std::max(S.nops, 1), 0);
  for (size_t w = 0; w < waves.size(); ++w) {
    const Wave& W = waves[w];
    const std::vector<int>* ids[7] = {&W.gemm_id, &W.lu_id, &W.trunc_id, &W.copy_id, &W.reduce_id, &W.rows_id, &W.vpart_id};
    for (int k = 0; k < 7; ++k)
      for (int id : *ids[k]) wave_of[id] = (int)w;
  }
  if (const char* fn = std::getenv("HM_TRACE_FILE")) {
    // one line per task: task op wave kind parts cta grabbed ready finished gathered summed (ns) sm : the op's producers
    std::string path = std::string(fn) + "." + what + ".txt";
    FILE* f = fopen(path.c_str(), "a");
    if (f) {
      fprintf(f, "# run\n");
      for (size_t t = 0; t < S.host_tasks.size(); ++t) {
        const Task& T = S.host_tasks[t];
        const unsigned long long* q = &tr[TRACE_STRIDE * t];
        fprintf(f, "%zu %d %d %d %d %llu %llu %llu %llu %llu %llu %llu :", t, T.id, wave_of[T.id], T.kind, T.nsub, q[3],
                q[0], q[1], q[2], q[4], q[5], q[6]);
        if (T.id < graph.size())
          for (const int* d = graph.begin(T.id); d != graph.end(T.id); ++d) fprintf(f, " %d", *d);
        fprintf(f, "\n");
      }
      fclose(f);
    }
    // one line per op: id kind dims (gemm m n k; lu m; trunc K kf; copy m n; reduce m n parts; rows nr; vpart len kf)
    FILE* g = fopen((std::string(fn) + "." + what + ".ops.txt").c_str(), "w");
    if (g) {
      for (const Wave& W : waves) {
        for (size_t j = 0; j < W.gemm.size(); ++j)
          fprintf(g, "%d 0 %d %d %d\n", W.gemm_id[j], W.gemm[j].m, W.gemm[j].n, W.gemm[j].k);
        for (size_t j = 0; j < W.lu.size(); ++j) fprintf(g, "%d 1 %d 0 0\n", W.lu_id[j], W.lu[j].m);
        for (size_t j = 0; j < W.trunc.size(); ++j) fprintf(g, "%d 2 %d %d 0\n", W.trunc_id[j], W.trunc[j].K, W.trunc[j].kf);
        for (size_t j = 0; j < W.copy.size(); ++j) fprintf(g, "%d 3 %d %d 0\n", W.copy_id[j], W.copy[j].m, W.copy[j].n);
        for (size_t j = 0; j < W.reduce.size(); ++j)
          fprintf(g, "%d 4 %d %d %d\n", W.reduce_id[j], W.reduce[j].m, W.reduce[j].n, W.reduce[j].nparts);
        for (size_t j = 0; j < W.rows.size(); ++j) fprintf(g, "%d 5 %d 0 0\n", W.rows_id[j], W.rows[j].nr);
        for (size_t j = 0; j < W.vpart.size(); ++j) fprintf(g, "%d 6 %d %d 0\n", W.vpart_id[j], W.vpart[j].len, W.vpart[j].kf);
      }
      fclose(g);
    }
  }
  unsigned long long t0 = ~0ull, t1 = 0;
  for (size_t t = 0; t < S.host_tasks.size(); ++t)
    if (tr[TRACE_STRIDE * t + 2]) { t0 = std::min(t0, tr[TRACE_STRIDE * t]); t1 = std::max(t1, tr[TRACE_STRIDE * t + 2]); }
  // busy time per kind (producers-ready to finished), summed over tasks
  const char* names[7] = {"gemm", "lu", "trunc", "copy", "reduce", "rows", "vpart"};
  double busy[7] = {0, 0, 0, 0, 0, 0, 0};
  int cnt[7] = {0, 0, 0, 0, 0, 0, 0};
  for (size_t t = 0; t < S.host_tasks.size(); ++t) {
    const int k = S.host_tasks[t].kind;
    if (k >= 0 && k < 7 && tr[TRACE_STRIDE * t + 2] > tr[TRACE_STRIDE * t + 1]) {
      busy[k] += (double)(tr[TRACE_STRIDE * t + 2] - tr[TRACE_STRIDE * t + 1]) * 1e-3;
      ++cnt[k];
    }
  }
  fprintf(stderr, "[trace] %s: %d waves, %d ops, %zu tasks, kernel %.3f ms, task span %.3f ms\n", what, S.nwaves,
          S.nops, S.host_tasks.size(), ms, (double)(t1 - t0) * 1e-6);
  for (int k = 0; k < 7; ++k)
    if (cnt[k] > 0)
      fprintf(stderr, "[trace]   %-6s %8d tasks, busy %10.1f us (%.2f us per task)\n", names[k], cnt[k], busy[k],
              busy[k] / cnt[k]);
}

// z = (LU)^{-1} b on Morton-order vectors (b may equal z)
int solve_morton(const hm_factors* F, const double* b, double* z, cudaStream_t st) {
  if (F->hinv) return hinv_solve(*F->hinv, b, z, st);
  const int N = F->H->plan.N;
  count_launches(2);
  copy_vec_kernel<<<vgrid(N), 256, 0, st>>>(N, b, F->d_y);
  HM_TRY(run_schedule(F->solve, F->H->d_err, st));
  copy_vec_kernel<<<vgrid(N), 256, 0, st>>>(N, F->d_sv + (size_t)N, z);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

// w = 2 u + theta (f0 + f1)   (f0, f1 may be null)
__global__ void cn_w_kernel(int N, const double* u, double th, const double* f0, const double* f1, double* w) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double v = 2.0 * u[i];
    if (f0 || f1) v += th * ((f0 ? f0[i] : 0.0) + (f1 ? f1[i] : 0.0));
    w[i] = v;
  }
}

// y = y - x
__global__ void sub_kernel(int N, const double* x, double* y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) y[i] = y[i] - x[i];
}

// One CN step on Morton-order vectors: u1 = CN(u0) with forcing f0, f1 (may be
// null), M = I - theta G, R = refine_max sweeps (the H-LU as preconditioner,
// the FP64 H-matvec residual setting the accuracy).
//  HM_CN_IDENTITY: I + theta G = 2I - M, so the scheme reads M v = w for
//    v = u^n + u^{n+1}, w = 2u + theta (f^n + f^{n+1}): v = (LU)^{-1} w, R sweeps
//    v += (LU)^{-1} (w - M v), u1 = v - u.  No H-matvec unless R > 0.
//  HM_CN_LITERAL: rhs = u + theta G u + theta (f^n + f^{n+1}) by the H-matvec
//    (Eq. scheme as written), u1 = (LU)^{-1} rhs, R sweeps u1 += (LU)^{-1}
//    (rhs - M u1).
int cn_step_morton(const hm_matrix* H, hm_factors* F, double dt, const double* u0,
                   const double* f0, const double* f1, double* u1, cudaStream_t st) {
  const int N = H->plan.N;
  const double th = 0.5 * dt;
  double* w = F->d_vec;  // right-hand side of M x = w: x = v (identity) or u1 (literal)
  double* s = F->d_vec + (size_t)N;
  const int sweeps = H->opts.refine_max;
  const bool literal = H->opts.cn_form == HM_CN_LITERAL;
  if (literal) {
    HM_TRY(hm_matvec_morton(H, 1.0, th, u0, th, f0, f1, nullptr, w, st));
  } else {
    count_launches(1);
    cn_w_kernel<<<vgrid(N), 256, 0, st>>>(N, u0, th, f0, f1, w);
  }
  HM_TRY(solve_morton(F, w, u1, st));  // x, kept in u1
  for (int it = 0; it < sweeps; ++it) {
    // s = w - (x - theta G x)
    HM_TRY(hm_matvec_morton(H, -1.0, th, u1, 0.0, nullptr, nullptr, w, s, st));
    if (it == sweeps - 1) {
      count_launches(1);
      norms_kernel<<<1, 1024, 0, st>>>(N, s, w, F->d_norm);
    }
    HM_TRY(solve_morton(F, s, s, st));
    count_launches(1);
    axpy_kernel<<<vgrid(N), 256, 0, st>>>(N, 1.0, s, u1);
  }
  if (literal) return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
  count_launches(1);
  sub_kernel<<<vgrid(N), 256, 0, st>>>(N, u0, u1);  // u1 = v - u0
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

// ---- batched vector operations: y = x (mode 0), y += a x (mode 1), y = 2 x
// (mode 2) or y = x - y (mode 3) for many vectors in one launch, 2048 elements
// per CTA

struct VecJob {
  const double* x;
  double* y;
  double a;
  int n;
  int mode;
};

__device__ __forceinline__ int batch_job_of(const int* off, int count, int b) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

constexpr int VEC_CHUNK = 2048;

__global__ void vec_batch_kernel(const VecJob* jobs, const int* off, int count) {
  const int j = batch_job_of(off, count, blockIdx.x);
  const VecJob J = jobs[j];
  const int i0 = (blockIdx.x - off[j]) * VEC_CHUNK, i1 = min(J.n, i0 + VEC_CHUNK);
  if (J.mode == 0) {
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) J.y[i] = J.x[i];
  } else if (J.mode == 1) {
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) J.y[i] += J.a * J.x[i];
  } else if (J.mode == 2) {
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) J.y[i] = 2.0 * J.x[i];
  } else {
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) J.y[i] = J.x[i] - J.y[i];
  }
}

// Device copy of a job table plus block offsets; freed by the owner.
template <class Job>
struct DevJobs {
  Job* jobs = nullptr;
  int* off = nullptr;
  int total = 0;
  int count = 0;
};

template <class Job, class Blocks>
int upload_jobs(const std::vector<Job>& h, Blocks blocks, DevJobs<Job>& d, std::vector<void*>& allocs) {
  std::vector<int> off(h.size() + 1, 0);
  for (size_t i = 0; i < h.size(); ++i) off[i + 1] = off[i] + blocks(h[i]);
  d.count = (int)h.size();
  d.total = off.back();
  if (cudaMalloc((void**)&d.jobs, sizeof(Job) * std::max<size_t>(h.size(), 1)) != cudaSuccess) return HM_ERR_OOM;
  allocs.push_back(d.jobs);
  if (cudaMalloc((void**)&d.off, sizeof(int) * off.size()) != cudaSuccess) return HM_ERR_OOM;
  allocs.push_back(d.off);
  if (!h.empty() && cudaMemcpy(d.jobs, h.data(), sizeof(Job) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return HM_ERR_CUDA;
  if (cudaMemcpy(d.off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return HM_ERR_CUDA;
  return HM_OK;
}

int launch_vec_batch(const DevJobs<VecJob>& d, cudaStream_t st) {
  if (d.total == 0) return HM_OK;
  count_launches(1);
  vec_batch_kernel<<<d.total, 256, 0, st>>>(d.jobs, d.off, d.count);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

// Batched H-matvec table: per job its plan, per launch kind its block offsets.
int upload_mv_batch(const std::vector<MvJob>& h, MvBatch& B, std::vector<void*>& allocs) {
  DevJobs<MvJob> d0, d1, d2;
  HM_TRY(upload_jobs(h, [](const MvJob& J) { return J.P.nvt > 0 ? J.P.nvt : 0; }, d0, allocs));
  HM_TRY(upload_jobs(h, [](const MvJob& J) { return J.P.nvt > 0 ? J.P.nlr : 0; }, d1, allocs));
  HM_TRY(upload_jobs(h, [](const MvJob& J) { return J.P.nchunk; }, d2, allocs));
  B.jobs = d0.jobs;
  B.off[0] = d0.off;
  B.off[1] = d1.off;
  B.off[2] = d2.off;
  B.total[0] = d0.total;
  B.total[1] = d1.total;
  B.total[2] = d2.total;
  B.count = (int)h.size();
  return HM_OK;
}

// Batched hierarchical-inverse products: per job its blocks of the two launches.
int upload_hinv_batch(const std::vector<HinvJob>& h, HinvBatch& B, std::vector<void*>& allocs) {
  if (h.empty()) return HM_OK;
  DevJobs<HinvJob> d0, d1;
  HM_TRY(upload_jobs(h, [](const HinvJob& J) { return J.A.ntch; }, d0, allocs));
  HM_TRY(upload_jobs(h, [](const HinvJob& J) { return J.A.nrch; }, d1, allocs));
  B.jobs = d0.jobs;
  B.off[0] = d0.off;
  B.off[1] = d1.off;
  B.total[0] = d0.total;
  B.total[1] = d1.total;
  B.count = (int)h.size();
  B.prec = h[0].A.prec;
  for (const HinvJob& J : h)
    if (J.A.prec != B.prec) B.prec = -1;
  return HM_OK;
}

// ---- factorisation in phases (shared by hm_factor and hm_factor_batch)

struct FactorJob {
  const hm_matrix* H = nullptr;
  hm_factors* F = nullptr;
  HluBuild hb;
  int status = HM_OK;
  std::string err;
};

void factor_discard(FactorJob& J) {
  if (!J.F) return;
  if (J.F->hinv) {
    J.F->hinv->release();
    delete J.F->hinv;
  }
  for (void* p : J.F->allocs) cudaFree(p);
  J.F->arena.release();
  J.F->tmp.release();
  delete J.F;
  J.F = nullptr;
}

// Rank cap, per-factor vectors and the copy of the ACA ranks (main thread).
int factor_alloc(FactorJob& J, const hm_matrix* H, double theta, cudaStream_t st) {
  if (!std::isfinite(theta)) { set_error("theta must be finite"); return HM_ERR_ARG; }
  int maxr = 0;
  for (int r : H->h_rank) maxr = std::max(maxr, r);
  int kf = std::max(H->opts.lu_max_rank, maxr);
  if (kf > TRUNC_MAXK / 2) {
    set_error("factor rank cap " + std::to_string(kf) + " exceeds " + std::to_string(TRUNC_MAXK / 2));
    return HM_ERR_RANK_CAP;
  }
  J.H = H;
  J.F = new hm_factors();
  hm_factors* F = J.F;
  F->H = H;
  F->theta = theta;
  F->solve_mode = solve_mode(H->prob, H->opts);
  F->kf = std::max(kf, 1);
  const int nlr = (int)H->h_ld.size();
  const int N = H->plan.N;
  auto alloc = [&](void** p, size_t bytes) {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) return HM_ERR_OOM;
    F->allocs.push_back(*p);
    return HM_OK;
  };
  int s;
  if ((s = alloc((void**)&F->d_rank, sizeof(int) * std::max(nlr, 1))) != HM_OK) return s;
  if ((s = alloc((void**)&F->d_y, sizeof(double) * N)) != HM_OK) return s;
  if ((s = alloc((void**)&F->d_sv, sizeof(double) * 4 * (size_t)N)) != HM_OK) return s;
  if ((s = alloc((void**)&F->d_vec, sizeof(double) * 6 * (size_t)N)) != HM_OK) return s;
  if ((s = alloc((void**)&F->d_norm, sizeof(double) * 4)) != HM_OK) return s;
  if (nlr && cudaMemcpyAsync(F->d_rank, H->d_rank, sizeof(int) * nlr, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return HM_ERR_CUDA;
  if (cudaMemsetAsync(F->d_norm, 0, sizeof(double) * 4, st) != cudaSuccess) return HM_ERR_CUDA;
  return HM_OK;
}

// H-LU planning (host; safe to run for different jobs on different threads).
void factor_plan(FactorJob& J) {
  const hm_matrix* H = J.H;
  hm_factors* F = J.F;
  J.status = plan_hlu(H->plan, H->h_dd, H->d_D, H->h_ld, H->d_U, H->d_V, F->kf, F->theta, H->opts.lu_tol,
                      F->d_rank, F->arena, J.hb, F->alpha, H->opts.solve_block, F->solve_mode == HM_SOLVE_SUBST,
                      &F->tmp);
  if (J.status != HM_OK) { J.err = J.hb.err; return; }
  F->fact_ops = J.hb.ops;
  F->fact_waves = (int)J.hb.waves.size();
  F->F = J.hb.F;
}

// Solve planning once the factor ranks are on the host (thread-safe per job).
void factor_plan_solve(FactorJob& J) {
  const hm_matrix* H = J.H;
  hm_factors* F = J.F;
  const int N = H->plan.N;
  SolveVectors sv{F->d_y, F->d_sv, F->d_sv + (size_t)N, F->d_sv + 2 * (size_t)N, F->d_sv + 3 * (size_t)N};
  J.status = plan_solve(H->plan, H->h_dd, H->h_ld, F->F, &F->h_rank, sv, F->arena, F->sw, F->srcs, F->sg);
  if (J.status != HM_OK) { J.err = "solve planning failed"; return; }
  F->solve_waves = (int)F->sw.size();
  // bytes the two sweeps read: leaf inverses, off-diagonal dense blocks, low-rank factors
  int64_t b = 0;
  for (size_t d = 0; d < H->h_dd.size(); ++d) {
    const DenseDesc& D = H->h_dd[d];
    b += (int64_t)D.m * D.n * (D.r0 == D.c0 ? 2 : 1);
  }
  for (size_t q = 0; q < H->h_ld.size(); ++q) b += (int64_t)(H->h_ld[q].m + H->h_ld[q].n) * F->kf;
  F->lu_bytes = 8 * b;
}

// Run fn(0..n-1) on up to hardware_concurrency host threads.
template <class Fn>
void parallel_for(int n, Fn fn) {
  const int nt = std::max(1, std::min<int>(n, (int)std::thread::hardware_concurrency()));
  if (nt <= 1) {
    for (int i = 0; i < n; ++i) fn(i);
    return;
  }
  std::atomic<int> next{0};
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t)
    pool.emplace_back([&]() {
      for (int i = next++; i < n; i = next++) fn(i);
    });
  for (auto& th : pool) th.join();
}


}  // namespace
}  // namespace hm

// A set of problems stepped together (hm_batch_create): the merged solve
// schedule, the batched H-matvec and vector job tables, the batch-owned
// Morton-order states and the recorded CUDA graph of one step.
struct hm_batch {
  std::vector<const hm_matrix*> H;
  std::vector<const hm_factors*> F;
  std::vector<double*> state;
  int refine = 0;
  bool literal = false;        // HM_CN_LITERAL (all problems share cn_form)
  DevSchedule sched;           // merged substitution schedule of the HM_SOLVE_SUBST problems
  hm::HinvBatch hL, hU;        // the HM_SOLVE_HINV problems: L^{-1}, then U^{-1} of every one
  hm::MvBatch A{}, B{};
  hm::DevJobs<hm::VecJob> rhs_in, w_in, w_solve, s_in, z_out, z_u1, z_v, u1_add, u1_out, u1_copy;
  std::vector<void*> allocs;
  cudaStream_t cs = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int64_t per_step = 0;
};

namespace hm {
namespace {

// One CN step of every problem of the batch (stream-ordered launches only,
// so that it can be recorded as a graph).
// The solves of every problem: z = (LU)^{-1} y from each factor's input
// vector y to its output z (the substitution schedule, the inverses' products).
int batch_solve(hm_batch* B, cudaStream_t cs) {
  HM_TRY(run_schedule(B->sched, B->H[0]->d_err, cs));
  HM_TRY(launch_hinv_batch(B->hL, cs));
  return launch_hinv_batch(B->hU, cs);
}

int batch_one_step(hm_batch* B, cudaStream_t cs) {
  if (B->literal) {
    // rhs = x + th G x, u1 = (LU)^{-1} rhs, sweeps u1 += (LU)^{-1} (rhs - M u1)
    HM_TRY(launch_matvec_batch(B->A, cs));
    HM_TRY(launch_vec_batch(B->rhs_in, cs));
    HM_TRY(batch_solve(B, cs));
    if (B->refine == 0) return launch_vec_batch(B->z_out, cs);
    HM_TRY(launch_vec_batch(B->z_u1, cs));
  } else if (B->refine == 0) {
    // the solve's input 2 x, then x = z - x with z = (LU)^{-1} (2 x) (the
    // hierarchical-inverse members do both inside their products)
    HM_TRY(launch_vec_batch(B->w_solve, cs));
    HM_TRY(batch_solve(B, cs));
    return launch_vec_batch(B->z_v, cs);
  } else {
    // w = 2 x (kept in rhs and given to the solve), v = (LU)^{-1} w in u1
    HM_TRY(launch_vec_batch(B->w_in, cs));
    HM_TRY(batch_solve(B, cs));
    HM_TRY(launch_vec_batch(B->z_u1, cs));
  }
  for (int it = 0; it < B->refine; ++it) {
    HM_TRY(launch_matvec_batch(B->B, cs));
    HM_TRY(launch_vec_batch(B->s_in, cs));
    HM_TRY(batch_solve(B, cs));
    HM_TRY(launch_vec_batch(B->u1_add, cs));
  }
  // identity: x = v - x; literal: x = u1
  return launch_vec_batch(B->literal ? B->u1_copy : B->u1_out, cs);
}

}  // namespace
}  // namespace hm

namespace hm {
namespace {
int factor_batch_impl(const hm_matrix* const* Hs, const double* alphas, const double* thetas, int count,
                      void* stream, hm_factors** out);
}
}  // namespace hm

extern "C" {

int hm_factor(const hm_matrix* H, double theta, void* stream, hm_factors** out) {
  return hm_factor_batch(&H, &theta, 1, stream, out);
}

int hm_factor_shifted(const hm_matrix* H, double alpha, double theta, void* stream, hm_factors** out) {
  if (!std::isfinite(alpha)) { set_error("alpha must be finite"); return HM_ERR_ARG; }
  return factor_batch_impl(&H, &alpha, &theta, 1, stream, out);
}

int hm_factor_batch(const hm_matrix* const* Hs, const double* thetas, int count, void* stream,
                    hm_factors** out) {
  return factor_batch_impl(Hs, nullptr, thetas, count, stream, out);
}

}  // extern "C"

namespace hm {
namespace {

#ifndef HM_SLICE_OPS
#define HM_SLICE_OPS (1 << 20)  // at most this many ops (whole planner chunks, at least one) per executor launch
#endif
#ifndef HM_CHUNK_OPS
#define HM_CHUNK_OPS 49152  // ops per planner chunk (build-time tuning parameter; 1D N = 65536: 131072 -> 49152 gave 231 -> 213 ms, the device waits less for each slice's merge and upload)
#endif

// dst += src with op ids shifted by -base
void append_rebased(Wave& dst, const Wave& src, int base) {
  auto cat = [base](auto& d, const auto& s, std::vector<int>& di, const std::vector<int>& si) {
    d.insert(d.end(), s.begin(), s.end());
    for (int id : si) di.push_back(id - base);
  };
  cat(dst.gemm, src.gemm, dst.gemm_id, src.gemm_id);
  cat(dst.lu, src.lu, dst.lu_id, src.lu_id);
  cat(dst.trunc, src.trunc, dst.trunc_id, src.trunc_id);
  cat(dst.copy, src.copy, dst.copy_id, src.copy_id);
  cat(dst.reduce, src.reduce, dst.reduce_id, src.reduce_id);
  cat(dst.rows, src.rows, dst.rows_id, src.rows_id);
  cat(dst.vpart, src.vpart, dst.vpart_id, src.vpart_id);
}

// Consecutive slices of one problem as one schedule part: ids relative to the
// first slice, producers in earlier launches dropped (they have finished: the
// launches run in stream order), the slices' waves merged in global wave order.
int merge_chunks(std::vector<HluChunk>& ch, std::vector<Wave>& waves, OpGraph& graph) {
  const int base = ch.front().first;
  int expect = base;
  std::vector<int> wv;
  for (const HluChunk& c : ch) {
    if (c.first != expect) return HM_ERR_ARG;
    expect += c.graph.size();
    wv.insert(wv.end(), c.wave_idx.begin(), c.wave_idx.end());
  }
  std::sort(wv.begin(), wv.end());
  wv.erase(std::unique(wv.begin(), wv.end()), wv.end());
  waves.assign(wv.size(), Wave());
  std::vector<int> d;
  for (HluChunk& c : ch) {
    for (size_t k = 0; k < c.wave_idx.size(); ++k) {
      const size_t lw = std::lower_bound(wv.begin(), wv.end(), c.wave_idx[k]) - wv.begin();
      append_rebased(waves[lw], c.waves[k], base);
    }
    for (int j = 0; j < c.graph.size(); ++j) {
      d.clear();
      for (const int* p = c.graph.begin(j); p != c.graph.end(j); ++p)
        if (*p >= base) d.push_back(*p - base);
      graph.add_op(d, c.graph.prio_of(j));
    }
    std::vector<Wave>().swap(c.waves);
    c.graph.release();
  }
  return HM_OK;
}

// Plans the H-LU again with a fake arena, handing it out in slices of
// `chunk` ops, merges consecutive slices in groups of 1, 2, 3, ... and checks
// each group against the one-piece plan `ref`: the same ops in the same wave
// order, with exactly the producers of `ref` that lie inside the group.
bool check_streamed_plan(const Plan& P, const std::vector<DenseDesc>& dd, const std::vector<LRDesc>& ld, int kf,
                         double theta, double lu_tol, int chunk, const HluBuild& ref) {
  Arena A;
  A.fake = true;
  std::vector<HluChunk> chunks;
  HluBuild hb;
  hb.chunk_ops = chunk;
  hb.sink = [&](HluChunk&& c) { chunks.push_back(std::move(c)); };
  // fake H storage (addresses only) sized from the block layout
  int64_t dp = 0;
  for (const DenseDesc& D : dd) dp = std::max<int64_t>(dp, D.off + (int64_t)D.m * D.ld);
  double* fD = A.alloc(std::max<int64_t>(dp, 1));
  int64_t uo = 0, vo = 0;
  for (const LRDesc& L : ld) {
    uo = std::max<int64_t>(uo, L.uoff + (int64_t)L.m * L.kcap);
    vo = std::max<int64_t>(vo, L.voff + (int64_t)L.n * L.kcap);
  }
  double* fU = A.alloc(std::max<int64_t>(uo, 1));
  double* fV = A.alloc(std::max<int64_t>(vo, 1));
  int* frank = (int*)A.alloc((int64_t)ld.size() / 2 + 1);
  if (plan_hlu(P, dd, fD, ld, fU, fV, kf, theta, lu_tol, frank, A, hb) != HM_OK) {
    set_error("streamed planning failed");
    return false;
  }
  const int nops = ref.graph.size();
  // global wave of every op in the one-piece plan
  std::vector<int> wave_of(nops, -1);
  for (size_t w = 0; w < ref.waves.size(); ++w) {
    const Wave& W = ref.waves[w];
    for (const std::vector<int>* ids : {&W.gemm_id, &W.lu_id, &W.trunc_id, &W.copy_id, &W.reduce_id})
      for (int id : *ids) wave_of[id] = (int)w;
  }
  size_t ci = 0;
  int next = 0, group = 1;
  std::vector<int> d;
  while (ci < chunks.size()) {
    std::vector<HluChunk> grp;
    for (int g = 0; g < group && ci < chunks.size(); ++g) grp.push_back(std::move(chunks[ci++]));
    ++group;
    const int base = grp.front().first;
    if (base != next) { set_error("streamed slices are not consecutive"); return false; }
    std::vector<Wave> waves;
    OpGraph graph;
    if (merge_chunks(grp, waves, graph) != HM_OK) { set_error("slices failed to merge"); return false; }
    next = base + graph.size();
    if (next > nops) { set_error("streamed plan has more ops than the one-piece plan"); return false; }
    for (int i = 0; i < graph.size(); ++i) {
      d.clear();
      for (const int* p = ref.graph.begin(base + i); p != ref.graph.end(base + i); ++p)
        if (*p >= base) d.push_back(*p - base);
      if (!std::equal(d.begin(), d.end(), graph.begin(i), graph.end(i)) || (int)d.size() != graph.end(i) - graph.begin(i)) {
        set_error("producers of op " + std::to_string(base + i) + " differ in the streamed plan");
        return false;
      }
    }
    int last = -1;
    for (const Wave& W : waves) {
      int wmin = 1 << 30, wmax = -1;
      for (const std::vector<int>* ids : {&W.gemm_id, &W.lu_id, &W.trunc_id, &W.copy_id, &W.reduce_id})
        for (int id : *ids) {
          const int gw = wave_of[base + id];
          wmin = std::min(wmin, gw);
          wmax = std::max(wmax, gw);
        }
      if (wmax < 0) continue;
      if (wmin != wmax || wmin <= last) { set_error("wave order differs in the streamed plan"); return false; }
      last = wmin;
    }
  }
  if (next != nops) { set_error("streamed plan misses ops"); return false; }
  return true;
}

// Streamed planning that runs out of (fake) memory at `limit` bytes: every op
// handed out before the failure must have all its operands inside the
// allocations that succeeded (no op with a missing operand reaches a launch).
bool check_streamed_failure(const Plan& P, const std::vector<DenseDesc>& dd, const std::vector<LRDesc>& ld,
                            int kf, double theta, double lu_tol, int chunk, int64_t limit) {
  Arena A;
  A.fake = true;
  A.fake_limit = limit;
  std::vector<HluChunk> chunks;
  HluBuild hb;
  hb.chunk_ops = chunk;
  hb.sink = [&](HluChunk&& c) { chunks.push_back(std::move(c)); };
  int64_t dp = 0, uo = 0, vo = 0;
  for (const DenseDesc& D : dd) dp = std::max<int64_t>(dp, D.off + (int64_t)D.m * D.ld);
  for (const LRDesc& L : ld) {
    uo = std::max<int64_t>(uo, L.uoff + (int64_t)L.m * L.kcap);
    vo = std::max<int64_t>(vo, L.voff + (int64_t)L.n * L.kcap);
  }
  double* fD = A.alloc(std::max<int64_t>(dp, 1));
  double* fU = A.alloc(std::max<int64_t>(uo, 1));
  double* fV = A.alloc(std::max<int64_t>(vo, 1));
  int* frank = (int*)A.alloc((int64_t)ld.size() / 2 + 1);
  if (plan_hlu(P, dd, fD, ld, fU, fV, kf, theta, lu_tol, frank, A, hb) != HM_ERR_OOM) {
    set_error("streamed planning did not report the injected allocation failure");
    return false;
  }
  std::string first;
  for (const HluChunk& c : chunks)
    if (check_spans(c.waves, A.ranges, first) != 0) {
      set_error("a streamed slice handed out after an allocation failure has an operand outside memory: " + first);
      return false;
    }
  return true;
}

// HM_PLAN_HIST (hm_plan_factor): the executor's tasks of an H-LU schedule by
// op kind (32 x 32 GEMM tiles), and the GEMMs by output and inner size
// rounded up to powers of two, on stderr
void plan_histogram(const std::vector<Wave>& waves) {
  auto p2 = [](int v) { int b = 1; while (b < v) b <<= 1; return b; };
  std::map<std::tuple<int, int, int>, std::pair<int64_t, int64_t>> gem;  // (m, n, k) -> ops, tasks
  int64_t ops[5] = {0, 0, 0, 0, 0}, tasks[5] = {0, 0, 0, 0, 0};
  double fma = 0.0;
  for (const Wave& W : waves) {
    for (const GemmOp& o : W.gemm) {
      const int t = gemm_tiles(o.m, o.n);
      auto& e = gem[std::make_tuple(p2(o.m), p2(o.n), p2(o.k))];
      e.first += 1;
      e.second += t;
      ops[0] += 1;
      tasks[0] += t;
      fma += (double)o.m * o.n * o.k;
    }
    ops[1] += (int64_t)W.lu.size();
    tasks[1] += (int64_t)W.lu.size();
    ops[2] += (int64_t)W.trunc.size();
    tasks[2] += (int64_t)W.trunc.size();
    for (const CopyOp& o : W.copy) {
      ops[3] += 1;
      tasks[3] += std::max<int64_t>(1, std::min<int64_t>(64, (int64_t)o.m * o.n / 2048));
    }
    for (const ReduceOp& o : W.reduce) {
      ops[4] += 1;
      tasks[4] += std::max<int64_t>(1, std::min<int64_t>(64, (int64_t)o.m * o.n * std::max(o.nparts, 1) / 2048));
    }
  }
  const char* names[5] = {"gemm", "lu", "trunc", "copy", "reduce"};
  for (int k = 0; k < 5; ++k)
    fprintf(stderr, "[plan] %-6s %10lld ops %11lld tasks\n", names[k], (long long)ops[k], (long long)tasks[k]);
  fprintf(stderr, "[plan] gemm FMAs %.3e (%.0f per task)\n", fma, fma / std::max<int64_t>(tasks[0], 1));
  std::vector<std::pair<int64_t, std::tuple<int, int, int>>> by;
  for (auto& kv : gem) by.push_back({kv.second.second, kv.first});
  std::sort(by.rbegin(), by.rend());
  for (size_t i = 0; i < by.size() && i < 24; ++i) {
    const auto& k = by[i].second;
    const auto& e = gem[k];
    fprintf(stderr, "[plan] gemm m<=%-5d n<=%-5d k<=%-5d %9lld ops %10lld tasks\n", std::get<0>(k), std::get<1>(k),
            std::get<2>(k), (long long)e.first, (long long)e.second);
  }
}

// H-LU planning streamed into execution: the planners (one host thread per
// problem, up to the core count) hand finished slices of their operation
// lists over; the main thread uploads whatever slices are ready (copies on a
// non-blocking stream, so the running launch is not waited for) and launches
// them as the next executor run on `st`.  Planning of later slices overlaps
// the execution of earlier ones.  e0/e1 bracket the launches.
int factor_streamed(std::vector<FactorJob>& jobs, cudaStream_t st, int* d_err, cudaEvent_t e0, cudaEvent_t e1,
                    std::vector<void*>& allocs, int& launches) {
  const int count = (int)jobs.size();
  std::mutex m;
  std::condition_variable cv;
  std::vector<std::deque<HluChunk>> ready(count);
  int finished = 0;
  const char* co = std::getenv("HM_CHUNK_OPS");  // slice size override (tests)
  const int64_t chunk = co && std::atoll(co) > 0 ? std::atoll(co) : HM_CHUNK_OPS;
  const char* so = std::getenv("HM_SLICE_OPS");
  const int64_t slice_cap = so && std::atoll(so) > 0 ? std::atoll(so) : HM_SLICE_OPS;
  for (int i = 0; i < count; ++i) {
    jobs[i].hb.chunk_ops = chunk;
    jobs[i].hb.sink = [&, i](HluChunk&& c) {
      std::lock_guard<std::mutex> g(m);
      ready[i].push_back(std::move(c));
      cv.notify_one();
    };
  }
  std::atomic<int> next{0};
  const int nt = std::max(1, std::min<int>(count, (int)std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t)
    pool.emplace_back([&]() {
      for (int i = next++; i < count; i = next++) {
        factor_plan(jobs[i]);
        std::lock_guard<std::mutex> g(m);
        ++finished;
        cv.notify_one();
      }
    });
  cudaStream_t cs = nullptr;
  int s = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess ? HM_OK : HM_ERR_CUDA;
  bool started = false;
  launches = 0;
  // HM_TIME_PHASES: per slice, when it was handed to the device (host clock)
  // and when its launch ended (device clock), both from the first launch
  const bool timing = std::getenv("HM_TIME_PHASES") != nullptr;
  struct SliceTime { int64_t tasks; double host_ms; cudaEvent_t end; };
  std::vector<SliceTime> slices;
  const auto t_host0 = std::chrono::steady_clock::now();
  // At most two slices in flight (one running, one queued behind it): while
  // the device is behind, the planners' chunks pile up and are merged into
  // one larger slice (fewer executor drains); while the planners are behind,
  // each chunk goes out as soon as it is ready.
  std::deque<cudaEvent_t> inflight;
  while (s == HM_OK) {
    while (inflight.size() >= 2) {
      cudaEventSynchronize(inflight.front());
      cudaEventDestroy(inflight.front());
      inflight.pop_front();
    }
    std::vector<std::vector<HluChunk>> got(count);
    bool any = false, done = false;
    {
      std::unique_lock<std::mutex> lk(m);
      cv.wait(lk, [&] {
        if (finished == count) return true;
        for (const auto& q : ready)
          if (!q.empty()) return true;
        return false;
      });
      // a prefix of every problem's queue, round robin over the problems,
      // up to slice_cap ops: a backlog goes out as several launches, so the
      // device starts on its first part while the host merges the next
      int64_t taken = 0;
      for (bool more = true; more && taken < slice_cap;) {
        more = false;
        for (int i = 0; i < count && taken < slice_cap; ++i) {
          if (ready[i].empty()) continue;
          taken += ready[i].front().graph.size();
          got[i].push_back(std::move(ready[i].front()));
          ready[i].pop_front();
          any = more = true;
        }
      }
      bool left = false;
      for (const auto& q : ready) left = left || !q.empty();
      done = finished == count && !left;
    }
    if (!any) {
      if (done) break;
      continue;
    }
    const auto t_m0 = std::chrono::steady_clock::now();
    std::vector<std::vector<Wave>> pw(count);
    std::vector<OpGraph> pg(count);
    std::vector<SchedPart> parts;
    std::vector<int> idx;  // the problems in this slice, merged in parallel
    for (int i = 0; i < count; ++i)
      if (!got[i].empty()) idx.push_back(i);
    std::vector<int> ms(idx.size(), HM_OK);
    parallel_for((int)idx.size(), [&](int k) { ms[k] = merge_chunks(got[idx[k]], pw[idx[k]], pg[idx[k]]); });
    for (size_t k = 0; k < idx.size(); ++k) {
      if (ms[k] != HM_OK) s = ms[k];
      parts.push_back(SchedPart{&pw[idx[k]], &pg[idx[k]], nullptr});
    }
    if (s != HM_OK) break;
    const auto t_m1 = std::chrono::steady_clock::now();
    DevSchedule S;
    s = upload_schedules(parts, S, allocs, 0, false, cs);
    if (s != HM_OK) break;
    const auto t_m2 = std::chrono::steady_clock::now();
    if (timing)
      fprintf(stderr, "[factor slices] merged in %.1f ms, uploaded in %.1f ms\n",
              std::chrono::duration<double, std::milli>(t_m1 - t_m0).count(),
              std::chrono::duration<double, std::milli>(t_m2 - t_m1).count());
    if (!started) {
      cudaEventRecord(e0, st);
      started = true;
    }
    s = run_schedule(S, d_err, st);
    ++launches;
    {
      cudaEvent_t ev = nullptr;
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(ev, st);
        inflight.push_back(ev);
      }
    }
    if (timing) {
      SliceTime T{S.ntasks, std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_host0).count(),
                  nullptr};
      cudaEventCreate(&T.end);
      cudaEventRecord(T.end, st);
      slices.push_back(T);
    }
  }
  for (cudaEvent_t ev : inflight) cudaEventDestroy(ev);
  if (!started) cudaEventRecord(e0, st);
  cudaEventRecord(e1, st);
  if (timing) {
    cudaEventSynchronize(e1);
    for (size_t k = 0; k < slices.size(); ++k) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, slices[k].end);
      fprintf(stderr, "[factor slices] %zu: %lld tasks, handed out at %.1f ms, done at %.1f ms\n", k,
              (long long)slices[k].tasks, slices[k].host_ms, ms);
      cudaEventDestroy(slices[k].end);
    }
  }
  for (auto& th : pool) th.join();  // after an error the planners still finish
  for (FactorJob& J : jobs) J.hb.sink = nullptr;
  if (cs) cudaStreamDestroy(cs);
  return s;
}

}  // namespace

namespace {
// alphas == nullptr: alpha = 1 for every problem
int factor_batch_impl(const hm_matrix* const* Hs, const double* alphas, const double* thetas, int count,
                      void* stream, hm_factors** out) {
  if (!out || !Hs || !thetas || count < 1) { set_error("bad argument"); return HM_ERR_ARG; }
  for (int i = 0; i < count; ++i) out[i] = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  // HM_TIME_PHASES=1: host wall time of every phase on stderr
  const bool timing = std::getenv("HM_TIME_PHASES") != nullptr;
  auto tp = std::chrono::steady_clock::now();
  auto phase = [&](const char* what) {
    if (!timing) return;
    cudaStreamSynchronize(st);
    auto t = std::chrono::steady_clock::now();
    fprintf(stderr, "[factor x%d] %-14s %8.1f ms\n", count, what, std::chrono::duration<double, std::milli>(t - tp).count());
    tp = t;
  };
  std::vector<FactorJob> jobs(count);
  auto fail_all = [&](int s) {
    cudaDeviceSynchronize();
    for (FactorJob& J : jobs) factor_discard(J);
    return s;
  };
  int s = HM_OK;
  for (int i = 0; i < count; ++i) {
    if (!Hs[i]) { set_error("null matrix"); return fail_all(HM_ERR_ARG); }
    if ((s = factor_alloc(jobs[i], Hs[i], thetas[i], st)) != HM_OK) return fail_all(s);
    jobs[i].F->alpha = alphas ? alphas[i] : 1.0;
  }
  phase("allocate");
  int* d_err = Hs[0]->d_err;  // the batch shares the first matrix's error word
  const bool tracing = std::getenv("HM_PHASE_TRACE") != nullptr;
  const char* pipe = std::getenv("HM_PIPELINE");
  const bool streamed = !tracing && !(pipe && pipe[0] == '0');
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<void*> fs_allocs;
  if (streamed) {
    // planning streamed into execution (slices of the operation lists)
    int launches = 0;
    s = factor_streamed(jobs, st, d_err, e0, e1, fs_allocs, launches);
    for (FactorJob& J : jobs)
      if (J.status != HM_OK) {
        cudaStreamSynchronize(st);
        for (void* p : fs_allocs) cudaFree(p);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        set_error(J.err);
        return fail_all(J.status);
      }
    if (timing) fprintf(stderr, "[factor x%d] streamed in %d launches\n", count, launches);
  } else {
    // host planning of every H-LU (independent problems: one host thread each)
    parallel_for(count, [&](int i) { factor_plan(jobs[i]); });
    for (FactorJob& J : jobs)
      if (J.status != HM_OK) { set_error(J.err); return fail_all(J.status); }
    phase("plan H-LU");
    // one schedule for all: the problems' operation graphs side by side
    std::vector<SchedPart> parts;
    for (FactorJob& J : jobs) parts.push_back(SchedPart{&J.hb.waves, &J.hb.graph, nullptr});
    DevSchedule fs;
    s = upload_schedules(parts, fs, fs_allocs, 0, false);
    phase("upload");
    cudaEventRecord(e0, st);
    if (s == HM_OK && tracing && count == 1) {
      trace_schedule("factor", jobs[0].hb.waves, jobs[0].hb.graph, fs, d_err, st);  // note: runs the factorisation
    } else if (s == HM_OK) {
      s = run_schedule(fs, d_err, st);
    }
    cudaEventRecord(e1, st);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) s = HM_ERR_CUDA;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (void* p : fs_allocs) cudaFree(p);
  for (FactorJob& J : jobs) {
    std::vector<Wave>().swap(J.hb.waves);
    J.hb.graph.release();
  }
  phase("run H-LU");
  if (s != HM_OK) {
    set_error("H-LU execution failed: " + std::string(cudaGetErrorString(cudaGetLastError())));
    return fail_all(s);
  }
  int e = 0;
  cudaMemcpy(&e, d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e & DEVERR_ZEROPIVOT) { set_error("zero pivot in a leaf LU"); return fail_all(HM_ERR_DEVICE_ASSERT); }
  if (e & DEVERR_TIMEOUT) { set_error("bounded wait gave up in the H-LU schedule"); return fail_all(HM_ERR_TIMEOUT); }
  if (e & DEVERR_NONFINITE) {
    set_error("non-finite value, or an H-LU GEMM operand of magnitude >= 2^128 (beyond double-float range)");
    return fail_all(HM_ERR_DEVICE_ASSERT);
  }
  if (e & DEVERR_RANKCAP) {
    int z = e & ~DEVERR_RANKCAP;
    cudaMemcpy(d_err, &z, sizeof(int), cudaMemcpyHostToDevice);
  }
  for (FactorJob& J : jobs) J.F->tmp.release();  // the schedule has run: its temporaries are dead
  for (FactorJob& J : jobs) {
    J.F->fact_ms = ms;
    J.F->fact_fma = J.hb.gemm_fma[0] + J.hb.gemm_fma[1] + J.hb.gemm_fma[2];
    J.F->capped = (e & DEVERR_RANKCAP) ? 1 : 0;  // in a batch: some problem reached its cap
    const int nlr = (int)J.H->h_ld.size();
    J.F->h_rank.assign(nlr, 0);
    if (nlr) cudaMemcpy(J.F->h_rank.data(), J.F->d_rank, sizeof(int) * nlr, cudaMemcpyDeviceToHost);
  }
  // the solve schedules (they read the factor ranks), planned in parallel;
  // or the hierarchical inverses of the factors
  phase("ranks");
  parallel_for(count, [&](int i) {
    if (jobs[i].F->solve_mode == HM_SOLVE_SUBST) factor_plan_solve(jobs[i]);
  });
  for (FactorJob& J : jobs)
    if (J.status != HM_OK) { set_error(J.err); return fail_all(J.status); }
  phase("plan solves");
  {
    // the inverses of every problem that solves with them, built together
    std::vector<HinvBuildJob> hjobs;
    for (FactorJob& J : jobs) {
      hm_factors* F = J.F;
      if (F->solve_mode != HM_SOLVE_HINV) continue;
      F->hinv = new HinvData();
      const int prec = J.H->opts.precision == HM_MIXED_FP32 ? HINV_F32
                       : (J.H->opts.precision == HM_MIXED_BF16 ? HINV_BF16 : HINV_F64);
      hjobs.push_back(HinvBuildJob{&J.H->plan, &J.H->h_dd, &F->F, F->d_rank, prec, hinv_tolerance(J.H->opts),
                                   F->hinv});
    }
    if (!hjobs.empty()) {
      std::string herr;
      s = hinv_build_batch(hjobs, d_err, st, herr);
      if (s != HM_OK) { set_error("hierarchical inverses: " + herr); return fail_all(s); }
    }
    for (FactorJob& J : jobs) {
      hm_factors* F = J.F;
      if (F->solve_mode != HM_SOLVE_HINV) continue;
      F->lu_bytes = F->hinv->step_bytes;
      // the solves read only the inverses: the factors and the planner's
      // temporaries are released (the layout's pointers are dropped with them)
      F->arena.release();
      F->F = FactorLayout();
    }
  }
  if (count > 0) phase("inverses");
  for (FactorJob& J : jobs) {
    hm_factors* F = J.F;
    if (F->solve_mode != HM_SOLVE_SUBST) continue;
    s = upload_schedule(F->sw, F->sg, F->solve, F->allocs, &F->srcs);
    if (s != HM_OK) { set_error("solve schedule upload failed"); return fail_all(s); }
    if (tracing && count == 1) {
      trace_schedule("solve", F->sw, F->sg, F->solve, J.H->d_err, st);
      trace_schedule("solve", F->sw, F->sg, F->solve, J.H->d_err, st);
    }
  }
  phase("upload solves");
  for (int i = 0; i < count; ++i) {
    out[i] = jobs[i].F;
    jobs[i].F = nullptr;
  }
  return HM_OK;
}
}  // namespace
}  // namespace hm

extern "C" {

int hm_batch_create(const hm_matrix* const* Hs, const hm_factors* const* Fs, const double* dts, int count,
                    hm_batch** out) {
  if (!out) { set_error("null argument"); return HM_ERR_ARG; }
  *out = nullptr;
  if (!Hs || !Fs || !dts || count < 1) { set_error("bad argument"); return HM_ERR_ARG; }
  const int R = Hs[0] ? Hs[0]->opts.refine_max : 0;
  for (int i = 0; i < count; ++i) {
    if (!Hs[i] || !Fs[i]) { set_error("null entry"); return HM_ERR_ARG; }
    if (Fs[i]->H != Hs[i]) { set_error("factors belong to another matrix"); return HM_ERR_ARG; }
    if (!(dts[i] > 0.0) || Fs[i]->alpha != 1.0 || std::fabs(Fs[i]->theta + 0.5 * dts[i]) > 1e-12 * std::fabs(0.5 * dts[i])) {
      set_error("factors must come from hm_factor(H, -dt/2)");
      return HM_ERR_ARG;
    }
    if (Hs[i]->opts.refine_max != R) { set_error("all matrices must share refine_max"); return HM_ERR_ARG; }
    if (Hs[i]->opts.cn_form != Hs[0]->opts.cn_form) { set_error("all matrices must share cn_form"); return HM_ERR_ARG; }
    for (int j = 0; j < i; ++j)
      if (Hs[j] == Hs[i] || Fs[j] == Fs[i]) { set_error("matrices and factors must be distinct"); return HM_ERR_ARG; }
  }
  hm_batch* B = new hm_batch();
  B->H.assign(Hs, Hs + count);
  B->F.assign(Fs, Fs + count);
  B->refine = R;
  B->literal = Hs[0]->opts.cn_form == HM_CN_LITERAL;
  auto fail = [&](int s) {
    hm_batch_free(B);
    return s;
  };
  // one solve schedule for all problems, in the throughput mode (more CTAs per
  // SM, smaller staging; staging changes where operands are read from, not
  // the arithmetic)
  int s = HM_OK;
  int nsub = 0;
  for (int i = 0; i < count; ++i) nsub += Fs[i]->solve_mode == HM_SOLVE_SUBST ? 1 : 0;
  if (count == 1 && nsub == 1) {
    B->sched = Fs[0]->solve;  // one problem: its own schedule, latency mode (borrowed, not freed here)
  } else if (nsub > 0) {
    std::vector<SchedPart> parts;
    for (int i = 0; i < count; ++i)
      if (Fs[i]->solve_mode == HM_SOLVE_SUBST) parts.push_back(SchedPart{&Fs[i]->sw, &Fs[i]->sg, &Fs[i]->srcs});
    s = upload_schedules(parts, B->sched, B->allocs, SOLVE_MODE_THROUGHPUT, true);
    if (s != HM_OK) { set_error("batched solve schedule upload failed"); return fail(s); }
  }
  // the unrefined identity form fuses its vector steps into the inverses'
  // products: v = (LU)^{-1} (2x) = 2 (LU)^{-1} x exactly (a power of two), so
  // L^{-1} reads the state x and U^{-1} writes x = 2 z - x in place
  const bool fused = !B->literal && R == 0;
  {
    std::vector<HinvJob> jl, ju;
    for (int i = 0; i < count; ++i) {
      const hm_factors* F = Fs[i];
      if (F->solve_mode != HM_SOLVE_HINV) continue;
      const int N = Hs[i]->plan.N;
      double* x = F->d_vec + 3 * (size_t)N;
      if (fused) {
        jl.push_back(HinvJob{F->hinv->tri[0].A, x, F->hinv->d_y, nullptr, 1.0});
        ju.push_back(HinvJob{F->hinv->tri[1].A, F->hinv->d_y, x, x, 2.0});
      } else {
        jl.push_back(HinvJob{F->hinv->tri[0].A, F->d_y, F->hinv->d_y, nullptr, 1.0});
        ju.push_back(HinvJob{F->hinv->tri[1].A, F->hinv->d_y, F->d_sv + (size_t)N, nullptr, 1.0});
      }
    }
    if ((s = upload_hinv_batch(jl, B->hL, B->allocs)) != HM_OK) return fail(s);
    if ((s = upload_hinv_batch(ju, B->hU, B->allocs)) != HM_OK) return fail(s);
  }
  // per problem: Morton-order state x (owned by the batch), rhs, residual,
  // refined iterate, solve output z
  std::vector<MvJob> jA(count), jB(count);
  std::vector<VecJob> rhs_in, w_in, w_solve, s_in, z_out, z_u1, z_v, u1_add, u1_out, u1_copy;
  for (int i = 0; i < count; ++i) {
    const hm_matrix* H = Hs[i];
    hm_factors* F = const_cast<hm_factors*>(Fs[i]);
    const int N = H->plan.N;
    const double th = 0.5 * dts[i];
    double* rhs = F->d_vec;
    double* res = F->d_vec + (size_t)N;
    double* u1 = F->d_vec + 2 * (size_t)N;
    double* x = F->d_vec + 3 * (size_t)N;
    double* z = F->d_sv + (size_t)N;
    B->state.push_back(x);
    jA[i] = MvJob{H->mv, 1.0, th, th, x, nullptr, nullptr, nullptr, rhs};   // rhs = x + th G x
    jB[i] = MvJob{H->mv, -1.0, th, 0.0, u1, nullptr, nullptr, rhs, res};    // res = rhs - (u1 - th G u1)
    rhs_in.push_back({rhs, F->d_y, 0.0, N, 0});
    w_in.push_back({x, rhs, 0.0, N, 2});      // w = 2 x
    w_in.push_back({x, F->d_y, 0.0, N, 2});   // the solve's input
    const bool own = !fused || F->solve_mode != HM_SOLVE_HINV;  // fused: nothing to do here
    if (own) w_solve.push_back({x, F->d_y, 0.0, N, 2});
    s_in.push_back({res, F->d_y, 0.0, N, 0});
    z_out.push_back({z, x, 0.0, N, 0});
    z_u1.push_back({z, u1, 0.0, N, 0});
    if (own) z_v.push_back({z, x, 0.0, N, 3});  // x = v - x, v the solve's output
    u1_add.push_back({z, u1, 1.0, N, 1});
    u1_out.push_back({u1, x, 0.0, N, 3});     // x = v - x
    u1_copy.push_back({u1, x, 0.0, N, 0});
  }
  auto vblocks = [](const VecJob& J) { return (J.n + VEC_CHUNK - 1) / VEC_CHUNK; };
  if ((s = upload_mv_batch(jA, B->A, B->allocs)) != HM_OK) return fail(s);
  if ((s = upload_mv_batch(jB, B->B, B->allocs)) != HM_OK) return fail(s);
  if ((s = upload_jobs(rhs_in, vblocks, B->rhs_in, B->allocs)) != HM_OK) return fail(s);
  if ((s = upload_jobs(w_in, vblocks, B->w_in, B->allocs)) != HM_OK) return fail(s);
  if ((s = upload_jobs(w_solve, vblocks, B->w_solve, B->allocs)) != HM_OK) return fail(s);
  if ((s = upload_jobs(z_v, vblocks, B->z_v, B->allocs)) != HM_OK) return fail(s);
  if ((s = upload_jobs(u1_copy, vblocks, B->u1_copy, B->allocs)) != HM_OK) return fail(s);
  if ((s = upload_jobs(s_in, vblocks, B->s_in, B->allocs)) != HM_OK) return fail(s);
  if ((s = upload_jobs(z_out, vblocks, B->z_out, B->allocs)) != HM_OK) return fail(s);
  if ((s = upload_jobs(z_u1, vblocks, B->z_u1, B->allocs)) != HM_OK) return fail(s);
  if ((s = upload_jobs(u1_add, vblocks, B->u1_add, B->allocs)) != HM_OK) return fail(s);
  if ((s = upload_jobs(u1_out, vblocks, B->u1_out, B->allocs)) != HM_OK) return fail(s);
  if ((s = prepare_executor(B->sched)) != HM_OK) return fail(s);
  if (cudaStreamCreateWithFlags(&B->cs, cudaStreamNonBlocking) != cudaSuccess) return fail(HM_ERR_CUDA);
  cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming);
  // record one step as a CUDA graph (replayed by hm_batch_step); without
  // capture support every step is launched directly
  if (cudaStreamBeginCapture(B->cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    const int64_t l0 = hm_launch_count();
    const int sc = batch_one_step(B, B->cs);
    const cudaError_t ec = cudaStreamEndCapture(B->cs, &B->graph);
    B->per_step = hm_launch_count() - l0;
    count_launches(-(int)B->per_step);  // counted when the graph runs
    if (sc != HM_OK || ec != cudaSuccess || cudaGraphInstantiate(&B->gexec, B->graph, 0) != cudaSuccess) {
      cudaGetLastError();
      if (B->gexec) cudaGraphExecDestroy(B->gexec);
      B->gexec = nullptr;
    }
  } else {
    cudaGetLastError();
  }
  g_batch_graphed = B->gexec != nullptr;
  *out = B;
  return HM_OK;
}

int hm_batch_step(hm_batch* B, double* const* u, int steps, void* stream) {
  if (!B || !u || steps < 0) { set_error("bad argument"); return HM_ERR_ARG; }
  const int count = (int)B->H.size();
  for (int i = 0; i < count; ++i)
    if (!u[i]) { set_error("null state vector"); return HM_ERR_ARG; }
  if (steps == 0) return HM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  // ordered after the caller's stream (which may be the legacy default stream)
  cudaEventRecord(B->ev, st);
  cudaStreamWaitEvent(B->cs, B->ev, 0);
  int s = HM_OK;
  for (int i = 0; i < count && s == HM_OK; ++i) {
    const hm_matrix* H = B->H[i];
    const int N = H->plan.N;
    if (H->plan.dim == 1) {
      count_launches(1);
      copy_vec_kernel<<<vgrid(N), 256, 0, B->cs>>>(N, u[i], B->state[i]);
      s = cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
    } else {
      s = launch_gather(H->d_perm, N, u[i], B->state[i], B->cs);
    }
  }
  for (int k = 0; k < steps && s == HM_OK; ++k) {
    if (B->gexec) {
      s = cudaGraphLaunch(B->gexec, B->cs) == cudaSuccess ? HM_OK : HM_ERR_CUDA;
      count_launches((int)B->per_step);
    } else {
      s = batch_one_step(B, B->cs);
    }
  }
  for (int i = 0; i < count && s == HM_OK; ++i) {
    const hm_matrix* H = B->H[i];
    const int N = H->plan.N;
    if (H->plan.dim == 1) {
      count_launches(1);
      copy_vec_kernel<<<vgrid(N), 256, 0, B->cs>>>(N, B->state[i], u[i]);
      s = cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
    } else {
      s = launch_scatter(H->d_perm, N, B->state[i], u[i], B->cs);
    }
  }
  cudaEventRecord(B->ev, B->cs);
  cudaStreamWaitEvent(st, B->ev, 0);
  if (s != HM_OK) set_error("batched CN steps failed: " + std::string(cudaGetErrorString(cudaGetLastError())));
  return s;
}

void hm_batch_free(hm_batch* B) {
  if (!B) return;
  if (B->cs) cudaStreamSynchronize(B->cs);
  if (B->gexec) cudaGraphExecDestroy(B->gexec);
  if (B->graph) cudaGraphDestroy(B->graph);
  if (B->ev) cudaEventDestroy(B->ev);
  if (B->cs) cudaStreamDestroy(B->cs);
  for (void* p : B->allocs) cudaFree(p);
  delete B;
}

int cn_solve_batch(const hm_matrix* const* Hs, const hm_factors* const* Fs, int count, double dt, int steps,
                   double* const* u, void* stream) {
  if (!Hs || !Fs || !u || count < 1 || steps < 0 || !(dt > 0.0)) { set_error("bad argument"); return HM_ERR_ARG; }
  for (int i = 0; i < count; ++i)
    if (!u[i]) { set_error("null state vector"); return HM_ERR_ARG; }
  std::vector<double> dts(count, dt);
  hm_batch* B = nullptr;
  HM_TRY(hm_batch_create(Hs, Fs, dts.data(), count, &B));
  const int s = hm_batch_step(B, u, steps, stream);
  if (s == HM_OK) cudaStreamSynchronize(B->cs);
  int e = 0;
  cudaMemcpy(&e, Hs[0]->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  hm_batch_free(B);
  if (s == HM_OK && (e & DEVERR_TIMEOUT)) { set_error("bounded wait gave up in a solve"); return HM_ERR_TIMEOUT; }
  return s;
}

int hm_batch_graphed(void) { return g_batch_graphed ? 1 : 0; }

void hm_factors_free(hm_factors* F) {
  if (!F) return;
  if (F->batch1) hm_batch_free(F->batch1);
  cudaDeviceSynchronize();
  if (F->hinv) {
    F->hinv->release();
    delete F->hinv;
  }
  for (void* p : F->allocs) cudaFree(p);
  F->arena.release();
  F->tmp.release();
  delete F;
}

int hm_solve(const hm_factors* F, const double* b, double* x, void* stream) {
  if (!F || !b || !x) { set_error("null argument"); return HM_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const hm_matrix* H = F->H;
  const int N = H->plan.N;
  if (H->plan.dim == 1) return solve_morton(F, b, x, st);
  double* t = F->d_vec + 5 * (size_t)N;
  HM_TRY(launch_gather(H->d_perm, N, b, t, st));
  HM_TRY(solve_morton(F, t, t, st));
  return launch_scatter(H->d_perm, N, t, x, st);
}

int hm_shifted_solve(const hm_matrix* H, const hm_factors* F, const double* b, double* x, double tol, int maxit,
                     void* stream, int* iters, double* resid) {
  if (!H || !F || !b || !x || maxit < 0 || !(tol >= 0.0)) { set_error("bad argument"); return HM_ERR_ARG; }
  if (b == x) { set_error("x must not alias b"); return HM_ERR_ARG; }
  // the preconditioner may be factored from another H-matrix of the same grid
  // (e.g. a coarser compression): both must share the unknowns' order
  if (F->H != H && (F->H->plan.N != H->plan.N || F->H->plan.perm != H->plan.perm)) {
    set_error("factors belong to a matrix of another grid");
    return HM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  hm_factors* Fm = const_cast<hm_factors*>(F);
  const int N = H->plan.N;
  double* bm = Fm->d_vec + 2 * (size_t)N;  // b, Morton order
  double* xm = Fm->d_vec + 3 * (size_t)N;  // iterate
  double* r = Fm->d_vec + 4 * (size_t)N;   // residual, then correction
  if (H->plan.dim == 2) HM_TRY(launch_gather(H->d_perm, N, b, bm, st));
  else {
    count_launches(1);
    copy_vec_kernel<<<vgrid(N), 256, 0, st>>>(N, b, bm);
  }
  // x_0 = M~^{-1} b, then x_{k+1} = x_k + M~^{-1} (b - M x_k) with M = alpha I + theta G
  HM_TRY(solve_morton(F, bm, xm, st));
  int it = 0;
  double rel = 0.0;
  for (;;) {
    HM_TRY(hm_matvec_morton(H, -F->alpha, -F->theta, xm, 0.0, nullptr, nullptr, bm, r, st));
    count_launches(1);
    norms_kernel<<<1, 1024, 0, st>>>(N, r, bm, F->d_norm);
    double nrm[2] = {0.0, 0.0};
    HM_CK(cudaMemcpyAsync(nrm, F->d_norm, sizeof(nrm), cudaMemcpyDeviceToHost, st));
    HM_CK(cudaStreamSynchronize(st));
    rel = nrm[1] > 0.0 ? std::sqrt(nrm[0] / nrm[1]) : std::sqrt(nrm[0]);
    if (!std::isfinite(rel) || rel <= tol || it >= maxit) break;
    HM_TRY(solve_morton(F, r, r, st));
    count_launches(1);
    axpy_kernel<<<vgrid(N), 256, 0, st>>>(N, 1.0, r, xm);
    ++it;
  }
  if (iters) *iters = it;
  if (resid) *resid = rel;
  if (H->plan.dim == 2) HM_TRY(launch_scatter(H->d_perm, N, xm, x, st));
  else {
    count_launches(1);
    copy_vec_kernel<<<vgrid(N), 256, 0, st>>>(N, xm, x);
  }
  HM_CK(cudaGetLastError());
  if (!(rel <= tol)) {
    set_error("residual " + std::to_string(rel) + " above tol after " + std::to_string(it) + " iterations");
    return HM_ERR_NOT_CONVERGED;
  }
  return HM_OK;
}

int cn_step(const hm_matrix* H, const hm_factors* F, double dt, const double* u_n, const double* f_n,
            const double* f_np1, double* u_np1, void* stream) {
  if (!H || !F || !u_n || !u_np1) { set_error("null argument"); return HM_ERR_ARG; }
  if (u_n == u_np1) { set_error("u_np1 must not alias u_n"); return HM_ERR_ARG; }
  if (F->H != H) { set_error("factors belong to another matrix"); return HM_ERR_ARG; }
  if (!(dt > 0.0) || F->alpha != 1.0 || std::fabs(F->theta + 0.5 * dt) > 1e-12 * std::fabs(0.5 * dt)) {
    set_error("factors must come from hm_factor(H, -dt/2)");
    return HM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  hm_factors* Fm = const_cast<hm_factors*>(F);
  const int N = H->plan.N;
  if (H->plan.dim == 1) return cn_step_morton(H, Fm, dt, u_n, f_n, f_np1, u_np1, st);
  double* um = Fm->d_vec + 2 * (size_t)N;
  double* f0 = Fm->d_vec + 3 * (size_t)N;
  double* f1 = Fm->d_vec + 4 * (size_t)N;
  double* u1 = Fm->d_vec + 5 * (size_t)N;
  HM_TRY(launch_gather(H->d_perm, N, u_n, um, st));
  if (f_n) HM_TRY(launch_gather(H->d_perm, N, f_n, f0, st));
  if (f_np1) HM_TRY(launch_gather(H->d_perm, N, f_np1, f1, st));
  HM_TRY(cn_step_morton(H, Fm, dt, um, f_n ? f0 : nullptr, f_np1 ? f1 : nullptr, u1, st));
  return launch_scatter(H->d_perm, N, u1, u_np1, st);
}

int cn_solve(const hm_matrix* H, const hm_factors* F, double dt, int steps, int step0, double* u,
             const double* f, void* stream) {
  if (!H || !F || !u || steps < 0 || step0 < 0) { set_error("bad argument"); return HM_ERR_ARG; }
  if (F->H != H) { set_error("factors belong to another matrix"); return HM_ERR_ARG; }
  if (!(dt > 0.0) || F->alpha != 1.0 || std::fabs(F->theta + 0.5 * dt) > 1e-12 * std::fabs(0.5 * dt)) {
    set_error("factors must come from hm_factor(H, -dt/2)");
    return HM_ERR_ARG;
  }
  (void)step0;  // the levels of f are relative to step0; the operator is time independent
  cudaStream_t st = (cudaStream_t)stream;
  if (!f && H->opts.refine_max == 0 && steps > 1) {
    // no forcing, no refinement: the persistent-batch path with one problem,
    // one step recorded as a CUDA graph and replayed (same arithmetic)
    hm_factors* Fb = const_cast<hm_factors*>(F);
    if (!Fb->batch1) HM_TRY(hm_batch_create(&H, &F, &dt, 1, &Fb->batch1));
    return hm_batch_step(Fb->batch1, &u, steps, stream);
  }
  hm_factors* Fm = const_cast<hm_factors*>(F);
  const int N = H->plan.N;
  double* ua = Fm->d_vec + 2 * (size_t)N;
  double* ub = Fm->d_vec + 5 * (size_t)N;
  double* f0 = Fm->d_vec + 3 * (size_t)N;
  double* f1 = Fm->d_vec + 4 * (size_t)N;
  const bool perm = H->plan.dim == 2;
  if (perm) HM_TRY(launch_gather(H->d_perm, N, u, ua, st));
  else {
    count_launches(1);
    copy_vec_kernel<<<vgrid(N), 256, 0, st>>>(N, u, ua);
  }
  for (int k = 0; k < steps; ++k) {
    const double* fa = nullptr;
    const double* fb = nullptr;
    if (f) {
      const double* g0 = f + (size_t)k * N;
      const double* g1 = f + (size_t)(k + 1) * N;
      if (perm) {
        HM_TRY(launch_gather(H->d_perm, N, g0, f0, st));
        HM_TRY(launch_gather(H->d_perm, N, g1, f1, st));
        fa = f0;
        fb = f1;
      } else {
        fa = g0;
        fb = g1;
      }
    }
    HM_TRY(cn_step_morton(H, Fm, dt, ua, fa, fb, ub, st));
    std::swap(ua, ub);
  }
  if (perm) return launch_scatter(H->d_perm, N, ua, u, st);
  count_launches(1);
  copy_vec_kernel<<<vgrid(N), 256, 0, st>>>(N, ua, u);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

int hm_plan_factor(const hm_problem* prob, const hm_opts* opts, double theta, hm_factor_plan_t* out) {
  if (!prob || !opts || !out) { set_error("null argument"); return HM_ERR_ARG; }
  std::memset(out, 0, sizeof(*out));
  Plan P;
  std::string err;
  if (make_plan(*prob, *opts, P, err) != HM_OK) { set_error(err); return HM_ERR_ARG; }
  std::vector<DenseDesc> dd;
  std::vector<LRDesc> ld;
  int64_t dp = 0, up = 0, vp = 0;
  make_descs(P, *opts, dd, ld, dp, up, vp);
  int maxr = 0;
  for (auto& L : ld) maxr = std::max(maxr, L.kcap);
  int kf = std::max(opts->lu_max_rank, maxr);
  if (kf > TRUNC_MAXK / 2) { set_error("factor rank cap too large"); return HM_ERR_RANK_CAP; }
  Arena A;
  A.fake = true;
  // host-side fault injection: HM_ARENA_LIMIT_BYTES makes the planner's
  // allocations fail past that many bytes, as a full device would
  if (const char* lim = std::getenv("HM_ARENA_LIMIT_BYTES")) A.fake_limit = std::atoll(lim);
  // fake storage of the H-matrix and of the factor ranks
  double* fD = A.alloc(std::max<int64_t>(dp, 1));
  double* fU = A.alloc(std::max<int64_t>(up, 1));
  double* fV = A.alloc(std::max<int64_t>(vp, 1));
  int* frank = (int*)A.alloc((int64_t)ld.size() / 2 + 1);
  double* fy = A.alloc(5 * (int64_t)P.N);
  HluBuild hb;
  int s = plan_hlu(P, dd, fD, ld, fU, fV, kf, theta, opts->lu_tol, frank, A, hb, 1.0, opts->solve_block, true);
  if (s != HM_OK) {
    const char* cs = std::getenv("HM_CHECK_STREAM");
    if (cs && s == HM_ERR_OOM && A.fake_limit >= 0 &&
        !check_streamed_failure(P, dd, ld, kf, theta, opts->lu_tol, std::max(1, std::atoi(cs)), A.fake_limit))
      return HM_ERR_ARG;
    set_error("planning failed: " + hb.err);
    return s;
  }
  if (const char* cs = std::getenv("HM_CHECK_STREAM")) {
    // self-check of the streamed planning (slices of HM_CHECK_STREAM ops): the
    // same planning handed out in slices, merged the way the executor
    // launches consume them (groups of 1, 2, 3, ... consecutive slices), must
    // give every op the producers it has in the one-piece plan that lie in its
    // own group, and the same order of waves
    if (!check_streamed_plan(P, dd, ld, kf, theta, opts->lu_tol, std::max(1, std::atoi(cs)), hb)) return HM_ERR_ARG;
  }
  if (std::getenv("HM_PLAN_HIST")) plan_histogram(hb.waves);
  std::vector<Wave> sw;
  std::vector<RowSrc> srcs;
  OpGraph sg;
  SolveVectors sv{fy, fy + P.N, fy + 2 * (int64_t)P.N, fy + 3 * (int64_t)P.N, fy + 4 * (int64_t)P.N};
  s = plan_solve(P, dd, ld, hb.F, nullptr, sv, A, sw, srcs, sg);
  if (s != HM_OK) { set_error("solve planning failed"); return s; }
  std::string first;
  int64_t bad = check_spans(hb.waves, A.ranges, first) + check_spans(sw, A.ranges, first, &srcs);
  int64_t sops = 0;
  for (auto& w : sw)
    sops += w.gemm.size() + w.copy.size() + w.lu.size() + w.trunc.size() + w.reduce.size() + w.rows.size() +
            w.vpart.size();
  out->fact_ops = hb.ops;
  out->fact_waves = (int)hb.waves.size();
  out->solve_ops = sops;
  out->solve_waves = (int)sw.size();
  out->bad_spans = bad;
  out->arena_bytes = A.total * (int64_t)sizeof(double);
  out->kf = kf;
  for (int i = 0; i < 3; ++i) out->gemm_fma[i] = hb.gemm_fma[i];
  if (bad) set_error("operand outside its allocation: " + first);
  return HM_OK;
}

int hm_stats(const hm_matrix* H, const hm_factors* F, hm_stats_t* out) {
  if (!H || !out) { set_error("null argument"); return HM_ERR_ARG; }
  std::memset(out, 0, sizeof(*out));
  const Plan& P = H->plan;
  out->n = P.N;
  out->clusters = (int)P.cl.size();
  out->leaves = (int)P.leaves.size();
  out->depth = P.depth;
  out->dense_blocks = (int)H->h_dd.size();
  out->lowrank_blocks = (int)H->h_ld.size();
  int64_t de = 0, le = 0;
  for (auto& D : H->h_dd) de += (int64_t)D.m * D.n;
  int mr = 0;
  for (size_t q = 0; q < H->h_ld.size(); ++q) {
    le += (int64_t)(H->h_ld[q].m + H->h_ld[q].n) * H->h_rank[q];
    mr = std::max(mr, H->h_rank[q]);
  }
  out->dense_entries = de;
  out->lowrank_entries = le;
  out->max_rank_seen = mr;
  out->rank_capped_blocks = H->capped_blocks;
  // bytes one H-matvec streams: dense leaves, and the U, V columns up to each block's cap
  int64_t hb = de;
  for (size_t q = 0; q < H->h_ld.size(); ++q) hb += (int64_t)(H->h_ld[q].m + H->h_ld[q].n) * H->h_rank[q];
  out->h_bytes = 8 * hb;
  out->device_bytes = H->arena.bytes_held;
  if (F) {
    for (auto& r : F->arena.ranges) out->device_bytes += (int64_t)(r.second - r.first);
    out->lu_bytes = F->lu_bytes;
    out->factor_fma = F->fact_fma;
    out->factor_ms = F->fact_ms;
    int m2 = 0;
    for (int r : F->h_rank) m2 = std::max(m2, r);
    out->lu_max_rank_seen = m2;
    out->lu_rank_capped = F->capped;
    double nrm[2] = {0, 0};
    if (cudaDeviceSynchronize() != cudaSuccess) return HM_ERR_CUDA;
    cudaMemcpy(nrm, F->d_norm, sizeof(nrm), cudaMemcpyDeviceToHost);
    out->last_refine_iters = H->opts.refine_max;
    out->last_refine_resid = nrm[1] > 0 ? std::sqrt(nrm[0] / nrm[1]) : 0.0;
    out->solve_mode = F->solve_mode;
    if (F->hinv) {
      out->device_bytes += F->hinv->bytes;
      out->hinv_max_rank = F->hinv->max_rank;
      out->hinv_capped = F->hinv->capped;
      out->hinv_ms = F->hinv->build_ms;
    }
  }
  return HM_OK;
}

}  // extern "C"
