// C ABI: planning, construction (hm_build), H-matvec and inspection calls.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <atomic>
#include <cstring>

#include "api_common.h"

namespace hm {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

static std::atomic<int64_t> g_launches{0};
void count_launches(int n) { g_launches += n; }

namespace {

int check_problem(const hm_problem* p, const hm_opts* o) {
  if (!p || !o) { set_error("null problem or options"); return HM_ERR_ARG; }
  if (p->kernel != HM_NU_GAUSS && p->kernel != HM_NU_STABLE) { set_error("unknown kernel"); return HM_ERR_ARG; }
  if (p->kernel == HM_NU_STABLE && !(p->s > 0.0 && p->s < 1.0)) { set_error("s must lie in (0, 1)"); return HM_ERR_ARG; }
  if (p->kernel == HM_NU_GAUSS && !(p->eps > 0.0)) { set_error("eps must be > 0"); return HM_ERR_ARG; }
  if (!(p->a >= 0.0)) { set_error("a must be >= 0"); return HM_ERR_ARG; }
  if (!(p->LW > 0.0)) { set_error("LW must be > 0"); return HM_ERR_ARG; }
  if (p->kernel == HM_NU_STABLE && !(p->r > 0.0 && p->r <= p->LW)) { set_error("need 0 < r <= LW"); return HM_ERR_ARG; }
  if (!(p->trunc > 0.0)) { set_error("trunc must be > 0"); return HM_ERR_ARG; }
  if (p->domain != HM_DOMAIN_BOX && p->domain != HM_DOMAIN_L) { set_error("unknown domain"); return HM_ERR_ARG; }
  if (p->domain == HM_DOMAIN_L && p->dim != 2) { set_error("the L-shaped domain is 2D"); return HM_ERR_ARG; }
  if (p->s_slope != 0.0) {
    if (!std::isfinite(p->s_slope) || p->kernel != HM_NU_STABLE || p->dim != 2 || p->a != 0.0 || p->b[0] != 0.0 ||
        p->b[1] != 0.0 || p->c != 0.0 || std::isfinite(p->trunc)) {
      set_error("a variable order needs the 2D stable kernel, a = b = c = 0 and no truncation");
      return HM_ERR_ARG;
    }
  }
  if (o->max_rank < 1 || o->max_rank > ACA_MAXK) { set_error("max_rank must lie in [1, 128]"); return HM_ERR_ARG; }
  if (!(o->aca_tol > 0.0)) { set_error("aca_tol must be > 0"); return HM_ERR_ARG; }
  return HM_OK;
}

int device_ok() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { set_error(std::string("no CUDA device: ") + cudaGetErrorString(e)); return HM_ERR_NO_DEVICE; }
  cudaDeviceProp pr;
  e = cudaGetDeviceProperties(&pr, dev);
  if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return HM_ERR_NO_DEVICE; }
  if (pr.major != 10 || pr.minor != 3) {
    set_error("kernels are built for sm_103a only; device is sm_" + std::to_string(pr.major) +
              std::to_string(pr.minor));
    return HM_ERR_NO_DEVICE;
  }
  return HM_OK;
}

NuParams nu_params(const hm_problem& p, const Plan& P, int* nw_out, std::string& err) {
  NuParams q{};
  q.dim = p.dim;
  q.kernel = p.kernel;
  q.h = P.h;
  q.n0 = P.n[0];
  q.n1 = P.dim == 2 ? P.n[1] : 1;
  q.s = p.s;
  q.eps = p.eps;
  q.lam = p.lam;
  q.trunc = p.trunc;
  q.LW = p.LW;
  q.r = p.r;
  double ratio = p.LW / P.h;
  int nw = (int)std::lround(ratio);
  if (nw < 1 || std::fabs(ratio - nw) > 1e-9 * std::max(1.0, ratio)) err = "LW must be a whole number of grid steps";
  q.nw = nw;
  *nw_out = nw;
  if (p.kernel == HM_NU_STABLE) {
    double d = p.dim;
    q.cds = std::pow(4.0, p.s) * std::tgamma(d / 2.0 + p.s) /
            (std::pow(M_PI, d / 2.0) * std::fabs(std::tgamma(-p.s)));
    q.expo = d + 2.0 * p.s;
  }
  return q;
}

}  // namespace

void make_descs(const Plan& P, const hm_opts& o, std::vector<DenseDesc>& dd, std::vector<LRDesc>& ld,
                int64_t& dpool, int64_t& upool, int64_t& vpool) {
  dd.clear();
  ld.clear();
  int64_t off = 0;
  for (int b : P.dense_block) {
    const Block& B = P.bl[b];
    DenseDesc D{};
    D.r0 = P.cl[B.t].begin;
    D.m = P.cl[B.t].end - D.r0;
    D.c0 = P.cl[B.s].begin;
    D.n = P.cl[B.s].end - D.c0;
    D.ld = (D.n + 3) & ~3;
    D.off = off;
    off += (int64_t)D.m * D.ld;
    dd.push_back(D);
  }
  int64_t uo = 0, vo = 0;
  for (int b : P.lr_block) {
    const Block& B = P.bl[b];
    LRDesc L{};
    L.r0 = P.cl[B.t].begin;
    L.m = P.cl[B.t].end - L.r0;
    L.c0 = P.cl[B.s].begin;
    L.n = P.cl[B.s].end - L.c0;
    L.kcap = std::min(o.max_rank, std::min(L.m, L.n));
    L.uoff = uo;
    L.voff = vo;
    uo += (int64_t)L.m * L.kcap;
    vo += (int64_t)L.n * L.kcap;
    ld.push_back(L);
  }
  dpool = off;
  upool = uo;
  vpool = vo;
}

}  // namespace hm

namespace hm {
int hm_matvec_morton(const hm_matrix* H, double alpha, double beta, const double* xm, double gamma,
                     const double* w1m, const double* w2m, const double* w3m, double* ym,
                     cudaStream_t st) {
  return launch_matvec(H->mv, alpha, beta, xm, gamma, w1m, w2m, w3m, ym, st);
}
}  // namespace hm

using namespace hm;

extern "C" {

const char* hm_error_string(int status) {
  switch (status) {
    case HM_OK: return "ok";
    case HM_ERR_ARG: return "invalid argument";
    case HM_ERR_OOM: return "device out of memory";
    case HM_ERR_CUDA: return "CUDA error";
    case HM_ERR_RANK_CAP: return "rank cap reached";
    case HM_ERR_NOT_CONVERGED: return "refinement did not converge";
    case HM_ERR_TIMEOUT: return "bounded device wait gave up";
    case HM_ERR_DEVICE_ASSERT: return "device-side check failed";
    case HM_ERR_NO_DEVICE: return "no usable CUDA device";
    default: return "unknown status";
  }
}

const char* hm_last_error(void) { return g_last_error.c_str(); }

int64_t hm_launch_count(void) { return g_launches.load(); }

int hm_plan_info(const hm_problem* prob, const hm_opts* opts, hm_stats_t* info) {
  if (!info) { set_error("null info"); return HM_ERR_ARG; }
  HM_TRY(check_problem(prob, opts));
  Plan P;
  std::string err;
  HM_TRY(make_plan(*prob, *opts, P, err) == HM_OK ? HM_OK : (set_error(err), HM_ERR_ARG));
  std::memset(info, 0, sizeof(*info));
  info->n = P.N;
  info->clusters = (int)P.cl.size();
  info->leaves = (int)P.leaves.size();
  info->depth = P.depth;
  info->dense_blocks = (int)P.dense_block.size();
  info->lowrank_blocks = (int)P.lr_block.size();
  int64_t de = 0;
  for (int b : P.dense_block) {
    const Block& B = P.bl[b];
    de += (int64_t)(P.cl[B.t].end - P.cl[B.t].begin) * (P.cl[B.s].end - P.cl[B.s].begin);
  }
  info->dense_entries = de;
  return HM_OK;
}

int hm_plan_blocks(const hm_problem* prob, const hm_opts* opts, int* count, int* row0, int* m,
                   int* col0, int* ncols, int* type, int* perm) {
  if (!count || !row0 || !m || !col0 || !ncols || !type) { set_error("null output array"); return HM_ERR_ARG; }
  HM_TRY(check_problem(prob, opts));
  Plan P;
  std::string err;
  if (make_plan(*prob, *opts, P, err) != HM_OK) { set_error(err); return HM_ERR_ARG; }
  int total = (int)(P.dense_block.size() + P.lr_block.size());
  if (*count < total) { *count = total; set_error("output arrays too small"); return HM_ERR_ARG; }
  int k = 0;
  for (int pass = 0; pass < 2; ++pass) {
    const std::vector<int>& L = pass == 0 ? P.lr_block : P.dense_block;
    for (int b : L) {
      const Block& B = P.bl[b];
      row0[k] = P.cl[B.t].begin;
      m[k] = P.cl[B.t].end - P.cl[B.t].begin;
      col0[k] = P.cl[B.s].begin;
      ncols[k] = P.cl[B.s].end - P.cl[B.s].begin;
      type[k] = B.type;
      ++k;
    }
  }
  *count = total;
  if (perm) std::copy(P.perm.begin(), P.perm.end(), perm);
  return HM_OK;
}

// Variable order (Sec. "Application: Variable-Order Fractional Poisson
// Equation"): s_p = s - s_slope d(x_p) per Morton row.  The row constants
// lambda_W(s), T(s), kappa(s) are smooth in s: they are computed by the
// constant-order kernels at 24 Chebyshev points of [min s_p, max s_p] and
// interpolated per row (Chebyshev series, Clenshaw's recurrence).
static int variable_order_rows(hm_matrix* H, cudaStream_t st) {
  const Plan& P = H->plan;
  const hm_problem& p = H->prob;
  const int N = P.N;
  const double h = P.h;
  const double cx = 0.5 * (p.lo[0] + p.hi[0]), cy = 0.5 * (p.lo[1] + p.hi[1]);
  std::vector<double> sp(N);
  double s_lo = 1e300, s_hi = -1e300;
  for (int q = 0; q < N; ++q) {
    const double x = p.lo[0] + (P.coord[2 * q] + 1) * h, y = p.lo[1] + (P.coord[2 * q + 1] + 1) * h;
    double d = std::min(std::min(x - p.lo[0], p.hi[0] - x), std::min(y - p.lo[1], p.hi[1] - y));
    if (p.domain == HM_DOMAIN_L) d = std::min(d, std::hypot(std::max(0.0, cx - x), std::max(0.0, cy - y)));
    sp[q] = p.s - p.s_slope * d;
    s_lo = std::min(s_lo, sp[q]);
    s_hi = std::max(s_hi, sp[q]);
  }
  if (!(s_lo > 0.0 && s_hi < 1.0)) { set_error("the variable order leaves (0, 1)"); return HM_ERR_ARG; }
  const int M = s_hi - s_lo > 1e-12 ? 24 : 1;
  const double mid = 0.5 * (s_lo + s_hi), half = 0.5 * (s_hi - s_lo);
  auto cds = [](double s) { return std::pow(4.0, s) * std::tgamma(1.0 + s) / (M_PI * std::fabs(std::tgamma(-s))); };
  std::vector<double> fl(M), ft(M), fk(M), tm(M);
  for (int m = 0; m < M; ++m) {
    tm[m] = M > 1 ? std::cos(M_PI * (m + 0.5) / M) : 0.0;
    NuParams q = H->nuq;
    q.s = mid + half * tm[m];
    q.cds = cds(q.s);
    q.expo = 2.0 + 2.0 * q.s;
    HM_CK(cudaMemsetAsync(H->d_cscratch, 0, sizeof(double) * 8, st));
    HM_TRY(launch_constants(q, H->d_tab, H->d_cscratch, st));
    HM_TRY(launch_finalize_constants(q, 0.0, p.b, 0.0, H->d_cscratch, H->d_gc, st));
    GenConst g;
    HM_CK(cudaMemcpyAsync(&g, H->d_gc, sizeof(GenConst), cudaMemcpyDeviceToHost, st));
    HM_CK(cudaStreamSynchronize(st));
    fl[m] = g.lam_w;
    ft[m] = g.tail;
    fk[m] = g.kappa;
  }
  // Chebyshev coefficients c_k = (2/M) sum_m f_m T_k(t_m), c_0 halved
  auto coeffs = [&](const std::vector<double>& f) {
    std::vector<double> c(M, 0.0);
    for (int k = 0; k < M; ++k) {
      for (int m = 0; m < M; ++m) c[k] += f[m] * std::cos(k * M_PI * (m + 0.5) / M);
      c[k] *= (k == 0 ? 1.0 : 2.0) / M;
    }
    return c;
  };
  auto clenshaw = [&](const std::vector<double>& c, double t) {
    double b1 = 0.0, b2 = 0.0;
    for (int k = M - 1; k >= 1; --k) {
      const double b0 = 2.0 * t * b1 - b2 + c[k];
      b2 = b1;
      b1 = b0;
    }
    return t * b1 - b2 + c[0];
  };
  const std::vector<double> cl = coeffs(fl), ct = coeffs(ft), ck = coeffs(fk);
  std::vector<double> rb(N), re(N), rk(N), rd(N);
  for (int q = 0; q < N; ++q) {
    const double t = M > 1 ? (sp[q] - mid) / half : 0.0;
    const double lam = clenshaw(cl, t), tail = clenshaw(ct, t), kap = clenshaw(ck, t);
    rb[q] = cds(sp[q]) * std::pow(h, -2.0 * sp[q]);
    re[q] = -(1.0 + sp[q]);
    rk[q] = kap;
    rd[q] = -4.0 * kap - lam - tail;
  }
  DevArena& A = H->arena;
  double *db = nullptr, *de = nullptr, *dk = nullptr, *dd = nullptr;
  HM_TRY(A.upload(&db, rb));
  HM_TRY(A.upload(&de, re));
  HM_TRY(A.upload(&dk, rk));
  HM_TRY(A.upload(&dd, rd));
  H->ectx.rowB = db;
  H->ectx.rowE = de;
  H->ectx.rowK = dk;
  H->ectx.rowD = dd;
  H->ectx.nw = H->nuq.nw;
  return HM_OK;
}

static int build_impl(const hm_problem* prob, const hm_opts* opts, cudaStream_t st, hm_matrix* H) {
  HM_TRY(check_problem(prob, opts));
  HM_TRY(device_ok());
  H->prob = *prob;
  H->opts = *opts;
  HM_CK(cudaGetDevice(&H->device));
  std::string err;
  if (make_plan(*prob, *opts, H->plan, err) != HM_OK) { set_error(err); return HM_ERR_ARG; }
  Plan& P = H->plan;
  int nw = 0;
  H->nuq = nu_params(*prob, P, &nw, err);
  if (!err.empty()) { set_error(err); return HM_ERR_ARG; }
  DevArena& A = H->arena;
  const int N = P.N;

  // grid tables
  HM_TRY(A.upload(&H->d_perm, P.perm));
  HM_TRY(A.upload(&H->d_iperm, P.iperm));
  std::vector<int2> coord(N);
  for (int q = 0; q < N; ++q) coord[q] = make_int2(P.coord[2 * q], P.coord[2 * q + 1]);
  HM_TRY(A.upload(&H->d_coord, coord));
  HM_TRY(A.alloc((void**)&H->d_tab, sizeof(double) * (size_t)H->nuq.n0 * H->nuq.n1));
  HM_TRY(A.alloc((void**)&H->d_cscratch, sizeof(double) * 8));
  HM_TRY(A.alloc((void**)&H->d_gc, sizeof(GenConst)));
  HM_TRY(A.alloc((void**)&H->d_err, sizeof(int) * 4));
  HM_CK(cudaMemsetAsync(H->d_err, 0, sizeof(int) * 4, st));
  HM_CK(cudaMemsetAsync(H->d_cscratch, 0, sizeof(double) * 8, st));
  HM_TRY(launch_constants(H->nuq, H->d_tab, H->d_cscratch, st));
  HM_TRY(launch_finalize_constants(H->nuq, prob->a, prob->b, prob->c, H->d_cscratch, H->d_gc, st));
  H->ectx.dim = P.dim;
  H->ectx.n0 = H->nuq.n0;
  H->ectx.n1 = H->nuq.n1;
  H->ectx.coord = H->d_coord;
  H->ectx.tab = H->d_tab;
  H->ectx.gc = H->d_gc;
  if (prob->s_slope != 0.0) HM_TRY(variable_order_rows(H, st));

  // dense leaves and low-rank descriptors (host layout)
  int64_t off = 0, uo = 0, vo = 0;
  make_descs(P, *opts, H->h_dd, H->h_ld, off, uo, vo);
  H->d_pool = off;
  HM_TRY(A.upload(&H->d_dd, H->h_dd));
  HM_TRY(A.alloc((void**)&H->d_D, sizeof(double) * (size_t)std::max<int64_t>(off, 1)));
  HM_CK(cudaMemsetAsync(H->d_D, 0, sizeof(double) * (size_t)std::max<int64_t>(off, 1), st));
  HM_TRY(launch_near_fill(H->ectx, H->d_dd, (int)H->h_dd.size(), H->d_D, st));

  // admissible blocks: ACA
  for (const LRDesc& L : H->h_ld) {
    H->max_m = std::max(H->max_m, L.m);
    H->kmax = std::max(H->kmax, L.kcap);
  }
  H->u_pool = uo;
  H->v_pool = vo;
  const int nlr = (int)H->h_ld.size();
  HM_TRY(A.upload(&H->d_ld, H->h_ld));
  HM_TRY(A.alloc((void**)&H->d_rank, sizeof(int) * std::max(nlr, 1)));
  HM_TRY(A.alloc((void**)&H->d_capped, sizeof(int) * std::max(nlr, 1)));
  HM_TRY(A.alloc((void**)&H->d_U, sizeof(double) * (size_t)std::max<int64_t>(uo, 1)));
  HM_TRY(A.alloc((void**)&H->d_V, sizeof(double) * (size_t)std::max<int64_t>(vo, 1)));
  HM_TRY(launch_aca(H->ectx, H->d_ld, nlr, H->max_m, H->d_U, H->d_V, H->d_rank, H->d_capped,
                    opts->aca_tol, st));

  // H-matvec plan: row chunks over leaves, far-field V' x tasks
  std::vector<std::vector<int>> lr_by_row(P.cl.size()), dense_by_row(P.cl.size());
  for (int q = 0; q < nlr; ++q) lr_by_row[P.bl[P.lr_block[q]].t].push_back(q);
  for (int d = 0; d < (int)P.dense_block.size(); ++d) dense_by_row[P.bl[P.dense_block[d]].t].push_back(d);
  for (int leaf : P.leaves) {
    RowChunk base{};
    base.dense_begin = (int)H->h_dense_items.size();
    for (int d : dense_by_row[leaf]) H->h_dense_items.push_back(d);
    base.dense_end = (int)H->h_dense_items.size();
    base.lr_begin = (int)H->h_lr_items.size();
    for (int c = leaf; c >= 0; c = P.cl[c].parent)
      for (int q : lr_by_row[c]) H->h_lr_items.push_back(q);
    base.lr_end = (int)H->h_lr_items.size();
    const Cluster& L = P.cl[leaf];
    for (int r = L.begin; r < L.end; r += MV_CHUNK) {
      RowChunk ch = base;
      ch.r0 = r;
      ch.nrow = std::min(MV_CHUNK, L.end - r);
      H->h_chunks.push_back(ch);
    }
  }
  std::vector<VTask> vt;
  std::vector<int> vt_range(2 * (size_t)std::max(nlr, 1), 0);
  for (int q = 0; q < nlr; ++q) {
    vt_range[2 * q] = (int)vt.size();
    for (int c = 0; c < H->h_ld[q].n; c += VT_CHUNK) {
      VTask t{q, c, std::min(VT_CHUNK, H->h_ld[q].n - c), (int)vt.size()};
      vt.push_back(t);
    }
    vt_range[2 * q + 1] = (int)vt.size();
  }
  MatvecPlan& M = H->mv;
  M.nlr = nlr;
  M.ndense = (int)H->h_dd.size();
  M.nvt = (int)vt.size();
  M.nchunk = (int)H->h_chunks.size();
  M.ld = H->d_ld;
  M.dd = H->d_dd;
  M.rank = H->d_rank;
  M.U = H->d_U;
  M.V = H->d_V;
  M.D = H->d_D;
  M.kmax = H->kmax;
  VTask* d_vt = nullptr;
  int* d_vtr = nullptr;
  RowChunk* d_ch = nullptr;
  int* d_di = nullptr;
  int* d_li = nullptr;
  HM_TRY(A.upload(&d_vt, vt));
  HM_TRY(A.upload(&d_vtr, vt_range));
  HM_TRY(A.upload(&d_ch, H->h_chunks));
  HM_TRY(A.upload(&d_di, H->h_dense_items));
  HM_TRY(A.upload(&d_li, H->h_lr_items));
  M.vt = d_vt;
  M.vt_range = d_vtr;
  M.chunks = d_ch;
  M.dense_items = d_di;
  M.lr_items = d_li;
  HM_TRY(A.alloc((void**)&M.partial, sizeof(double) * (size_t)std::max(M.nvt, 1) * ACA_MAXK));
  HM_TRY(A.alloc((void**)&M.tvec, sizeof(double) * (size_t)std::max(nlr, 1) * ACA_MAXK));
  HM_TRY(A.alloc((void**)&H->d_work, sizeof(double) * (size_t)N * 8));

  HM_CK(cudaStreamSynchronize(st));
  H->h_rank.assign(nlr, 0);
  std::vector<int> capped(nlr, 0);
  if (nlr) {
    HM_CK(cudaMemcpy(H->h_rank.data(), H->d_rank, sizeof(int) * nlr, cudaMemcpyDeviceToHost));
    HM_CK(cudaMemcpy(capped.data(), H->d_capped, sizeof(int) * nlr, cudaMemcpyDeviceToHost));
  }
  H->capped_blocks = 0;
  for (int c : capped) H->capped_blocks += c;

  // low-rank storage compacted to the ranks ACA reached (it was sized for
  // the cap max_rank): U (m x rank) and V (n x rank), column-major
  if (nlr) {
    int64_t uo2 = 0, vo2 = 0;
    std::vector<LRDesc> ld2 = H->h_ld;
    std::vector<int64_t> ju, jv;  // (source offset, target offset, count) triples, in doubles
    for (int q = 0; q < nlr; ++q) {
      LRDesc& L = ld2[q];
      const int k = std::max(1, H->h_rank[q]);
      ju.insert(ju.end(), {H->h_ld[q].uoff, uo2, (int64_t)L.m * k});
      jv.insert(jv.end(), {H->h_ld[q].voff, vo2, (int64_t)L.n * k});
      L.uoff = uo2;
      L.voff = vo2;
      L.kcap = k;
      uo2 += ((int64_t)L.m * k + 3) & ~int64_t(3);
      vo2 += ((int64_t)L.n * k + 3) & ~int64_t(3);
    }
    double *U2 = nullptr, *V2 = nullptr;
    HM_TRY(A.alloc((void**)&U2, sizeof(double) * (size_t)std::max<int64_t>(uo2, 1)));
    HM_TRY(A.alloc((void**)&V2, sizeof(double) * (size_t)std::max<int64_t>(vo2, 1)));
    int64_t *d_ju = nullptr, *d_jv = nullptr;
    HM_TRY(A.upload(&d_ju, ju));
    HM_TRY(A.upload(&d_jv, jv));
    HM_TRY(launch_copy_segments(d_ju, nlr, H->d_U, U2, st));
    HM_TRY(launch_copy_segments(d_jv, nlr, H->d_V, V2, st));
    LRDesc* d_ld2 = nullptr;
    HM_TRY(A.upload(&d_ld2, ld2));
    HM_CK(cudaStreamSynchronize(st));
    A.free_one(H->d_U);
    A.free_one(H->d_V);
    A.free_one(H->d_ld);
    A.free_one(d_ju);
    A.free_one(d_jv);
    H->d_U = U2;
    H->d_V = V2;
    H->d_ld = d_ld2;
    H->h_ld = ld2;
    H->u_pool = uo2;
    H->v_pool = vo2;
    H->kmax = 1;
    for (const LRDesc& L : ld2) H->kmax = std::max(H->kmax, L.kcap);
    M.U = U2;
    M.V = V2;
    M.ld = d_ld2;
    M.kmax = H->kmax;
    uo = uo2;
    vo = vo2;
  }
  // split form G = S + J for constant-order problems on a box (HM_MATVEC_FP64=1: FP64 products)
  const char* mv64 = std::getenv("HM_MATVEC_FP64");
  if (prob->s_slope == 0.0 && prob->domain == HM_DOMAIN_BOX && !(mv64 && mv64[0] == '1')) {
    float2 *dj = nullptr, *udf = nullptr, *vdf = nullptr;
    HM_TRY(A.alloc((void**)&dj, sizeof(float2) * (size_t)std::max<int64_t>(off, 1)));
    HM_TRY(A.alloc((void**)&udf, sizeof(float2) * (size_t)std::max<int64_t>(uo, 1)));
    HM_TRY(A.alloc((void**)&vdf, sizeof(float2) * (size_t)std::max<int64_t>(vo, 1)));
    HM_TRY(A.alloc((void**)&M.tdf, sizeof(float2) * (size_t)std::max(nlr, 1) * ACA_MAXK));
    HM_TRY(launch_near_fill_jump(H->ectx, H->d_dd, (int)H->h_dd.size(), dj, st));
    HM_TRY(launch_split(H->d_U, udf, uo, st));
    HM_TRY(launch_split(H->d_V, vdf, vo, st));
    // axis neighbours of every Morton row: (-axis 0, +axis 0, -axis 1, +axis 1)
    std::vector<int4> nb(N);
    for (int q = 0; q < N; ++q) {
      const int i0 = P.coord[2 * q], i1 = P.coord[2 * q + 1];
      auto at = [&](int a0, int a1) {
        if (a0 < 0 || a0 >= P.n[0] || a1 < 0 || a1 >= P.n[1]) return -1;
        return P.iperm[(size_t)a1 * P.n[0] + a0];
      };
      nb[q] = make_int4(at(i0 - 1, i1), at(i0 + 1, i1), P.dim == 2 ? at(i0, i1 - 1) : -1,
                        P.dim == 2 ? at(i0, i1 + 1) : -1);
    }
    int4* d_nb = nullptr;
    HM_TRY(A.upload(&d_nb, nb));
    M.Ddf = dj;
    M.Udf = udf;
    M.Vdf = vdf;
    M.nb = d_nb;
    M.gc = H->d_gc;
  }
  HM_CK(cudaStreamSynchronize(st));
  return HM_OK;
}

int hm_build(const hm_problem* prob, const hm_opts* opts, void* stream, hm_matrix** out) {
  if (!out) { set_error("null out"); return HM_ERR_ARG; }
  *out = nullptr;
  hm_matrix* H = new hm_matrix();
  int s = build_impl(prob, opts, (cudaStream_t)stream, H);
  if (s != HM_OK) {
    cudaDeviceSynchronize();
    H->arena.release();
    delete H;
    return s;
  }
  *out = H;
  return HM_OK;
}

void hm_free(hm_matrix* H) {
  if (!H) return;
  cudaDeviceSynchronize();
  H->arena.release();
  delete H;
}

int hm_matvec(const hm_matrix* H, double alpha, double beta, const double* x, double gamma,
              const double* w1, const double* w2, double* y, void* stream) {
  if (!H || !x || !y) { set_error("null argument"); return HM_ERR_ARG; }
  if (x == y) { set_error("y must not alias x"); return HM_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const int N = H->plan.N;
  if (H->plan.dim == 1) return hm_matvec_morton(H, alpha, beta, x, gamma, w1, w2, nullptr, y, st);
  double* xm = H->d_work;
  double* ym = H->d_work + N;
  double* a = H->d_work + 2 * (size_t)N;
  double* b = H->d_work + 3 * (size_t)N;
  HM_TRY(launch_gather(H->d_perm, N, x, xm, st));
  if (w1) HM_TRY(launch_gather(H->d_perm, N, w1, a, st));
  if (w2) HM_TRY(launch_gather(H->d_perm, N, w2, b, st));
  HM_TRY(hm_matvec_morton(H, alpha, beta, xm, gamma, w1 ? a : nullptr, w2 ? b : nullptr, nullptr, ym, st));
  return launch_scatter(H->d_perm, N, ym, y, st);
}

int hm_matvec_noalloc(const hm_matrix* H, double alpha, double beta, const double* x, double gamma,
                      const double* w1, const double* w2, double* y, void* stream) {
  if (!H || !x || !y) { set_error("null argument"); return HM_ERR_ARG; }
  if (x == y) { set_error("y must not alias x"); return HM_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const int N = H->plan.N;
  const size_t part = (size_t)H->mv.nvt * ACA_MAXK, tv = (size_t)H->mv.nlr * ACA_MAXK;
  const size_t vecs = H->plan.dim == 2 ? 4 * (size_t)N : 0;
  const size_t need = part + tv + vecs;
  if (need > noalloc_capacity()) {
    set_error("hm_matvec_noalloc: this H-matrix needs " + std::to_string(need) +
              " doubles of scratch; the fixed scratch holds " + std::to_string(noalloc_capacity()));
    return HM_ERR_ARG;
  }
  double* s = nullptr;
  if (noalloc_scratch(&s) != HM_OK) { set_error("cudaGetSymbolAddress of the fixed scratch failed"); return HM_ERR_CUDA; }
  MatvecPlan Q = H->mv;
  Q.partial = s;
  Q.tvec = s + part;
  Q.Ddf = nullptr;  // FP64 products: the split form's float-pair coefficients would need more scratch
  Q.tdf = nullptr;
  if (H->plan.dim == 1) return launch_matvec(Q, alpha, beta, x, gamma, w1, w2, nullptr, y, st);
  double* xm = s + part + tv;
  double* ym = xm + N;
  double* a = ym + N;
  double* c = a + N;
  HM_TRY(launch_gather(H->d_perm, N, x, xm, st));
  if (w1) HM_TRY(launch_gather(H->d_perm, N, w1, a, st));
  if (w2) HM_TRY(launch_gather(H->d_perm, N, w2, c, st));
  HM_TRY(launch_matvec(Q, alpha, beta, xm, gamma, w1 ? a : nullptr, w2 ? c : nullptr, nullptr, ym, st));
  return launch_scatter(H->d_perm, N, ym, y, st);
}

int hm_to_dense(const hm_matrix* H, double* out, void* stream) {
  if (!H || !out) { set_error("null argument"); return HM_ERR_ARG; }
  return launch_to_dense(H->d_dd, (int)H->h_dd.size(), H->d_D, H->d_ld, (int)H->h_ld.size(),
                         H->d_rank, H->d_U, H->d_V, H->d_perm, H->plan.N, out, (cudaStream_t)stream);
}

int hm_entries(const hm_matrix* H, int64_t count, const int* rows, const int* cols, double* out,
               void* stream) {
  if (!H || count < 0 || (count > 0 && (!rows || !cols || !out))) { set_error("bad argument"); return HM_ERR_ARG; }
  return launch_entries(H->ectx, H->d_iperm, H->plan.N, count, rows, cols, out, H->d_err,
                        (cudaStream_t)stream);
}

int hm_sync(const hm_matrix* H, void* stream) {
  if (!H) { set_error("null argument"); return HM_ERR_ARG; }
  HM_CK(cudaStreamSynchronize((cudaStream_t)stream));
  int e = 0;
  HM_CK(cudaMemcpy(&e, H->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) { set_error("device error flags " + std::to_string(e)); return HM_ERR_DEVICE_ASSERT; }
  return HM_OK;
}

}  // extern "C"
