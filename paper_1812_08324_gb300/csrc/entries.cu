// Entry generation: row-independent constants, the offset table of w nu,
// and the dense near-field leaves (Eq. Aij; Eqs. I1approx, I2approx, I3approx).
#include <cmath>

#include "hm_device.cuh"
#include "hm_kernels.h"

namespace hm {

// Levy density at distance R (radial kernels; Sec. "H-matrix construction"
// for the Gaussian, Sec. "Singular ..." for the fractional Laplacian).
__device__ __forceinline__ double nu_radial(const NuParams& q, double R) {
  double v;
  if (q.kernel == HM_NU_GAUSS) v = q.lam * exp((-(q.eps * q.eps) * R) * R);
  else v = q.cds / pow(R, q.expo);
  return R <= q.trunc ? v : 0.0;
}

// rho(y) = (1 - (|y|/r)^4)^3 on |y| < r: C^2 window with 1 - rho = O(|y|^4)
// (Eq. rho_condition).
__device__ __forceinline__ double rho_win(double R, double r) {
  double t = R / r;
  if (t >= 1.0) return 0.0;
  double t4 = t * t * t * t;
  double u = 1.0 - t4;
  return u * u * u;
}

// tab[j1 * n0 + j0] = w(j) nu(|j| h), w = h^d halved per axis on the window face.
__global__ void nu_table_kernel(NuParams q, int n0, int n1, double* tab) {
  int64_t total = (int64_t)n0 * n1;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int j0 = (int)(t % n0), j1 = (int)(t / n0);
    if (j0 == 0 && j1 == 0) { tab[t] = 0.0; continue; }
    double w = q.dim == 1 ? q.h : q.h * q.h;
    if (j0 == q.nw) w = w * 0.5;
    if (q.dim == 2 && j1 == q.nw) w = w * 0.5;
    double y0 = j0 * q.h, y1 = j1 * q.h;
    double R = q.dim == 1 ? sqrt(y0 * y0) : sqrt(y0 * y0 + y1 * y1);
    tab[t] = w * nu_radial(q, R);
  }
}

// Window sums lambda_W = sum' w nu and D = sum' w rho nu y_0^2 over the whole
// window (offsets beyond the grid included), by quadrant with multiplicities.
__global__ void window_sums_kernel(NuParams q, double* out2) {
  __shared__ double sc[32];
  int nw = q.nw;
  int64_t cnt = q.dim == 1 ? (int64_t)(nw + 1) : (int64_t)(nw + 1) * (nw + 1);
  double lam = 0.0, dis = 0.0;
  for (int64_t t = threadIdx.x; t < cnt; t += blockDim.x) {
    int j0 = (int)(t % (nw + 1)), j1 = q.dim == 1 ? 0 : (int)(t / (nw + 1));
    if (j0 == 0 && j1 == 0) continue;
    double w = q.dim == 1 ? q.h : q.h * q.h;
    if (j0 == nw) w = w * 0.5;
    if (q.dim == 2 && j1 == nw) w = w * 0.5;
    double mult = (j0 > 0 ? 2.0 : 1.0) * (j1 > 0 ? 2.0 : 1.0);
    double y0 = j0 * q.h, y1 = j1 * q.h;
    double R = q.dim == 1 ? sqrt(y0 * y0) : sqrt(y0 * y0 + y1 * y1);
    double wn = w * nu_radial(q, R);
    lam += mult * wn;
    if (q.kernel == HM_NU_STABLE) {
      // per-axis second moment: average of the two axes is exact by symmetry
      double y2 = q.dim == 1 ? y0 * y0 : 0.5 * (y0 * y0 + y1 * y1);
      dis += mult * wn * rho_win(R, q.r) * y2;
    }
  }
  lam = block_sum(lam, sc);
  dis = block_sum(dis, sc);
  if (threadIdx.x == 0) { out2[0] = lam; out2[1] = dis; }
}

// T for the 2D square window: 8 int_0^{pi/4} radial(L_W / cos phi) dphi,
// radial(R) = int_R^{trunc} nu(rho) rho drho in closed form; composite Simpson.
__device__ double radial_tail(const NuParams& q, double R) {
  if (R >= q.trunc) return 0.0;
  if (q.kernel == HM_NU_STABLE) {
    double s = q.s;
    double hi = isinf(q.trunc) ? 0.0 : pow(q.trunc, -2.0 * s);
    return q.cds * (pow(R, -2.0 * s) - hi) / (2.0 * s);
  }
  double e2 = q.eps * q.eps;
  double hi = isinf(q.trunc) ? 0.0 : exp(-e2 * q.trunc * q.trunc);
  return q.lam * (exp(-e2 * R * R) - hi) / (2.0 * e2);
}

__global__ void tail2d_kernel(NuParams q, double* out) {
  __shared__ double sc[32];
  const int M = 1 << 14;  // Simpson intervals (even)
  const double a = 0.0, b = 0.78539816339744830962;
  double hs = (b - a) / M;
  double acc = 0.0;
  for (int i = threadIdx.x; i <= M; i += blockDim.x) {
    double phi = a + i * hs;
    double wgt = (i == 0 || i == M) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
    acc += wgt * radial_tail(q, q.LW / cos(phi));
  }
  acc = block_sum(acc, sc);
  if (threadIdx.x == 0) out[0] = 8.0 * acc * hs / 3.0;
}

// Dense near-field leaves: D[i, j] = G(r0 + i, c0 + j), row-major.
__global__ void near_fill_kernel(EntryCtx E, const DenseDesc* dd, double* pool) {
  const DenseDesc D = dd[blockIdx.x];
  const GenConst g = *E.gc;
  double* out = pool + D.off;
  int64_t tot = (int64_t)D.m * D.n;
  for (int64_t t = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.y * blockDim.x) {
    int i = (int)(t / D.n), j = (int)(t % D.n);
    out[(int64_t)i * D.ld + j] = gen_entry(E, g, D.r0 + i, D.c0 + j);
  }
}

// The jump entries of the dense leaves as float pairs (split form of the
// H-matvec): every entry but the diagonal from the offset table (no stencil:
// it is applied in FP64 from the constants), zero on the diagonal and in the
// row padding.  Constant-order problems only.
__global__ void near_fill_jump_kernel(EntryCtx E, const DenseDesc* dd, float2* pool) {
  const DenseDesc D = dd[blockIdx.x];
  float2* out = pool + D.off;
  const int64_t tot = (int64_t)D.m * D.ld;
  bool bad = false;
  for (int64_t t = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.y * blockDim.x) {
    const int i = (int)(t / D.ld), j = (int)(t % D.ld);
    const int p = D.r0 + i, q = D.c0 + j;
    out[(int64_t)i * D.ld + j] = (j < D.n && p != q) ? df_split(far_entry(E, p, q), bad) : make_float2(0.f, 0.f);
  }
}

// segments (source offset, target offset, count) of src copied into dst, one
// segment per CTA
__global__ void copy_segments_kernel(const int64_t* jobs, const double* src, double* dst) {
  const int64_t s = jobs[3 * (int64_t)blockIdx.x], d = jobs[3 * (int64_t)blockIdx.x + 1], n = jobs[3 * (int64_t)blockIdx.x + 2];
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) dst[d + e] = src[s + e];
}

__global__ void split_kernel(const double* src, float2* dst, int64_t n) {
  bool bad = false;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = df_split(src[e], bad);
}

__global__ void entries_kernel(EntryCtx E, const int* iperm, int N, int64_t count, const int* rows,
                               const int* cols, double* out, int* err) {
  const GenConst g = *E.gc;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x) {
    int r = rows[t], c = cols[t];
    if (r < 0 || r >= N || c < 0 || c >= N) { atomicOr(err, DEVERR_INDEX); out[t] = 0.0; continue; }
    out[t] = gen_entry(E, g, iperm[r], iperm[c]);
  }
}

// Expand the H-matrix into a dense natural-order N x N array.
__global__ void to_dense_dense_kernel(const DenseDesc* dd, const double* pool, const int* perm,
                                      int N, double* out) {
  const DenseDesc D = dd[blockIdx.x];
  int64_t tot = (int64_t)D.m * D.n;
  for (int64_t t = threadIdx.x; t < tot; t += blockDim.x) {
    int i = (int)(t / D.n), j = (int)(t % D.n);
    out[(int64_t)perm[D.r0 + i] * N + perm[D.c0 + j]] = pool[D.off + (int64_t)i * D.ld + j];
  }
}

__global__ void to_dense_lr_kernel(const LRDesc* ld, const int* rank, const double* U,
                                   const double* V, const int* perm, int N, double* out) {
  const LRDesc L = ld[blockIdx.x];
  int k = rank[blockIdx.x];
  int64_t tot = (int64_t)L.m * L.n;
  for (int64_t t = threadIdx.x; t < tot; t += blockDim.x) {
    int i = (int)(t / L.n), j = (int)(t % L.n);
    double acc = 0.0;
    for (int l = 0; l < k; ++l) acc += U[L.uoff + i + (int64_t)l * L.m] * V[L.voff + j + (int64_t)l * L.n];
    out[(int64_t)perm[L.r0 + i] * N + perm[L.c0 + j]] = acc;
  }
}

// ------------------------------------------------------------------ launchers

int launch_constants(const NuParams& q, double* d_tab, double* d_scratch, cudaStream_t st) {
  int64_t total = (int64_t)q.n0 * q.n1;
  int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  count_launches(q.dim == 2 ? 3 : 2);
  nu_table_kernel<<<grid, 256, 0, st>>>(q, q.n0, q.n1, d_tab);
  window_sums_kernel<<<1, 1024, 0, st>>>(q, d_scratch);
  if (q.dim == 2) tail2d_kernel<<<1, 1024, 0, st>>>(q, d_scratch + 2);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

int launch_near_fill(const EntryCtx& E, const DenseDesc* d_dd, int ndense, double* pool,
                     cudaStream_t st) {
  if (ndense == 0) return HM_OK;
  dim3 grid(ndense, 8);
  count_launches(1);
  near_fill_kernel<<<grid, 256, 0, st>>>(E, d_dd, pool);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

int launch_near_fill_jump(const EntryCtx& E, const DenseDesc* d_dd, int ndense, float2* pool, cudaStream_t st) {
  if (ndense == 0) return HM_OK;
  count_launches(1);
  dim3 grid(ndense, 16);
  near_fill_jump_kernel<<<grid, 256, 0, st>>>(E, d_dd, pool);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

int launch_copy_segments(const int64_t* d_jobs, int njobs, const double* src, double* dst, cudaStream_t st) {
  if (njobs <= 0) return HM_OK;
  count_launches(1);
  copy_segments_kernel<<<njobs, 256, 0, st>>>(d_jobs, src, dst);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

int launch_split(const double* src, float2* dst, int64_t n, cudaStream_t st) {
  if (n <= 0) return HM_OK;
  count_launches(1);
  split_kernel<<<1216, 256, 0, st>>>(src, dst, n);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

int launch_entries(const EntryCtx& E, const int* iperm, int N, int64_t count, const int* rows,
                   const int* cols, double* out, int* err, cudaStream_t st) {
  if (count <= 0) return HM_OK;
  int grid = (int)std::min<int64_t>((count + 255) / 256, 152 * 16);
  entries_kernel<<<grid, 256, 0, st>>>(E, iperm, N, count, rows, cols, out, err);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

int launch_to_dense(const DenseDesc* d_dd, int ndense, const double* pool, const LRDesc* d_ld,
                    int nlr, const int* rank, const double* U, const double* V, const int* perm,
                    int N, double* out, cudaStream_t st) {
  if (ndense) to_dense_dense_kernel<<<ndense, 256, 0, st>>>(d_dd, pool, perm, N, out);
  if (nlr) to_dense_lr_kernel<<<nlr, 256, 0, st>>>(d_ld, rank, U, V, perm, N, out);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

}  // namespace hm

namespace hm {

// Finish the row-independent constants: tail T (Eq. I2approx), the window
// correction kappa of the second difference (Eqs. I1approx, I3approx, with the
// closed-form moment int rho nu y_d^2 of rho = (1 - (|y|/r)^4)^3), the
// diagonal and the two axis stencils.
__global__ void finalize_constants_kernel(NuParams q, double a, double b0, double b1, double c,
                                          const double* sc, GenConst* gc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double h = q.h;
  const double d = (double)q.dim;
  const double PI = 3.14159265358979323846;
  double lam = sc[0], disc = sc[1];
  double T = 0.0;
  if (q.dim == 2) {
    T = sc[2];
  } else if (q.trunc > q.LW) {
    if (q.kernel == HM_NU_STABLE) {
      double hi = isinf(q.trunc) ? 0.0 : pow(q.trunc, -2.0 * q.s);
      T = (q.cds / q.s) * (pow(q.LW, -2.0 * q.s) - hi);
    } else {
      double hi = isinf(q.trunc) ? 0.0 : erfc(q.eps * q.trunc);
      T = q.lam * (sqrt(PI) / q.eps) * (erfc(q.eps * q.LW) - hi);
    }
  }
  double kappa = 0.0;
  if (q.kernel == HM_NU_STABLE) {
    double S = 0.0;
    const double binom[4] = {1.0, -3.0, 3.0, -1.0};
    for (int k = 0; k < 4; ++k) S += binom[k] / (2.0 - 2.0 * q.s + 4.0 * k);
    double rp = pow(q.r, 2.0 - 2.0 * q.s);
    double moment = q.dim == 1 ? 2.0 * q.cds * rp * S : PI * q.cds * rp * S;
    kappa = (moment - disc) / (2.0 * h * h);
  }
  GenConst g;
  g.h = h;
  g.a = a;
  g.b0 = b0;
  g.b1 = b1;
  g.c = c;
  g.lam_w = lam;
  g.tail = T;
  g.kappa = kappa;
  g.diag = c - 2.0 * d * a / (h * h) - 2.0 * d * kappa - lam - T;
  double base = kappa + a / (h * h);
  g.stencil_p[0] = base + b0 / (2.0 * h);
  g.stencil_m[0] = base + (-b0) / (2.0 * h);
  g.stencil_p[1] = base + b1 / (2.0 * h);
  g.stencil_m[1] = base + (-b1) / (2.0 * h);
  *gc = g;
}

int launch_finalize_constants(const NuParams& q, double a, const double* b, double c,
                              const double* d_scratch, GenConst* d_gc, cudaStream_t st) {
  count_launches(1);
  finalize_constants_kernel<<<1, 32, 0, st>>>(q, a, b[0], q.dim == 2 ? b[1] : 0.0, c, d_scratch, d_gc);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

}  // namespace hm
