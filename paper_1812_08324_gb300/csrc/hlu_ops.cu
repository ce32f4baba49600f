// Batched executors of the H-LU schedule (FP64): strided GEMM tiles, leaf LU
// with triangular inverses, low-rank truncation cores, copies and reductions.
#include <algorithm>

#include "hm_device.cuh"
#include "hlu_ops.h"
#include "hm_internal.h"

namespace hm {

namespace {

constexpr int GT = 32;   // GEMM output tile
constexpr int GK = 16;   // GEMM k chunk

__global__ void __launch_bounds__(256)
gemm_batch_kernel(const GemmOp* ops, const int* prefix, int nops) {
  __shared__ double As[GT][GK + 1];
  __shared__ double Bs[GK][GT + 1];
  const int tile = blockIdx.x;
  // locate the op owning this tile: prefix[o] <= tile < prefix[o + 1]
  int lo = 0, hi = nops - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= tile) lo = mid; else hi = mid - 1;
  }
  const GemmOp op = ops[lo];
  const int local = tile - prefix[lo];
  const int tn = (op.n + GT - 1) / GT;
  const int i0 = (local / tn) * GT, j0 = (local % tn) * GT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 2 x 2 outputs each
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int k0 = 0; k0 < op.k; k0 += GK) {
    for (int e = threadIdx.x; e < GT * GK; e += 256) {
      int r = e / GK, c = e % GK;
      int gi = i0 + r, gk = k0 + c;
      As[r][c] = (gi < op.m && gk < op.k) ? op.A[gi * op.ars + gk * op.acs] : 0.0;
    }
    for (int e = threadIdx.x; e < GK * GT; e += 256) {
      int r = e / GT, c = e % GT;
      int gk = k0 + r, gj = j0 + c;
      Bs[r][c] = (gk < op.k && gj < op.n) ? op.B[gk * op.brs + gj * op.bcs] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a0 = As[ty * 2][kk], a1 = As[ty * 2 + 1][kk];
      double b0 = Bs[kk][tx * 2], b1 = Bs[kk][tx * 2 + 1];
      acc[0][0] += a0 * b0;
      acc[0][1] += a0 * b1;
      acc[1][0] += a1 * b0;
      acc[1][1] += a1 * b1;
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      int gi = i0 + ty * 2 + a, gj = j0 + tx * 2 + b;
      if (gi < op.m && gj < op.n) {
        double* c = op.C + gi * op.crs + gj * op.ccs;
        double v = op.alpha * acc[a][b];
        *c = op.beta == 0.0 ? v : op.beta * (*c) + v;
      }
    }
}

// Base LU (m <= LU_BASE) in shared memory, then the inverses of L (unit
// lower) and U by substitution against the identity.
__global__ void lu_base_kernel(const LuOp* ops, int* err) {
  __shared__ double A[LU_BASE][LU_BASE + 1];
  __shared__ double X[LU_BASE][LU_BASE + 1];
  const LuOp op = ops[blockIdx.x];
  const int m = op.m, t = threadIdx.x;
  for (int e = t; e < m * m; e += blockDim.x) A[e / m][e % m] = op.A[(e / m) * op.lda + e % m];
  __syncthreads();
  for (int p = 0; p < m; ++p) {
    double piv = A[p][p];
    if (piv == 0.0 || !isfinite(piv)) {
      if (t == 0) atomicOr(err, DEVERR_ZEROPIVOT);
      piv = 1e-300;
    }
    __syncthreads();
    for (int i = p + 1 + t; i < m; i += blockDim.x) A[i][p] /= piv;
    __syncthreads();
    for (int e = t; e < (m - p - 1) * (m - p - 1); e += blockDim.x) {
      int i = p + 1 + e / (m - p - 1), j = p + 1 + e % (m - p - 1);
      A[i][j] -= A[i][p] * A[p][j];
    }
    __syncthreads();
  }
  // L^{-1}: column j by forward substitution (thread per column)
  if (t < m) {
    const int j = t;
    for (int i = 0; i < m; ++i) {
      double v = (i == j) ? 1.0 : 0.0;
      for (int k = j; k < i; ++k) v -= A[i][k] * X[k][j];
      X[i][j] = i < j ? 0.0 : v;
    }
  }
  __syncthreads();
  for (int e = t; e < m * m; e += blockDim.x) op.Li[(e / m) * op.ldl + e % m] = X[e / m][e % m];
  __syncthreads();
  // U^{-1}: column j by back substitution
  if (t < m) {
    const int j = t;
    for (int i = m - 1; i >= 0; --i) {
      double v = (i == j) ? 1.0 : 0.0;
      if (i > j) { X[i][j] = 0.0; continue; }
      for (int k = i + 1; k <= j; ++k) v -= A[i][k] * X[k][j];
      double d = A[i][i];
      X[i][j] = v / (d == 0.0 ? 1e-300 : d);
    }
  }
  __syncthreads();
  for (int e = t; e < m * m; e += blockDim.x) op.Ui[(e / m) * op.ldu + e % m] = X[e / m][e % m];
}

// ---- truncation core (one CTA): pivoted Cholesky of both Gram matrices,
// core C = R_A P_A' P_B R_B', column-pivoted Householder QR of C, then the
// coefficient matrices TA, TB (see TruncOp).
struct TruncSmem {
  double* GA;   // K x K
  double* GB;   // K x K
  double* C;    // K x K
};

// In-place pivoted Cholesky of the symmetric K x K matrix G (row-major);
// perm[c] = original index of pivot c; returns the rank (pivots above thresh).
__device__ int pivoted_cholesky(double* G, int K, int* perm, double rel_thresh, double* red_v,
                                int* red_i) {
  const int t = threadIdx.x;
  for (int c = t; c < K; c += blockDim.x) perm[c] = c;
  __syncthreads();
  double dmax0 = 0.0;
  for (int c = 0; c < K; ++c) dmax0 = fmax(dmax0, G[c * K + c]);
  const double thresh = rel_thresh * dmax0;
  int rank = 0;
  for (int p = 0; p < K; ++p) {
    __syncthreads();
    if (t == 0) {
      int q = p;
      double best = G[p * K + p];
      for (int j = p + 1; j < K; ++j)
        if (G[j * K + j] > best) { best = G[j * K + j]; q = j; }
      red_v[0] = best;
      red_i[0] = q;
    }
    __syncthreads();
    const double best = red_v[0];
    const int q = red_i[0];
    if (!(best > thresh) || dmax0 <= 0.0) break;
    // symmetric swap of p and q
    if (q != p) {
      for (int j = t; j < K; j += blockDim.x) {
        double a = G[p * K + j];
        G[p * K + j] = G[q * K + j];
        G[q * K + j] = a;
      }
      __syncthreads();
      for (int i = t; i < K; i += blockDim.x) {
        double a = G[i * K + p];
        G[i * K + p] = G[i * K + q];
        G[i * K + q] = a;
      }
      if (t == 0) {
        int a = perm[p];
        perm[p] = perm[q];
        perm[q] = a;
      }
      __syncthreads();
    }
    const double d = sqrt(best);
    __syncthreads();
    for (int j = p + t; j < K; j += blockDim.x) G[p * K + j] = (j == p) ? d : G[p * K + j] / d;
    __syncthreads();
    const int w = K - p - 1;
    for (int e = t; e < w * w; e += blockDim.x) {
      int i = p + 1 + e / w, j = p + 1 + e % w;
      G[i * K + j] -= G[p * K + i] * G[p * K + j];
    }
    ++rank;
  }
  __syncthreads();
  return rank;
}

__global__ void trunc_core_kernel(const TruncOp* ops, int* err) {
  extern __shared__ double sm[];
  __shared__ int permA[TRUNC_MAXK], permB[TRUNC_MAXK], permC[TRUNC_MAXK];
  __shared__ int posA[TRUNC_MAXK], posB[TRUNC_MAXK];
  __shared__ double cn[TRUNC_MAXK], tau[TRUNC_MAXK];
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  const TruncOp op = ops[blockIdx.x];
  const int K = op.K, kf = op.kf, t = threadIdx.x;
  double* GA = sm;
  double* GB = sm + K * K;
  double* C = sm + 2 * K * K;
  for (int e = t; e < K * K; e += blockDim.x) {
    GA[e] = op.GA[e];
    GB[e] = op.GB[e];
  }
  __syncthreads();
  // Gram entries below (tol/10)^2 of the largest carry nothing the truncation keeps
  const double rel = fmax(0.01 * op.tol * op.tol, 1e-15);
  const int rA = pivoted_cholesky(GA, K, permA, rel, red_v, red_i);
  const int rB = pivoted_cholesky(GB, K, permB, rel, red_v, red_i);
  for (int c = t; c < K; c += blockDim.x) {
    posA[permA[c]] = c;
    posB[permB[c]] = c;
  }
  __syncthreads();
  // C[i][j] = sum_o R_A[i][posA(o)] R_B[j][posB(o)]  (R upper: entry nonzero for col >= row)
  for (int e = t; e < rA * rB; e += blockDim.x) {
    int i = e / rB, j = e % rB;
    double acc = 0.0;
    for (int o = 0; o < K; ++o) {
      int ca = posA[o], cb = posB[o];
      if (ca >= i && cb >= j) acc += GA[i * K + ca] * GB[j * K + cb];
    }
    C[i * K + j] = acc;
  }
  __syncthreads();
  // Householder QR of C (rA x rB) with column pivoting; stop on the trailing norm
  for (int j = t; j < rB; j += blockDim.x) {
    permC[j] = j;
    double s = 0.0;
    for (int i = 0; i < rA; ++i) s += C[i * K + j] * C[i * K + j];
    cn[j] = s;
  }
  __syncthreads();
  double total = 0.0;
  for (int j = 0; j < rB; ++j) total += cn[j];
  int r = 0;
  const int rmax = min(min(rA, rB), kf);
  bool capped = false;
  for (int p = 0; p < min(rA, rB); ++p) {
    __syncthreads();
    if (t == 0) {
      double rem = 0.0;
      int q = p;
      double best = -1.0;
      for (int j = p; j < rB; ++j) {
        rem += cn[j];
        if (cn[j] > best) { best = cn[j]; q = j; }
      }
      red_v[0] = rem;
      red_i[0] = q;
    }
    __syncthreads();
    const double rem = red_v[0];
    if (!(rem > op.tol * op.tol * total) || total <= 0.0) break;
    if (p == rmax) { capped = true; break; }
    const int q = red_i[0];
    if (q != p) {
      for (int i = t; i < rA; i += blockDim.x) {
        double a = C[i * K + p];
        C[i * K + p] = C[i * K + q];
        C[i * K + q] = a;
      }
      if (t == 0) {
        int a = permC[p]; permC[p] = permC[q]; permC[q] = a;
        double b = cn[p]; cn[p] = cn[q]; cn[q] = b;
      }
    }
    __syncthreads();
    // Householder vector for column p, rows p..rA-1 (stored below the diagonal)
    if (t == 0) {
      double s = 0.0;
      for (int i = p; i < rA; ++i) s += C[i * K + p] * C[i * K + p];
      double nrm = sqrt(s);
      double x0 = C[p * K + p];
      double alpha = x0 >= 0.0 ? -nrm : nrm;
      double v0 = x0 - alpha;
      double vnorm2 = s - x0 * x0 + v0 * v0;
      tau[p] = (vnorm2 > 0.0) ? 2.0 / vnorm2 : 0.0;
      red_v[1] = v0;
      red_v[2] = alpha;
    }
    __syncthreads();
    const double v0 = red_v[1], alpha = red_v[2], tp = tau[p];
    // apply H = I - tau v v' to columns p+1.. (v = [v0, C[p+1..rA-1][p]])
    for (int j = p + 1 + t; j < rB; j += blockDim.x) {
      double dot = v0 * C[p * K + j];
      for (int i = p + 1; i < rA; ++i) dot += C[i * K + p] * C[i * K + j];
      dot *= tp;
      C[p * K + j] -= dot * v0;
      for (int i = p + 1; i < rA; ++i) C[i * K + j] -= dot * C[i * K + p];
      cn[j] -= C[p * K + j] * C[p * K + j];
    }
    __syncthreads();
    if (t == 0) {
      C[p * K + p] = alpha;  // R diagonal; v0 kept in red-free storage below
      cn[p] = v0;            // reuse: v0 of reflector p
    }
    __syncthreads();
    // trailing column norms, recomputed (no downdating drift)
    for (int j = p + 1 + t; j < rB; j += blockDim.x) {
      double s = 0.0;
      for (int i = p + 1; i < rA; ++i) s += C[i * K + j] * C[i * K + j];
      cn[j] = s;
    }
    ++r;
  }
  __syncthreads();
  // Q_C[:, :r]: apply reflectors to E = [I_r; 0], stored into GB's free rows? use TA scratch in global
  // Q (rA x r) is formed in the first rA x r entries of a scratch area: reuse GA rows >= rA? Not safe;
  // write Q into op.TA temporarily (K x kf, row-major) then overwrite with the final T_A.
  double* Q = op.TA;  // rows 0..rA-1, cols 0..r-1 (row-major with stride kf)
  for (int e = t; e < K * kf; e += blockDim.x) Q[e] = 0.0;
  __syncthreads();
  for (int c = t; c < r; c += blockDim.x) Q[c * kf + c] = 1.0;
  __syncthreads();
  for (int p = r - 1; p >= 0; --p) {
    const double v0 = cn[p], tp = tau[p];
    for (int c = t; c < r; c += blockDim.x) {
      double dot = v0 * Q[p * kf + c];
      for (int i = p + 1; i < rA; ++i) dot += C[i * K + p] * Q[i * kf + c];
      dot *= tp;
      Q[p * kf + c] -= dot * v0;
      for (int i = p + 1; i < rA; ++i) Q[i * kf + c] -= dot * C[i * K + p];
    }
    __syncthreads();
  }
  // T_A (pivoted rows) = R11_A^{-1} Q; R11_A is the leading rA x rA block of GA (upper)
  // solve in place column by column (back substitution), then scatter rows by permA.
  for (int c = t; c < r; c += blockDim.x) {
    for (int i = rA - 1; i >= 0; --i) {
      double v = Q[i * kf + c];
      for (int k = i + 1; k < rA; ++k) v -= GA[i * K + k] * Q[k * kf + c];
      Q[i * kf + c] = v / GA[i * K + i];
    }
  }
  __syncthreads();
  // move to original row order: use C's strictly-unused space? rows of TA are K x kf:
  // copy pivoted rows into smem GA (no longer needed after this point: R11_A consumed)
  for (int e = t; e < K * kf; e += blockDim.x) {
    int i = e / kf, c = e % kf;
    GA[e] = (i < rA && c < r) ? Q[i * kf + c] : 0.0;
  }
  __syncthreads();
  for (int e = t; e < K * kf; e += blockDim.x) {
    int i = e / kf, c = e % kf;
    op.TA[permA[i] * kf + c] = GA[i * kf + c];
  }
  // T_B (pivoted rows) = R11_B^{-1} Z, Z[j][c] = R_C[c][posC(j)] for j < rB
  __syncthreads();
  double* Z = C + 0;  // reuse? C holds R_C and reflectors needed for Z -> build Z in GA
  for (int e = t; e < K * kf; e += blockDim.x) {
    int j = e / kf, c = e % kf;
    double v = 0.0;
    if (j < rB && c < r) {
      // column j of C in original order sits at pivoted position pc where permC[pc] = j
      int pc = 0;
      for (int u = 0; u < rB; ++u)
        if (permC[u] == j) { pc = u; break; }
      v = (pc >= c) ? C[c * K + pc] : 0.0;
      if (pc == c) v = C[c * K + c];
    }
    GA[e] = v;
  }
  (void)Z;
  __syncthreads();
  for (int c = t; c < r; c += blockDim.x) {
    for (int i = rB - 1; i >= 0; --i) {
      double v = GA[i * kf + c];
      for (int k = i + 1; k < rB; ++k) v -= GB[i * K + k] * GA[k * kf + c];
      GA[i * kf + c] = v / GB[i * K + i];
    }
  }
  __syncthreads();
  for (int e = t; e < K * kf; e += blockDim.x) {
    int i = e / kf, c = e % kf;
    op.TB[permB[i] * kf + c] = (i < rB && c < r) ? GA[i * kf + c] : 0.0;
  }
  if (t == 0) {
    *op.rank = r;
    if (capped) atomicOr(err, DEVERR_RANKCAP);
  }
}

__global__ void copy_batch_kernel(const CopyOp* ops) {
  const CopyOp op = ops[blockIdx.y];
  const int64_t tot = (int64_t)op.m * op.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / op.n), j = (int)(e % op.n);
    double v = op.src ? op.alpha * op.src[i * op.srs + j * op.scs] : op.alpha;
    double* d = op.dst + i * op.drs + j * op.dcs;
    *d = op.beta == 0.0 ? v : op.beta * (*d) + v;
  }
}

__global__ void reduce_batch_kernel(const ReduceOp* ops) {
  const ReduceOp op = ops[blockIdx.y];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < op.count;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < op.nparts; ++p) s += op.parts[p * op.stride + i];
    op.dst[i] = s;
  }
}

}  // namespace

int gemm_tiles(int m, int n) { return ((m + GT - 1) / GT) * ((n + GT - 1) / GT); }

int upload_schedule(const std::vector<Wave>& waves, DevSchedule& S, std::vector<void*>& allocs) {
  std::vector<GemmOp> g;
  std::vector<LuOp> l;
  std::vector<TruncOp> tr;
  std::vector<CopyOp> c;
  std::vector<ReduceOp> r;
  std::vector<int> prefix;
  S.nwaves = (int)waves.size();
  S.begin.assign(5 * S.nwaves, 0);
  S.end.assign(5 * S.nwaves, 0);
  S.h_gemm_tiles_total.assign(S.nwaves, 0);
  for (int w = 0; w < S.nwaves; ++w) {
    const Wave& W = waves[w];
    S.begin[5 * w + 0] = (int)g.size();
    int tiles = 0;
    for (const GemmOp& o : W.gemm) {
      prefix.push_back(tiles);
      tiles += gemm_tiles(o.m, o.n);
      g.push_back(o);
    }
    S.end[5 * w + 0] = (int)g.size();
    S.h_gemm_tiles_total[w] = tiles;
    S.begin[5 * w + 1] = (int)l.size();
    l.insert(l.end(), W.lu.begin(), W.lu.end());
    S.end[5 * w + 1] = (int)l.size();
    S.begin[5 * w + 2] = (int)tr.size();
    tr.insert(tr.end(), W.trunc.begin(), W.trunc.end());
    S.end[5 * w + 2] = (int)tr.size();
    S.begin[5 * w + 3] = (int)c.size();
    c.insert(c.end(), W.copy.begin(), W.copy.end());
    S.end[5 * w + 3] = (int)c.size();
    S.begin[5 * w + 4] = (int)r.size();
    r.insert(r.end(), W.reduce.begin(), W.reduce.end());
    S.end[5 * w + 4] = (int)r.size();
  }
  auto up = [&](auto& vec, auto** dst) -> int {
    size_t bytes = std::max<size_t>(vec.size() * sizeof(vec[0]), 16);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return HM_ERR_OOM;
    allocs.push_back(p);
    if (!vec.empty() && cudaMemcpy(p, vec.data(), vec.size() * sizeof(vec[0]), cudaMemcpyHostToDevice) != cudaSuccess)
      return HM_ERR_CUDA;
    *dst = (std::remove_reference_t<decltype(**dst)>*)p;
    return HM_OK;
  };
  int s;
  if ((s = up(g, &S.gemm)) != HM_OK) return s;
  if ((s = up(l, &S.lu)) != HM_OK) return s;
  if ((s = up(tr, &S.trunc)) != HM_OK) return s;
  if ((s = up(c, &S.copy)) != HM_OK) return s;
  if ((s = up(r, &S.reduce)) != HM_OK) return s;
  if ((s = up(prefix, &S.gemm_tile_prefix)) != HM_OK) return s;
  return HM_OK;
}

int run_schedule(const DevSchedule& S, int* d_err, cudaStream_t st) {
  static bool attr_set = false;
  const size_t trunc_smem = 3 * sizeof(double) * TRUNC_MAXK * TRUNC_MAXK;
  if (!attr_set) {
    if (cudaFuncSetAttribute(trunc_core_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)trunc_smem) != cudaSuccess)
      return HM_ERR_CUDA;
    attr_set = true;
  }
  for (int w = 0; w < S.nwaves; ++w) {
    int b, e;
    b = S.begin[5 * w + 0]; e = S.end[5 * w + 0];
    if (e > b) gemm_batch_kernel<<<S.h_gemm_tiles_total[w], 256, 0, st>>>(S.gemm + b, S.gemm_tile_prefix + b, e - b);
    b = S.begin[5 * w + 1]; e = S.end[5 * w + 1];
    if (e > b) lu_base_kernel<<<e - b, 256, 0, st>>>(S.lu + b, d_err);
    b = S.begin[5 * w + 2]; e = S.end[5 * w + 2];
    if (e > b) trunc_core_kernel<<<e - b, 256, trunc_smem, st>>>(S.trunc + b, d_err);
    b = S.begin[5 * w + 3]; e = S.end[5 * w + 3];
    if (e > b) copy_batch_kernel<<<dim3(32, e - b), 256, 0, st>>>(S.copy + b);
    b = S.begin[5 * w + 4]; e = S.end[5 * w + 4];
    if (e > b) reduce_batch_kernel<<<dim3(16, e - b), 256, 0, st>>>(S.reduce + b);
  }
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

}  // namespace hm
