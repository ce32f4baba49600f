// Construction of the hierarchical inverses of the triangular factors
// (see hinv.h).  Bottom-up over the levels of the 1D cluster tree; at a
// level every cluster tau with children (a, b) gets its inverse block
//     L^{-1}: W = -X_b L_ba X_a   (rows b, columns a)
//     U^{-1}: W = -Y_a U_ab Y_b   (rows a, columns b)
// from two sketches made of products only:
//     range      R3 = X (T_off (X Omega))        = -W Omega     (Omega on the source rows)
//     co-range   C3 = X^T (T_off^T (X^T Psi))    = -W^T Psi     (Psi on the target rows)
// where X is the inverse formed so far (the leaves' inverses and the blocks
// of the deeper levels: block diagonal over the children) and T_off the
// factor blocks between the children.  With the core G = Psi^T R3 and its
// column-pivoted QR  G Pi = Q_c R  truncated at the first |R_kk| <= tol |R_00|,
//     W ~ -(R3 Pi_k R_11^{-1}) (C3 Q_c,k)^T        (generalised Nystrom).
// FP64 values; the products run in double-float arithmetic (below).
// Products are "multi-vector" kernels: a reduction
// T = V^T IN for every low-rank piece (chunks of 128 rows, the last CTA of a
// piece sums the chunks in order) and a row kernel summing, per 32-row chunk,
// its dense pieces (optionally one triangle) and its low-rank pieces U T.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include <cuda_bf16.h>

#include "hinv.h"
#include "hlu_plan.h"
#include "api_common.h"
#include "hm_device.cuh"
#include "hm_kernels.h"

namespace hm {

// ---- multi-vector products (construction only)
struct MrRed {          // T[slot] (k x S, row-major, stride S) = V^T IN[in0 : in0 + n, :]
  const double* V;
  int64_t vrs, vcs;     // V(j, l) = V[j * vrs + l * vcs]
  int in0, n;
  const int* rank;      // k = *rank (nullptr: kc)
  int kc;
  int c_begin, c_end;   // its reduction chunks
};
struct MrItem {         // contribution to the rows of a chunk
  int kind;             // 0: dense piece, 1: low-rank piece U T[slot]
  int mask;             // dense square pieces: 1 keeps j <= i, 2 keeps j >= i (local indices)
  const double* A;      // dense: A(i, j) = A[i rs + j cs]; low rank: U(i, l) = A[i rs + l cs]
  int64_t rs, cs;
  int row0;             // output row of local row 0
  int col0, ncol;       // dense: input rows read
  const int* rank;      // low rank: k = *rank (nullptr: kc)
  int kc, slot;
};
struct MrChunk { int r0, nr, ib, ie; };
struct MrPlan {
  const MrRed* reds;
  const int2* rch;      // (red item, first row) per reduction chunk
  int nrch;
  const MrChunk* chunks;
  int nchunk;
  const MrItem* items;
  double* partial;      // nrch x MAXS^2
  double* tbuf;         // red items x MAXS^2
  unsigned* count;      // per red item
  int S;                // columns of IN and OUT
};

constexpr int MR_T = HINV_MAXS * HINV_MAXS;

namespace {

__device__ __forceinline__ double urand(unsigned long long key) {
  // splitmix64 finaliser (Steele, Lea, Flood 2014) -> uniform in (-1, 1)
  unsigned long long z = key + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// rows [r0, r0 + n) of a row-major block of S columns get seeded uniform values
struct FillJob { double* buf; int r0, n, S; unsigned long long seed; };
__global__ void fill_kernel(const FillJob* jobs, int njobs) {
  const FillJob J = jobs[blockIdx.x];
  const int total = J.n * J.S;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int64_t i = J.r0 + e / J.S, c = e % J.S;
    J.buf[i * J.S + c] = urand(J.seed * 0x100000001B3ull + (unsigned long long)(i * HINV_MAXS + c));
  }
}

__global__ void __launch_bounds__(256) mr_red_kernel(MrPlan P, const double* __restrict__ in) {
  __shared__ int last;
  const int2 rc = P.rch[blockIdx.x];
  const MrRed R = P.reds[rc.x];
  const int k = R.rank ? *R.rank : R.kc;
  const int S = P.S;
  const int j0 = rc.y, len = min(HINV_MCH, R.n - j0);
  const int g = threadIdx.x & 7, lg = threadIdx.x >> 3;  // columns g + 8 q, pieces lg and lg + 32
  double acc[2][8];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[a][q] = 0.0;
  const bool l0 = lg < k, l1 = lg + 32 < k;
  if (l0) {
    for (int j = 0; j < len; ++j) {
      const int64_t jj = j0 + j;
      const double v0 = R.V[jj * R.vrs + (int64_t)lg * R.vcs];
      const double v1 = l1 ? R.V[jj * R.vrs + (int64_t)(lg + 32) * R.vcs] : 0.0;
      const double* x = in + (int64_t)(R.in0 + jj) * S;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int c = g + 8 * q;
        if (c < S) {
          const double xv = x[c];
          acc[0][q] = fma(v0, xv, acc[0][q]);
          acc[1][q] = fma(v1, xv, acc[1][q]);
        }
      }
    }
  }
  double* part = P.partial + (int64_t)blockIdx.x * MR_T;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int c = g + 8 * q;
    if (c < S) {
      if (l0) part[lg * S + c] = acc[0][q];
      if (l1) part[(lg + 32) * S + c] = acc[1][q];
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(P.count + rc.x, 1u) == (unsigned)(R.c_end - R.c_begin - 1) ? 1 : 0;
  __syncthreads();
  if (!last) return;
  __threadfence();
  double* T = P.tbuf + (int64_t)rc.x * MR_T;
  for (int e = threadIdx.x; e < k * S; e += blockDim.x) {
    double s = 0.0;
    for (int cc = R.c_begin; cc < R.c_end; ++cc) s += __ldcg(P.partial + (int64_t)cc * MR_T + e);
    T[e] = s;
  }
  if (threadIdx.x == 0) P.count[rc.x] = 0u;
}

__global__ void __launch_bounds__(256) mr_row_kernel(MrPlan P, const double* __restrict__ in, double* __restrict__ out) {
  const MrChunk C = P.chunks[blockIdx.x];
  const int S = P.S;
  const int g = threadIdx.x & 7, r = threadIdx.x >> 3;
  const int row = C.r0 + r;
  double acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = 0.0;
  for (int it = C.ib; it < C.ie; ++it) {
    const MrItem I = P.items[it];
    const int i = row - I.row0;  // local row of this thread
    if (I.kind == 0) {
      int jlo = 0, jhi = I.ncol;
      const int ifirst = C.r0 - I.row0, ilast = C.r0 + C.nr - 1 - I.row0;
      if (I.mask == 1) jhi = min(jhi, ilast + 1);
      if (I.mask == 2) jlo = max(0, ifirst);
      const double* arow = I.A + (int64_t)i * I.rs;
      for (int j = jlo; j < jhi; ++j) {
        double a = (r < C.nr) ? arow[(int64_t)j * I.cs] : 0.0;
        if ((I.mask == 1 && j > i) || (I.mask == 2 && j < i)) a = 0.0;
        const double* x = in + (int64_t)(I.col0 + j) * S;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int c = g + 8 * q;
          if (c < S) acc[q] = fma(a, x[c], acc[q]);
        }
      }
    } else {
      const int k = I.rank ? *I.rank : I.kc;
      const double* T = P.tbuf + (int64_t)I.slot * MR_T;
      const double* urow = I.A + (int64_t)i * I.rs;
      for (int l = 0; l < k; ++l) {
        const double u = (r < C.nr) ? urow[(int64_t)l * I.cs] : 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int c = g + 8 * q;
          if (c < S) acc[q] = fma(u, T[l * S + c], acc[q]);
        }
      }
    }
  }
  if (r < C.nr) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int c = g + 8 * q;
      if (c < S) out[(int64_t)row * S + c] = acc[q];
    }
  }
}

// ---- the same two products in double-float arithmetic on the FP32 pipes
// (FP64 runs at about two multiply-adds per clock per SM on this GPU): every
// FP64 operand is split into a float pair with integer operations (df_split),
// the vectors' rows are split once per CTA into shared memory, products and
// sums as Dekker / Knuth (about 48 significant bits, far below the sketches'
// truncation tolerances).  HM_HINV_BUILD_FP64=1 selects the FP64 kernels.
__device__ __forceinline__ void dd_mac(float2& s, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float t = __fadd_rn(s.x, p);
  const float bb = __fsub_rn(t, s.x);
  const float r = __fadd_rn(__fsub_rn(s.x, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  s.x = t;
  s.y = __fadd_rn(s.y, __fadd_rn(r, e));
}

constexpr int DD_JB = 32;  // rows of the input staged per block

template <int SC>
__global__ void __launch_bounds__(256) mr_red_dd_kernel(MrPlan P, const double* __restrict__ in) {
  __shared__ float2 xs[DD_JB][HINV_MAXS];
  __shared__ int last;
  const int2 rc = P.rch[blockIdx.x];
  const MrRed R = P.reds[rc.x];
  const int k = R.rank ? *R.rank : R.kc;
  constexpr int S = SC, NQ = SC / 8;  // columns per thread: NQ, all live
  const int j0 = rc.y, len = min(HINV_MCH, R.n - j0);
  const int g = threadIdx.x & 7, lg = threadIdx.x >> 3;
  const float2 z = make_float2(0.f, 0.f);
  float2 acc[2][8];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[a][q] = z;
  const bool l0 = lg < k, l1 = lg + 32 < k;
  bool bad = false;
  for (int jb = 0; jb < len; jb += DD_JB) {
    const int nb = min(DD_JB, len - jb);
    __syncthreads();
    for (int e = threadIdx.x; e < nb * S; e += blockDim.x) {
      const int r = e / S, c = e % S;
      xs[r][c] = df_split(in[(int64_t)(R.in0 + j0 + jb + r) * S + c], bad);
    }
    __syncthreads();
    if (l0) {
      for (int jq = 0; jq < nb; jq += 4) {  // four rows of V loaded before any is used
        double w0[4], w1[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t jj = j0 + jb + jq + u;
          const bool in = jq + u < nb;
          w0[u] = in ? R.V[jj * R.vrs + (int64_t)lg * R.vcs] : 0.0;
          w1[u] = in && l1 ? R.V[jj * R.vrs + (int64_t)(lg + 32) * R.vcs] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (jq + u >= nb) break;
          const float2 v0 = df_split(w0[u], bad);
          const float2 v1 = l1 ? df_split(w1[u], bad) : z;
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            const int c = g + 8 * q;
            {
              dd_mac(acc[0][q], v0, xs[jq + u][c]);
              if (l1) dd_mac(acc[1][q], v1, xs[jq + u][c]);
            }
          }
        }
      }
    }
  }
  double* part = P.partial + (int64_t)blockIdx.x * MR_T;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int c = g + 8 * q;
    {
      if (l0) part[lg * S + c] = (double)acc[0][q].x + (double)acc[0][q].y;
      if (l1) part[(lg + 32) * S + c] = (double)acc[1][q].x + (double)acc[1][q].y;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(P.count + rc.x, 1u) == (unsigned)(R.c_end - R.c_begin - 1) ? 1 : 0;
  __syncthreads();
  if (!last) return;
  __threadfence();
  double* T = P.tbuf + (int64_t)rc.x * MR_T;
  for (int e = threadIdx.x; e < k * S; e += blockDim.x) {
    double s = 0.0;
    for (int cc = R.c_begin; cc < R.c_end; ++cc) s += __ldcg(P.partial + (int64_t)cc * MR_T + e);
    T[e] = s;
  }
  if (threadIdx.x == 0) P.count[rc.x] = 0u;
}

template <int SC>
__global__ void __launch_bounds__(256) mr_row_dd_kernel(MrPlan P, const double* __restrict__ in,
                                                         double* __restrict__ out) {
  constexpr int JB = 64;
  __shared__ float2 xs[JB][HINV_MAXS];
  const MrChunk C = P.chunks[blockIdx.x];
  constexpr int S = SC, NQ = SC / 8;  // columns per thread: NQ, all live
  const int g = threadIdx.x & 7, r = threadIdx.x >> 3;
  const int row = C.r0 + r;
  const bool live = r < C.nr;
  const float2 z = make_float2(0.f, 0.f);
  float2 acc[8];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = z;
  bool bad = false;
  for (int it = C.ib; it < C.ie; ++it) {
    const MrItem I = P.items[it];
    const int i = row - I.row0;
    if (I.kind == 0) {
      int jlo = 0, jhi = I.ncol;
      const int ifirst = C.r0 - I.row0, ilast = C.r0 + C.nr - 1 - I.row0;
      if (I.mask == 1) jhi = min(jhi, ilast + 1);
      if (I.mask == 2) jlo = max(0, ifirst);
      const double* arow = I.A + (int64_t)i * I.rs;
      for (int jb = jlo; jb < jhi; jb += JB) {
        const int nb = min(JB, jhi - jb);
        __syncthreads();
        for (int e = threadIdx.x; e < nb * S; e += blockDim.x) {
          const int rr = e / S, c = e % S;
          xs[rr][c] = df_split(in[(int64_t)(I.col0 + jb + rr) * S + c], bad);
        }
        __syncthreads();
        if (live) {
          // eight matrix entries loaded before any is used
          for (int j0 = jb; j0 < jb + nb; j0 += 8) {
            double av[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int j = j0 + u;
              const bool keep = j < jb + nb && !((I.mask == 1 && j > i) || (I.mask == 2 && j < i));
              av[u] = keep ? arow[(int64_t)j * I.cs] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              if (j0 + u >= jb + nb) break;
              const float2 a = df_split(av[u], bad);
#pragma unroll
              for (int q = 0; q < NQ; ++q) {
                const int c = g + 8 * q;
                dd_mac(acc[q], a, xs[j0 + u - jb][c]);
              }
            }
          }
        }
      }
    } else {
      const int k = I.rank ? *I.rank : I.kc;
      const double* T = P.tbuf + (int64_t)I.slot * MR_T;
      const double* urow = I.A + (int64_t)i * I.rs;
      for (int lb = 0; lb < k; lb += JB) {
        const int nb = min(JB, k - lb);
        __syncthreads();
        for (int e = threadIdx.x; e < nb * S; e += blockDim.x) {
          const int rr = e / S, c = e % S;
          xs[rr][c] = df_split(T[(lb + rr) * S + c], bad);
        }
        __syncthreads();
        if (live) {
          for (int l0 = lb; l0 < lb + nb; l0 += 8) {
            double uv[8];
#pragma unroll
            for (int w = 0; w < 8; ++w) uv[w] = l0 + w < lb + nb ? urow[(int64_t)(l0 + w) * I.cs] : 0.0;
#pragma unroll
            for (int w = 0; w < 8; ++w) {
              if (l0 + w >= lb + nb) break;
              const float2 u = df_split(uv[w], bad);
#pragma unroll
              for (int q = 0; q < NQ; ++q) {
                const int c = g + 8 * q;
                dd_mac(acc[q], u, xs[l0 + w - lb][c]);
              }
            }
          }
        }
      }
    }
  }
  if (live) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int c = g + 8 * q;
      out[(int64_t)row * S + c] = (double)acc[q].x + (double)acc[q].y;
    }
  }
}

// ---- column-pivoted Householder QR of the core G (SP x S, row-major, stride
// S) of one block, truncated at |R_kk| <= tol |R_00| or the rank cap.  Writes
// the rank, the pivots, R_11^{-1} (k x k) and the first k columns of Q_c.
struct Core {
  int k, capped, pad[2];
  int piv[HINV_S];
  double rinv[HINV_KCAP * HINV_KCAP];  // row-major
  double qc[HINV_SP * HINV_KCAP];      // row-major SP x KCAP
};

struct CoreOut {   // where the rank of core b goes, and its truncation tolerance
  int* rank;
  double tol;
};
__global__ void __launch_bounds__(256) cpqr_kernel(const double* __restrict__ tbuf, Core* cores,
                                                   const CoreOut* core_out, int* err) {
  constexpr int M = HINV_SP, NC = HINV_S;
  __shared__ double A[M][NC + 1];
  __shared__ double nrm2[NC];
  __shared__ double tauv[HINV_KCAP], diagR[HINV_KCAP];
  __shared__ int piv[NC];
  __shared__ int s_p, s_stop;
  __shared__ double s_ref, s_norm;
  const int b = blockIdx.x;
  const double tol = core_out[b].tol;
  const double* G = tbuf + (int64_t)b * MR_T;  // the core of block b is reduction slot b
  for (int e = threadIdx.x; e < M * NC; e += blockDim.x) A[e / NC][e % NC] = G[e];
  if (threadIdx.x < NC) piv[threadIdx.x] = threadIdx.x;
  __syncthreads();
  int k = 0;
  int capped = 0;
  for (int j = 0; j < NC && j < M; ++j) {
    if (threadIdx.x < NC && threadIdx.x >= j) {
      double s = 0.0;
      for (int i = j; i < M; ++i) s = fma(A[i][threadIdx.x], A[i][threadIdx.x], s);
      nrm2[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int p = j;
      for (int c = j + 1; c < NC; ++c)
        if (nrm2[c] > nrm2[p]) p = c;
      const double nm = sqrt(nrm2[p]);
      if (j == 0) s_ref = nm;
      int stop = !(nm > tol * s_ref) || nm == 0.0 || !isfinite(nm);
      if (!stop && j == HINV_KCAP) { stop = 1; capped = 1; }
      s_stop = stop;
      s_p = p;
      s_norm = nm;
    }
    __syncthreads();
    if (s_stop) break;
    const int p = s_p;
    if (p != j) {
      for (int i = threadIdx.x; i < M; i += blockDim.x) {
        const double t = A[i][j];
        A[i][j] = A[i][p];
        A[i][p] = t;
      }
      if (threadIdx.x == 0) {
        const int t = piv[j];
        piv[j] = piv[p];
        piv[p] = t;
      }
    }
    __syncthreads();
    // Householder reflector H = I - tau v v^T with v = x - alpha e_1, alpha = -sign(x_0) |x|
    if (threadIdx.x == 0) {
      const double x0 = A[j][j];
      const double alpha = x0 >= 0.0 ? -s_norm : s_norm;
      const double v0 = x0 - alpha;
      tauv[j] = -1.0 / (alpha * v0);
      diagR[j] = alpha;
      A[j][j] = v0;
    }
    __syncthreads();
    const int c = j + 1 + (int)threadIdx.x;
    if (c < NC) {
      double d = 0.0;
      for (int i = j; i < M; ++i) d = fma(A[i][j], A[i][c], d);
      d *= tauv[j];
      for (int i = j; i < M; ++i) A[i][c] = fma(-d, A[i][j], A[i][c]);
    }
    __syncthreads();
    k = j + 1;
  }
  Core* out = cores + b;
  // R_11^{-1}: thread per column, back substitution (R_ii = diagR, R_ic = A[i][c] for i < c)
  if ((int)threadIdx.x < k) {
    const int c = threadIdx.x;
    double x[HINV_KCAP];
    for (int i = 0; i < HINV_KCAP; ++i) x[i] = 0.0;
    x[c] = 1.0 / diagR[c];
    for (int i = c - 1; i >= 0; --i) {
      double s = 0.0;
      for (int m = i + 1; m <= c; ++m) s = fma(A[i][m], x[m], s);
      x[i] = -s / diagR[i];
    }
    for (int i = 0; i < HINV_KCAP; ++i) out->rinv[i * HINV_KCAP + c] = i <= c ? x[i] : 0.0;
  }
  // Q_c columns: e_c through the reflectors in reverse order
  if ((int)threadIdx.x < k) {
    const int c = threadIdx.x;
    double q[M];
    for (int i = 0; i < M; ++i) q[i] = i == c ? 1.0 : 0.0;
    for (int h = k - 1; h >= 0; --h) {
      double d = 0.0;
      for (int i = h; i < M; ++i) d = fma(A[i][h], q[i], d);
      d *= tauv[h];
      for (int i = h; i < M; ++i) q[i] = fma(-d, A[i][h], q[i]);
    }
    for (int i = 0; i < M; ++i) out->qc[i * HINV_KCAP + c] = q[i];
  }
  if (threadIdx.x < NC) out->piv[threadIdx.x] = piv[threadIdx.x];
  if (threadIdx.x == 0) {
    out->k = k;
    out->capped = capped;
    *core_out[b].rank = k;
    if (!isfinite(s_ref)) atomicOr(err, DEVERR_NONFINITE);
  }
}

// P = -R3[tgt rows][:, piv_k] R_11^{-1}, Q = C3[src rows] Q_c,k (both
// column-major, column stride ld); zero beyond k
struct FormJob { int which, core, node_row0, nrow, r_lo; double* dst; int ld; const double* src; int S; };
__global__ void __launch_bounds__(256) form_kernel(const FormJob* jobs, const Core* cores) {
  const FormJob J = jobs[blockIdx.x];
  const Core& K = cores[J.core];
  const int k = K.k;
  const int g = threadIdx.x & 7, r = threadIdx.x >> 3;
  const int i = J.r_lo + r;  // local row of the block
  if (i >= J.nrow || r >= HINV_RCH) return;
  const double* x = J.src + (int64_t)(J.node_row0 + i) * J.S;
  for (int l = g; l < HINV_KCAP; l += 8) {
    double s = 0.0;
    if (l < k) {
      if (J.which == 0) {
        for (int c = 0; c <= l; ++c) s = fma(x[K.piv[c]], K.rinv[c * HINV_KCAP + l], s);
        s = -s;
      } else {
        for (int c = 0; c < HINV_SP; ++c) s = fma(x[c], K.qc[c * HINV_KCAP + l], s);
      }
    }
    J.dst[(int64_t)l * J.ld + i] = s;
  }
}

// leaf inverse (row-major, stride sld) -> its triangle, column-major with
// column stride ld, zeros elsewhere (padding rows included)
struct LeafCopy { const double* src; int64_t sld; double* dst; int ld, m, lower; };
__global__ void leaf_copy_kernel(const LeafCopy* jobs) {
  const LeafCopy J = jobs[blockIdx.x];
  const int64_t total = (int64_t)J.m * J.ld;
  for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
    const int j = (int)(e / J.ld), i = (int)(e % J.ld);
    const bool keep = i < J.m && (J.lower ? j <= i : j >= i);
    J.dst[e] = keep ? J.src[(int64_t)i * J.sld + j] : 0.0;
  }
}

// FP64 pools -> the per-step storage: FP32, BF16, or pairs of floats
// (hi = v rounded to float, lo = the rest rounded to float: 48 bits of v)
template <class T>
__global__ void convert_kernel(const double* src, T* dst, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = src[e];
    if constexpr (sizeof(T) == 8) {
      const float hi = __double2float_rn(v);
      dst[e] = make_float2(hi, __double2float_rn(v - (double)hi));
    } else if constexpr (sizeof(T) == 4) {
      dst[e] = (float)v;
    } else {
      dst[e] = __double2bfloat16(v);
    }
  }
}

}  // namespace

// ---------------------------------------------------------------- host side

void HinvData::release() {
  for (void* p : allocs) cudaFree(p);
  allocs.clear();
  bytes = 0;
}

namespace {

int round8(int n) { return (n + 7) & ~7; }

// Host image of one multi-vector product; its arrays live in shared host
// vectors (one upload for every plan of the construction).
struct HostMr {
  int S = 0;
  int red0 = 0, nred = 0;      // into all reds
  int rch0 = 0, nrch = 0;      // into all rch
  int ch0 = 0, nch = 0;        // into all chunks
  int it0 = 0;                 // into all items
};

static_assert(HINV_S % 8 == 0 && HINV_SP % 8 == 0 && HINV_SP <= HINV_MAXS, "multi-vector widths: whole groups of 8");

struct Planner {
  std::vector<MrRed> reds;
  std::vector<int2> rch;
  std::vector<MrChunk> chunks;
  std::vector<MrItem> items;
  HostMr cur;
  int max_red = 0, max_rch = 0;
  int base = 0;  // row offset of the current problem in the shared buffers (added to every row below)

  void begin(int S) {
    cur = HostMr();
    cur.S = S;
    cur.red0 = (int)reds.size();
    cur.rch0 = (int)rch.size();
    cur.ch0 = (int)chunks.size();
    cur.it0 = (int)items.size();
  }
  // T slot = returned id (relative to the plan)
  int red(const double* V, int64_t vrs, int64_t vcs, int in0, int n, const int* rank, int kc) {
    MrRed R{V, vrs, vcs, in0 + base, n, rank, kc, (int)rch.size() - cur.rch0, 0};
    const int id = (int)reds.size() - cur.red0;
    for (int j0 = 0; j0 < n; j0 += HINV_MCH) rch.push_back(make_int2(id, j0));
    R.c_end = (int)rch.size() - cur.rch0;
    reds.push_back(R);
    return id;
  }
  void chunk(int r0, int nr) { chunks.push_back(MrChunk{r0 + base, nr, (int)items.size() - cur.it0, 0}); }
  void item(MrItem I) {
    I.row0 += base;
    if (I.kind == 0) I.col0 += base;
    items.push_back(I);
    chunks.back().ie = (int)items.size() - cur.it0;
  }
  HostMr end() {
    cur.nred = (int)reds.size() - cur.red0;
    cur.nrch = (int)rch.size() - cur.rch0;
    cur.nch = (int)chunks.size() - cur.ch0;
    max_red = std::max(max_red, cur.nred);
    max_rch = std::max(max_rch, cur.nrch);
    return cur;
  }
};

MrItem dense_item(const double* A, int64_t rs, int64_t cs, int row0, int col0, int ncol, int mask) {
  MrItem I{};
  I.kind = 0;
  I.mask = mask;
  I.A = A;
  I.rs = rs;
  I.cs = cs;
  I.row0 = row0;
  I.col0 = col0;
  I.ncol = ncol;
  return I;
}
MrItem lr_item(const double* U, int64_t rs, int64_t cs, int row0, const int* rank, int kc, int slot) {
  MrItem I{};
  I.kind = 1;
  I.A = U;
  I.rs = rs;
  I.cs = cs;
  I.row0 = row0;
  I.rank = rank;
  I.kc = kc;
  I.slot = slot;
  return I;
}

struct TNode {   // an internal cluster of the 1D tree
  int cl, level;
  int a, b;      // children (clusters)
};

struct OffBlock { bool lowrank; int id; int t, s; };

// One problem of a construction: its tree, the factor blocks between
// children, its pools and its first row in the shared construction buffers.
struct Ctx {
  const Plan* P = nullptr;
  const std::vector<DenseDesc>* dd = nullptr;
  const FactorLayout* F = nullptr;
  const int* d_rank_f = nullptr;
  HinvData* out = nullptr;
  double tol = 0.0;
  int N = 0, nl = 0, nn = 0, maxlev = -1;
  int base = 0;
  std::vector<int> dense_of_leaf, node_of;
  std::vector<TNode> nodes;
  std::vector<std::vector<int>> anc_t[2], anc_s[2];  // per leaf: nodes whose target (source) holds it, upwards
  std::vector<std::vector<int>> level_nodes;
  std::vector<std::vector<OffBlock>> toff[2];        // per node: factor blocks between its children
  int* d_rank = nullptr;                             // 2 x nn inverse-block ranks
  double* leafpool[2] = {nullptr, nullptr};
  double* ppool[2] = {nullptr, nullptr};
  double* qpool[2] = {nullptr, nullptr};
  int64_t leaf_elems = 0, p_elems[2] = {0, 0}, q_elems[2] = {0, 0};
  std::vector<int> h_rank;

  std::pair<int, int> range(int c) const { return std::make_pair(P->cl[c].begin, P->cl[c].end); }
  // per triangle: target and source cluster of a node
  static int tgt(int tri, const TNode& T) { return tri == 0 ? T.b : T.a; }
  static int src(int tri, const TNode& T) { return tri == 0 ? T.a : T.b; }
};

int out_alloc(HinvData& out, void** p, size_t bytes, std::string& err) {
  *p = nullptr;
  if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
    cudaGetLastError();
    err = "device allocation of " + std::to_string(bytes) + " bytes failed";
    return HM_ERR_OOM;
  }
  out.allocs.push_back(*p);
  out.bytes += (int64_t)std::max<size_t>(bytes, 16);
  return HM_OK;
}

template <class T>
int out_upload(HinvData& out, T** dst, const std::vector<T>& vec, cudaStream_t st, std::string& err) {
  const size_t n = vec.size() * sizeof(T);
  void* p = nullptr;
  HM_TRY(out_alloc(out, &p, n, err));
  if (n && cudaMemcpyAsync(p, vec.data(), n, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    err = std::string("table upload failed: ") + cudaGetErrorString(cudaGetLastError());
    return HM_ERR_CUDA;
  }
  *dst = (T*)p;
  return HM_OK;
}

// The tree, the ancestors of every leaf and the blocks between children, and
// the layout of the per-step pools (host only).
int ctx_prepare(Ctx& C, std::string& err) {
  const Plan& P = *C.P;
  const FactorLayout& F = *C.F;
  const std::vector<DenseDesc>& dd = *C.dd;
  if (P.dim != 1) { err = "hierarchical inverses are built for 1D problems only"; return HM_ERR_ARG; }
  if (F.kf > HINV_MAXS) { err = "factor rank cap above 64"; return HM_ERR_ARG; }
  if (P.depth > HINV_MAX_ANC) { err = "cluster tree deeper than " + std::to_string(HINV_MAX_ANC); return HM_ERR_ARG; }
  C.N = P.N;
  // ---- tree: leaves (Morton order) with their diagonal dense block, internal nodes
  C.nl = (int)P.leaves.size();
  const int nl = C.nl;
  std::vector<int> leaf_of(P.cl.size(), -1);
  C.dense_of_leaf.assign(nl, -1);
  for (int l = 0; l < nl; ++l) leaf_of[P.leaves[l]] = l;
  for (int d = 0; d < (int)dd.size(); ++d) {
    if (dd[d].r0 != dd[d].c0) continue;
    const int t = P.bl[P.dense_block[d]].t;
    if (leaf_of[t] >= 0) C.dense_of_leaf[leaf_of[t]] = d;
  }
  for (int l = 0; l < nl; ++l) {
    const int d = C.dense_of_leaf[l];
    if (d < 0 || !F.linv[d] || !F.uinv[d]) { err = "a leaf has no inverse of its factors"; return HM_ERR_ARG; }
    if (P.cl[P.leaves[l]].end - P.cl[P.leaves[l]].begin > 1024) { err = "leaves above 1024 rows"; return HM_ERR_ARG; }
  }
  C.node_of.assign(P.cl.size(), -1);
  for (int c = 0; c < (int)P.cl.size(); ++c) {
    if (P.cl[c].nchild == 0) continue;
    if (P.cl[c].nchild != 2) { err = "the 1D cluster tree must be binary"; return HM_ERR_ARG; }
    C.node_of[c] = (int)C.nodes.size();
    C.nodes.push_back(TNode{c, P.cl[c].level, P.cl[c].child[0], P.cl[c].child[1]});
    C.maxlev = std::max(C.maxlev, P.cl[c].level);
  }
  C.nn = (int)C.nodes.size();
  const int nn = C.nn;
  C.level_nodes.assign(std::max(C.maxlev + 1, 0), {});
  for (int v = 0; v < nn; ++v) C.level_nodes[C.nodes[v].level].push_back(v);
  for (int tri = 0; tri < 2; ++tri) {
    C.anc_t[tri].resize(nl);
    C.anc_s[tri].resize(nl);
    for (int l = 0; l < nl; ++l) {
      int c = P.leaves[l];
      while (P.cl[c].parent >= 0) {
        const int par = P.cl[c].parent;
        const TNode& T = C.nodes[C.node_of[par]];
        if (Ctx::tgt(tri, T) == c) C.anc_t[tri][l].push_back(C.node_of[par]);
        else C.anc_s[tri][l].push_back(C.node_of[par]);
        c = par;
      }
    }
  }
  // ---- factor blocks between the children of each node (T_off), by triangle
  C.toff[0].assign(nn, {});
  C.toff[1].assign(nn, {});
  auto lca = [&](int t, int s) {
    int c = t;
    while (!(P.cl[c].begin <= P.cl[s].begin && P.cl[s].end <= P.cl[c].end)) c = P.cl[c].parent;
    return c;
  };
  for (int d = 0; d < (int)dd.size(); ++d) {
    const Block& B = P.bl[P.dense_block[d]];
    if (B.t == B.s) continue;
    const int A = lca(B.t, B.s);
    const bool lower = P.cl[B.t].begin >= P.cl[P.cl[A].child[1]].begin;
    C.toff[lower ? 0 : 1][C.node_of[A]].push_back(OffBlock{false, d, B.t, B.s});
  }
  for (int q = 0; q < (int)P.lr_block.size(); ++q) {
    const Block& B = P.bl[P.lr_block[q]];
    const int A = lca(B.t, B.s);
    const bool lower = P.cl[B.t].begin >= P.cl[P.cl[A].child[1]].begin;
    C.toff[lower ? 0 : 1][C.node_of[A]].push_back(OffBlock{true, q, B.t, B.s});
  }
  // ---- layout of the pools: leaves, P, Q
  C.leaf_elems = 0;
  for (int l = 0; l < nl; ++l) {
    const int m = P.cl[P.leaves[l]].end - P.cl[P.leaves[l]].begin;
    C.leaf_elems += (int64_t)m * round8(m);
  }
  for (int tri = 0; tri < 2; ++tri) {
    HinvTriangle& H = C.out->tri[tri];
    H.h_leaves.resize(nl);
    H.h_nodes.resize(nn);
    int64_t lo = 0, po = 0, qo = 0;
    for (int l = 0; l < nl; ++l) {
      const auto r = C.range(P.leaves[l]);
      HinvLeaf& L = H.h_leaves[l];
      L.r0 = r.first;
      L.m = r.second - r.first;
      L.ld = round8(L.m);
      L.off = lo;
      lo += (int64_t)L.m * L.ld;
    }
    for (int v = 0; v < nn; ++v) {
      HinvNode& Nd = H.h_nodes[v];
      const auto rt = C.range(Ctx::tgt(tri, C.nodes[v])), rs = C.range(Ctx::src(tri, C.nodes[v]));
      Nd.tgt0 = rt.first;
      Nd.tgt_n = rt.second - rt.first;
      Nd.src0 = rs.first;
      Nd.src_n = rs.second - rs.first;
      Nd.pld = round8(Nd.tgt_n);
      Nd.qld = round8(Nd.src_n);
      Nd.poff = po;
      Nd.qoff = qo;
      po += (int64_t)Nd.pld * HINV_KCAP;
      qo += (int64_t)Nd.qld * HINV_KCAP;
    }
    C.p_elems[tri] = po;
    C.q_elems[tri] = qo;
  }
  return HM_OK;
}

// X (transposed or not) on the source (target) part of every node of the
// level: the leaf inverses and the inverse blocks of the deeper levels
void plan_x(Planner& PL, const Ctx& C, int tri, int lev, bool trans, bool on_src) {
  const HinvTriangle& H = C.out->tri[tri];
  const int* rk = C.d_rank + tri * C.nn;
  std::vector<int> slot(C.nn, -1);
  for (int v : C.level_nodes[lev]) {
    const int part = on_src ? Ctx::src(tri, C.nodes[v]) : Ctx::tgt(tri, C.nodes[v]);
    const auto pr = C.range(part);
    for (int l = 0; l < C.nl; ++l) {
      const HinvLeaf& L = H.h_leaves[l];
      if (L.r0 < pr.first || L.r0 + L.m > pr.second) continue;
      const std::vector<int>& anc = trans ? C.anc_s[tri][l] : C.anc_t[tri][l];
      for (int q : anc) {
        if (C.nodes[q].level <= lev || slot[q] >= 0) continue;
        const HinvNode& Q = H.h_nodes[q];
        slot[q] = trans ? PL.red(C.ppool[tri] + Q.poff, 1, Q.pld, Q.tgt0, Q.tgt_n, rk + q, HINV_KCAP)
                        : PL.red(C.qpool[tri] + Q.qoff, 1, Q.qld, Q.src0, Q.src_n, rk + q, HINV_KCAP);
      }
      for (int i0 = 0; i0 < L.m; i0 += HINV_RCH) {
        PL.chunk(L.r0 + i0, std::min(HINV_RCH, L.m - i0));
        const double* X = C.leafpool[tri] + L.off;
        const int mask = (tri == 0) != trans ? 1 : 2;
        // the leaf is stored column-major: X(i, j) = X[j ld + i]
        PL.item(trans ? dense_item(X, L.ld, 1, L.r0, L.r0, L.m, mask)
                      : dense_item(X, 1, L.ld, L.r0, L.r0, L.m, mask));
        for (int q : anc) {
          if (C.nodes[q].level <= lev) continue;
          const HinvNode& Q = H.h_nodes[q];
          PL.item(trans ? lr_item(C.qpool[tri] + Q.qoff, 1, Q.qld, Q.src0, rk + q, HINV_KCAP, slot[q])
                        : lr_item(C.ppool[tri] + Q.poff, 1, Q.pld, Q.tgt0, rk + q, HINV_KCAP, slot[q]));
        }
      }
    }
  }
}

// T_off (transposed or not) of every node of the level: output rows = its
// target (source) part
void plan_t(Planner& PL, const Ctx& C, int tri, int lev, bool trans) {
  const Plan& P = *C.P;
  const FactorLayout& F = *C.F;
  const HinvTriangle& H = C.out->tri[tri];
  const int kf = F.kf;
  for (int v : C.level_nodes[lev]) {
    const int part = trans ? Ctx::src(tri, C.nodes[v]) : Ctx::tgt(tri, C.nodes[v]);
    const auto pr = C.range(part);
    const std::vector<OffBlock>& ob = C.toff[tri][v];
    std::vector<int> slot(ob.size(), -1);
    for (size_t k = 0; k < ob.size(); ++k) {
      if (!ob[k].lowrank) continue;
      const int q = ob[k].id;
      const int m = P.cl[ob[k].t].end - P.cl[ob[k].t].begin, n = P.cl[ob[k].s].end - P.cl[ob[k].s].begin;
      slot[k] = trans ? PL.red(F.lr_u[q], 1, m, P.cl[ob[k].t].begin, m, C.d_rank_f + q, kf)
                      : PL.red(F.lr_v[q], 1, n, P.cl[ob[k].s].begin, n, C.d_rank_f + q, kf);
    }
    for (int l = 0; l < C.nl; ++l) {
      const HinvLeaf& L = H.h_leaves[l];
      if (L.r0 < pr.first || L.r0 + L.m > pr.second) continue;
      for (int i0 = 0; i0 < L.m; i0 += HINV_RCH) {
        PL.chunk(L.r0 + i0, std::min(HINV_RCH, L.m - i0));
        for (size_t k = 0; k < ob.size(); ++k) {
          const Cluster& T = P.cl[ob[k].t];
          const Cluster& Sc = P.cl[ob[k].s];
          const Cluster& out_cl = trans ? Sc : T;
          if (L.r0 < out_cl.begin || L.r0 + L.m > out_cl.end) continue;
          if (!ob[k].lowrank) {
            const View& V = F.dense[ob[k].id];
            PL.item(trans ? dense_item(V.p, V.cs, V.rs, Sc.begin, T.begin, T.end - T.begin, 0)
                          : dense_item(V.p, V.rs, V.cs, T.begin, Sc.begin, Sc.end - Sc.begin, 0));
          } else {
            const int q = ob[k].id;
            const int m = T.end - T.begin, n = Sc.end - Sc.begin;
            PL.item(trans ? lr_item(F.lr_v[q], 1, n, Sc.begin, C.d_rank_f + q, kf, slot[k])
                          : lr_item(F.lr_u[q], 1, m, T.begin, C.d_rank_f + q, kf, slot[k]));
          }
        }
      }
    }
  }
}

// The inverses of a group of problems.  The problems' rows are stacked in the
// shared construction buffers; every construction step (level, triangle)
// runs for all problems with nodes on that level in one launch per kernel.
// The values do not depend on the grouping: every reduction sums its chunks
// in a fixed order, the sketches are seeded by level, triangle and the
// problem's own row.  Synchronises the stream.
int build_group(std::vector<Ctx>& G, int* d_err, cudaStream_t st, std::string& err) {
  const auto t_start = std::chrono::steady_clock::now();
  std::vector<void*> tmp;
  auto free_tmp = [&]() {
    for (void* p : tmp) cudaFree(p);
    tmp.clear();
  };
  auto tmp_alloc = [&](void** p, size_t bytes) -> int {
    *p = nullptr;
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      cudaGetLastError();
      err = "device allocation of construction buffers failed";
      return HM_ERR_OOM;
    }
    tmp.push_back(*p);
    return HM_OK;
  };
  auto tmp_upload = [&](auto** dst, const auto& vec) -> int {
    const size_t n = vec.size() * sizeof(vec[0]);
    void* p = nullptr;
    HM_TRY(tmp_alloc(&p, n));
    if (n && cudaMemcpyAsync(p, vec.data(), n, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      err = std::string("construction table upload failed: ") + cudaGetErrorString(cudaGetLastError());
      return HM_ERR_CUDA;
    }
    *dst = (std::remove_reference_t<decltype(**dst)>*)p;
    return HM_OK;
  };
  auto fail = [&](int s) {
    free_tmp();
    if (err.empty()) err = "hierarchical inverse construction failed";
    return s;
  };
  // ---- rows in the shared buffers; pools (FP64: the construction's; they
  // are the per-step storage only in FP64, otherwise one shared temporary)
  int64_t rows = 0, tmp_pool = 0;
  auto pad32 = [](int64_t n) { return (n + 31) & ~int64_t(31); };
  int gmax = -1;
  for (Ctx& C : G) {
    if (rows + C.N > INT32_MAX) return fail(HM_ERR_ARG);
    C.base = (int)rows;
    rows += C.N;
    gmax = std::max(gmax, C.maxlev);
    if (C.out->prec != HINV_F64)
      for (int tri = 0; tri < 2; ++tri) tmp_pool += pad32(C.p_elems[tri]) + pad32(C.q_elems[tri]) + pad32(C.leaf_elems);
  }
  int s = HM_OK;
  double* pool64 = nullptr;
  if ((s = tmp_alloc((void**)&pool64, sizeof(double) * std::max<int64_t>(tmp_pool, 1))) != HM_OK) return fail(s);
  // P and Q pools first (one clear for all), then the leaves
  int64_t at = 0;
  for (Ctx& C : G)
    if (C.out->prec != HINV_F64)
      for (int tri = 0; tri < 2; ++tri) {
        C.ppool[tri] = pool64 + at;
        at += pad32(C.p_elems[tri]);
        C.qpool[tri] = pool64 + at;
        at += pad32(C.q_elems[tri]);
      }
  const int64_t pq_elems = at;
  for (Ctx& C : G)
    if (C.out->prec != HINV_F64)
      for (int tri = 0; tri < 2; ++tri) {
        C.leafpool[tri] = pool64 + at;
        at += pad32(C.leaf_elems);
      }
  if (pq_elems && cudaMemsetAsync(pool64, 0, sizeof(double) * pq_elems, st) != cudaSuccess) {
    err = "clearing the inverse pools failed";
    return fail(HM_ERR_CUDA);
  }
  for (Ctx& C : G) {
    HinvData& out = *C.out;
    if ((s = out_alloc(out, (void**)&C.d_rank, sizeof(int) * 2 * std::max(C.nn, 1), err)) != HM_OK) return fail(s);
    if (cudaMemsetAsync(C.d_rank, 0, sizeof(int) * 2 * std::max(C.nn, 1), st) != cudaSuccess) {
      err = std::string("clearing the ranks failed: ") + cudaGetErrorString(cudaGetLastError());
      return fail(HM_ERR_CUDA);
    }
    if (out.prec != HINV_F64) continue;
    for (int tri = 0; tri < 2; ++tri) {
      if ((s = out_alloc(out, (void**)&C.leafpool[tri], sizeof(double) * std::max<int64_t>(C.leaf_elems, 1), err)) != HM_OK ||
          (s = out_alloc(out, (void**)&C.ppool[tri], sizeof(double) * std::max<int64_t>(C.p_elems[tri], 1), err)) != HM_OK ||
          (s = out_alloc(out, (void**)&C.qpool[tri], sizeof(double) * std::max<int64_t>(C.q_elems[tri], 1), err)) != HM_OK)
        return fail(s);
      if (cudaMemsetAsync(C.ppool[tri], 0, sizeof(double) * std::max<int64_t>(C.p_elems[tri], 1), st) != cudaSuccess ||
          cudaMemsetAsync(C.qpool[tri], 0, sizeof(double) * std::max<int64_t>(C.q_elems[tri], 1), st) != cudaSuccess) {
        err = "clearing the inverse pools failed";
        return fail(HM_ERR_CUDA);
      }
    }
  }
  // ---- leaf inverses -> triangles (one launch)
  {
    std::vector<LeafCopy> lc;
    for (Ctx& C : G)
      for (int tri = 0; tri < 2; ++tri)
        for (int l = 0; l < C.nl; ++l) {
          const int d = C.dense_of_leaf[l];
          const HinvLeaf& L = C.out->tri[tri].h_leaves[l];
          lc.push_back(LeafCopy{tri == 0 ? C.F->linv[d] : C.F->uinv[d], C.F->linv_ld[d], C.leafpool[tri] + L.off, L.ld,
                                L.m, tri == 0 ? 1 : 0});
        }
    LeafCopy* d_lc = nullptr;
    if ((s = tmp_upload(&d_lc, lc)) != HM_OK) return fail(s);
    if (!lc.empty()) {
      count_launches(1);
      leaf_copy_kernel<<<(unsigned)lc.size(), 256, 0, st>>>(d_lc);
    }
  }
  // ---- shared construction buffers (rows x width, row-major), per triangle
  double* bufA[2];
  double* bufB[2];
  double* bufC[2];
  double* bufD[2];
  double* bufE[2];
  for (int tri = 0; tri < 2; ++tri) {
    double* blk = nullptr;
    if ((s = tmp_alloc((void**)&blk, sizeof(double) * std::max<int64_t>(rows, 1) * (2 * HINV_S + 3 * HINV_SP))) != HM_OK)
      return fail(s);
    bufA[tri] = blk;
    bufB[tri] = bufA[tri] + rows * HINV_S;
    bufC[tri] = bufB[tri] + rows * HINV_S;
    bufD[tri] = bufC[tri] + rows * HINV_SP;
    bufE[tri] = bufD[tri] + rows * HINV_SP;
  }
  // ---- construction plans, level by level (deepest first), both triangles
  Planner PL;
  struct Step {
    int tri, level;
    HostMr mr[7];              // XR, TR, XR2, XC, TC, XC2, gram
    std::vector<FillJob> fill;
    std::vector<FormJob> form;
    std::vector<CoreOut> core_out;  // per core (reduction slot of the gram plan)
  };
  std::vector<Step> steps;
  for (int lev = gmax; lev >= 0; --lev) {
    std::vector<Ctx*> on;  // problems with nodes on this level
    for (Ctx& C : G)
      if (lev <= C.maxlev && !C.level_nodes[lev].empty()) on.push_back(&C);
    if (on.empty()) continue;
    for (int tri = 0; tri < 2; ++tri) {
      Step S;
      S.tri = tri;
      S.level = lev;
      auto plan_all = [&](int width, auto&& body) {
        PL.begin(width);
        for (Ctx* C : on) {
          PL.base = C->base;
          body(*C);
        }
        PL.base = 0;
        return PL.end();
      };
      S.mr[0] = plan_all(HINV_S, [&](const Ctx& C) { plan_x(PL, C, tri, lev, false, true); });
      S.mr[1] = plan_all(HINV_S, [&](const Ctx& C) { plan_t(PL, C, tri, lev, false); });
      S.mr[2] = plan_all(HINV_S, [&](const Ctx& C) { plan_x(PL, C, tri, lev, false, false); });
      S.mr[3] = plan_all(HINV_SP, [&](const Ctx& C) { plan_x(PL, C, tri, lev, true, false); });
      S.mr[4] = plan_all(HINV_SP, [&](const Ctx& C) { plan_t(PL, C, tri, lev, true); });
      S.mr[5] = plan_all(HINV_SP, [&](const Ctx& C) { plan_x(PL, C, tri, lev, true, true); });
      S.mr[6] = plan_all(HINV_S, [&](const Ctx& C) {
        for (int v : C.level_nodes[lev]) {
          const HinvNode& Nd = C.out->tri[tri].h_nodes[v];
          PL.red(bufC[tri] + ((int64_t)C.base + Nd.tgt0) * HINV_SP, HINV_SP, 1, Nd.tgt0, Nd.tgt_n, nullptr, HINV_SP);
        }
      });
      const unsigned long long seed = 1000003ull * (unsigned long long)(lev + 1) + 17ull * tri;
      int b = 0;
      for (Ctx* C : on) {
        double* A0 = bufA[tri] + (int64_t)C->base * HINV_S;
        double* B0 = bufB[tri] + (int64_t)C->base * HINV_S;
        double* C0 = bufC[tri] + (int64_t)C->base * HINV_SP;
        double* D0 = bufD[tri] + (int64_t)C->base * HINV_SP;
        for (int v : C->level_nodes[lev]) {
          const HinvNode& Nd = C->out->tri[tri].h_nodes[v];
          // 128-row pieces (one CTA each; the values depend on the problem's own row only)
          for (int r = 0; r < Nd.src_n; r += HINV_MCH)
            S.fill.push_back(FillJob{A0, Nd.src0 + r, std::min(HINV_MCH, Nd.src_n - r), HINV_S, 2 * seed});
          for (int r = 0; r < Nd.tgt_n; r += HINV_MCH)
            S.fill.push_back(FillJob{C0, Nd.tgt0 + r, std::min(HINV_MCH, Nd.tgt_n - r), HINV_SP, 2 * seed + 1});
          S.core_out.push_back(CoreOut{C->d_rank + tri * C->nn + v, C->tol});
          for (int r = 0; r < Nd.tgt_n; r += HINV_RCH)
            S.form.push_back(FormJob{0, b, Nd.tgt0, Nd.tgt_n, r, C->ppool[tri] + Nd.poff, Nd.pld, B0, HINV_S});
          for (int r = 0; r < Nd.src_n; r += HINV_RCH)
            S.form.push_back(FormJob{1, b, Nd.src0, Nd.src_n, r, C->qpool[tri] + Nd.qoff, Nd.qld, D0, HINV_SP});
          ++b;
        }
      }
      steps.push_back(std::move(S));
    }
  }
  // ---- upload every plan at once, then run the steps in order
  std::vector<FillJob> all_fill;
  std::vector<FormJob> all_form;
  std::vector<CoreOut> all_core;
  std::vector<int> fill_off, form_off, core_off;
  int max_cores = 1;
  for (const Step& S : steps) {
    fill_off.push_back((int)all_fill.size());
    form_off.push_back((int)all_form.size());
    core_off.push_back((int)all_core.size());
    all_fill.insert(all_fill.end(), S.fill.begin(), S.fill.end());
    all_form.insert(all_form.end(), S.form.begin(), S.form.end());
    all_core.insert(all_core.end(), S.core_out.begin(), S.core_out.end());
    max_cores = std::max(max_cores, (int)S.core_out.size());
  }
  MrRed* d_reds = nullptr;
  int2* d_rch = nullptr;
  MrChunk* d_chunks = nullptr;
  MrItem* d_items = nullptr;
  FillJob* d_fill = nullptr;
  FormJob* d_form = nullptr;
  CoreOut* d_core = nullptr;
  double* d_partial = nullptr;
  double* d_tbuf = nullptr;
  unsigned* d_count = nullptr;
  Core* d_cores = nullptr;
  if (s == HM_OK) s = tmp_upload(&d_reds, PL.reds);
  if (s == HM_OK) s = tmp_upload(&d_rch, PL.rch);
  if (s == HM_OK) s = tmp_upload(&d_chunks, PL.chunks);
  if (s == HM_OK) s = tmp_upload(&d_items, PL.items);
  if (s == HM_OK) s = tmp_upload(&d_fill, all_fill);
  if (s == HM_OK) s = tmp_upload(&d_form, all_form);
  if (s == HM_OK) s = tmp_upload(&d_core, all_core);
  if (s == HM_OK) s = tmp_alloc((void**)&d_partial, sizeof(double) * std::max(PL.max_rch, 1) * MR_T);
  if (s == HM_OK) s = tmp_alloc((void**)&d_tbuf, sizeof(double) * std::max(PL.max_red, 1) * MR_T);
  if (s == HM_OK) s = tmp_alloc((void**)&d_count, sizeof(unsigned) * std::max(PL.max_red, 1));
  if (s == HM_OK) s = tmp_alloc((void**)&d_cores, sizeof(Core) * max_cores);
  if (s == HM_OK && cudaMemsetAsync(d_count, 0, sizeof(unsigned) * std::max(PL.max_red, 1), st) != cudaSuccess)
    s = HM_ERR_CUDA;
  if (s != HM_OK) return fail(s);
  const char* b64 = std::getenv("HM_HINV_BUILD_FP64");  // FP64 products in the construction (checks)
  const bool build_fp64 = b64 && b64[0] == '1';
  auto run_mr = [&](const HostMr& h, const double* in, double* o) {
    MrPlan M{d_reds + h.red0, d_rch + h.rch0, h.nrch, d_chunks + h.ch0, h.nch, d_items + h.it0,
             d_partial, d_tbuf, d_count, h.S};
    if (h.nrch > 0) {
      count_launches(1);
      if (build_fp64) mr_red_kernel<<<h.nrch, 256, 0, st>>>(M, in);
      else if (h.S == HINV_S) mr_red_dd_kernel<HINV_S><<<h.nrch, 256, 0, st>>>(M, in);
      else mr_red_dd_kernel<HINV_SP><<<h.nrch, 256, 0, st>>>(M, in);
    }
    if (h.nch > 0 && o) {
      count_launches(1);
      if (build_fp64) mr_row_kernel<<<h.nch, 256, 0, st>>>(M, in, o);
      else if (h.S == HINV_S) mr_row_dd_kernel<HINV_S><<<h.nch, 256, 0, st>>>(M, in, o);
      else mr_row_dd_kernel<HINV_SP><<<h.nch, 256, 0, st>>>(M, in, o);
    }
  };
  for (size_t k = 0; k < steps.size(); ++k) {
    const Step& S = steps[k];
    const int t = S.tri;
    if (!S.fill.empty()) {
      count_launches(1);
      fill_kernel<<<(unsigned)S.fill.size(), 256, 0, st>>>(d_fill + fill_off[k], (int)S.fill.size());
    }
    run_mr(S.mr[0], bufA[t], bufB[t]);   // X Omega          (source rows)
    run_mr(S.mr[1], bufB[t], bufA[t]);   // T_off X Omega    (target rows)
    run_mr(S.mr[2], bufA[t], bufB[t]);   // R3               (target rows)
    run_mr(S.mr[3], bufC[t], bufD[t]);   // X^T Psi          (target rows)
    run_mr(S.mr[4], bufD[t], bufE[t]);   // T_off^T X^T Psi  (source rows)
    run_mr(S.mr[5], bufE[t], bufD[t]);   // C3               (source rows)
    run_mr(S.mr[6], bufB[t], nullptr);   // cores Psi^T R3 in slots 0..
    const int nb = (int)S.core_out.size();
    count_launches(2);
    cpqr_kernel<<<nb, 256, 0, st>>>(d_tbuf, d_cores, d_core + core_off[k], d_err);
    form_kernel<<<(unsigned)S.form.size(), 256, 0, st>>>(d_form + form_off[k], d_cores);
  }
  if (cudaGetLastError() != cudaSuccess) {
    err = "construction launch failed";
    return fail(HM_ERR_CUDA);
  }
  // ---- per-step tables and storage of every problem
  for (Ctx& C : G) {
    HinvData& out = *C.out;
    const int aprec = out.prec;
    for (int tri = 0; tri < 2 && s == HM_OK; ++tri) {
      HinvTriangle& H = out.tri[tri];
      int ntch = 0;
      for (int v = 0; v < C.nn; ++v) {
        HinvNode& Nd = H.h_nodes[v];
        Nd.tch_begin = ntch;
        ntch += (Nd.src_n + HINV_TCH - 1) / HINV_TCH;
        Nd.tch_end = ntch;
      }
      HinvApply& A = H.A64;
      A.lower = tri == 0 ? 1 : 0;
      A.prec = HINV_F64;
      A.nleaf = C.nl;
      A.nnode = C.nn;
      A.ntch = ntch;
      A.nrch = 0;  // the chunk tables follow once the ranks are on the host
      if (s == HM_OK) s = out_upload(out, (HinvNode**)&A.nodes, H.h_nodes, st, err);
      A.leaf_pool = C.leafpool[tri];
      A.p_pool = C.ppool[tri];
      A.q_pool = C.qpool[tri];
      A.rank = C.d_rank + tri * C.nn;
      if (s == HM_OK) s = out_alloc(out, (void**)&A.tpart, sizeof(double) * HINV_KCAP * std::max(ntch, 1), err);
      if (s == HM_OK) s = out_alloc(out, (void**)&A.tvec, sizeof(double) * HINV_KCAP * std::max(C.nn, 1), err);
      if (s == HM_OK) s = out_alloc(out, (void**)&A.tcount, sizeof(unsigned) * std::max(C.nn, 1), err);
      if (s == HM_OK && cudaMemsetAsync(A.tcount, 0, sizeof(unsigned) * std::max(C.nn, 1), st) != cudaSuccess)
        s = HM_ERR_CUDA;
      H.A = A;
      if (s == HM_OK && aprec != HINV_F64) {
        const size_t es = aprec == HINV_DF ? 8 : (aprec == HINV_F32 ? 4 : 2);
        void* pl = nullptr;
        void* pp = nullptr;
        void* pq = nullptr;
        if (s == HM_OK) s = out_alloc(out, &pl, es * std::max<int64_t>(C.leaf_elems, 1), err);
        if (s == HM_OK) s = out_alloc(out, &pp, es * std::max<int64_t>(C.p_elems[tri], 1), err);
        if (s == HM_OK) s = out_alloc(out, &pq, es * std::max<int64_t>(C.q_elems[tri], 1), err);
        if (s == HM_OK) {
          count_launches(3);
          if (aprec == HINV_DF) {
            convert_kernel<float2><<<1216, 256, 0, st>>>(C.leafpool[tri], (float2*)pl, C.leaf_elems);
            convert_kernel<float2><<<1216, 256, 0, st>>>(C.ppool[tri], (float2*)pp, C.p_elems[tri]);
            convert_kernel<float2><<<1216, 256, 0, st>>>(C.qpool[tri], (float2*)pq, C.q_elems[tri]);
          } else if (aprec == HINV_F32) {
            convert_kernel<float><<<1216, 256, 0, st>>>(C.leafpool[tri], (float*)pl, C.leaf_elems);
            convert_kernel<float><<<1216, 256, 0, st>>>(C.ppool[tri], (float*)pp, C.p_elems[tri]);
            convert_kernel<float><<<1216, 256, 0, st>>>(C.qpool[tri], (float*)pq, C.q_elems[tri]);
          } else {
            convert_kernel<__nv_bfloat16><<<1216, 256, 0, st>>>(C.leafpool[tri], (__nv_bfloat16*)pl, C.leaf_elems);
            convert_kernel<__nv_bfloat16><<<1216, 256, 0, st>>>(C.ppool[tri], (__nv_bfloat16*)pp, C.p_elems[tri]);
            convert_kernel<__nv_bfloat16><<<1216, 256, 0, st>>>(C.qpool[tri], (__nv_bfloat16*)pq, C.q_elems[tri]);
          }
          H.A.prec = aprec;
          H.A.leaf_pool = pl;
          H.A.p_pool = pp;
          H.A.q_pool = pq;
          // the FP64 pools of the construction are temporaries: gone after this group
          H.A64.leaf_pool = H.A64.p_pool = H.A64.q_pool = nullptr;
        }
      }
    }
    if (s == HM_OK) s = out_alloc(out, (void**)&out.d_y, sizeof(double) * std::max(C.N, 1), err);
    // ranks to the host (the group synchronises once below)
    C.h_rank.assign(2 * std::max(C.nn, 1), 0);
    if (s == HM_OK && cudaMemcpyAsync(C.h_rank.data(), C.d_rank, sizeof(int) * C.h_rank.size(),
                                      cudaMemcpyDeviceToHost, st) != cudaSuccess)
      s = HM_ERR_CUDA;
    if (s != HM_OK) break;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && s == HM_OK) s = HM_ERR_CUDA;
  free_tmp();
  if (s != HM_OK) return fail(s);
  // ---- per problem: row chunks of the per-step products and their column runs
  for (Ctx& C : G) {
    HinvData& out = *C.out;
    const int aprec = out.prec;
    const size_t es = (aprec == HINV_F64 || aprec == HINV_DF) ? 8 : (aprec == HINV_F32 ? 4 : 2);
    int64_t sb = 0;
    for (int tri = 0; tri < 2; ++tri) {
      HinvTriangle& H = out.tri[tri];
      H.h_rank.assign(C.h_rank.begin() + tri * C.nn, C.h_rank.begin() + tri * C.nn + C.nn);
      // the leaf's triangle (lower: columns [0, i0 + nr), upper: [i0, m)),
      // then P of every block above the leaf whose target holds it, at its rank
      std::vector<HinvRChunk> rch;
      std::vector<HinvSeg> segs;
      for (int l = 0; l < C.nl; ++l) {
        const HinvLeaf& L = H.h_leaves[l];
        for (int i0 = 0; i0 < L.m; i0 += HINV_ACH) {
          const int nr = std::min(HINV_ACH, L.m - i0);
          HinvRChunk R{L.r0 + i0, nr, (int)segs.size(), 0};
          HinvSeg t{};
          t.kind = 0;
          t.ld = L.ld;
          if (tri == 0) {
            t.off = L.off + i0;
            t.voff = L.r0;
            t.n = i0 + nr;
            t.a_hi = std::min(t.n, i0 + 32);
            t.b_lo = 0;
          } else {
            t.off = L.off + (int64_t)i0 * L.ld + i0;
            t.voff = L.r0 + i0;
            t.n = L.m - i0;
            t.a_hi = t.n;
            t.b_lo = 32;
          }
          segs.push_back(t);
          for (int q : C.anc_t[tri][l]) {
            const HinvNode& Nd = H.h_nodes[q];
            const int k = H.h_rank[q];
            if (k <= 0) continue;
            HinvSeg g{};
            g.kind = 1;
            g.off = Nd.poff + (L.r0 + i0 - Nd.tgt0);
            g.voff = (int64_t)q * HINV_KCAP;
            g.ld = Nd.pld;
            g.n = k;
            g.a_hi = k;
            g.b_lo = 0;
            segs.push_back(g);
          }
          R.seg_end = (int)segs.size();
          rch.push_back(R);
        }
      }
      // the chunks of one launch are all resident at once; heaviest first, so
      // that the CTAs handed to each SM mix heavy and light chunks
      auto rcost = [&](const HinvRChunk& R) {
        int64_t c = 0;
        for (int k = R.seg_begin; k < R.seg_end; ++k) c += segs[k].n;
        return c * (R.nr > 32 ? 2 : 1);
      };
      std::stable_sort(rch.begin(), rch.end(),
                       [&](const HinvRChunk& a, const HinvRChunk& b) { return rcost(a) > rcost(b); });
      std::vector<int4> tch;
      for (int v = 0; v < C.nn; ++v) {
        const HinvNode& Nd = H.h_nodes[v];
        for (int j0 = 0, q = Nd.tch_begin; j0 < Nd.src_n; j0 += HINV_TCH, ++q) tch.push_back(make_int4(v, j0, q, 0));
      }
      auto tcost = [&](const int4& c) {
        const HinvNode& Nd = H.h_nodes[c.x];
        return (int64_t)H.h_rank[c.x] * std::min(HINV_TCH, Nd.src_n - c.y);
      };
      std::stable_sort(tch.begin(), tch.end(), [&](const int4& a, const int4& b) { return tcost(a) > tcost(b); });
      HinvRChunk* d_rch_t = nullptr;
      HinvSeg* d_segs = nullptr;
      int4* d_tch = nullptr;
      if (s == HM_OK) s = out_upload(out, &d_rch_t, rch, st, err);
      if (s == HM_OK) s = out_upload(out, &d_segs, segs, st, err);
      if (s == HM_OK) s = out_upload(out, &d_tch, tch, st, err);
      if (s != HM_OK) return fail(s);
      for (HinvApply* A : {&H.A, &H.A64}) {
        A->nrch = (int)rch.size();
        A->rch = d_rch_t;
        A->segs = d_segs;
        A->tch = d_tch;
      }
      for (const HinvLeaf& L : H.h_leaves) sb += (int64_t)L.m * (L.m + 1) / 2;
      for (int v = 0; v < C.nn; ++v) {
        const HinvNode& Nd = H.h_nodes[v];
        sb += (int64_t)(Nd.tgt_n + Nd.src_n) * H.h_rank[v];
        out.max_rank = std::max(out.max_rank, H.h_rank[v]);
        out.capped += H.h_rank[v] >= HINV_KCAP ? 1 : 0;
      }
    }
    out.step_bytes = sb * (int64_t)es;
  }
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  for (Ctx& C : G) C.out->build_ms = ms;
  return HM_OK;
}

}  // namespace

int hinv_build_batch(const std::vector<HinvBuildJob>& jobs, int* d_err, cudaStream_t st, std::string& err) {
  // groups of at most HM_HINV_GROUP_ROWS stacked rows (default 2^19): the
  // construction's temporaries grow with the rows of a group (about 10 KB per row)
  int64_t limit = int64_t(1) << 19;
  if (const char* g = std::getenv("HM_HINV_GROUP_ROWS")) limit = std::max<int64_t>(1, std::atoll(g));
  const auto t0 = std::chrono::steady_clock::now();
  size_t i = 0;
  while (i < jobs.size()) {
    std::vector<Ctx> G;
    int64_t rows = 0;
    while (i < jobs.size() && (G.empty() || rows + jobs[i].P->N <= limit)) {
      const HinvBuildJob& J = jobs[i++];
      G.emplace_back();
      Ctx& C = G.back();
      C.P = J.P;
      C.dd = J.dd;
      C.F = J.F;
      C.d_rank_f = J.d_rank_f;
      C.out = J.out;
      C.tol = J.tol;
      *C.out = HinvData();
      // FP64 accuracy: pairs of floats in double-float arithmetic (HM_HINV_FP64=1: FP64 storage and arithmetic)
      const char* f64 = std::getenv("HM_HINV_FP64");
      C.out->prec = J.prec == HINV_F64 && !(f64 && f64[0] == '1') ? HINV_DF : J.prec;
      C.out->tol = J.tol;
      HM_TRY(ctx_prepare(C, err));
      rows += C.N;
    }
    HM_TRY(build_group(G, d_err, st, err));
  }
  if (jobs.size() > 1) {
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (const HinvBuildJob& J : jobs) J.out->build_ms = ms;
  }
  return HM_OK;
}

int hinv_solve(const HinvData& D, const double* b, double* z, cudaStream_t st) {
  HM_TRY(launch_hinv_apply(D.tri[0].A, b, D.d_y, st));
  return launch_hinv_apply(D.tri[1].A, D.d_y, z, st);
}

}  // namespace hm
