// Batched executors of the H-LU schedule (FP64): strided GEMM tiles, leaf LU
// with triangular inverses, low-rank truncation cores, copies and reductions.
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "hm_device.cuh"
#include "hlu_ops.h"
#include "hm_internal.h"
#include "hm_kernels.h"

namespace hm {

namespace {

constexpr int GK = 16;   // GEMM k chunk
#ifndef HM_GEMM_BIG_TILES
#define HM_GEMM_BIG_TILES 16  // 32 x 32 tiles from which a GEMM may take 64 x 64 tiles (0: never; build-time tuning parameter)
#endif
#ifndef HM_GEMM_BIG_WAVE
#define HM_GEMM_BIG_WAVE 4096  // ... when its wave has at least this many 32 x 32 GEMM tiles (build-time tuning parameter)
#endif

// (sh, sl) += a b for double-float a, b: the product's high part exactly
// (FMA), the cross terms rounded (the lo lo term, below 2^-48, is dropped),
// the sum by Knuth's two-sum.  __f*_rn keep the compiler from contracting or
// reordering the error terms.
__device__ __forceinline__ void df_acc(float& sh, float& sl, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float s = __fadd_rn(sh, p);
  const float bb = __fsub_rn(s, sh);
  const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(t, e));
}

// One TM x TN output tile of C = beta C + alpha A B (256 threads; 32 x 32,
// 64 x 16 and 16 x 64 tiles give each thread 2 x 2 outputs, 64 x 64 tiles
// 4 x 4).  Thread (tx, ty) owns rows ty + TY a and columns tx + TX b, so the
// shared-memory reads of a warp are broadcasts (A) and consecutive words (B).
// Narrow outputs (n or m <= 16) take the 64 x 16 or 16 x 64 shape so that no
// thread computes padding; large ones may take 64 x 64 (fewer, longer tasks).
// The next k chunk is loaded into registers while the current one is
// multiplied.  DF: the products and sums in double-float arithmetic on the
// FP32 pipes (about 48 significant bits: operands to 2^-49, each product and
// addition to about 2^-48 of its terms), otherwise FP64.  Every output sums
// its k terms in the same order whatever the tile shape.
template <int TM, int TN, bool DF>
__device__ void gemm_tile(const GemmOp& op, int local, double* smem, int* err) {
  constexpr int RN = TM * TN / 256 == 16 ? 4 : 2;        // outputs per thread along n
  constexpr int TX = TN / RN, TY = 256 / TX, RM = TM / TY;  // threads along n, m; outputs along m
  static_assert(RM * RN * 256 == TM * TN, "tile shape");
  constexpr int NA = TM * GK / 256, NB = GK * TN / 256;     // chunk elements per thread
  using T = typename std::conditional<DF, float2, double>::type;
  static_assert(sizeof(T) == sizeof(double), "same shared-memory layout");
  T (*As)[GK + 1] = reinterpret_cast<T (*)[GK + 1]>(smem);
  T (*Bs)[TN + 1] = reinterpret_cast<T (*)[TN + 1]>(smem + TM * (GK + 1));
  const int tn = (op.n + TN - 1) / TN;
  const int i0 = (local / tn) * TM, j0 = (local % tn) * TN;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  double ra[NA], rb[NB];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const int e = threadIdx.x + 256 * q, r = e / GK, c = e % GK, gi = i0 + r, gk = k0 + c;
      ra[q] = (gi < op.m && gk < op.k) ? op.A[gi * op.ars + gk * op.acs] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int e = threadIdx.x + 256 * q, r = e / TN, c = e % TN, gk = k0 + r, gj = j0 + c;
      rb[q] = (gk < op.k && gj < op.n) ? op.B[gk * op.brs + gj * op.bcs] : 0.0;
    }
  };
  auto stash = [&]() {
    bool bad = false;
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const int e = threadIdx.x + 256 * q;
      if constexpr (DF) As[e / GK][e % GK] = df_split(ra[q], bad);
      else As[e / GK][e % GK] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int e = threadIdx.x + 256 * q;
      if constexpr (DF) Bs[e / TN][e % TN] = df_split(rb[q], bad);
      else Bs[e / TN][e % TN] = rb[q];
    }
    if (bad) atomicOr(err, DEVERR_NONFINITE);
  };
  constexpr int RO = RM * RN;
  double acc[RO];
  float sh[RO], sl[RO];
#pragma unroll
  for (int q = 0; q < RO; ++q) {
    acc[q] = 0.0;
    sh[q] = 0.f;
    sl[q] = 0.f;
  }
  load(0);
  for (int k0 = 0; k0 < op.k; k0 += GK) {
    stash();
    __syncthreads();
    if (k0 + GK < op.k) load(k0 + GK);  // in flight during this chunk's arithmetic
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      T a[RM], b[RN];
#pragma unroll
      for (int x = 0; x < RM; ++x) a[x] = As[ty + TY * x][kk];
#pragma unroll
      for (int y = 0; y < RN; ++y) b[y] = Bs[kk][tx + TX * y];
      if constexpr (DF) {
#pragma unroll
        for (int x = 0; x < RM; ++x)
#pragma unroll
          for (int y = 0; y < RN; ++y) df_acc(sh[x * RN + y], sl[x * RN + y], a[x], b[y]);
        if ((kk & 3) == 3) {
#pragma unroll
          for (int q = 0; q < RO; ++q) {  // renormalise every 4 terms: sl stays within an ulp of sh
            const float s = __fadd_rn(sh[q], sl[q]);
            sl[q] = __fsub_rn(sl[q], __fsub_rn(s, sh[q]));
            sh[q] = s;
          }
        }
      } else {
#pragma unroll
        for (int x = 0; x < RM; ++x)
#pragma unroll
          for (int y = 0; y < RN; ++y) acc[x * RN + y] += a[x] * b[y];
      }
    }
    if (k0 + GK < op.k) __syncthreads();  // the next chunk overwrites As, Bs
  }
#pragma unroll
  for (int x = 0; x < RM; ++x)
#pragma unroll
    for (int y = 0; y < RN; ++y) {
      const int gi = i0 + ty + TY * x, gj = j0 + tx + TX * y;
      if (gi < op.m && gj < op.n) {
        double* c = op.C + gi * op.crs + gj * op.ccs;
        const double r = DF ? (double)sh[x * RN + y] + (double)sl[x * RN + y] : acc[x * RN + y];
        double v = op.alpha * r;
        *c = op.beta == 0.0 ? v : op.beta * (*c) + v;
      }
    }
  // no barrier here: the executor's completion barrier follows every task
  // before shared memory is written again
}

// op.shape: bits 0-1 the tile shape (gemm_shape; 3 = 64 x 64), bit 2 set = FP64 arithmetic
__device__ void dev_gemm_tile(const GemmOp& op, int local, double* smem, int* err) {
  const int sh = op.shape & 3;
  if (op.shape & GEMM_FP64) {
    if (sh == 1) gemm_tile<64, 16, false>(op, local, smem, err);
    else if (sh == 2) gemm_tile<16, 64, false>(op, local, smem, err);
    else if (sh == 3) gemm_tile<64, 64, false>(op, local, smem, err);
    else gemm_tile<32, 32, false>(op, local, smem, err);
  } else {
    if (sh == 1) gemm_tile<64, 16, true>(op, local, smem, err);
    else if (sh == 2) gemm_tile<16, 64, true>(op, local, smem, err);
    else if (sh == 3) gemm_tile<64, 64, true>(op, local, smem, err);
    else gemm_tile<32, 32, true>(op, local, smem, err);
  }
}

// Base LU (m <= LU_BASE) in shared memory, then the inverses of L (unit
// lower) and U.  FP64 on this GPU issues one warp instruction per 64 cycles
// on each SM sub-partition and a division takes about ten of them, so the
// work is laid out to keep dependent FP64 chains short: one reciprocal per
// pivot (warp 0, overlapped with the other warps' updates), and blocked
// inverses (8 x 8 diagonal blocks by substitution, then two doubling steps of
// small products).  The block is padded to 32 with the identity.
constexpr int LB = LU_BASE;
struct LuSmem {
  double (*A)[LB + 1];
  double (*XL)[LB + 1];
  double (*XU)[LB + 1];
  double* TL;   // 2 x 16 x 16 products of the doubling steps
  double* TU;
  double* rd;   // 1 / U[i][i]
  double* rp;   // reciprocal of the current pivot
};

__device__ __forceinline__ LuSmem lu_smem(double* smem) {
  LuSmem S;
  S.A = reinterpret_cast<double (*)[LB + 1]>(smem);
  S.XL = reinterpret_cast<double (*)[LB + 1]>(smem + LB * (LB + 1));
  S.XU = reinterpret_cast<double (*)[LB + 1]>(smem + 2 * LB * (LB + 1));
  S.TL = smem + 3 * LB * (LB + 1);
  S.TU = S.TL + 512;
  S.rd = S.TU + 512;
  S.rp = S.rd + LB;
  return S;
}

// One doubling step of the blocked inverses: blocks of size s combine into
// blocks of size 2s (XL21 = -XL22 L21 XL11, XU12 = -XU11 U12 XU22).
__device__ void lu_inv_double(const LuSmem& S, int s) {
  const int np = LB / (2 * s), per = np * s * s, t = threadIdx.x;
  for (int e = t; e < 2 * per; e += blockDim.x) {
    const int f = e / per, r = e % per, pr = r / (s * s), i = (r % (s * s)) / s, j = r % s, b = pr * 2 * s;
    double acc = 0.0;
    if (f == 0) {
      for (int k = 0; k < s; ++k) acc += S.A[b + s + i][b + k] * S.XL[b + k][b + j];
      S.TL[r] = acc;
    } else {
      for (int k = 0; k < s; ++k) acc += S.A[b + i][b + s + k] * S.XU[b + s + k][b + s + j];
      S.TU[r] = acc;
    }
  }
  __syncthreads();
  for (int e = t; e < 2 * per; e += blockDim.x) {
    const int f = e / per, r = e % per, pr = r / (s * s), i = (r % (s * s)) / s, j = r % s, b = pr * 2 * s;
    const double* T = (f == 0 ? S.TL : S.TU) + pr * s * s;
    double acc = 0.0;
    if (f == 0) {
      for (int k = 0; k < s; ++k) acc += S.XL[b + s + i][b + s + k] * T[k * s + j];
      S.XL[b + s + i][b + j] = -acc;
    } else {
      for (int k = 0; k < s; ++k) acc += S.XU[b + i][b + k] * T[k * s + j];
      S.XU[b + i][b + s + j] = -acc;
    }
  }
  __syncthreads();
}

__device__ void dev_lu_base(const LuOp& op, int* err, double* smem) {
  const LuSmem S = lu_smem(smem);
  const int m = op.m, t = threadIdx.x, warp = t >> 5, lane = t & 31;
  for (int e = t; e < LB * LB; e += blockDim.x) {
    const int i = e / LB, j = e % LB;
    S.A[i][j] = (i < m && j < m) ? op.A[i * op.lda + j] : (i == j ? 1.0 : 0.0);
    S.XL[i][j] = 0.0;
    S.XU[i][j] = 0.0;
  }
  __syncthreads();
  auto recip = [&](double piv) {
    if (piv == 0.0 || !isfinite(piv)) {
      atomicOr(err, DEVERR_ZEROPIVOT);
      piv = 1e-300;
    }
    return 1.0 / piv;
  };
  if (t == 0) S.rp[0] = recip(S.A[0][0]);
  __syncthreads();
  // right-looking elimination; warp 0 updates the next pivot first and takes
  // its reciprocal while warps 1..7 update the rest
  for (int p = 0; p < m; ++p) {
    const double rp = S.rp[0];
    for (int i = p + 1 + t; i < m; i += blockDim.x) S.A[i][p] *= rp;
    __syncthreads();
    const int w = m - p - 1;
    if (warp == 0) {
      if (lane == 0 && w > 0) {
        const double v = S.A[p + 1][p + 1] - S.A[p + 1][p] * S.A[p][p + 1];
        S.A[p + 1][p + 1] = v;
        S.rp[0] = recip(v);
      }
    } else {
      for (int e = t - 32; e < w * w; e += blockDim.x - 32) {
        if (e == 0) continue;  // the next pivot: warp 0
        const int i = p + 1 + e / w, j = p + 1 + e % w;
        S.A[i][j] -= S.A[i][p] * S.A[p][j];
      }
    }
    __syncthreads();
  }
  // diagonal 8 x 8 blocks of both inverses by substitution: warp 0 L, warp 1 U
  if (warp == 1) {  // padded rows have 1 on the diagonal; a zero pivot was flagged above
    const double d = S.A[lane][lane];
    S.rd[lane] = 1.0 / (d == 0.0 ? 1e-300 : d);
  }
  __syncwarp();
  if (warp == 0) {
    const int b = (lane >> 3) * 8, j = lane & 7;
    S.XL[b + j][b + j] = 1.0;
    for (int i = j + 1; i < 8; ++i) {
      double v = 0.0;
      for (int k = j; k < i; ++k) v -= S.A[b + i][b + k] * S.XL[b + k][b + j];
      S.XL[b + i][b + j] = v;
    }
  } else if (warp == 1) {
    const int b = (lane >> 3) * 8, j = lane & 7;
    S.XU[b + j][b + j] = S.rd[b + j];
    for (int i = j - 1; i >= 0; --i) {
      double v = 0.0;
      for (int k = i + 1; k <= j; ++k) v += S.A[b + i][b + k] * S.XU[b + k][b + j];
      S.XU[b + i][b + j] = -v * S.rd[b + i];
    }
  }
  __syncthreads();
  lu_inv_double(S, 8);
  lu_inv_double(S, 16);
  for (int e = t; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    op.Li[i * op.ldl + j] = S.XL[i][j];
    op.Ui[i * op.ldu + j] = S.XU[i][j];
  }
  __syncthreads();
}

// ---- the same base LU in double-float arithmetic on the FP32 pipes (the
// helpers in hm_device.cuh; HM_LU_DF=1).  Unevaluated float pairs (about 48
// significant bits, as the GEMM tiles) shorten the pivot steps (1D N = 65536:
// executor 220.9 -> 216.5 ms) but are not the default: the pivots carry the
// cancellation between the identity and the stiff part of I - dt/2 G, and
// their rounding reaches the Crank-Nicolson solution (1D Levy workload at
// N = 32768, 1000 steps against the dense FP64 oracle: 1.5e-8 with a
// double-float 64 x 64 base, 7e-9 with FP64, the compression's own error).
struct LuSmemDD {
  float2 (*A)[LB + 1];
  float2 (*XL)[LB + 1];
  float2 (*XU)[LB + 1];
  float2* TL;
  float2* TU;
  float2* rd;
  float2* rp;
};

__device__ __forceinline__ LuSmemDD lu_smem_dd(double* smem) {
  float2* f = reinterpret_cast<float2*>(smem);  // the FP64 layout, one float pair per double
  LuSmemDD S;
  S.A = reinterpret_cast<float2 (*)[LB + 1]>(f);
  S.XL = reinterpret_cast<float2 (*)[LB + 1]>(f + LB * (LB + 1));
  S.XU = reinterpret_cast<float2 (*)[LB + 1]>(f + 2 * LB * (LB + 1));
  S.TL = f + 3 * LB * (LB + 1);
  S.TU = S.TL + 512;
  S.rd = S.TU + 512;
  S.rp = S.rd + LB;
  return S;
}

__device__ void lu_inv_double_dd(const LuSmemDD& S, int s) {
  const int np = LB / (2 * s), per = np * s * s, t = threadIdx.x;
  const float2 z = make_float2(0.f, 0.f);
  for (int e = t; e < 2 * per; e += blockDim.x) {
    const int f = e / per, r = e % per, pr = r / (s * s), i = (r % (s * s)) / s, j = r % s, b = pr * 2 * s;
    float2 acc = z;
    if (f == 0) {
      for (int k = 0; k < s; ++k) acc = dd_add(acc, dd_mul(S.A[b + s + i][b + k], S.XL[b + k][b + j]));
      S.TL[r] = acc;
    } else {
      for (int k = 0; k < s; ++k) acc = dd_add(acc, dd_mul(S.A[b + i][b + s + k], S.XU[b + s + k][b + s + j]));
      S.TU[r] = acc;
    }
  }
  __syncthreads();
  for (int e = t; e < 2 * per; e += blockDim.x) {
    const int f = e / per, r = e % per, pr = r / (s * s), i = (r % (s * s)) / s, j = r % s, b = pr * 2 * s;
    const float2* T = (f == 0 ? S.TL : S.TU) + pr * s * s;
    float2 acc = z;
    if (f == 0) {
      for (int k = 0; k < s; ++k) acc = dd_add(acc, dd_mul(S.XL[b + s + i][b + s + k], T[k * s + j]));
      S.XL[b + s + i][b + j] = dd_neg(acc);
    } else {
      for (int k = 0; k < s; ++k) acc = dd_add(acc, dd_mul(S.XU[b + i][b + k], T[k * s + j]));
      S.XU[b + i][b + s + j] = dd_neg(acc);
    }
  }
  __syncthreads();
}

__device__ void dev_lu_base_dd(const LuOp& op, int* err, double* smem) {
  const LuSmemDD S = lu_smem_dd(smem);
  const int m = op.m, t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const float2 z = make_float2(0.f, 0.f);
  bool bad = false;
  for (int e = t; e < LB * LB; e += blockDim.x) {
    const int i = e / LB, j = e % LB;
    S.A[i][j] = (i < m && j < m) ? df_split(op.A[i * op.lda + j], bad) : make_float2(i == j ? 1.f : 0.f, 0.f);
    S.XL[i][j] = z;
    S.XU[i][j] = z;
  }
  if (bad) atomicOr(err, DEVERR_NONFINITE);
  __syncthreads();
  auto recip = [&](float2 piv) {
    if (piv.x == 0.f || !isfinite(piv.x)) {
      atomicOr(err, DEVERR_ZEROPIVOT);
      piv = make_float2(1e-30f, 0.f);
    }
    return dd_recip(piv);
  };
  if (t == 0) S.rp[0] = recip(S.A[0][0]);
  __syncthreads();
  for (int p = 0; p < m; ++p) {
    const float2 rp = S.rp[0];
    for (int i = p + 1 + t; i < m; i += blockDim.x) S.A[i][p] = dd_mul(S.A[i][p], rp);
    __syncthreads();
    const int w = m - p - 1;
    if (warp == 0) {
      if (lane == 0 && w > 0) {
        const float2 v = dd_fnms(S.A[p + 1][p + 1], S.A[p + 1][p], S.A[p][p + 1]);
        S.A[p + 1][p + 1] = v;
        S.rp[0] = recip(v);
      }
    } else {
      for (int e = t - 32; e < w * w; e += blockDim.x - 32) {
        if (e == 0) continue;
        const int i = p + 1 + e / w, j = p + 1 + e % w;
        S.A[i][j] = dd_fnms(S.A[i][j], S.A[i][p], S.A[p][j]);
      }
    }
    __syncthreads();
  }
  if (warp == 1) {
    const float2 d = S.A[lane][lane];
    S.rd[lane] = dd_recip(d.x == 0.f ? make_float2(1e-30f, 0.f) : d);
  }
  __syncwarp();
  if (warp == 0) {
    const int b = (lane >> 3) * 8, j = lane & 7;
    S.XL[b + j][b + j] = make_float2(1.f, 0.f);
    for (int i = j + 1; i < 8; ++i) {
      float2 v = z;
      for (int k = j; k < i; ++k) v = dd_fnms(v, S.A[b + i][b + k], S.XL[b + k][b + j]);
      S.XL[b + i][b + j] = v;
    }
  } else if (warp == 1) {
    const int b = (lane >> 3) * 8, j = lane & 7;
    S.XU[b + j][b + j] = S.rd[b + j];
    for (int i = j - 1; i >= 0; --i) {
      float2 v = z;
      for (int k = i + 1; k <= j; ++k) v = dd_add(v, dd_mul(S.A[b + i][b + k], S.XU[b + k][b + j]));
      S.XU[b + i][b + j] = dd_neg(dd_mul(v, S.rd[b + i]));
    }
  }
  __syncthreads();
  lu_inv_double_dd(S, 8);
  lu_inv_double_dd(S, 16);
  for (int e = t; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    const float2 l = S.XL[i][j], u = S.XU[i][j];
    op.Li[i * op.ldl + j] = (double)l.x + (double)l.y;
    op.Ui[i * op.ldu + j] = (double)u.x + (double)u.y;
  }
  __syncthreads();
}

// Biased exponent of a Gram diagonal entry (0 for zero or subnormal) and an
// exact power of two 2^n (|n| clamped to the normal range).
__device__ __forceinline__ int gram_exponent(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}
__device__ __forceinline__ double pow2i(int n) {
  n = max(-1000, min(1000, n));
  return __longlong_as_double((long long)(1023 + n) << 52);
}

// ---- truncation core (one CTA): pivoted Cholesky of both Gram matrices,
// core C = R_A P_A' P_B R_B', column-pivoted Householder QR of C, then the
// coefficient matrices TA, TB (see TruncOp).
struct TruncSmem {
  double* GA;   // K x K
  double* GB;   // K x K
  double* C;    // K x K
};

// Warp 0: largest v[j * stride] over p <= j < K (ties -> smallest j) and the
// sum of those entries; results in red_v[0] (max), red_v[1] (sum), red_i[0].
__device__ __forceinline__ void warp0_max_sum(const double* v, int stride, int p, int K, double* red_v,
                                              int* red_i) {
  if ((threadIdx.x >> 5) != 0) return;
  const int lane = threadIdx.x & 31;
  double best = -1.0, sum = 0.0;
  int q = -1;
  for (int j = p + lane; j < K; j += 32) {
    double x = v[j * stride];
    sum += x;
    if (q < 0 || x > best) { best = x; q = j; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double ob = __shfl_xor_sync(0xffffffffu, best, o);
    int oq = __shfl_xor_sync(0xffffffffu, q, o);
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (oq >= 0 && (q < 0 || ob > best || (ob == best && oq < q))) { best = ob; q = oq; }
  }
  if (lane == 0) {
    red_v[0] = best;
    red_v[1] = sum;
    red_i[0] = q < 0 ? p : q;
  }
}

// Barrier over `n` threads: the whole CTA (id 0) or one half (ids 1, 2).
__device__ __forceinline__ void group_sync(int id, int n) {
  if (id == 0) __syncthreads();
  else asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// In-place pivoted Cholesky P' G P = R' R of the symmetric K x K matrix G
// (row-major), run by the `nthr` threads of a group (index ht, barrier bar).
// Only the upper triangle is read and written (entry (i, j), i <= j, at
// G[i K + j]); rows are swapped physically.  On return R is the upper
// triangle of G's first `rank` rows, perm[c] the original index of pivot c.
// Pivots stop at rel_thresh times the largest initial diagonal.  FP64 issue
// is the limit here: one rsqrt per pivot, multiplications for the row
// scaling, and the symmetric half of the trailing update.
__device__ int pivoted_cholesky(double* G, int K, int* perm, double rel_thresh, double* red_v, int* red_i,
                                int ht, int nthr, int bar) {
  for (int c = ht; c < K; c += nthr) perm[c] = c;
  if (ht < 32) {
    double m = 0.0;
    for (int c = ht; c < K; c += 32) m = fmax(m, G[c * K + c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (ht == 0) red_v[0] = m;
  }
  group_sync(bar, nthr);
  const double dmax0 = red_v[0];
  const double thresh = rel_thresh * dmax0;
  int rank = 0;
  for (int p = 0; p < K; ++p) {
    // pivot: the largest remaining diagonal (ties: smallest index); warp 0 of the group
    if (ht < 32) {
      double best = -1.0;
      int q = -1;
      for (int c = p + ht; c < K; c += 32) {
        const double x = G[c * K + c];
        if (q < 0 || x > best) { best = x; q = c; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oq = __shfl_xor_sync(0xffffffffu, q, o);
        if (oq >= 0 && (q < 0 || ob > best || (ob == best && oq < q))) { best = ob; q = oq; }
      }
      if (ht == 0) {
        red_v[1] = best;
        red_i[0] = q;
      }
    }
    group_sync(bar, nthr);
    const double best = red_v[1];
    const int q = red_i[0];
    if (q < 0 || !(best > thresh) || dmax0 <= 0.0) break;
    if (q != p) {
      // symmetric swap of indices p and q in the upper-triangle storage
      for (int x = ht; x < K; x += nthr) {
        if (x == p || x == q) continue;
        double* a = &G[min(p, x) * K + max(p, x)];
        double* b = &G[min(q, x) * K + max(q, x)];
        const double t = *a;
        *a = *b;
        *b = t;
      }
      if (ht == 0) {
        const double t = G[p * K + p];
        G[p * K + p] = G[q * K + q];
        G[q * K + q] = t;
        const int u = perm[p];
        perm[p] = perm[q];
        perm[q] = u;
      }
      group_sync(bar, nthr);
    }
    const double rs = rsqrt(best);  // every thread: one reciprocal square root per pivot
    for (int j = p + ht; j < K; j += nthr) G[p * K + j] = (j == p) ? best * rs : G[p * K + j] * rs;
    group_sync(bar, nthr);
    // trailing update of the upper triangle: (i, j), p < i <= j
    const int w = K - p - 1;
    const int tri = w * (w + 1) / 2;
    for (int e = ht; e < tri; e += nthr) {
      // e -> (i, j), i <= j: rows k and w-1-k paired (w + 1 entries per pair)
      const int k = e / (w + 1), o = e % (w + 1);
      int i, j;
      if (o < w - k) {
        i = k;
        j = k + o;
      } else {
        i = w - 1 - k;
        j = i + (o - (w - k));
      }
      const int gi = p + 1 + i, gj = p + 1 + j;
      G[gi * K + gj] -= G[p * K + gi] * G[p * K + gj];
    }
    ++rank;
    group_sync(bar, nthr);
  }
  group_sync(bar, nthr);
  return rank;
}

// Tail of the truncation when Q and Z do not fit beside the K x K matrices:
// Q is formed in the output TA (global memory), then staged through GA.
template <int KM>
__device__ void trunc_tail_global(const TruncOp& op, int* err, double* sm, int K, int kf, int rA, int rB, int r,
                                  bool capped) {
  double* cn = sm + 3 * KM * KM;
  double* tau = cn + KM;
  double* red_v = tau + KM;
  int* permA = reinterpret_cast<int*>(red_v + 32);
  int* permB = permA + KM;
  int* permC = permB + KM;
  int* posA = permC + KM;
  int* posB = posA + KM;
  int* red_i = posB + KM;
  int* kexp = red_i + 8;
  const int t = threadIdx.x;
  double* GA = sm;
  double* GB = sm + K * K;
  double* C = sm + 2 * K * K;
  (void)posA;
  (void)posB;
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
  // reciprocal diagonals of R_A and R_B (cn and tau are free now): the same
  // arithmetic as the shared-memory tail, so the factors do not depend on
  // which tail (which executor mode) ran
  for (int i = t; i < rA; i += blockDim.x) cn[i] = 1.0 / GA[i * K + i];
  for (int i = t; i < rB; i += blockDim.x) tau[i] = 1.0 / GB[i * K + i];
  __syncthreads();
  // T_A (pivoted rows) = R11_A^{-1} Q; R11_A is the leading rA x rA block of GA (upper)
  // solve in place column by column (back substitution), then scatter rows by permA.
  for (int c = t; c < r; c += blockDim.x) {
    for (int i = rA - 1; i >= 0; --i) {
      double v = Q[i * kf + c];
      for (int k = i + 1; k < rA; ++k) v -= GA[i * K + k] * Q[k * kf + c];
      Q[i * kf + c] = v * cn[i];
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
    op.TA[permA[i] * kf + c] = GA[i * kf + c] * pow2i(kexp[permA[i]]);
  }
  // T_B (pivoted rows) = R11_B^{-1} Z, Z[j][c] = R_C[c][posC(j)] for j < rB
  __syncthreads();
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
  __syncthreads();
  for (int c = t; c < r; c += blockDim.x) {
    for (int i = rB - 1; i >= 0; --i) {
      double v = GA[i * kf + c];
      for (int k = i + 1; k < rB; ++k) v -= GB[i * K + k] * GA[k * kf + c];
      GA[i * kf + c] = v * tau[i];
    }
  }
  __syncthreads();
  for (int e = t; e < K * kf; e += blockDim.x) {
    int i = e / kf, c = e % kf;
    op.TB[permB[i] * kf + c] = (i < rB && c < r) ? GA[i * kf + c] * pow2i(-kexp[permB[i]]) : 0.0;
  }
  if (t == 0) {
    *op.rank = r;
    if (capped) atomicOr(err, DEVERR_RANKCAP);
  }
  __syncthreads();
}

// Tail of the truncation with Q and Z in shared memory: Q = the first r
// columns of C's orthogonal factor, TA = R_A^{-1} Q (half 0) and Z = R_C P_C',
// TB = R_B^{-1} Z (half 1) side by side; reciprocal diagonals precomputed.
template <int KM>
__device__ void trunc_tail_smem(const TruncOp& op, int* err, double* sm, int K, int kf, int rA, int rB, int r,
                                bool capped) {
  double* cn = sm + 3 * KM * KM;
  double* tau = cn + KM;
  double* red_v = tau + KM;
  int* permA = reinterpret_cast<int*>(red_v + 32);
  int* permB = permA + KM;
  int* permC = permB + KM;
  int* posA = permC + KM;
  int* posB = posA + KM;
  int* red_i = posB + KM;
  int* kexp = red_i + 8;
  const int t = threadIdx.x;
  double* GA = sm;
  double* GB = sm + K * K;
  double* C = sm + 2 * K * K;
  double* Q = sm + 3 * K * K;   // rA x r, stride kf
  double* Z = Q + K * kf;       // rB x r, stride kf
  (void)posA;
  (void)posB;
  for (int e = t; e < K * kf; e += blockDim.x) Q[e] = 0.0;
  __syncthreads();
  for (int c = t; c < r; c += blockDim.x) Q[c * kf + c] = 1.0;
  // Z[j][c] = R_C[c][pos(j)] (zero below R_C's diagonal), pos(j): permC[pos] = j
  for (int e = t; e < rB * r; e += blockDim.x) {
    const int j = e / r, c = e % r;
    int pc = 0;
    for (int u = 0; u < rB; ++u)
      if (permC[u] == j) { pc = u; break; }
    Z[j * kf + c] = (pc >= c) ? C[c * K + pc] : 0.0;
  }
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
  // reciprocal diagonals of R_A and R_B (cn and tau are free now)
  for (int i = t; i < rA; i += blockDim.x) cn[i] = 1.0 / GA[i * K + i];
  for (int i = t; i < rB; i += blockDim.x) tau[i] = 1.0 / GB[i * K + i];
  __syncthreads();
  // back substitutions: half 0 solves R_A X = Q, half 1 solves R_B Y = Z
  {
    const int h = t >> 7, ht = t & 127;
    const double* R = h ? GB : GA;
    double* X = h ? Z : Q;
    const double* rd = h ? tau : cn;
    const int n = h ? rB : rA;
    for (int c = ht; c < r; c += 128) {
      for (int i = n - 1; i >= 0; --i) {
        double v = X[i * kf + c];
        for (int k = i + 1; k < n; ++k) v -= R[i * K + k] * X[k * kf + c];
        X[i * kf + c] = v * rd[i];
      }
    }
  }
  __syncthreads();
  for (int e = t; e < K * kf; e += blockDim.x) {
    const int i = e / kf, c = e % kf;
    op.TA[permA[i] * kf + c] = (i < rA && c < r) ? Q[i * kf + c] * pow2i(kexp[permA[i]]) : 0.0;
    op.TB[permB[i] * kf + c] = (i < rB && c < r) ? Z[i * kf + c] * pow2i(-kexp[permB[i]]) : 0.0;
  }
  if (t == 0) {
    *op.rank = r;
    if (capped) atomicOr(err, DEVERR_RANKCAP);
  }
  __syncthreads();
}

template <int KM>
__device__ void dev_trunc(const TruncOp& op, int* err, double* sm) {
  // scratch after the three K x K matrices
  double* cn = sm + 3 * KM * KM;
  double* tau = cn + KM;
  double* red_v = tau + KM;
  int* permA = reinterpret_cast<int*>(red_v + 32);
  int* permB = permA + KM;
  int* permC = permB + KM;
  int* posA = permC + KM;
  int* posB = posA + KM;
  int* red_i = posB + KM;
  const int K = op.K, kf = op.kf, t = threadIdx.x;
  double* GA = sm;
  double* GB = sm + K * K;
  double* C = sm + 2 * K * K;
  int* kexp = red_i + 8;  // K ints (the int scratch holds 7 x KM)
  for (int e = t; e < K * K; e += blockDim.x) {
    GA[e] = op.GA[e];
    GB[e] = op.GB[e];
  }
  __syncthreads();
  // Balance every column pair (a_i, b_i) by an exact power of two,
  // a_i 2^k_i and b_i 2^-k_i with |a_i| ~ |b_i|, so that the Gram diagonals
  // measure the norms |a_i||b_i| of the terms of the sum: otherwise a small
  // column of A whose partner in B is large falls below the Cholesky cut.
  for (int i = t; i < K; i += blockDim.x) {
    const int ea = gram_exponent(GA[i * K + i]), eb = gram_exponent(GB[i * K + i]);
    kexp[i] = (ea > 0 && eb > 0) ? (eb - ea) >> 2 : 0;
  }
  __syncthreads();
  for (int e = t; e < K * K; e += blockDim.x) {
    const int s = kexp[e / K] + kexp[e % K];
    GA[e] *= pow2i(s);
    GB[e] *= pow2i(-s);
  }
  __syncthreads();
  // Gram entries below (tol/10)^2 of the largest carry nothing the truncation
  // keeps.  The two factorizations run side by side on the CTA's halves.
  const double rel = fmax(0.01 * op.tol * op.tol, 1e-15);
  {
    const int h = t >> 7;
    const int r = pivoted_cholesky(h ? GB : GA, K, h ? permB : permA, rel, red_v + 8 * h, red_i + 4 * h,
                                   t & 127, 128, 1 + h);
    if ((t & 127) == 0) red_i[2 + 4 * h] = r;
  }
  __syncthreads();
  const int rA = red_i[2], rB = red_i[6];
  for (int c = t; c < K; c += blockDim.x) {
    posA[permA[c]] = c;
    posB[permB[c]] = c;
  }
  __syncthreads();
  // C[i][j] = sum_o R_A[i][posA(o)] R_B[j][posB(o)] over the upper triangles:
  // walk A's pivot positions c >= i and keep the terms with posB(o) >= j
  for (int e = t; e < rA * rB; e += blockDim.x) {
    const int i = e / rB, j = e % rB;
    double acc = 0.0;
    for (int c = i; c < K; ++c) {
      const int cb = posB[permA[c]];
      if (cb >= j) acc += GA[i * K + c] * GB[j * K + cb];
    }
    C[i * K + j] = acc;
  }
  __syncthreads();
  // Householder QR of C (rA x rB) with column pivoting; stop on the trailing norm
  for (int j = t; j < rB; j += blockDim.x) {
    permC[j] = j;
    double sq = 0.0;
    for (int i = 0; i < rA; ++i) sq += C[i * K + j] * C[i * K + j];
    cn[j] = sq;
  }
  __syncthreads();
  if (t < 32) {
    double sm_ = 0.0;
    for (int j = t; j < rB; j += 32) sm_ += cn[j];
    sm_ = warp_sum(sm_);
    if (t == 0) red_v[4] = sm_;
  }
  __syncthreads();
  const double total = red_v[4];
  int r = 0;
  const int rmax = min(min(rA, rB), kf);
  bool capped = false;
  for (int p = 0; p < min(rA, rB); ++p) {
    warp0_max_sum(cn, 1, p, rB, red_v, red_i);
    __syncthreads();
    const double rem = red_v[1];
    if (!(rem > op.tol * op.tol * total) || total <= 0.0) break;
    if (p == rmax) { capped = true; break; }
    const int q = red_i[0];
    // swap columns p and q; the thread that owns row p in the swap (thread p,
    // rA <= KM < blockDim.x) first forms the reflector of column q:
    // s = sum_{i >= p} C[i][q]^2 is its trailing norm, the maximum red_v[0]
    if (t == p) {
      const double sq = red_v[0];
      const double nrm = sqrt(sq);
      const double x0 = C[p * K + q];
      const double alpha = x0 >= 0.0 ? -nrm : nrm;
      const double v0 = x0 - alpha;
      const double vnorm2 = sq - x0 * x0 + v0 * v0;
      tau[p] = (vnorm2 > 0.0) ? 2.0 / vnorm2 : 0.0;
      red_v[2] = v0;
      red_v[3] = alpha;
    }
    if (q != p) {
      for (int i = t; i < rA; i += blockDim.x) {
        const double a = C[i * K + p];
        C[i * K + p] = C[i * K + q];
        C[i * K + q] = a;
      }
      if (t == 32) {
        const int a = permC[p];
        permC[p] = permC[q];
        permC[q] = a;
        const double b = cn[p];
        cn[p] = cn[q];
        cn[q] = b;
      }
    }
    __syncthreads();
    const double v0 = red_v[2], alpha = red_v[3], tp = tau[p];
    // apply H = I - tau v v' to columns p+1.. (v = [v0, C[p+1..rA-1][p]]) and
    // recompute their trailing norms in the same pass
    for (int j = p + 1 + t; j < rB; j += blockDim.x) {
      double dot = v0 * C[p * K + j];
      for (int i = p + 1; i < rA; ++i) dot += C[i * K + p] * C[i * K + j];
      dot *= tp;
      C[p * K + j] -= dot * v0;
      double sq = 0.0;
      for (int i = p + 1; i < rA; ++i) {
        const double x = C[i * K + j] - dot * C[i * K + p];
        C[i * K + j] = x;
        sq += x * x;
      }
      cn[j] = sq;
    }
    if (t == 0) {
      C[p * K + p] = alpha;  // R diagonal; v0 of reflector p kept in cn[p]
      cn[p] = v0;
    }
    ++r;
    __syncthreads();
  }
  __syncthreads();
  if (3 * K * K + 2 * K * kf <= 3 * KM * KM) {
    trunc_tail_smem<KM>(op, err, sm, K, kf, rA, rB, r, capped);
    return;
  }
  trunc_tail_global<KM>(op, err, sm, K, kf, rA, rB, r, capped);
}

__device__ void dev_copy(const CopyOp& op, int chunk, int nchunks) {
  const int64_t tot = (int64_t)op.m * op.n;
  for (int64_t e = chunk * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)nchunks * blockDim.x) {
    int i = (int)(e / op.n), j = (int)(e % op.n);
    double v = op.src ? op.alpha * op.src[i * op.srs + j * op.scs] : op.alpha;
    double* d = op.dst + i * op.drs + j * op.dcs;
    *d = op.beta == 0.0 ? v : op.beta * (*d) + v;
  }
}

__device__ void dev_reduce(const ReduceOp& op, int chunk, int nchunks) {
  const int64_t count = (int64_t)op.m * op.n;
  if (count <= 64 && op.nparts > 8) {
    // few outputs, many parts: a warp per output, lanes over the parts
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t e = chunk * 8 + warp; e < count; e += (int64_t)nchunks * 8) {
      double s = 0.0;
      for (int p = lane; p < op.nparts; p += 32) s += op.parts[p * op.stride + e];
      s = warp_sum(s);
      if (lane == 0) {
        const int i = (int)(e / op.n), j = (int)(e % op.n);
        double* d = op.dst + i * op.drs + j * op.dcs;
        *d = op.beta == 0.0 ? op.alpha * s : op.beta * (*d) + op.alpha * s;
      }
    }
    return;
  }
  for (int64_t e = chunk * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)nchunks * blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < op.nparts; ++p) s += op.parts[p * op.stride + e];
    const int i = (int)(e / op.n), j = (int)(e % op.n);
    double* d = op.dst + i * op.drs + j * op.dcs;
    *d = op.beta == 0.0 ? op.alpha * s : op.beta * (*d) + op.alpha * s;
  }
}


// Row task: 8 warps.  Dense sources: warp per row (rows w, w+8, ...), lanes
// over columns.  Low-rank sources: warp per source (round robin), lane per
// row, after summing the source's partial products.  Per-row totals are
// combined in a fixed order, so results are bitwise reproducible.
// 8-byte asynchronous global -> shared copy (operands written by an earlier
// kernel only: the copy goes through L1) and the wait for all of a thread's copies.
__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Shared-memory layout of a row task: accumulators, per-warp coefficient
// vectors, staged descriptors, copied static rows, gathered dynamic inputs.
struct RowsSmem {
  double* acc_d;    // 32
  double* acc_l;    // 8 x 32
  double* wsum;     // 8 x 64
  RowSrc* srcs;     // up to ROWS_MAX_SRC descriptors
  double* pre;      // copied rows of M
  double* dyn;      // gathered dynamic inputs
};

__device__ __forceinline__ RowsSmem rows_smem(double* smem, int pre_cap) {
  RowsSmem L;
  L.acc_d = smem;
  L.acc_l = smem + 32;
  L.wsum = smem + 32 + 256;
  L.srcs = reinterpret_cast<RowSrc*>(smem + 32 + 256 + 512);
  L.pre = smem + 32 + 256 + 512 + ROWS_MAX_SRC * (sizeof(RowSrc) / sizeof(double));
  L.dyn = L.pre + pre_cap;
  return L;
}

__device__ __forceinline__ int dyn_start(const RowSrc& S) { return S.dyn_off >= 0 ? S.dyn_off : -(S.dyn_off + 1); }

// Before the wait: stage the descriptors and start the asynchronous copies of
// the static rows; they complete while the CTA waits for its producers.
__device__ void dev_rows_prefetch(const RowsOp& op, const RowSrc* srcs_g, double* smem, int pre_cap) {
  RowsSmem L = rows_smem(smem, pre_cap);
  const int nsrc = min(op.src_end - op.src_begin, ROWS_MAX_SRC);
  {
    const int words = nsrc * (int)(sizeof(RowSrc) / sizeof(long long));
    const long long* g = reinterpret_cast<const long long*>(srcs_g + op.src_begin);
    long long* d = reinterpret_cast<long long*>(L.srcs);
    for (int w = threadIdx.x; w < words; w += blockDim.x) d[w] = g[w];
  }
  __syncthreads();
  for (int s = 0; s < nsrc; ++s) {
    const RowSrc& S = L.srcs[s];
    if (S.pre_off < 0) continue;
    const int nc = S.ncols, tot = op.nr * nc, ld = S.nparts ? nc + 1 : nc;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
      const int r = e / nc, c = e % nc;
      cp_async8(L.pre + S.pre_off + r * ld + c, S.M + r * S.rs + c * S.cs);
    }
  }
}

// After the wait: gather every dynamic input (x vectors, partial products,
// base rows) with eight independent loads in flight per thread.
__device__ void dev_rows_gather(const RowsOp& op, double* smem, int pre_cap) {
  RowsSmem L = rows_smem(smem, pre_cap);
  const int nsrc = min(op.src_end - op.src_begin, ROWS_MAX_SRC);
  const int total = op.dyn_total;
  for (int e0 = threadIdx.x; e0 < total; e0 += 8 * blockDim.x) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * blockDim.x;
      v[u] = 0.0;
      if (e < total) {
        if (e >= op.dyn_base) {
          v[u] = op.base[op.r0 + (e - op.dyn_base)];
        } else {
          // owning source: the last s whose range starts at or before e
          // (sources read from global memory own empty ranges)
          int lo = 0, hi = nsrc - 1;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (dyn_start(L.srcs[mid]) <= e) lo = mid; else hi = mid - 1;
          }
          v[u] = L.srcs[lo].x[e - L.srcs[lo].dyn_off];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < total) L.dyn[e] = v[u];
    }
  }
  __syncthreads();
}

// ts (tracing only, else nullptr): times after the gather and after the sums
__device__ void dev_rows(const RowsOp& op, double* smem, int pre_cap, unsigned long long* ts) {
  RowsSmem L = rows_smem(smem, pre_cap);
  cp_async_wait_all();
  dev_rows_gather(op, smem, pre_cap);
  if (ts && threadIdx.x == 0) ts[0] = global_ns();
  const int nsrc = min(op.src_end - op.src_begin, ROWS_MAX_SRC);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nr = op.nr;
  for (int r = warp; r < nr; r += 8) {
    double acc = 0.0;
    {
      for (int s = 0; s < nsrc; ++s) {
        const RowSrc& S = L.srcs[s];
        if (S.nparts) continue;
        double a = 0.0;
        const int off = S.pre_off, xo = S.dyn_off;
        for (int c0 = lane; c0 < S.ncols; c0 += 256) {
          double xv[8], mv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int c = c0 + 32 * u;
            const bool in = c < S.ncols;
            xv[u] = in ? (xo >= 0 ? L.dyn[xo + c] : S.x[c]) : 0.0;
            mv[u] = in ? (off >= 0 ? L.pre[off + r * S.ncols + c] : S.M[r * S.rs + c * S.cs]) : 0.0;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) a += mv[u] * xv[u];
        }
        acc += S.sign * a;
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) L.acc_d[r] = acc;
  }
  double la = 0.0;
  int k = 0;
  for (int s = 0; s < nsrc; ++s) {
    const RowSrc& S = L.srcs[s];
    if (!S.nparts) continue;
    if ((k++ & 7) != warp) continue;
    double* w = L.wsum + warp * 64;
    const int xo = S.dyn_off;
    for (int l = lane; l < S.ncols; l += 32) {
      double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      int p = 0;
      for (; p + 8 <= S.nparts; p += 8)
#pragma unroll
        for (int u = 0; u < 8; ++u)
          v[u] += xo >= 0 ? L.dyn[xo + (p + u) * S.ncols + l] : S.x[(p + u) * S.ncols + l];
      for (; p < S.nparts; ++p) v[0] += xo >= 0 ? L.dyn[xo + p * S.ncols + l] : S.x[p * S.ncols + l];
      w[l] = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
    }
    __syncwarp();
    if (lane < nr) {
      const int off = S.pre_off;
      double a = 0.0;
      if (off >= 0) {
        const double* Mr = L.pre + off + lane * (S.ncols + 1);
        for (int l = 0; l < S.ncols; ++l) a += Mr[l] * w[l];
      } else {
        const double* Mr = S.M + lane * S.rs;
#pragma unroll 8
        for (int l = 0; l < S.ncols; ++l) a += Mr[l * S.cs] * w[l];
      }
      la += S.sign * a;
    }
    __syncwarp();
  }
  L.acc_l[warp * 32 + lane] = la;
  __syncthreads();
  if (ts && threadIdx.x == 0) ts[1] = global_ns();
  if (threadIdx.x < nr) {
    const int r = threadIdx.x;
    double v = op.base ? L.dyn[op.dyn_base + r] : 0.0;
    v += L.acc_d[r];
    for (int w = 0; w < 8; ++w) v += L.acc_l[w * 32 + r];
    op.out[op.r0 + r] = v;
  }
  __syncthreads();
}

// V' y over one piece: V (static) is copied to shared memory before the
// wait (when it fits), y is gathered after it.
__device__ void dev_vpart_prefetch(const VPartOp& op, double* smem, int vcap) {
  if (op.len * op.kf > vcap) return;
  for (int e = threadIdx.x; e < op.len * op.kf; e += blockDim.x) {
    const int l = e / op.len, r = e % op.len;
    cp_async8(smem + e, op.V + l * op.ldv + r);
  }
}

__device__ void dev_vpart(const VPartOp& op, double* smem, int vcap) {
  const bool pre = op.len * op.kf <= vcap;
  cp_async_wait_all();
  double* ys = smem + vcap;
  for (int r0 = threadIdx.x; r0 < op.len; r0 += 8 * blockDim.x) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int r = r0 + u * blockDim.x;
      v[u] = r < op.len ? op.y[r] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int r = r0 + u * blockDim.x;
      if (r < op.len) ys[r] = v[u];
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int l = warp; l < op.kf; l += 8) {
    double a = 0.0;
    for (int r = lane; r < op.len; r += 32) a += (pre ? smem[l * op.len + r] : op.V[l * op.ldv + r]) * ys[r];
    a = warp_sum(a);
    if (lane == 0) op.part[l] = a;
  }
}

constexpr int EXEC_THREADS = 256;
static_assert(TRUNC_MAXK < EXEC_THREADS, "the truncation core maps rows of C to threads");
static_assert(TRUNC_MAXK_2CTA <= TRUNC_MAXK, "the two-CTA mode takes a subset of the schedules");
// shared memory of an H-LU mode: the truncation core's three K x K matrices and scratch
constexpr size_t factor_smem(int km) { return sizeof(double) * (3 * km * km + 2 * km + 32) + sizeof(int) * 7 * km; }
__host__ __device__ constexpr int mode_trunc_maxk(int m) { return m == FACTOR_MODE_2CTA ? TRUNC_MAXK_2CTA : TRUNC_MAXK; }
// shared memory of a solve mode: the larger of a row task's and a partial-product task's needs
constexpr size_t rows_smem_bytes(int m) {
  return sizeof(double) * (32 + 256 + 512 + mode_prefetch(m) + mode_dyn(m)) + sizeof(RowSrc) * ROWS_MAX_SRC;
}
constexpr size_t vpart_smem_bytes(int m) { return sizeof(double) * (mode_vpart(m) + 256); }
constexpr size_t mode_smem(int m) {
  return mode_factor(m) ? factor_smem(mode_trunc_maxk(m))
                        : (rows_smem_bytes(m) > vpart_smem_bytes(m) ? rows_smem_bytes(m) : vpart_smem_bytes(m));
}
static_assert(mode_ctas(FACTOR_MODE_2CTA) * (mode_smem(FACTOR_MODE_2CTA) + 1024) <= 228 * 1024,
              "two-CTA H-LU mode shared memory");
static_assert(mode_ctas(1) * (mode_smem(1) + 1024) <= 228 * 1024, "latency solve mode shared memory");
static_assert(mode_ctas(2) * (mode_smem(2) + 1024) <= 228 * 1024, "throughput solve mode shared memory");
constexpr unsigned long long WAIT_LIMIT_NS = 4000000000ull;  // 4 s for one dependency wait
#ifndef HM_POLL_NS
#define HM_POLL_NS 0  // pause between two polls of a producer counter (build-time tuning parameter)
#endif

struct ExecArgs {
  const GemmOp* gemm;
  const LuOp* lu;
  const TruncOp* trunc;
  const CopyOp* copy;
  const ReduceOp* reduce;
  const RowsOp* rows;
  const VPartOp* vpart;
  const RowSrc* srcs;
  const Task* tasks;
  const int* wave_begin;
  const OpInfo* ops;
  const int2* deps;  // per dependency edge: (producer op, tasks it has)
  int* counters;
  int* grab;        // next task to hand out
  int ntasks;
  int nops;
  int* err;
  unsigned long long* trace;  // optional, TRACE_STRIDE per task: grabbed, producers-ready, finished (ns), CTA, sub-steps
  unsigned long long wait_ns; // limit of one dependency wait
};

// Release add at GPU scope: a CTA-wide barrier followed by one thread's
// release publishes all of the CTA's prior writes; a reader that observes the
// count and then executes an acquire fence sees them, and so does the rest of
// its CTA after the next barrier.
__device__ __forceinline__ void red_release_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until every producer of op `id` has finished all its tasks.  Warp 0
// polls the counters with relaxed loads (lanes split the producer list); each
// polling lane's acquire fence after observing the counts pairs with the
// producers' release adds.  Bounded in time.
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ bool wait_deps(const ExecArgs& a, int id) {
  __shared__ int ok;
  if (threadIdx.x < 32) {
    const OpInfo op = a.ops[id];
    bool good = true;
    const unsigned long long t0 = global_ns();
    for (int k = op.dep_begin + (int)threadIdx.x; k < op.dep_end && good; k += 32) {
      const int2 dn = a.deps[k];  // the producer's task count travels with the edge
      const int need = dn.y;
      const int* c = a.counters + dn.x;
      unsigned polls = 0;
      while (ld_relaxed(c) < need) {
#if HM_POLL_NS > 0
        __nanosleep(HM_POLL_NS);
#endif
        if ((++polls & 255u) == 0 && global_ns() - t0 > a.wait_ns) {
          atomicOr(a.err, DEVERR_TIMEOUT);
          good = false;
          break;
        }
      }
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    good = __all_sync(0xffffffffu, good);
    if (threadIdx.x == 0) ok = good ? 1 : 0;
  }
  __syncthreads();
  return ok != 0;
}

// Tasks are taken in topological order from a global counter, so a CTA
// waiting on a producer never holds up a task that is ready elsewhere.
template <int MODE>
__global__ void __launch_bounds__(EXEC_THREADS, mode_ctas(MODE)) exec_kernel(ExecArgs a) {
  constexpr bool SOLVE = !mode_factor(MODE);
  extern __shared__ double smem[];
  // the task index, in two slots used alternately: thread 0 writes the other
  // slot next time, after barriers that every thread passes only once it has
  // read this one, so no barrier is needed between the read and the next write
  __shared__ int next[2];
  int slot = 0;
  // descriptor of the current op (factorisation), copied before the wait
  __shared__ union OpDesc {
    int w[1];
    GemmOp gemm;
    LuOp lu;
    TruncOp trunc;
    CopyOp copy;
    ReduceOp reduce;
  } opdesc;
  for (;;) {
    if (threadIdx.x == 0) next[slot] = atomicAdd(a.grab, 1);
    __syncthreads();
    const int t = next[slot];
    slot ^= 1;
    if (t >= a.ntasks) return;
    const Task T = a.tasks[t];
    if (a.trace && threadIdx.x == 0) {
      a.trace[TRACE_STRIDE * (size_t)t] = global_ns();
      a.trace[TRACE_STRIDE * (size_t)t + 3] = blockIdx.x;
      unsigned sm;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
      a.trace[TRACE_STRIDE * (size_t)t + 6] = sm;
    }
    if constexpr (SOLVE) {
      if (T.kind == TK_ROWS) dev_rows_prefetch(a.rows[T.op], a.srcs, smem, mode_prefetch(MODE));
      if (T.kind == TK_VPART) dev_vpart_prefetch(a.vpart[T.op], smem, mode_vpart(MODE));
    } else {
      // the op's descriptor to shared memory while warp 0 waits for its producers
      if (threadIdx.x >= 32) {
        const int* src = nullptr;
        int words = 0;
        switch (T.kind) {
          case TK_GEMM: src = reinterpret_cast<const int*>(a.gemm + T.op); words = sizeof(GemmOp) / 4; break;
          case TK_LU: src = reinterpret_cast<const int*>(a.lu + T.op); words = sizeof(LuOp) / 4; break;
          case TK_TRUNC: src = reinterpret_cast<const int*>(a.trunc + T.op); words = sizeof(TruncOp) / 4; break;
          case TK_COPY: src = reinterpret_cast<const int*>(a.copy + T.op); words = sizeof(CopyOp) / 4; break;
          case TK_REDUCE: src = reinterpret_cast<const int*>(a.reduce + T.op); words = sizeof(ReduceOp) / 4; break;
          default: break;
        }
        for (int w = threadIdx.x - 32; w < words; w += blockDim.x - 32) opdesc.w[w] = src[w];
      }
    }
    if (!wait_deps(a, T.id)) {
      cp_async_wait_all();  // no copy may outlive the CTA
      return;
    }
    if (a.trace && threadIdx.x == 0) a.trace[TRACE_STRIDE * (size_t)t + 1] = global_ns();
    if constexpr (!SOLVE) {
      switch (T.kind) {
        case TK_GEMM: dev_gemm_tile(opdesc.gemm, T.sub, smem, a.err); break;
        case TK_LU:
          if (opdesc.lu.pad & LU_DF) dev_lu_base_dd(opdesc.lu, a.err, smem);
          else dev_lu_base(opdesc.lu, a.err, smem);
          break;
        case TK_TRUNC: dev_trunc<mode_trunc_maxk(MODE)>(opdesc.trunc, a.err, smem); break;
        case TK_COPY: dev_copy(opdesc.copy, T.sub, T.nsub); break;
        case TK_REDUCE: dev_reduce(opdesc.reduce, T.sub, T.nsub); break;
        default: break;
      }
    }
    switch (T.kind) {
      case TK_COPY:
        if constexpr (SOLVE) dev_copy(a.copy[T.op], T.sub, T.nsub);
        break;
      case TK_REDUCE:
        if constexpr (SOLVE) dev_reduce(a.reduce[T.op], T.sub, T.nsub);
        break;
      case TK_ROWS:
        if constexpr (SOLVE)
          dev_rows(a.rows[T.op], smem, mode_prefetch(MODE), a.trace ? a.trace + TRACE_STRIDE * (size_t)t + 4 : nullptr);
        break;
      case TK_VPART:
        if constexpr (SOLVE) dev_vpart(a.vpart[T.op], smem, mode_vpart(MODE));
        break;
      default: break;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      red_release_add(a.counters + T.id, 1);  // publishes the CTA's writes (after the barrier)
      if (a.trace) a.trace[TRACE_STRIDE * (size_t)t + 2] = global_ns();
    }
  }
}

}  // namespace

void plan_rows_staging(RowsOp& op, RowSrc* src, int mode) {
  const int pre_cap = mode_prefetch(mode), dyn_cap = mode_dyn(mode);
  const int nsrc = op.src_end - op.src_begin;
  int used = 0, dused = 0;
  for (int s = 0; s < nsrc; ++s) {
    RowSrc& S = src[s];
    const int need = op.nr * (S.nparts ? S.ncols + 1 : S.ncols);
    if (s < ROWS_MAX_SRC && used + need <= pre_cap) {
      S.pre_off = used;
      used += need;
    } else {
      S.pre_off = -1;
    }
    const int dneed = S.nparts ? S.nparts * S.ncols : S.ncols;
    if (s < ROWS_MAX_SRC && dused + dneed <= dyn_cap - 32) {
      S.dyn_off = dused;
      dused += dneed;
    } else {
      S.dyn_off = -(dused + 1);
    }
  }
  op.dyn_base = dused;
  op.dyn_total = dused + (op.base ? op.nr : 0);
}

int gemm_shape(int m, int n) { return n <= 16 && m > 16 ? 1 : (m <= 16 && n > 16 ? 2 : 0); }
int shape_tiles(int sh, int m, int n) {
  const int tm = sh == 1 || sh == 3 ? 64 : sh == 2 ? 16 : 32, tn = sh == 2 || sh == 3 ? 64 : sh == 1 ? 16 : 32;
  return ((m + tm - 1) / tm) * ((n + tn - 1) / tn);
}
int gemm_tiles(int m, int n) { return shape_tiles(gemm_shape(m, n), m, n); }

int upload_schedule(const std::vector<Wave>& waves, const OpGraph& graph, DevSchedule& S,
                    std::vector<void*>& allocs, const std::vector<RowSrc>* srcs, int mode) {
  return upload_schedules({SchedPart{&waves, &graph, srcs}}, S, allocs, mode, false);
}

int upload_schedules(const std::vector<SchedPart>& parts, DevSchedule& S, std::vector<void*>& allocs, int mode,
                     bool restage, cudaStream_t copy_stream) {
  std::vector<RowsOp> ro;
  std::vector<VPartOp> vp;
  std::vector<GemmOp> g;
  std::vector<LuOp> l;
  std::vector<TruncOp> tr;
  std::vector<CopyOp> c;
  std::vector<ReduceOp> r;
  std::vector<Task> tasks;
  std::vector<int> wb;
  std::vector<RowSrc> msrc;
  // op id and row-source offsets of every part
  std::vector<int> off(parts.size() + 1, 0), soff(parts.size() + 1, 0);
  size_t nw = 0;
  for (size_t p = 0; p < parts.size(); ++p) {
    off[p + 1] = off[p] + parts[p].graph->size();
    soff[p + 1] = soff[p] + (parts[p].srcs ? (int)parts[p].srcs->size() : 0);
    nw = std::max(nw, parts[p].waves->size());
  }
  const int nops = off.back();
  std::vector<OpInfo> info(std::max(nops, 1), OpInfo{0, 0, 0, 0});
  std::vector<int> prio(std::max(nops, 1), 0);
  std::vector<int> deps;
  size_t ndeps = 0;
  for (const SchedPart& P : parts) ndeps += P.graph->flat.size();
  deps.reserve(ndeps);
  for (size_t p = 0; p < parts.size(); ++p) {
    const OpGraph& gr = *parts[p].graph;
    for (int i = 0; i < gr.size(); ++i) {
      const int id = off[p] + i;
      prio[id] = gr.prio_of(i);
      info[id].dep_begin = (int)deps.size();
      for (const int* d = gr.begin(i); d != gr.end(i); ++d) deps.push_back(*d + off[p]);
      info[id].dep_end = (int)deps.size();
    }
  }
  if (soff.back() > 0) {
    msrc.reserve(soff.back());
    for (const SchedPart& P : parts)
      if (P.srcs) msrc.insert(msrc.end(), P.srcs->begin(), P.srcs->end());
  }
  // copies and reductions are split so that one task does about 2048 FP64
  // operations (a few microseconds on one SM)
  auto chunks = [](int64_t work) { return (int)std::max<int64_t>(1, std::min<int64_t>(64, work / 2048)); };
  const char* g64 = std::getenv("HM_GEMM_FP64");  // FP64 instead of double-float GEMM tiles
  const bool gemm_fp64 = g64 && g64[0] == '1';
  // GEMMs of at least big_tiles 32 x 32 tiles, in waves of at least big_wave
  // such tiles, run as 64 x 64 tiles (a quarter of the tasks; the same
  // arithmetic per output)
  int big_tiles = HM_GEMM_BIG_TILES;
  if (const char* gb = std::getenv("HM_GEMM_BIG_TILES")) big_tiles = std::atoi(gb);
  int64_t big_wave = HM_GEMM_BIG_WAVE;
  if (const char* gw = std::getenv("HM_GEMM_BIG_WAVE")) big_wave = std::atoll(gw);
  const char* ldf = std::getenv("HM_LU_DF");  // double-float instead of FP64 base LUs
  const bool lu_df = ldf && ldf[0] == '1';
  // the tasks of one op (kind, index k in its wave's list of that kind)
  auto emit = [&](size_t p, const Wave& W, int kind, size_t k, bool wide) {
    const int o0 = off[p];
    if (kind == TK_GEMM) {
      GemmOp o = W.gemm[k];
      int sh = gemm_shape(o.m, o.n);
      if (sh == 0 && wide && big_tiles > 0 && shape_tiles(0, o.m, o.n) >= big_tiles) sh = 3;
      o.shape = sh | (gemm_fp64 ? GEMM_FP64 : 0);
      int nt = shape_tiles(sh, o.m, o.n), id = W.gemm_id[k] + o0;
      for (int t = 0; t < nt; ++t) tasks.push_back({TK_GEMM, (int)g.size(), t, nt, id});
      info[id].ntasks = nt;
      g.push_back(o);
    } else if (kind == TK_LU) {
      tasks.push_back({TK_LU, (int)l.size(), 0, 1, W.lu_id[k] + o0});
      info[W.lu_id[k] + o0].ntasks = 1;
      LuOp o = W.lu[k];
      o.pad = lu_df ? LU_DF : 0;
      l.push_back(o);
    } else if (kind == TK_TRUNC) {
      tasks.push_back({TK_TRUNC, (int)tr.size(), 0, 1, W.trunc_id[k] + o0});
      info[W.trunc_id[k] + o0].ntasks = 1;
      tr.push_back(W.trunc[k]);
    } else if (kind == TK_COPY) {
      const CopyOp& o = W.copy[k];
      int nc = chunks((int64_t)o.m * o.n), id = W.copy_id[k] + o0;
      for (int t = 0; t < nc; ++t) tasks.push_back({TK_COPY, (int)c.size(), t, nc, id});
      info[id].ntasks = nc;
      c.push_back(o);
    } else if (kind == TK_REDUCE) {
      const ReduceOp& o = W.reduce[k];
      int nc = chunks((int64_t)o.m * o.n * std::max(o.nparts, 1)), id = W.reduce_id[k] + o0;
      for (int t = 0; t < nc; ++t) tasks.push_back({TK_REDUCE, (int)r.size(), t, nc, id});
      info[id].ntasks = nc;
      r.push_back(o);
    } else if (kind == TK_ROWS) {
      RowsOp o = W.rows[k];
      o.src_begin += soff[p];
      o.src_end += soff[p];
      if (restage) plan_rows_staging(o, msrc.data() + o.src_begin, mode);
      const int id = W.rows_id[k] + o0;
      tasks.push_back({TK_ROWS, (int)ro.size(), 0, o.nr, id});  // nsub: rows of the chunk
      info[id].ntasks += 1;  // the chunks of one row op share its id
      ro.push_back(o);
    } else {
      tasks.push_back({TK_VPART, (int)vp.size(), 0, 1, W.vpart_id[k] + o0});
      info[W.vpart_id[k] + o0].ntasks = 1;
      vp.push_back(W.vpart[k]);
    }
  };
  auto count_of = [](const Wave& W, int kind) -> size_t {
    switch (kind) {
      case TK_GEMM: return W.gemm.size();
      case TK_LU: return W.lu.size();
      case TK_TRUNC: return W.trunc.size();
      case TK_COPY: return W.copy.size();
      case TK_REDUCE: return W.reduce.size();
      case TK_ROWS: return W.rows.size();
      default: return W.vpart.size();
    }
  };
  // Tasks are handed out in this order: wave by wave (an op's producers lie
  // in earlier waves, so a CTA only ever waits for tasks handed out before its
  // own).  Within a wave by the ops' urgency (OpGraph::prio: for the H-LU the
  // diagonal position at which the result is first needed), ties by kind
  // (base LUs, truncations, split-K reductions and copies before GEMM tiles),
  // so that the ops on the factorisation's dependency chain start as soon as
  // their producers finish instead of after the wave's far-field work.  (A
  // topological order by urgency alone, across waves, defers the far field
  // until the chain waits for it: 2x slower at 1D N = 65536.)
  static const int kinds[] = {TK_LU, TK_TRUNC, TK_REDUCE, TK_COPY, TK_GEMM, TK_ROWS, TK_VPART};
  for (size_t w = 0; w < nw; ++w) {
    wb.push_back((int)tasks.size());
    // a wave of many GEMM tiles keeps every SM busy whatever the tile size:
    // its large GEMMs take 64 x 64 tiles (a wave of few tiles keeps 32 x 32
    // ones, which finish sooner on the dependency chain)
    int64_t wt = 0;
    for (size_t p = 0; p < parts.size(); ++p)
      if (w < parts[p].waves->size())
        for (const GemmOp& o : (*parts[p].waves)[w].gemm) wt += gemm_tiles(o.m, o.n);
    const bool wide = wt >= big_wave;
    for (int kind : kinds)
      for (size_t p = 0; p < parts.size(); ++p) {
        if (w >= parts[p].waves->size()) continue;
        const Wave& W = (*parts[p].waves)[w];
        for (size_t k = 0; k < count_of(W, kind); ++k) emit(p, W, kind, k, wide);
      }
    std::stable_sort(tasks.begin() + wb.back(), tasks.end(),
                     [&](const Task& x, const Task& y) { return prio[x.id] < prio[y.id]; });
  }
  wb.push_back((int)tasks.size());
  S.nwaves = (int)nw;
  S.nops = nops;
  S.ntasks = (int64_t)tasks.size();
  auto up = [&](auto& vec, auto** dst) -> int {
    size_t bytes = std::max<size_t>(vec.size() * sizeof(vec[0]), 16);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return HM_ERR_OOM;
    allocs.push_back(p);
    if (!vec.empty()) {
      const size_t n = vec.size() * sizeof(vec[0]);
      const cudaError_t e = copy_stream ? cudaMemcpyAsync(p, vec.data(), n, cudaMemcpyHostToDevice, copy_stream)
                                        : cudaMemcpy(p, vec.data(), n, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return HM_ERR_CUDA;
    }
    *dst = (std::remove_reference_t<decltype(**dst)>*)p;
    return HM_OK;
  };
  int st;
  if ((st = up(g, &S.gemm)) != HM_OK) return st;
  if ((st = up(l, &S.lu)) != HM_OK) return st;
  if ((st = up(tr, &S.trunc)) != HM_OK) return st;
  if ((st = up(c, &S.copy)) != HM_OK) return st;
  if ((st = up(r, &S.reduce)) != HM_OK) return st;
  if ((st = up(ro, &S.rows)) != HM_OK) return st;
  if ((st = up(vp, &S.vpart)) != HM_OK) return st;
  if ((st = up(msrc, &S.srcs)) != HM_OK) return st;
  if ((st = up(tasks, &S.tasks)) != HM_OK) return st;
  if (g.empty() && l.empty() && tr.empty()) {
    S.mode = mode == SOLVE_MODE_THROUGHPUT ? 2 : 1;
  } else {
    // H-LU: two CTAs per SM when every truncation core fits the smaller
    // shared-memory layout (HM_EXEC_2CTA=0: always one)
    int kmax = 0;
    for (const TruncOp& o : tr) kmax = std::max(kmax, o.K);
    const char* two = std::getenv("HM_EXEC_2CTA");
    S.mode = kmax <= TRUNC_MAXK_2CTA && !(two && two[0] == '0') ? FACTOR_MODE_2CTA : 0;
  }
  if (std::getenv("HM_PHASE_TRACE")) S.host_tasks.swap(tasks);  // kept for tracing only
  if ((st = up(wb, &S.wave_begin)) != HM_OK) return st;
  // Test-only fault injection (failure detection of the bounded waits):
  // HM_TEST_STALL_OP=<op> makes op <op> of this schedule require one task more
  // than it has, so its consumers' waits can only run out; HM_WAIT_LIMIT_MS
  // shortens the limit of every dependency wait of the schedule.
  if (const char* so = std::getenv("HM_TEST_STALL_OP")) {
    const int id = std::atoi(so);
    if (id >= 0 && id < nops) info[id].ntasks += 1;
  }
  if ((st = up(info, &S.ops)) != HM_OK) return st;
  {  // dependency edges with the producer's task count (one load fewer per wait)
    std::vector<int2> deps2(deps.size());
    for (size_t e = 0; e < deps.size(); ++e) deps2[e] = make_int2(deps[e], info[deps[e]].ntasks);
    if ((st = up(deps2, &S.deps)) != HM_OK) return st;
  }
  S.wait_ns = WAIT_LIMIT_NS;
  if (const char* wl = std::getenv("HM_WAIT_LIMIT_MS"))
    if (std::atoll(wl) > 0) S.wait_ns = (unsigned long long)std::atoll(wl) * 1000000ull;
  std::vector<int> cnt(nops + 1, 0);
  if ((st = up(cnt, &S.counters)) != HM_OK) return st;
  if (copy_stream && cudaStreamSynchronize(copy_stream) != cudaSuccess) return HM_ERR_CUDA;
  return HM_OK;
}

namespace {
int g_exec_grid[EXEC_MODES] = {0, 0, 0, 0};
void* exec_fn(int m) {
  switch (m) {
    case 0: return (void*)exec_kernel<0>;
    case 1: return (void*)exec_kernel<1>;
    case 2: return (void*)exec_kernel<2>;
    default: return (void*)exec_kernel<FACTOR_MODE_2CTA>;
  }
}
}

int prepare_executor(const DevSchedule& S) {
  const int m = S.mode;
  if (g_exec_grid[m] != 0) return HM_OK;
  void* fn = exec_fn(m);
  const size_t smem = mode_smem(m);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return HM_ERR_CUDA;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, EXEC_THREADS, smem) != cudaSuccess || per < 1)
    return HM_ERR_CUDA;
  g_exec_grid[m] = sms * std::min(per, mode_ctas(m));
  return HM_OK;
}

int run_schedule(const DevSchedule& S, int* d_err, cudaStream_t st, unsigned long long* trace) {
  if (S.ntasks == 0) return HM_OK;
  const int m = S.mode;
  void* fn = exec_fn(m);
  const size_t smem = mode_smem(m);
  int s = prepare_executor(S);
  if (s != HM_OK) return s;
  int* grid = g_exec_grid;
  // counters[nops] is the task dispenser
  if (cudaMemsetAsync(S.counters, 0, sizeof(int) * (S.nops + 1), st) != cudaSuccess) return HM_ERR_CUDA;
  ExecArgs a{S.gemm, S.lu, S.trunc, S.copy, S.reduce, S.rows, S.vpart, S.srcs, S.tasks, S.wave_begin,
             S.ops, S.deps, S.counters, S.counters + S.nops, (int)S.ntasks, S.nops, d_err, trace, S.wait_ns};
  void* args[] = {&a};
  count_launches(1);
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid[m]), dim3(EXEC_THREADS), args, smem, st);
  return e == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

}  // namespace hm
