// Device-side helpers shared by the kernels: entry evaluation and reductions.
#pragma once

#include <cuda_runtime.h>

#include "hm_internal.h"

namespace hm {

// Device error word bits (set by kernels, read back by hm_sync / hm_stats).
enum : int {
  DEVERR_INDEX = 1,      // an index fell outside its buffer (access skipped)
  DEVERR_NONFINITE = 2,  // a non-finite value appeared where it must not
  DEVERR_RANKCAP = 4,    // a low-rank sum needed more than its capacity
  DEVERR_ZEROPIVOT = 8,  // a zero pivot in an unpivoted dense LU
  DEVERR_TIMEOUT = 16,   // a bounded wait in a persistent kernel gave up
};

// ---- double-float arithmetic (unevaluated pairs of floats, about 48 bits)

// Double-float split of an FP64 operand, integer operations only (no FP64
// instruction, which this GPU issues at 1/64 of the FP32 rate): hi is the
// significand rounded to nearest at 24 bits (an integer add on the float's bit
// pattern carries into the exponent), lo the signed remainder, 29 bits rounded
// to 24, so a = hi + lo + r with |r| <= 2^-49 |a|.  |a| < 2^-126 is flushed
// to zero and the low part of |a| < 2^-74 is dropped (absolute error below
// 2^-74); |a| >= 2^128 (after rounding), inf and NaN set `bad`.
__device__ __forceinline__ float2 df_split(double a, bool& bad) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(a);
  const unsigned hw = (unsigned)(u >> 32), lw = (unsigned)u;
  const int e = (int)((hw >> 20) & 0x7ffu) - 1023;
  if (e < -126) return make_float2(0.f, 0.f);
  if (e > 127) {
    bad = true;
    return make_float2(0.f, 0.f);
  }
  const unsigned sgn = hw & 0x80000000u;
  const unsigned r = lw & 0x1fffffffu;  // the 29 bits below hi's last, in units of 2^(e-52)
  const unsigned up = r >> 28;          // round half up on the magnitude
  const unsigned hb = (((unsigned)(e + 127) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29)) + up;
  if ((hb >> 23) >= 255u) {
    bad = true;
    return make_float2(0.f, 0.f);
  }
  float lo = 0.f;
  if (e >= -74) lo = __fmul_rn(__int2float_rn((int)r - (int)(up << 29)), __int_as_float((e - 52 + 127) << 23));
  return make_float2(__uint_as_float(sgn | hb), sgn ? -lo : lo);
}

// Products by Dekker's method, sums by Knuth's two-sum (Dekker 1971; Knuth,
// TAOCP 2, sec. 4.2.2), reciprocal by one Newton step from the float
// reciprocal; __f*_rn keep the compiler from contracting the error terms.
__device__ __forceinline__ float2 dd_renorm(float hi, float lo) {
  const float s = __fadd_rn(hi, lo);
  return make_float2(s, __fsub_rn(lo, __fsub_rn(s, hi)));
}
__device__ __forceinline__ float2 dd_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return dd_renorm(p, e);
}
__device__ __forceinline__ float2 dd_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float bb = __fsub_rn(s, a.x);
  const float t = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
  return dd_renorm(s, __fadd_rn(t, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 dd_neg(float2 a) { return make_float2(-a.x, -a.y); }
// c - a b
__device__ __forceinline__ float2 dd_fnms(float2 c, float2 a, float2 b) { return dd_add(c, dd_neg(dd_mul(a, b))); }
// 1 / d: r0 = float reciprocal, r = r0 + r0 (1 - d r0) with the residual in double-float
__device__ __forceinline__ float2 dd_recip(float2 d) {
  const float r0 = __frcp_rn(d.x);
  const float2 e = dd_add(make_float2(1.f, 0.f), dd_neg(dd_mul(d, make_float2(r0, 0.f))));
  return dd_add(make_float2(r0, 0.f), dd_mul(make_float2(r0, 0.f), e));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for a cooperative launch: bar[0] counts arrivals, bar[1]
// is the generation.  Waits at most limit_ns; returns false (and sets
// DEVERR_TIMEOUT) if the other CTAs did not arrive in time.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* err,
                                             unsigned long long limit_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    const unsigned g = *vgen;
    __threadfence();
    ok = 1;
    if (atomicAdd(bar, 1u) == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      // pure polling (a sleeping warp wakes up far later than requested);
      // the clock is checked every 256 polls to bound the wait
      const unsigned long long t0 = global_ns();
      unsigned polls = 0;
      while (*vgen == g) {
        if ((++polls & 255u) == 0 && global_ns() - t0 > limit_ns) {
          atomicOr(err, DEVERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Jump entry of a variable-order row p (2D stable kernel): trapezoid weight
// times c_{2,s_p} / |y|^{2+2 s_p} at y = h j, i.e. B_p (|j|^2)^{E_p} with
// B_p = c_{2,s_p} h^{-2 s_p}, E_p = -(1 + s_p), halved on each window face.
__device__ __forceinline__ double var_jump(const EntryCtx& E, int p, int a0, int a1) {
  if (a0 > E.nw || a1 > E.nw) return 0.0;  // outside the window [-L_W, L_W]^2
  double v = E.rowB[p] * pow((double)a0 * a0 + (double)a1 * a1, E.rowE[p]);
  if (a0 == E.nw) v *= 0.5;
  if (a1 == E.nw) v *= 0.5;
  return v;
}

// G between Morton positions p (row) and q (column): the formula of Eq. Aij
// (sign-flipped) with the singular corrections, evaluated from the offset
// table w(j) nu(|j| h) and the row-independent constants.
__device__ __forceinline__ double gen_entry(const EntryCtx& E, const GenConst& g, int p, int q) {
  int2 cp = E.coord[p];
  int2 cq = E.coord[q];
  int d0 = cq.x - cp.x;
  int d1 = cq.y - cp.y;
  int a0 = d0 < 0 ? -d0 : d0;
  int a1 = d1 < 0 ? -d1 : d1;
  if (E.rowB) {  // variable order: per-row constants, stencil kappa_p (a = b = c = 0)
    if (d0 == 0 && d1 == 0) return E.rowD[p];
    double v = var_jump(E, p, a0, a1);
    if (a0 + a1 == 1) v += E.rowK[p];
    return v;
  }
  if (d0 == 0 && d1 == 0) return g.diag;
  double v = E.tab[(size_t)a1 * E.n0 + a0];
  if (a0 + a1 == 1) {
    if (a0 == 1) v = v + (d0 > 0 ? g.stencil_p[0] : g.stencil_m[0]);
    else v = v + (d1 > 0 ? g.stencil_p[1] : g.stencil_m[1]);
  }
  return v;
}

// Far entries (never the diagonal or an axis neighbour): table lookup only.
__device__ __forceinline__ double far_entry(const EntryCtx& E, int p, int q) {
  int2 cp = E.coord[p];
  int2 cq = E.coord[q];
  int a0 = abs(cq.x - cp.x);
  int a1 = abs(cq.y - cp.y);
  if (E.rowB) return var_jump(E, p, a0, a1);
  return E.tab[(size_t)a1 * E.n0 + a0];
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; every thread gets the result.  scratch: >= 32 elements.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* scratch) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  T r = 0;
  for (int i = 0; i < nw; ++i) r += scratch[i];
  __syncthreads();
  return r;
}

// Block-wide argmax of |v| with ties to the smallest index.  Every thread gets
// (best value (signed), best index); idx < 0 means "no candidate".
__device__ __forceinline__ void argmax_merge(double& bv, int& bi, double v, int i) {
  double av = fabs(v), ab = fabs(bv);
  if (i >= 0 && (bi < 0 || av > ab || (av == ab && i < bi))) { bv = v; bi = i; }
}

__device__ __forceinline__ void block_argmax(double& v, int& idx, double* sv, int* si) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, v, o);
    int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    argmax_merge(v, idx, ov, oi);
  }
  __syncthreads();
  if (lane == 0) { sv[w] = v; si[w] = idx; }
  __syncthreads();
  double bv = 0;
  int bi = -1;
  for (int i = 0; i < nw; ++i) argmax_merge(bv, bi, sv[i], si[i]);
  __syncthreads();
  v = bv;
  idx = bi;
}

}  // namespace hm
