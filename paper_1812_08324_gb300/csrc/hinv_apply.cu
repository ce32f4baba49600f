// Per-step application of the hierarchical inverses of the triangular factors
// (the H-triangular solves of App. "LU Decomposition" as products):
//
//   y = X b,   y_i = sum_{j in leaf(i), j <= i (L) / j >= i (U)} X_leaf[i, j] b_j
//                    + sum_{tau: i in tgt(tau)} P_tau[i, :] (Q_tau^T b[src(tau)])
//
//   1. hinv_t_kernel  t_tau = Q_tau^T b[src(tau)]: one CTA per 256-row chunk of
//                     every source range (Q column-major, warp per column);
//                     the last CTA of a block sums the chunks' partials in
//                     chunk order
//   2. hinv_r_kernel  one CTA per 64-row chunk of a leaf, lane per two rows:
//                     the leaf's triangle (stored column-major) plus P rows
//                     times t of every block whose target holds the rows,
//                     split evenly over the warps by host-built column runs
// Every load is a run of consecutive entries and every entry is read once:
// the step is bandwidth-bound if the arithmetic keeps up.  GB300 issues FP64
// at about two multiply-adds per clock per SM, below what these products
// need, so the FP64-accurate path stores each entry as an unevaluated pair
// of floats (hi + lo, 48-bit significand, the same 8 bytes) and multiplies
// and accumulates in double-float arithmetic on the FP32 pipes (Dekker's
// product and Knuth's two-sum; Dekker 1971, Knuth TAOCP 2 sec. 4.2.2).  The
// other storages: FP64 with FP64 arithmetic (kept for checks), FP32 and BF16
// with FP32 accumulation (mixed precision).  Vectors are FP64, Morton order.
#include <cuda_bf16.h>

#include "hinv.h"
#include "hm_device.cuh"
#include "hm_kernels.h"

namespace hm {

namespace {

// ---- double-float arithmetic (no contraction: every step rounds as written;
// FP64 vector entries are split with integer operations, df_split of
// hm_device.cuh)
// s += a x   (a, x and s unevaluated pairs; the lo * lo term is dropped)
__device__ __forceinline__ void df_mac(float2& s, float2 a, float2 x) {
  const float p = __fmul_rn(a.x, x.x);
  const float e = fmaf(a.x, x.x, -p);                // exact error of the product
  const float c = fmaf(a.x, x.y, fmaf(a.y, x.x, e));  // cross terms
  const float t = __fadd_rn(s.x, p);                  // two-sum of the high parts
  const float z = __fsub_rn(t, s.x);
  const float err = __fadd_rn(__fsub_rn(s.x, __fsub_rn(t, z)), __fsub_rn(p, z));
  s.x = t;
  s.y = __fadd_rn(s.y, __fadd_rn(err, c));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float t = __fadd_rn(a.x, b.x);
  const float z = __fsub_rn(t, a.x);
  const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(t, z)), __fsub_rn(b.x, z));
  const float lo = __fadd_rn(__fadd_rn(a.y, b.y), err);
  const float hi = __fadd_rn(t, lo);
  return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, t)));
}

// ---- storage / arithmetic traits per precision
//   S: stored element, X: multiplicand (staged vector entries), A: accumulator
template <int P> struct Tr;
template <> struct Tr<HINV_F64> {
  using S = double; using X = double; using A = double;
  static __device__ __forceinline__ X cvt(double v) { return v; }
  static __device__ __forceinline__ S ld(const S* p) { return __ldg(p); }
  static __device__ __forceinline__ S sz() { return 0.0; }
  static __device__ __forceinline__ void mac(A& s, S a, X x) { s = fma(a, x, s); }
  static __device__ __forceinline__ A zero() { return 0.0; }
  static __device__ __forceinline__ A add(A a, A b) { return a + b; }
  static __device__ __forceinline__ double fin(A a) { return a; }
};
template <> struct Tr<HINV_DF> {
  using S = float2; using X = float2; using A = float2;
  static __device__ __forceinline__ X cvt(double v) {
    bool bad = false;  // vector entries are finite
    return df_split(v, bad);
  }
  static __device__ __forceinline__ S ld(const S* p) { return __ldg(p); }
  static __device__ __forceinline__ S sz() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ void mac(A& s, S a, X x) { df_mac(s, a, x); }
  static __device__ __forceinline__ A zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ A add(A a, A b) { return df_add(a, b); }
  static __device__ __forceinline__ double fin(A a) { return (double)a.x + (double)a.y; }
};
template <> struct Tr<HINV_F32> {
  using S = float; using X = float; using A = float;
  static __device__ __forceinline__ X cvt(double v) { return (float)v; }
  static __device__ __forceinline__ S ld(const S* p) { return __ldg(p); }
  static __device__ __forceinline__ S sz() { return 0.f; }
  static __device__ __forceinline__ void mac(A& s, S a, X x) { s = fmaf(a, x, s); }
  static __device__ __forceinline__ A zero() { return 0.f; }
  static __device__ __forceinline__ A add(A a, A b) { return a + b; }
  static __device__ __forceinline__ double fin(A a) { return (double)a; }
};
template <> struct Tr<HINV_BF16> {
  using S = __nv_bfloat16; using X = float; using A = float;
  static __device__ __forceinline__ X cvt(double v) { return (float)v; }
  static __device__ __forceinline__ S ld(const S* p) { return *p; }
  static __device__ __forceinline__ S sz() { return __float2bfloat16(0.f); }
  static __device__ __forceinline__ void mac(A& s, S a, X x) { s = fmaf(__bfloat162float(a), x, s); }
  static __device__ __forceinline__ A zero() { return 0.f; }
  static __device__ __forceinline__ A add(A a, A b) { return a + b; }
  static __device__ __forceinline__ double fin(A a) { return (double)a; }
};

// Warp sum by a fixed xor butterfly; lane 0's result is used.
__device__ __forceinline__ double shfl_x(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float shfl_x(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float2 shfl_x(float2 v, int o) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}
__device__ __forceinline__ double shfl_i(double v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ float shfl_i(float v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ float2 shfl_i(float2 v, int l) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, l), __shfl_sync(0xffffffffu, v.y, l));
}
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ float2 ld_cg(const float2* p) { return __ldcg(p); }
template <int P>
__device__ __forceinline__ typename Tr<P>::A warp_sum(typename Tr<P>::A a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = Tr<P>::add(a, shfl_x(a, o));
  return a;
}

constexpr int T_WARPS = 4;

// t_tau = Q_tau^T b over one 256-row chunk of the source range.  Q is stored
// column-major, so a warp reads a column of the chunk as 256 consecutive
// entries: lane takes rows lane + 32u (u < 8) and holds their b values in
// registers; warps take columns, two at a time (sixteen loads issued before
// any is used).  Each column's sum is reduced over the warp by a fixed
// butterfly and written per chunk; the last chunk of a block sums the chunks'
// partials in chunk order.  Deterministic.
template <int P>
__device__ __forceinline__ void t_body(const HinvApply& H, int c, const double* __restrict__ b) {
  using T = Tr<P>;
  __shared__ int last;
  const int4 tc = H.tch[c];
  const HinvNode nd = H.nodes[tc.x];
  const int k = H.rank[tc.x];
  const int j0 = tc.y, len = min(HINV_TCH, nd.src_n - j0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  typename T::X x[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int r = lane + 32 * u;
    x[u] = T::cvt(r < len ? b[nd.src0 + j0 + r] : 0.0);
  }
  const typename T::S* Q = static_cast<const typename T::S*>(H.q_pool) + nd.qoff + j0 + lane;
  for (int l = warp; l < k; l += 2 * T_WARPS) {  // warp-uniform
    const int l2 = l + T_WARPS;
    typename T::S va[8], vb[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const bool in = lane + 32 * u < len;
      va[u] = in ? T::ld(Q + (int64_t)l * nd.qld + 32 * u) : T::sz();
      vb[u] = (in && l2 < k) ? T::ld(Q + (int64_t)l2 * nd.qld + 32 * u) : T::sz();
    }
    typename T::A sa = T::zero(), sb = T::zero();
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      T::mac(sa, va[u], x[u]);
      T::mac(sb, vb[u], x[u]);
    }
    sa = warp_sum<P>(sa);
    sb = warp_sum<P>(sb);
    if (lane == 0) {  // kept in the accumulator type: no FP64 instruction
      typename T::A* tp = static_cast<typename T::A*>(H.tpart) + (int64_t)tc.z * HINV_KCAP;
      tp[l] = sa;
      if (l2 < k) tp[l2] = sb;
    }
  }
  // the CTA's partials are published by one acquire-release count after the
  // barrier (release is cumulative over what the barrier ordered); the last
  // chunk's CTA acquires everyone's and sums them
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned n = (unsigned)(nd.tch_end - nd.tch_begin);
    unsigned prev;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(H.tcount + tc.x) : "memory");
    last = prev == n - 1 ? 1 : 0;
  }
  __syncthreads();
  if (last) {
    // warp per column, lanes over the chunks (fixed assignment and tree);
    // four columns of a warp at a time, so that their partials' loads are in
    // flight together (each column's sum keeps its order)
    const int nch = nd.tch_end - nd.tch_begin;
    const typename T::A* tp = static_cast<const typename T::A*>(H.tpart);
    for (int l0 = warp; l0 < k; l0 += 4 * T_WARPS) {
      typename T::A s[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) s[q] = T::zero();
      for (int cc = lane; cc < nch; cc += 32) {
        const typename T::A* row = tp + (int64_t)(nd.tch_begin + cc) * HINV_KCAP;
        typename T::A v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = l0 + q * T_WARPS < k ? ld_cg(row + l0 + q * T_WARPS) : T::zero();
#pragma unroll
        for (int q = 0; q < 4; ++q) s[q] = T::add(s[q], v[q]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int l = l0 + q * T_WARPS;
        const typename T::A r = warp_sum<P>(s[q]);
        if (lane == 0 && l < k) static_cast<typename T::A*>(H.tvec)[(int64_t)tc.x * HINV_KCAP + l] = r;
      }
    }
    if (threadIdx.x == 0) H.tcount[tc.x] = 0u;
  }
}

// y rows of one 64-row chunk: lane takes rows lane and lane + 32.  The
// chunk's column runs (its leaf's triangle against b, then P of every block
// whose target holds the rows, against t) are split into equal column ranges
// over the warps (the zeros of a triangle outside the rows' own half are
// skipped, not read).  Every load is 32 consecutive rows of one column,
// sixteen issued before any is used; the vector entries of eight columns are
// loaded and converted by eight lanes and broadcast.  The warps' sums meet in
// shared memory and are added in warp order.  Deterministic.
template <int P>
__device__ __forceinline__ void r_body(const HinvApply& H, int c, const double* __restrict__ b, double* y,
                                       const double* sub, double scale) {
  using T = Tr<P>;
  __shared__ typename T::A part[HINV_AWARPS][HINV_ACH];
  const HinvRChunk ch = H.rch[c];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int total = 0;
  for (int s = ch.seg_begin; s < ch.seg_end; ++s) total += H.segs[s].n;
  const int w0 = (int)((int64_t)total * warp / HINV_AWARPS);
  const int w1 = (int)((int64_t)total * (warp + 1) / HINV_AWARPS);
  const bool ra = lane < ch.nr, rb = lane + 32 < ch.nr;
  typename T::A fa = T::zero(), fb = T::zero();
  int base = 0;
  for (int s = ch.seg_begin; s < ch.seg_end && base < w1; ++s) {
    const HinvSeg g = H.segs[s];
    const int lo = max(w0 - base, 0), hi = min(w1 - base, g.n);
    base += g.n;
    if (lo >= hi) continue;
    const typename T::S* M = static_cast<const typename T::S*>(g.kind ? H.p_pool : H.leaf_pool) + g.off + lane;
    const typename T::A* tv = static_cast<const typename T::A*>(H.tvec) + g.voff;  // t: already converted
    const double* v = b + g.voff;
    for (int j0 = lo; j0 < hi; j0 += 8) {
      typename T::S va[8], vb[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + u;
        va[u] = (j < hi && ra && j < g.a_hi) ? T::ld(M + (int64_t)j * g.ld) : T::sz();
        vb[u] = (j < hi && rb && j >= g.b_lo) ? T::ld(M + (int64_t)j * g.ld + 32) : T::sz();
      }
      typename T::X xl = T::cvt(0.0);
      if (lane < 8 && j0 + lane < hi) xl = g.kind ? tv[j0 + lane] : T::cvt(__ldg(v + j0 + lane));
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const typename T::X x = shfl_i(xl, u);
        T::mac(fa, va[u], x);
        T::mac(fb, vb[u], x);
      }
    }
  }
  part[warp][lane] = fa;
  part[warp][lane + 32] = fb;
  __syncthreads();
  if ((int)threadIdx.x < ch.nr) {
    const int r = threadIdx.x;
    typename T::A s = part[0][r];
#pragma unroll
    for (int w = 1; w < HINV_AWARPS; ++w) s = T::add(s, part[w][r]);
    double o = T::fin(s);
    if (sub) o = scale * o - sub[ch.row0 + r];
    y[ch.row0 + r] = o;
  }
}

constexpr int R_THREADS = 32 * HINV_AWARPS;

template <int P>
__global__ void __launch_bounds__(32 * T_WARPS, 8) hinv_t_kernel(HinvApply H, const double* __restrict__ b) {
  t_body<P>(H, blockIdx.x, b);
}

template <int P>
__global__ void __launch_bounds__(R_THREADS, 7) hinv_r_kernel(HinvApply H, const double* __restrict__ b, double* y,
                                                              const double* sub, double scale) {
  r_body<P>(H, blockIdx.x, b, y, sub, scale);
}

__device__ __forceinline__ int job_of(const int* off, int count, int blk) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// one precision for every job (the common case: no switch, no spills)
template <int P>
__global__ void __launch_bounds__(32 * T_WARPS, 8) hinv_t_batch1_kernel(const HinvJob* jobs, const int* off, int count) {
  const int j = job_of(off, count, blockIdx.x);
  t_body<P>(jobs[j].A, blockIdx.x - off[j], jobs[j].b);
}
template <int P>
__global__ void __launch_bounds__(R_THREADS, 7) hinv_r_batch1_kernel(const HinvJob* jobs, const int* off, int count) {
  const int j = job_of(off, count, blockIdx.x);
  const HinvJob& J = jobs[j];
  r_body<P>(J.A, blockIdx.x - off[j], J.b, J.y, J.sub, J.scale);
}

__global__ void __launch_bounds__(32 * T_WARPS, 8) hinv_t_batch_kernel(const HinvJob* jobs, const int* off, int count) {
  const int j = job_of(off, count, blockIdx.x);
  const HinvJob& J = jobs[j];
  const int c = blockIdx.x - off[j];
  switch (J.A.prec) {
    case HINV_F64: t_body<HINV_F64>(J.A, c, J.b); break;
    case HINV_DF: t_body<HINV_DF>(J.A, c, J.b); break;
    case HINV_F32: t_body<HINV_F32>(J.A, c, J.b); break;
    default: t_body<HINV_BF16>(J.A, c, J.b); break;
  }
}

__global__ void __launch_bounds__(R_THREADS, 7) hinv_r_batch_kernel(const HinvJob* jobs, const int* off, int count) {
  const int j = job_of(off, count, blockIdx.x);
  const HinvJob& J = jobs[j];
  const int c = blockIdx.x - off[j];
  switch (J.A.prec) {
    case HINV_F64: r_body<HINV_F64>(J.A, c, J.b, J.y, J.sub, J.scale); break;
    case HINV_DF: r_body<HINV_DF>(J.A, c, J.b, J.y, J.sub, J.scale); break;
    case HINV_F32: r_body<HINV_F32>(J.A, c, J.b, J.y, J.sub, J.scale); break;
    default: r_body<HINV_BF16>(J.A, c, J.b, J.y, J.sub, J.scale); break;
  }
}

template <int P>
int launch_typed(const HinvApply& H, const double* b, double* y, cudaStream_t st) {
  count_launches(H.ntch > 0 ? 2 : 1);
  if (H.ntch > 0) hinv_t_kernel<P><<<H.ntch, 32 * T_WARPS, 0, st>>>(H, b);
  hinv_r_kernel<P><<<H.nrch, R_THREADS, 0, st>>>(H, b, y, nullptr, 1.0);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

}  // namespace

int launch_hinv_apply(const HinvApply& H, const double* b, double* y, cudaStream_t st) {
  if (H.nrch == 0) return HM_OK;
  switch (H.prec) {
    case HINV_F64: return launch_typed<HINV_F64>(H, b, y, st);
    case HINV_DF: return launch_typed<HINV_DF>(H, b, y, st);
    case HINV_F32: return launch_typed<HINV_F32>(H, b, y, st);
    default: return launch_typed<HINV_BF16>(H, b, y, st);
  }
}

template <int P>
void launch_batch1(const HinvBatch& B, cudaStream_t st) {
  if (B.total[0] > 0) hinv_t_batch1_kernel<P><<<B.total[0], 32 * T_WARPS, 0, st>>>(B.jobs, B.off[0], B.count);
  hinv_r_batch1_kernel<P><<<B.total[1], R_THREADS, 0, st>>>(B.jobs, B.off[1], B.count);
}

int launch_hinv_batch(const HinvBatch& B, cudaStream_t st) {
  if (B.count == 0) return HM_OK;
  count_launches(B.total[0] > 0 ? 2 : 1);
  switch (B.prec) {
    case HINV_F64: launch_batch1<HINV_F64>(B, st); break;
    case HINV_DF: launch_batch1<HINV_DF>(B, st); break;
    case HINV_F32: launch_batch1<HINV_F32>(B, st); break;
    case HINV_BF16: launch_batch1<HINV_BF16>(B, st); break;
    default:
      if (B.total[0] > 0) hinv_t_batch_kernel<<<B.total[0], 32 * T_WARPS, 0, st>>>(B.jobs, B.off[0], B.count);
      hinv_r_batch_kernel<<<B.total[1], R_THREADS, 0, st>>>(B.jobs, B.off[1], B.count);
  }
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

}  // namespace hm
