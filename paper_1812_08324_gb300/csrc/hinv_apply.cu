// Per-step application of the hierarchical inverses of the triangular factors
// (the H-triangular solves of App. "LU Decomposition" as products):
//
//   y = X b,   y_i = sum_{j in leaf(i), j <= i (L) / j >= i (U)} X_leaf[i, j] b_j
//                    + sum_{tau: i in tgt(tau)} P_tau[i, :] (Q_tau^T b[src(tau)])
//
//   1. hinv_t_kernel  t_tau = Q_tau^T b[src(tau)]: one CTA per 256-row chunk of
//                     every source range (Q row-major); the last CTA of a
//                     block sums the chunks' partials in chunk order
//   2. hinv_r_kernel  one CTA per 32-row chunk of a leaf, lane per row: the
//                     leaf's triangle (stored column-major) plus P rows times
//                     t of every block whose target holds the leaf
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
#include "hm_kernels.h"

namespace hm {

namespace {

// ---- double-float arithmetic (no contraction: every step rounds as written)
__device__ __forceinline__ float2 df_split(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}
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
  static __device__ __forceinline__ X cvt(double v) { return df_split(v); }
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

constexpr int LEAF_SMEM = 1024;  // largest leaf the row kernel stages
constexpr int ANC_SMEM = HINV_MAX_ANC;  // blocks above a leaf whose coefficients are staged

// t_tau = Q_tau^T b over one 256-row chunk (Q row-major, stride KCAP).  Lanes
// take columns (W = 8, 16 or 32 of them, 32 / W rows at a time), warps take
// 32-row slices, two accumulators per lane.  The warps' partial sums meet in
// shared memory (fixed order); the last chunk of a block sums the chunks'
// partials in chunk order.  Deterministic.
template <int P>
constexpr int t_smem() { return (int)(sizeof(typename Tr<P>::X) * HINV_TCH + sizeof(typename Tr<P>::A) * 32 * HINV_KCAP); }
template <int P>
constexpr int r_smem() {
  return (int)(sizeof(typename Tr<P>::X) * (LEAF_SMEM + ANC_SMEM * HINV_KCAP) + sizeof(typename Tr<P>::A) * 8 * HINV_RCH);
}
constexpr int T_SMEM_MAX = 12288, R_SMEM_MAX = 17920;  // the largest of the precisions (FP64 and pairs)
static_assert(t_smem<HINV_F64>() <= T_SMEM_MAX && t_smem<HINV_DF>() <= T_SMEM_MAX, "t smem");
static_assert(r_smem<HINV_F64>() <= R_SMEM_MAX && r_smem<HINV_DF>() <= R_SMEM_MAX, "r smem");

template <int P>
__device__ __forceinline__ void t_body(const HinvApply& H, int c, const double* __restrict__ b, char* sm) {
  using T = Tr<P>;
  typename T::X* xs = reinterpret_cast<typename T::X*>(sm);
  auto red = reinterpret_cast<typename T::A(*)[HINV_KCAP]>(sm + sizeof(typename T::X) * HINV_TCH);
  __shared__ int last;
  const int2 tc = H.tch[c];
  const HinvNode nd = H.nodes[tc.x];
  const int k = H.rank[tc.x];
  const int j0 = tc.y, len = min(HINV_TCH, nd.src_n - j0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < len; j += blockDim.x) xs[j] = T::cvt(b[nd.src0 + j0 + j]);
  __syncthreads();
  const typename T::S* Q = static_cast<const typename T::S*>(H.q_pool) + nd.qoff + (int64_t)j0 * HINV_KCAP;
  const int rb = warp * 32, re = min(len, rb + 32);
  const int W = k <= 8 ? 8 : (k <= 16 ? 16 : 32), G = 32 / W;
  const int col = lane % W, sub = lane / W;
  typename T::A a0 = T::zero(), a1 = T::zero();
  if (col < k) {
    // all of the lane's rows of the slice (32 / G) are loaded before any is used
    for (int m0 = 0; m0 < 32 / G; m0 += 16) {
      typename T::S v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int r = rb + sub + (m0 + u) * G;
        v[u] = (m0 + u < 32 / G && r < re) ? T::ld(Q + (int64_t)r * HINV_KCAP + col) : T::sz();
      }
#pragma unroll
      for (int u = 0; u < 16; u += 2) {
        const int r = rb + sub + (m0 + u) * G;
        if (m0 + u < 32 / G && r < re) T::mac(a0, v[u], xs[r]);
        if (m0 + u + 1 < 32 / G && r + G < re) T::mac(a1, v[u + 1], xs[r + G]);
      }
    }
  }
  typename T::A a2 = T::zero();  // columns [32, KCAP): 8 lanes per row, 4 rows at a time
  const int col2 = 32 + (lane & 7), sub2 = lane >> 3;
  if (k > 32 && col2 < k) {
    typename T::S v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int r = rb + sub2 + 4 * u;
      v[u] = r < re ? T::ld(Q + (int64_t)r * HINV_KCAP + col2) : T::sz();
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (rb + sub2 + 4 * u < re) T::mac(a2, v[u], xs[rb + sub2 + 4 * u]);
  }
  if (col < k) red[warp * G + sub][col] = T::add(a0, a1);
  if (k > 32 && col2 < k) red[warp * 4 + sub2][col2] = a2;
  __syncthreads();
  if ((int)threadIdx.x < k) {
    const int l = threadIdx.x;
    const int ns = l < 32 ? 8 * G : 32;
    typename T::A s = red[0][l];
    for (int q = 1; q < ns; ++q) s = T::add(s, red[q][l]);
    H.tpart[(int64_t)c * HINV_KCAP + l] = T::fin(s);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned n = (unsigned)(nd.tch_end - nd.tch_begin);
    last = atomicAdd(H.tcount + tc.x, 1u) == n - 1 ? 1 : 0;
  }
  __syncthreads();
  if (last) {
    // warp per column, lanes over the chunks (fixed assignment and tree)
    __threadfence();
    const int nch = nd.tch_end - nd.tch_begin;
    for (int l = warp; l < k; l += 8) {
      double s = 0.0;
      for (int cc = lane; cc < nch; cc += 32) s += __ldcg(H.tpart + (int64_t)(nd.tch_begin + cc) * HINV_KCAP + l);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) H.tvec[(int64_t)tc.x * HINV_KCAP + l] = s;
    }
    if (threadIdx.x == 0) H.tcount[tc.x] = 0u;
  }
}

// y rows of one 32-row chunk of a leaf: lane = row, warps split the columns.
// The leaf inverse and P are stored column-major, so every load is 32
// consecutive rows of one column.  Dense triangle: the columns that can be
// nonzero for the chunk's rows (lower: [0, i0 + nr), upper: [i0, m); the
// zeros inside the chunk's diagonal block are stored); low-rank blocks:
// (block, half of its columns) items over the warps, their coefficients t
// staged in shared memory.  The warps' sums meet in shared memory.
template <int P>
__device__ __forceinline__ void r_body(const HinvApply& H, int c, const double* __restrict__ b,
                                       double* __restrict__ y, char* sm) {
  using T = Tr<P>;
  typename T::X* bs = reinterpret_cast<typename T::X*>(sm);
  auto ts = reinterpret_cast<typename T::X(*)[HINV_KCAP]>(sm + sizeof(typename T::X) * LEAF_SMEM);
  auto part = reinterpret_cast<typename T::A(*)[HINV_RCH]>(sm + sizeof(typename T::X) * (LEAF_SMEM + ANC_SMEM * HINV_KCAP));
  const int2 rc = H.rch[c];
  const HinvLeaf L = H.leaves[rc.x];
  const int i0 = rc.y, nr = min(HINV_RCH, L.m - i0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int na = L.anc_end - L.anc_begin;
  for (int j = threadIdx.x; j < L.m; j += blockDim.x) bs[j] = T::cvt(b[L.r0 + j]);
  for (int e = threadIdx.x; e < na * HINV_KCAP; e += blockDim.x) {
    const int a = e / HINV_KCAP, l = e % HINV_KCAP;
    const int q = H.anc[L.anc_begin + a];
    ts[a][l] = T::cvt(l < H.rank[q] ? H.tvec[(int64_t)q * HINV_KCAP + l] : 0.0);
  }
  __syncthreads();
  typename T::A f0 = T::zero(), f1 = T::zero();
  if (lane < nr) {
    const int c0 = H.lower ? 0 : i0, c1 = H.lower ? i0 + nr : L.m;
    const int span = (c1 - c0 + 7) >> 3;
    const int jb = c0 + warp * span, je = min(c1, jb + span);
    const typename T::S* X = static_cast<const typename T::S*>(H.leaf_pool) + L.off + i0 + lane;
    // blocks of 16 columns: the loads are issued before any is used
    for (int j0 = jb; j0 < je; j0 += 16) {
      typename T::S v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) v[u] = j0 + u < je ? T::ld(X + (int64_t)(j0 + u) * L.ld) : T::sz();
#pragma unroll
      for (int u = 0; u < 16; u += 2) {
        if (j0 + u < je) T::mac(f0, v[u], bs[j0 + u]);
        if (j0 + u + 1 < je) T::mac(f1, v[u + 1], bs[j0 + u + 1]);
      }
    }
    for (int it = warp; it < 2 * na; it += 8) {
      const int a = it >> 1;
      const int q = H.anc[L.anc_begin + a];
      const HinvNode nd = H.nodes[q];
      const int k = H.rank[q];
      const int kh = (k + 1) >> 1;
      const int lb = (it & 1) ? kh : 0, le = (it & 1) ? k : kh;
      const typename T::S* Pp = static_cast<const typename T::S*>(H.p_pool) + nd.poff + (L.r0 + i0 + lane - nd.tgt0);
      for (int l0 = lb; l0 < le; l0 += 16) {
        typename T::S v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = l0 + u < le ? T::ld(Pp + (int64_t)(l0 + u) * nd.pld) : T::sz();
#pragma unroll
        for (int u = 0; u < 16; u += 2) {
          if (l0 + u < le) T::mac(f0, v[u], ts[a][l0 + u]);
          if (l0 + u + 1 < le) T::mac(f1, v[u + 1], ts[a][l0 + u + 1]);
        }
      }
    }
  }
  part[warp][lane] = T::add(f0, f1);
  __syncthreads();
  if ((int)threadIdx.x < nr) {
    const int r = threadIdx.x;
    typename T::A s = part[0][r];
#pragma unroll
    for (int w = 1; w < 8; ++w) s = T::add(s, part[w][r]);
    y[L.r0 + i0 + r] = T::fin(s);
  }
}

template <int P>
__global__ void __launch_bounds__(256) hinv_t_kernel(HinvApply H, const double* __restrict__ b) {
  extern __shared__ __align__(16) char smem_t[];
  t_body<P>(H, blockIdx.x, b, smem_t);
}

template <int P>
__global__ void __launch_bounds__(256) hinv_r_kernel(HinvApply H, const double* __restrict__ b, double* y) {
  extern __shared__ __align__(16) char smem_r[];
  r_body<P>(H, blockIdx.x, b, y, smem_r);
}

__device__ __forceinline__ int job_of(const int* off, int count, int blk) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(256) hinv_t_batch_kernel(const HinvJob* jobs, const int* off, int count) {
  const int j = job_of(off, count, blockIdx.x);
  const HinvJob& J = jobs[j];
  const int c = blockIdx.x - off[j];
  extern __shared__ __align__(16) char smem_tb[];
  switch (J.A.prec) {
    case HINV_F64: t_body<HINV_F64>(J.A, c, J.b, smem_tb); break;
    case HINV_DF: t_body<HINV_DF>(J.A, c, J.b, smem_tb); break;
    case HINV_F32: t_body<HINV_F32>(J.A, c, J.b, smem_tb); break;
    default: t_body<HINV_BF16>(J.A, c, J.b, smem_tb); break;
  }
}

__global__ void __launch_bounds__(256) hinv_r_batch_kernel(const HinvJob* jobs, const int* off, int count) {
  const int j = job_of(off, count, blockIdx.x);
  const HinvJob& J = jobs[j];
  const int c = blockIdx.x - off[j];
  extern __shared__ __align__(16) char smem_rb[];
  switch (J.A.prec) {
    case HINV_F64: r_body<HINV_F64>(J.A, c, J.b, J.y, smem_rb); break;
    case HINV_DF: r_body<HINV_DF>(J.A, c, J.b, J.y, smem_rb); break;
    case HINV_F32: r_body<HINV_F32>(J.A, c, J.b, J.y, smem_rb); break;
    default: r_body<HINV_BF16>(J.A, c, J.b, J.y, smem_rb); break;
  }
}

template <int P>
int launch_typed(const HinvApply& H, const double* b, double* y, cudaStream_t st) {
  count_launches(H.ntch > 0 ? 2 : 1);
  if (H.ntch > 0) hinv_t_kernel<P><<<H.ntch, 256, t_smem<P>(), st>>>(H, b);
  hinv_r_kernel<P><<<H.nrch, 256, r_smem<P>(), st>>>(H, b, y);
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

int launch_hinv_batch(const HinvBatch& B, cudaStream_t st) {
  if (B.count == 0) return HM_OK;
  count_launches(B.total[0] > 0 ? 2 : 1);
  if (B.total[0] > 0) hinv_t_batch_kernel<<<B.total[0], 256, T_SMEM_MAX, st>>>(B.jobs, B.off[0], B.count);
  hinv_r_batch_kernel<<<B.total[1], 256, R_SMEM_MAX, st>>>(B.jobs, B.off[1], B.count);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

}  // namespace hm
