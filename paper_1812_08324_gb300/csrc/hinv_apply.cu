// Per-step application of the hierarchical inverses of the triangular factors
// (the H-triangular solves of App. "LU Decomposition" as products):
//
//   y = X b,   y_i = sum_{j in leaf(i), j <= i (L) / j >= i (U)} X_leaf[i, j] b_j
//                    + sum_{tau: i in tgt(tau)} P_tau[i, :] (Q_tau^T b[src(tau)])
//
//   1. hinv_t_kernel  t_tau = Q_tau^T b[src(tau)]: one CTA per 256-row chunk of
//                     every source range; the last CTA of a block sums the
//                     chunks' partials in chunk order (deterministic)
//   2. hinv_r_kernel  one CTA per 32-row chunk of a leaf: the leaf's triangle
//                     (warp per 4 rows, 2-element loads) plus P rows times t of
//                     every block whose target holds the leaf
// Storage FP64 (FP64 accumulation) or FP32 / BF16 (FP32 accumulation); the
// vectors are FP64 and in Morton order.  Every read of the two kernels is a
// stored entry of the inverses read once: the step is bandwidth-bound.
#include <cuda_bf16.h>

#include "hinv.h"
#include "hm_kernels.h"

namespace hm {

namespace {

template <class T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// element and pair loads converted to the accumulation type
template <class ST, class AT> struct Ld;
template <> struct Ld<double, double> {
  static __device__ __forceinline__ double one(const double* p) { return __ldg(p); }
  static __device__ __forceinline__ double2 two(const double* p) { return __ldg(reinterpret_cast<const double2*>(p)); }
};
template <> struct Ld<float, float> {
  static __device__ __forceinline__ float one(const float* p) { return __ldg(p); }
  static __device__ __forceinline__ float2 two(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }
};
template <> struct Ld<__nv_bfloat16, float> {
  static __device__ __forceinline__ float one(const __nv_bfloat16* p) { return __bfloat162float(p[0]); }
  static __device__ __forceinline__ float2 two(const __nv_bfloat16* p) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
  }
};

constexpr int LEAF_SMEM = 1024;  // largest leaf the row kernel stages

template <class ST, class AT>
__device__ __forceinline__ void t_body(const HinvApply& A, int c, const double* __restrict__ b) {
  __shared__ AT xs[HINV_TCH];
  __shared__ int last;
  const int2 tc = A.tch[c];
  const HinvNode nd = A.nodes[tc.x];
  const int k = A.rank[tc.x];
  const int j0 = tc.y, len = min(HINV_TCH, nd.src_n - j0);
  for (int j = threadIdx.x; j < len; j += blockDim.x) xs[j] = (AT)b[nd.src0 + j0 + j];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const ST* Q = static_cast<const ST*>(A.q_pool) + nd.qoff + j0;  // j0 is a multiple of 256: pairs aligned
  const int npair = len >> 1;
  for (int l = warp; l < k; l += nwarp) {
    const ST* Ql = Q + (int64_t)l * nd.qld;
    AT acc = 0;
    for (int p = lane; p < npair; p += 32) {
      const auto v = Ld<ST, AT>::two(Ql + 2 * p);
      acc = fma(v.x, xs[2 * p], acc);
      acc = fma(v.y, xs[2 * p + 1], acc);
    }
    if ((len & 1) && lane == 0) acc = fma(Ld<ST, AT>::one(Ql + len - 1), xs[len - 1], acc);
    acc = wsum(acc);
    if (lane == 0) A.tpart[(int64_t)c * HINV_KCAP + l] = (double)acc;
  }
  // the last chunk of the block sums the partials in chunk order
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned n = (unsigned)(nd.tch_end - nd.tch_begin);
    last = atomicAdd(A.tcount + tc.x, 1u) == n - 1 ? 1 : 0;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    for (int l = threadIdx.x; l < k; l += blockDim.x) {
      double s = 0.0;
      for (int cc = nd.tch_begin; cc < nd.tch_end; ++cc) s += __ldcg(A.tpart + (int64_t)cc * HINV_KCAP + l);
      A.tvec[(int64_t)tc.x * HINV_KCAP + l] = s;
    }
    if (threadIdx.x == 0) A.tcount[tc.x] = 0u;
  }
}

template <class ST, class AT>
__device__ __forceinline__ void r_body(const HinvApply& A, int c, const double* __restrict__ b,
                                       double* __restrict__ y) {
  __shared__ AT bs[LEAF_SMEM + 2];
  __shared__ AT part[9][HINV_RCH];
  const int2 rc = A.rch[c];
  const HinvLeaf L = A.leaves[rc.x];
  const int i0 = rc.y, nr = min(HINV_RCH, L.m - i0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < L.m + 2; j += blockDim.x) bs[j] = j < L.m ? (AT)b[L.r0 + j] : (AT)0;
  __syncthreads();
  // ---- the leaf's triangle: warp w has rows i0 + 4w .. i0 + 4w + 3, lanes
  // over column pairs (entries outside the triangle are stored as zeros, and
  // the row stride leaves room for the pair that straddles the row end)
  const ST* X = static_cast<const ST*>(A.leaf_pool) + L.off;
  const int mp = (L.m + 1) >> 1;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + 4 * warp + r;
    AT acc = 0;
    if (i < i0 + nr) {
      const ST* row = X + (int64_t)i * L.ld;
      const int p0 = A.lower ? 0 : (i >> 1), p1 = A.lower ? ((i >> 1) + 1) : mp;
      for (int p = p0 + lane; p < p1; p += 32) {
        const auto v = Ld<ST, AT>::two(row + 2 * p);
        acc = fma(v.x, bs[2 * p], acc);
        acc = fma(v.y, bs[2 * p + 1], acc);
      }
    }
    acc = wsum(acc);
    if (lane == 0) part[8][4 * warp + r] = acc;
  }
  // ---- low-rank blocks: warp per block, lane per row
  AT facc = 0;
  for (int a = L.anc_begin + warp; a < L.anc_end; a += 8) {
    const int q = A.anc[a];
    const HinvNode nd = A.nodes[q];
    const int k = A.rank[q];
    if (lane < nr) {
      const ST* P = static_cast<const ST*>(A.p_pool) + nd.poff + (L.r0 + i0 + lane - nd.tgt0);
      const double* t = A.tvec + (int64_t)q * HINV_KCAP;
      for (int l = 0; l < k; ++l) facc = fma(Ld<ST, AT>::one(P + (int64_t)l * nd.pld), (AT)t[l], facc);
    }
  }
  part[warp][lane] = facc;
  __syncthreads();
  if (threadIdx.x < nr) {
    const int r = threadIdx.x;
    AT s = part[8][r];
#pragma unroll
    for (int w = 0; w < 8; ++w) s += part[w][r];
    y[L.r0 + i0 + r] = (double)s;
  }
}

template <class ST, class AT>
__global__ void __launch_bounds__(256) hinv_t_kernel(HinvApply A, const double* __restrict__ b) {
  t_body<ST, AT>(A, blockIdx.x, b);
}

template <class ST, class AT>
__global__ void __launch_bounds__(256) hinv_r_kernel(HinvApply A, const double* __restrict__ b, double* y) {
  r_body<ST, AT>(A, blockIdx.x, b, y);
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
  switch (J.A.prec) {
    case HINV_F64: t_body<double, double>(J.A, c, J.b); break;
    case HINV_F32: t_body<float, float>(J.A, c, J.b); break;
    default: t_body<__nv_bfloat16, float>(J.A, c, J.b); break;
  }
}

__global__ void __launch_bounds__(256) hinv_r_batch_kernel(const HinvJob* jobs, const int* off, int count) {
  const int j = job_of(off, count, blockIdx.x);
  const HinvJob& J = jobs[j];
  const int c = blockIdx.x - off[j];
  switch (J.A.prec) {
    case HINV_F64: r_body<double, double>(J.A, c, J.b, J.y); break;
    case HINV_F32: r_body<float, float>(J.A, c, J.b, J.y); break;
    default: r_body<__nv_bfloat16, float>(J.A, c, J.b, J.y); break;
  }
}

template <class ST, class AT>
int launch_typed(const HinvApply& A, const double* b, double* y, cudaStream_t st) {
  count_launches(A.ntch > 0 ? 2 : 1);
  if (A.ntch > 0) hinv_t_kernel<ST, AT><<<A.ntch, 256, 0, st>>>(A, b);
  hinv_r_kernel<ST, AT><<<A.nrch, 256, 0, st>>>(A, b, y);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

}  // namespace

int launch_hinv_apply(const HinvApply& A, const double* b, double* y, cudaStream_t st) {
  if (A.nrch == 0) return HM_OK;
  switch (A.prec) {
    case HINV_F64: return launch_typed<double, double>(A, b, y, st);
    case HINV_F32: return launch_typed<float, float>(A, b, y, st);
    default: return launch_typed<__nv_bfloat16, float>(A, b, y, st);
  }
}

int launch_hinv_batch(const HinvBatch& B, cudaStream_t st) {
  if (B.count == 0) return HM_OK;
  count_launches(B.total[0] > 0 ? 2 : 1);
  if (B.total[0] > 0) hinv_t_batch_kernel<<<B.total[0], 256, 0, st>>>(B.jobs, B.off[0], B.count);
  hinv_r_batch_kernel<<<B.total[1], 256, 0, st>>>(B.jobs, B.off[1], B.count);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

}  // namespace hm
