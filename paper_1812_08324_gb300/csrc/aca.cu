// Batched partially pivoted adaptive cross approximation (ACA) of the
// admissible blocks (the low-rank construction named in Sec. "H-matrix
// construction"; storage U V' of App. "Construction and Storage").
//
// One CTA per block.  Step k: the residual of pivot row i* is generated
// entry by entry (offset table), its largest entry picks the column j*
// (ties -> smallest Morton index), v_k = row / pivot, u_k = residual column j*.
// The Frobenius norm of the approximant is updated exactly,
//   |S_k|^2 = |S_{k-1}|^2 + 2 sum_{l<k} (u_l.u_k)(v_l.v_k) + |u_k|^2 |v_k|^2,
// and the loop stops when |u_k| |v_k| <= tol |S_k| or k reaches the cap.
// The next pivot row is the largest entry of |u_k| among unused rows.
// Pivots and norms are FP64.
#include "hm_device.cuh"
#include "hm_kernels.h"

namespace hm {

namespace {

constexpr int ACA_THREADS = 256;
constexpr int ZERO_ROW_TRIES = 8;

__device__ __forceinline__ bool is_used(const unsigned* used, int i) {
  return (used[i >> 5] >> (i & 31)) & 1u;
}

__global__ void __launch_bounds__(ACA_THREADS)
aca_kernel(EntryCtx E, const LRDesc* ld, double* Upool, double* Vpool, int* rank, int* capped,
           double tol) {
  extern __shared__ unsigned used[];
  __shared__ double urow[ACA_MAXK], vcol[ACA_MAXK], cu[ACA_MAXK], cv[ACA_MAXK];
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ double sc[32];
  __shared__ int s_next;

  const LRDesc L = ld[blockIdx.x];
  const int m = L.m, n = L.n, kcap = L.kcap;
  double* U = Upool + L.uoff;
  double* V = Vpool + L.voff;
  const int tid = threadIdx.x, bs = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = bs >> 5;
  const int words = (m + 31) >> 5;
  for (int w = tid; w < words; w += bs) used[w] = 0u;
  __syncthreads();

  int istar = 0, k = 0, zero_rows = 0;
  bool converged = false;
  double norm2 = 0.0;
  while (k < kcap) {
    for (int l = tid; l < k; l += bs) urow[l] = U[istar + (int64_t)l * m];
    __syncthreads();
    // residual of row i*, stored as candidate column k of V
    double bv = 0.0;
    int bi = -1;
    double* Vk = V + (int64_t)k * n;
    for (int j = tid; j < n; j += bs) {
      double val = far_entry(E, L.r0 + istar, L.c0 + j);
      for (int l = 0; l < k; ++l) val -= urow[l] * V[j + (int64_t)l * n];
      Vk[j] = val;
      argmax_merge(bv, bi, val, j);
    }
    block_argmax(bv, bi, sv, si);
    if (tid == 0) used[istar >> 5] |= 1u << (istar & 31);
    __syncthreads();
    if (bi < 0 || bv == 0.0) {
      // a zero residual row: sample another unused row, a bounded number of times
      if (++zero_rows > ZERO_ROW_TRIES) { converged = true; break; }
      if (tid == 0) {
        int start = (istar + 1 + m / (ZERO_ROW_TRIES + 1)) % m, found = -1;
        for (int t = 0; t < m && found < 0; ++t) {
          int i = (start + t) % m;
          if (!is_used(used, i)) found = i;
        }
        s_next = found;
      }
      __syncthreads();
      istar = s_next;
      __syncthreads();
      if (istar < 0) { converged = true; break; }
      continue;
    }
    const int jstar = bi;
    const double delta = bv;
    for (int j = tid; j < n; j += bs) Vk[j] = Vk[j] / delta;
    __syncthreads();
    for (int l = tid; l <= k; l += bs) vcol[l] = V[jstar + (int64_t)l * n];
    __syncthreads();
    // residual of column j*
    double* Uk = U + (int64_t)k * m;
    for (int i = tid; i < m; i += bs) {
      double val = far_entry(E, L.r0 + i, L.c0 + jstar);
      for (int l = 0; l < k; ++l) val -= U[i + (int64_t)l * m] * vcol[l];
      Uk[i] = val;
    }
    __syncthreads();
    // exact norm update: cross terms (u_l.u_k)(v_l.v_k), l < k, one warp per l
    for (int l = warp; l < k; l += nwarp) {
      double a = 0.0, b = 0.0;
      const double* Ul = U + (int64_t)l * m;
      const double* Vl = V + (int64_t)l * n;
      for (int i = lane; i < m; i += 32) a += Ul[i] * Uk[i];
      for (int j = lane; j < n; j += 32) b += Vl[j] * Vk[j];
      a = warp_sum(a);
      b = warp_sum(b);
      if (lane == 0) { cu[l] = a; cv[l] = b; }
    }
    double uu = 0.0, vv = 0.0;
    for (int i = tid; i < m; i += bs) uu += Uk[i] * Uk[i];
    for (int j = tid; j < n; j += bs) vv += Vk[j] * Vk[j];
    uu = block_sum(uu, sc);
    vv = block_sum(vv, sc);
    double cross = 0.0;
    for (int l = 0; l < k; ++l) cross += cu[l] * cv[l];
    norm2 += uu * vv + 2.0 * cross;
    ++k;
    if (sqrt(uu * vv) <= tol * sqrt(fmax(norm2, 0.0))) { converged = true; break; }
    // next pivot row: largest |u_k| among unused rows
    bv = 0.0;
    bi = -1;
    for (int i = tid; i < m; i += bs)
      if (!is_used(used, i)) argmax_merge(bv, bi, Uk[i], i);
    block_argmax(bv, bi, sv, si);
    if (bi < 0) { converged = true; break; }
    istar = bi;
  }
  // zero the unused columns so that fixed-capacity consumers may read them
  for (int l = k; l < kcap; ++l) {
    for (int i = tid; i < m; i += bs) U[i + (int64_t)l * m] = 0.0;
    for (int j = tid; j < n; j += bs) V[j + (int64_t)l * n] = 0.0;
  }
  if (tid == 0) {
    rank[blockIdx.x] = k;
    capped[blockIdx.x] = (!converged && k == kcap) ? 1 : 0;
  }
}

}  // namespace

int launch_aca(const EntryCtx& E, const LRDesc* d_ld, int nlr, int max_m, double* U, double* V,
               int* rank, int* capped, double tol, cudaStream_t st) {
  if (nlr == 0) return HM_OK;
  size_t smem = (size_t)((max_m + 31) / 32) * sizeof(unsigned);
  if (smem > 200 * 1024) return HM_ERR_ARG;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(aca_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  count_launches(1);
  aca_kernel<<<nlr, ACA_THREADS, smem, st>>>(E, d_ld, U, V, rank, capped, tol);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

}  // namespace hm
