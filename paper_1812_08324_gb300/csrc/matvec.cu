// H-matvec (App. "Matrix Vector Multiplication"): dense leaves by GEMV and
// low-rank blocks as U (V' x), flattened over the leaf blocks of the tree.
//
//   1. vt_kernel      partial products V[chunk]' x[chunk] of every low-rank
//                     block, one CTA per 256-row chunk of its column cluster
//   2. vt_reduce      t_q = sum of the partials of block q
//   3. rows_kernel    one CTA per 32-row chunk: the dense leaves of its rows
//                     (warp per 4 rows, 16-byte loads) plus U[rows] t_q of
//                     every low-rank block covering the rows, then the
//                     epilogue y = alpha x + beta (H x) + gamma (w1 + w2) + w3.
// All vectors are in Morton order.  FP64 storage and FP64 accumulation, or the
// split form (below): the stiff stencil part in FP64, the jump part from
// float-pair storage in double-float arithmetic.
#include <atomic>

#include "hm_device.cuh"
#include "hm_kernels.h"

namespace hm {

namespace {

// ---- bodies shared by the single and the batched launches

__device__ __forceinline__ void vt_body(const MatvecPlan& P, int task, const double* __restrict__ x) {
  __shared__ double xs[VT_CHUNK];
  const VTask T = P.vt[task];
  const LRDesc L = P.ld[T.lr];
  const int k = P.rank[T.lr];
  const double* xc = x + L.c0 + T.c_lo;
  for (int j = threadIdx.x; j < T.len; j += blockDim.x) xs[j] = xc[j];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const double* V = P.V + L.voff + T.c_lo;
  for (int l = warp; l < k; l += nwarp) {
    const double* Vl = V + (int64_t)l * L.n;
    double acc = 0.0;
    for (int j = lane; j < T.len; j += 32) acc += Vl[j] * xs[j];
    acc = warp_sum(acc);
    if (lane == 0) P.partial[(int64_t)T.out * ACA_MAXK + l] = acc;
  }
}

__device__ __forceinline__ void vt_reduce_body(const MatvecPlan& P, int q) {
  const int b = P.vt_range[2 * q], e = P.vt_range[2 * q + 1];
  const int k = P.rank[q];
  for (int l = threadIdx.x; l < k; l += blockDim.x) {
    double acc = 0.0;
    for (int o = b; o < e; ++o) acc += P.partial[(int64_t)o * ACA_MAXK + l];
    P.tvec[(int64_t)q * ACA_MAXK + l] = acc;
    if (P.tdf) {
      bool bad = false;
      P.tdf[(int64_t)q * ACA_MAXK + l] = df_split(acc, bad);
    }
  }
}

constexpr int ROWS_PER_WARP = MV_CHUNK / 8;  // 8 warps x 4 rows

__device__ __forceinline__ void rows_body(const MatvecPlan& P, int chunk, double alpha, double beta,
                                          const double* __restrict__ x, double gamma, const double* w1,
                                          const double* w2, const double* w3, double* y) {
  __shared__ double acc_d[MV_CHUNK];
  __shared__ double acc_f[8][MV_CHUNK];
  const RowChunk C = P.chunks[chunk];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < MV_CHUNK) acc_d[threadIdx.x] = 0.0;
  acc_f[warp][lane] = 0.0;
  __syncthreads();

  // ---- dense leaves: warp handles ROWS_PER_WARP consecutive rows
  double rsum[ROWS_PER_WARP];
#pragma unroll
  for (int r = 0; r < ROWS_PER_WARP; ++r) rsum[r] = 0.0;
  const int rw0 = warp * ROWS_PER_WARP;
  for (int it = C.dense_begin; it < C.dense_end; ++it) {
    const DenseDesc D = P.dd[P.dense_items[it]];
    const int i0 = C.r0 - D.r0 + rw0;
    const double* xc = x + D.c0;
    const double* base = P.D + D.off + (int64_t)i0 * D.ld;
    // 16-byte loads over column pairs; D.ld is a multiple of 4, D.off even
    const int npair = D.n >> 1;
    for (int p = lane; p < npair; p += 32) {
      double x0 = xc[2 * p], x1 = xc[2 * p + 1];
#pragma unroll
      for (int r = 0; r < ROWS_PER_WARP; ++r) {
        if (rw0 + r < C.nrow) {
          double2 v = *reinterpret_cast<const double2*>(base + (int64_t)r * D.ld + 2 * p);
          // two chained FMAs: one FP64 instruction per matrix entry (the
          // kernel issues FP64 close to the HBM rate)
          rsum[r] = fma(v.x, x0, rsum[r]);
          rsum[r] = fma(v.y, x1, rsum[r]);
        }
      }
    }
    if ((D.n & 1) && lane == 0) {
      double xl = xc[D.n - 1];
#pragma unroll
      for (int r = 0; r < ROWS_PER_WARP; ++r)
        if (rw0 + r < C.nrow) rsum[r] += base[(int64_t)r * D.ld + D.n - 1] * xl;
    }
  }
#pragma unroll
  for (int r = 0; r < ROWS_PER_WARP; ++r) {
    double s = warp_sum(rsum[r]);
    if (lane == 0) acc_d[rw0 + r] = s;
  }

  // ---- low-rank blocks: warp per block, lane per row
  double facc = 0.0;
  for (int it = C.lr_begin + warp; it < C.lr_end; it += 8) {
    const int q = P.lr_items[it];
    const LRDesc L = P.ld[q];
    const int k = P.rank[q];
    const int i = C.r0 - L.r0 + lane;
    if (lane < C.nrow) {
      const double* U = P.U + L.uoff + i;
      const double* t = P.tvec + (int64_t)q * ACA_MAXK;
      for (int l = 0; l < k; ++l) facc += U[(int64_t)l * L.m] * t[l];
    }
  }
  acc_f[warp][lane] = facc;
  __syncthreads();

  if (threadIdx.x < C.nrow) {
    const int r = threadIdx.x;
    double hx = acc_d[r];
    for (int w = 0; w < 8; ++w) hx += acc_f[w][r];
    const int row = C.r0 + r;
    double out = alpha * x[row] + beta * hx;
    if (w1) out += gamma * w1[row];
    if (w2) out += gamma * w2[row];
    if (w3) out += w3[row];
    y[row] = out;
  }
}

// ---- split form G = S + J (constant-order problems on a box): the stiff
// part S -- the diagonal and the axis-neighbour stencil, entries up to
// 4 a / h^2 -- in FP64 from the constants, the jump part J (every other
// entry; the diagonal and the stencil removed from the dense leaves) from
// float-pair storage in double-float arithmetic on the FP32 pipes (FP64 on
// this GPU issues about two multiply-adds per clock per SM, below the HBM
// rate of these products).  The double-float rounding is about 2^-47 of
// sum |J_ij x_j|, which stays far below the FP64 rounding of the stiff part's
// terms.  Products by Dekker's method, sums by Knuth's two-sum.
__device__ __forceinline__ void mv_mac(float2& s, float2 a, float2 b) {
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
__device__ __forceinline__ float2 mv_wsum(float2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float2 w = make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
    v = dd_add(v, w);
  }
  return v;
}

__device__ __forceinline__ void vt_df_body(const MatvecPlan& P, int task, const double* __restrict__ x) {
  __shared__ float2 xs[VT_CHUNK];
  const VTask T = P.vt[task];
  const LRDesc L = P.ld[T.lr];
  const int k = P.rank[T.lr];
  const double* xc = x + L.c0 + T.c_lo;
  bool bad = false;
  for (int j = threadIdx.x; j < T.len; j += blockDim.x) xs[j] = df_split(xc[j], bad);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const float2* V = P.Vdf + L.voff + T.c_lo;
  for (int l = warp; l < k; l += nwarp) {
    const float2* Vl = V + (int64_t)l * L.n;
    float2 acc = make_float2(0.f, 0.f);
    for (int j = lane; j < T.len; j += 32) mv_mac(acc, Vl[j], xs[j]);
    acc = mv_wsum(acc);
    if (lane == 0) P.partial[(int64_t)T.out * ACA_MAXK + l] = (double)acc.x + (double)acc.y;
  }
}

__device__ __forceinline__ void rows_df_body(const MatvecPlan& P, int chunk, double alpha, double beta,
                                             const double* __restrict__ x, double gamma, const double* w1,
                                             const double* w2, const double* w3, double* y) {
  __shared__ float2 acc_d[MV_CHUNK];
  __shared__ float2 acc_f[8][MV_CHUNK];
  const RowChunk C = P.chunks[chunk];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float2 z = make_float2(0.f, 0.f);
  bool bad = false;
  float2 rsum[ROWS_PER_WARP];
#pragma unroll
  for (int r = 0; r < ROWS_PER_WARP; ++r) rsum[r] = z;
  const int rw0 = warp * ROWS_PER_WARP;
  const int nrw = max(0, min(ROWS_PER_WARP, C.nrow - rw0));
  // dense leaves: warp has ROWS_PER_WARP rows, lanes over column pairs, two
  // pairs per lane in flight (16-byte loads of two float pairs; D.ld is a
  // multiple of 4 and D.off even, the padding holds zeros); x is read and
  // split in registers (no staging barrier between the blocks)
  for (int it = C.dense_begin; it < C.dense_end; ++it) {
    const DenseDesc D = P.dd[P.dense_items[it]];
    const int i0 = C.r0 - D.r0 + rw0;
    const float2* base = P.Ddf + D.off + (int64_t)i0 * D.ld;
    const double* xc = x + D.c0;
    const int npair = (D.n + 1) >> 1;
    for (int p0 = lane; p0 < npair; p0 += 64) {
      const int p1 = p0 + 32;
      float4 v[2][ROWS_PER_WARP];
#pragma unroll
      for (int r = 0; r < ROWS_PER_WARP; ++r) {
        v[0][r] = r < nrw ? *reinterpret_cast<const float4*>(base + (int64_t)r * D.ld + 2 * p0) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[1][r] = (r < nrw && p1 < npair) ? *reinterpret_cast<const float4*>(base + (int64_t)r * D.ld + 2 * p1)
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      const float2 xa = df_split(__ldg(xc + 2 * p0), bad);
      const float2 xb = 2 * p0 + 1 < D.n ? df_split(__ldg(xc + 2 * p0 + 1), bad) : z;
      const float2 xc0 = p1 < npair ? df_split(__ldg(xc + 2 * p1), bad) : z;
      const float2 xc1 = (p1 < npair && 2 * p1 + 1 < D.n) ? df_split(__ldg(xc + 2 * p1 + 1), bad) : z;
#pragma unroll
      for (int r = 0; r < ROWS_PER_WARP; ++r) {
        mv_mac(rsum[r], make_float2(v[0][r].x, v[0][r].y), xa);
        mv_mac(rsum[r], make_float2(v[0][r].z, v[0][r].w), xb);
        mv_mac(rsum[r], make_float2(v[1][r].x, v[1][r].y), xc0);
        mv_mac(rsum[r], make_float2(v[1][r].z, v[1][r].w), xc1);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < ROWS_PER_WARP; ++r) {
    const float2 sr = mv_wsum(rsum[r]);
    if (lane == 0) acc_d[rw0 + r] = sr;
  }
  // low-rank blocks: warp per block, lane per row
  float2 facc = z;
  for (int it = C.lr_begin + warp; it < C.lr_end; it += 8) {
    const int q = P.lr_items[it];
    const LRDesc L = P.ld[q];
    const int k = P.rank[q];
    const int i = C.r0 - L.r0 + lane;
    if (lane < C.nrow) {
      const float2* U = P.Udf + L.uoff + i;
      const float2* t = P.tdf + (int64_t)q * ACA_MAXK;
      for (int l = 0; l < k; ++l) mv_mac(facc, U[(int64_t)l * L.m], t[l]);
    }
  }
  acc_f[warp][lane] = facc;
  __syncthreads();
  if (threadIdx.x < C.nrow) {
    const int r = threadIdx.x;
    float2 jx = acc_d[r];
    for (int w = 0; w < 8; ++w) jx = dd_add(jx, acc_f[w][r]);
    const int row = C.r0 + r;
    // S x in FP64: the diagonal and the axis neighbours
    const GenConst* g = P.gc;
    const int4 nb = P.nb[row];
    double sx = g->diag * x[row];
    if (nb.x >= 0) sx = fma(g->stencil_m[0], x[nb.x], sx);
    if (nb.y >= 0) sx = fma(g->stencil_p[0], x[nb.y], sx);
    if (nb.z >= 0) sx = fma(g->stencil_m[1], x[nb.z], sx);
    if (nb.w >= 0) sx = fma(g->stencil_p[1], x[nb.w], sx);
    const double hx = sx + ((double)jx.x + (double)jx.y);
    double out = alpha * x[row] + beta * hx;
    if (w1) out += gamma * w1[row];
    if (w2) out += gamma * w2[row];
    if (w3) out += w3[row];
    y[row] = out;
  }
}

__global__ void __launch_bounds__(256) vt_kernel(MatvecPlan P, const double* __restrict__ x) {
  if (P.Ddf) vt_df_body(P, blockIdx.x, x);
  else vt_body(P, blockIdx.x, x);
}

__global__ void vt_reduce_kernel(MatvecPlan P) {
  if ((int)blockIdx.x < P.nlr) vt_reduce_body(P, blockIdx.x);
}

__global__ void __launch_bounds__(256, 4)
rows_kernel(MatvecPlan P, double alpha, double beta, const double* __restrict__ x, double gamma, const double* w1,
            const double* w2, const double* w3, double* y) {
  if (P.Ddf) rows_df_body(P, blockIdx.x, alpha, beta, x, gamma, w1, w2, w3, y);
  else rows_body(P, blockIdx.x, alpha, beta, x, gamma, w1, w2, w3, y);
}

// ---- batched: many independent H-matvecs in three launches.  off[j] is the
// first block of job j in the launch (kind: 0 = V'x tasks, 1 = reductions,
// 2 = row chunks), off[count] the total.
__device__ __forceinline__ int batch_job(const int* off, int count, int b) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(256) vt_batch_kernel(const MvJob* jobs, const int* off, int count) {
  const int j = batch_job(off, count, blockIdx.x);
  if (jobs[j].P.Ddf) vt_df_body(jobs[j].P, blockIdx.x - off[j], jobs[j].x);
  else vt_body(jobs[j].P, blockIdx.x - off[j], jobs[j].x);
}

__global__ void vt_reduce_batch_kernel(const MvJob* jobs, const int* off, int count) {
  const int j = batch_job(off, count, blockIdx.x);
  vt_reduce_body(jobs[j].P, blockIdx.x - off[j]);
}

__global__ void __launch_bounds__(256, 4) rows_batch_kernel(const MvJob* jobs, const int* off, int count) {
  const int j = batch_job(off, count, blockIdx.x);
  const MvJob& J = jobs[j];
  if (J.P.Ddf) rows_df_body(J.P, blockIdx.x - off[j], J.alpha, J.beta, J.x, J.gamma, J.w1, J.w2, J.w3, J.y);
  else rows_body(J.P, blockIdx.x - off[j], J.alpha, J.beta, J.x, J.gamma, J.w1, J.w2, J.w3, J.y);
}

__global__ void gather_kernel(const int* perm, int N, const double* src, double* dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    dst[i] = src[perm[i]];
}

__global__ void scatter_kernel(const int* perm, int N, const double* src, double* dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    dst[perm[i]] = src[i];
}

}  // namespace

// ---- scratch for hm_matvec_noalloc ------------------------------------------
// A fixed array of 2^21 doubles (16 MiB) in device global memory, loaded with
// the library on every GPU that uses it and held until the process exits.  It
// takes the V'x partial products and the per-block coefficient vectors of one
// H-matvec (and, in 2D, the Morton-order copies of the vectors).
constexpr size_t NOALLOC_DOUBLES = size_t(1) << 21;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

size_t noalloc_capacity() { return NOALLOC_DOUBLES; }

// Device address of the array for the current device.  In host code the
// symbol name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
// The cache slots are atomics: threads that make their first call on a device
// at the same time each look the address up and store the same value.  The
// cache assumes the device is not reset while the library is loaded.
int noalloc_scratch(double** out) {
  static std::atomic<double*> addr[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return HM_ERR_CUDA;
  double* a = addr[dev].load(std::memory_order_acquire);
  if (!a) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return HM_ERR_CUDA;
    a = static_cast<double*>(p);
    addr[dev].store(a, std::memory_order_release);
  }
  *out = a;
  return HM_OK;
}

int launch_matvec(const MatvecPlan& P, double alpha, double beta, const double* x, double gamma,
                  const double* w1, const double* w2, const double* w3, double* y,
                  cudaStream_t st) {
  count_launches(P.nvt > 0 ? 3 : 1);
  if (P.nvt > 0) {
    vt_kernel<<<P.nvt, 256, 0, st>>>(P, x);
    vt_reduce_kernel<<<P.nlr, 64, 0, st>>>(P);
  }
  rows_kernel<<<P.nchunk, 256, 0, st>>>(P, alpha, beta, x, gamma, w1, w2, w3, y);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

int launch_matvec_batch(const MvBatch& B, cudaStream_t st) {
  if (B.count == 0) return HM_OK;
  count_launches(B.total[0] > 0 ? 3 : 1);
  if (B.total[0] > 0) {
    vt_batch_kernel<<<B.total[0], 256, 0, st>>>(B.jobs, B.off[0], B.count);
    vt_reduce_batch_kernel<<<B.total[1], 64, 0, st>>>(B.jobs, B.off[1], B.count);
  }
  rows_batch_kernel<<<B.total[2], 256, 0, st>>>(B.jobs, B.off[2], B.count);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

int launch_gather(const int* perm, int N, const double* src, double* dst, cudaStream_t st) {
  count_launches(1);
  gather_kernel<<<std::min((N + 255) / 256, 152 * 8), 256, 0, st>>>(perm, N, src, dst);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

int launch_scatter(const int* perm, int N, const double* src, double* dst, cudaStream_t st) {
  count_launches(1);
  scatter_kernel<<<std::min((N + 255) / 256, 152 * 8), 256, 0, st>>>(perm, N, src, dst);
  return cudaGetLastError() == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

}  // namespace hm
