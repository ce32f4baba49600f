// Internal state behind the opaque handles of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdio>
#include <string>
#include <vector>

#include "hm_internal.h"
#include "hm_kernels.h"

namespace hm {

void set_error(const std::string& msg);
void count_launches(int n);

// Record a failed CUDA call and turn it into a status code.
#define HM_CK(call)                                                                    \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      ::hm::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));             \
      return e_ == cudaErrorMemoryAllocation ? HM_ERR_OOM : HM_ERR_CUDA;               \
    }                                                                                  \
  } while (0)

#define HM_TRY(expr)               \
  do {                             \
    int s_ = (expr);               \
    if (s_ != HM_OK) return s_;    \
  } while (0)

// Device allocations owned by one handle, freed together.
struct DevArena {
  std::vector<void*> ptrs;
  int64_t bytes_held = 0;
  int alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
      set_error(std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
      *p = nullptr;
      return HM_ERR_OOM;
    }
    ptrs.push_back(*p);
    sizes.push_back(bytes);
    bytes_held += (int64_t)bytes;
    return HM_OK;
  }
  template <typename T>
  int upload(T** p, const std::vector<T>& h) {
    HM_TRY(alloc((void**)p, h.size() * sizeof(T)));
    if (!h.empty()) HM_CK(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return HM_OK;
  }
  // free one allocation made by this arena (its bytes leave bytes_held)
  void free_one(void* p, size_t bytes = 0) {
    for (size_t i = 0; i < ptrs.size(); ++i)
      if (ptrs[i] == p) {
        size_t b = bytes;
        if (!b) b = sizes.size() > i ? sizes[i] : 0;
        cudaFree(p);
        bytes_held -= (int64_t)b;
        ptrs.erase(ptrs.begin() + i);
        if (sizes.size() > i) sizes.erase(sizes.begin() + i);
        return;
      }
  }
  std::vector<size_t> sizes;  // bytes of each allocation (parallel to ptrs)
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
    sizes.clear();
  }
};

}  // namespace hm

struct hm_matrix {
  hm::Plan plan;
  hm_problem prob;
  hm_opts opts;
  int device = 0;
  hm::DevArena arena;
  hm::NuParams nuq;
  // device tables
  int* d_perm = nullptr;
  int* d_iperm = nullptr;
  int2* d_coord = nullptr;
  double* d_tab = nullptr;
  double* d_cscratch = nullptr;
  hm::GenConst* d_gc = nullptr;
  hm::EntryCtx ectx;
  // storage
  std::vector<hm::LRDesc> h_ld;
  std::vector<hm::DenseDesc> h_dd;
  hm::LRDesc* d_ld = nullptr;
  hm::DenseDesc* d_dd = nullptr;
  int* d_rank = nullptr;
  int* d_capped = nullptr;
  double* d_U = nullptr;
  double* d_V = nullptr;
  double* d_D = nullptr;
  int64_t u_pool = 0, v_pool = 0, d_pool = 0;
  int max_m = 0, kmax = 0;
  // matvec plan
  hm::MatvecPlan mv;
  std::vector<hm::RowChunk> h_chunks;
  std::vector<int> h_dense_items, h_lr_items;
  // work vectors (Morton order)
  double* d_work = nullptr;  // 6 x N
  int* d_err = nullptr;
  // host copies of results
  std::vector<int> h_rank;
  int capped_blocks = 0;
  int last_refine_iters = 0;
  double last_refine_resid = 0.0;
};

namespace hm {
// Host layout of the dense leaves and low-rank blocks of the plan.
void make_descs(const Plan& P, const hm_opts& o, std::vector<DenseDesc>& dd, std::vector<LRDesc>& ld,
                int64_t& dpool, int64_t& upool, int64_t& vpool);
// y = alpha x + beta G x + gamma (w1 + w2) + w3 on Morton-order device vectors.
int hm_matvec_morton(const hm_matrix* H, double alpha, double beta, const double* xm, double gamma,
                     const double* w1m, const double* w2m, const double* w3m, double* ym,
                     cudaStream_t st);
}  // namespace hm
