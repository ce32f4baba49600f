// C ABI: H-LU factorisation, triangular solves and Crank-Nicolson steps.
#include <algorithm>
#include <cstring>

#include "api_common.h"

using namespace hm;

struct hm_factors {
  int dummy;
};

extern "C" {

int hm_factor(const hm_matrix*, double, void*, hm_factors** out) {
  if (out) *out = nullptr;
  set_error("hm_factor: not built yet");
  return HM_ERR_ARG;
}
int hm_solve(const hm_factors*, const double*, double*, void*) { set_error("not built yet"); return HM_ERR_ARG; }
int cn_step(const hm_matrix*, const hm_factors*, double, const double*, const double*, const double*,
            double*, void*) { set_error("not built yet"); return HM_ERR_ARG; }
int cn_solve(const hm_matrix*, const hm_factors*, double, int, int, double*, const double*, void*) {
  set_error("not built yet");
  return HM_ERR_ARG;
}
int hm_stats(const hm_matrix* H, const hm_factors*, hm_stats_t* out) {
  if (!H || !out) { set_error("null argument"); return HM_ERR_ARG; }
  std::memset(out, 0, sizeof(*out));
  const Plan& P = H->plan;
  out->n = P.N;
  out->clusters = (int)P.cl.size();
  out->leaves = (int)P.leaves.size();
  out->depth = P.depth;
  out->dense_blocks = (int)H->h_dd.size();
  out->lowrank_blocks = (int)H->h_ld.size();
  int64_t de = 0, le = 0;
  for (auto& D : H->h_dd) de += (int64_t)D.m * D.n;
  int mr = 0;
  for (size_t q = 0; q < H->h_ld.size(); ++q) {
    le += (int64_t)(H->h_ld[q].m + H->h_ld[q].n) * H->h_rank[q];
    mr = std::max(mr, H->h_rank[q]);
  }
  out->dense_entries = de;
  out->lowrank_entries = le;
  out->h_bytes = 8 * (de + le);
  out->max_rank_seen = mr;
  out->rank_capped_blocks = H->capped_blocks;
  return HM_OK;
}
void hm_factors_free(hm_factors* F) { delete F; }

}  // extern "C"
