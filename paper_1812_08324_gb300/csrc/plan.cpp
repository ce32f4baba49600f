// Host-side planning: grid, Morton order, cluster tree and block tree
// (App. "H Matrix", Sec. "Construction and Storage"; admissibility Eq. adm).
// Integer-only: the admissibility test runs on cell-unit bounding boxes, so
// the classification is exact and identical on every machine.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include <vector_types.h>
#include <vector_functions.h>

#include "hm_internal.h"

namespace hm {

namespace {

uint64_t spread_bits(uint32_t v) {
  uint64_t x = v;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

struct Builder {
  Plan& P;
  std::vector<uint64_t> code;  // Morton code per Morton position (2D)

  explicit Builder(Plan& p) : P(p) {}

  void bbox(Cluster& c) {
    c.lo[0] = c.lo[1] = INT32_MAX;
    c.hi[0] = c.hi[1] = INT32_MIN;
    for (int q = c.begin; q < c.end; ++q) {
      for (int a = 0; a < P.dim; ++a) {
        int v = P.coord[2 * q + a];
        c.lo[a] = std::min(c.lo[a], v);
        c.hi[a] = std::max(c.hi[a], v + 1);  // cell [v, v+1)
      }
    }
    if (P.dim == 1) { c.lo[1] = 0; c.hi[1] = 0; }  // no extent along the absent axis
  }

  // Split a cluster: 1D halves the index range; 2D splits by the next pair of
  // Morton-code bits (quadtree), keeping non-empty quadrants.
  void split(int id, int bit) {
    Cluster c = P.cl[id];
    int cnt = c.end - c.begin;
    if (cnt <= P.leaf) return;
    std::vector<std::pair<int, int>> parts;
    if (P.dim == 1) {
      int mid = c.begin + cnt / 2;
      parts.push_back({c.begin, mid});
      parts.push_back({mid, c.end});
    } else {
      // find the next bit level where the range actually separates
      while (bit >= 0) {
        int b = c.begin;
        std::vector<std::pair<int, int>> pr;
        for (int quad = 0; quad < 4; ++quad) {
          int e = b;
          while (e < c.end && (int)((code[e] >> (2 * bit)) & 3u) == quad) ++e;
          if (e > b) pr.push_back({b, e});
          b = e;
        }
        if (pr.size() > 1) { parts = pr; break; }
        --bit;
      }
      if (parts.empty()) return;
    }
    int first = (int)P.cl.size();
    P.cl[id].nchild = (int)parts.size();
    for (size_t k = 0; k < parts.size(); ++k) {
      Cluster ch{};
      ch.begin = parts[k].first;
      ch.end = parts[k].second;
      ch.level = c.level + 1;
      ch.parent = id;
      ch.nchild = 0;
      bbox(ch);
      P.cl[id].child[k] = first + (int)k;
      P.cl.push_back(ch);
    }
    P.depth = std::max(P.depth, c.level + 1);
    for (size_t k = 0; k < parts.size(); ++k) split(first + (int)k, bit - 1);
  }

  bool admissible(int t, int s) const {
    const Cluster& A = P.cl[t];
    const Cluster& B = P.cl[s];
    int64_t da = 0, db = 0, dist = 0;
    for (int a = 0; a < 2; ++a) {
      int64_t wa = A.hi[a] - A.lo[a], wb = B.hi[a] - B.lo[a];
      da += wa * wa;
      db += wb * wb;
      int64_t g = std::max<int64_t>({0, (int64_t)B.lo[a] - A.hi[a], (int64_t)A.lo[a] - B.hi[a]});
      dist += g * g;
    }
    int64_t dmin = std::min(da, db);
    if (P.eta == 1.0) return dmin <= dist;                        // exact in integers
    return std::sqrt((double)dmin) <= P.eta * std::sqrt((double)dist);
  }

  void block(int bid) {
    Block b = P.bl[bid];
    const Cluster& T = P.cl[b.t];
    const Cluster& S = P.cl[b.s];
    if (b.t != b.s && admissible(b.t, b.s)) {
      P.bl[bid].type = BT_LR;
      P.bl[bid].id = (int)P.lr_block.size();
      P.lr_block.push_back(bid);
      return;
    }
    if (T.nchild == 0 && S.nchild == 0) {
      P.bl[bid].type = BT_DENSE;
      P.bl[bid].id = (int)P.dense_block.size();
      P.dense_block.push_back(bid);
      return;
    }
    int nrc = T.nchild ? T.nchild : 1;
    int ncc = S.nchild ? S.nchild : 1;
    int first = (int)P.bl.size();
    P.bl[bid].type = BT_H;
    P.bl[bid].child0 = first;
    P.bl[bid].nrc = nrc;
    P.bl[bid].ncc = ncc;
    for (int i = 0; i < nrc; ++i)
      for (int j = 0; j < ncc; ++j) {
        Block c{};
        c.t = T.nchild ? T.child[i] : b.t;
        c.s = S.nchild ? S.child[j] : b.s;
        c.type = BT_H;
        c.level = b.level + 1;
        c.id = -1;
        P.bl.push_back(c);
      }
    for (int k = 0; k < nrc * ncc; ++k) block(first + k);
  }
};

}  // namespace

int solve_mode(const hm_problem& p, const hm_opts& o) {
  if (o.solve == HM_SOLVE_SUBST || o.solve == HM_SOLVE_HINV) return o.solve;
  return (p.dim == 1 && p.domain == HM_DOMAIN_BOX && o.leaf <= 1024) ? HM_SOLVE_HINV : HM_SOLVE_SUBST;
}

double hinv_tolerance(const hm_opts& o) {
  if (o.hinv_tol > 0.0) return o.hinv_tol;
  if (o.precision == HM_MIXED_FP32) return 1e-7;
  if (o.precision == HM_MIXED_BF16) return 2e-3;
  return std::min(1e-6, std::max(1e-14, 1e-2 * o.lu_tol));
}

int make_plan(const hm_problem& p, const hm_opts& o, Plan& P, std::string& err) {
  if (p.dim != 1 && p.dim != 2) { err = "dim must be 1 or 2"; return HM_ERR_ARG; }
  if (p.n[0] < 1 || (p.dim == 2 && p.n[1] < 1)) { err = "n must be positive"; return HM_ERR_ARG; }
  if (o.leaf < 1) { err = "leaf must be >= 1"; return HM_ERR_ARG; }
  if (!(o.eta > 0)) { err = "eta must be > 0"; return HM_ERR_ARG; }
  if (o.precision != HM_FP64 && o.precision != HM_MIXED_FP32 && o.precision != HM_MIXED_BF16) {
    err = "precision must be HM_FP64, HM_MIXED_FP32 or HM_MIXED_BF16";
    return HM_ERR_ARG;
  }
  if (o.solve != HM_SOLVE_AUTO && o.solve != HM_SOLVE_SUBST && o.solve != HM_SOLVE_HINV) {
    err = "unknown solve mode";
    return HM_ERR_ARG;
  }
  if (o.solve_block < 0) { err = "solve_block must be >= 0"; return HM_ERR_ARG; }
  if (!(o.hinv_tol >= 0.0 && o.hinv_tol < 1.0)) { err = "hinv_tol must lie in [0, 1)"; return HM_ERR_ARG; }
  if (o.cn_form != HM_CN_IDENTITY && o.cn_form != HM_CN_LITERAL) { err = "unknown cn_form"; return HM_ERR_ARG; }
  const bool hinv_ok = p.dim == 1 && p.domain == HM_DOMAIN_BOX && o.leaf <= 1024;
  if (o.solve == HM_SOLVE_HINV && !hinv_ok) {
    err = "HM_SOLVE_HINV needs a 1D problem and leaves of at most 1024 points";
    return HM_ERR_ARG;
  }
  if (o.precision != HM_FP64 && solve_mode(p, o) != HM_SOLVE_HINV) {
    err = "mixed precision storage is built for the hierarchical-inverse solve (1D problems)";
    return HM_ERR_ARG;
  }
  P = Plan();
  P.dim = p.dim;
  P.n[0] = p.n[0];
  P.n[1] = p.dim == 2 ? p.n[1] : 1;
  int64_t full = (int64_t)P.n[0] * P.n[1];
  if (full > (1 << 26)) { err = "too many unknowns"; return HM_ERR_ARG; }
  // the L-shaped domain drops the grid points with both coordinates at or
  // beyond the box centre: x_a = lo_a + (i_a + 1) h >= centre_a iff 2 (i_a + 1) >= n_a + 1
  const bool lshape = p.domain == HM_DOMAIN_L && p.dim == 2;
  auto inside = [&](int i0, int i1) { return !(lshape && 2 * (i0 + 1) >= P.n[0] + 1 && 2 * (i1 + 1) >= P.n[1] + 1); };
  int64_t N = 0;
  for (int i1 = 0; i1 < P.n[1]; ++i1)
    for (int i0 = 0; i0 < P.n[0]; ++i0) N += inside(i0, i1);
  if (N < 1) { err = "the domain holds no grid point"; return HM_ERR_ARG; }
  P.N = (int)N;
  P.leaf = o.leaf;
  P.eta = o.eta;
  P.h = (p.hi[0] - p.lo[0]) / (p.n[0] + 1);
  if (!(P.h > 0)) { err = "hi must exceed lo"; return HM_ERR_ARG; }
  if (p.dim == 2) {
    double h1 = (p.hi[1] - p.lo[1]) / (p.n[1] + 1);
    if (std::fabs(h1 - P.h) > 1e-12 * P.h) { err = "2D grid needs square cells"; return HM_ERR_ARG; }
  }
  P.perm.resize(P.N);
  P.iperm.resize(P.N);
  P.coord.assign(2 * (size_t)P.N, 0);
  Builder B(P);
  if (p.dim == 1) {
    for (int i = 0; i < P.N; ++i) { P.perm[i] = i; P.coord[2 * i] = i; }
  } else {
    // natural order: the domain's grid points row by row (axis 0 fastest)
    std::vector<std::pair<uint64_t, int>> key;
    std::vector<int2> ij;
    key.reserve(P.N);
    ij.reserve(P.N);
    for (int i1 = 0; i1 < P.n[1]; ++i1)
      for (int i0 = 0; i0 < P.n[0]; ++i0) {
        if (!inside(i0, i1)) continue;
        const int nat = (int)key.size();
        key.push_back({spread_bits((uint32_t)i0) | (spread_bits((uint32_t)i1) << 1), nat});
        ij.push_back(make_int2(i0, i1));
      }
    std::sort(key.begin(), key.end());
    B.code.resize(P.N);
    for (int q = 0; q < P.N; ++q) {
      P.perm[q] = key[q].second;
      B.code[q] = key[q].first;
      P.coord[2 * q] = ij[key[q].second].x;
      P.coord[2 * q + 1] = ij[key[q].second].y;
    }
  }
  for (int q = 0; q < P.N; ++q) P.iperm[P.perm[q]] = q;

  Cluster root{};
  root.begin = 0;
  root.end = P.N;
  root.level = 0;
  root.parent = -1;
  B.bbox(root);
  P.cl.push_back(root);
  int topbit = 0;
  while ((1 << topbit) < std::max(P.n[0], P.n[1])) ++topbit;
  B.split(0, topbit);
  for (int c = 0; c < (int)P.cl.size(); ++c)
    if (P.cl[c].nchild == 0) P.leaves.push_back(c);
  std::sort(P.leaves.begin(), P.leaves.end(),
            [&](int x, int y) { return P.cl[x].begin < P.cl[y].begin; });

  Block rb{};
  rb.t = rb.s = 0;
  rb.type = BT_H;
  rb.level = 0;
  rb.id = -1;
  P.bl.push_back(rb);
  B.block(0);
  return HM_OK;
}

}  // namespace hm
