// Symbolic expansion of H-LU and of the H-triangular solves (App. "LU
// Decomposition") into dense operations with row-segment dependency waves.
//
// H-LU of a diagonal H-block with children A_ij (rows/cols split alike):
//   for i: LU(A_ii); for j > i: L_ii U_ij = A_ij, L_ji U_ii = A_ji;
//          for j, l > i: A_jl -= L_ji U_il
// with the triangular solves of the appendix (full right-hand side: dense
// solve; low-rank right-hand side B1 B2': (L^{-1} B1) B2'; H right-hand side:
// block forward substitution).  Leaf LU is unpivoted and also forms the
// inverses of the leaf factors, so leaf triangular solves become products.
// Sums of low-rank terms are recompressed at relative tolerance lu_tol
// (eps_2 of Sec. "Application") and the rank cap kf.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <queue>
#include <unordered_map>
#include <string>

#include "hlu_plan.h"

namespace hm {

double* Arena::alloc(int64_t n) {
  n = (n + 3) & ~int64_t(3);
  if (n > left) {
    int64_t chunk = std::max<int64_t>(n, int64_t(1) << 25);
    void* p = nullptr;
    if (fake) {
      if (fake_limit >= 0 && (int64_t)((fake_next - (uintptr_t(1) << 40)) + chunk * sizeof(double)) > fake_limit) {
        status = HM_ERR_OOM;  // injected allocation failure (dry runs only)
        return nullptr;
      }
      p = (void*)fake_next;
      fake_next += (uintptr_t)(chunk * sizeof(double)) + 4096;
    } else {
      if (cudaMalloc(&p, chunk * sizeof(double)) != cudaSuccess) {
        status = HM_ERR_OOM;
        return nullptr;
      }
      chunks.push_back(p);
    }
    ranges.push_back({(uintptr_t)p, (uintptr_t)p + (uintptr_t)(chunk * sizeof(double))});
    cur = (double*)p;
    left = chunk;
  }
  double* r = cur;
  cur += n;
  left -= n;
  total += n;
  return r;
}

void Arena::release() {
  for (void* p : chunks) cudaFree(p);
  chunks.clear();
  ranges.clear();
  cur = nullptr;
  left = 0;
}

namespace {

// Last write / last read wave per segment of every buffer.  Regular buffers
// are split into row segments; pooled temporaries into 64 element ranges.
struct Tracker {
  struct Buf {
    int seg;
    bool elem = false;
    const double* base = nullptr;
    std::vector<int> lw, lr;              // waves of the last write / latest read
    std::vector<int> wop;                 // op id of the last write (-1: none)
    std::vector<std::vector<int>> rops;   // op ids of the reads since the last write
    int maxw = -1;                        // latest wave of any access
    // Segments [u0, u1] share one state (set by a write of exactly that
    // range and kept while accesses cover exactly that range), held here
    // instead of in the per-segment arrays: most operations read and write
    // whole buffers, and this makes their tracking O(1).  A write leaves
    // ulr = -1: a later op's wave already exceeds the writer's, which
    // exceeds every earlier read.
    bool uni = false;
    int u0 = 0, u1 = -1, ulw = -1, ulr = -1, uwop = -1;
    std::vector<int> urops;
    int nseg = 1;  // segments; the per-segment arrays are allocated on first use
    void ensure() {
      if (!lw.empty()) return;
      lw.assign(nseg, -1);
      lr.assign(nseg, -1);
      wop.assign(nseg, -1);
      rops.resize(nseg);
    }
    void materialize() {
      ensure();
      for (int s = u0; s <= u1; ++s) {
        lw[s] = ulw;
        lr[s] = ulr;
        wop[s] = uwop;
        rops[s] = urops;
      }
      uni = false;
    }
  };
  std::vector<Buf> bufs;
  int add_elem(const double* base, int64_t cap) {
    Buf b;
    b.elem = true;
    b.base = base;
    b.seg = (int)std::max<int64_t>(1, (cap + 63) / 64);
    b.nseg = 64;
    bufs.push_back(std::move(b));
    return (int)bufs.size() - 1;
  }
  int add(int rows, int seg) {
    Buf b;
    b.seg = std::max(1, seg);
    b.nseg = std::max(1, (rows + b.seg - 1) / b.seg);
    bufs.push_back(std::move(b));
    return (int)bufs.size() - 1;
  }
};

struct Acc {
  const View* v;
  bool write;
};

#ifndef HM_KSLICE
#define HM_KSLICE 64  // smallest split-K slice (build-time tuning parameter)
#endif
#ifndef HM_TMP_LAG
#define HM_TMP_LAG 512  // waves between the last use of a temporary and its reuse (build-time tuning parameter)
#endif
#ifndef HM_GRAM_CHUNK
#define HM_GRAM_CHUNK 64  // rows per partial Gram product (build-time tuning parameter)
#endif
constexpr int GRAM_CHUNK = HM_GRAM_CHUNK;

class Emitter {
 public:
  Emitter(std::vector<Wave>& w, OpGraph& g, Arena& a, int seg) : waves(w), graph(g), A(a), seg_default(seg) {}

  std::vector<Wave>& waves;
  OpGraph& graph;
  int cur_id = -1;  // op id assigned by the last place()
  Arena& A;
  Arena* TA = nullptr;  // pooled temporaries (nullptr: A); no op after the H-LU reads them
  Tracker T;
  int seg_default;
  int64_t nops = 0;
  int status = HM_OK;
  int phase = 0;                        // FMA accounting bucket of the ops emitted now
  int prio = 0;                         // urgency recorded with the ops emitted now (OpGraph::prio)
  double gemm_fma[3] = {0.0, 0.0, 0.0};

  View new_mat(int rows, int cols, bool colmajor, int seg = -1, bool scratch = false) {
    View v;
    v.rows = rows;
    v.cols = cols;
    v.p = (scratch && TA ? *TA : A).alloc((int64_t)rows * cols);
    if (!v.p) status = HM_ERR_OOM;
    if (colmajor) { v.rs = 1; v.cs = rows; } else { v.rs = cols; v.cs = 1; }
    v.buf = T.add(rows, seg < 0 ? seg_default : seg);
    v.br0 = 0;
    v.br1 = rows;
    return v;
  }

  // Temporaries come from a pool per size class.  A buffer is reused only
  // once the last op that touched it lies at least tmp_lag waves behind the
  // deepest wave placed so far: its next writer then waits for ops that are
  // long finished when the executor reaches it, so reuse adds no false
  // dependency to the critical path (a plain FIFO reuse chains unrelated
  // operations of the same size class into one long sequence).
  struct Pooled {
    int lastw;
    double* p;
    int buf;
    bool operator>(const Pooled& o) const { return lastw > o.lastw; }
  };
  using Heap = std::priority_queue<Pooled, std::vector<Pooled>, std::greater<Pooled>>;
  std::vector<Heap> pool = std::vector<Heap>(64);
  int tmp_lag = HM_TMP_LAG;

  static int size_class(int64_t n) {
    int c = 0;
    while ((int64_t(1) << c) < n) ++c;
    return c;
  }

  View tmp(int rows, int cols, bool colmajor) {
    int64_t n = std::max<int64_t>(1, (int64_t)rows * cols);
    int c = size_class(n);
    View v;
    v.rows = rows;
    v.cols = cols;
    if (colmajor) { v.rs = 1; v.cs = rows; } else { v.rs = cols; v.cs = 1; }
    v.br0 = 0;
    v.br1 = 1;
    Heap& h = pool[c];
    if (!h.empty() && h.top().lastw < (int)waves.size() - tmp_lag) {
      v.p = h.top().p;
      v.buf = h.top().buf;
      h.pop();
    } else {
      v.p = (TA ? *TA : A).alloc(int64_t(1) << c);
      if (!v.p) status = HM_ERR_OOM;
      v.buf = T.add_elem(v.p, int64_t(1) << c);
    }
    v.tr = false;
    return v;
  }

  // Pooled scratch for `ns` parts of rows x cols (row-major): part i starts at
  // element i * stride, a multiple of the dependency tracker's segment of the
  // pooled buffer (1/64 of its capacity), so that operations on different
  // parts are independent.  Returns the whole buffer (one row) and the stride.
  // (The tracker has 64 segments per pooled buffer: more than 64 parts are
  // laid out contiguously, with some false dependencies between neighbours.)
  View tmp_parts(int ns, int rows, int cols, int64_t& stride) {
    const int64_t n = std::max<int64_t>(1, (int64_t)rows * cols);
    stride = n;
    if (ns > 64) return tmp(1, (int)(ns * n), false);
    int c = size_class(ns * n);
    for (int it = 0; it < 64; ++it) {
      const int64_t cap = int64_t(1) << c, seg = std::max<int64_t>(1, (cap + 63) / 64);
      stride = (n + seg - 1) / seg * seg;
      const int c2 = size_class(ns * stride);
      if (c2 <= c) break;
      c = c2;
    }
    return tmp(1, (int)(ns * stride), false);
  }
  static View part_of(const View& whole, int64_t stride, int i, int rows, int cols) {
    View v = whole;
    v.p = whole.p + i * stride;
    v.rows = rows;
    v.cols = cols;
    v.rs = cols;
    v.cs = 1;
    return v;
  }

  void release(const View& v) {
    int64_t n = std::max<int64_t>(1, (int64_t)v.rows * v.cols);
    pool[size_class(n)].push({T.bufs[v.buf].maxw, v.p, v.buf});
  }

  View wrap(double* p, int rows, int cols, int64_t rs, int64_t cs, int seg = -1) {
    View v;
    v.p = p;
    v.rows = rows;
    v.cols = cols;
    v.rs = rs;
    v.cs = cs;
    v.buf = T.add(rows, seg < 0 ? seg_default : seg);
    v.br0 = 0;
    v.br1 = rows;
    return v;
  }

  static void seg_range(const Tracker::Buf& B, const View& v, int& s0, int& s1) {
    const int ns = B.nseg;
    if (B.elem) {
      int64_t off = v.p - B.base;
      int64_t span = (int64_t)(std::max(v.rows, 1) - 1) * (v.rs < 0 ? -v.rs : v.rs) +
                     (int64_t)(std::max(v.cols, 1) - 1) * (v.cs < 0 ? -v.cs : v.cs) + 1;
      s0 = (int)std::min<int64_t>(off / B.seg, ns - 1);
      s1 = (int)std::min<int64_t>((off + span - 1) / B.seg, ns - 1);
    } else {
      s0 = std::min(v.br0 / B.seg, ns - 1);
      s1 = std::min((std::max(v.br1, v.br0 + 1) - 1) / B.seg, ns - 1);
    }
  }

  // Wave and producers of a new op from its accesses; records the op.
  // streaming of finished slices (HluBuild::sink)
  std::function<void(HluChunk&&)>* sink = nullptr;
  int64_t chunk_ops = 0;   // slice size; the first slices are smaller (8x, 4x, 2x) so the GPU starts early
  int64_t chunk_cur = 0;
  int chunk_first = 0;
  int chunk_wmin = 1 << 30;  // lowest wave holding an op of the open slice

  // Hand the ops placed since the last slice to the sink.  Called only at the
  // start of place() or after the last op: every op placed so far has been
  // added to its wave by then.
  void take_chunk() {
    const int last = graph.size();
    if (!sink || last == chunk_first) return;
    // once an allocation has failed, ops may hold null operands: nothing more
    // is handed out (the slices given earlier precede the failure)
    if (status != HM_OK || A.status != HM_OK) return;
    HluChunk c;
    c.first = chunk_first;
    for (int w = std::min(chunk_wmin, (int)waves.size()); w < (int)waves.size(); ++w) {
      if (waves[w].size() == 0) continue;
      c.wave_idx.push_back(w);
      c.waves.push_back(std::move(waves[w]));
      waves[w] = Wave();
    }
    for (int i = chunk_first; i < last; ++i) c.graph.add_op(graph.begin(i), graph.end(i), graph.prio_of(i));
    chunk_first = last;
    chunk_wmin = 1 << 30;
    chunk_cur = std::min(chunk_ops, 2 * chunk_cur);
    (*sink)(std::move(c));
  }

  std::vector<int> deps;  // scratch of place()
  int place(std::initializer_list<Acc> acc) {
    if (sink && graph.size() - chunk_first >= chunk_cur) take_chunk();
    int w = -1;
    deps.clear();
    for (const Acc& a : acc) {
      const View& v = *a.v;
      Tracker::Buf& B = T.bufs[v.buf];
      int s0, s1;
      seg_range(B, v, s0, s1);
      if (B.uni && s0 == B.u0 && s1 == B.u1) {
        w = std::max(w, B.ulw);
        if (B.uwop >= 0) deps.push_back(B.uwop);
        if (a.write) {
          w = std::max(w, B.ulr);
          deps.insert(deps.end(), B.urops.begin(), B.urops.end());
        }
        continue;
      }
      if (B.uni) B.materialize();
      B.ensure();
      for (int s = s0; s <= s1; ++s) {
        // neighbouring segments mostly share their writer and readers: skip repeats
        w = std::max(w, B.lw[s]);
        if (B.wop[s] >= 0 && (deps.empty() || deps.back() != B.wop[s])) deps.push_back(B.wop[s]);
        if (a.write) {
          w = std::max(w, B.lr[s]);
          if (s == s0 || B.rops[s] != B.rops[s - 1]) deps.insert(deps.end(), B.rops[s].begin(), B.rops[s].end());
        }
      }
    }
    ++w;
    if (deps.size() > 1) {
      std::sort(deps.begin(), deps.end());
      deps.erase(std::unique(deps.begin(), deps.end()), deps.end());
    }
    const int id = graph.add_op(deps, prio);
    for (const Acc& a : acc) {
      const View& v = *a.v;
      Tracker::Buf& B = T.bufs[v.buf];
      int s0, s1;
      seg_range(B, v, s0, s1);
      B.maxw = std::max(B.maxw, w);
      if (B.uni && s0 == B.u0 && s1 == B.u1) {
        if (a.write) {
          B.ulw = w;
          B.uwop = id;
          B.ulr = -1;
          B.urops.clear();
        } else {
          B.ulr = std::max(B.ulr, w);
          B.urops.push_back(id);
        }
        continue;
      }
      if (B.uni) B.materialize();
      B.ensure();
      if (a.write && s1 - s0 >= 3) {  // a written range of several segments becomes one shared state
        B.uni = true;
        B.u0 = s0;
        B.u1 = s1;
        B.ulw = w;
        B.uwop = id;
        B.ulr = -1;
        B.urops.clear();
      } else {
        for (int s = s0; s <= s1; ++s) {
          if (a.write) {
            B.lw[s] = w;
            B.wop[s] = id;
            B.rops[s].clear();
          } else {
            B.lr[s] = std::max(B.lr[s], w);
            B.rops[s].push_back(id);
          }
        }
      }
    }
    if ((int)waves.size() <= w) waves.resize(w + 1);
    chunk_wmin = std::min(chunk_wmin, w);
    ++nops;
    cur_id = id;
    return w;
  }

  // C = beta C + alpha sum_p parts[p]  (parts: nparts blocks of C.rows x C.cols, row-major)
  // stride: elements from one part to the next (0: C.rows * C.cols)
  void reduce(const View& C, double alpha, const View& parts, int nparts, double beta, int64_t stride = 0) {
    int w = beta != 0.0 ? place({{&parts, false}, {&C, false}, {&C, true}}) : place({{&parts, false}, {&C, true}});
    ReduceOp o{};
    o.parts = parts.p;
    o.dst = C.p;
    o.stride = stride > 0 ? stride : (int64_t)C.rows * C.cols;
    o.drs = C.rs;
    o.dcs = C.cs;
    o.m = C.rows;
    o.n = C.cols;
    o.nparts = nparts;
    o.alpha = alpha;
    o.beta = beta;
    waves[w].add(o, cur_id);
  }

  // C = beta C + alpha A B; a long inner dimension with few output tiles is
  // split into 256-wide slices reduced afterwards (FP64 throughput per SM is
  // low, so the work must reach many SMs).
  void gemm(const View& C, double alpha, const View& Am, const View& Bm, double beta) {
    if (C.rows == 0 || C.cols == 0) return;
    if (Am.cols != Bm.rows || Am.rows != C.rows || Bm.cols != C.cols) { status = HM_ERR_ARG; return; }
    if (Am.cols == 0) {
      if (beta != 1.0) copy(C, 0.0, nullptr, beta);
      return;
    }
    const int K = Am.cols;
    const int tiles = gemm_tiles(C.rows, C.cols);
    // a tile costs 1024 k FP64 FMAs on one SM (about 0.27 us per unit of k at
    // two FP64 FMAs per cycle): long inner dimensions with few tiles are split
    // so that the work reaches more SMs, in slices of at least HM_KSLICE
    int KS = 0;
    if (tiles < 76 && K >= 2 * HM_KSLICE) {
      const int want = std::max(2, 152 / tiles);            // slices that fill the SMs
      const int ns = std::min(want, K / HM_KSLICE);
      if (ns >= 2) KS = ((K + ns - 1) / ns + 15) / 16 * 16;
    }
    if (KS) {
      const int ns = (K + KS - 1) / KS;
      int64_t stride = 0;
      View parts = tmp_parts(ns, C.rows, C.cols, stride);
      for (int c = 0; c < ns; ++c) {
        int k0 = c * KS, kn = std::min(KS, K - k0);
        gemm_direct(part_of(parts, stride, c, C.rows, C.cols), 1.0, Am.sub(0, k0, Am.rows, kn),
                    Bm.sub(k0, 0, kn, Bm.cols), 0.0);
      }
      reduce(C, alpha, parts, ns, beta, stride);
      release(parts);
      return;
    }
    gemm_direct(C, alpha, Am, Bm, beta);
  }

  void gemm_direct(const View& C, double alpha, const View& Am, const View& Bm, double beta) {
    gemm_fma[phase] += (double)C.rows * C.cols * Am.cols;
    int w = beta != 0.0 ? place({{&Am, false}, {&Bm, false}, {&C, false}, {&C, true}})
                        : place({{&Am, false}, {&Bm, false}, {&C, true}});
    GemmOp o{};
    o.A = Am.p;
    o.B = Bm.p;
    o.C = C.p;
    o.m = C.rows;
    o.n = C.cols;
    o.k = Am.cols;
    o.shape = gemm_shape(o.m, o.n);
    o.ars = Am.rs;
    o.acs = Am.cs;
    o.brs = Bm.rs;
    o.bcs = Bm.cs;
    o.crs = C.rs;
    o.ccs = C.cs;
    o.alpha = alpha;
    o.beta = beta;
    waves[w].add(o, cur_id);
  }

  // dst = beta dst + alpha src (src null: constant alpha)
  void copy(const View& dst, double alpha, const View* src, double beta) {
    if (dst.rows == 0 || dst.cols == 0) return;
    int w;
    if (src) {
      w = beta != 0.0 ? place({{src, false}, {&dst, false}, {&dst, true}}) : place({{src, false}, {&dst, true}});
    } else {
      w = beta != 0.0 ? place({{&dst, false}, {&dst, true}}) : place({{&dst, true}});
    }
    CopyOp o{};
    o.src = src ? src->p : nullptr;
    o.dst = dst.p;
    o.m = dst.rows;
    o.n = dst.cols;
    o.srs = src ? src->rs : 0;
    o.scs = src ? src->cs : 0;
    o.drs = dst.rs;
    o.dcs = dst.cs;
    o.alpha = alpha;
    o.beta = beta;
    waves[w].add(o, cur_id);
  }

  void lu(const View& Am, const View& Li, const View& Ui) {
    int w = place({{&Am, false}, {&Am, true}, {&Li, true}, {&Ui, true}});
    LuOp o{};
    o.A = Am.p;
    o.Li = Li.p;
    o.Ui = Ui.p;
    o.lda = Am.rs;
    o.ldl = Li.rs;
    o.ldu = Ui.rs;
    o.m = Am.rows;
    waves[w].add(o, cur_id);
  }

  // Gram matrix G = X' X (K x K row-major, fresh), split over GRAM_CHUNK-row
  // chunks so that the K x K x rows FMAs of one Gram matrix spread over SMs.
  View gram(const View& X) {
    const int K = X.cols;
    View G = tmp(K, K, false);
    const int CH = GRAM_CHUNK;
    int nch = (X.rows + CH - 1) / CH;
    if (nch <= 1) {
      gemm_direct(G, 1.0, X.T(), X, 0.0);
      return G;
    }
    int64_t stride = 0;
    View parts = tmp_parts(nch, K, K, stride);
    for (int c = 0; c < nch; ++c) {
      int r0 = c * CH, nr = std::min(CH, X.rows - r0);
      View Xc = X.sub(r0, 0, nr, K);
      gemm_direct(part_of(parts, stride, c, K, K), 1.0, Xc.T(), Xc, 0.0);
    }
    reduce(G, 1.0, parts, nch, 0.0, stride);
    release(parts);
    return G;
  }

  void trunc(const View& GA, const View& GB, const View& TA, const View& TB, int* rank,
             const View& rankv, int K, int kf, double tol) {
    int w = place({{&GA, false}, {&GB, false}, {&TA, true}, {&TB, true}, {&rankv, true}});
    TruncOp o{};
    o.GA = GA.p;
    o.GB = GB.p;
    o.TA = TA.p;
    o.TB = TB.p;
    o.rank = rank;
    o.K = K;
    o.kf = kf;
    o.tol = tol;
    waves[w].add(o, cur_id);
  }
};

// ---------------------------------------------------------------- H-LU

// Low-rank updates are accumulated: a block's current slot holds its factor in
// the first kf columns and pending update terms after them; the sum is
// recompressed once, when the pending columns are full or the block is read.
#ifndef HM_LR_ACC
#define HM_LR_ACC 3  // pending capacity in multiples of kf (build-time tuning parameter)
#endif
#ifndef HM_TRUNC_KCAP
#define HM_TRUNC_KCAP 96  // widest accumulated sum, kf + pending (build-time tuning parameter)
#endif
struct LRState {
  View U[2], V[2];   // slots: m x (1 + nacc) kf and n x (1 + nacc) kf, column-major
  View rankv;        // dependency token for the rank word
  int cur = 0;
  int pend = 0;      // pending columns after the first kf of the current slot
  int m = 0, n = 0;
  int urg = 0;       // urgency of its recompressions: max(row, column) of the block
  int* rank = nullptr;
};

struct Target {
  int b;          // block id
  int ro, co;     // offset inside the block
  int nr, nc;
};

class HLU {
 public:
  HLU(const Plan& P_, Emitter& E_, int kf_, double tol_) : P(P_), E(E_), kf(kf_), tol(tol_) {}

  const Plan& P;
  Emitter& E;
  int kf;
  double tol;
  int lu_base = LU_BASE;          // base-case size of the dense leaf LUs (HM_LU_BASE, <= LU_BASE)
  std::vector<View> dense;        // per dense id: current storage
  std::vector<View> linv, uinv;   // per dense id (diagonal leaves only)
  std::vector<LRState> lr;

  const Block& B(int b) const { return P.bl[b]; }
  int rows(int b) const { const Cluster& c = P.cl[B(b).t]; return c.end - c.begin; }
  int cols(int b) const { const Cluster& c = P.cl[B(b).s]; return c.end - c.begin; }
  int child(int b, int i, int j) const { return B(b).child0 + i * B(b).ncc + j; }
  int nrc(int b) const { return B(b).type == BT_H ? B(b).nrc : 1; }
  int ncc(int b) const { return B(b).type == BT_H ? B(b).ncc : 1; }
  int sub(int b, int i, int j) const { return B(b).type == BT_H ? child(b, i, j) : b; }

  // Urgency of the ops that write (rows ro.., columns co.. of) block b: the
  // elimination along the diagonal first needs the result when it reaches
  // the block's later corner, max(row, column).  Among the ops of one wave
  // the executor hands out the lower values first, so the ops on the
  // diagonal's dependency chain go ahead of the far-field updates.
  int urgency(int b, int ro = 0, int co = 0) const {
    return std::max(P.cl[B(b).t].begin + ro, P.cl[B(b).s].begin + co);
  }
  struct Prio {  // sets the emitter's urgency for a scope
    Emitter& E;
    int old;
    Prio(Emitter& e, int p) : E(e), old(e.prio) { E.prio = p; }
    ~Prio() { E.prio = old; }
  };
  // offset of child row cluster inside the parent row cluster
  int roff(int parent, int ch) const { return P.cl[B(ch).t].begin - P.cl[B(parent).t].begin; }
  int coff(int parent, int ch) const { return P.cl[B(ch).s].begin - P.cl[B(parent).s].begin; }

  // pending update columns a block may hold: the recompression of kf + pending
  // columns costs about K^3 FP64 operations on one SM, so the accumulated width
  // K stays within HM_TRUNC_KCAP (and the truncation core's TRUNC_MAXK)
  int nacc() const { return std::max(1, std::min(HM_LR_ACC, std::min(TRUNC_MAXK, HM_TRUNC_KCAP) / kf - 1)); }
  int pend_cap() const { return nacc() * kf; }
  // readers see the recompressed factor
  View lrU(int q) { flush(q); return lr[q].U[lr[q].cur].sub(0, 0, lr[q].m, kf); }
  View lrV(int q) { flush(q); return lr[q].V[lr[q].cur].sub(0, 0, lr[q].n, kf); }
  void flush(int q) {
    if (lr[q].pend > 0) {
      Prio g(E, lr[q].urg);
      const int K = kf + lr[q].pend;
      lr[q].pend = 0;
      truncate(q, K);
    }
  }

  // ---- leaf LU with inverses of both factors
  void luinv(const View& Am, const View& Li, const View& Ui) {
    const int m = Am.rows;
    if (m <= lu_base) { E.lu(Am, Li, Ui); return; }
    const int h = m / 2, r = m - h;
    View A11 = Am.sub(0, 0, h, h), A12 = Am.sub(0, h, h, r), A21 = Am.sub(h, 0, r, h), A22 = Am.sub(h, h, r, r);
    View Li11 = Li.sub(0, 0, h, h), Li21 = Li.sub(h, 0, r, h), Li12 = Li.sub(0, h, h, r), Li22 = Li.sub(h, h, r, r);
    View Ui11 = Ui.sub(0, 0, h, h), Ui12 = Ui.sub(0, h, h, r), Ui21 = Ui.sub(h, 0, r, h), Ui22 = Ui.sub(h, h, r, r);
    // the zero blocks of the triangular inverses first: they depend on nothing,
    // so the products that read a whole inverse do not wait for them at the end
    E.copy(Li12, 0.0, nullptr, 0.0);
    E.copy(Ui21, 0.0, nullptr, 0.0);
    luinv(A11, Li11, Ui11);
    View T12 = E.tmp(h, r, false), T21 = E.tmp(r, h, false);
    E.gemm(T12, 1.0, Li11, A12, 0.0);   // U12 = L11^{-1} A12
    E.gemm(T21, 1.0, A21, Ui11, 0.0);   // L21 = A21 U11^{-1}
    E.gemm(A22, -1.0, T21, T12, 1.0);   // Schur complement
    // the halves of the off-diagonal inverse blocks that need no factor of
    // A22, formed while A22 is factored: one product after its LU, not two
    View X = E.tmp(r, h, false), Y = E.tmp(h, r, false);
    E.gemm(X, 1.0, T21, Li11, 0.0);     // L21 L11^{-1}
    E.gemm(Y, 1.0, Ui11, T12, 0.0);     // U11^{-1} U12
    luinv(A22, Li22, Ui22);
    E.gemm(Li21, -1.0, Li22, X, 0.0);   // (L^{-1})_21 = -L22^{-1} L21 L11^{-1}
    E.gemm(Ui12, -1.0, Y, Ui22, 0.0);   // (U^{-1})_12 = -U11^{-1} U12 U22^{-1}
    E.release(T12);
    E.release(T21);
    E.release(X);
    E.release(Y);
  }

  // ---- recompression of the low-rank sum held in the current slot (K columns)
  void truncate(int q, int K) {
    LRState& S = lr[q];
    View Aall = S.U[S.cur].sub(0, 0, S.m, K), Ball = S.V[S.cur].sub(0, 0, S.n, K);
    View GA = E.gram(Aall), GB = E.gram(Ball);
    View TA = E.tmp(K, kf, false), TB = E.tmp(K, kf, false);
    E.trunc(GA, GB, TA, TB, S.rank, S.rankv, K, kf, tol);
    int nx = 1 - S.cur;
    E.gemm(S.U[nx].sub(0, 0, S.m, kf), 1.0, Aall, TA, 0.0);
    E.gemm(S.V[nx].sub(0, 0, S.n, kf), 1.0, Ball, TB, 0.0);
    E.release(GA);
    E.release(GB);
    E.release(TA);
    E.release(TB);
    S.cur = nx;
  }

  // ---- tgt += alpha Up Vp'
  void add_lr(const Target& tg, const View& Up, const View& Vp, double alpha) {
    const Block& C = B(tg.b);
    Prio g(E, urgency(tg.b, tg.ro, tg.co));
    const int w = Up.cols;
    if (w == 0 || tg.nr == 0 || tg.nc == 0) return;
    if (C.type == BT_DENSE) {
      E.gemm(dense[C.id].sub(tg.ro, tg.co, tg.nr, tg.nc), alpha, Up, Vp.T(), 1.0);
      return;
    }
    if (C.type == BT_LR) {
      if (w > kf) {
        for (int c0 = 0; c0 < w; c0 += kf) {
          int wc = std::min(kf, w - c0);
          add_lr(tg, Up.sub(0, c0, Up.rows, wc), Vp.sub(0, c0, Vp.rows, wc), alpha);
        }
        return;
      }
      LRState& S = lr[C.id];
      if (S.pend + w > pend_cap()) flush(C.id);
      View Upend = S.U[S.cur].sub(0, kf + S.pend, S.m, w), Vpend = S.V[S.cur].sub(0, kf + S.pend, S.n, w);
      if (tg.ro != 0 || tg.nr != S.m) E.copy(Upend, 0.0, nullptr, 0.0);
      if (tg.co != 0 || tg.nc != S.n) E.copy(Vpend, 0.0, nullptr, 0.0);
      E.copy(Upend.sub(tg.ro, 0, tg.nr, w), alpha, &Up, 0.0);
      E.copy(Vpend.sub(tg.co, 0, tg.nc, w), 1.0, &Vp, 0.0);
      S.pend += w;
      return;
    }
    // H target: split over the children that intersect the target range
    for (int i = 0; i < C.nrc; ++i)
      for (int j = 0; j < C.ncc; ++j) {
        int ch = child(tg.b, i, j);
        int r0 = roff(tg.b, ch), r1 = r0 + rows(ch);
        int c0 = coff(tg.b, ch), c1 = c0 + cols(ch);
        int a0 = std::max(r0, tg.ro), a1 = std::min(r1, tg.ro + tg.nr);
        int b0 = std::max(c0, tg.co), b1 = std::min(c1, tg.co + tg.nc);
        if (a0 >= a1 || b0 >= b1) continue;
        Target t2{ch, a0 - r0, b0 - c0, a1 - a0, b1 - b0};
        add_lr(t2, Up.sub(a0 - tg.ro, 0, a1 - a0, w), Vp.sub(b0 - tg.co, 0, b1 - b0, w), alpha);
      }
  }

  // ---- out += alpha A in   (A block (t, r), in |r| x k, out |t| x k)
  void hgemm(const View& out, double alpha, int a, const View& in) {
    const Block& A = B(a);
    if (A.type == BT_DENSE) { E.gemm(out, alpha, dense[A.id], in, 1.0); return; }
    if (A.type == BT_LR) {
      View W = E.tmp(kf, in.cols, false);
      E.gemm(W, 1.0, lrV(A.id).T(), in, 0.0);
      E.gemm(out, alpha, lrU(A.id), W, 1.0);
      E.release(W);
      return;
    }
    for (int i = 0; i < A.nrc; ++i)
      for (int j = 0; j < A.ncc; ++j) {
        int c = child(a, i, j);
        hgemm(out.sub(roff(a, c), 0, rows(c), out.cols), alpha, c, in.sub(coff(a, c), 0, cols(c), in.cols));
      }
  }

  // ---- out += alpha A' in   (A block (r, t), in |r| x k, out |t| x k)
  void hgemm_t(const View& out, double alpha, int a, const View& in) {
    const Block& A = B(a);
    if (A.type == BT_DENSE) { E.gemm(out, alpha, dense[A.id].T(), in, 1.0); return; }
    if (A.type == BT_LR) {
      View W = E.tmp(kf, in.cols, false);
      E.gemm(W, 1.0, lrU(A.id).T(), in, 0.0);
      E.gemm(out, alpha, lrV(A.id), W, 1.0);
      E.release(W);
      return;
    }
    for (int i = 0; i < A.nrc; ++i)
      for (int j = 0; j < A.ncc; ++j) {
        int c = child(a, i, j);
        hgemm_t(out.sub(coff(a, c), 0, cols(c), out.cols), alpha, c, in.sub(roff(a, c), 0, rows(c), in.cols));
      }
  }

  // ---- X <- L^{-1} X for the diagonal block l (X: |t| x k, a view into storage)
  void lsolve_mat(int l, const View& X) {
    const Block& L = B(l);
    if (L.type == BT_DENSE) {
      View Tm = E.tmp(X.rows, X.cols, false);
      E.gemm(Tm, 1.0, linv[L.id], X, 0.0);
      E.copy(X, 1.0, &Tm, 0.0);
      E.release(Tm);
      return;
    }
    const int nc = L.nrc;
    for (int a = 0; a < nc; ++a) {
      int la = child(l, a, a);
      View Xa = X.sub(roff(l, la), 0, rows(la), X.cols);
      lsolve_mat(la, Xa);
      for (int a2 = a + 1; a2 < nc; ++a2) {
        int lb = child(l, a2, a);
        hgemm(X.sub(roff(l, lb), 0, rows(lb), X.cols), -1.0, lb, Xa);
      }
    }
  }

  // ---- Y <- U^{-T} Y for the diagonal block u (Y: |s| x k)
  void usolve_t_mat(int u, const View& Y) {
    const Block& U = B(u);
    if (U.type == BT_DENSE) {
      View Tm = E.tmp(Y.rows, Y.cols, false);
      E.gemm(Tm, 1.0, uinv[U.id].T(), Y, 0.0);
      E.copy(Y, 1.0, &Tm, 0.0);
      E.release(Tm);
      return;
    }
    const int nc = U.nrc;
    for (int a = 0; a < nc; ++a) {
      int ua = child(u, a, a);
      View Ya = Y.sub(roff(u, ua), 0, rows(ua), Y.cols);
      usolve_t_mat(ua, Ya);
      for (int a2 = a + 1; a2 < nc; ++a2) {
        int ub = child(u, a, a2);  // U_{a, a2}; rows of Y_{a2} are its columns
        hgemm_t(Y.sub(coff(u, ub), 0, cols(ub), Y.cols), -1.0, ub, Ya);
      }
    }
  }

  // ---- X <- L_l^{-1} [D | I] for the diagonal block l: X (rows(l) x (c0 +
  // rows(l))) holds arbitrary columns D in [0, c0) and, implicitly, the identity
  // of l's rows in [c0, c0 + rows(l)); the columns after that are zero and
  // stay zero (the inverse is lower triangular), so they are not touched.
  void linv_ident(int l, const View& X, int c0) {
    const Block& L = B(l);
    const int m = rows(l);
    if (L.type == BT_DENSE) {
      if (c0 > 0) {
        View Tm = E.tmp(m, c0, false);
        E.gemm(Tm, 1.0, linv[L.id], X.sub(0, 0, m, c0), 0.0);
        E.copy(X.sub(0, 0, m, c0), 1.0, &Tm, 0.0);
        E.release(Tm);
      }
      E.copy(X.sub(0, c0, m, m), 1.0, &linv[L.id], 0.0);  // L^{-1} I
      return;
    }
    for (int a = 0; a < L.nrc; ++a) {
      const int la = child(l, a, a), ra = roff(l, la), w = c0 + ra + rows(la);
      View Xa = X.sub(ra, 0, rows(la), w);
      linv_ident(la, Xa, c0 + ra);
      for (int a2 = a + 1; a2 < L.nrc; ++a2) {
        const int lb = child(l, a2, a);
        hgemm(X.sub(roff(l, lb), 0, rows(lb), w), -1.0, lb, Xa);
      }
    }
  }

  // ---- Y <- U_u^{-T} [D | I], the same for the transposed upper factor
  void uinvt_ident(int u, const View& Y, int c0) {
    const Block& U = B(u);
    const int m = rows(u);
    if (U.type == BT_DENSE) {
      View UiT = uinv[U.id].T();
      if (c0 > 0) {
        View Tm = E.tmp(m, c0, false);
        E.gemm(Tm, 1.0, UiT, Y.sub(0, 0, m, c0), 0.0);
        E.copy(Y.sub(0, 0, m, c0), 1.0, &Tm, 0.0);
        E.release(Tm);
      }
      E.copy(Y.sub(0, c0, m, m), 1.0, &UiT, 0.0);  // U^{-T} I
      return;
    }
    for (int a = 0; a < U.nrc; ++a) {
      const int ua = child(u, a, a), ra = roff(u, ua), w = c0 + ra + rows(ua);
      View Ya = Y.sub(ra, 0, rows(ua), w);
      uinvt_ident(ua, Ya, c0 + ra);
      for (int a2 = a + 1; a2 < U.nrc; ++a2) {
        const int ub = child(u, a, a2);  // U_{a, a2}; rows of Y_{a2} are its columns
        hgemm_t(Y.sub(coff(u, ub), 0, cols(ub), w), -1.0, ub, Ya);
      }
    }
  }

  // ---- X <- L_ll^{-1} X  (X block with the row cluster of l)
  void trsm_l(int l, int x) {
    const Block& X = B(x);
    Prio g(E, urgency(x));
    if (X.type == BT_DENSE) {
      const Block& L = B(l);
      View Tm = E.new_mat(rows(x), cols(x), false);
      E.gemm(Tm, 1.0, linv[L.id], dense[X.id], 0.0);
      dense[X.id] = Tm;
      return;
    }
    if (X.type == BT_LR) { lsolve_mat(l, lrU(X.id)); return; }
    const Block& L = B(l);
    if (L.type != BT_H) {
      for (int j = 0; j < X.ncc; ++j) trsm_l(l, child(x, 0, j));
      return;
    }
    for (int a = 0; a < L.nrc; ++a) {
      for (int j = 0; j < X.ncc; ++j) trsm_l(child(l, a, a), child(x, a, j));
      for (int a2 = a + 1; a2 < L.nrc; ++a2)
        for (int j = 0; j < X.ncc; ++j) {
          int c = child(x, a2, j);
          mulsub(Target{c, 0, 0, rows(c), cols(c)}, child(l, a2, a), child(x, a, j));
        }
    }
  }

  // ---- X <- X U_uu^{-1}  (X block with the column cluster of u)
  void trsm_u(int u, int x) {
    const Block& X = B(x);
    Prio g(E, urgency(x));
    if (X.type == BT_DENSE) {
      const Block& U = B(u);
      View Tm = E.new_mat(rows(x), cols(x), false);
      E.gemm(Tm, 1.0, dense[X.id], uinv[U.id], 0.0);
      dense[X.id] = Tm;
      return;
    }
    if (X.type == BT_LR) { usolve_t_mat(u, lrV(X.id)); return; }
    const Block& U = B(u);
    if (U.type != BT_H) {
      for (int i = 0; i < X.nrc; ++i) trsm_u(u, child(x, i, 0));
      return;
    }
    for (int a = 0; a < U.nrc; ++a) {
      for (int i = 0; i < X.nrc; ++i) trsm_u(child(u, a, a), child(x, i, a));
      for (int a2 = a + 1; a2 < U.nrc; ++a2)
        for (int i = 0; i < X.nrc; ++i) {
          int c = child(x, i, a2);
          mulsub(Target{c, 0, 0, rows(c), cols(c)}, child(x, i, a), child(u, a, a2));
        }
    }
  }

  // ---- tgt -= A B  (A block (t', r), B block (r, s'), tgt rows t', cols s')
  void mulsub(const Target& tg, int a, int b) {
    const Block& A = B(a);
    const Block& Bb = B(b);
    Prio g(E, urgency(tg.b, tg.ro, tg.co));
    if (A.type == BT_LR) {
      View W = E.tmp(cols(b), kf, true);
      E.copy(W, 0.0, nullptr, 0.0);
      hgemm_t(W, 1.0, b, lrV(A.id));           // W = B' V_A
      add_lr(tg, lrU(A.id), W, -1.0);
      E.release(W);
      return;
    }
    if (Bb.type == BT_LR) {
      View W = E.tmp(rows(a), kf, true);
      E.copy(W, 0.0, nullptr, 0.0);
      hgemm(W, 1.0, a, lrU(Bb.id));            // W = A U_B
      add_lr(tg, W, lrV(Bb.id), -1.0);
      E.release(W);
      return;
    }
    const Block& C = B(tg.b);
    if (A.type == BT_DENSE && Bb.type == BT_DENSE) {
      if (C.type == BT_DENSE) {
        E.gemm(dense[C.id].sub(tg.ro, tg.co, tg.nr, tg.nc), -1.0, dense[A.id], dense[Bb.id], 1.0);
      } else {
        // product of two dense leaves into a low-rank target: exact pieces of
        // width <= kf over the inner dimension
        add_lr(tg, dense[A.id], dense[Bb.id].T(), -1.0);
      }
      return;
    }
    const bool full = tg.ro == 0 && tg.co == 0 && tg.nr == rows(tg.b) && tg.nc == cols(tg.b);
    const int nk = A.type == BT_H ? A.ncc : Bb.nrc;
    if (C.type == BT_H && full) {
      for (int i = 0; i < C.nrc; ++i)
        for (int j = 0; j < C.ncc; ++j)
          for (int l = 0; l < nk; ++l) {
            int c = child(tg.b, i, j);
            mulsub(Target{c, 0, 0, rows(c), cols(c)}, sub(a, i, l), sub(b, l, j));
          }
      return;
    }
    // low-rank / dense / partial target: recurse on virtual sub-blocks
    const int nr = nrc(a), ncl = ncc(b);
    for (int i = 0; i < nr; ++i)
      for (int j = 0; j < ncl; ++j)
        for (int l = 0; l < nk; ++l) {
          int ai = sub(a, i, l), bj = sub(b, l, j);
          int ro = tg.ro + (P.cl[B(ai).t].begin - P.cl[A.t].begin);
          int co = tg.co + (P.cl[B(bj).s].begin - P.cl[Bb.s].begin);
          mulsub(Target{tg.b, ro, co, rows(ai), cols(bj)}, ai, bj);
        }
  }

  void hlu(int b) {
    const Block& X = B(b);
    if (X.type == BT_DENSE) {
      Prio g(E, urgency(b));
      int m = rows(b);
      linv[X.id] = E.new_mat(m, m, false, LU_SEG);
      uinv[X.id] = E.new_mat(m, m, false, LU_SEG);
      luinv(dense[X.id], linv[X.id], uinv[X.id]);
      return;
    }
    const int nc = X.nrc;
    for (int i = 0; i < nc; ++i) {
      hlu(child(b, i, i));
      for (int j = i + 1; j < nc; ++j) {
        trsm_l(child(b, i, i), child(b, i, j));
        trsm_u(child(b, i, i), child(b, j, i));
      }
      for (int j = i + 1; j < nc; ++j)
        for (int l = i + 1; l < nc; ++l) {
          int c = child(b, j, l);
          mulsub(Target{c, 0, 0, rows(c), cols(c)}, child(b, j, i), child(b, i, l));
        }
    }
  }
};

}  // namespace

int plan_hlu(const Plan& P, const std::vector<DenseDesc>& dd, const double* d_dense,
             const std::vector<LRDesc>& ld, const double* d_U, const double* d_V, int kf,
             double theta, double lu_tol, int* d_rank_f, Arena& arena, HluBuild& out, double alpha,
             int sb_rows_opt, bool solve_blocks, Arena* tmp_arena) {
  Emitter E(out.waves, out.graph, arena, std::max(1, std::min(P.leaf, 256)));
  E.TA = tmp_arena;
  if (const char* lag = std::getenv("HM_TMP_LAG")) E.tmp_lag = std::atoi(lag);
  if (out.sink && out.chunk_ops > 0) {
    E.sink = &out.sink;
    E.chunk_ops = out.chunk_ops;
    E.chunk_cur = std::max<int64_t>(1, out.chunk_ops / 8);
  }
  HLU H(P, E, kf, lu_tol);
  if (const char* lb = std::getenv("HM_LU_BASE")) H.lu_base = std::max(8, std::min(LU_BASE, std::atoi(lb)));
  const int nd = (int)dd.size(), nl = (int)ld.size();
  H.dense.resize(nd);
  H.linv.resize(nd);
  H.uinv.resize(nd);
  H.lr.resize(nl);
  // M = I + theta G in factor storage
  for (int d = 0; d < nd; ++d) {
    const DenseDesc& D = dd[d];
    View src = E.wrap(const_cast<double*>(d_dense) + D.off, D.m, D.n, D.ld, 1);
    View dst = E.new_mat(D.m, D.n, false, LU_SEG);
    E.copy(dst, theta, &src, 0.0);
    if (D.r0 == D.c0 && alpha != 0.0) {
      View diag = dst;
      diag.cols = 1;
      diag.rs = dst.rs + 1;
      diag.cs = 0;
      E.copy(diag, alpha, nullptr, 1.0);  // + alpha on the diagonal
    }
    H.dense[d] = dst;
  }
  for (int q = 0; q < nl; ++q) {
    const LRDesc& L = ld[q];
    LRState& S = H.lr[q];
    S.m = L.m;
    S.n = L.n;
    S.urg = std::max(L.r0, L.c0);
    S.rank = d_rank_f + q;
    for (int s = 0; s < 2; ++s) {
      // working slots (factor + pending update columns, ping-pong): scratch when
      // a temporaries arena is given; the final factor is copied out below
      S.U[s] = E.new_mat(L.m, (1 + H.nacc()) * kf, true, -1, true);
      S.V[s] = E.new_mat(L.n, (1 + H.nacc()) * kf, true, -1, true);
    }
    S.rankv = E.new_mat(1, 1, false, 1);
    int kc = std::min(L.kcap, kf);
    View Us = E.wrap(const_cast<double*>(d_U) + L.uoff, L.m, kc, 1, L.m);
    View Vs = E.wrap(const_cast<double*>(d_V) + L.voff, L.n, kc, 1, L.n);
    E.copy(S.U[0].sub(0, 0, L.m, kc), theta, &Us, 0.0);
    E.copy(S.V[0].sub(0, 0, L.n, kc), 1.0, &Vs, 0.0);
    if (kc < kf) {
      E.copy(S.U[0].sub(0, kc, L.m, kf - kc), 0.0, nullptr, 0.0);
      E.copy(S.V[0].sub(0, kc, L.n, kf - kc), 0.0, nullptr, 0.0);
    }
  }
  H.hlu(0);
  for (int q = 0; q < nl; ++q) H.flush(q);  // recompress what is still pending
  // the final low-rank factors in tight storage (m x kf, n x kf), copied out of
  // the working slots (which lie with the temporaries when tmp_arena is given)
  std::vector<View> fin_u(nl), fin_v(nl);
  for (int q = 0; q < nl; ++q) {
    if (tmp_arena) {
      fin_u[q] = E.new_mat(ld[q].m, kf, true);
      fin_v[q] = E.new_mat(ld[q].n, kf, true);
      View su = H.lrU(q), sv = H.lrV(q);
      E.copy(fin_u[q], 1.0, &su, 0.0);
      E.copy(fin_v[q], 1.0, &sv, 0.0);
    } else {
      fin_u[q] = H.lrU(q);
      fin_v[q] = H.lrV(q);
    }
  }
  if (solve_blocks) {
    E.phase = 1;
    // Solve blocks and their exact diagonal inverses, then the scaled couplings.
    FactorLayout& FL = out.F;
    {
      // 1D problems from 32768 unknowns use solve blocks twice as large: half as
      // many steps on the solve's dependency chain for 36 % more inverse FMAs
      // (measured at N = 65536: solve 1.57 -> 1.42 ms, factor +0.06 s)
      const int sb_rows = sb_rows_opt > 0 ? sb_rows_opt : ((P.dim == 1 && P.N >= 32768) ? 2 * SOLVE_BLOCK : SOLVE_BLOCK);
      std::vector<int> stack = {0};
      while (!stack.empty()) {
        int c = stack.back();
        stack.pop_back();
        const Cluster& C = P.cl[c];
        if (C.end - C.begin <= sb_rows || C.nchild == 0) {
          FL.sb_cluster.push_back(c);
        } else {
          for (int k = C.nchild - 1; k >= 0; --k) stack.push_back(C.child[k]);
        }
      }
      std::sort(FL.sb_cluster.begin(), FL.sb_cluster.end(),
                [&](int x, int y) { return P.cl[x].begin < P.cl[y].begin; });
    }
    std::vector<int> diag_block(P.cl.size(), -1);
    for (int bi = 0; bi < (int)P.bl.size(); ++bi)
      if (P.bl[bi].t == P.bl[bi].s) diag_block[P.bl[bi].t] = bi;
    const int nsb = (int)FL.sb_cluster.size();
    std::vector<View> sbL(nsb), sbU(nsb);
    for (int k = 0; k < nsb; ++k) {
      const Cluster& C = P.cl[FL.sb_cluster[k]];
      const int S = C.end - C.begin;
      const int db = diag_block[FL.sb_cluster[k]];
      View Li = E.new_mat(S, S, false), UiT = E.new_mat(S, S, false), Ui = E.new_mat(S, S, false);
      for (View* X : {&Li, &UiT}) E.copy(*X, 0.0, nullptr, 0.0);
      H.linv_ident(db, Li, 0);    // L_BB^{-1}
      H.uinvt_ident(db, UiT, 0);  // U_BB^{-T}
      View UiTt = UiT.T();
      E.copy(Ui, 1.0, &UiTt, 0.0);
      sbL[k] = Li;
      sbU[k] = Ui;
      FL.sb_linv.push_back(Li.p);
      FL.sb_uinv.push_back(Ui.p);
    }
    std::vector<int> sb_of_row(P.N, 0);
    for (int k = 0; k < nsb; ++k)
      for (int r = P.cl[FL.sb_cluster[k]].begin; r < P.cl[FL.sb_cluster[k]].end; ++r) sb_of_row[r] = k;
    E.phase = 2;
    auto couple = [&](int tcl, int scl, bool lowrank, int id, bool lower, const View& rowsrc) {
      // rowsrc: the block's rows (dense m x n, or U m x kf); scale each part in a solve block
      const Cluster& T = P.cl[tcl];
      const Cluster& Sc = P.cl[scl];
      for (int r = T.begin; r < T.end;) {
        const int k = sb_of_row[r];
        const Cluster& C = P.cl[FL.sb_cluster[k]];
        const int e = std::min(T.end, C.end);
        const bool internal = Sc.begin >= C.begin && Sc.end <= C.end && T.begin >= C.begin && T.end <= C.end;
        if (!internal) {
          const int S = C.end - C.begin, len = e - r;
          const View& inv = lower ? sbL[k] : sbU[k];
          View o = E.new_mat(S, rowsrc.cols, false);
          // a lower (upper) triangular inverse leaves the rows above (below) the
          // source rows zero: only rows [lo, hi) are products, the rest is zero
          const int lo = lower ? r - C.begin : 0, hi = lower ? S : e - C.begin;
          E.gemm(o.sub(lo, 0, hi - lo, rowsrc.cols), 1.0, inv.sub(lo, r - C.begin, hi - lo, len),
                 rowsrc.sub(r - T.begin, 0, len, rowsrc.cols), 0.0);
          if (lo > 0) E.copy(o.sub(0, 0, lo, rowsrc.cols), 0.0, nullptr, 0.0);
          if (hi < S) E.copy(o.sub(hi, 0, S - hi, rowsrc.cols), 0.0, nullptr, 0.0);
          FL.scaled.push_back({lower, lowrank, id, k, o.p, rowsrc.cols, lo, hi});
        }
        r = e;
      }
    };
    for (int d = 0; d < nd; ++d) {
      if (dd[d].r0 == dd[d].c0) continue;
      const Block& Bk = P.bl[P.dense_block[d]];
      couple(Bk.t, Bk.s, false, d, dd[d].r0 > dd[d].c0, H.dense[d]);
    }
    for (int q = 0; q < nl; ++q) {
      const Block& Bk = P.bl[P.lr_block[q]];
      couple(Bk.t, Bk.s, true, q, ld[q].r0 > ld[q].c0, H.lrU(q));
    }
  }
  if (E.status != HM_OK || arena.status != HM_OK) {
    out.err = "H-LU planning failed (device memory or shape)";
    return E.status != HM_OK ? E.status : arena.status;
  }
  out.ops = E.nops;
  for (int i = 0; i < 3; ++i) out.gemm_fma[i] = E.gemm_fma[i];
  E.take_chunk();  // the last slice (streaming only)
  if (std::getenv("HM_CRIT") && !E.sink) {
    // planning diagnostic: the longest dependency path of the op graph under
    // a rough cost model (microseconds: 2 per hand-off, 0.16 k per 32 x 32
    // GEMM tile, 0.3 m per base LU, 0.5 K per truncation) and what it is made of
    const int nops = out.graph.size();
    std::vector<int> kind(nops, -1);
    std::vector<double> cost(nops, 0.0);
    std::vector<std::string> desc(nops);
    for (const Wave& W : out.waves) {
      for (size_t j = 0; j < W.gemm.size(); ++j) {
        const GemmOp& o = W.gemm[j];
        kind[W.gemm_id[j]] = 0;
        cost[W.gemm_id[j]] = 2.0 + 0.16 * o.k * (double)std::min(o.m * o.n, 1024) / 1024.0;
        desc[W.gemm_id[j]] = "gemm " + std::to_string(o.m) + "x" + std::to_string(o.n) + "x" + std::to_string(o.k);
      }
      for (size_t j = 0; j < W.lu.size(); ++j) {
        kind[W.lu_id[j]] = 1;
        cost[W.lu_id[j]] = 2.0 + 0.3 * W.lu[j].m;
        desc[W.lu_id[j]] = "lu " + std::to_string(W.lu[j].m);
      }
      for (size_t j = 0; j < W.trunc.size(); ++j) {
        kind[W.trunc_id[j]] = 2;
        cost[W.trunc_id[j]] = 2.0 + 0.5 * W.trunc[j].K;
        desc[W.trunc_id[j]] = "trunc K" + std::to_string(W.trunc[j].K);
      }
      for (size_t j = 0; j < W.copy.size(); ++j) {
        kind[W.copy_id[j]] = 3;
        cost[W.copy_id[j]] = 2.0;
        desc[W.copy_id[j]] = "copy " + std::to_string(W.copy[j].m) + "x" + std::to_string(W.copy[j].n);
      }
      for (size_t j = 0; j < W.reduce.size(); ++j) {
        kind[W.reduce_id[j]] = 4;
        cost[W.reduce_id[j]] = 2.0;
        desc[W.reduce_id[j]] = "reduce " + std::to_string(W.reduce[j].m) + "x" + std::to_string(W.reduce[j].n) + " p" + std::to_string(W.reduce[j].nparts);
      }
    }
    std::vector<double> fin(nops, 0.0);
    std::vector<int> from(nops, -1);
    int last = 0;
    for (int i = 0; i < nops; ++i) {  // ids are topological (deps < id)
      double st = 0.0;
      for (const int* d = out.graph.begin(i); d != out.graph.end(i); ++d)
        if (fin[*d] > st) { st = fin[*d]; from[i] = *d; }
      fin[i] = st + cost[i];
      if (fin[i] > fin[last]) last = i;
    }
    double kc[5] = {0, 0, 0, 0, 0};
    int kn[5] = {0, 0, 0, 0, 0};
    int len = 0;
    std::map<std::string, std::pair<int, double>> dh;
    for (int i = last; i >= 0; i = from[i]) {
      if (kind[i] >= 0) { kc[kind[i]] += cost[i]; kn[kind[i]]++; }
      auto& e = dh[desc[i]]; e.first++; e.second += cost[i];
      ++len;
    }
    fprintf(stderr, "crit: %d waves, weighted path %.1f ms over %d ops\n", (int)out.waves.size(), fin[last] * 1e-3, len);
    const char* nm[5] = {"gemm", "lu", "trunc", "copy", "reduce"};
    for (int k = 0; k < 5; ++k) fprintf(stderr, "crit:   %-6s %7d ops %9.1f ms\n", nm[k], kn[k], kc[k] * 1e-3);
    std::vector<std::pair<double, std::string>> v;
    for (auto& kv : dh) v.push_back({kv.second.second, kv.first + " x" + std::to_string(kv.second.first)});
    std::sort(v.rbegin(), v.rend());
    for (size_t i = 0; i < v.size() && i < 15; ++i) fprintf(stderr, "crit:     %8.1f ms  %s\n", v[i].first * 1e-3, v[i].second.c_str());
  }
  FactorLayout& F = out.F;
  F.kf = kf;
  (void)F;
  F.d_rank = d_rank_f;
  F.dense = H.dense;
  F.linv.resize(nd, nullptr);
  F.uinv.resize(nd, nullptr);
  F.linv_ld.resize(nd, 0);
  for (int d = 0; d < nd; ++d) {
    if (H.linv[d].p) {
      F.linv[d] = H.linv[d].p;
      F.uinv[d] = H.uinv[d].p;
      F.linv_ld[d] = H.linv[d].rs;
    }
  }
  F.lr_u.resize(nl);
  F.lr_v.resize(nl);
  for (int q = 0; q < nl; ++q) {
    F.lr_u[q] = fin_u[q].p;
    F.lr_v[q] = fin_v[q].p;
  }
  return HM_OK;
}

// ---------------------------------------------------------------- solves
//
// Forward substitution L y = b leaf by leaf (Morton order).  With the leaf
// inverses folded into the factors (P_pj = L_pp^{-1} L_pj, and likewise for
// the rows of low-rank U factors),
//     y_p = L_pp^{-1} b_p - sum_{j < p} P_pj y_j - sum_{q in L, rows(q) > p} (L_pp^{-1} U_q)[p] (V_q' y_s(q)),
// a sum of independent row dot products.  Each source becomes ready when its
// input is final; sources ready two phases early are summed by a
// non-critical task one phase ahead, the rest by the critical task that
// writes y_p.  V_q' y is accumulated as one partial product per leaf of the
// column cluster.  Backward substitution U z = y runs the same way in reverse.

namespace {

struct Src {
  RowSrc s;
  int ready;
  std::vector<int64_t> res;  // resources the source reads
  int row_lo = 0, row_hi = 1 << 30;  // rows (relative to the task rows' start) where M can be nonzero
  int tri = 0;                       // 1: M lower triangular, 2: upper triangular (square, cs == 1)
};

// Stable sort of sources by the phase they are ready in (through an index
// permutation: a source carries a vector, so moving them in merges is slow).
void sort_by_ready(std::vector<Src>& v) {
  std::vector<int> idx(v.size());
  for (size_t i = 0; i < v.size(); ++i) idx[i] = (int)i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return v[a].ready < v[b].ready; });
  std::vector<Src> out;
  out.reserve(v.size());
  for (int i : idx) out.push_back(std::move(v[i]));
  v.swap(out);
}

// Producer tracking on named resources (vector segments, partial products).
struct ResTracker {
  struct Res {
    int wop = -1;
    std::vector<int> rops;
  };
  std::unordered_map<int64_t, Res> res;  // looked up by key only (no ordered walk)
  OpGraph& graph;
  std::vector<int> op_wave;
  std::vector<int> deps;  // scratch
  int bad = 0;
  explicit ResTracker(OpGraph& g) : graph(g) { res.reserve(1 << 16); }
  int add(int wave, const std::vector<int64_t>& reads, const std::vector<int64_t>& writes) {
    deps.clear();
    for (int64_t r : reads) {
      auto it = res.find(r);
      if (it != res.end() && it->second.wop >= 0) deps.push_back(it->second.wop);
    }
    for (int64_t r : writes) {
      Res& R = res[r];
      if (R.wop >= 0) deps.push_back(R.wop);
      deps.insert(deps.end(), R.rops.begin(), R.rops.end());
    }
    std::sort(deps.begin(), deps.end());
    deps.erase(std::unique(deps.begin(), deps.end()), deps.end());
    for (int d : deps)
      if (op_wave[d] >= wave) {
        ++bad;  // producers must sit in earlier waves
        if (getenv("HM_DEBUG_PLAN")) fprintf(stderr, "dep %d (wave %d) of new op in wave %d\n", d, op_wave[d], wave);
      }
    const int id = graph.add_op(deps);
    op_wave.push_back(wave);
    for (int64_t r : reads) res[r].rops.push_back(id);
    for (int64_t r : writes) {
      Res& R = res[r];
      R.wop = id;
      R.rops.clear();
    }
    return id;
  }
};

// y / z / accumulator rows of a leaf are written chunk by chunk (one op per
// chunk of rows); a reader of the leaf depends on every chunk.
int64_t key_y(int sweep, int p, int c = 0) { return (int64_t(1 + sweep) << 40) | (int64_t(p) << 12) | c; }
int64_t key_acc(int sweep, int p, int c = 0) { return (int64_t(7 + sweep) << 44) | (int64_t(p) << 12) | c; }
#ifndef HM_CR_ROWS
#define HM_CR_ROWS 8  // rows per critical row task (build-time tuning parameter)
#endif
#ifndef HM_NC_ROWS
#define HM_NC_ROWS 32  // rows per non-critical row task (build-time tuning parameter)
#endif
constexpr int CR_ROWS = HM_CR_ROWS, NC_ROWS = HM_NC_ROWS;
#ifndef HM_NC_LEAD
#define HM_NC_LEAD 8  // phases by which non-critical row groups precede their block (tuning parameter)
#endif
constexpr int NC_LEAD = HM_NC_LEAD;
std::vector<int64_t> chunk_keys(int64_t base, int nr, int chunk) {
  std::vector<int64_t> k;
  for (int c = 0; c * chunk < nr; ++c) k.push_back(base | c);
  return k;
}
int64_t key_part(int sweep, int q, int seg) { return (int64_t(3 + sweep) << 40) | (int64_t(q) << 16) | seg; }
int64_t key_w(int sweep, int q) { return (int64_t(5 + sweep) << 40) | q; }

class SolvePlanner {
 public:
  SolvePlanner(const Plan& P_, const std::vector<DenseDesc>& dd_, const std::vector<LRDesc>& ld_,
               const FactorLayout& F_, const std::vector<int>* rank_, Arena& A_, std::vector<Wave>& W_,
               std::vector<RowSrc>& S_, OpGraph& G_)
      : P(P_), dd(dd_), ld(ld_), F(F_), rank(rank_), A(A_), waves(W_), srcs(S_), RT(G_) {}
  const Plan& P;
  const std::vector<DenseDesc>& dd;
  const std::vector<LRDesc>& ld;
  const FactorLayout& F;
  const std::vector<int>* rank;
  Arena& A;
  std::vector<Wave>& waves;
  std::vector<RowSrc>& srcs;
  ResTracker RT;
  int status = HM_OK;

  Wave& at(int ph) {
    if ((int)waves.size() <= ph) waves.resize(ph + 1);
    return waves[ph];
  }

  // rows r0 .. r0 + nr - 1 in chunks of `chunk` rows; chunk c writes resource wbase | c
  void emit_rows(int ph, double* out, const double* base, int r0, int nr, int chunk, const std::vector<Src>& list,
                 const std::vector<int64_t>& extra_reads, int64_t wbase) {
    std::vector<int64_t> reads = extra_reads;
    for (const Src& s : list) reads.insert(reads.end(), s.res.begin(), s.res.end());
    if (list.size() > ROWS_MAX_SRC) status = HM_ERR_ARG;  // a row task stages at most this many sources
    // one op for all chunks: its consumers wait on a single counter
    std::vector<int64_t> writes;
    for (int c = 0; c < nr; c += chunk) writes.push_back(wbase | (int64_t)(c / chunk));
    const int id = RT.add(ph, reads, writes);
    for (int c = 0; c < nr; c += chunk) {
      RowsOp o{};
      o.out = out;
      o.base = base;
      o.r0 = r0 + c;
      o.nr = std::min(chunk, nr - c);
      o.src_begin = (int)srcs.size();
      for (const Src& s : list) {
        if (s.row_hi <= c || s.row_lo >= c + o.nr) continue;  // zero rows in this chunk
        RowSrc r = s.s;
        r.M = r.M + (int64_t)c * r.rs;
        if (s.tri == 1) {
          r.ncols = std::min(r.ncols, c + o.nr);  // columns <= the chunk's last row
        } else if (s.tri == 2) {
          r.M += c;                               // columns >= the chunk's first row
          r.x += c;
          r.ncols -= c;
        }
        srcs.push_back(r);
      }
      o.src_end = (int)srcs.size();
      plan_rows_staging(o, srcs.data() + o.src_begin, SOLVE_MODE_LATENCY);
      at(ph).add(o, id);
    }
  }

  // One sweep over the solve blocks; lower = forward with L, otherwise
  // backward with U.  Block k: out_k = Binv_k in_k - sum of scaled couplings.
  void sweep(int sw, bool lower, const double* in, const std::vector<int>& in_ready, double* out, double* acc,
             std::vector<int>& out_ready) {
    const int nb = (int)F.sb_cluster.size();
    const int kf = F.kf;
    std::vector<int> sb_of(P.N, 0);
    for (int k = 0; k < nb; ++k)
      for (int r = P.cl[F.sb_cluster[k]].begin; r < P.cl[F.sb_cluster[k]].end; ++r) sb_of[r] = k;
    auto sbeg = [&](int k) { return P.cl[F.sb_cluster[k]].begin; };
    auto send = [&](int k) { return P.cl[F.sb_cluster[k]].end; };
    // low-rank blocks of this triangle: one partial V_q' y per piece of at most
    // 256 columns inside one solve block; consumers sum the partials
    constexpr int VP_ROWS = 256;
    std::vector<double*> part(ld.size(), nullptr), wfin(ld.size(), nullptr);
    std::vector<int> nparts(ld.size(), 0), w_ready(ld.size(), -1), seen(ld.size(), 0);
    std::vector<std::vector<std::pair<int, int>>> pieces(ld.size());  // (first col, length) per part
    std::vector<std::vector<int>> lr_by_colsb(nb);
    std::vector<bool> used(ld.size(), false);
    auto kq = [&](int q) { return rank ? std::max(0, std::min((*rank)[q], kf)) : kf; };
    for (const FactorLayout::Scaled& s : F.scaled)
      if (s.lowrank && s.lower == lower && kq(s.id) > 0) used[s.id] = true;
    for (size_t q = 0; q < ld.size(); ++q) {
      if (!used[q]) continue;
      const int c0 = ld[q].c0, c1 = ld[q].c0 + ld[q].n;
      for (int r = c0; r < c1;) {
        const int k = sb_of[r], e = std::min(send(k), c1);
        if (lr_by_colsb[k].empty() || lr_by_colsb[k].back() != (int)q) lr_by_colsb[k].push_back((int)q);
        for (int a = r; a < e; a += VP_ROWS) pieces[q].push_back({a, std::min(VP_ROWS, e - a)});
        r = e;
      }
      nparts[q] = (int)pieces[q].size();
      part[q] = A.alloc((int64_t)nparts[q] * kq(q));
      wfin[q] = nparts[q] > 4 ? A.alloc(kq(q)) : nullptr;
      if (!part[q] || (nparts[q] > 4 && !wfin[q])) status = HM_ERR_OOM;
    }
    std::vector<std::vector<const FactorLayout::Scaled*>> by_row(nb);
    for (const FactorLayout::Scaled& s : F.scaled)
      if (s.lower == lower) by_row[s.sb].push_back(&s);
    out_ready.assign(nb, -1);
    for (int it = 0; it < nb; ++it) {
      const int k = lower ? it : nb - 1 - it;
      const int rb = sbeg(k), nr = send(k) - rb;
      std::vector<Src> list;
      {
        Src s{};
        s.s.M = lower ? F.sb_linv[k] : F.sb_uinv[k];
        s.s.rs = nr;
        s.s.cs = 1;
        s.s.x = in + rb;
        s.s.ncols = nr;
        s.s.nparts = 0;
        s.s.sign = 1.0;
        s.ready = in_ready[k];
        s.tri = lower ? 1 : 2;
        if (sw == 1) s.res = chunk_keys(key_y(0, k), nr, CR_ROWS);
        list.push_back(s);
      }
      for (const FactorLayout::Scaled* e : by_row[k]) {
        if (e->lowrank && !used[e->id]) continue;  // rank 0
        Src s{};
        s.s.M = e->M;
        s.s.rs = e->ncols;
        s.s.cs = 1;
        s.s.ncols = e->lowrank ? kq(e->id) : e->ncols;
        s.s.sign = -1.0;
        s.row_lo = e->row_lo;
        s.row_hi = e->row_hi;
        if (e->lowrank) {
          const int q = e->id;
          if (wfin[q]) {  // summed once by a reduction task
            s.s.x = wfin[q];
            s.s.nparts = 1;
            s.res.push_back(key_w(sw, q));
          } else {        // few partials: summed by the consumer
            s.s.x = part[q];
            s.s.nparts = nparts[q];
            for (int sg = 0; sg < nparts[q]; ++sg) s.res.push_back(key_part(sw, q, sg));
          }
          s.ready = w_ready[q];
        } else {
          const int c0 = dd[e->id].c0, j = sb_of[c0];
          s.s.x = out + c0;
          s.s.nparts = 0;
          s.ready = out_ready[j];
          s.res = chunk_keys(key_y(sw, j), send(j) - sbeg(j), CR_ROWS);
        }
        list.push_back(s);
      }
      // sources ready early are summed by a non-critical task placed as soon
      // as they are ready; the critical task adds the late ones
      int latest = -1;
      for (const Src& s : list) latest = std::max(latest, s.ready);
      std::vector<Src> nc, cr;
      for (const Src& s : list) (s.ready < latest - 1 ? nc : cr).push_back(s);
      if ((int)cr.size() > ROWS_MAX_SRC) {
        // the critical task stages a bounded number of sources: the earliest
        // ready of the rest join the non-critical groups
        sort_by_ready(cr);
        const size_t extra = cr.size() - ROWS_MAX_SRC;
        nc.insert(nc.end(), cr.begin(), cr.begin() + extra);
        cr.erase(cr.begin(), cr.begin() + extra);
      }
      int ph;
      if (!nc.empty()) {
        // non-critical sources in groups of at most ROWS_MAX_SRC, chained through
        // per-group accumulators (acc_g = acc_{g-1} + group g)
        sort_by_ready(nc);
        // the first group is the block-inverse product alone when it is ready
        // first, so every block's share of it runs in bulk at the start
        std::vector<std::vector<Src>> groups;
        size_t i0 = 0;
        if (nc.size() > 1 && nc[0].ready < nc[1].ready) groups.push_back({nc[0]}), i0 = 1;
        for (size_t g0 = i0; g0 < nc.size(); g0 += ROWS_MAX_SRC)
          groups.emplace_back(nc.begin() + g0, nc.begin() + std::min(nc.size(), g0 + ROWS_MAX_SRC));
        const double* prev = nullptr;
        int64_t prev_key = -1;
        int phn = 0;
        // the chain reaches this block about two phases after the previous
        // one: the early groups go NC_LEAD phases ahead of that, overlapping the chain
        const int prev_ph = it > 0 ? out_ready[lower ? k - 1 : k + 1] : 0;
        phn = std::max(0, prev_ph - NC_LEAD);
        for (size_t gi = 0; gi < groups.size(); ++gi) {
          const size_t g0 = gi;
          const std::vector<Src>& grp = groups[gi];
          for (const Src& s : grp) phn = std::max(phn, s.ready + 1);
          double* accg = g0 == 0 ? acc : A.alloc(P.N) ;
          if (!accg) { status = HM_ERR_OOM; return; }
          const int64_t gk = key_acc(sw, k) + (int64_t(g0) << 32);
          std::vector<int64_t> rd;
          if (prev) rd = chunk_keys(prev_key, nr, NC_ROWS);
          emit_rows(phn, accg, prev, rb, nr, NC_ROWS, grp, rd, gk);
          prev = accg;
          prev_key = gk;
          ++phn;
        }
        ph = std::max(phn, latest + 1);
        emit_rows(ph, out, prev, rb, nr, CR_ROWS, cr, chunk_keys(prev_key, nr, NC_ROWS), key_y(sw, k));
      } else {
        ph = latest + 1;
        emit_rows(ph, out, nullptr, rb, nr, CR_ROWS, cr, {}, key_y(sw, k));
      }
      out_ready[k] = ph;
      // partial products V_q' y over the pieces of this solve block's columns
      for (int q : lr_by_colsb[k]) {
        for (int sg = 0; sg < nparts[q]; ++sg) {
          const int lo = pieces[q][sg].first, len = pieces[q][sg].second;
          if (lo < rb || lo >= send(k)) continue;
          VPartOp v{};
          v.V = F.lr_v[q] + (lo - ld[q].c0);
          v.ldv = ld[q].n;
          v.y = out + lo;
          v.len = len;
          v.kf = kq(q);
          v.part = part[q] + (int64_t)sg * kq(q);
          int id = RT.add(ph + 1, chunk_keys(key_y(sw, k), nr, CR_ROWS), {key_part(sw, q, sg)});
          at(ph + 1).add(v, id);
          w_ready[q] = std::max(w_ready[q], ph + 1);
          if (++seen[q] == nparts[q] && wfin[q]) {
            ReduceOp o{};
            o.parts = part[q];
            o.dst = wfin[q];
            o.stride = kq(q);
            o.drs = 0;
            o.dcs = 1;
            o.m = 1;
            o.n = kq(q);
            o.nparts = nparts[q];
            o.alpha = 1.0;
            o.beta = 0.0;
            std::vector<int64_t> rd;
            for (int g = 0; g < nparts[q]; ++g) rd.push_back(key_part(sw, q, g));
            int rid = RT.add(w_ready[q] + 1, rd, {key_w(sw, q)});
            at(w_ready[q] + 1).add(o, rid);
            w_ready[q] += 1;
          }
        }
      }
    }
  }
};

}  // namespace

int plan_solve(const Plan& P, const std::vector<DenseDesc>& dd, const std::vector<LRDesc>& ld,
               const FactorLayout& F, const std::vector<int>* rank, const SolveVectors& v, Arena& arena,
               std::vector<Wave>& waves, std::vector<RowSrc>& srcs, OpGraph& graph) {
  SolvePlanner S(P, dd, ld, F, rank, arena, waves, srcs, graph);
  const int nb = (int)F.sb_cluster.size();
  std::vector<int> b_ready(nb, -1), y_ready, z_ready;
  S.sweep(0, true, v.b, b_ready, v.y, v.acc1, y_ready);
  S.sweep(1, false, v.y, y_ready, v.z, v.acc2, z_ready);
  if (S.RT.bad) return HM_ERR_ARG;
  if (S.status != HM_OK || arena.status != HM_OK) return S.status != HM_OK ? S.status : arena.status;
  return HM_OK;
}

}  // namespace hm

namespace hm {

namespace {
struct SpanCheck {
  const std::vector<std::pair<uintptr_t, uintptr_t>>& R;
  const std::vector<RowSrc>* srcs = nullptr;
  int64_t bad = 0;
  std::string first;
  bool inside(const double* p, int64_t lo, int64_t hi) const {
    uintptr_t a = (uintptr_t)(p + lo), b = (uintptr_t)(p + hi) + sizeof(double);
    for (auto& r : R)
      if (a >= r.first && b <= r.second) return true;
    return false;
  }
  // element span of a strided m x n view
  void view(const double* p, int m, int n, int64_t rs, int64_t cs, const char* what) {
    if (m <= 0 || n <= 0) return;
    int64_t lo = 0, hi = 0;
    int64_t a = (int64_t)(m - 1) * rs, b = (int64_t)(n - 1) * cs;
    lo = std::min<int64_t>(0, a) + std::min<int64_t>(0, b);
    hi = std::max<int64_t>(0, a) + std::max<int64_t>(0, b);
    if (!inside(p, lo, hi)) {
      if (bad == 0) first = what;
      ++bad;
    }
  }
};
}  // namespace

int64_t check_spans(const std::vector<Wave>& waves,
                    const std::vector<std::pair<uintptr_t, uintptr_t>>& ranges, std::string& first,
                    const std::vector<RowSrc>* srcs) {
  SpanCheck C{ranges, srcs};
  for (const Wave& w : waves) {
    for (const GemmOp& o : w.gemm) {
      C.view(o.A, o.m, o.k, o.ars, o.acs, "gemm A");
      C.view(o.B, o.k, o.n, o.brs, o.bcs, "gemm B");
      C.view(o.C, o.m, o.n, o.crs, o.ccs, "gemm C");
    }
    for (const LuOp& o : w.lu) {
      C.view(o.A, o.m, o.m, o.lda, 1, "lu A");
      C.view(o.Li, o.m, o.m, o.ldl, 1, "lu Li");
      C.view(o.Ui, o.m, o.m, o.ldu, 1, "lu Ui");
      if (o.m > LU_BASE) { if (C.bad == 0) C.first = "lu size"; ++C.bad; }
    }
    for (const TruncOp& o : w.trunc) {
      C.view(o.GA, o.K, o.K, o.K, 1, "trunc GA");
      C.view(o.GB, o.K, o.K, o.K, 1, "trunc GB");
      C.view(o.TA, o.K, o.kf, o.kf, 1, "trunc TA");
      C.view(o.TB, o.K, o.kf, o.kf, 1, "trunc TB");
      if (o.K > TRUNC_MAXK || o.kf > o.K) { if (C.bad == 0) C.first = "trunc size"; ++C.bad; }
    }
    for (const CopyOp& o : w.copy) {
      if (o.src) C.view(o.src, o.m, o.n, o.srs, o.scs, "copy src");
      C.view(o.dst, o.m, o.n, o.drs, o.dcs, "copy dst");
    }
    for (const ReduceOp& o : w.reduce) {
      C.view(o.parts, o.nparts, o.m * o.n, o.stride, 1, "reduce parts");
      C.view(o.dst, o.m, o.n, o.drs, o.dcs, "reduce dst");
    }
    for (const VPartOp& o : w.vpart) {
      C.view(o.V, o.len, o.kf, 1, o.ldv, "vpart V");
      C.view(o.y, o.len, 1, 1, 0, "vpart y");
      C.view(o.part, o.kf, 1, 1, 0, "vpart part");
    }
    for (const RowsOp& o : w.rows) {
      C.view(o.out + o.r0, o.nr, 1, 1, 0, "rows out");
      if (o.base) C.view(o.base + o.r0, o.nr, 1, 1, 0, "rows base");
      if (C.srcs) {
        for (int k = o.src_begin; k < o.src_end; ++k) {
          const RowSrc& r = (*C.srcs)[k];
          C.view(r.M, o.nr, r.ncols, r.rs, r.cs, "rows src M");
          C.view(r.x, std::max(r.nparts, 1) * r.ncols, 1, 1, 0, "rows src x");
        }
      }
    }
  }
  first = C.first;
  return C.bad;
}

}  // namespace hm
