/*
 * levy_hmat.h -- C ABI of the GB300 (sm_103a) H-matrix Crank-Nicolson solver for
 * convection-diffusion equations driven by a Levy process.
 *
 * Method: Xu & Darve, "Efficient Numerical Method for Models Driven by Levy
 * Process via Hierarchical Matrices" (arXiv 1812.08324).
 *
 *   u_t = a u_xx + b u_x + c u + L u,  L u = int (u(x+y) - u(x) - ...) nu(y) dy
 *                                           (Sec. "Model Problem", Eq. ut)
 *
 * discretised on a uniform interior grid with u = 0 outside the domain into a
 * dense generator G (Eq. Aij with G = -A, trapezoidal jump sum Eq. dl, and the
 * singularity subtraction of Eqs. I1approx-I3approx for singular nu), stored
 * as an H-matrix (App. "H Matrix", Sec. "Construction and Storage"), factored
 * by H-LU (App. "LU Decomposition") and advanced by Crank-Nicolson
 * (Eq. scheme):  (I - dt/2 G) u^{n+1} = (I + dt/2 G) u^n + dt/2 (f^n + f^{n+1}).
 *
 * Conventions for every entry point:
 *   - Return value: HM_OK (0) or a negative HM_ERR_* code.  No exception or
 *     abort crosses the ABI.  hm_error_string() names a code; hm_last_error()
 *     gives the message of the last failure on the calling thread.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls are stream-ordered; device errors found by kernels are reported by
 *     the next call that synchronises (hm_stats, hm_sync) as HM_ERR_DEVICE_ASSERT.
 *   - Vectors exchanged with the caller are device pointers to N doubles in
 *     natural grid order (axis 0 fastest); the caller owns them.  The library
 *     owns the H-matrix and the factors (freed by hm_free / hm_factors_free).
 *   - The library allocates device memory only inside hm_build and hm_factor.
 */
#ifndef LEVY_HMAT_H
#define LEVY_HMAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define HM_OK 0
#define HM_ERR_ARG (-1)            /* invalid argument (sizes, pointers, parameters) */
#define HM_ERR_OOM (-2)            /* device allocation failed */
#define HM_ERR_CUDA (-3)           /* a CUDA runtime call failed */
#define HM_ERR_RANK_CAP (-4)       /* a low-rank block needed more than its rank cap */
#define HM_ERR_NOT_CONVERGED (-5)  /* refinement did not reach refine_tol in refine_max */
#define HM_ERR_TIMEOUT (-6)        /* a bounded device wait gave up */
#define HM_ERR_DEVICE_ASSERT (-7)  /* a kernel found an invalid index or a non-finite value */
#define HM_ERR_NO_DEVICE (-8)      /* no usable CUDA device (or not an sm_103 part) */

/* ---- Levy measure families ---- */
#define HM_NU_GAUSS 0   /* nu(y) = lam * exp(-eps^2 |y|^2)   (Merton jumps, Sec. H-matrix construction) */
#define HM_NU_STABLE 1  /* nu(y) = c_{d,s} / |y|^{d+2s}      (fractional Laplacian, Introduction) */

/* ---- storage precision of what the triangular solves read (HM_FP64 keeps
 * everything FP64).  The mixed modes store the hierarchical inverses of the
 * factors in FP32 or BF16 and multiply with FP32 accumulation; the H-matrix
 * of G, the H-LU factorisation itself (its diagonal-leaf LUs included), the
 * right-hand side and the refinement residual stay FP64, and the accuracy is
 * won back by the FP64 refinement sweeps of every CN solve (refine_max). ---- */
#define HM_FP64 0
#define HM_MIXED_FP32 1
#define HM_MIXED_BF16 2

/* ---- how the triangular solves run ---- */
#define HM_SOLVE_AUTO 0   /* HM_SOLVE_HINV for 1D problems on a box, HM_SOLVE_SUBST otherwise */
#define HM_SOLVE_SUBST 1  /* block forward/backward substitution over solve blocks (dataflow executor) */
#define HM_SOLVE_HINV 2   /* products with hierarchical inverses of the factors (1D problems only) */

/* hm_opts.cn_form: how a Crank-Nicolson step is arranged (Sec. "Crank Nicolson
 * Scheme Based on H-matrix", Eq. scheme: (I - theta G) u^{n+1} = (I + theta G) u^n
 * + theta (f^n + f^{n+1}), theta = dt/2).  Both compute the same scheme.
 *  HM_CN_IDENTITY: since I + theta G = 2I - (I - theta G), the scheme is
 *    (I - theta G) v = w with v = u^n + u^{n+1}, w = 2u^n + theta (f^n + f^{n+1});
 *    v = (LU)^{-1} w, u^{n+1} = v - u^n.  Needs no H-matvec without refinement
 *    sweeps; each sweep refines v against the FP64 H-matvec residual w - Mv.
 *  HM_CN_LITERAL: the right-hand side (I + theta G) u^n + theta (f^n + f^{n+1})
 *    by the H-matvec, u^{n+1} = (LU)^{-1} rhs; sweeps refine u^{n+1}. */
#define HM_CN_IDENTITY 0
#define HM_CN_LITERAL 1

/*
 * Problem (Sec. "Model Problem"; Sec. "Singular and/or Slow Decaying Levy Measure").
 * Interior grid: n[d] points per axis strictly inside [lo[d], hi[d]], spacing
 * h = (hi - lo) / (n + 1), the same on both axes in 2D; u = 0 outside.
 * The jump window is |y| <= LW (1D) or max-norm <= LW (2D); LW must be a
 * whole number of grid steps.  r is the support radius of the subtraction
 * window rho(y) = (1 - (|y|/r)^4)^3 (used only for HM_NU_STABLE).
 * trunc: nu = 0 for |y| > trunc (INFINITY = no truncation).
 */
typedef struct hm_problem {
  int dim;          /* 1 or 2 */
  int n[2];         /* points per axis (n[1] ignored in 1D) */
  double lo[2], hi[2];
  double a;         /* diffusion coefficient a >= 0 (a = sigma^2 / 2) */
  double b[2];      /* drift per axis */
  double c;         /* reaction c <= 0 */
  int kernel;       /* HM_NU_GAUSS or HM_NU_STABLE */
  double s;         /* stable index s in (0, 1) (alpha = 2 s) */
  double eps, lam;  /* Gaussian kernel parameters */
  double trunc;     /* truncation radius of nu */
  double LW;        /* window half-width L_W */
  double r;         /* rho support radius */
  /* Variable-order application (Sec. "Application: Variable-Order Fractional
   * Poisson Equation"); zero for the problems above. */
  int domain;       /* HM_DOMAIN_BOX, or HM_DOMAIN_L (2D): the box minus its closed upper-right
                       quadrant (points with both coordinates >= the box centre are not unknowns) */
  double s_slope;   /* order of the row at x: s(x) = s - s_slope d(x), d = distance from x to the
                       domain boundary; 0 = constant order.  Non-zero needs HM_NU_STABLE, 2D,
                       a = b = c = 0 and untruncated nu. */
} hm_problem;

#define HM_DOMAIN_BOX 0
#define HM_DOMAIN_L 1

/*
 * Options (App. "Construction and Storage": N_min = leaf, eta of Eq. adm;
 * Sec. "Application": eps_1 = aca_tol for construction, eps_2 = lu_tol for the
 * additions inside H-LU).
 */
typedef struct hm_opts {
  int leaf;          /* N_min: clusters with at most leaf points are not split */
  double eta;        /* admissibility min(diam) <= eta * dist */
  double aca_tol;    /* ACA stopping tolerance (relative Frobenius estimate) */
  int max_rank;      /* rank cap of the ACA blocks */
  double lu_tol;     /* relative truncation tolerance of low-rank sums in H-LU */
  int lu_max_rank;   /* rank cap of the low-rank blocks of the factors */
  int precision;     /* HM_FP64, HM_MIXED_FP32 or HM_MIXED_BF16 (the mixed modes need HM_SOLVE_HINV) */
  double refine_tol; /* stop refinement when ||s||_2 <= refine_tol ||rhs||_2 */
  int refine_max;    /* max refinement sweeps per CN step (0 = plain H-LU solve) */
  int solve;         /* HM_SOLVE_AUTO, HM_SOLVE_SUBST or HM_SOLVE_HINV */
  int solve_block;   /* HM_SOLVE_SUBST: rows of the largest solve block (0 = 1024, and 2048 for
                        1D problems of at least 32768 unknowns) */
  double hinv_tol;   /* HM_SOLVE_HINV: relative truncation of the inverse blocks (0 = 1e-2 lu_tol
                        for HM_FP64, 1e-7 for HM_MIXED_FP32, 2e-3 for HM_MIXED_BF16) */
  int cn_form;       /* HM_CN_IDENTITY (default) or HM_CN_LITERAL */
} hm_opts;

typedef struct hm_matrix hm_matrix;    /* opaque: H-matrix of G on the device */
typedef struct hm_factors hm_factors;  /* opaque: H-LU factors of I + theta G */

typedef struct hm_stats_t {
  int64_t n;                  /* unknowns N */
  int clusters, leaves, depth;
  int dense_blocks, lowrank_blocks;
  int64_t dense_entries;      /* entries stored in dense leaves */
  int64_t lowrank_entries;    /* (m + n) * rank summed over low-rank blocks (actual ranks) */
  int64_t h_bytes;            /* bytes of the H-matrix actually read by one H-matvec */
  int64_t lu_bytes;           /* bytes read by one pair of triangular solves: the factors
                                 (HM_SOLVE_SUBST) or their hierarchical inverses (HM_SOLVE_HINV) */
  int max_rank_seen;          /* largest ACA rank */
  int rank_capped_blocks;     /* ACA blocks that stopped at max_rank before aca_tol */
  int lu_max_rank_seen;       /* largest rank in the factors */
  int lu_rank_capped;         /* factor blocks truncated at lu_max_rank before lu_tol */
  int last_refine_iters;      /* refinement sweeps used by the last cn_step */
  double last_refine_resid;   /* ||s|| / ||rhs|| after the last cn_step */
  int64_t device_bytes;       /* device memory held by H (and by F when given) */
  double factor_fma;          /* FP64 FMAs of the factorisation's GEMM tiles (H-LU, solve-block
                                 inverses, scaled couplings; F given) */
  double factor_ms;           /* device time of the factorisation's executor launch (F given;
                                 shared by all problems of one hm_factor_batch) */
  int solve_mode;             /* HM_SOLVE_SUBST or HM_SOLVE_HINV (F given) */
  int hinv_max_rank;          /* largest rank of an inverse block (HM_SOLVE_HINV) */
  int hinv_capped;            /* inverse blocks that reached the rank cap 40 */
  double hinv_ms;             /* host wall time of forming the inverses */
} hm_stats_t;

/* ---- errors ---- */
const char* hm_error_string(int status);
const char* hm_last_error(void);

/*
 * Host-only planning (no GPU needed): the cluster tree (Morton order, binary
 * in 1D / quadtree in 2D, App. "Construction and Storage") and the block tree
 * with the admissibility of Eq. adm, evaluated exactly in integer cell units.
 * Fills n, clusters, leaves, depth, dense_blocks, lowrank_blocks and
 * dense_entries of *info; other fields are zero.
 */
int hm_plan_info(const hm_problem* prob, const hm_opts* opts, hm_stats_t* info);

/*
 * hm_plan_blocks: host-only export of the leaf blocks of the block tree, for
 * checking the admissibility split.  For block b < *count: rows
 * [row0[b], row0[b]+m[b]) and columns [col0[b], col0[b]+ncols[b]) in Morton
 * order, type[b] = 1 (low rank) or 2 (dense).  perm (N ints, may be NULL)
 * receives the natural index of each Morton position.  Arrays are caller
 * owned; *count is in/out (capacity in, blocks out); HM_ERR_ARG if too small.
 */
int hm_plan_blocks(const hm_problem* prob, const hm_opts* opts, int* count, int* row0,
                   int* m, int* col0, int* ncols, int* type, int* perm);

/* Host-only dry run of hm_factor's planning (no GPU needed). */
typedef struct hm_factor_plan_t {
  int64_t fact_ops;      /* dense operations in the H-LU schedule */
  int fact_waves;        /* dependency waves of the H-LU schedule */
  int64_t solve_ops;     /* operations of one forward + backward H-triangular solve */
  int solve_waves;
  int64_t bad_spans;     /* operands outside every allocation (must be 0) */
  int64_t arena_bytes;   /* device bytes the factors and temporaries would take */
  int kf;                /* rank cap of the factors' low-rank blocks */
  double gemm_fma[3];    /* FP64 FMAs of the factor's GEMMs at the rank cap: H-LU proper,
                            solve-block inverses, scaled couplings */
} hm_factor_plan_t;

/*
 * hm_plan_factor: expand the H-LU of I + theta G (App. "LU Decomposition")
 * and the triangular solves into their operation schedules with fake device
 * addresses, assuming every ACA block reaches its rank cap, and check that
 * every operand lies inside an allocation.  Host memory only.
 */
int hm_plan_factor(const hm_problem* prob, const hm_opts* opts, double theta, hm_factor_plan_t* out);

/*
 * hm_build: assemble G as an H-matrix on the current device.
 * Steps (all on the device after the host-side tree): row-independent
 * constants lambda_W, T, kappa (Eqs. dl, I2approx, I3approx) and the table of
 * w nu(|y|) over grid offsets; dense leaves filled entry by entry (Eq. Aij);
 * admissible blocks compressed by partially pivoted ACA to aca_tol or
 * max_rank.  On success *out owns all device memory of the matrix.
 */
int hm_build(const hm_problem* prob, const hm_opts* opts, void* stream, hm_matrix** out);

/*
 * hm_matvec: y = alpha x + beta G x + gamma (w1 + w2)  (the H-matvec of App.
 * "Matrix Vector Multiplication": dense leaves by GEMV, low-rank blocks as
 * U (V' x)).  x, w1, w2 (w1/w2 may be NULL) and y are device vectors of N
 * doubles in natural order; y must not alias x.
 */
int hm_matvec(const hm_matrix* H, double alpha, double beta, const double* x, double gamma,
              const double* w1, const double* w2, double* y, void* stream);

/*
 * hm_matvec_noalloc: the same product as hm_matvec, for callers that must not
 * allocate device memory when they call it -- e.g. a server that admits work
 * against a fixed device-memory budget, or code running where cudaMalloc
 * would synchronise the device or is forbidden by the host application.  It
 * allocates nothing: its scratch (the V'x partial products, the per-block
 * coefficient vectors and, in 2D, Morton-order copies of the vectors) is one
 * fixed library-wide array of 2^21 doubles (16 MiB) in device global memory,
 * which every GPU that loads the library holds until the process exits.
 * H must need at most that much scratch (about N/256 * 3 * depth partials of
 * 128 doubles in 1D); larger problems get HM_ERR_ARG and a message with the
 * size needed.  The first call on a device looks up the array's device address
 * with cudaGetSymbolAddress (that device current) and caches it for the life
 * of the process (threads racing on that first call are safe; the cache
 * assumes the device is not reset while the library is loaded); make that
 * first call before any stream capture.  All calls share the array and it keeps the last
 * call's contents; every entry a call reads is written earlier in the same
 * call, so nothing needs clearing.  Calls that overlap on the GPU (other
 * streams, other threads) race on the array: serialise them.  The paper has
 * no counterpart; this is a library facility.  Arguments as hm_matvec.
 */
int hm_matvec_noalloc(const hm_matrix* H, double alpha, double beta, const double* x, double gamma,
                      const double* w1, const double* w2, double* y, void* stream);

/*
 * hm_to_dense: expand H into a dense N x N row-major device array (natural
 * order), for checks at small N.  out must hold N*N doubles.
 */
int hm_to_dense(const hm_matrix* H, double* out, void* stream);

/*
 * hm_entries: G_{rows[q], cols[q]} for q < count from the device entry
 * generator (natural indices; device arrays).  Evaluates the formula of
 * Eq. Aij with the singular corrections, independent of the compression.
 */
int hm_entries(const hm_matrix* H, int64_t count, const int* rows, const int* cols, double* out,
               void* stream);

/*
 * hm_factor: H-LU factorisation of M = I + theta G (App. "LU Decomposition":
 * LU(A11); L11 U12 = A12; L21 U11 = A21; LU(A22 - L21 U12)), without pivoting
 * (M = I - dt/2 G of Crank-Nicolson is row diagonally dominant).  Low-rank
 * sums are truncated at opts.lu_tol / lu_max_rank.  Crank-Nicolson uses
 * theta = -dt/2.  *out owns its device memory.
 * With HM_SOLVE_HINV (opts.solve; the default for 1D problems) it then forms
 * hierarchical inverses of both factors: for every cluster tau with children
 * a, b the off-diagonal block -X_b L_ba X_a of L^{-1} (and -Y_a U_ab Y_b of
 * U^{-1}) is compressed to rank <= 40 at opts.hinv_tol by a randomised
 * two-sided sketch built from products with the factors and the deeper
 * levels of the inverse only (seeded, deterministic).  The triangular solves
 * are then two fully parallel products; the compression error is corrected by
 * the CN step's FP64 refinement sweeps.  The paper solves by substitution
 * (App. "LU Decomposition"); the inverses are this library's GPU form of it.
 */
int hm_factor(const hm_matrix* H, double theta, void* stream, hm_factors** out);

/*
 * hm_factor_shifted: H-LU of M = alpha I + theta G, the same algorithm as
 * hm_factor (which is alpha = 1).  alpha = 0, theta = 1 factors the generator
 * itself for the variable-order fractional Poisson problem G u = f (Sec.
 * "Application: Variable-Order Fractional Poisson Equation"); -G is an
 * M-matrix there (positive diagonal, non-positive off-diagonal, row sums >= 0),
 * so LU without pivoting applies.  Factors with alpha != 1 are refused by the
 * Crank-Nicolson entry points (HM_ERR_ARG); HM_ERR_ARG for non-finite alpha.
 */
int hm_factor_shifted(const hm_matrix* H, double alpha, double theta, void* stream, hm_factors** out);

/*
 * hm_shifted_solve: x with M x = b, M = alpha I + theta G of F's factors,
 * by Richardson iteration preconditioned with the H-LU:  x_0 = (L U)^{-1} b,
 * x_{k+1} = x_k + (L U)^{-1} (b - M x_k), M applied by the H-matvec of H.
 * F comes from hm_factor / hm_factor_shifted of H or of another H-matrix of
 * the same problem grid (same unknowns, e.g. compressed at a coarser aca_tol:
 * the paper preconditions with the H-LU of a 1e-4 compression, Sec.
 * "Application: Variable-Order Fractional Poisson Equation"); HM_ERR_ARG if
 * the grids differ.  Stops
 * when |b - M x_k| <= tol |b| (2-norms) or after maxit corrections; *iters
 * gets the corrections taken and *resid the last relative residual (either
 * may be NULL).  Natural-order device vectors of N doubles; x must not alias
 * b.  Synchronises the stream once per iteration to test convergence.
 * HM_ERR_NOT_CONVERGED (x holds the last iterate) when tol was not reached.
 */
int hm_shifted_solve(const hm_matrix* H, const hm_factors* F, const double* b, double* x, double tol,
                     int maxit, void* stream, int* iters, double* resid);

/*
 * hm_factor_batch: hm_factor of `count` independent matrices in one
 * persistent launch.  The H-LU operation graphs of all problems are planned
 * on host threads and executed side by side by one dataflow schedule, so small
 * problems share the GPU; out[i] equals hm_factor(H[i], theta[i]) bit for bit
 * (the same operations in the same order of arithmetic).  out has count
 * entries, each owning its device memory; on error all are NULL.  Device-side
 * failures are reported through H[0]'s error word.  The paper has no batched
 * form (it factors one problem at a time).
 */
int hm_factor_batch(const hm_matrix* const* H, const double* theta, int count, void* stream,
                    hm_factors** out);

/*
 * hm_solve: x = (L U)^{-1} b by the H-triangular solves of App. "LU
 * Decomposition": forward then backward substitution over the block tree
 * (HM_SOLVE_SUBST), or x = U^{-1} (L^{-1} b) with the hierarchical inverses
 * (HM_SOLVE_HINV).  Natural-order device vectors; x may alias b.
 */
int hm_solve(const hm_factors* F, const double* b, double* x, void* stream);

/*
 * cn_step: one Crank-Nicolson step (Eq. scheme) with theta = dt/2:
 *   rhs = u_n + theta G u_n + theta (f_n + f_np1)      (H-matvec)
 *   u_np1 = (I - theta G)^{-1} rhs                      (H-LU solve, then
 *   refinement s = rhs - (I - theta G) z, z += (LU)^{-1} s with the H-matvec
 *   residual, the H-LU acting as preconditioner as in Sec. "Solution to the
 *   Model Problem", until ||s|| <= refine_tol ||rhs|| or refine_max sweeps).
 * F must come from hm_factor(H, -dt/2); HM_ERR_ARG otherwise.  f_n / f_np1
 * may be NULL (zero forcing).  u_np1 must not alias u_n.
 */
int cn_step(const hm_matrix* H, const hm_factors* F, double dt, const double* u_n,
            const double* f_n, const double* f_np1, double* u_np1, void* stream);

/*
 * cn_solve: `steps` CN steps starting at level step0; u holds u^{step0} on
 * entry and u^{step0+steps} on return.  f (may be NULL) holds the forcing at
 * levels step0 .. step0+steps as (steps+1) consecutive N-vectors.  Resuming a
 * run = rebuild (deterministic) + cn_solve from the saved level.
 */
int cn_solve(const hm_matrix* H, const hm_factors* F, double dt, int steps, int step0, double* u,
             const double* f, void* stream);

/*
 * cn_solve_batch: `steps` Crank-Nicolson steps without forcing (Eq. scheme)
 * of `count` independent problems sharing dt.  Per step: one batched
 * H-matvec (three launches for all problems), one merged solve schedule (one
 * persistent launch) and batched copies (plus the same per refinement sweep),
 * recorded once as a CUDA graph and replayed `steps` times.  u[i] (device,
 * natural order, N_i doubles) holds problem i's state and is updated in
 * place; the u[i] must not overlap.  Each F[i] must come from
 * hm_factor(H[i], -dt/2) or hm_factor_batch, and all H[i] must share
 * opts.refine_max; HM_ERR_ARG otherwise.  Results equal count separate
 * cn_solve calls bit for bit.
 */
int cn_solve_batch(const hm_matrix* const* H, const hm_factors* const* F, int count, double dt, int steps,
                   double* const* u, void* stream);

/*
 * Persistent batches (continuous batching of independent problems).
 * hm_batch_create: stepping state for `count` problems with their own dt[i]
 * (each F[i] from hm_factor(H[i], -dt[i]/2); distinct matrices and factors;
 * a common opts.refine_max).  It uploads the merged solve schedule and the
 * batched H-matvec tables once and records one step of all problems as a CUDA
 * graph.  The batch borrows H[i] and F[i]: free it before them.
 * hm_batch_step: `steps` CN steps (no forcing) of every problem; u[i] (device,
 * natural order) is read on entry and written on return; results equal
 * separate cn_solve calls bit for bit.  Stream-ordered after `stream`.
 */
typedef struct hm_batch hm_batch;
int hm_batch_create(const hm_matrix* const* H, const hm_factors* const* F, const double* dt, int count,
                    hm_batch** out);
int hm_batch_step(hm_batch* B, double* const* u, int steps, void* stream);
void hm_batch_free(hm_batch* B);

/* 1 if the last batch created replays its step as a CUDA graph, 0 if every
 * step is launched directly (stream capture refused). */
int hm_batch_graphed(void);

/* Number of kernel launches this library has issued in the process so far
 * (every launch helper counts itself; a persistent schedule counts once). */
int64_t hm_launch_count(void);

/* Synchronise the stream and report device-side errors of earlier calls. */
int hm_sync(const hm_matrix* H, void* stream);

/* Statistics (synchronises the stream).  F may be NULL. */
int hm_stats(const hm_matrix* H, const hm_factors* F, hm_stats_t* out);

void hm_free(hm_matrix* H);
void hm_factors_free(hm_factors* F);

#ifdef __cplusplus
}
#endif
#endif /* LEVY_HMAT_H */
