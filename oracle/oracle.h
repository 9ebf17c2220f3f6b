/*
 * CPU oracle for PC-alphaAMG (Hu, Lin, Zikatanov, "An Adaptive Multigrid Method
 * Based on Path Cover", arXiv 1806.07028).
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, single-threaded FP64
 * restatement of the method, written to check the CUDA library against. Only the
 * test-suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Conventions
 *  - A is a weighted graph Laplacian (Section 2.2) in CSR: rowptr[n+1] (int32),
 *    col[nnz] (int32, ascending per row, diagonal stored), val[nnz] (double).
 *  - Levels are numbered from 0 (level 0 is A itself, the paper's A_1).
 *  - Every function returns ORC_OK (0) or a positive error code.
 *  - Host memory only. Arrays passed in are caller-owned; arrays the oracle
 *    allocates are released with orc_free / orc_hier_free.
 *
 * Parity status per part (what pins it) is stated beside each declaration.
 */
#ifndef PCAMG_ORACLE_H
#define PCAMG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ORC_OK = 0, ORC_ERR_INVALID = 1, ORC_ERR_NOT_LAPLACIAN = 2, ORC_ERR_OOM = 3,
    ORC_ERR_ROUND_CAP = 5, ORC_ERR_SINGULAR = 6, ORC_ERR_NOT_CONVERGED = 7,
    ORC_ERR_DIVERGED = 8, ORC_ERR_COARSE_TOO_BIG = 9
};

enum { ORC_P1_E_SCALED = 0, ORC_P1_BOOLEAN = 1 };          /* prolongation at level 0 */
enum { ORC_LEFT_ROUNDS = 0, ORC_LEFT_SEQUENTIAL = 1 };      /* leftover handling (Alg. 3) */
enum { ORC_COVER_LD = 0, ORC_COVER_GREEDY = 1 };            /* path cover (Alg. 1) */
/* Alg. 5 after a re-setup: the smooth error only drives the rebuild (the
 * printed update lands on an iterate that is never used again), or the raw
 * PCG solution is added to the new iterate and the residual recomputed. */
enum { ORC_UPD_REBUILD_ONLY = 0, ORC_UPD_ADD_CORRECTION = 1 };
/* Outer iteration of Alg. 5: the paper's stationary V-cycle iteration, or
 * flexible conjugate gradients preconditioned by the current hierarchy's
 * V-cycle (not in the paper; the re-setup rule is the same, and a re-setup
 * restarts the search direction). */
enum { ORC_OUTER_STATIONARY = 0, ORC_OUTER_FCG = 1 };

typedef struct {
    double tol;           /* relative residual target ||b-Ax||/||b|| */
    int32_t max_iter;     /* V-cycle iterations cap (Alg. 5) */
    double threshold;     /* re-setup when mean ConvR since last setup exceeds it */
    int32_t numW;         /* re-setups that use the W-cycle PCG (Alg. 2) */
    int32_t iterW;        /* PCG iterations with the W-cycle */
    int32_t iterV;        /* PCG iterations with the composite V-cycle */
    int32_t nu_pre;       /* forward multicolour GS sweeps before restriction */
    int32_t nu_post;      /* backward sweeps after prolongation */
    int32_t relax_sweeps; /* sweeps on Au=0 for the random start vector */
    uint64_t seed;        /* start-vector and colouring seed */
    int32_t n_min;        /* stop coarsening at or below this size */
    int32_t max_levels;
    int32_t round_cap;    /* leftover rounds before the sequential tail */
    int32_t p1_mode;      /* ORC_P1_* */
    int32_t leftover_mode;/* ORC_LEFT_* */
    int32_t cover_mode;   /* ORC_COVER_* */
    int32_t dense_max;    /* largest coarsest level solved densely */
    int32_t l1jac_rows;   /* levels >= 1 with at most this many unknowns are smoothed
                             by l1-Jacobi instead of multicolour Gauss-Seidel */
    int32_t update_mode;  /* ORC_UPD_*: what Alg. 5 does with the smooth error */
    int32_t keep_setup;   /* keep each level's reweighted graph after the build (for
                             export); 0 frees it and saves memory on large graphs */
    int32_t init_mwm;     /* 1: the initial hierarchy of Alg. 5 / Alg. 6 is MWM_setup(A)
                             (the paper's); 0: Alg. 4 from the start vector */
    int32_t outer;        /* ORC_OUTER_*: the outer iteration of Alg. 5 */
} orc_params;

typedef struct {
    int32_t iters;        /* V-cycle iterations done */
    int32_t resetups;     /* hierarchies built inside the loop (initial one excluded) */
    int32_t levels;       /* levels of the last hierarchy */
    int32_t status;
    double rel_res;       /* final ||r||/||b|| */
    double oc_mean;       /* operator complexity averaged over all hierarchies */
    int64_t cycles;       /* multigrid cycles applied (V and W, Alg. 5 and Alg. 2) */
    int64_t wcycles;      /* of which W-cycles */
} orc_stats;

void orc_default_params(orc_params* p);
void orc_free(void* p);

/* ---- counter-based random numbers (published definitions) --------------- */
/* Philox4x64 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
/* SplitMix64 output function applied to x (Steele, Lea, Flood 2014; Vigna). */
uint64_t orc_splitmix64(uint64_t x);
/* out[i] = (word_i >> 11) * 2^-52 - 1 in [-1,1), word_i = Philox(ctr=(i/4,0,0,0), key=(seed,0))[i%4] */
void orc_uniform_pm1(uint64_t seed, int64_t n, double* out);

/* ---- level operators -------------------------------------------------------- */
/* r = b - A x, row sums taken left to right in CSR order, one fused
 * multiply-add (single rounding) per entry. */
void orc_residual(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                  const double* x, const double* b, double* r);
/* Jones-Plassmann colouring: priority (splitmix64(seed^i), i), larger wins; a
 * winner takes the smallest colour unused by its already coloured neighbours.
 * Returns the number of colours (>0) or -error. */
int32_t orc_colour(int32_t n, const int32_t* rowptr, const int32_t* col, uint64_t seed,
                   int32_t* colour, int32_t* rounds);
/* Smoother colouring: a connected bipartite graph is coloured by the parity of
 * the breadth-first distance from vertex 0 (two colours); any other graph by
 * orc_colour. Returns the number of colours or -error. */
int32_t orc_colour_smoother(int32_t n, const int32_t* rowptr, const int32_t* col, uint64_t seed,
                            int32_t* colour, int32_t* rounds);
/* One Gauss-Seidel sweep in colour order (forward: colour 0..C-1, backward:
 * C-1..0; rows ascending inside a colour). */
void orc_mcgs_sweep(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                    const int32_t* colour, int32_t ncolour, const double* b, double* x,
                    int32_t forward);
/* One l1-Jacobi sweep: x += (b - A x) / d, d_i = sum_j |a_ij| (row order). */
void orc_l1jac_sweep(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                     const double* b, double* x);
/* One Gauss-Seidel sweep visiting rows in the order perm[0..n-1]. */
void orc_gs_perm_sweep(int32_t n, const int32_t* rowptr, const int32_t* col,
                       const double* val, const int32_t* perm, const double* b, double* x);

/* ---- setup pieces (Alg. 4 step 2, Alg. 1, Alg. 3) --------------------------- */
/* Reweighted A^2 pattern: row u lists v != u with (A^2)_uv structurally nonzero,
 * columns ascending, w_uv = 1/max(|e_u - e_v|, delta), delta = 2^-52 max|e|
 * (delta = 1 when e == 0). Allocates *cptr (n+1), *ccol, *cw. */
int32_t orc_candidates(int32_t n, const int32_t* rowptr, const int32_t* col, const double* e,
                       int32_t** cptr, int32_t** ccol, double** cw);
/* Path cover of the weighted graph (cptr, ccol, cw). nbr0/nbr1 get each vertex's
 * cover neighbours (smaller id in nbr0; -1 where absent).
 * greedy: Alg. 1 over edges in the order (w desc, min id asc, max id asc).
 * ld:     locally-dominant rounds over paths (same result as greedy). */
int32_t orc_cover_greedy(int32_t n, const int32_t* cptr, const int32_t* ccol, const double* cw,
                         int32_t* nbr0, int32_t* nbr1);
int32_t orc_cover_ld(int32_t n, const int32_t* cptr, const int32_t* ccol, const double* cw,
                     int32_t* nbr0, int32_t* nbr1, int32_t* rounds);
/* Path-cover aggregation of one level (Alg. 3) on the weighted graph
 * (tptr, tcol, tw) and cover (nbr0, nbr1). Outputs agg[n] (coarse ids numbered
 * by ascending smallest member), *nc, and the shortened cover cnbr0/cnbr1
 * (first *nc entries used; arrays of length n). */
int32_t orc_aggregate(int32_t n, const int32_t* nbr0, const int32_t* nbr1,
                      const int32_t* tptr, const int32_t* tcol, const double* tw,
                      int32_t round_cap, int32_t leftover_mode,
                      int32_t* agg, int32_t* nc, int32_t* cnbr0, int32_t* cnbr1,
                      int32_t* rounds);
/* Galerkin product B^T A B (pval == NULL: boolean) or P^T A P with P_ui = pval[u]
 * for u in aggregate i. Entry (I,J) is summed left to right over members of I
 * ascending, then row position; each term is (p_u * a_uv) * p_v. drop_diag
 * removes I == J entries. Allocates the output CSR. */
int32_t orc_galerkin(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                     const int32_t* agg, int32_t nc, const double* pval, int32_t drop_diag,
                     int32_t** optr, int32_t** ocol, double** oval, int64_t* onnz);

/* ---- hierarchy (Alg. 4) ------------------------------------------------------ */
typedef struct orc_hier orc_hier;
/* Build the hierarchy from smooth error e (not modified). status in *status. */
orc_hier* orc_build(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                    const double* e, const orc_params* p, int32_t* status);
void orc_hier_free(orc_hier* h);
/* MWM aggregation of one level (Section 2.1) on the weighted adjacency of A
 * (edge weight -a_uv): heaviest-first matching (ld = 0: the sequential greedy
 * over sorted edges; ld = 1: locally-dominant rounds, the same matching, with
 * their count in *rounds), then each unmatched vertex joins the pair of its
 * heaviest neighbour. agg[n] numbered by ascending smallest member. */
int32_t orc_mwm_aggregate(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                          int32_t ld, int32_t* agg, int32_t* nc, int32_t* rounds);
/* MWM_setup (Alg. 5, 6): the hierarchy of MWM aggregations with boolean P on
 * every level (UA-AMG), Galerkin coarse matrices, same stopping rules. */
orc_hier* orc_build_mwm(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                        const orc_params* p, int32_t* status);
int32_t orc_hier_nlevels(const orc_hier* h);
/* sizes[0]=n, [1]=nnz, [2]=nc (0 at the coarsest), [3]=ncolour, [4]=cover rounds,
 * [5]=leftover rounds, [6]=pinned (coarsest), [7]=candidate nnz (level 0). */
void orc_hier_sizes(const orc_hier* h, int32_t lev, int64_t sizes[8]);
/* Copy out one level. Any pointer may be NULL. agg/pval are absent at the
 * coarsest level; pval is absent above level 0 and in boolean mode. */
void orc_hier_export(const orc_hier* h, int32_t lev, int32_t* agg, int32_t* nbr0,
                     int32_t* nbr1, int32_t* rowptr, int32_t* col, double* val,
                     double* pval, int32_t* colour);
/* Level-0 reweighted candidates (CSR, column order). */
void orc_hier_export_candidates(const orc_hier* h, int32_t* cptr, int32_t* ccol, double* cw);
double orc_hier_oc(const orc_hier* h);
/* c = one V-cycle (or W-cycle, gamma=2) correction for A c = r from c = 0. */
void orc_vcycle(const orc_hier* h, const double* r, double* c);
void orc_wcycle(const orc_hier* h, const double* r, double* c);
/* x = pseudo-inverse of the coarsest matrix applied to r (pinned Cholesky). */
void orc_coarse_solve(const orc_hier* h, const double* r, double* x);

/* ---- driver (Alg. 2, Alg. 5, Alg. 6) ---------------------------------------- */
/* Relaxed random start: uniform(seed), relax_sweeps forward MCGS sweeps on Au=0,
 * mean removed, unit 2-norm. */
int32_t orc_start_vector(int32_t n, const int32_t* rowptr, const int32_t* col,
                         const double* val, const orc_params* p, double* e);
/* Alg. 2: flexible PCG on A e = r from e = 0, W-cycle on the newest hierarchy
 * when re <= numW, else the composite V-cycle over hist[0..re-1]. */
int32_t orc_smooth_error(int32_t n, const int32_t* rowptr, const int32_t* col,
                         const double* val, const double* r, orc_hier* const* hist,
                         int32_t re, const orc_params* p, double* e_raw);
/* The preconditioner that Alg. 2's PCG applies: z = W-cycle of hist[re-1] when
 * re <= numW, else the symmetric composite of V-cycles over hist[0..re-1]. */
void orc_precond(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                 orc_hier* const* hist, int32_t re, const orc_params* p, const double* r,
                 double* z);
/* Alg. 5 (general b). x is the initial guess on entry and the solution on exit.
 * e0: start vector (NULL: relaxed random start). res_hist (may be NULL) gets
 * ||r_k||/||b|| for k = 0..iters; rebuilt (may be NULL, same capacity) gets 1 at
 * step k when a re-setup followed the k-th V-cycle, else 0. */
int32_t orc_solve(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                  const double* b, double* x, const orc_params* p, const double* e0,
                  orc_stats* st, double* res_hist, int32_t res_hist_cap, int32_t* rebuilt);
/* Several right-hand sides (B, X column-major n x k), each column by the outer
 * iteration of Alg. 5 without re-setup (p->outer), preconditioned by Alg. 2's
 * composite product of V-cycles over hist[0..re-1]. iters, rel_res: k entries
 * each (may be NULL). */
int32_t orc_solve_multi(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                        int32_t k, const double* B, double* X, const orc_params* p,
                        orc_hier* const* hist, int32_t re, int32_t* iters, double* rel_res);
/* Alg. 6 (b = 0): the iterate itself becomes the smooth error. */
int32_t orc_solve_zero_rhs(int32_t n, const int32_t* rowptr, const int32_t* col,
                           const double* val, double* x, const orc_params* p,
                           const double* e0, orc_stats* st, double* res_hist,
                           int32_t res_hist_cap);

#ifdef __cplusplus
}
#endif
#endif
