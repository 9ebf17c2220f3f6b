/*
 * pcamg.h -- C ABI of the GB300 (sm_103a) PC-alphaAMG library.
 *
 * PC-alphaAMG is the path-cover adaptive unsmoothed-aggregation algebraic
 * multigrid method of Hu, Lin and Zikatanov, "An Adaptive Multigrid Method
 * Based on Path Cover" (arXiv 1806.07028), for weighted graph Laplacians.
 * Every step runs as a CUDA kernel of this library on one GPU.
 *
 * General rules
 *  - Matrices are graph Laplacians (Section 2.2): CSR with int32 row pointers
 *    and column indices (columns ascending in each row, diagonal stored) and
 *    float64 values; symmetric, off-diagonals <= 0, zero row sums (up to
 *    rounding), positive diagonal, connected graph.
 *  - Pointers named d_* are device pointers, h_* host pointers. Inputs are
 *    borrowed for the duration of the call only: the library copies what it
 *    keeps. Outputs are caller-owned buffers the library writes.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). A handle runs
 *    its device work on a private non-blocking stream that each call orders
 *    after the caller's prior work on `stream` and before the caller's later
 *    work on it (event record/wait), so results are ready for `stream` when a
 *    call returns. Calls synchronise where they must read sizes or scalars
 *    back, and before they return results in host memory.
 *  - Every call returns a pcamg_status; nothing is thrown across the ABI and the
 *    library never exits or traps. pcamg_last_error(h) gives a message.
 *  - A handle is not thread safe: use one handle from one host thread at a time.
 */
#ifndef PCAMG_H
#define PCAMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define PCAMG_API __attribute__((visibility("default")))
#else
#define PCAMG_API
#endif

typedef struct pcamg_ctx* pcamg_handle;

typedef enum {
    PCAMG_OK = 0,
    PCAMG_ERR_INVALID = 1,        /* bad argument or malformed CSR / vector */
    PCAMG_ERR_NOT_LAPLACIAN = 2,  /* asymmetric, positive off-diagonal, row sum, ... */
    PCAMG_ERR_OOM = 3,            /* device allocation failed */
    PCAMG_ERR_CUDA = 4,           /* a CUDA runtime call or launch failed */
    PCAMG_ERR_ROUND_CAP = 5,      /* an iterative setup round hit its cap */
    PCAMG_ERR_SINGULAR = 6,       /* reserved, not returned: a coarsest-level pivot at or
                                     below 1e-12 of the largest diagonal entry is pinned
                                     (its row and column replaced by the identity), so the
                                     dense factorisation does not break down */
    PCAMG_ERR_NOT_CONVERGED = 7,  /* max_iter reached before tol (stats are filled) */
    PCAMG_ERR_DIVERGED = 8,       /* NaN/Inf residual */
    PCAMG_ERR_COARSE_TOO_BIG = 9, /* coarsening stalled above dense_max */
    PCAMG_ERR_UNSUPPORTED = 10    /* feature not available in this build */
} pcamg_status;

enum { PCAMG_FP64 = 0, PCAMG_FP32_IR = 1 };                 /* precision */
/* How pcamg_setup builds the first hierarchy: by Alg. 4 from a start vector
 * (RANDOM: the relaxed random vector; USER: d_e0; LEARNED: the network's
 * output), or by MWM_setup (Section 2.1: heaviest-first matching of each
 * level's weighted adjacency, unmatched vertices joined to the pair of their
 * heaviest neighbour, boolean prolongations -- the paper's initial hierarchy
 * of Alg. 5 and 6, and with a threshold no factor reaches, its plain UA-AMG
 * comparator). */
enum { PCAMG_START_RANDOM = 0, PCAMG_START_USER = 1, PCAMG_START_LEARNED = 2, PCAMG_START_MWM = 3 };

/* A start-vector network (see the pcamg_mpnn_* calls below). */
typedef struct pcamg_mpnn_s* pcamg_mpnn;
enum { PCAMG_P1_E_SCALED = 0, PCAMG_P1_BOOLEAN = 1 };       /* level-1 prolongation */
/* Alg. 5 after a re-setup. REBUILD_ONLY (default): the smooth error only drives
 * the new hierarchy; the iterate and its residual are left as the V-cycle made
 * them, so the next convergence factor is measured against that residual (the
 * printed update adds e to an iterate that is never used again; this reading
 * gives the paper's Re = Iter - 1 for Alg. 5(1) and its Re counts for Alg. 5(2)).
 * ADD_CORRECTION: the raw PCG solution of A e = r is added to the iterate and
 * the residual recomputed before the next step. */
enum { PCAMG_UPD_REBUILD_ONLY = 0, PCAMG_UPD_ADD_CORRECTION = 1 };
/* Outer iteration of pcamg_solve. STATIONARY (default): Alg. 5 as the paper
 * gives it, x <- x + V r. FCG: flexible conjugate gradients (Polak-Ribiere)
 * preconditioned by the current hierarchy's V-cycle, x <- x + alpha p; the
 * re-setup rule is Alg. 5's, and a re-setup restarts the search direction.
 * The paper uses plain V-cycles; FCG is this library's addition. */
enum { PCAMG_OUTER_STATIONARY = 0, PCAMG_OUTER_FCG = 1 };

/* Parameters. Defaults (pcamg_default_params) follow Section 4 of the paper:
 * threshold 0.4 (Alg. 5(2)), numW 2, iterW 7, iterV 4, Gauss-Seidel smoothing,
 * V-cycle, tol 1e-8. */
typedef struct {
    double tol;            /* stop when ||b - A x||_2 / ||b||_2 <= tol */
    int32_t max_iter;      /* cap on V-cycle iterations */
    double threshold;      /* re-setup when the mean convergence factor since the
                              last setup exceeds it (Alg. 5) */
    int32_t numW;          /* re-setups whose smooth error uses W-cycle PCG (Alg. 2) */
    int32_t iterW;         /* PCG iterations with the W-cycle */
    int32_t iterV;         /* PCG iterations with the composite V-cycle */
    int32_t nu_pre;        /* forward multicolour Gauss-Seidel sweeps per level */
    int32_t nu_post;       /* backward sweeps per level */
    int32_t relax_sweeps;  /* sweeps on A u = 0 that smooth the random start */
    uint64_t seed;         /* start vector and colouring priorities */
    int32_t n_min;         /* stop coarsening at or below this many unknowns */
    int32_t max_levels;    /* at most this many levels (<= 32) */
    int32_t round_cap;     /* leftover rounds before the sequential tail (Alg. 3) */
    int32_t p1_mode;       /* PCAMG_P1_*: level-1 prolongation carries e or is boolean */
    int32_t precision;     /* PCAMG_FP64 or PCAMG_FP32_IR */
    int32_t start;         /* PCAMG_START_RANDOM, PCAMG_START_USER (d_e0 given) or
                              PCAMG_START_LEARNED (the network `mpnn` maps the relaxed
                              random start and the graph's degrees to the start vector) */
    int32_t dense_max;     /* largest coarsest level factorised densely (<= 4096) */
    int32_t use_graphs;    /* capture each cycle in a CUDA graph and replay it */
    int32_t keep_setup;    /* keep covers and reweighted graphs for export */
    int32_t profile;       /* bit 0: time the FP64 fine-level residual of Alg. 5 with CUDA
                              events; bit 1: time the finest-level pre-smoothing sweep and
                              residual inside every V-cycle (event-record nodes in the
                              cycle graph) */
    int32_t tail_rows;     /* levels with at most this many unknowns (the finest level: at
                              most half as many) run inside one thread-block cluster per
                              cycle visit, or as their dense operator (0 = never) */
    int32_t l1jac_rows;    /* coarse levels (not the finest) with at most this many
                              unknowns are smoothed by l1-Jacobi, x += (b - A x)/d with
                              d_i = sum_j |a_ij|, instead of multicolour Gauss-Seidel */
    int32_t tail_dense;    /* bit 0: V-cycles, bit 1: W-cycles (default 3: both). For the selected cycle
                              kinds the levels below tail_rows are applied as their
                              dense linear operator N (formed once per hierarchy, on
                              first use: one visit of those levels from a zero start is
                              x = N b, later visits x += N (b - A x); a W-cycle's two
                              visits from the level above are one operator and one
                              product), instead of recursing through them. Same result up to rounding; used
                              when the tail has two or more levels and its vectors fit
                              one block's shared memory, else the recursion runs. */
    int32_t max_resetups;  /* pcamg_solve builds at most this many new hierarchies and
                              stops (PCAMG_ERR_NOT_CONVERGED) right after the last one,
                              or instead of one more; -1 = no limit. Used to collect
                              the first smooth error of a run (training data). */
    pcamg_mpnn mpnn;       /* the network for PCAMG_START_LEARNED, else NULL */
    int32_t update_mode;   /* PCAMG_UPD_*: what Alg. 5 does with the Alg. 2 smooth error
                              after a re-setup (default PCAMG_UPD_REBUILD_ONLY) */
    int32_t max_cover_rounds; /* cap on the path-cover rounds of one build (0: n + 1, which
                              always suffices: every round adds at least one edge); a build
                              that needs more returns PCAMG_ERR_ROUND_CAP */
    int32_t outer;         /* PCAMG_OUTER_*: stationary Alg. 5 (default) or flexible CG */
} pcamg_params;

typedef struct {
    int32_t iters;         /* V-cycle iterations done */
    int32_t resetups;      /* hierarchies built inside the solve (initial one excluded) */
    int32_t levels;        /* levels of the current hierarchy */
    int32_t status;        /* pcamg_status of the solve */
    double rel_res;        /* final ||b - A x|| / ||b|| (FP64, on the device) */
    double oc_mean;        /* operator complexity averaged over all hierarchies */
    double t_setup_ms;     /* host wall time inside re-setups (Alg. 2 + Alg. 4) */
    double t_solve_ms;     /* host wall time of the whole call */
    double t_alg2_ms;      /* of t_setup_ms: smooth-error PCG (Alg. 2) */
    double t_alg4_ms;      /* of t_setup_ms: hierarchy builds (Alg. 4) */
    int64_t cycles;        /* multigrid cycles applied (V and W, all hierarchies) */
    double* res_hist;      /* optional host buffer: ||r_k||/||b||, k = 0..iters */
    int32_t res_hist_cap;  /* its capacity (0 = none) */
    int32_t res_hist_len;  /* entries written */
    /* fine-level residual kernel timing (params.profile != 0) */
    int64_t prof_launches;
    double prof_ms;        /* summed CUDA-event time of those launches */
    double prof_bytes;     /* their algorithmic bytes: 12 nnz + 28 n each */
    int32_t* rebuilt;      /* optional host buffer of res_hist_cap entries: 1 at step k
                              when a new hierarchy was built after the k-th V-cycle, else 0 */
    int64_t wcycles;       /* of cycles: W-cycles */
    /* finest-level residual inside every V-cycle (params.profile bit 1), timed with
       CUDA events on the handle's stream (event-record nodes in the cycle graph) */
    int64_t cyc_launches;
    double cyc_ms;         /* summed event time of those launches */
    double cyc_bytes;      /* their algorithmic bytes: (4 + w) nnz + (4 + 3 w) n each,
                              w = 4 (FP32_IR) or 8 (FP64) */
    /* the finest level's pre-smoothing sweep of every V-cycle (all colours of the
       Gauss-Seidel sweep), timed the same way (params.profile bit 1) */
    int64_t gs_sweeps;
    double gs_ms;          /* summed event time of those sweeps */
    double gs_bytes;       /* their algorithmic bytes, (4 + w) nnz + (4 + 3 w) n each: A,
                              b, x written, and every x gathered once by the other colours */
} pcamg_stats;

/* Fill p with the defaults above. */
PCAMG_API pcamg_status pcamg_default_params(pcamg_params* p);

/* ---- device memory --------------------------------------------------------
 * Every device buffer the library allocates (handles, hierarchies, work
 * vectors, networks, the partial sums of pcamg_residual) is allocated and freed
 * in stream order on the stream the work runs on. By default the memory comes
 * from a memory pool the library creates per device, which keeps freed memory
 * cached for reuse (pcamg_trim_memory returns it to the device).
 * pcamg_set_allocator installs caller callbacks instead -- for instance a
 * framework's caching allocator, so that the library and the framework share
 * one pool: alloc(bytes, stream, ctx) returns device memory of the current
 * device usable in stream order on `stream` (a cudaStream_t; NULL = legacy
 * default stream), or NULL on failure (reported as PCAMG_ERR_OOM);
 * free(ptr, stream, ctx) releases it, ordered after the work queued on
 * `stream`. A handle or network keeps the allocator that was installed when it
 * was created and frees through it, so the callbacks and ctx must stay valid
 * until it is destroyed. alloc == free == NULL restores the library pool; one
 * of them NULL alone is PCAMG_ERR_INVALID. Process wide; do not call it while
 * another thread is inside the library. The paper has no counterpart. */
typedef void* (*pcamg_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*pcamg_free_fn)(void* ptr, void* stream, void* ctx);
PCAMG_API pcamg_status pcamg_set_allocator(pcamg_alloc_fn alloc, pcamg_free_fn free, void* ctx);
/* Return the memory the library pool of the current device holds unused. */
PCAMG_API pcamg_status pcamg_trim_memory(void);

/* Create a handle for A and build the first hierarchy (Alg. 5 setup, with the
 * initial hierarchy built by Alg. 4 from a start vector instead of MWM).
 * n >= 2, nnz = d_rowptr[n]. d_e0: start vector (device, length n) when
 * p->start == PCAMG_START_USER, else NULL: the relaxed random start is used
 * (uniform Philox4x64-10 numbers, relax_sweeps forward Gauss-Seidel sweeps on
 * A u = 0, mean removed, unit 2-norm). The CSR is validated first; on error no
 * handle is returned (*out = NULL). */
PCAMG_API pcamg_status pcamg_setup(pcamg_handle* out, const pcamg_params* p, int32_t n,
                                   int64_t nnz, const int32_t* d_rowptr, const int32_t* d_col,
                                   const double* d_val, const double* d_e0, void* stream);

/* PathCoverAMG_setup (Alg. 4) from the smooth error d_e (device, length n, used
 * as given; the solver itself passes the Alg. 2 output made orthogonal to 1 and
 * normalised, and P_1 carries e): reweighting on the A^2 pattern,
 * path cover (Alg. 1), path-cover aggregation (Alg. 3) and Galerkin products on
 * every level. The new hierarchy becomes the current one and joins the history
 * used by the composite preconditioner (Alg. 2). */
PCAMG_API pcamg_status pcamg_adapt(pcamg_handle h, const double* d_e);

/* AdaptiveAMG for general b (Alg. 5): V-cycles on the current hierarchy, x kept
 * orthogonal to 1, re-setup through Alg. 2 + Alg. 4 when the mean convergence
 * factor since the last setup exceeds threshold. d_b (length n, sum zero) and
 * d_x (initial guess in, solution out) are device pointers. st may be NULL. */
PCAMG_API pcamg_status pcamg_solve(pcamg_handle h, const double* d_b, double* d_x,
                                   pcamg_stats* st);

/* AdaptiveAMG for b = 0 (Alg. 6): the iterate itself is the smooth error;
 * rebuild when one step's convergence factor exceeds threshold. d_x holds the
 * initial guess and receives the last iterate. The stopping test is relative
 * to the first residual. */
PCAMG_API pcamg_status pcamg_solve_zero_rhs(pcamg_handle h, double* d_x, pcamg_stats* st);

/* Several right-hand sides at once: A X = B for k columns. Adaptivity is per
 * operator, so no column builds a hierarchy: every column runs the outer
 * iteration of Alg. 5 without re-setup -- stationary (x += z) or flexible CG
 * (params.outer), the column's residual and stopping test in FP64 as in
 * pcamg_solve -- with z = M r, M Alg. 2's symmetric composite product of
 * V-cycles over every hierarchy the handle holds (those pcamg_setup,
 * pcamg_adapt and earlier solves built; z += B_j (r - A z) for j = 1..Re,
 * Re..1 from z = 0). The cycles of up to 8 columns run together: every pass
 * over a level's matrix serves all of them (the level's vectors
 * row-interleaved, K = 2, 4 or 8 per pass); a batch of one column runs the
 * single-vector cycles of pcamg_solve. A column agrees with the same
 * iteration on that column alone to rounding (the batched row sums take the
 * sub-warp order).
 * d_B, d_X: device, column-major n x k (column c at offset c*n); d_X holds the
 * initial guesses and receives the solutions (each with zero mean). iters,
 * rel_res: optional host arrays of k entries (V-cycles done, final
 * ||b - A x|| / ||b|| per column). Returns PCAMG_OK when every column reached
 * params.tol, PCAMG_ERR_NOT_CONVERGED when one stopped at params.max_iter,
 * PCAMG_ERR_DIVERGED on a non-finite residual, PCAMG_ERR_INVALID for k < 1 or
 * a zero or non-finite column of B. */
PCAMG_API pcamg_status pcamg_solve_multi(pcamg_handle h, int32_t k, const double* d_B, double* d_X,
                                         int32_t* iters, double* rel_res);

/* End-to-end call on HOST buffers: copies A, b, x to the device, runs
 * pcamg_setup + pcamg_solve, copies x back, frees everything. */
PCAMG_API pcamg_status pcamg_solve_host(const pcamg_params* p, int32_t n, int64_t nnz,
                                        const int32_t* h_rowptr, const int32_t* h_col,
                                        const double* h_val, const double* h_b, double* h_x,
                                        pcamg_stats* st, void* stream);

/* One multigrid cycle (gamma = 1: V-cycle, 2: W-cycle) of hierarchy `hist`
 * (0 = first built) as a correction: d_c = B d_r from a zero start, in the
 * handle's precision (FP32_IR: r is scaled by ||r||_2 and cast to float, the
 * correction is scaled back). Section 4: Gauss-Seidel pre- (forward colour
 * order) and post- (backward) smoothing, restriction by P^T, prolongation by P,
 * pinned dense solve on the coarsest level. */
PCAMG_API pcamg_status pcamg_cycle(pcamg_handle h, int32_t hist, int32_t gamma,
                                   const double* d_r, double* d_c);

/* ApproximateSmoothError (Alg. 2) for residual d_r with the handle's current
 * history: flexible PCG on A e = r from e = 0, preconditioned by a W-cycle on the
 * newest hierarchy while the history holds <= numW hierarchies, else by the
 * symmetric composite of V-cycles over all of them. Writes the raw PCG iterate. */
PCAMG_API pcamg_status pcamg_smooth_error(pcamg_handle h, const double* d_r, double* d_e);

/* The relaxed random start vector of this handle's parameters (device out). */
PCAMG_API pcamg_status pcamg_start_vector(pcamg_handle h, double* d_e);

/* Inspection. hist: 0-based hierarchy index; lev: 0-based level (0 = A).
 * sizes[0]=n, [1]=nnz, [2]=nc (0 at the coarsest), [3]=colours, [4]=cover
 * rounds (level 0), [5]=leftover rounds, [6]=pinned unknowns (coarsest),
 * [7]=reweighted-graph nnz of this level (needs keep_setup). */
PCAMG_API int32_t pcamg_num_hierarchies(pcamg_handle h);
PCAMG_API int32_t pcamg_num_levels(pcamg_handle h, int32_t hist);
PCAMG_API pcamg_status pcamg_level_sizes(pcamg_handle h, int32_t hist, int32_t lev,
                                         int64_t sizes[8]);
/* Copy one level to HOST buffers (any may be NULL): agg[n] coarse aggregate of
 * each unknown (absent at the coarsest), nbr0/nbr1[n] its path-cover neighbours
 * (smaller id first, -1 = none; needs keep_setup), the level matrix CSR,
 * pval[n] the level-1 prolongation values (e-scaled mode, level 0 only),
 * colour[n] smoother colours. */
PCAMG_API pcamg_status pcamg_export_level(pcamg_handle h, int32_t hist, int32_t lev,
                                          int32_t* agg, int32_t* nbr0, int32_t* nbr1,
                                          int32_t* rowptr, int32_t* col, double* val,
                                          double* pval, int32_t* colour);
/* The reweighted graph of one level (level 0: the A^2 pattern with weights
 * 1/max(|e_i - e_j|, 2^-52 max|e|), Alg. 4 step 2) as host CSR; needs keep_setup. */
PCAMG_API pcamg_status pcamg_export_reweighted(pcamg_handle h, int32_t hist, int32_t lev,
                                               int32_t* ptr, int32_t* col, double* w);

/* Number of CUDA kernels this library has launched in this process so far (a
 * replayed cycle graph counts the kernels it holds). */
PCAMG_API int64_t pcamg_kernel_launches(void);

PCAMG_API const char* pcamg_last_error(pcamg_handle h);
PCAMG_API const char* pcamg_status_string(pcamg_status s);
PCAMG_API void pcamg_destroy(pcamg_handle h);

/* The normalised smooth error (zero mean, unit 2-norm) from which the newest
 * hierarchy of h was built (the start vector after pcamg_setup, the Alg. 2
 * output after a re-setup). d_e: device, length n. */
PCAMG_API pcamg_status pcamg_last_smooth_error(pcamg_handle h, double* d_e);

/* ---- learned start vector ------------------------------------------------
 * The paper has no learned component; this network is the library's own. It
 * maps per-vertex features -- the relaxed random start u (times sqrt(n)), log
 * degree and log weighted degree D_i = sum_{j != i} |a_ij| (both minus their
 * means over the vertices) -- through an input layer (3 -> 64), four
 * message-passing layers h' = C(GELU(W_l [h ; m] + b_l)) with the weighted
 * neighbour mean m_i = sum_{j != i} |a_ij| h_j / D_i (128 -> 64), C removing
 * every channel's mean over the vertices, and a linear output (64 -> 1) to y;
 * the start vector is (y - mean y) / ||y - mean y||. Weights are applied
 * rounded to bfloat16, the layer products on the tensor cores with FP32
 * accumulation. Training minimises, per vertex over its A^2 candidate pairs,
 * the cross-entropy between the softmax of -|e_i - e_j|/tau_i of a target
 * smooth error e and that of the prediction (tau_i: standard deviation of
 * |e_i - e_j| over the pairs), with Adam on FP32 master weights.
 * Parameters: a flat FP32 vector of pcamg_mpnn_num_params() entries in the
 * order W_in (64x3 row-major), b_in, then per layer W_l (64x128 row-major,
 * columns 0-63 act on h, 64-127 on m) and b_l, then w_out (64), b_out (1).
 * All calls are synchronous; the network owns its device memory. */
PCAMG_API int64_t pcamg_mpnn_num_params(void);
/* New network with the given host parameters (Adam state zero). */
PCAMG_API pcamg_status pcamg_mpnn_create(pcamg_mpnn* out, const float* h_params);
PCAMG_API void pcamg_mpnn_destroy(pcamg_mpnn m);
PCAMG_API pcamg_status pcamg_mpnn_get_params(pcamg_mpnn m, float* h_params);
/* Replace the parameters and reset the Adam state. */
PCAMG_API pcamg_status pcamg_mpnn_set_params(pcamg_mpnn m, const float* h_params);
/* The gradient of the last pcamg_mpnn_loss_grad call (host, num_params). */
PCAMG_API pcamg_status pcamg_mpnn_get_grad(pcamg_mpnn m, float* h_grad);
/* The network's start vector on the graph of g: d_u is the relaxed random
 * start (pcamg_start_vector), d_y receives the output (device, length n). */
PCAMG_API pcamg_status pcamg_mpnn_forward(pcamg_mpnn m, pcamg_handle g, const double* d_u, double* d_y);
/* Loss against the target smooth error d_target (device, zero mean, unit norm)
 * into *h_loss, and its gradient kept in the network for pcamg_mpnn_adam_step. */
PCAMG_API pcamg_status pcamg_mpnn_loss_grad(pcamg_mpnn m, pcamg_handle g, const double* d_u,
                                            const double* d_target, double* h_loss);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) with learning rate lr. */
PCAMG_API pcamg_status pcamg_mpnn_adam_step(pcamg_mpnn m, float lr);
/* Save / load: one JSON header line, then the FP32 parameters, little-endian. */
PCAMG_API pcamg_status pcamg_mpnn_save(pcamg_mpnn m, const char* path);
PCAMG_API pcamg_status pcamg_mpnn_load(pcamg_mpnn* out, const char* path);

/* ---- single kernels, for measurement and parity tests -------------------- */
/* r = b - A x (FP64), optionally ||r||_2^2 into *d_norm2 (device scalar, may be
 * NULL). The fine-level residual of Alg. 5. Allocates a small device buffer of
 * per-block partial sums when d_norm2 is given. */
PCAMG_API pcamg_status pcamg_residual(int32_t n, const int32_t* d_rowptr, const int32_t* d_col,
                                      const double* d_val, const double* d_x, const double* d_b,
                                      double* d_r, double* d_norm2, void* stream);
/* The same residual and ||r||_2^2 WITHOUT any device allocation. The paper has
 * no counterpart: this is for callers that cannot allocate device memory --
 * e.g. a time-critical loop that may not pay for cudaMalloc/cudaFree (they can
 * synchronise the device), or a process whose device memory is all handed out
 * by its own pool. The per-block partial sums live in one fixed device array of
 * 65536 doubles (512 KB) that every GPU which loads the library holds until the
 * process exits, so n <= 67,108,864 rows (larger n: PCAMG_ERR_INVALID). d_norm2
 * is required. The first call on a device looks up that array's device address
 * (with the device current) and caches it for the life of the process (the
 * device's primary context must not be reset in between); make that first call
 * before any stream capture. A call reads nothing back and does not
 * synchronise: it returns once its two kernels are queued on `stream`. All
 * calls share the array: calls whose work overlaps on the GPU (other streams,
 * other host threads) race on it and must be serialised by the caller. Each
 * call overwrites every entry it reads, so no clearing is needed. Errors:
 * pcamg_last_error(NULL). */
PCAMG_API pcamg_status pcamg_residual_noalloc(int32_t n, const int32_t* d_rowptr,
                                              const int32_t* d_col, const double* d_val,
                                              const double* d_x, const double* d_b, double* d_r,
                                              double* d_norm2, void* stream);
/* Same in FP32 (values, x, b, r float). */
PCAMG_API pcamg_status pcamg_residual_f32(int32_t n, const int32_t* d_rowptr,
                                          const int32_t* d_col, const float* d_val,
                                          const float* d_x, const float* d_b, float* d_r,
                                          void* stream);
/* d_out[i] = (w_i >> 11) 2^-52 - 1, w_i = word i%4 of Philox4x64-10 with counter
 * (i/4, 0, 0, 0) and key (seed, 0). */
PCAMG_API pcamg_status pcamg_uniform(uint64_t seed, int64_t n, double* d_out, void* stream);
/* Jones-Plassmann colouring of the pattern (rowptr, col): priority
 * (splitmix64(seed ^ i), i), a round winner takes the smallest colour unused by
 * its coloured neighbours. Writes d_colour[n]; *ncolour on the host. */
PCAMG_API pcamg_status pcamg_colour(int32_t n, const int32_t* d_rowptr, const int32_t* d_col,
                                    uint64_t seed, int32_t* d_colour, int32_t* ncolour,
                                    void* stream);

#ifdef __cplusplus
}
#endif
#endif
