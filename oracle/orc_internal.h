/* CPU oracle internals. TEST INFRASTRUCTURE ONLY (see oracle.h). */
#ifndef PCAMG_ORC_INTERNAL_H
#define PCAMG_ORC_INTERNAL_H
#include <stddef.h>
#include "oracle.h"

#define ORC_MAX_LEVELS 64

typedef struct {
    int32_t n;
    int64_t nnz;
    int32_t *rowptr, *col;   /* A_l (level 0: a private copy of A) */
    double* val;
    int32_t ncolour;
    int32_t* colour;
    int32_t jac;             /* smoothed by l1-Jacobi (no colouring) */
    /* reweighted graph of this level (level 0: candidates on the A^2 pattern) */
    int32_t *tptr, *tcol;
    double* tw;
    int32_t *nbr0, *nbr1;    /* path cover of this level */
    /* transfer to the next level (absent at the coarsest) */
    int32_t nc;
    int32_t* agg;
    int32_t *agg_ptr, *agg_mem;  /* members of each aggregate, ascending */
    double* pval;                /* level 0 in e-scaled mode only */
    int32_t cover_rounds, leftover_rounds;
} orc_level;

struct orc_hier {
    int32_t nlev;
    orc_level lev[ORC_MAX_LEVELS];
    int32_t nL;
    double* Xinv;      /* nL x nL pinned pseudo-inverse of the coarsest matrix */
    int32_t npinned;
    int32_t nu_pre, nu_post;
    int64_t cand_nnz;
};

void* orc_xmalloc(size_t bytes);
int32_t orc_dense_pinned_inverse(int32_t m, const double* Adense, int32_t force_last,
                                 double tau, double* X, int32_t* npinned);

#endif
