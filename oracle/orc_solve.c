/*
 * CPU oracle, part 3: cycles (Section 3, V- and W-cycle with Gauss-Seidel),
 * smooth-error estimate (Alg. 2), and the adaptive drivers (Alg. 5, Alg. 6).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include "orc_internal.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static double vsum(int32_t n, const double* x) {
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i) s += x[i];
    return s;
}

static double vdot(int32_t n, const double* x, const double* y) {
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i) s += x[i] * y[i];
    return s;
}

static double vnorm(int32_t n, const double* x) { return sqrt(vdot(n, x, x)); }

static void remove_mean(int32_t n, double* x) {
    double m = vsum(n, x) / (double)n;
    for (int32_t i = 0; i < n; ++i) x[i] -= m;
}

void orc_coarse_solve(const orc_hier* h, const double* r, double* x) {
    int32_t m = h->nL;
    for (int32_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int32_t j = 0; j < m; ++j) s += h->Xinv[(size_t)i * m + j] * r[j];
        x[i] = s;
    }
}

/* One multigrid cycle on level l for A_l x = b (x holds the start value):
 * nu_pre forward colour-ordered Gauss-Seidel sweeps, residual, restriction by
 * P_l^T, gamma coarse cycles from zero, prolongation x += P_l x_c, nu_post
 * backward sweeps. The coarsest level is solved directly. */
static void cycle(const orc_hier* h, int32_t l, const double* b, double* x, int32_t gamma) {
    if (l == h->nlev - 1) { orc_coarse_solve(h, b, x); return; }
    const orc_level* L = &h->lev[l];
    for (int32_t s = 0; s < h->nu_pre; ++s) {
        if (L->jac) orc_l1jac_sweep(L->n, L->rowptr, L->col, L->val, b, x);
        else orc_mcgs_sweep(L->n, L->rowptr, L->col, L->val, L->colour, L->ncolour, b, x, 1);
    }
    double* r = (double*)orc_xmalloc(sizeof(double) * (size_t)L->n);
    double* bc = (double*)orc_xmalloc(sizeof(double) * (size_t)L->nc);
    double* xc = (double*)calloc((size_t)L->nc, sizeof(double));
    orc_residual(L->n, L->rowptr, L->col, L->val, x, b, r);
    for (int32_t I = 0; I < L->nc; ++I) {
        double s = 0.0;
        for (int32_t t = L->agg_ptr[I]; t < L->agg_ptr[I + 1]; ++t) {
            int32_t u = L->agg_mem[t];
            s += L->pval ? L->pval[u] * r[u] : r[u];
        }
        bc[I] = s;
    }
    for (int32_t g = 0; g < gamma; ++g) cycle(h, l + 1, bc, xc, gamma);
    for (int32_t u = 0; u < L->n; ++u)
        x[u] += L->pval ? L->pval[u] * xc[L->agg[u]] : xc[L->agg[u]];
    for (int32_t s = 0; s < h->nu_post; ++s) {
        if (L->jac) orc_l1jac_sweep(L->n, L->rowptr, L->col, L->val, b, x);
        else orc_mcgs_sweep(L->n, L->rowptr, L->col, L->val, L->colour, L->ncolour, b, x, 0);
    }
    free(r); free(bc); free(xc);
}

/* cycles applied since the library was loaded (the oracle is single-threaded) */
static int64_t g_vcycles = 0, g_wcycles = 0;

void orc_vcycle(const orc_hier* h, const double* r, double* c) {
    ++g_vcycles;
    memset(c, 0, sizeof(double) * (size_t)h->lev[0].n);
    cycle(h, 0, r, c, 1);
}

void orc_wcycle(const orc_hier* h, const double* r, double* c) {
    ++g_wcycles;
    memset(c, 0, sizeof(double) * (size_t)h->lev[0].n);
    cycle(h, 0, r, c, 2);
}

int32_t orc_start_vector(int32_t n, const int32_t* rowptr, const int32_t* col,
                         const double* val, const orc_params* p, double* e) {
    orc_uniform_pm1(p->seed, n, e);
    int32_t* colour = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n);
    double* zero = (double*)calloc((size_t)n, sizeof(double));
    if (!colour || !zero) { free(colour); free(zero); return ORC_ERR_OOM; }
    int32_t nc = orc_colour_smoother(n, rowptr, col, p->seed, colour, NULL);
    for (int32_t s = 0; s < p->relax_sweeps; ++s)
        orc_mcgs_sweep(n, rowptr, col, val, colour, nc, zero, e, 1);
    remove_mean(n, e);
    double nr = vnorm(n, e);
    if (nr > 0.0) for (int32_t i = 0; i < n; ++i) e[i] /= nr;
    free(colour); free(zero);
    return ORC_OK;
}

/* Preconditioner of Alg. 2: a W-cycle on the newest hierarchy while
 * re <= numW, else the symmetric composite product over all hierarchies
 * built so far, applied as z += B_j (r - A z) for j = 1..re, re..1. */
static void precond(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                    orc_hier* const* hist, int32_t re, const orc_params* p,
                    const double* r, double* z, double* t1, double* t2) {
    if (re <= p->numW) { orc_wcycle(hist[re - 1], r, z); return; }
    memset(z, 0, sizeof(double) * (size_t)n);
    for (int32_t s = 0; s < 2 * re; ++s) {
        int32_t j = (s < re) ? s : 2 * re - 1 - s;
        orc_residual(n, rowptr, col, val, z, r, t1);
        orc_vcycle(hist[j], t1, t2);
        for (int32_t i = 0; i < n; ++i) z[i] += t2[i];
    }
}

void orc_precond(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                 orc_hier* const* hist, int32_t re, const orc_params* p, const double* r,
                 double* z) {
    double* t1 = (double*)orc_xmalloc(sizeof(double) * (size_t)n);
    double* t2 = (double*)orc_xmalloc(sizeof(double) * (size_t)n);
    precond(n, rowptr, col, val, hist, re, p, r, z, t1, t2);
    free(t1); free(t2);
}

/* Several right-hand sides of one operator, column by column: the outer
 * iteration of Alg. 5 (stationary x += z, or flexible CG with the same
 * Polak-Ribiere update as orc_solve) without re-setup, z the symmetric
 * composite product of V-cycles over hist[0..re-1] (Alg. 2's preconditioner
 * with every hierarchy given, applied as z += B_j (r - A z) for j = 1..re,
 * re..1 from z = 0). B, X column-major n x k; X holds the initial guesses and
 * receives the solutions. */
int32_t orc_solve_multi(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                        int32_t k, const double* B, double* X, const orc_params* p,
                        orc_hier* const* hist, int32_t re, int32_t* iters, double* rel_res) {
    if (k < 1 || re < 1) return ORC_ERR_INVALID;
    orc_params q = *p;
    q.numW = 0;   /* the composite product for every re */
    double *r = (double*)orc_xmalloc(sizeof(double) * (size_t)n),
           *z = (double*)orc_xmalloc(sizeof(double) * (size_t)n),
           *t1 = (double*)orc_xmalloc(sizeof(double) * (size_t)n),
           *t2 = (double*)orc_xmalloc(sizeof(double) * (size_t)n),
           *fp = (double*)orc_xmalloc(sizeof(double) * (size_t)n),
           *fq = (double*)orc_xmalloc(sizeof(double) * (size_t)n),
           *frold = (double*)orc_xmalloc(sizeof(double) * (size_t)n),
           *fzold = (double*)orc_xmalloc(sizeof(double) * (size_t)n),
           *fzero = (double*)calloc((size_t)n, sizeof(double));
    int32_t status = ORC_OK;
    if (!r || !z || !t1 || !t2 || !fp || !fq || !frold || !fzold || !fzero) { status = ORC_ERR_OOM; goto out; }
    for (int32_t c = 0; c < k; ++c) {
        const double* b = B + (size_t)c * n;
        double* x = X + (size_t)c * n;
        for (int32_t i = 0; i < n; ++i) if (!isfinite(b[i]) || !isfinite(x[i])) { status = ORC_ERR_INVALID; goto out; }
        const double bn = vnorm(n, b);
        if (!(bn > 0.0)) { status = ORC_ERR_INVALID; goto out; }
        remove_mean(n, x);
        orc_residual(n, rowptr, col, val, x, b, r);
        double res = vnorm(n, r);
        int32_t it = 0, restart = 1;
        while (it < p->max_iter && res / bn > p->tol) {
            precond(n, rowptr, col, val, hist, re, &q, r, z, t1, t2);
            if (p->outer == ORC_OUTER_FCG) {
                double rz = vdot(n, r, z);
                if (restart) {
                    memcpy(fp, z, sizeof(double) * (size_t)n);
                    restart = 0;
                } else {
                    double num = 0.0, den = vdot(n, fzold, frold);
                    for (int32_t i = 0; i < n; ++i) num += z[i] * (r[i] - frold[i]);
                    double beta = (den != 0.0) ? num / den : 0.0;
                    for (int32_t i = 0; i < n; ++i) fp[i] = z[i] + beta * fp[i];
                }
                orc_residual(n, rowptr, col, val, fp, fzero, fq);   /* fq = -A p */
                double pq = -vdot(n, fp, fq);
                double alpha = (pq > 0.0 && rz > 0.0) ? rz / pq : 0.0;
                for (int32_t i = 0; i < n; ++i) x[i] += alpha * fp[i];
                memcpy(frold, r, sizeof(double) * (size_t)n);
                memcpy(fzold, z, sizeof(double) * (size_t)n);
            } else {
                for (int32_t i = 0; i < n; ++i) x[i] += z[i];
            }
            remove_mean(n, x);
            orc_residual(n, rowptr, col, val, x, b, r);
            double nres = vnorm(n, r);
            ++it;
            if (!isfinite(nres)) { status = ORC_ERR_DIVERGED; res = nres; break; }
            res = nres;
        }
        if (iters) iters[c] = it;
        if (rel_res) rel_res[c] = res / bn;
        if (status == ORC_OK && !(res / bn <= p->tol)) status = ORC_ERR_NOT_CONVERGED;
    }
out:
    free(r); free(z); free(t1); free(t2); free(fp); free(fq); free(frold); free(fzold); free(fzero);
    return status;
}

/* Alg. 2: flexible (Polak-Ribiere) PCG on A e = r from e = 0. */
int32_t orc_smooth_error(int32_t n, const int32_t* rowptr, const int32_t* col,
                         const double* val, const double* rhs, orc_hier* const* hist,
                         int32_t re, const orc_params* p, double* e) {
    int32_t iters = (re <= p->numW) ? p->iterW : p->iterV;
    double *r = (double*)orc_xmalloc(sizeof(double) * (size_t)n),
           *rold = (double*)orc_xmalloc(sizeof(double) * (size_t)n),
           *z = (double*)orc_xmalloc(sizeof(double) * (size_t)n),
           *pp = (double*)orc_xmalloc(sizeof(double) * (size_t)n),
           *q = (double*)orc_xmalloc(sizeof(double) * (size_t)n),
           *t1 = (double*)orc_xmalloc(sizeof(double) * (size_t)n),
           *t2 = (double*)orc_xmalloc(sizeof(double) * (size_t)n),
           *zero = (double*)calloc((size_t)n, sizeof(double));
    if (!r || !rold || !z || !pp || !q || !t1 || !t2 || !zero) {
        free(r); free(rold); free(z); free(pp); free(q); free(t1); free(t2); free(zero);
        return ORC_ERR_OOM;
    }
    memset(e, 0, sizeof(double) * (size_t)n);
    memcpy(r, rhs, sizeof(double) * (size_t)n);
    precond(n, rowptr, col, val, hist, re, p, r, z, t1, t2);
    memcpy(pp, z, sizeof(double) * (size_t)n);
    double rz = vdot(n, r, z);
    for (int32_t it = 1; it <= iters; ++it) {
        /* q = A p */
        orc_residual(n, rowptr, col, val, pp, zero, q);
        for (int32_t i = 0; i < n; ++i) q[i] = -q[i];
        double pq = vdot(n, pp, q);
        if (!(pq > 0.0) || !(rz > 0.0)) break;
        double alpha = rz / pq;
        for (int32_t i = 0; i < n; ++i) e[i] += alpha * pp[i];
        memcpy(rold, r, sizeof(double) * (size_t)n);
        for (int32_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
        if (it == iters) break;
        precond(n, rowptr, col, val, hist, re, p, r, z, t1, t2);
        double num = 0.0;
        for (int32_t i = 0; i < n; ++i) num += z[i] * (r[i] - rold[i]);
        double beta = num / rz;
        rz = vdot(n, r, z);
        for (int32_t i = 0; i < n; ++i) pp[i] = z[i] + beta * pp[i];
    }
    free(r); free(rold); free(z); free(pp); free(q); free(t1); free(t2); free(zero);
    return ORC_OK;
}

#define ORC_MAX_HIST 4096

int32_t orc_solve(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                  const double* b, double* x, const orc_params* p, const double* e0,
                  orc_stats* stt, double* res_hist, int32_t cap, int32_t* rebuilt) {
    orc_stats st;
    memset(&st, 0, sizeof(st));
    const int64_t v0 = g_vcycles, w0 = g_wcycles;
    for (int32_t i = 0; i < n; ++i) if (!isfinite(b[i]) || !isfinite(x[i])) return ORC_ERR_INVALID;
    double bn = vnorm(n, b);
    if (!(bn > 0.0)) return ORC_ERR_INVALID;
    orc_hier** hist = (orc_hier**)calloc(ORC_MAX_HIST, sizeof(orc_hier*));
    double *r = (double*)orc_xmalloc(sizeof(double) * (size_t)n),
           *c = (double*)orc_xmalloc(sizeof(double) * (size_t)n),
           *e = (double*)orc_xmalloc(sizeof(double) * (size_t)n);
    int32_t status = ORC_OK, re = 0;
    double oc_sum = 0.0;
    if (!hist || !r || !c || !e) { status = ORC_ERR_OOM; goto out; }
    remove_mean(n, x);
    orc_residual(n, rowptr, col, val, x, b, r);
    double res = vnorm(n, r);
    if (p->init_mwm) {
        hist[0] = orc_build_mwm(n, rowptr, col, val, p, &status);
    } else {
        if (e0) memcpy(e, e0, sizeof(double) * (size_t)n);
        else if ((status = orc_start_vector(n, rowptr, col, val, p, e))) goto out;
        hist[0] = orc_build(n, rowptr, col, val, e, p, &status);
    }
    if (!hist[0]) goto out;
    re = 1;
    oc_sum += orc_hier_oc(hist[0]);
    int32_t k = 0;
    double wsum = 0.0;
    int32_t wcnt = 0;
    if (res_hist && cap > 0) res_hist[0] = res / bn;
    if (rebuilt) for (int32_t i = 0; i < cap; ++i) rebuilt[i] = 0;
    /* flexible CG state (outer = FCG): direction, A times it, previous r and z */
    double *fp = NULL, *fq = NULL, *frold = NULL, *fzold = NULL, *fzero = NULL;
    int32_t restart = 1;
    if (p->outer == ORC_OUTER_FCG) {
        fp = (double*)orc_xmalloc(sizeof(double) * (size_t)n);
        fq = (double*)orc_xmalloc(sizeof(double) * (size_t)n);
        frold = (double*)orc_xmalloc(sizeof(double) * (size_t)n);
        fzold = (double*)orc_xmalloc(sizeof(double) * (size_t)n);
        fzero = (double*)calloc((size_t)n, sizeof(double));
        if (!fp || !fq || !frold || !fzold || !fzero) { status = ORC_ERR_OOM; goto fcg_out; }
    }
    while (k < p->max_iter && res / bn > p->tol) {
        /* z = V-cycle on the current hierarchy */
        orc_vcycle(hist[re - 1], r, c);
        if (p->outer == ORC_OUTER_FCG) {
            /* flexible CG: p = z + beta p (Polak-Ribiere beta; restart after a
             * re-setup), x += alpha p, alpha = r.z / p.Ap */
            double rz = vdot(n, r, c);
            if (restart) {
                memcpy(fp, c, sizeof(double) * (size_t)n);
                restart = 0;
            } else {
                double num = 0.0, den = vdot(n, fzold, frold);
                for (int32_t i = 0; i < n; ++i) num += c[i] * (r[i] - frold[i]);
                double beta = (den != 0.0) ? num / den : 0.0;
                for (int32_t i = 0; i < n; ++i) fp[i] = c[i] + beta * fp[i];
            }
            orc_residual(n, rowptr, col, val, fp, fzero, fq);   /* fq = -A p */
            double pq = -vdot(n, fp, fq);
            double alpha = (pq > 0.0 && rz > 0.0) ? rz / pq : 0.0;
            for (int32_t i = 0; i < n; ++i) x[i] += alpha * fp[i];
            memcpy(frold, r, sizeof(double) * (size_t)n);
            memcpy(fzold, c, sizeof(double) * (size_t)n);
        } else {
            /* x_{k+1} = x_k + V-cycle correction */
            for (int32_t i = 0; i < n; ++i) x[i] += c[i];
        }
        remove_mean(n, x);
        orc_residual(n, rowptr, col, val, x, b, r);
        double nres = vnorm(n, r);
        if (!isfinite(nres)) { status = ORC_ERR_DIVERGED; break; }
        wsum += nres / res; ++wcnt;
        res = nres;
        ++k;
        if (res_hist && k < cap) res_hist[k] = res / bn;
        if (res / bn <= p->tol) break;
        if (wsum / (double)wcnt > p->threshold && re < ORC_MAX_HIST) {
            /* re-setup: Alg. 2 smooth error, Alg. 4 hierarchy, then x += e */
            if ((status = orc_smooth_error(n, rowptr, col, val, r, hist, re, p, e))) break;
            double* eh = c;
            memcpy(eh, e, sizeof(double) * (size_t)n);
            remove_mean(n, eh);
            double en = vnorm(n, eh);
            if (en > 0.0) for (int32_t i = 0; i < n; ++i) eh[i] /= en;
            hist[re] = orc_build(n, rowptr, col, val, eh, p, &status);
            if (!hist[re]) break;
            oc_sum += orc_hier_oc(hist[re]);
            ++re;
            if (rebuilt && k < cap) rebuilt[k] = 1;
            restart = 1;
            if (p->update_mode == ORC_UPD_ADD_CORRECTION) {
                for (int32_t i = 0; i < n; ++i) x[i] += e[i];
                remove_mean(n, x);
                orc_residual(n, rowptr, col, val, x, b, r);
                res = vnorm(n, r);
                if (res_hist && k < cap) res_hist[k] = res / bn;
            }
            wsum = 0.0; wcnt = 0;
        }
    }
    st.iters = k;
    st.rel_res = res / bn;
    if (status == ORC_OK && !(st.rel_res <= p->tol)) status = ORC_ERR_NOT_CONVERGED;
fcg_out:
    free(fp); free(fq); free(frold); free(fzold); free(fzero);
out:
    st.resetups = re > 0 ? re - 1 : 0;
    st.levels = re > 0 && hist[re - 1] ? hist[re - 1]->nlev : 0;
    st.oc_mean = re > 0 ? oc_sum / (double)re : 0.0;
    st.status = status;
    st.cycles = (g_vcycles - v0) + (g_wcycles - w0);
    st.wcycles = g_wcycles - w0;
    if (stt) *stt = st;
    if (hist) for (int32_t j = 0; j < ORC_MAX_HIST; ++j) orc_hier_free(hist[j]);
    free(hist); free(r); free(c); free(e);
    return status;
}

int32_t orc_solve_zero_rhs(int32_t n, const int32_t* rowptr, const int32_t* col,
                           const double* val, double* x, const orc_params* p,
                           const double* e0, orc_stats* stt, double* res_hist, int32_t cap) {
    orc_stats st;
    memset(&st, 0, sizeof(st));
    const int64_t v0 = g_vcycles;
    double *r = (double*)orc_xmalloc(sizeof(double) * (size_t)n),
           *c = (double*)orc_xmalloc(sizeof(double) * (size_t)n),
           *zero = (double*)calloc((size_t)n, sizeof(double)),
           *e = (double*)orc_xmalloc(sizeof(double) * (size_t)n);
    orc_hier* h = NULL;
    int32_t status = ORC_OK, builds = 0;
    double oc_sum = 0.0;
    if (!r || !c || !zero || !e) { status = ORC_ERR_OOM; goto out; }
    remove_mean(n, x);
    orc_residual(n, rowptr, col, val, x, zero, r);
    double r0 = vnorm(n, r), res = r0;
    if (!(r0 > 0.0)) { status = ORC_OK; goto out; }
    if (p->init_mwm) {
        h = orc_build_mwm(n, rowptr, col, val, p, &status);
    } else {
        if (e0) memcpy(e, e0, sizeof(double) * (size_t)n);
        else if ((status = orc_start_vector(n, rowptr, col, val, p, e))) goto out;
        h = orc_build(n, rowptr, col, val, e, p, &status);
    }
    if (!h) goto out;
    builds = 1; oc_sum += orc_hier_oc(h);
    int32_t k = 0;
    if (res_hist && cap > 0) res_hist[0] = 1.0;
    while (k < p->max_iter && res / r0 > p->tol) {
        orc_vcycle(h, r, c);
        for (int32_t i = 0; i < n; ++i) x[i] += c[i];
        remove_mean(n, x);
        orc_residual(n, rowptr, col, val, x, zero, r);
        double nres = vnorm(n, r);
        if (!isfinite(nres)) { status = ORC_ERR_DIVERGED; break; }
        double conv = nres / res;
        res = nres;
        ++k;
        if (res_hist && k < cap) res_hist[k] = res / r0;
        if (res / r0 <= p->tol) break;
        if (conv > p->threshold) {
            /* the exact error is the iterate itself: e = x / ||x|| */
            double xn = vnorm(n, x);
            for (int32_t i = 0; i < n; ++i) e[i] = x[i] / xn;
            orc_hier_free(h);
            h = orc_build(n, rowptr, col, val, e, p, &status);
            if (!h) break;
            ++builds; oc_sum += orc_hier_oc(h);
        }
    }
    st.iters = k;
    st.rel_res = res / r0;
    if (status == ORC_OK && !(st.rel_res <= p->tol)) status = ORC_ERR_NOT_CONVERGED;
out:
    st.resetups = builds > 0 ? builds - 1 : 0;
    st.levels = h ? h->nlev : 0;
    st.oc_mean = builds > 0 ? oc_sum / (double)builds : 0.0;
    st.status = status;
    st.cycles = g_vcycles - v0;
    if (stt) *stt = st;
    orc_hier_free(h);
    free(r); free(c); free(zero); free(e);
    return status;
}
