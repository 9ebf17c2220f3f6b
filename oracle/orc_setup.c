/*
 * CPU oracle, part 2: the setup of one hierarchy (Alg. 4) and its pieces:
 * reweighting on the A^2 pattern (Alg. 4 step 2), path cover (Alg. 1),
 * path-cover aggregation (Alg. 3), prolongation (Section 3.3), Galerkin
 * products and path shortening (Alg. 4 steps 6-8).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include "orc_internal.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

int32_t orc_candidates(int32_t n, const int32_t* rowptr, const int32_t* col, const double* e,
                       int32_t** cptr_out, int32_t** ccol_out, double** cw_out) {
    int32_t* stamp = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n);
    int32_t* cptr = (int32_t*)orc_xmalloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!stamp || !cptr) { free(stamp); free(cptr); return ORC_ERR_OOM; }
    for (int32_t i = 0; i < n; ++i) stamp[i] = -1;
    int64_t total = 0;
    cptr[0] = 0;
    for (int32_t u = 0; u < n; ++u) {
        int64_t cnt = 0;
        for (int32_t k = rowptr[u]; k < rowptr[u + 1]; ++k) {
            int32_t j = col[k];
            for (int32_t kk = rowptr[j]; kk < rowptr[j + 1]; ++kk) {
                int32_t v = col[kk];
                if (v != u && stamp[v] != u) { stamp[v] = u; ++cnt; }
            }
        }
        total += cnt;
        if (total >= 2147483647LL) { free(stamp); free(cptr); return ORC_ERR_INVALID; }
        cptr[u + 1] = (int32_t)total;
    }
    int32_t* ccol = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)total);
    double* cw = (double*)orc_xmalloc(sizeof(double) * (size_t)total);
    if (!ccol || !cw) { free(stamp); free(cptr); free(ccol); free(cw); return ORC_ERR_OOM; }
    double emax = 0.0;
    for (int32_t i = 0; i < n; ++i) if (fabs(e[i]) > emax) emax = fabs(e[i]);
    double delta = ldexp(emax, -52);
    if (delta == 0.0) delta = 1.0;
    for (int32_t i = 0; i < n; ++i) stamp[i] = -1;
    for (int32_t u = 0; u < n; ++u) {
        int32_t p = cptr[u];
        for (int32_t k = rowptr[u]; k < rowptr[u + 1]; ++k) {
            int32_t j = col[k];
            for (int32_t kk = rowptr[j]; kk < rowptr[j + 1]; ++kk) {
                int32_t v = col[kk];
                if (v != u && stamp[v] != u) { stamp[v] = u; ccol[p++] = v; }
            }
        }
        qsort(ccol + cptr[u], (size_t)(cptr[u + 1] - cptr[u]), sizeof(int32_t), cmp_i32);
        for (int32_t k = cptr[u]; k < cptr[u + 1]; ++k) {
            double d = fabs(e[u] - e[ccol[k]]);
            if (d < delta) d = delta;
            cw[k] = 1.0 / d;
        }
    }
    free(stamp);
    *cptr_out = cptr; *ccol_out = ccol; *cw_out = cw;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* The total order on weighted edges: heavier first, then smaller min endpoint,
 * then smaller max endpoint. Returns 1 when (a1,b1,w1) comes before (a2,b2,w2). */
static int edge_before(double w1, int32_t a1, int32_t b1, double w2, int32_t a2, int32_t b2) {
    int32_t lo1 = a1 < b1 ? a1 : b1, hi1 = a1 < b1 ? b1 : a1;
    int32_t lo2 = a2 < b2 ? a2 : b2, hi2 = a2 < b2 ? b2 : a2;
    if (w1 != w2) return w1 > w2;
    if (lo1 != lo2) return lo1 < lo2;
    return hi1 < hi2;
}

typedef struct { double w; int32_t u, v; } orc_edge;

static int cmp_edge(const void* a, const void* b) {
    const orc_edge* x = (const orc_edge*)a;
    const orc_edge* y = (const orc_edge*)b;
    if (edge_before(x->w, x->u, x->v, y->w, y->u, y->v)) return -1;
    if (edge_before(y->w, y->u, y->v, x->w, x->u, x->v)) return 1;
    return 0;
}

static int32_t uf_find(int32_t* parent, int32_t x) {
    while (parent[x] != x) { parent[x] = parent[parent[x]]; x = parent[x]; }
    return x;
}

static void cover_add(int32_t* nbr0, int32_t* nbr1, int32_t u, int32_t v) {
    if (nbr0[u] < 0) nbr0[u] = v; else nbr1[u] = v;
}

static void cover_canonical(int32_t n, int32_t* nbr0, int32_t* nbr1) {
    for (int32_t u = 0; u < n; ++u) {
        if (nbr0[u] >= 0 && nbr1[u] >= 0 && nbr1[u] < nbr0[u]) {
            int32_t t = nbr0[u]; nbr0[u] = nbr1[u]; nbr1[u] = t;
        } else if (nbr0[u] < 0 && nbr1[u] >= 0) {
            nbr0[u] = nbr1[u]; nbr1[u] = -1;
        }
    }
}

/* Alg. 1: scan edges heaviest first; keep an edge when both ends still have
 * fewer than two cover edges and the ends lie on different paths. */
int32_t orc_cover_greedy(int32_t n, const int32_t* cptr, const int32_t* ccol, const double* cw,
                         int32_t* nbr0, int32_t* nbr1) {
    int64_t m = 0;
    for (int32_t u = 0; u < n; ++u)
        for (int32_t k = cptr[u]; k < cptr[u + 1]; ++k) if (ccol[k] > u) ++m;
    orc_edge* E = (orc_edge*)orc_xmalloc(sizeof(orc_edge) * (size_t)m);
    int32_t* parent = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n);
    int32_t* deg = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n);
    if (!E || !parent || !deg) { free(E); free(parent); free(deg); return ORC_ERR_OOM; }
    m = 0;
    for (int32_t u = 0; u < n; ++u)
        for (int32_t k = cptr[u]; k < cptr[u + 1]; ++k)
            if (ccol[k] > u) { E[m].w = cw[k]; E[m].u = u; E[m].v = ccol[k]; ++m; }
    qsort(E, (size_t)m, sizeof(orc_edge), cmp_edge);
    for (int32_t u = 0; u < n; ++u) { parent[u] = u; deg[u] = 0; nbr0[u] = -1; nbr1[u] = -1; }
    for (int64_t t = 0; t < m; ++t) {
        int32_t u = E[t].u, v = E[t].v;
        if (deg[u] >= 2 || deg[v] >= 2) continue;
        int32_t ru = uf_find(parent, u), rv = uf_find(parent, v);
        if (ru == rv) continue;            /* would close a cycle */
        parent[ru] = rv;
        cover_add(nbr0, nbr1, u, v); cover_add(nbr0, nbr1, v, u);
        ++deg[u]; ++deg[v];
    }
    cover_canonical(n, nbr0, nbr1);
    free(E); free(parent); free(deg);
    return ORC_OK;
}

/* Locally-dominant rounds. Paths (singletons included) act as super-vertices;
 * each path proposes the best eligible edge at its two endpoints; an edge
 * proposed by both of its paths is added. An edge (u,v) is eligible when both
 * ends have fewer than two cover edges and lie on different paths; since both
 * are then endpoints, "different paths" means v is not the far end of u's path. */
int32_t orc_cover_ld(int32_t n, const int32_t* cptr, const int32_t* ccol, const double* cw,
                     int32_t* nbr0, int32_t* nbr1, int32_t* rounds_out) {
    int32_t nn = cptr[n];
    int32_t* scol = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)nn);
    double* sw = (double*)orc_xmalloc(sizeof(double) * (size_t)nn);
    orc_edge* tmp = NULL;
    int32_t maxrow = 0;
    for (int32_t u = 0; u < n; ++u) if (cptr[u + 1] - cptr[u] > maxrow) maxrow = cptr[u + 1] - cptr[u];
    tmp = (orc_edge*)orc_xmalloc(sizeof(orc_edge) * (size_t)(maxrow + 1));
    int32_t *deg = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n),
            *oe = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n),
            *ptr = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n),
            *bv = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n),
            *cf = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n),
            *ct = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n),
            *acc = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n * 2);
    double* bw = (double*)orc_xmalloc(sizeof(double) * (size_t)n);
    if (!scol || !sw || !tmp || !deg || !oe || !ptr || !bv || !cf || !ct || !acc || !bw) {
        free(scol); free(sw); free(tmp); free(deg); free(oe); free(ptr); free(bv);
        free(cf); free(ct); free(acc); free(bw);
        return ORC_ERR_OOM;
    }
    /* each row in the edge order (w desc, then neighbour id asc) */
    for (int32_t u = 0; u < n; ++u) {
        int32_t len = cptr[u + 1] - cptr[u];
        for (int32_t k = 0; k < len; ++k) {
            tmp[k].w = cw[cptr[u] + k]; tmp[k].u = u; tmp[k].v = ccol[cptr[u] + k];
        }
        qsort(tmp, (size_t)len, sizeof(orc_edge), cmp_edge);
        for (int32_t k = 0; k < len; ++k) { scol[cptr[u] + k] = tmp[k].v; sw[cptr[u] + k] = tmp[k].w; }
    }
    for (int32_t u = 0; u < n; ++u) {
        deg[u] = 0; oe[u] = u; ptr[u] = cptr[u]; nbr0[u] = -1; nbr1[u] = -1;
    }
    int32_t rounds = 0;
    for (;;) {
        /* 1. every endpoint finds its best eligible edge (pointers only move forward:
         *    an ineligible edge never becomes eligible again) */
        for (int32_t u = 0; u < n; ++u) {
            if (deg[u] >= 2) continue;
            while (ptr[u] < cptr[u + 1]) {
                int32_t v = scol[ptr[u]];
                if (deg[v] >= 2 || oe[u] == v) ++ptr[u]; else break;
            }
            if (ptr[u] < cptr[u + 1]) { bv[u] = scol[ptr[u]]; bw[u] = sw[ptr[u]]; }
            else bv[u] = -1;
        }
        /* 2. every path keeps the better of its two endpoints' proposals */
        for (int32_t u = 0; u < n; ++u) {
            if (deg[u] >= 2 || u > oe[u]) continue;
            int32_t o = oe[u];
            int32_t x = -1, y = -1;
            if (bv[u] >= 0) { x = u; y = bv[u]; }
            if (o != u && bv[o] >= 0) {
                if (x < 0 || edge_before(bw[o], o, bv[o], bw[u], u, bv[u])) { x = o; y = bv[o]; }
            }
            cf[u] = x; ct[u] = y; cf[o] = x; ct[o] = y;
        }
        /* 3. an edge chosen by both of its paths is accepted */
        int32_t nacc = 0;
        for (int32_t u = 0; u < n; ++u) {
            if (deg[u] >= 2 || cf[u] != u) continue;
            int32_t y = ct[u];
            if (y >= 0 && u < y && cf[y] == y && ct[y] == u) { acc[2 * nacc] = u; acc[2 * nacc + 1] = y; ++nacc; }
        }
        /* 4. merge the paths */
        for (int32_t t = 0; t < nacc; ++t) {
            int32_t u = acc[2 * t], y = acc[2 * t + 1];
            int32_t a = oe[u], b = oe[y];
            oe[a] = b; oe[b] = a;
            cover_add(nbr0, nbr1, u, y); cover_add(nbr0, nbr1, y, u);
            ++deg[u]; ++deg[y];
        }
        ++rounds;
        if (nacc == 0) break;
    }
    cover_canonical(n, nbr0, nbr1);
    if (rounds_out) *rounds_out = rounds;
    free(scol); free(sw); free(tmp); free(deg); free(oe); free(ptr); free(bv);
    free(cf); free(ct); free(acc); free(bw);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
typedef struct { int32_t g, u; } orc_join;

static int cmp_join(const void* a, const void* b) {
    const orc_join* x = (const orc_join*)a;
    const orc_join* y = (const orc_join*)b;
    if (x->g != y->g) return (x->g > y->g) - (x->g < y->g);
    return (x->u > y->u) - (x->u < y->u);
}

/* The rule of Alg. 3 for one unaggregated vertex u whose best neighbour is v:
 * v unaggregated -> new pair {u,v} (case 1); v in an aggregate of size 2 -> u
 * joins it (case 2); size 3 -> v leaves it and {u,v} becomes a new aggregate
 * (case 3). Aggregates are named by a "label" vertex id. */
static void leftover_apply(int32_t u, int32_t v, int32_t* lab, int32_t* size) {
    if (lab[v] < 0) {
        lab[u] = u; lab[v] = u; size[u] = 2;
    } else {
        int32_t h = lab[v];
        if (size[h] == 2) { lab[u] = h; size[h] = 3; }
        else { lab[v] = u; size[h] -= 1; lab[u] = u; size[u] = 2; }
    }
}

int32_t orc_aggregate(int32_t n, const int32_t* nbr0, const int32_t* nbr1,
                      const int32_t* tptr, const int32_t* tcol, const double* tw,
                      int32_t round_cap, int32_t leftover_mode,
                      int32_t* agg, int32_t* nc_out, int32_t* cnbr0, int32_t* cnbr1,
                      int32_t* rounds_out) {
    int32_t *lab = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n),
            *size = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n),
            *path = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n),
            *ishead = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n),
            *sprev = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n),
            *snext = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n),
            *best = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n),
            *inU = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n),
            *minmem = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n),
            *cidl = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n);
    orc_join* J = (orc_join*)orc_xmalloc(sizeof(orc_join) * (size_t)n);
    int32_t st = ORC_OK;
    if (!lab || !size || !path || !ishead || !sprev || !snext || !best || !inU || !minmem || !cidl || !J) {
        st = ORC_ERR_OOM; goto done;
    }
    for (int32_t u = 0; u < n; ++u) {
        lab[u] = -1; size[u] = 0; ishead[u] = 0; sprev[u] = -1; snext[u] = -1;
    }
    /* --- pairing along paths: each path is read from its endpoint with the smaller
     *     id; positions (0,1), (2,3), ... form aggregates; an odd tail is left over */
    for (int32_t s = 0; s < n; ++s) {
        int32_t d = (nbr0[s] >= 0) + (nbr1[s] >= 0);
        if (d != 1) continue;
        int32_t L = 0, prev = -1, cur = s;
        while (cur >= 0) {
            if (L >= n) { st = ORC_ERR_INVALID; goto done; }   /* not a path */
            path[L++] = cur;
            int32_t nx = (nbr0[cur] >= 0 && nbr0[cur] != prev) ? nbr0[cur]
                       : ((nbr1[cur] >= 0 && nbr1[cur] != prev) ? nbr1[cur] : -1);
            prev = cur; cur = nx;
        }
        if (path[L - 1] < s) continue;     /* read it from the other end */
        for (int32_t k = 0; 2 * k + 1 < L; ++k) {
            int32_t h = path[2 * k];
            lab[path[2 * k]] = h; lab[path[2 * k + 1]] = h; size[h] = 2; ishead[h] = 1;
            sprev[h] = (k > 0) ? path[2 * k - 2] : -1;
            snext[h] = (2 * k + 3 < L) ? path[2 * k + 2] : -1;
        }
    }
    /* --- best neighbour in the reweighted graph: heaviest edge, ties to smaller id */
    for (int32_t u = 0; u < n; ++u) {
        int32_t b = -1; double bwv = 0.0;
        for (int32_t k = tptr[u]; k < tptr[u + 1]; ++k) {
            if (b < 0 || tw[k] > bwv || (tw[k] == bwv && tcol[k] < b)) { b = tcol[k]; bwv = tw[k]; }
        }
        best[u] = b;
        if (b < 0 && lab[u] < 0) { lab[u] = u; size[u] = 1; }   /* isolated vertex */
    }
    /* --- leftovers */
    int32_t rounds = 0;
    int32_t cap = (leftover_mode == ORC_LEFT_SEQUENTIAL) ? 0 : round_cap;
    for (;;) {
        int32_t left = 0;
        for (int32_t u = 0; u < n; ++u) left += (lab[u] < 0);
        if (left == 0) break;
        if (rounds >= cap) {
            /* sequential tail: the paper's loop, vertices in ascending order */
            for (int32_t u = 0; u < n; ++u)
                if (lab[u] < 0) leftover_apply(u, best[u], lab, size);
            ++rounds;
            break;
        }
        for (int32_t u = 0; u < n; ++u) inU[u] = (lab[u] < 0);
        int32_t nj = 0;
        for (int32_t u = 0; u < n; ++u) {
            if (!inU[u]) continue;
            int32_t v = best[u];
            if (!inU[v]) { J[nj].g = lab[v]; J[nj].u = u; ++nj; }
        }
        /* case 1: mutual best pairs among unaggregated vertices */
        for (int32_t u = 0; u < n; ++u) {
            if (!inU[u]) continue;
            int32_t v = best[u];
            if (inU[v] && best[v] == u && u < v) { lab[u] = u; lab[v] = u; size[u] = 2; }
        }
        /* cases 2/3: joiners grouped by the aggregate they aim at, each group in
         * ascending vertex order */
        qsort(J, (size_t)nj, sizeof(orc_join), cmp_join);
        for (int32_t t = 0; t < nj; ++t) leftover_apply(J[t].u, best[J[t].u], lab, size);
        ++rounds;
    }
    /* --- numbering by ascending smallest member */
    for (int32_t u = 0; u < n; ++u) minmem[u] = -1;
    for (int32_t u = 0; u < n; ++u) if (minmem[lab[u]] < 0) minmem[lab[u]] = u;
    int32_t nc = 0;
    for (int32_t v = 0; v < n; ++v) if (minmem[lab[v]] == v) cidl[lab[v]] = nc++;
    for (int32_t u = 0; u < n; ++u) agg[u] = cidl[lab[u]];
    /* --- shortened cover: the k-th aggregate matched along a path is joined to the
     *     (k-1)-th and (k+1)-th ones of the same path */
    for (int32_t I = 0; I < nc; ++I) { cnbr0[I] = -1; cnbr1[I] = -1; }
    for (int32_t h = 0; h < n; ++h) {
        if (!ishead[h]) continue;
        int32_t I = cidl[h];
        int32_t a = sprev[h] >= 0 ? cidl[sprev[h]] : -1;
        int32_t b = snext[h] >= 0 ? cidl[snext[h]] : -1;
        if (a >= 0 && b >= 0) { cnbr0[I] = a < b ? a : b; cnbr1[I] = a < b ? b : a; }
        else if (a >= 0) cnbr0[I] = a;
        else if (b >= 0) cnbr0[I] = b;
    }
    *nc_out = nc;
    if (rounds_out) *rounds_out = rounds;
done:
    free(lab); free(size); free(path); free(ishead); free(sprev); free(snext); free(best);
    free(inU); free(minmem); free(cidl); free(J);
    return st;
}

/* ------------------------------------------------------------------------- */
int32_t orc_galerkin(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                     const int32_t* agg, int32_t nc, const double* pval, int32_t drop_diag,
                     int32_t** optr_out, int32_t** ocol_out, double** oval_out, int64_t* onnz) {
    int32_t *mptr = (int32_t*)calloc((size_t)nc + 1, sizeof(int32_t)),
            *mem = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n),
            *fill = (int32_t*)orc_xmalloc(sizeof(int32_t) * ((size_t)nc + 1)),
            *stamp = (int32_t*)orc_xmalloc(sizeof(int32_t) * ((size_t)nc + 1)),
            *list = (int32_t*)orc_xmalloc(sizeof(int32_t) * ((size_t)nc + 1)),
            *optr = (int32_t*)orc_xmalloc(sizeof(int32_t) * ((size_t)nc + 1));
    double* acc = (double*)orc_xmalloc(sizeof(double) * ((size_t)nc + 1));
    int32_t* ocol = NULL;
    double* oval = NULL;
    if (!mptr || !mem || !fill || !stamp || !list || !optr || !acc) goto oom;
    for (int32_t u = 0; u < n; ++u) mptr[agg[u] + 1]++;
    for (int32_t I = 0; I < nc; ++I) mptr[I + 1] += mptr[I];
    for (int32_t I = 0; I <= nc; ++I) fill[I] = mptr[I];
    for (int32_t u = 0; u < n; ++u) mem[fill[agg[u]]++] = u;    /* ascending members */
    for (int32_t I = 0; I < nc; ++I) stamp[I] = -1;
    int64_t total = 0;
    optr[0] = 0;
    for (int32_t I = 0; I < nc; ++I) {
        int32_t cnt = 0;
        for (int32_t t = mptr[I]; t < mptr[I + 1]; ++t) {
            int32_t u = mem[t];
            for (int32_t k = rowptr[u]; k < rowptr[u + 1]; ++k) {
                int32_t Jc = agg[col[k]];
                if (drop_diag && Jc == I) continue;
                if (stamp[Jc] != I) { stamp[Jc] = I; ++cnt; }
            }
        }
        total += cnt;
        if (total >= 2147483647LL) { free(mptr); free(mem); free(fill); free(stamp); free(list); free(optr); free(acc); return ORC_ERR_INVALID; }
        optr[I + 1] = (int32_t)total;
    }
    ocol = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)total);
    oval = (double*)orc_xmalloc(sizeof(double) * (size_t)total);
    if (!ocol || !oval) goto oom;
    for (int32_t I = 0; I < nc; ++I) stamp[I] = -1;
    for (int32_t I = 0; I < nc; ++I) {
        int32_t cnt = 0;
        for (int32_t t = mptr[I]; t < mptr[I + 1]; ++t) {
            int32_t u = mem[t];
            for (int32_t k = rowptr[u]; k < rowptr[u + 1]; ++k) {
                int32_t v = col[k];
                int32_t Jc = agg[v];
                if (drop_diag && Jc == I) continue;
                double term = pval ? (pval[u] * val[k]) * pval[v] : val[k];
                if (stamp[Jc] != I) { stamp[Jc] = I; list[cnt++] = Jc; acc[Jc] = term; }
                else acc[Jc] += term;
            }
        }
        qsort(list, (size_t)cnt, sizeof(int32_t), cmp_i32);
        for (int32_t t = 0; t < cnt; ++t) {
            ocol[optr[I] + t] = list[t];
            oval[optr[I] + t] = acc[list[t]];
        }
    }
    free(mptr); free(mem); free(fill); free(stamp); free(list); free(acc);
    *optr_out = optr; *ocol_out = ocol; *oval_out = oval; *onnz = total;
    return ORC_OK;
oom:
    free(mptr); free(mem); free(fill); free(stamp); free(list); free(optr); free(acc);
    free(ocol); free(oval);
    return ORC_ERR_OOM;
}

/* ------------------------------------------------------------------------- */
static void level_free(orc_level* L) {
    free(L->rowptr); free(L->col); free(L->val); free(L->colour);
    free(L->tptr); free(L->tcol); free(L->tw); free(L->nbr0); free(L->nbr1);
    free(L->agg); free(L->agg_ptr); free(L->agg_mem); free(L->pval);
    memset(L, 0, sizeof(*L));
}

void orc_hier_free(orc_hier* h) {
    if (!h) return;
    for (int32_t l = 0; l < h->nlev; ++l) level_free(&h->lev[l]);
    free(h->Xinv);
    free(h);
}

static int32_t build_members(orc_level* L) {
    L->agg_ptr = (int32_t*)calloc((size_t)L->nc + 1, sizeof(int32_t));
    L->agg_mem = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)L->n);
    int32_t* fill = (int32_t*)orc_xmalloc(sizeof(int32_t) * ((size_t)L->nc + 1));
    if (!L->agg_ptr || !L->agg_mem || !fill) { free(fill); return ORC_ERR_OOM; }
    for (int32_t u = 0; u < L->n; ++u) L->agg_ptr[L->agg[u] + 1]++;
    for (int32_t I = 0; I < L->nc; ++I) L->agg_ptr[I + 1] += L->agg_ptr[I];
    for (int32_t I = 0; I <= L->nc; ++I) fill[I] = L->agg_ptr[I];
    for (int32_t u = 0; u < L->n; ++u) L->agg_mem[fill[L->agg[u]]++] = u;
    free(fill);
    return ORC_OK;
}

/* Smoother colouring of every level but the coarsest, the coarsest level's
 * pinned dense inverse (boolean_chain: every prolongation is boolean, so the
 * constant null space is kept exactly and the last unknown is pinned), and the
 * reweighted graphs dropped unless kept for export. */
static int32_t finish_hierarchy(orc_hier* h, const orc_params* p, int32_t boolean_chain) {
    int32_t st = ORC_OK;
    /* smoother colouring on every level but the coarsest; small coarse levels
     * are smoothed by l1-Jacobi and need none */
    for (int32_t l = 0; l + 1 < h->nlev; ++l) {
        orc_level* L = &h->lev[l];
        L->jac = (l >= 1 && L->n <= p->l1jac_rows);
        if (L->jac) continue;
        L->colour = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)L->n);
        if (!L->colour) return ORC_ERR_OOM;
        L->ncolour = orc_colour_smoother(L->n, L->rowptr, L->col, p->seed, L->colour, NULL);
        if (L->ncolour < 0) return -L->ncolour;
    }
    /* coarsest level: dense pinned Cholesky -> explicit inverse */
    {
        orc_level* C = &h->lev[h->nlev - 1];
        int32_t m = C->n;
        if (m > p->dense_max) return ORC_ERR_COARSE_TOO_BIG;
        double* D = (double*)calloc((size_t)m * (size_t)m, sizeof(double));
        h->Xinv = (double*)orc_xmalloc(sizeof(double) * (size_t)m * (size_t)m);
        if (!D || !h->Xinv) { free(D); return ORC_ERR_OOM; }
        for (int32_t i = 0; i < m; ++i)
            for (int32_t k = C->rowptr[i]; k < C->rowptr[i + 1]; ++k)
                D[(size_t)i * m + C->col[k]] = C->val[k];
        /* a chain of boolean prolongations from a Laplacian keeps the constant
         * null space exactly: pin the last unknown */
        st = orc_dense_pinned_inverse(m, D, boolean_chain, 1e-12, h->Xinv, &h->npinned);
        free(D);
        h->nL = m;
        if (st) return st;
    }
    if (!p->keep_setup)
        for (int32_t l = 0; l < h->nlev; ++l) {
            orc_level* L = &h->lev[l];
            free(L->tptr); free(L->tcol); free(L->tw);
            L->tptr = NULL; L->tcol = NULL; L->tw = NULL;
        }
    return ORC_OK;
}

orc_hier* orc_build(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                    const double* e, const orc_params* p, int32_t* status) {
    int32_t st = ORC_OK;
    orc_hier* h = (orc_hier*)calloc(1, sizeof(orc_hier));
    if (!h) { *status = ORC_ERR_OOM; return NULL; }
    h->nu_pre = p->nu_pre; h->nu_post = p->nu_post;
    int64_t nnz = rowptr[n];
    orc_level* L0 = &h->lev[0];
    L0->n = n; L0->nnz = nnz;
    L0->rowptr = (int32_t*)orc_xmalloc(sizeof(int32_t) * ((size_t)n + 1));
    L0->col = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)nnz);
    L0->val = (double*)orc_xmalloc(sizeof(double) * (size_t)nnz);
    if (!L0->rowptr || !L0->col || !L0->val) { st = ORC_ERR_OOM; goto fail; }
    memcpy(L0->rowptr, rowptr, sizeof(int32_t) * ((size_t)n + 1));
    memcpy(L0->col, col, sizeof(int32_t) * (size_t)nnz);
    memcpy(L0->val, val, sizeof(double) * (size_t)nnz);
    h->nlev = 1;
    /* Alg. 4 step 2: reweight on the A^2 pattern; step 3: path cover */
    st = orc_candidates(n, rowptr, col, e, &L0->tptr, &L0->tcol, &L0->tw);
    if (st) goto fail;
    h->cand_nnz = L0->tptr[n];
    L0->nbr0 = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n);
    L0->nbr1 = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n);
    if (!L0->nbr0 || !L0->nbr1) { st = ORC_ERR_OOM; goto fail; }
    if (p->cover_mode == ORC_COVER_GREEDY) st = orc_cover_greedy(n, L0->tptr, L0->tcol, L0->tw, L0->nbr0, L0->nbr1);
    else st = orc_cover_ld(n, L0->tptr, L0->tcol, L0->tw, L0->nbr0, L0->nbr1, &L0->cover_rounds);
    if (st) goto fail;
    /* Alg. 4 steps 5-9, one level at a time */
    for (int32_t l = 0;; ++l) {
        orc_level* L = &h->lev[l];
        if (L->n <= p->n_min || l == p->max_levels - 1 || l == ORC_MAX_LEVELS - 1) break;
        L->agg = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)L->n);
        int32_t* cn0 = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)L->n);
        int32_t* cn1 = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)L->n);
        if (!L->agg || !cn0 || !cn1) { free(cn0); free(cn1); st = ORC_ERR_OOM; goto fail; }
        st = orc_aggregate(L->n, L->nbr0, L->nbr1, L->tptr, L->tcol, L->tw, p->round_cap,
                           p->leftover_mode, L->agg, &L->nc, cn0, cn1, &L->leftover_rounds);
        if (st) { free(cn0); free(cn1); goto fail; }
        if ((double)L->nc > 0.9 * (double)L->n) {
            free(cn0); free(cn1); free(L->agg); L->agg = NULL; L->nc = 0;
            break;
        }
        st = build_members(L);
        if (st) { free(cn0); free(cn1); goto fail; }
        if (l == 0 && p->p1_mode == ORC_P1_E_SCALED) {
            /* P_1 carries the smooth error: (P_1)_ki = e_k for k in aggregate i;
             * an aggregate on which e vanishes entirely uses 1 instead */
            L->pval = (double*)orc_xmalloc(sizeof(double) * (size_t)L->n);
            if (!L->pval) { free(cn0); free(cn1); st = ORC_ERR_OOM; goto fail; }
            for (int32_t I = 0; I < L->nc; ++I) {
                int allzero = 1;
                for (int32_t t = L->agg_ptr[I]; t < L->agg_ptr[I + 1]; ++t)
                    if (e[L->agg_mem[t]] != 0.0) allzero = 0;
                for (int32_t t = L->agg_ptr[I]; t < L->agg_ptr[I + 1]; ++t)
                    L->pval[L->agg_mem[t]] = allzero ? 1.0 : e[L->agg_mem[t]];
            }
        }
        orc_level* C = &h->lev[l + 1];
        C->n = L->nc;
        st = orc_galerkin(L->n, L->rowptr, L->col, L->val, L->agg, L->nc, L->pval, 0,
                          &C->rowptr, &C->col, &C->val, &C->nnz);
        if (st) { free(cn0); free(cn1); goto fail; }
        int64_t tnnz = 0;
        st = orc_galerkin(L->n, L->tptr, L->tcol, L->tw, L->agg, L->nc, NULL, 1,
                          &C->tptr, &C->tcol, &C->tw, &tnnz);
        if (st) { free(cn0); free(cn1); goto fail; }
        C->nbr0 = cn0; C->nbr1 = cn1;
        h->nlev = l + 2;
    }
    st = finish_hierarchy(h, p, (p->p1_mode == ORC_P1_BOOLEAN) || h->nlev == 1);
    if (st) goto fail;
    *status = ORC_OK;
    return h;
fail:
    orc_hier_free(h);
    *status = st;
    return NULL;
}

/* ------------------------------------------------------------------------- */
/* MWM (Section 2.1): heaviest-first matching on the weighted adjacency of A_l
 * (edge {u,v} weighs -a_uv > 0), visiting edges in the total order of Alg. 1
 * (weight descending, then the smaller end, then the larger end) and matching
 * both ends when both are still free. Each vertex left free then joins the
 * pair of its heaviest neighbour (that neighbour is matched: a free neighbour
 * would have been matched to it); an aggregate is a pair with vertices hung on
 * either end, so its diameter is at most three. A vertex without neighbours
 * stays alone. Aggregates are numbered by ascending smallest member. */
typedef struct { double w; int32_t u, v; } mwm_edge;

static int edge_cmp(const void* a, const void* b) {
    const mwm_edge* x = (const mwm_edge*)a;
    const mwm_edge* y = (const mwm_edge*)b;
    if (x->w != y->w) return x->w > y->w ? -1 : 1;
    if (x->u != y->u) return x->u < y->u ? -1 : 1;
    return (x->v > y->v) - (x->v < y->v);
}

/* edge (u, v) of weight w before edge (u2, v2) of weight w2 in the order above */
static int mwm_before(double w, int32_t u, int32_t v, double w2, int32_t u2, int32_t v2) {
    int32_t a = u < v ? u : v, b = u < v ? v : u, a2 = u2 < v2 ? u2 : v2, b2 = u2 < v2 ? v2 : u2;
    if (w != w2) return w > w2;
    if (a != a2) return a < a2;
    return b < b2;
}

static int32_t mwm_match_greedy(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                                int32_t* mate) {
    int64_t m = 0;
    for (int32_t u = 0; u < n; ++u)
        for (int32_t k = rowptr[u]; k < rowptr[u + 1]; ++k) if (col[k] > u) ++m;
    mwm_edge* E = (mwm_edge*)orc_xmalloc(sizeof(mwm_edge) * (size_t)(m ? m : 1));
    if (!E) return ORC_ERR_OOM;
    m = 0;
    for (int32_t u = 0; u < n; ++u)
        for (int32_t k = rowptr[u]; k < rowptr[u + 1]; ++k)
            if (col[k] > u) { E[m].w = -val[k]; E[m].u = u; E[m].v = col[k]; ++m; }
    qsort(E, (size_t)m, sizeof(mwm_edge), edge_cmp);
    for (int32_t i = 0; i < n; ++i) mate[i] = -1;
    for (int64_t t = 0; t < m; ++t)
        if (mate[E[t].u] < 0 && mate[E[t].v] < 0) { mate[E[t].u] = E[t].v; mate[E[t].v] = E[t].u; }
    free(E);
    return ORC_OK;
}

/* the same matching by locally-dominant rounds: every free vertex points at its
 * heaviest free neighbour; two vertices pointing at each other are matched */
static int32_t mwm_match_ld(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                            int32_t* mate, int32_t* rounds_out) {
    int32_t* best = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    if (!best) return ORC_ERR_OOM;
    for (int32_t i = 0; i < n; ++i) mate[i] = -1;
    int32_t rounds = 0;
    for (;;) {
        int32_t any = 0;
        for (int32_t v = 0; v < n; ++v) {
            best[v] = -1;
            if (mate[v] >= 0) continue;
            double bw = 0.0;
            for (int32_t k = rowptr[v]; k < rowptr[v + 1]; ++k) {
                int32_t u = col[k];
                if (u == v || mate[u] >= 0) continue;
                if (best[v] < 0 || mwm_before(-val[k], v, u, bw, v, best[v])) { best[v] = u; bw = -val[k]; }
            }
        }
        ++rounds;
        for (int32_t v = 0; v < n; ++v) {
            int32_t u = best[v];
            if (u >= 0 && best[u] == v) { mate[v] = u; any = 1; }
        }
        if (!any) break;
    }
    free(best);
    if (rounds_out) *rounds_out = rounds;
    return ORC_OK;
}

int32_t orc_mwm_aggregate(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                          int32_t ld, int32_t* agg, int32_t* nc_out, int32_t* rounds) {
    int32_t* mate = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    int32_t* lab = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    int32_t* minm = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    if (!mate || !lab || !minm) { free(mate); free(lab); free(minm); return ORC_ERR_OOM; }
    int32_t st = ld ? mwm_match_ld(n, rowptr, col, val, mate, rounds)
                    : mwm_match_greedy(n, rowptr, col, val, mate);
    if (!ld && rounds) *rounds = 0;
    if (st) { free(mate); free(lab); free(minm); return st; }
    /* label = the smaller vertex of the pair; a free vertex takes the label of
     * its heaviest neighbour's pair */
    for (int32_t v = 0; v < n; ++v) lab[v] = mate[v] >= 0 ? (v < mate[v] ? v : mate[v]) : -1;
    for (int32_t v = 0; v < n; ++v) {
        if (mate[v] >= 0) continue;
        int32_t b = -1;
        double bw = 0.0;
        for (int32_t k = rowptr[v]; k < rowptr[v + 1]; ++k) {
            int32_t u = col[k];
            if (u == v) continue;
            if (b < 0 || mwm_before(-val[k], v, u, bw, v, b)) { b = u; bw = -val[k]; }
        }
        lab[v] = (b < 0) ? v : (b < mate[b] ? b : mate[b]);
    }
    /* number aggregates by their smallest member */
    for (int32_t v = 0; v < n; ++v) minm[v] = n;
    for (int32_t v = 0; v < n; ++v) if (v < minm[lab[v]]) minm[lab[v]] = v;
    int32_t nc = 0;
    int32_t* id = mate;   /* reuse: id of the aggregate whose smallest member is v */
    for (int32_t v = 0; v < n; ++v) id[v] = (minm[lab[v]] == v) ? nc++ : -1;
    for (int32_t v = 0; v < n; ++v) agg[v] = id[minm[lab[v]]];
    *nc_out = nc;
    free(mate); free(lab); free(minm);
    return ORC_OK;
}

orc_hier* orc_build_mwm(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                        const orc_params* p, int32_t* status) {
    int32_t st = ORC_OK;
    orc_hier* h = (orc_hier*)calloc(1, sizeof(orc_hier));
    if (!h) { *status = ORC_ERR_OOM; return NULL; }
    h->nu_pre = p->nu_pre; h->nu_post = p->nu_post;
    int64_t nnz = rowptr[n];
    orc_level* L0 = &h->lev[0];
    L0->n = n; L0->nnz = nnz;
    L0->rowptr = (int32_t*)orc_xmalloc(sizeof(int32_t) * ((size_t)n + 1));
    L0->col = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)nnz);
    L0->val = (double*)orc_xmalloc(sizeof(double) * (size_t)nnz);
    if (!L0->rowptr || !L0->col || !L0->val) { st = ORC_ERR_OOM; goto fail; }
    memcpy(L0->rowptr, rowptr, sizeof(int32_t) * ((size_t)n + 1));
    memcpy(L0->col, col, sizeof(int32_t) * (size_t)nnz);
    memcpy(L0->val, val, sizeof(double) * (size_t)nnz);
    h->nlev = 1;
    for (int32_t l = 0;; ++l) {
        orc_level* L = &h->lev[l];
        if (L->n <= p->n_min || l == p->max_levels - 1 || l == ORC_MAX_LEVELS - 1) break;
        L->agg = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)L->n);
        if (!L->agg) { st = ORC_ERR_OOM; goto fail; }
        st = orc_mwm_aggregate(L->n, L->rowptr, L->col, L->val, p->cover_mode == ORC_COVER_LD, L->agg,
                               &L->nc, &L->cover_rounds);
        if (st) goto fail;
        if ((double)L->nc > 0.9 * (double)L->n) {
            free(L->agg); L->agg = NULL; L->nc = 0;
            break;
        }
        st = build_members(L);
        if (st) goto fail;
        orc_level* C = &h->lev[l + 1];
        C->n = L->nc;
        st = orc_galerkin(L->n, L->rowptr, L->col, L->val, L->agg, L->nc, NULL, 0,
                          &C->rowptr, &C->col, &C->val, &C->nnz);
        if (st) goto fail;
        h->nlev = l + 2;
    }
    st = finish_hierarchy(h, p, 1);
    if (st) goto fail;
    *status = ORC_OK;
    return h;
fail:
    orc_hier_free(h);
    *status = st;
    return NULL;
}

int32_t orc_hier_nlevels(const orc_hier* h) { return h->nlev; }

void orc_hier_sizes(const orc_hier* h, int32_t lev, int64_t s[8]) {
    const orc_level* L = &h->lev[lev];
    s[0] = L->n; s[1] = L->nnz; s[2] = (lev + 1 < h->nlev) ? L->nc : 0; s[3] = L->ncolour;
    s[4] = L->cover_rounds; s[5] = L->leftover_rounds; s[6] = h->npinned; s[7] = h->cand_nnz;
}

void orc_hier_export(const orc_hier* h, int32_t lev, int32_t* agg, int32_t* nbr0,
                     int32_t* nbr1, int32_t* rowptr, int32_t* col, double* val,
                     double* pval, int32_t* colour) {
    const orc_level* L = &h->lev[lev];
    if (agg && L->agg) memcpy(agg, L->agg, sizeof(int32_t) * (size_t)L->n);
    if (nbr0 && L->nbr0) memcpy(nbr0, L->nbr0, sizeof(int32_t) * (size_t)L->n);
    if (nbr1 && L->nbr1) memcpy(nbr1, L->nbr1, sizeof(int32_t) * (size_t)L->n);
    if (rowptr) memcpy(rowptr, L->rowptr, sizeof(int32_t) * ((size_t)L->n + 1));
    if (col) memcpy(col, L->col, sizeof(int32_t) * (size_t)L->nnz);
    if (val) memcpy(val, L->val, sizeof(double) * (size_t)L->nnz);
    if (pval && L->pval) memcpy(pval, L->pval, sizeof(double) * (size_t)L->n);
    if (colour && L->colour) memcpy(colour, L->colour, sizeof(int32_t) * (size_t)L->n);
}

void orc_hier_export_candidates(const orc_hier* h, int32_t* cptr, int32_t* ccol, double* cw) {
    const orc_level* L = &h->lev[0];
    if (!L->tptr) return;                 /* built with keep_setup = 0 */
    if (cptr) memcpy(cptr, L->tptr, sizeof(int32_t) * ((size_t)L->n + 1));
    if (ccol) memcpy(ccol, L->tcol, sizeof(int32_t) * (size_t)L->tptr[L->n]);
    if (cw) memcpy(cw, L->tw, sizeof(double) * (size_t)L->tptr[L->n]);
}

double orc_hier_oc(const orc_hier* h) {
    double s = 0.0;
    for (int32_t l = 0; l < h->nlev; ++l) s += (double)h->lev[l].nnz;
    return s / (double)h->lev[0].nnz;
}
