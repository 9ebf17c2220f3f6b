/*
 * CPU oracle, part 1: random numbers, level operators, coarsest solve.
 * TEST INFRASTRUCTURE ONLY (see oracle.h). Plain FP64, single thread,
 * compiled with -ffp-contract=off so every product and sum rounds once.
 */
#include "orc_internal.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

void orc_free(void* p) { free(p); }

void* orc_xmalloc(size_t bytes) {
    void* p = malloc(bytes ? bytes : 1);
    return p;
}

void orc_default_params(orc_params* p) {
    memset(p, 0, sizeof(*p));
    p->tol = 1e-8;            /* Section 4, scalability tests */
    p->max_iter = 300;
    p->threshold = 0.4;       /* Alg. 5(2) */
    p->numW = 2;              /* Section 4 parameter choices */
    p->iterW = 7;
    p->iterV = 4;
    p->nu_pre = 1;
    p->nu_post = 1;
    p->relax_sweeps = 8;
    p->seed = 12345;
    p->n_min = 256;
    p->max_levels = 25;
    p->round_cap = 64;
    p->p1_mode = ORC_P1_E_SCALED;
    p->leftover_mode = ORC_LEFT_ROUNDS;
    p->cover_mode = ORC_COVER_LD;
    p->dense_max = 4096;
    p->l1jac_rows = 2147483647;
    p->update_mode = ORC_UPD_REBUILD_ONLY;  /* the printed order of Alg. 5 */
    p->keep_setup = 1;
}

/* ------------------------------------------------------------------------- */
/* Philox4x64-10, from the published definition: each round multiplies words 0
 * and 2 by fixed odd constants, keeps the 128-bit products' halves, and mixes
 * the high halves with words 1, 3 and the round key; the key is bumped by two
 * Weyl constants between rounds. */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *lo = (uint64_t)p;
    *hi = (uint64_t)(p >> 64);
}

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, c0, &hi0, &lo0);
        mulhilo64(M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

uint64_t orc_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void orc_uniform_pm1(uint64_t seed, int64_t n, double* out) {
    uint64_t key[2] = {seed, 0};
    for (int64_t i = 0; i < n; ++i) {
        uint64_t ctr[4] = {(uint64_t)(i >> 2), 0, 0, 0};
        uint64_t w[4];
        orc_philox4x64_10(ctr, key, w);
        uint64_t word = w[i & 3];
        out[i] = ldexp((double)(word >> 11), -52) - 1.0;
    }
}

/* ------------------------------------------------------------------------- */
void orc_residual(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                  const double* x, const double* b, double* r) {
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        /* one fused multiply-add per entry, left to right */
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s = fma(val[k], x[col[k]], s);
        r[i] = b[i] - s;
    }
}

static int beats(uint64_t hu, int32_t u, uint64_t hv, int32_t v) {
    return hu > hv || (hu == hv && u > v);
}

int32_t orc_colour(int32_t n, const int32_t* rowptr, const int32_t* col, uint64_t seed,
                   int32_t* colour, int32_t* rounds_out) {
    uint64_t* h = (uint64_t*)orc_xmalloc(sizeof(uint64_t) * (size_t)n);
    int32_t* next = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n);
    int32_t* mark = (int32_t*)orc_xmalloc(sizeof(int32_t) * ((size_t)n + 2));
    if (!h || !next || !mark) { free(h); free(next); free(mark); return -ORC_ERR_OOM; }
    for (int32_t i = 0; i < n; ++i) { h[i] = orc_splitmix64(seed ^ (uint64_t)(int64_t)i); colour[i] = -1; }
    for (int32_t i = 0; i < n + 2; ++i) mark[i] = -1;
    int32_t left = n, ncol = 0, rounds = 0;
    while (left > 0) {
        memcpy(next, colour, sizeof(int32_t) * (size_t)n);
        for (int32_t v = 0; v < n; ++v) {
            if (colour[v] >= 0) continue;
            int win = 1;
            for (int32_t k = rowptr[v]; k < rowptr[v + 1]; ++k) {
                int32_t u = col[k];
                if (u == v || colour[u] >= 0) continue;
                if (beats(h[u], u, h[v], v)) { win = 0; break; }
            }
            if (!win) continue;
            /* smallest colour not used by a neighbour coloured in earlier rounds */
            for (int32_t k = rowptr[v]; k < rowptr[v + 1]; ++k) {
                int32_t u = col[k];
                if (u != v && colour[u] >= 0 && colour[u] <= n) mark[colour[u]] = v;
            }
            int32_t c = 0;
            while (mark[c] == v) ++c;
            next[v] = c;
            if (c + 1 > ncol) ncol = c + 1;
        }
        int32_t done = 0;
        for (int32_t v = 0; v < n; ++v) if (colour[v] < 0 && next[v] >= 0) ++done;
        memcpy(colour, next, sizeof(int32_t) * (size_t)n);
        left -= done;
        ++rounds;
    }
    free(h); free(next); free(mark);
    if (rounds_out) *rounds_out = rounds;
    return ncol;
}

/* Smoother colouring. A connected bipartite graph (every 2D/3D grid graph) is
 * coloured by the parity of each vertex's breadth-first distance from vertex 0:
 * two colours, unique once vertex 0 has colour 0. Any other graph (an odd
 * cycle: some edge joins two vertices at the same distance; or disconnected)
 * gets the Jones-Plassmann colouring above. *rounds_out = the number of
 * distance levels, or the Jones-Plassmann rounds. */
int32_t orc_colour_smoother(int32_t n, const int32_t* rowptr, const int32_t* col, uint64_t seed,
                            int32_t* colour, int32_t* rounds_out) {
    int32_t* dist = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n);
    int32_t* queue = (int32_t*)orc_xmalloc(sizeof(int32_t) * (size_t)n);
    if (!dist || !queue) { free(dist); free(queue); return -ORC_ERR_OOM; }
    for (int32_t i = 0; i < n; ++i) dist[i] = -1;
    int32_t head = 0, tail = 0, levels = 0, ok = n > 0;
    if (ok) { dist[0] = 0; queue[tail++] = 0; }
    while (head < tail) {
        int32_t v = queue[head++];
        if (dist[v] + 1 > levels) levels = dist[v] + 1;
        for (int32_t k = rowptr[v]; k < rowptr[v + 1]; ++k) {
            int32_t u = col[k];
            if (u == v) continue;
            if (dist[u] < 0) { dist[u] = dist[v] + 1; queue[tail++] = u; }
            else if (dist[u] == dist[v]) ok = 0;     /* odd cycle */
        }
    }
    if (tail != n) ok = 0;                           /* not connected */
    int32_t nc;
    if (ok) {
        for (int32_t i = 0; i < n; ++i) colour[i] = dist[i] & 1;
        nc = n > 1 ? 2 : 1;
        if (rounds_out) *rounds_out = levels;
    } else {
        nc = orc_colour(n, rowptr, col, seed, colour, rounds_out);
    }
    free(dist); free(queue);
    return nc;
}

static void gs_row(const int32_t* rowptr, const int32_t* col, const double* val,
                   const double* b, double* x, int32_t i) {
    double s = 0.0, d = 0.0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        int32_t j = col[k];
        if (j == i) d = val[k];
        else s = fma(val[k], x[j], s);
    }
    x[i] = (b[i] - s) / d;
}

void orc_mcgs_sweep(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                    const int32_t* colour, int32_t ncolour, const double* b, double* x,
                    int32_t forward) {
    for (int32_t t = 0; t < ncolour; ++t) {
        int32_t c = forward ? t : ncolour - 1 - t;
        for (int32_t i = 0; i < n; ++i)
            if (colour[i] == c) gs_row(rowptr, col, val, b, x, i);
    }
}

void orc_l1jac_sweep(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                     const double* b, double* x) {
    double* r = (double*)orc_xmalloc(sizeof(double) * (size_t)n);
    orc_residual(n, rowptr, col, val, x, b, r);
    for (int32_t i = 0; i < n; ++i) {
        double d = 0.0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) d += fabs(val[k]);
        x[i] += r[i] / d;
    }
    free(r);
}

void orc_gs_perm_sweep(int32_t n, const int32_t* rowptr, const int32_t* col,
                       const double* val, const int32_t* perm, const double* b, double* x) {
    for (int32_t t = 0; t < n; ++t) gs_row(rowptr, col, val, b, x, perm[t]);
}

/* ------------------------------------------------------------------------- */
/* Coarsest level: Cholesky A = L L^T where a pivot <= tau * max diag (or any
 * index listed in force_pin) is "pinned": its row and column are replaced by
 * the identity and its right-hand-side entry by 0, so its solution entry is 0.
 * The explicit inverse X (n x n, row-major) is then formed column by column by
 * forward and back substitution, so the coarse solve is x = X r. */
int32_t orc_dense_pinned_inverse(int32_t m, const double* Adense, int32_t force_last,
                                 double tau, double* X, int32_t* npinned) {
    double* L = (double*)calloc((size_t)m * (size_t)m, sizeof(double));
    int32_t* pin = (int32_t*)calloc((size_t)m, sizeof(int32_t));
    double* y = (double*)orc_xmalloc(sizeof(double) * (size_t)m);
    if (!L || !pin || !y) { free(L); free(pin); free(y); return ORC_ERR_OOM; }
    double maxd = 0.0;
    for (int32_t i = 0; i < m; ++i) if (Adense[(size_t)i * m + i] > maxd) maxd = Adense[(size_t)i * m + i];
    int32_t np = 0;
    for (int32_t k = 0; k < m; ++k) {
        double d = Adense[(size_t)k * m + k];
        for (int32_t j = 0; j < k; ++j) d -= L[(size_t)k * m + j] * L[(size_t)k * m + j];
        if ((force_last && k == m - 1) || !(d > tau * maxd)) {
            pin[k] = 1; ++np;
            continue;                       /* column k of L stays zero */
        }
        double lkk = sqrt(d);
        L[(size_t)k * m + k] = lkk;
        for (int32_t i = k + 1; i < m; ++i) {
            double s = Adense[(size_t)i * m + k];
            for (int32_t j = 0; j < k; ++j) s -= L[(size_t)i * m + j] * L[(size_t)k * m + j];
            L[(size_t)i * m + k] = s / lkk;
        }
    }
    for (int32_t c = 0; c < m; ++c) {
        /* forward: L y = e_c */
        for (int32_t i = 0; i < m; ++i) {
            if (pin[i]) { y[i] = 0.0; continue; }
            double s = (i == c) ? 1.0 : 0.0;
            for (int32_t j = 0; j < i; ++j) s -= L[(size_t)i * m + j] * y[j];
            y[i] = s / L[(size_t)i * m + i];
        }
        /* backward: L^T x = y */
        for (int32_t i = m - 1; i >= 0; --i) {
            if (pin[i]) { X[(size_t)i * m + c] = 0.0; continue; }
            double s = y[i];
            for (int32_t j = i + 1; j < m; ++j) s -= L[(size_t)j * m + i] * X[(size_t)j * m + c];
            X[(size_t)i * m + c] = s / L[(size_t)i * m + i];
        }
    }
    free(L); free(pin); free(y);
    if (npinned) *npinned = np;
    return ORC_OK;
}
