// PathCoverAMG_setup (Alg. 4) orchestration: reweighting on the A^2 pattern,
// path cover, then per level path-cover aggregation (Alg. 3), prolongation
// (level 1 carries e, Section 3.3), Galerkin products of A and of the reweighted
// graph, path shortening, smoother colouring, and the coarsest factorisation.
#include <cstring>
#include <memory>
#include <vector>
#include <utility>

#include "pcamg_internal.cuh"

namespace pc {

Hier::~Hier() {
    for (auto& g : graph)
        if (g) cudaGraphExecDestroy(g);
    for (auto& g : graph_tmpl)
        if (g) cudaGraphDestroy(g);
}

static Csr make_csr(const Level& L, int32_t n, int64_t nnz, const int32_t* rp, const int32_t* ci,
                    const double* v, const float* v32) {
    (void)L;
    Csr A;
    A.n = n;
    A.nnz = nnz;
    A.rowptr = rp;
    A.col = ci;
    A.val = v;
    A.val32 = v32;
    A.lpr = lanes_per_row(n, nnz);
    return A;
}

template <class T>
static T* vx(Level& L) { if constexpr (sizeof(T) == 8) return L.x64v; else return L.x32v; }
template <class T>
static T* vb(Level& L) { if constexpr (sizeof(T) == 8) return L.b64v; else return L.b32v; }
template <class T>
static T* vr(Level& L) { if constexpr (sizeof(T) == 8) return L.r64v; else return L.r32v; }

template <class T>
static void setup_tail(Ctx& c, Hier& h) {
    std::vector<TailLevel<T>> tl(h.nlev);
    for (int32_t l = h.lt; l < h.nlev; ++l) {
        Level& L = h.lev[l];
        TailLevel<T>& t = tl[l];
        std::memset(&t, 0, sizeof(t));
        t.n = L.n;
        t.nc = (l + 1 < h.nlev) ? L.nc : 0;
        t.ncolour = (l + 1 < h.nlev) ? L.ncolour : 0;
        t.jac = L.jac;
        if constexpr (sizeof(T) == 8) t.dl1 = L.dl1_64.p; else t.dl1 = L.dl1_32.p;
        t.lpr = L.A.lpr;
        t.rowptr = L.A.rowptr;
        t.col = L.A.col;
        if constexpr (sizeof(T) == 8) t.val = L.A.val; else t.val = L.A.val32;
        if (l + 1 < h.nlev) {
            if (!L.jac) {
                L.d_cptr.alloc(c.mem, L.h_colour_ptr.size());
                PC_CUDA(cudaMemcpyAsync(L.d_cptr.p, L.h_colour_ptr.data(), sizeof(int32_t) * L.h_colour_ptr.size(),
                                        cudaMemcpyHostToDevice, c.stream));
                t.cptr = L.d_cptr.p;
            }
            t.crows = L.colour_rows_v;
            t.agg = L.agg.p;
            t.agg_ptr = L.agg_ptr.p;
            t.agg_mem = L.agg_mem.p;
            if (l == 0) {
                if constexpr (sizeof(T) == 8) t.pval = L.pval.p; else t.pval = L.pval32.p;
            }
        }
        t.x = vx<T>(L);
        t.b = vb<T>(L);
        t.r = vr<T>(L);
    }
    h.tail.alloc(c.mem, sizeof(TailLevel<T>) * h.nlev);
    PC_CUDA(cudaMemcpyAsync(h.tail.p, tl.data(), sizeof(TailLevel<T>) * h.nlev, cudaMemcpyHostToDevice, c.stream));
    sync(c);
}

// Everything after the levels exist: smoothers (l1-Jacobi diagonals or
// colourings), the coarsest level's pinned dense inverse (boolean_chain: every
// prolongation is boolean, so the last unknown is pinned), work vectors,
// operator complexity, the coarse tail and the row-permuted smoother copies.
static void finish_hierarchy(Ctx& c, Hier& hh, bool boolean_chain) {
    const pcamg_params& p = c.p;
    const bool f32 = p.precision == PCAMG_FP32_IR;
    Hier* h = &hh;
    const int32_t nlev = h->nlev;
    // smoother of every level but the coarsest: small coarse levels use
    // l1-Jacobi (diagonal of row l1 norms), the others multicolour Gauss-Seidel
    // (level 0's colouring is shared)
    for (int32_t l = 1; l + 1 < nlev; ++l) {
        Level& L = h->lev[l];
        if (L.n <= p.l1jac_rows) {
            L.jac = 1;
            L.dl1_64.alloc(c.mem, L.n);
            l1_diagonal(c.stream, L.n, L.A.rowptr, L.A.val, L.dl1_64.p);
            if (f32) {
                L.dl1_32.alloc(c.mem, L.n);
                cast_f32(c.stream, L.n, L.dl1_64.p, L.dl1_32.p);
            }
            continue;
        }
        L.colour.alloc(c.mem, L.n);
        L.ncolour = colour_smoother(c, L.n, L.A.rowptr, L.A.col, p.seed, L.colour.p);
        colour_lists(c, L.n, L.colour.p, L.ncolour, L.colour_rows, L.h_colour_ptr);
        L.colour_v = L.colour.p;
        L.colour_rows_v = L.colour_rows.p;
    }
    // coarsest level
    Level& LC = h->lev[nlev - 1];
    if (LC.n > p.dense_max) fail(PCAMG_ERR_COARSE_TOO_BIG, "coarsening stalled above dense_max");
    coarse_factor(c, LC.n, LC.A.rowptr, LC.A.col, LC.A.val, boolean_chain, h->Xinv, &h->npinned);
    h->nL = LC.n;
    // work vectors
    double nnz_sum = 0.0;
    for (int32_t l = 0; l < nlev; ++l) {
        Level& L = h->lev[l];
        nnz_sum += (double)L.nnz;
        if (f32) {
            if (l > 0) { L.x32.alloc(c.mem, L.n); L.b32.alloc(c.mem, L.n); L.r32.alloc(c.mem, L.n); }
            if (l == nlev - 1) { L.x64.alloc(c.mem, L.n); L.b64.alloc(c.mem, L.n); }
        } else if (l > 0) {
            L.x64.alloc(c.mem, L.n); L.b64.alloc(c.mem, L.n); L.r64.alloc(c.mem, L.n);
        }
        if (l == 0) {   // the finest level's vectors are the context's
            L.x32v = c.l0_x32.p; L.b32v = c.l0_b32.p; L.r32v = c.l0_r32.p;
            L.x64v = L.x64.p ? L.x64.p : c.l0_x64.p;
            L.b64v = L.b64.p ? L.b64.p : c.l0_b64.p;
            L.r64v = c.l0_r64.p;
        } else {
            L.x32v = L.x32.p; L.b32v = L.b32.p; L.r32v = L.r32.p;
            L.x64v = L.x64.p; L.b64v = L.b64.p; L.r64v = L.r64.p;
        }
    }
    h->oc = nnz_sum / (double)c.nnz;
    // levels from lt down run inside the single-block tail kernel
    // (the finest level joins only below half the limit: the tail's dense
    // operator then stays a small part of a small problem)
    h->lt = nlev;
    if (p.tail_rows > 0)
        for (int32_t l = 0; l < nlev; ++l)
            if (h->lev[l].n <= (l == 0 ? p.tail_rows / 2 : p.tail_rows)) { h->lt = l; break; }
    if (h->lt < nlev) {
        if (f32) setup_tail<float>(c, *h); else setup_tail<double>(c, *h);
    }
    // second iterate buffers of the l1-Jacobi levels the cycle runs level by level
    for (int32_t l = 1; l < h->lt && l + 1 < nlev; ++l) {
        Level& L = h->lev[l];
        if (!L.jac) continue;
        if (f32) L.xa32.alloc(c.mem, L.n); else L.xa64.alloc(c.mem, L.n);
    }
    // row-permuted copies for the streaming smoother on levels above the tail
    for (int32_t l = 1; l < h->lt && l + 1 < nlev; ++l) {
        Level& L = h->lev[l];
        if (L.jac || L.ncolour < 1 || !use_stream(L.n / L.ncolour, L.A.lpr)) continue;
        if (f32) {
            permute_rows<float>(c, L.n, L.colour_rows_v, L.A.rowptr, L.A.col, L.A.val, L.gs_ptr, L.gs_col, L.gs_val32);
            L.gs_val32_v = L.gs_val32.p;
        } else {
            permute_rows<double>(c, L.n, L.colour_rows_v, L.A.rowptr, L.A.col, L.A.val, L.gs_ptr, L.gs_col, L.gs_val64);
            L.gs_val64_v = L.gs_val64.p;
        }
        L.gs_ptr_v = L.gs_ptr.p;
        L.gs_col_v = L.gs_col.p;
    }
    // the finest level in colour order (the context keeps its matrix that way):
    // restate this hierarchy's level-0 transfer data by position
    Level& L0 = h->lev[0];
    if (c.perm0 && nlev > 1 && h->lt >= 1) {
        L0.perm = true;
        L0.Ap = make_csr(L0, c.n, c.nnz, c.gs_ptr0.p, c.gs_col0.p, c.gs_val0_64.p, f32 ? c.gs_val0_32.p : nullptr);
        L0.Ap.dmark = true;
        L0.aggp.alloc(c.mem, L0.n);
        gather<int32_t>(c.stream, L0.n, c.colour_rows0.p, L0.agg.p, L0.aggp.p);
        L0.memp.alloc(c.mem, L0.n);
        map_index(c.stream, L0.n, c.iperm0.p, L0.agg_mem.p, L0.memp.p);
        if (L0.pval.p) {
            if (f32) {
                L0.pvalp32.alloc(c.mem, L0.n);
                gather<float>(c.stream, L0.n, c.colour_rows0.p, L0.pval32.p, L0.pvalp32.p);
            } else {
                L0.pvalp.alloc(c.mem, L0.n);
                gather<double>(c.stream, L0.n, c.colour_rows0.p, L0.pval.p, L0.pvalp.p);
            }
        }
    }
}

Hier* build_hierarchy(Ctx& c, const double* e) {
    const pcamg_params& p = c.p;
    std::unique_ptr<Hier> h(new Hier());
    const bool f32 = p.precision == PCAMG_FP32_IR;
    Level& L0 = h->lev[0];
    L0.n = c.n;
    L0.nnz = c.nnz;
    L0.A = make_csr(L0, c.n, c.nnz, c.rowptr.p, c.col.p, c.val.p, f32 ? c.val32.p : nullptr);
    L0.ncolour = c.ncolour0;
    L0.colour_v = c.colour0.p;
    L0.colour_rows_v = c.colour_rows0.p;
    L0.h_colour_ptr = c.h_colour_ptr0;
    L0.gs_ptr_v = c.gs_ptr0.p;
    L0.gs_col_v = c.gs_col0.p;
    L0.gs_val64_v = f32 ? nullptr : c.gs_val0_64.p;
    L0.gs_val32_v = f32 ? c.gs_val0_32.p : nullptr;

    // Alg. 4 steps 2-3: reweighted A^2 pattern and its path cover
    Reweighted t;
    build_candidates(c, e, t);
    DBuf<int32_t> nbr0, nbr1;
    nbr0.alloc(c.mem, c.n);
    nbr1.alloc(c.mem, c.n);
    L0.cover_rounds = path_cover(c, c.n, t, nbr0.p, nbr1.p);

    int32_t nlev = 1;
    for (int32_t l = 0;; ++l) {
        Level& L = h->lev[l];
        if (L.n <= p.n_min || l == p.max_levels - 1 || l == kMaxLevels - 1) break;
        DBuf<int32_t> agg, cn0, cn1;
        int32_t rounds = 0;
        int32_t nc = aggregate_level(c, L.n, nbr0.p, nbr1.p, t, agg, cn0, cn1, &rounds);
        L.leftover_rounds = rounds;
        if ((double)nc > 0.9 * (double)L.n) break;   // coarsening stalled: L is the coarsest
        L.nc = nc;
        L.agg = std::move(agg);
        build_members(c, L.n, nc, L.agg.p, L.agg_ptr, L.agg_mem);
        if (l == 0 && p.p1_mode == PCAMG_P1_E_SCALED) {
            build_pval(c, L.n, nc, L.agg_ptr.p, L.agg_mem.p, e, L.pval);
            if (f32) {
                L.pval32.alloc(c.mem, L.n);
                cast_f32(c.stream, L.n, L.pval.p, L.pval32.p);
            }
        }
        Level& C = h->lev[l + 1];
        C.n = nc;
        C.nnz = galerkin(c, L.n, L.A.rowptr, L.A.col, L.A.val, nc, L.agg.p, L.agg_ptr.p,
                         L.agg_mem.p, L.pval.p, false, C.rowptr, C.col, C.val);
        Reweighted tc;
        tc.nnz = galerkin(c, L.n, t.ptr.p, t.col.p, t.w.p, nc, L.agg.p, L.agg_ptr.p, L.agg_mem.p,
                          nullptr, true, tc.ptr, tc.col, tc.w);
        if (f32) {
            C.val32.alloc(c.mem, C.nnz);
            cast_f32(c.stream, C.nnz, C.val.p, C.val32.p);
        }
        C.A = make_csr(C, C.n, C.nnz, C.rowptr.p, C.col.p, C.val.p, f32 ? C.val32.p : nullptr);
        if (p.keep_setup) {
            L.nbr0 = std::move(nbr0);
            L.nbr1 = std::move(nbr1);
            L.tptr = std::move(t.ptr);
            L.tcol = std::move(t.col);
            L.tw = std::move(t.w);
            L.tnnz = t.nnz;
        }
        t = Reweighted();
        t.ptr = std::move(tc.ptr);
        t.col = std::move(tc.col);
        t.w = std::move(tc.w);
        t.nnz = tc.nnz;
        nbr0 = std::move(cn0);
        nbr1 = std::move(cn1);
        nlev = l + 2;
    }
    h->nlev = nlev;
    if (p.keep_setup) {
        Level& Lc = h->lev[nlev - 1];
        Lc.nbr0 = std::move(nbr0);
        Lc.nbr1 = std::move(nbr1);
        Lc.tptr = std::move(t.ptr);
        Lc.tcol = std::move(t.col);
        Lc.tw = std::move(t.w);
        Lc.tnnz = t.nnz;
    }
    finish_hierarchy(c, *h, (p.p1_mode == PCAMG_P1_BOOLEAN) || nlev == 1);
    sync(c);
    return h.release();
}

// MWM_setup (Alg. 5 and 6, Section 2.1): MWM aggregation of every level's
// weighted adjacency, boolean prolongations (UA-AMG), Galerkin coarse
// matrices, the same stopping rules as Alg. 4.
Hier* build_hierarchy_mwm(Ctx& c) {
    const pcamg_params& p = c.p;
    std::unique_ptr<Hier> h(new Hier());
    const bool f32 = p.precision == PCAMG_FP32_IR;
    Level& L0 = h->lev[0];
    L0.n = c.n;
    L0.nnz = c.nnz;
    L0.A = make_csr(L0, c.n, c.nnz, c.rowptr.p, c.col.p, c.val.p, f32 ? c.val32.p : nullptr);
    L0.ncolour = c.ncolour0;
    L0.colour_v = c.colour0.p;
    L0.colour_rows_v = c.colour_rows0.p;
    L0.h_colour_ptr = c.h_colour_ptr0;
    L0.gs_ptr_v = c.gs_ptr0.p;
    L0.gs_col_v = c.gs_col0.p;
    L0.gs_val64_v = f32 ? nullptr : c.gs_val0_64.p;
    L0.gs_val32_v = f32 ? c.gs_val0_32.p : nullptr;
    int32_t nlev = 1;
    for (int32_t l = 0;; ++l) {
        Level& L = h->lev[l];
        if (L.n <= p.n_min || l == p.max_levels - 1 || l == kMaxLevels - 1) break;
        DBuf<int32_t> agg;
        int32_t rounds = 0;
        const int32_t nc = mwm_aggregate_level(c, L.n, L.A.rowptr, L.A.col, L.A.val, agg, &rounds);
        if (l == 0) L.cover_rounds = rounds;
        if ((double)nc > 0.9 * (double)L.n) break;
        L.nc = nc;
        L.agg = std::move(agg);
        build_members(c, L.n, nc, L.agg.p, L.agg_ptr, L.agg_mem);
        Level& C = h->lev[l + 1];
        C.n = nc;
        C.nnz = galerkin(c, L.n, L.A.rowptr, L.A.col, L.A.val, nc, L.agg.p, L.agg_ptr.p,
                         L.agg_mem.p, nullptr, false, C.rowptr, C.col, C.val);
        if (f32) {
            C.val32.alloc(c.mem, C.nnz);
            cast_f32(c.stream, C.nnz, C.val.p, C.val32.p);
        }
        C.A = make_csr(C, C.n, C.nnz, C.rowptr.p, C.col.p, C.val.p, f32 ? C.val32.p : nullptr);
        nlev = l + 2;
    }
    h->nlev = nlev;
    finish_hierarchy(c, *h, true);
    sync(c);
    return h.release();
}

}  // namespace pc
