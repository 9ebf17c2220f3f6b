// C ABI of the library (see include/pcamg.h): argument checks, CSR validation,
// handle life cycle, and error translation (no exception crosses the ABI).
#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>

#include "pcamg_internal.cuh"

using namespace pc;

// The opaque handle type of the ABI is the library context.
struct pcamg_ctx : public pc::Ctx {};

namespace {

thread_local std::string g_last_error;

enum : int {
    V_BAD_PTR = 1, V_BAD_COL = 2, V_UNSORTED = 4, V_NONFINITE = 8,
    V_POS_OFFDIAG = 16, V_ASYM = 32, V_ROWSUM = 64, V_NO_DIAG = 128
};

// Checks of Section 2.2's Laplacian structure, one thread per row.
__global__ void k_validate(int n, int64_t nnz, const int* __restrict__ rowptr,
                           const int* __restrict__ col, const double* __restrict__ val,
                           int* __restrict__ flags) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int b = rowptr[i], e = rowptr[i + 1];
        if (b < 0 || e < b || (int64_t)e > nnz) { atomicOr(flags, V_BAD_PTR); continue; }
        int prev = -1, f = 0;
        double diag = 0.0, sum = 0.0, amax = 0.0;
        bool has_diag = false;
        for (int k = b; k < e; ++k) {
            int j = col[k];
            double v = val[k];
            if (j < 0 || j >= n) { f |= V_BAD_COL; continue; }
            if (j <= prev) f |= V_UNSORTED;
            prev = j;
            if (!isfinite(v)) { f |= V_NONFINITE; continue; }
            sum += v;
            amax = fmax(amax, fabs(v));
            if (j == i) { diag = v; has_diag = true; continue; }
            if (v > 0.0) f |= V_POS_OFFDIAG;
            // the transposed entry must exist with the same value
            int lo = rowptr[j], hi = rowptr[j + 1] - 1;
            if (lo < 0 || (int64_t)hi >= nnz || hi < lo - 1) { f |= V_BAD_PTR; continue; }
            bool found = false;
            while (lo <= hi) {
                int mid = (lo + hi) >> 1;
                int cm = col[mid];
                if (cm == i) { found = (val[mid] == v); break; }
                if (cm < i) lo = mid + 1; else hi = mid - 1;
            }
            if (!found) f |= V_ASYM;
        }
        if (!has_diag || !(diag > 0.0)) f |= V_NO_DIAG;
        if (fabs(sum) > 1e-8 * amax) f |= V_ROWSUM;
        if (f) atomicOr(flags, f);
    }
}

__global__ void k_check_finite(int64_t n, const double* __restrict__ x, int* __restrict__ flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(x[i])) atomicOr(flag, 1);
}

pcamg_status set_err(Ctx* c, pcamg_status s, const std::string& m) {
    g_last_error = m;
    if (c) c->last_error = m;
    return s;
}

template <class F>
pcamg_status guarded(Ctx* c, F&& f) {
    try {
        return f();
    } catch (const Error& e) {
        return set_err(c, e.status, e.msg);
    } catch (const std::bad_alloc&) {
        return set_err(c, PCAMG_ERR_OOM, "host allocation failed");
    } catch (...) {
        return set_err(c, PCAMG_ERR_CUDA, "unexpected internal error");
    }
}

void check_params(const pcamg_params& p) {
    if (!(p.tol > 0.0) || p.max_iter < 0 || !(p.threshold >= 0.0) || p.numW < 0 || p.iterW < 1 ||
        p.iterV < 1 || p.nu_pre < 0 || p.nu_post < 0 || p.relax_sweeps < 0 || p.n_min < 1 ||
        p.max_levels < 1 || p.max_levels > kMaxLevels || p.round_cap < 0 ||
        (p.p1_mode != PCAMG_P1_E_SCALED && p.p1_mode != PCAMG_P1_BOOLEAN) ||
        (p.precision != PCAMG_FP64 && p.precision != PCAMG_FP32_IR) ||
        (p.start != PCAMG_START_RANDOM && p.start != PCAMG_START_USER && p.start != PCAMG_START_LEARNED &&
         p.start != PCAMG_START_MWM) ||
        (p.start == PCAMG_START_LEARNED && !p.mpnn) || p.max_resetups < -1 || p.dense_max < 1 ||
        p.dense_max > 4096 || p.tail_rows < 0 || p.l1jac_rows < 0 || p.tail_dense < 0 ||
        p.tail_dense > 3 ||
        (p.update_mode != PCAMG_UPD_REBUILD_ONLY && p.update_mode != PCAMG_UPD_ADD_CORRECTION) ||
        p.max_cover_rounds < 0 || (p.outer != PCAMG_OUTER_STATIONARY && p.outer != PCAMG_OUTER_FCG))
        fail(PCAMG_ERR_INVALID, "invalid parameters");
}

void check_finite(Ctx& c, const double* x, int64_t n, const char* what) {
    DBuf<int32_t> f;
    f.alloc(c.mem, 1);
    PC_CUDA(cudaMemsetAsync(f.p, 0, sizeof(int32_t), c.stream));
    int g = (int)std::min<int64_t>((n + 255) / 256, 4096);
    if (g < 1) g = 1;
    k_check_finite<<<g, 256, 0, c.stream>>>(n, x, f.p); ::pc::count_launches(1);
    PC_LAUNCH("check_finite");
    if (read_i32(c, f.p)) fail(PCAMG_ERR_INVALID, std::string(what) + " has a NaN or Inf entry");
}

void validate_csr(Ctx& c) {
    int32_t h[2] = {0, 0};
    PC_CUDA(cudaMemcpyAsync(&h[0], c.rowptr.p, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    PC_CUDA(cudaMemcpyAsync(&h[1], c.rowptr.p + c.n, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    sync(c);
    if (h[0] != 0 || (int64_t)h[1] != c.nnz) fail(PCAMG_ERR_INVALID, "rowptr[0] must be 0 and rowptr[n] must equal nnz");
    DBuf<int32_t> f;
    f.alloc(c.mem, 1);
    PC_CUDA(cudaMemsetAsync(f.p, 0, sizeof(int32_t), c.stream));
    int g = std::min((c.n + 255) / 256, 4096);
    k_validate<<<g, 256, 0, c.stream>>>(c.n, c.nnz, c.rowptr.p, c.col.p, c.val.p, f.p); ::pc::count_launches(1);
    PC_LAUNCH("validate");
    int fl = read_i32(c, f.p);
    if (fl & (V_BAD_PTR | V_BAD_COL | V_UNSORTED | V_NONFINITE))
        fail(PCAMG_ERR_INVALID, "malformed CSR (row pointers, column range/order or non-finite values)");
    if (fl & V_NO_DIAG) fail(PCAMG_ERR_NOT_LAPLACIAN, "a diagonal entry is missing or not positive");
    if (fl & V_POS_OFFDIAG) fail(PCAMG_ERR_NOT_LAPLACIAN, "positive off-diagonal entry");
    if (fl & V_ASYM) fail(PCAMG_ERR_NOT_LAPLACIAN, "matrix is not symmetric");
    if (fl & V_ROWSUM) fail(PCAMG_ERR_NOT_LAPLACIAN, "row sums are not zero");
}

void alloc_work(Ctx& c) {
    DBuf<double>* vs[] = {&c.w_r, &c.w_c, &c.w_e, &c.w_t1, &c.w_t2, &c.w_z, &c.w_p,
                          &c.w_q, &c.w_rold, &c.w_eh, &c.w_ein, &c.w_cin};
    for (auto* v : vs) v->alloc(c.mem, c.n);
    if (c.p.precision == PCAMG_FP32_IR) {
        c.l0_x32.alloc(c.mem, c.n); c.l0_b32.alloc(c.mem, c.n); c.l0_r32.alloc(c.mem, c.n);
    } else {
        c.l0_x64.alloc(c.mem, c.n); c.l0_b64.alloc(c.mem, c.n); c.l0_r64.alloc(c.mem, c.n);
    }
    c.npartials = std::max<int64_t>(4096, residual_partials(c.n));
    c.red.alloc(c.mem, c.npartials + 64);
    PC_CUDA(cudaMemsetAsync(c.red.p, 0, sizeof(double) * (c.npartials + 64), c.stream));
    PC_CUDA(cudaMallocHost(&c.h_red, sizeof(double) * 64));
    PC_CUDA(cudaEventCreate(&c.ev0));
    PC_CUDA(cudaEventCreate(&c.ev1));
}

// Work of a call runs on the context's stream, after the caller's prior work
// and before the caller's later work.
struct Enter {
    Ctx& c;
    explicit Enter(Ctx& cc) : c(cc) {
        PC_CUDA(cudaEventRecord(c.ev_in, c.user));
        PC_CUDA(cudaStreamWaitEvent(c.stream, c.ev_in, 0));
    }
    ~Enter() {
        if (cudaEventRecord(c.ev_out, c.stream) == cudaSuccess) cudaStreamWaitEvent(c.user, c.ev_out, 0);
        cudaGetLastError();
    }
};

Hier* get_hier(Ctx* c, int32_t hist) {
    if (hist < 0 || hist >= (int32_t)c->hist.size()) fail(PCAMG_ERR_INVALID, "hierarchy index out of range");
    return c->hist[hist];
}

template <class T>
void copy_out(Ctx& c, T* host, const T* dev, size_t count) {
    if (!host || count == 0) return;
    if (!dev) fail(PCAMG_ERR_INVALID, "requested data was not kept (set keep_setup)");
    PC_CUDA(cudaMemcpyAsync(host, dev, sizeof(T) * count, cudaMemcpyDeviceToHost, c.stream));
}

}  // namespace

namespace pc {
void set_global_error(const std::string& m) { g_last_error = m; }
}  // namespace pc

extern "C" {

PCAMG_API pcamg_status pcamg_default_params(pcamg_params* p) {
    if (!p) return set_err(nullptr, PCAMG_ERR_INVALID, "null params");
    std::memset(p, 0, sizeof(*p));
    p->tol = 1e-8;
    p->max_iter = 300;
    p->threshold = 0.4;
    p->numW = 2;
    p->iterW = 7;
    p->iterV = 4;
    p->nu_pre = 1;
    p->nu_post = 1;
    p->relax_sweeps = 8;
    p->seed = 12345;
    p->n_min = 256;
    p->max_levels = 25;
    p->round_cap = 64;
    p->p1_mode = PCAMG_P1_E_SCALED;
    p->precision = PCAMG_FP64;
    p->start = PCAMG_START_RANDOM;
    p->dense_max = 4096;
    p->use_graphs = 1;
    p->keep_setup = 0;
    p->profile = 0;
    p->tail_rows = 4096;
    p->l1jac_rows = 2147483647;
    p->tail_dense = 3;
    p->max_resetups = -1;
    p->mpnn = nullptr;
    p->update_mode = PCAMG_UPD_REBUILD_ONLY;
    return PCAMG_OK;
}

PCAMG_API pcamg_status pcamg_set_allocator(pcamg_alloc_fn alloc, pcamg_free_fn free, void* ctx) {
    if ((alloc == nullptr) != (free == nullptr))
        return set_err(nullptr, PCAMG_ERR_INVALID, "alloc and free must both be given or both be NULL");
    pc::set_allocator(alloc, free, ctx);
    return PCAMG_OK;
}

PCAMG_API pcamg_status pcamg_trim_memory(void) {
    return guarded(nullptr, [&]() -> pcamg_status {
        pc::trim_memory();
        return PCAMG_OK;
    });
}

PCAMG_API pcamg_status pcamg_setup(pcamg_handle* out, const pcamg_params* p, int32_t n, int64_t nnz,
                                   const int32_t* d_rowptr, const int32_t* d_col, const double* d_val,
                                   const double* d_e0, void* stream) {
    if (!out) return set_err(nullptr, PCAMG_ERR_INVALID, "null output handle");
    *out = nullptr;
    std::unique_ptr<pcamg_ctx> c(new pcamg_ctx());
    pcamg_status st = guarded(c.get(), [&]() -> pcamg_status {
        if (!p) fail(PCAMG_ERR_INVALID, "null params");
        check_params(*p);
        if (n < 2 || nnz < n || nnz >= ((int64_t)1 << 31) || !d_rowptr || !d_col || !d_val)
            fail(PCAMG_ERR_INVALID, "invalid sizes or null CSR pointers");
        if (p->start == PCAMG_START_USER && !d_e0) fail(PCAMG_ERR_INVALID, "start == USER needs d_e0");
        c->p = *p;
        c->user = (cudaStream_t)stream;
        PC_CUDA(cudaStreamCreateWithFlags(&c->own.s, cudaStreamNonBlocking));
        c->stream = c->own.s;
        c->mem.stream = c->stream;
        PC_CUDA(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
        PC_CUDA(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
        Enter guard(*c);
        c->n = n;
        c->nnz = nnz;
        c->rowptr.alloc(c->mem, (size_t)n + 1);
        c->col.alloc(c->mem, nnz);
        c->val.alloc(c->mem, nnz);
        PC_CUDA(cudaMemcpyAsync(c->rowptr.p, d_rowptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, c->stream));
        PC_CUDA(cudaMemcpyAsync(c->col.p, d_col, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, c->stream));
        PC_CUDA(cudaMemcpyAsync(c->val.p, d_val, sizeof(double) * nnz, cudaMemcpyDeviceToDevice, c->stream));
        validate_csr(*c);
        if (c->p.precision == PCAMG_FP32_IR) {
            c->val32.alloc(c->mem, nnz);
            cast_f32(c->stream, nnz, c->val.p, c->val32.p);
        }
        alloc_work(*c);
        c->colour0.alloc(c->mem, n);
        c->ncolour0 = colour_smoother(*c, n, c->rowptr.p, c->col.p, c->p.seed, c->colour0.p);
        colour_lists(*c, n, c->colour0.p, c->ncolour0, c->colour_rows0, c->h_colour_ptr0);
        // rows grouped by colour, for the streaming smoother (FP64 for the start
        // vector and the FP64 cycle; FP32 for the FP32 cycle), when its launches
        // are large enough to pay off
        if (use_stream(n / std::max(1, c->ncolour0), lanes_per_row(n, nnz))) {
            permute_rows<double>(*c, n, c->colour_rows0.p, c->rowptr.p, c->col.p, c->val.p, c->gs_ptr0,
                                 c->gs_col0, c->gs_val0_64);
            if (c->p.precision == PCAMG_FP32_IR) {
                DBuf<int32_t> p2, c2;
                permute_rows<float>(*c, n, c->colour_rows0.p, c->rowptr.p, c->col.p, c->val.p, p2, c2,
                                    c->gs_val0_32);
            }
            // the cycles then keep the finest level in colour order, unless it
            // joins the coarse tail (which works in row order): columns of the
            // copy become positions, so a colour's rows read b and write x
            // contiguously and gather their neighbours by position
            if (c->p.tail_rows == 0 || n > c->p.tail_rows / 2) {
                c->iperm0.alloc(c->mem, n);
                invert_perm(c->stream, n, c->colour_rows0.p, c->iperm0.p);
                map_index(c->stream, nnz, c->iperm0.p, c->gs_col0.p, c->gs_col0.p);
                mark_diagonal(c->stream, n, c->gs_ptr0.p, c->gs_col0.p);
                c->perm0 = true;
            }
        }
        if (c->p.start == PCAMG_START_MWM) {
            c->hist.push_back(build_hierarchy_mwm(*c));
            c->last_e = nullptr;
            sync(*c);
            return PCAMG_OK;
        }
        if (c->p.start == PCAMG_START_USER) {
            check_finite(*c, d_e0, n, "start vector");
            copy(c->stream, n, d_e0, c->w_e.p);
        } else if (c->p.start == PCAMG_START_LEARNED) {
            start_vector(*c, c->w_t2.p);
            mpnn_forward(*c, *reinterpret_cast<pc::Mpnn*>(c->p.mpnn), c->w_t2.p, c->w_e.p);
        } else {
            start_vector(*c, c->w_e.p);
        }
        c->hist.push_back(build_hierarchy(*c, c->w_e.p));
        c->last_e = c->w_e.p;
        sync(*c);
        return PCAMG_OK;
    });
    if (st == PCAMG_OK) *out = c.release();
    else { try { cudaStreamSynchronize((cudaStream_t)stream); } catch (...) {} }
    return st;
}

PCAMG_API pcamg_status pcamg_adapt(pcamg_handle h, const double* d_e) {
    if (!h || !d_e) return set_err(h, PCAMG_ERR_INVALID, "null argument");
    return guarded(h, [&]() -> pcamg_status {
        Enter guard(*h);
        check_finite(*h, d_e, h->n, "smooth error");
        copy(h->stream, h->n, d_e, h->w_eh.p);
        h->hist.push_back(build_hierarchy(*h, h->w_eh.p));
        h->last_e = h->w_eh.p;
        return PCAMG_OK;
    });
}

PCAMG_API pcamg_status pcamg_solve(pcamg_handle h, const double* d_b, double* d_x, pcamg_stats* st) {
    if (!h || !d_b || !d_x) return set_err(h, PCAMG_ERR_INVALID, "null argument");
    return guarded(h, [&]() -> pcamg_status {
        Enter guard(*h);
        check_finite(*h, d_b, h->n, "b");
        check_finite(*h, d_x, h->n, "x");
        pcamg_status s = solve(*h, d_b, d_x, st);
        if (s == PCAMG_ERR_NOT_CONVERGED) set_err(h, s, "max_iter reached before tol");
        if (s == PCAMG_ERR_DIVERGED) set_err(h, s, "residual became NaN/Inf");
        return s;
    });
}

PCAMG_API pcamg_status pcamg_solve_zero_rhs(pcamg_handle h, double* d_x, pcamg_stats* st) {
    if (!h || !d_x) return set_err(h, PCAMG_ERR_INVALID, "null argument");
    return guarded(h, [&]() -> pcamg_status {
        Enter guard(*h);
        check_finite(*h, d_x, h->n, "x");
        return solve_zero_rhs(*h, d_x, st);
    });
}

PCAMG_API pcamg_status pcamg_solve_multi(pcamg_handle h, int32_t k, const double* d_B, double* d_X,
                                         int32_t* iters, double* rel_res) {
    if (!h || !d_B || !d_X || k < 1) return set_err(h, PCAMG_ERR_INVALID, "invalid argument");
    return guarded(h, [&]() -> pcamg_status {
        Enter guard(*h);
        for (int32_t j = 0; j < k; ++j) {
            check_finite(*h, d_B + (size_t)j * h->n, h->n, "B");
            check_finite(*h, d_X + (size_t)j * h->n, h->n, "X");
        }
        return solve_multi(*h, k, d_B, d_X, iters, rel_res);
    });
}

PCAMG_API pcamg_status pcamg_solve_host(const pcamg_params* p, int32_t n, int64_t nnz,
                                        const int32_t* h_rowptr, const int32_t* h_col,
                                        const double* h_val, const double* h_b, double* h_x,
                                        pcamg_stats* st, void* stream) {
    if (!p || !h_rowptr || !h_col || !h_val || !h_b || !h_x || n < 2 || nnz < n)
        return set_err(nullptr, PCAMG_ERR_INVALID, "invalid argument");
    Ctx tmp;
    tmp.stream = (cudaStream_t)stream;
    tmp.user = tmp.stream;
    tmp.mem.stream = tmp.stream;
    pcamg_handle h = nullptr;
    pcamg_status s = guarded(&tmp, [&]() -> pcamg_status {
        DBuf<int32_t> rp, ci;
        DBuf<double> v, b, x;
        rp.alloc(tmp.mem, (size_t)n + 1); ci.alloc(tmp.mem, nnz); v.alloc(tmp.mem, nnz);
        b.alloc(tmp.mem, n); x.alloc(tmp.mem, n);
        PC_CUDA(cudaMemcpyAsync(rp.p, h_rowptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, tmp.stream));
        PC_CUDA(cudaMemcpyAsync(ci.p, h_col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, tmp.stream));
        PC_CUDA(cudaMemcpyAsync(v.p, h_val, sizeof(double) * nnz, cudaMemcpyHostToDevice, tmp.stream));
        PC_CUDA(cudaMemcpyAsync(b.p, h_b, sizeof(double) * n, cudaMemcpyHostToDevice, tmp.stream));
        PC_CUDA(cudaMemcpyAsync(x.p, h_x, sizeof(double) * n, cudaMemcpyHostToDevice, tmp.stream));
        pcamg_status r = pcamg_setup(&h, p, n, nnz, rp.p, ci.p, v.p, nullptr, stream);
        if (r != PCAMG_OK) fail(r, g_last_error);
        r = pcamg_solve(h, b.p, x.p, st);
        std::string msg = (r != PCAMG_OK) ? h->last_error : std::string();
        pcamg_destroy(h);
        h = nullptr;
        PC_CUDA(cudaMemcpyAsync(h_x, x.p, sizeof(double) * n, cudaMemcpyDeviceToHost, tmp.stream));
        sync(tmp);
        if (r != PCAMG_OK) set_err(nullptr, r, msg);
        return r;
    });
    if (h) pcamg_destroy(h);
    return s;
}

PCAMG_API pcamg_status pcamg_cycle(pcamg_handle h, int32_t hist, int32_t gamma, const double* d_r,
                                   double* d_c) {
    if (!h || !d_r || !d_c || (gamma != 1 && gamma != 2)) return set_err(h, PCAMG_ERR_INVALID, "invalid argument");
    return guarded(h, [&]() -> pcamg_status {
        Enter guard(*h);
        Hier* hh = get_hier(h, hist);
        cycle(*h, *hh, gamma, d_r, d_c);
        sync(*h);
        return PCAMG_OK;
    });
}

PCAMG_API pcamg_status pcamg_smooth_error(pcamg_handle h, const double* d_r, double* d_e) {
    if (!h || !d_r || !d_e) return set_err(h, PCAMG_ERR_INVALID, "null argument");
    return guarded(h, [&]() -> pcamg_status {
        Enter guard(*h);
        smooth_error(*h, d_r, d_e);
        sync(*h);
        return PCAMG_OK;
    });
}

PCAMG_API pcamg_status pcamg_start_vector(pcamg_handle h, double* d_e) {
    if (!h || !d_e) return set_err(h, PCAMG_ERR_INVALID, "null argument");
    return guarded(h, [&]() -> pcamg_status {
        Enter guard(*h);
        start_vector(*h, d_e);
        sync(*h);
        return PCAMG_OK;
    });
}

PCAMG_API pcamg_status pcamg_last_smooth_error(pcamg_handle h, double* d_e) {
    if (!h || !d_e) return set_err(h, PCAMG_ERR_INVALID, "null argument");
    return guarded(h, [&]() -> pcamg_status {
        if (!h->last_e) fail(PCAMG_ERR_INVALID, "the newest hierarchy was not built from a smooth error (MWM)");
        Enter guard(*h);
        copy(h->stream, h->n, h->last_e, d_e);
        sync(*h);
        return PCAMG_OK;
    });
}

// ---- learned start vector
static void check_params_finite(const float* w) {
    for (int64_t i = 0; i < kMpnnParams; ++i)
        if (!std::isfinite(w[i])) fail(PCAMG_ERR_INVALID, "mpnn parameters are not finite");
}

PCAMG_API int64_t pcamg_mpnn_num_params(void) { return kMpnnParams; }

PCAMG_API pcamg_status pcamg_mpnn_create(pcamg_mpnn* out, const float* h_params) {
    if (!out || !h_params) return set_err(nullptr, PCAMG_ERR_INVALID, "null argument");
    *out = nullptr;
    return guarded(nullptr, [&]() -> pcamg_status {
        check_params_finite(h_params);
        *out = reinterpret_cast<pcamg_mpnn>(mpnn_create(h_params));
        return PCAMG_OK;
    });
}

PCAMG_API void pcamg_mpnn_destroy(pcamg_mpnn m) { mpnn_destroy(reinterpret_cast<pc::Mpnn*>(m)); }

PCAMG_API pcamg_status pcamg_mpnn_get_params(pcamg_mpnn m, float* h_params) {
    if (!m || !h_params) return set_err(nullptr, PCAMG_ERR_INVALID, "null argument");
    return guarded(nullptr, [&]() -> pcamg_status {
        mpnn_get_params(*reinterpret_cast<pc::Mpnn*>(m), h_params);
        return PCAMG_OK;
    });
}

PCAMG_API pcamg_status pcamg_mpnn_set_params(pcamg_mpnn m, const float* h_params) {
    if (!m || !h_params) return set_err(nullptr, PCAMG_ERR_INVALID, "null argument");
    return guarded(nullptr, [&]() -> pcamg_status {
        check_params_finite(h_params);
        mpnn_set_params(*reinterpret_cast<pc::Mpnn*>(m), h_params);
        return PCAMG_OK;
    });
}

PCAMG_API pcamg_status pcamg_mpnn_get_grad(pcamg_mpnn m, float* h_grad) {
    if (!m || !h_grad) return set_err(nullptr, PCAMG_ERR_INVALID, "null argument");
    return guarded(nullptr, [&]() -> pcamg_status {
        mpnn_get_grad(*reinterpret_cast<pc::Mpnn*>(m), h_grad);
        return PCAMG_OK;
    });
}

PCAMG_API pcamg_status pcamg_mpnn_forward(pcamg_mpnn m, pcamg_handle g, const double* d_u, double* d_y) {
    if (!m || !g || !d_u || !d_y) return set_err(g, PCAMG_ERR_INVALID, "null argument");
    return guarded(g, [&]() -> pcamg_status {
        Enter guard(*g);
        mpnn_forward(*g, *reinterpret_cast<pc::Mpnn*>(m), d_u, d_y);
        return PCAMG_OK;
    });
}

PCAMG_API pcamg_status pcamg_mpnn_loss_grad(pcamg_mpnn m, pcamg_handle g, const double* d_u,
                                            const double* d_target, double* h_loss) {
    if (!m || !g || !d_u || !d_target || !h_loss) return set_err(g, PCAMG_ERR_INVALID, "null argument");
    return guarded(g, [&]() -> pcamg_status {
        Enter guard(*g);
        *h_loss = mpnn_loss_grad(*g, *reinterpret_cast<pc::Mpnn*>(m), d_u, d_target);
        return PCAMG_OK;
    });
}

PCAMG_API pcamg_status pcamg_mpnn_adam_step(pcamg_mpnn m, float lr) {
    if (!m || !(lr > 0.0f) || !std::isfinite(lr)) return set_err(nullptr, PCAMG_ERR_INVALID, "invalid argument");
    return guarded(nullptr, [&]() -> pcamg_status {
        mpnn_adam(*reinterpret_cast<pc::Mpnn*>(m), lr);
        return PCAMG_OK;
    });
}

static const char kMpnnHead[] = "{\"format\": \"pcamg-mpnn\", \"version\": 1, \"dtype\": \"f32-le\", \"params\": ";

static bool little_endian() {
    const uint32_t one = 1;
    unsigned char b;
    std::memcpy(&b, &one, 1);
    return b == 1;
}

static std::string mpnn_header() { return std::string(kMpnnHead) + std::to_string((long long)kMpnnParams) + "}\n"; }

PCAMG_API pcamg_status pcamg_mpnn_save(pcamg_mpnn m, const char* path) {
    if (!m || !path) return set_err(nullptr, PCAMG_ERR_INVALID, "null argument");
    return guarded(nullptr, [&]() -> pcamg_status {
        if (!little_endian()) fail(PCAMG_ERR_UNSUPPORTED, "mpnn files are little-endian");
        std::vector<float> w(kMpnnParams);
        mpnn_get_params(*reinterpret_cast<pc::Mpnn*>(m), w.data());
        FILE* f = std::fopen(path, "wb");
        if (!f) fail(PCAMG_ERR_INVALID, "cannot open file for writing");
        const std::string head = mpnn_header();
        bool ok = std::fwrite(head.data(), 1, head.size(), f) == head.size() &&
                  std::fwrite(w.data(), sizeof(float), w.size(), f) == w.size();
        ok = (std::fclose(f) == 0) && ok;
        if (!ok) fail(PCAMG_ERR_INVALID, "write failed");
        return PCAMG_OK;
    });
}

PCAMG_API pcamg_status pcamg_mpnn_load(pcamg_mpnn* out, const char* path) {
    if (!out || !path) return set_err(nullptr, PCAMG_ERR_INVALID, "null argument");
    *out = nullptr;
    return guarded(nullptr, [&]() -> pcamg_status {
        if (!little_endian()) fail(PCAMG_ERR_UNSUPPORTED, "mpnn files are little-endian");
        FILE* f = std::fopen(path, "rb");
        if (!f) fail(PCAMG_ERR_INVALID, "cannot open file");
        const std::string head = mpnn_header();
        std::string got(head.size(), '\0');
        std::vector<float> w(kMpnnParams);
        bool ok = std::fread(&got[0], 1, got.size(), f) == got.size() && got == head &&
                  std::fread(w.data(), sizeof(float), w.size(), f) == w.size();
        std::fclose(f);
        if (!ok) fail(PCAMG_ERR_INVALID, "not a pcamg-mpnn file of this layout");
        check_params_finite(w.data());
        *out = reinterpret_cast<pcamg_mpnn>(mpnn_create(w.data()));
        return PCAMG_OK;
    });
}

PCAMG_API int32_t pcamg_num_hierarchies(pcamg_handle h) { return h ? (int32_t)h->hist.size() : -1; }

PCAMG_API int32_t pcamg_num_levels(pcamg_handle h, int32_t hist) {
    if (!h || hist < 0 || hist >= (int32_t)h->hist.size()) return -1;
    return h->hist[hist]->nlev;
}

PCAMG_API pcamg_status pcamg_level_sizes(pcamg_handle h, int32_t hist, int32_t lev, int64_t sizes[8]) {
    if (!h || !sizes) return set_err(h, PCAMG_ERR_INVALID, "null argument");
    return guarded(h, [&]() -> pcamg_status {
        Hier* hh = get_hier(h, hist);
        if (lev < 0 || lev >= hh->nlev) fail(PCAMG_ERR_INVALID, "level out of range");
        Level& L = hh->lev[lev];
        sizes[0] = L.n;
        sizes[1] = L.nnz;
        sizes[2] = (lev + 1 < hh->nlev) ? L.nc : 0;
        sizes[3] = L.ncolour;
        sizes[4] = L.cover_rounds;
        sizes[5] = L.leftover_rounds;
        sizes[6] = hh->npinned;
        sizes[7] = L.tnnz;
        return PCAMG_OK;
    });
}

PCAMG_API pcamg_status pcamg_export_level(pcamg_handle h, int32_t hist, int32_t lev, int32_t* agg,
                                          int32_t* nbr0, int32_t* nbr1, int32_t* rowptr, int32_t* col,
                                          double* val, double* pval, int32_t* colour) {
    if (!h) return set_err(h, PCAMG_ERR_INVALID, "null handle");
    return guarded(h, [&]() -> pcamg_status {
        Enter guard(*h);
        Hier* hh = get_hier(h, hist);
        if (lev < 0 || lev >= hh->nlev) fail(PCAMG_ERR_INVALID, "level out of range");
        Level& L = hh->lev[lev];
        bool coarsest = lev + 1 == hh->nlev;
        if (agg && !coarsest) copy_out(*h, agg, L.agg.p, L.n);
        copy_out(*h, nbr0, L.nbr0.p, nbr0 ? L.n : 0);
        copy_out(*h, nbr1, L.nbr1.p, nbr1 ? L.n : 0);
        copy_out(*h, rowptr, L.A.rowptr, (size_t)L.n + 1);
        copy_out(*h, col, L.A.col, L.nnz);
        copy_out(*h, val, L.A.val, L.nnz);
        if (pval && L.pval.p) copy_out(*h, pval, L.pval.p, L.n);
        if (colour && L.colour_v) copy_out(*h, colour, L.colour_v, L.n);
        sync(*h);
        return PCAMG_OK;
    });
}

PCAMG_API pcamg_status pcamg_export_reweighted(pcamg_handle h, int32_t hist, int32_t lev, int32_t* ptr,
                                               int32_t* col, double* w) {
    if (!h) return set_err(h, PCAMG_ERR_INVALID, "null handle");
    return guarded(h, [&]() -> pcamg_status {
        Hier* hh = get_hier(h, hist);
        if (lev < 0 || lev >= hh->nlev) fail(PCAMG_ERR_INVALID, "level out of range");
        Level& L = hh->lev[lev];
        if (!L.tptr.p) fail(PCAMG_ERR_INVALID, "reweighted graph was not kept (set keep_setup)");
        Enter guard(*h);
        copy_out(*h, ptr, L.tptr.p, (size_t)L.n + 1);
        copy_out(*h, col, L.tcol.p, L.tnnz);
        copy_out(*h, w, L.tw.p, L.tnnz);
        sync(*h);
        return PCAMG_OK;
    });
}

PCAMG_API int64_t pcamg_kernel_launches(void) { return launch_count(); }

PCAMG_API const char* pcamg_last_error(pcamg_handle h) {
    return h ? h->last_error.c_str() : g_last_error.c_str();
}

PCAMG_API const char* pcamg_status_string(pcamg_status s) {
    switch (s) {
        case PCAMG_OK: return "OK";
        case PCAMG_ERR_INVALID: return "INVALID";
        case PCAMG_ERR_NOT_LAPLACIAN: return "NOT_LAPLACIAN";
        case PCAMG_ERR_OOM: return "OOM";
        case PCAMG_ERR_CUDA: return "CUDA";
        case PCAMG_ERR_ROUND_CAP: return "ROUND_CAP";
        case PCAMG_ERR_SINGULAR: return "SINGULAR";
        case PCAMG_ERR_NOT_CONVERGED: return "NOT_CONVERGED";
        case PCAMG_ERR_DIVERGED: return "DIVERGED";
        case PCAMG_ERR_COARSE_TOO_BIG: return "COARSE_TOO_BIG";
        case PCAMG_ERR_UNSUPPORTED: return "UNSUPPORTED";
    }
    return "UNKNOWN";
}

PCAMG_API void pcamg_destroy(pcamg_handle h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    delete h;
    cudaGetLastError();
}

PCAMG_API pcamg_status pcamg_residual(int32_t n, const int32_t* d_rowptr, const int32_t* d_col,
                                      const double* d_val, const double* d_x, const double* d_b,
                                      double* d_r, double* d_norm2, void* stream) {
    if (n < 1 || !d_rowptr || !d_col || !d_val || !d_x || !d_b || !d_r)
        return set_err(nullptr, PCAMG_ERR_INVALID, "invalid argument");
    Ctx tmp;
    tmp.stream = (cudaStream_t)stream;
    tmp.mem.stream = tmp.stream;
    return guarded(nullptr, [&]() -> pcamg_status {
        int32_t nnz = 0;
        PC_CUDA(cudaMemcpyAsync(&nnz, d_rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, tmp.stream));
        sync(tmp);
        Csr A;
        A.n = n; A.nnz = nnz; A.rowptr = d_rowptr; A.col = d_col; A.val = d_val;
        A.lpr = lanes_per_row(n, nnz);
        DBuf<double> part;
        if (d_norm2) part.alloc(tmp.mem, std::max<int64_t>(4096, residual_partials(n)));
        residual64(tmp.stream, A, d_x, d_b, d_r, part.p, d_norm2);
        sync(tmp);
        return PCAMG_OK;
    });
}

PCAMG_API pcamg_status pcamg_residual_f32(int32_t n, const int32_t* d_rowptr, const int32_t* d_col,
                                          const float* d_val, const float* d_x, const float* d_b,
                                          float* d_r, void* stream) {
    if (n < 1 || !d_rowptr || !d_col || !d_val || !d_x || !d_b || !d_r)
        return set_err(nullptr, PCAMG_ERR_INVALID, "invalid argument");
    Ctx tmp;
    tmp.stream = (cudaStream_t)stream;
    tmp.mem.stream = tmp.stream;
    return guarded(nullptr, [&]() -> pcamg_status {
        int32_t nnz = 0;
        PC_CUDA(cudaMemcpyAsync(&nnz, d_rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, tmp.stream));
        sync(tmp);
        Csr A;
        A.n = n; A.nnz = nnz; A.rowptr = d_rowptr; A.col = d_col; A.val32 = d_val;
        A.lpr = lanes_per_row(n, nnz);
        residual32(tmp.stream, A, d_x, d_b, d_r);
        sync(tmp);
        return PCAMG_OK;
    });
}

PCAMG_API pcamg_status pcamg_uniform(uint64_t seed, int64_t n, double* d_out, void* stream) {
    if (n < 0 || (n > 0 && !d_out)) return set_err(nullptr, PCAMG_ERR_INVALID, "invalid argument");
    return guarded(nullptr, [&]() -> pcamg_status {
        philox_uniform((cudaStream_t)stream, seed, n, d_out);
        PC_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
        return PCAMG_OK;
    });
}

PCAMG_API pcamg_status pcamg_colour(int32_t n, const int32_t* d_rowptr, const int32_t* d_col,
                                    uint64_t seed, int32_t* d_colour, int32_t* ncolour, void* stream) {
    if (n < 1 || !d_rowptr || !d_col || !d_colour || !ncolour)
        return set_err(nullptr, PCAMG_ERR_INVALID, "invalid argument");
    Ctx tmp;
    tmp.stream = (cudaStream_t)stream;
    tmp.mem.stream = tmp.stream;
    return guarded(nullptr, [&]() -> pcamg_status {
        *ncolour = colour_graph(tmp, n, d_rowptr, d_col, seed, d_colour);
        sync(tmp);
        return PCAMG_OK;
    });
}

}  // extern "C"
