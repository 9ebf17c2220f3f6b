// Cycles and the adaptive drivers:
//  * the multigrid cycle of Section 4 (Gauss-Seidel pre/post smoothing in
//    colour order, restriction by P^T, prolongation by P, dense coarsest solve),
//    run in FP64 or in FP32 inside FP64 iterative refinement, optionally
//    captured once per hierarchy in a CUDA graph;
//  * ApproximateSmoothError (Alg. 2): flexible PCG with a W-cycle or the
//    symmetric composite of V-cycles over all hierarchies;
//  * AdaptiveAMG for general b (Alg. 5) and for b = 0 (Alg. 6).
#include <atomic>
#include <chrono>
#include <mutex>
#include <cmath>
#include <cstring>

#include "pcamg_internal.cuh"

namespace pc {

// ---------------------------------------------------------------- basics
void fail(pcamg_status s, const std::string& msg) { throw Error{s, msg}; }

static std::atomic<int64_t> g_launches{0};
static thread_local int64_t* t_capture_acc = nullptr;
void count_launches(int64_t k) {
    if (t_capture_acc) *t_capture_acc += k;   // recorded into a graph, not run yet
    else g_launches.fetch_add(k, std::memory_order_relaxed);
}
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
bool capturing() { return t_capture_acc != nullptr; }

static thread_local bool t_pdl_prev_copy = false;
bool pdl_next() {
    const bool ok = t_capture_acc != nullptr && !t_pdl_prev_copy;
    t_pdl_prev_copy = false;
    return ok;
}
void pdl_after_copy() { t_pdl_prev_copy = true; }

void check_cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    cudaGetLastError();
    pcamg_status s = (e == cudaErrorMemoryAllocation) ? PCAMG_ERR_OOM : PCAMG_ERR_CUDA;
    throw Error{s, std::string(what) + ": " + cudaGetErrorString(e)};
}

// ---------------------------------------------------------------- device memory
static std::mutex g_alloc_mu;
static pcamg_alloc_fn g_afn = nullptr;
static pcamg_free_fn g_ffn = nullptr;
static void* g_actx = nullptr;
static cudaMemPool_t g_pool[64] = {};

void set_allocator(pcamg_alloc_fn a, pcamg_free_fn f, void* ctx) {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_afn = a;
    g_ffn = f;
    g_actx = ctx;
}

// The library pool of the current device: freed memory stays cached (release
// threshold unlimited) instead of going back to the device at every
// synchronisation.
static cudaMemPool_t library_pool() {
    int dev = 0;
    PC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(PCAMG_ERR_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        PC_CUDA(cudaMemPoolCreate(&pool, &props));
        uint64_t keep = UINT64_MAX;
        PC_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        g_pool[dev] = pool;
    }
    return g_pool[dev];
}

void trim_memory() {
    int dev = 0;
    PC_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        if (dev >= 0 && dev < 64) pool = g_pool[dev];
    }
    if (pool) PC_CUDA(cudaMemPoolTrimTo(pool, 0));
}

Mem::Mem() {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    afn = g_afn;
    ffn = g_ffn;
    actx = g_actx;
}

void* Mem::alloc(size_t bytes) {
    void* p = nullptr;
    if (afn) {
        p = afn(bytes, (void*)stream, actx);
        if (!p) throw Error{PCAMG_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed"};
    } else {
        cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, library_pool(), stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error{PCAMG_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed"};
        }
    }
    live += bytes;
    if (live > peak) peak = live;
    return p;
}

void Mem::release(void* p, size_t bytes) {
    if (ffn) ffn(p, (void*)stream, actx);
    else cudaFreeAsync(p, stream);
    live -= bytes;
}

Ctx::~Ctx() {
    for (Hier* h : hist) delete h;
    hist.clear();
    for (cudaEvent_t e : cyc_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : cyc_tmpl) if (e) cudaEventDestroy(e);
    if (h_red) cudaFreeHost(h_red);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
}

void sync(Ctx& c) { PC_CUDA(cudaStreamSynchronize(c.stream)); }

template <class T>
void d2h(Ctx& c, T* host, const T* dev, size_t count) {
    if (count == 0) return;
    PC_CUDA(cudaMemcpyAsync(host, dev, sizeof(T) * count, cudaMemcpyDeviceToHost, c.stream));
    sync(c);
}
template void d2h<int32_t>(Ctx&, int32_t*, const int32_t*, size_t);
template void d2h<int64_t>(Ctx&, int64_t*, const int64_t*, size_t);
template void d2h<double>(Ctx&, double*, const double*, size_t);

int64_t read_i64(Ctx& c, const int64_t* dev) {
    int64_t v = 0;
    d2h(c, &v, dev, 1);
    return v;
}
int32_t read_i32(Ctx& c, const int32_t* dev) {
    int32_t v = 0;
    d2h(c, &v, dev, 1);
    return v;
}
double read_f64(Ctx& c, const double* dev) {
    double v = 0;
    d2h(c, &v, dev, 1);
    return v;
}

// scalar slots after the reduction partials
enum Slot { S_T0 = 0, S_T1, S_T2, S_NORM2, S_RZ, S_PQ, S_ALPHA, S_NUM, S_BETA, S_SCALE, S_INV, S_SUM,
            S_FRZ, S_FPQ, S_FALPHA, S_FNUM, S_FDEN, S_FBETA, S_NSLOTS };
static double* slot(Ctx& c, int k) { return c.red.p + c.npartials + k; }
static double* partials(Ctx& c) { return c.red.p; }

double* red_partials(Ctx& c) { return partials(c); }
double* mpnn_slots(Ctx& c) { return slot(c, 32); }
const double* norm_slot(Ctx& c) { return slot(c, S_T1); }

void normalise_orth(Ctx& c, const double* e, double* out) {
    cudaStream_t s = c.stream;
    if (out != e) copy(s, c.n, e, out);
    sum(s, c.n, out, partials(c), slot(c, S_SUM));
    sub_mean(s, c.n, out, slot(c, S_SUM));
    dot(s, c.n, out, out, partials(c), slot(c, S_T0));
    scalar_ops(s, SOP_SQRT, slot(c, 0), S_T0, 0, S_T1);
    scale_dev(s, c.n, out, nullptr, slot(c, S_T1));  // out *= 1 / ||out||
}

// ---------------------------------------------------------------- cycle
template <class T>
struct LV;
template <>
struct LV<double> {
    static double* x(Level& L) { return L.x64v; }
    static double* b(Level& L) { return L.b64v; }
    static double* r(Level& L) { return L.r64v; }
    static const double* pv(Level& L) { return L.perm ? L.pvalp.p : L.pval.p; }
};
template <>
struct LV<float> {
    static float* x(Level& L) { return L.x32v; }
    static float* b(Level& L) { return L.b32v; }
    static float* r(Level& L) { return L.r32v; }
    static const float* pv(Level& L) { return L.perm ? L.pvalp32.p : L.pval32.p; }
};

// The buffer that holds level L's iterate now, and the other one (l1-Jacobi
// levels with a second buffer alternate between them)
template <class T>
static T* xalt(Level& L) { if constexpr (sizeof(T) == 8) return L.xa64.p; else return L.xa32.p; }
template <class T>
static T* X(Level& L) { return L.xcur ? xalt<T>(L) : LV<T>::x(L); }

template <class T>
static void smooth(Ctx& c, Level& L, const T* b, T* x, bool forward, bool skip_first = false) {
    if (L.jac && xalt<T>(L)) {   // l1-Jacobi in one pass: x' = x + (b - A x) / d
        const T* d;
        if constexpr (sizeof(T) == 8) d = L.dl1_64.p; else d = L.dl1_32.p;
        T* out = L.xcur ? LV<T>::x(L) : xalt<T>(L);
        jacobi_sweep<T>(c.stream, L.A, x, b, d, out);
        L.xcur ^= 1;
        return;
    }
    if (L.jac) {   // l1-Jacobi: x += (b - A x) / d
        T* r;
        const T* d;
        if constexpr (sizeof(T) == 8) { r = L.r64v; d = L.dl1_64.p; } else { r = L.r32v; d = L.dl1_32.p; }
        if constexpr (sizeof(T) == 8) residual64(c.stream, L.A, x, b, r, nullptr, nullptr);
        else residual32(c.stream, L.A, x, b, r);
        jacobi_update<T>(c.stream, L.n, r, d, x);
        return;
    }
    const T* pv;
    if constexpr (sizeof(T) == 8) pv = L.gs_val64_v; else pv = L.gs_val32_v;
    for (int32_t t = skip_first ? 1 : 0; t < L.ncolour; ++t) {
        int32_t k = forward ? t : L.ncolour - 1 - t;
        int32_t beg = L.h_colour_ptr[k], end = L.h_colour_ptr[k + 1];
        if (pv) gs_colour_perm<T>(c.stream, beg, end, L.perm ? nullptr : L.colour_rows_v, L.gs_ptr_v, L.gs_col_v, pv, b, x);
        else gs_colour<T>(c.stream, L.A, L.colour_rows_v + beg, end - beg, b, x);
    }
}

// Rows the prolongation must update: on a level kept in colour order and
// smoothed by Gauss-Seidel after the coarse correction, the backward post-sweep
// begins with the last colour, whose new values do not read their own old x:
// the prolongation of those rows (the last range of the order) would be
// overwritten unread.
static int32_t prolong_rows(const Level& L, int32_t nu_post) {
    if (L.perm && !L.jac && nu_post >= 1 && L.ncolour >= 2) return L.h_colour_ptr[L.ncolour - 1];
    return L.n;
}

// ---------------------------------------------------------------- live timing
// params.profile bit 1: CUDA events around the finest-level residual of every
// V-cycle. Inside a captured graph they are event-record nodes, retargeted to a
// fresh pair of pool events before each replay; without graphs the pool events
// are recorded on the stream directly. The pairs are resolved when the solve
// ends (pcamg_stats.cyc_*).
static constexpr size_t kMaxProfEvents = 1 << 16;   // events beyond this are not recorded (4 per V-cycle)

static cudaEvent_t pool_event(Ctx& c) {
    if (c.cyc_used >= kMaxProfEvents) return nullptr;
    if (c.cyc_used == c.cyc_ev.size()) {
        cudaEvent_t e = nullptr;
        PC_CUDA(cudaEventCreate(&e));
        c.cyc_ev.push_back(e);
    }
    return c.cyc_ev[c.cyc_used++];
}

static void prof_mark(Ctx& c, Hier& h, int k) {
    if (capturing()) {
        if (!c.cyc_tmpl[k]) PC_CUDA(cudaEventCreate(&c.cyc_tmpl[k]));
        PC_CUDA(cudaEventRecordWithFlags(c.cyc_tmpl[k], c.stream, cudaEventRecordExternal));
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        PC_CUDA(cudaStreamGetCaptureInfo(c.stream, &cs, nullptr, nullptr, &deps, nullptr, &nd));
        if (nd != 1) fail(PCAMG_ERR_CUDA, "profiling node not found in the captured cycle");
        h.prof_node[c.cur_kind][k] = deps[0];
        pdl_after_copy();   // the next kernel follows a non-kernel node
    } else if (cudaEvent_t e = pool_event(c)) {
        PC_CUDA(cudaEventRecord(e, c.stream));
    }
}

// events come in fours per V-cycle: pre-sweep start, end, residual start, end
static void prof_resolve(Ctx& c) {
    for (size_t i = 0; i + 3 < c.cyc_used; i += 4) {
        float ms = 0.f;
        PC_CUDA(cudaEventElapsedTime(&ms, c.cyc_ev[i], c.cyc_ev[i + 1]));
        c.gs_ms += ms;
        c.gs_sweeps += 1;
        PC_CUDA(cudaEventElapsedTime(&ms, c.cyc_ev[i + 2], c.cyc_ev[i + 3]));
        c.cyc_ms += ms;
        c.cyc_launches += 1;
    }
    c.cyc_used = 0;
}

// One visit of level l. `fresh`: x arrives as the result of one l1-Jacobi
// sweep from zero (the parent wrote b/d), so the first pre-sweep is done.
// `first`: x is zero or that fresh start, i.e. this is the child's first visit.
template <class T>
static void cycle_level(Ctx& c, Hier& h, int32_t l, int gamma, bool fresh, bool first) {
    cudaStream_t s = c.stream;
    Level& L = h.lev[l];
    if (l == h.lt && h.tail_op[gamma - 1].p) {
        // the tail levels as their dense operator N (reached here for the
        // finest level only, lt = 0: one visit per product): a visit from a
        // zero start is x = N b; a later visit continues from x, x += N (b - A x)
        const T* Nm = reinterpret_cast<const T*>(h.tail_op[gamma - 1].p);
        T* x = LV<T>::x(L);
        T* b = LV<T>::b(L);
        if (first) {
            tail_gemv<T>(s, L.n, h.tail_ld, Nm, b, x, false);
        } else {
            T* r = LV<T>::r(L);
            if constexpr (sizeof(T) == 8) residual64(s, L.A, x, b, r, nullptr, nullptr);
            else residual32(s, L.A, x, b, r);
            tail_gemv<T>(s, L.n, h.tail_ld, Nm, r, x, true);
        }
        return;
    }
    if (l == h.lt) {
        tail_cycle<T>(s, reinterpret_cast<const TailLevel<T>*>(h.tail.p), l, h.nlev, gamma,
                      c.p.nu_pre, c.p.nu_post, h.Xinv.p, fresh ? 1 : 0);
        return;
    }
    if (l == h.nlev - 1) {
        coarse_apply<T>(s, L.n, h.Xinv.p, LV<T>::b(L), LV<T>::x(L));
        return;
    }
    T* b = LV<T>::b(L);
    const bool prof = l == 0 && gamma == 1 && (c.p.profile & 2) && c.cur_kind != 3;
    // kind 3: the finest level's first colour was the last one updated, from
    // the same b and the same other colours
    const bool skip = l == 0 && c.cur_kind == 3 && !L.jac;
    if (prof) prof_mark(c, h, 0);
    for (int32_t k = fresh ? 1 : 0; k < c.p.nu_pre; ++k) smooth<T>(c, L, b, X<T>(L), true, skip && k == 0);
    if (prof) prof_mark(c, h, 1);
    T* x = X<T>(L);
    Level& C = h.lev[l + 1];
    // the child is the tail levels as one dense operator standing for all
    // gamma visits: x_c = N b_c, one product
    const bool child_dense = l + 1 == h.lt && h.tail_op[gamma - 1].p && h.tail_visits[gamma - 1] == gamma;
    // the child starts from zero; an l1-Jacobi child's first sweep from zero is
    // b/d, written by the restriction itself (the tail child does the same)
    const bool child_fresh = !child_dense && C.jac && c.p.nu_pre >= 1 && l + 1 < h.nlev - 1;
    const T* dc = nullptr;
    if (child_fresh) { if constexpr (sizeof(T) == 8) dc = C.dl1_64.p; else dc = C.dl1_32.p; }
    T* r = LV<T>::r(L);
    if (prof) prof_mark(c, h, 2);
    const Csr& A = L.perm ? L.Ap : L.A;
    if constexpr (sizeof(T) == 8) residual64(s, A, x, b, r, nullptr, nullptr);
    else residual32(s, A, x, b, r);
    if (prof) prof_mark(c, h, 3);
    restrict_agg<T>(s, L.nc, L.agg_ptr.p, L.perm ? L.memp.p : L.agg_mem.p, l == 0 ? LV<T>::pv(L) : nullptr, r,
                    LV<T>::b(C), child_dense ? nullptr : X<T>(C), dc);
    if (child_dense)
        tail_gemv<T>(s, C.n, h.tail_ld, reinterpret_cast<const T*>(h.tail_op[gamma - 1].p), LV<T>::b(C),
                     LV<T>::x(C), false);
    else
        for (int g = 0; g < gamma; ++g) cycle_level<T>(c, h, l + 1, gamma, child_fresh && g == 0, g == 0);
    prolong_add<T>(s, prolong_rows(L, c.p.nu_post), L.perm ? L.aggp.p : L.agg.p, l == 0 ? LV<T>::pv(L) : nullptr,
                   X<T>(C), x);
    for (int32_t k = 0; k < c.p.nu_post; ++k) smooth<T>(c, L, b, X<T>(L), false);
}

// kind 0: V-cycle from zero, 1: W-cycle from zero, 2: V-cycle continuing from
// the finest level's current x (x <- x + B (b - A x): a cycle from a start
// vector is the zero-start cycle applied to the start's residual)
template <class T>
static void cycle_body(Ctx& c, Hier& h, int kind) {
    for (int32_t l = 0; l < h.nlev; ++l) h.lev[l].xcur = 0;
    Level& L0 = h.lev[0];
    const bool cont = kind == 2 || kind == 3;
    if (!cont) {
        PC_CUDA(cudaMemsetAsync(LV<T>::x(L0), 0, sizeof(T) * L0.n, c.stream));
        pdl_after_copy();
    }
    cycle_level<T>(c, h, 0, kind == 1 ? 2 : 1, false, !cont);
}

// Forms the tail levels' dense operator for this cycle kind once per
// hierarchy, when params.tail_dense selects the kind, the tail has more than
// the coarsest level and its vectors fit one block's shared memory.
template <class T>
static void ensure_tail_op(Ctx& c, Hier& h, int gamma) {
    const int k = gamma - 1;
    if (h.tail_op_tried[k]) return;
    h.tail_op_tried[k] = true;
    if (!(c.p.tail_dense & (1 << k)) || h.lt >= h.nlev - 1) return;
    int n[kMaxLevels] = {0};
    for (int32_t l = 0; l < h.nlev; ++l) n[l] = h.lev[l].n;
    if (!tail_operator_fits<T>(n, h.lt, h.nlev)) return;
    const int m = n[h.lt];
    constexpr int w = 16 / sizeof(T);
    h.tail_ld = (m + w - 1) / w * w;
    const size_t bytes = sizeof(T) * (size_t)m * h.tail_ld;
    h.tail_op[k].alloc(c.mem, bytes);
    PC_CUDA(cudaMemsetAsync(h.tail_op[k].p, 0, bytes, c.stream));
    int dev = 0, nsm = 0;
    PC_CUDA(cudaGetDevice(&dev));
    PC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    h.tail_visits[k] = h.lt >= 1 ? gamma : 1;
    tail_operator<T>(c.stream, reinterpret_cast<const TailLevel<T>*>(h.tail.p), n, h.lt, h.nlev, gamma,
                     c.p.nu_pre, c.p.nu_post, h.Xinv.p, reinterpret_cast<T*>(h.tail_op[k].p), h.tail_ld, nsm,
                     h.tail_visits[k]);
}

static void run_body(Ctx& c, Hier& h, int kind) {
    const int gamma = kind == 1 ? 2 : 1;
    bool f32 = c.p.precision == PCAMG_FP32_IR;
    if (f32) ensure_tail_op<float>(c, h, gamma); else ensure_tail_op<double>(c, h, gamma);
    c.cur_kind = kind;
    if (!c.p.use_graphs) {
        if (f32) cycle_body<float>(c, h, kind); else cycle_body<double>(c, h, kind);
        return;
    }
    cudaGraphExec_t& ge = h.graph[kind];
    if (!ge) {
        cudaGraph_t g = nullptr;
        h.graph_kernels[kind] = 0;
        PC_CUDA(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
        t_capture_acc = &h.graph_kernels[kind];
        try {
            if (f32) cycle_body<float>(c, h, kind); else cycle_body<double>(c, h, kind);
        } catch (...) {
            t_capture_acc = nullptr;
            cudaStreamEndCapture(c.stream, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        t_capture_acc = nullptr;
        PC_CUDA(cudaStreamEndCapture(c.stream, &g));
        cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
        // a graph holding profiling nodes is kept: its nodes name the ones to retarget
        if (h.prof_node[kind][0]) h.graph_tmpl[kind] = g; else cudaGraphDestroy(g);
        PC_CUDA(e);
    }
    if (h.prof_node[kind][0] && (c.p.profile & 2)) {
        for (int k = 0; k < 4; ++k) {
            cudaEvent_t e = pool_event(c);
            PC_CUDA(cudaGraphExecEventRecordNodeSetEvent(ge, h.prof_node[kind][k], e ? e : c.cyc_tmpl[k]));
        }
    }
    PC_CUDA(cudaGraphLaunch(ge, c.stream));
    count_launches(h.graph_kernels[kind]);
}

// Vectors into and out of the finest level's cycle vectors: scaled to float
// (FP32 cycles) and, when the finest level is kept in colour order, gathered
// into it (position t holds row colour_rows0[t]) and back (row u from
// position iperm0[u]).
static void to_cycle_f32(Ctx& c, Level& L0, const double* r, float* b) {
    if (L0.perm) gather_scaled_f32(c.stream, c.n, c.colour_rows0.p, r, slot(c, S_INV), b);
    else cast_scaled_f32(c.stream, c.n, r, slot(c, S_INV), b);
}
static void from_cycle_f32(Ctx& c, Level& L0, const float* x, double* out) {
    if (L0.perm) gather_set_scaled_f32(c.stream, c.n, c.iperm0.p, x, slot(c, S_SCALE), out);
    else set_scaled_f32(c.stream, c.n, x, slot(c, S_SCALE), out);
}
static void to_cycle_f64(Ctx& c, Level& L0, const double* r, double* b) {
    if (L0.perm) gather<double>(c.stream, c.n, c.colour_rows0.p, r, b);
    else copy(c.stream, c.n, r, b);
}
static void from_cycle_f64(Ctx& c, Level& L0, const double* x, double* out) {
    if (L0.perm) gather<double>(c.stream, c.n, c.iperm0.p, x, out);
    else copy(c.stream, c.n, x, out);
}

// out = B r, the correction of one cycle from a zero start
void cycle(Ctx& c, Hier& h, int gamma, const double* r, double* out) {
    cudaStream_t s = c.stream;
    c.ncycles += 1;
    if (gamma == 2) c.nwcycles += 1;
    Level& L0 = h.lev[0];
    if (c.p.precision == PCAMG_FP32_IR) {
        // scale so the float cycle sees data of order one, then scale back:
        // inside a solve by the power of two fixed from ||b|| (exact; residuals
        // only shrink from there, far above float's smallest normal), else by
        // this residual's ||r||_2
        if (!c.fixed_scale) {
            dot(s, c.n, r, r, partials(c), slot(c, S_T0));
            scalar_ops(s, SOP_SQRT, slot(c, 0), S_T0, 0, S_SCALE);
            scalar_ops(s, SOP_INV, slot(c, 0), S_SCALE, 0, S_INV);
        }
        to_cycle_f32(c, L0, r, L0.b32v);
        run_body(c, h, gamma - 1);
        from_cycle_f32(c, L0, L0.x32v, out);
    } else {
        to_cycle_f64(c, L0, r, L0.b64v);
        run_body(c, h, gamma - 1);
        from_cycle_f64(c, L0, L0.x64v, out);
    }
}

// z = the symmetric composite of V-cycles over hist[0..re-1] applied to r
// (Alg. 2): z starts at 0 and each factor continues from it,
// z <- z + B_j (r - A z) for j = 1..re, re..1. The finest-level cycle vectors
// are shared by all hierarchies, so z stays in them between the factors.
static void composite(Ctx& c, const double* r, double* z) {
    cudaStream_t s = c.stream;
    const int32_t re = (int32_t)c.hist.size();
    const bool f32 = c.p.precision == PCAMG_FP32_IR;
    bool single = false;   // a one-level hierarchy is a bare coarse solve, x = X b
    for (Hier* h : c.hist) single = single || h->nlev < 2;
    if (single) {          // then each factor runs explicitly on r - A z
        fill(s, c.n, 0.0, z);
        Csr A;
        A.n = c.n; A.nnz = c.nnz; A.rowptr = c.rowptr.p; A.col = c.col.p; A.val = c.val.p;
        A.lpr = lanes_per_row(c.n, c.nnz);
        for (int32_t k = 0; k < 2 * re; ++k) {
            const int32_t j = (k < re) ? k : 2 * re - 1 - k;
            residual64(s, A, z, r, c.w_t1.p, nullptr, nullptr);
            cycle(c, *c.hist[j], 1, c.w_t1.p, c.w_t2.p);
            axpy(s, c.n, 1.0, c.w_t2.p, z);
        }
        return;
    }
    Level& L0 = c.hist[0]->lev[0];
    if (f32) {
        if (!c.fixed_scale) {
            dot(s, c.n, r, r, partials(c), slot(c, S_T0));
            scalar_ops(s, SOP_SQRT, slot(c, 0), S_T0, 0, S_SCALE);
            scalar_ops(s, SOP_INV, slot(c, 0), S_SCALE, 0, S_INV);
        }
        to_cycle_f32(c, L0, r, L0.b32v);
        PC_CUDA(cudaMemsetAsync(L0.x32v, 0, sizeof(float) * c.n, s));
    } else {
        to_cycle_f64(c, L0, r, L0.b64v);
        PC_CUDA(cudaMemsetAsync(L0.x64v, 0, sizeof(double) * c.n, s));
    }
    // after the first factor, each one follows the previous factor's
    // post-sweep on the same finest level (kind 3) when that level is smoothed
    // by Gauss-Seidel above the coarse tail
    Level& F = c.hist[0]->lev[0];
    const bool follow = !F.jac && F.ncolour >= 1 && c.hist[0]->lt >= 1;
    for (int32_t k = 0; k < 2 * re; ++k) {
        const int32_t j = (k < re) ? k : 2 * re - 1 - k;
        c.ncycles += 1;
        run_body(c, *c.hist[j], (k > 0 && follow) ? 3 : 2);
    }
    if (f32) from_cycle_f32(c, L0, L0.x32v, z);
    else from_cycle_f64(c, L0, L0.x64v, z);
}

// ---------------------------------------------------------------- residual with profiling
static void fine_residual(Ctx& c, const double* x, const double* b, double* r, double* norm2) {
    Csr A;
    A.n = c.n; A.nnz = c.nnz; A.rowptr = c.rowptr.p; A.col = c.col.p; A.val = c.val.p;
    A.lpr = lanes_per_row(c.n, c.nnz);
    if (c.p.profile & 1) PC_CUDA(cudaEventRecord(c.ev0, c.stream));
    residual64(c.stream, A, x, b, r, partials(c), norm2);
    if (c.p.profile & 1) {
        PC_CUDA(cudaEventRecord(c.ev1, c.stream));
        PC_CUDA(cudaEventSynchronize(c.ev1));
        float ms = 0.f;
        PC_CUDA(cudaEventElapsedTime(&ms, c.ev0, c.ev1));
        c.prof_ms += ms;
        c.prof_launches += 1;
    }
}

static void spmv_A(Ctx& c, const double* x, double* y) {
    Csr A;
    A.n = c.n; A.nnz = c.nnz; A.rowptr = c.rowptr.p; A.col = c.col.p; A.val = c.val.p;
    A.lpr = lanes_per_row(c.n, c.nnz);
    spmv64(c.stream, A, x, y);
}

static void remove_mean(Ctx& c, double* x) {
    sum(c.stream, c.n, x, partials(c), slot(c, S_SUM));
    sub_mean(c.stream, c.n, x, slot(c, S_SUM));
}

// ---------------------------------------------------------------- Alg. 2
static void precond(Ctx& c, const double* r, double* z) {
    int32_t re = (int32_t)c.hist.size();
    if (re <= c.p.numW) {
        cycle(c, *c.hist[re - 1], 2, r, z);
        return;
    }
    composite(c, r, z);
}

void smooth_error(Ctx& c, const double* rhs, double* e) {
    cudaStream_t s = c.stream;
    int32_t re = (int32_t)c.hist.size();
    if (re < 1) fail(PCAMG_ERR_INVALID, "no hierarchy built");
    int32_t iters = (re <= c.p.numW) ? c.p.iterW : c.p.iterV;
    double* r = c.w_ein.p;  // running residual
    double* rold = c.w_rold.p;
    double* z = c.w_z.p;
    double* pp = c.w_p.p;
    double* q = c.w_q.p;
    fill(s, c.n, 0.0, e);
    copy(s, c.n, rhs, r);
    precond(c, r, z);
    copy(s, c.n, z, pp);
    dot(s, c.n, r, z, partials(c), slot(c, S_RZ));
    for (int32_t it = 1; it <= iters; ++it) {
        spmv_A(c, pp, q);
        dot(s, c.n, pp, q, partials(c), slot(c, S_PQ));
        scalar_ops(s, SOP_PCG_ALPHA, slot(c, 0), S_RZ, S_PQ, S_ALPHA);  // alpha = rz/pq (0 on breakdown)
        axpy_dev(s, c.n, slot(c, S_ALPHA), 1.0, pp, e);
        copy(s, c.n, r, rold);
        axpy_dev(s, c.n, slot(c, S_ALPHA), -1.0, q, r);
        if (it == iters) break;
        precond(c, r, z);
        // beta = z^T (r - r_old) / (z_old^T r_old)   (Polak-Ribiere)
        copy(s, c.n, r, c.w_t1.p);
        axpy(s, c.n, -1.0, rold, c.w_t1.p);
        dot(s, c.n, z, c.w_t1.p, partials(c), slot(c, S_NUM));
        scalar_ops(s, SOP_DIV, slot(c, 0), S_NUM, S_RZ, S_BETA);
        dot(s, c.n, r, z, partials(c), slot(c, S_RZ));
        xpby_dev(s, c.n, z, slot(c, S_BETA), pp);
    }
}

void start_vector(Ctx& c, double* e) {
    cudaStream_t s = c.stream;
    philox_uniform(s, c.p.seed, c.n, e);
    fill(s, c.n, 0.0, c.w_t1.p);
    Csr A;
    A.n = c.n; A.nnz = c.nnz; A.rowptr = c.rowptr.p; A.col = c.col.p; A.val = c.val.p;
    A.lpr = lanes_per_row(c.n, c.nnz);
    // with the finest level in colour order the sweeps run on e in that order
    double* ep = e;
    if (c.perm0 && c.p.relax_sweeps > 0) {
        ep = (e == c.w_q.p) ? c.w_p.p : c.w_q.p;
        gather<double>(s, c.n, c.colour_rows0.p, e, ep);
    }
    for (int32_t k = 0; k < c.p.relax_sweeps; ++k) {
        for (int32_t t = 0; t < c.ncolour0; ++t) {
            int32_t beg = c.h_colour_ptr0[t], end = c.h_colour_ptr0[t + 1];
            if (c.gs_val0_64.p)
                gs_colour_perm<double>(s, beg, end, c.perm0 ? nullptr : c.colour_rows0.p, c.gs_ptr0.p,
                                       c.gs_col0.p, c.gs_val0_64.p, c.w_t1.p, ep);
            else
                gs_colour<double>(s, A, c.colour_rows0.p + beg, end - beg, c.w_t1.p, e);
        }
    }
    if (ep != e) gather<double>(s, c.n, c.iperm0.p, ep, e);
    normalise_orth(c, e, e);
}

// ---------------------------------------------------------------- Alg. 5 / Alg. 6
static double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Fix the FP32 cycles' scale for a solve: the power of two nearest to the root
// mean square of the right-hand side (norm2 = ||b||_2), so scaling is exact.
static void fix_scale(Ctx& c, double norm2) {
    double rms = norm2 / std::sqrt((double)c.n);
    int e = (rms > 0.0 && std::isfinite(rms)) ? std::ilogb(rms) : 0;
    c.h_red[40] = std::ldexp(1.0, e);
    c.h_red[41] = std::ldexp(1.0, -e);
    PC_CUDA(cudaMemcpyAsync(slot(c, S_SCALE), c.h_red + 40, sizeof(double), cudaMemcpyHostToDevice, c.stream));
    PC_CUDA(cudaMemcpyAsync(slot(c, S_INV), c.h_red + 41, sizeof(double), cudaMemcpyHostToDevice, c.stream));
    c.fixed_scale = true;
}

struct ScaleGuard {
    Ctx& c;
    ~ScaleGuard() { c.fixed_scale = false; }
};

static double read_norm(Ctx& c) {
    PC_CUDA(cudaMemcpyAsync(c.h_red, slot(c, S_NORM2), sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    sync(c);
    return std::sqrt(c.h_red[0]);
}

static void rebuild(Ctx& c, double* e_raw_out) {
    double t0 = now_ms();
    smooth_error(c, c.w_r.p, e_raw_out);
    normalise_orth(c, e_raw_out, c.w_eh.p);
    sync(c);
    double t1 = now_ms();
    Hier* h = build_hierarchy(c, c.w_eh.p);
    c.hist.push_back(h);
    c.last_e = c.w_eh.p;
    c.t_alg2 += t1 - t0;
    c.t_alg4 += now_ms() - t1;
}

pcamg_status solve(Ctx& c, const double* b, double* x, pcamg_stats* st) {
    cudaStream_t s = c.stream;
    double t0 = now_ms(), t_setup = 0.0;
    c.prof_ms = 0.0;
    c.prof_launches = 0;
    c.cyc_ms = 0.0;
    c.cyc_launches = 0;
    c.gs_ms = 0.0;
    c.gs_sweeps = 0;
    c.cyc_used = 0;
    c.ncycles = 0;
    c.nwcycles = 0;
    c.t_alg2 = c.t_alg4 = 0.0;
    int32_t re0 = (int32_t)c.hist.size();
    if (st && st->rebuilt)
        for (int32_t i = 0; i < st->res_hist_cap; ++i) st->rebuilt[i] = 0;
    dot(s, c.n, b, b, partials(c), slot(c, S_NORM2));
    double bn = read_norm(c);
    if (!std::isfinite(bn) || !(bn > 0.0)) fail(PCAMG_ERR_INVALID, "right-hand side is zero or not finite");
    ScaleGuard sg{c};
    fix_scale(c, bn);
    remove_mean(c, x);
    fine_residual(c, x, b, c.w_r.p, slot(c, S_NORM2));
    double res = read_norm(c);
    if (!std::isfinite(res)) fail(PCAMG_ERR_INVALID, "initial guess is not finite");
    int32_t k = 0, hl = 0;
    double wsum = 0.0;
    int32_t wcnt = 0;
    pcamg_status status = PCAMG_OK;
    auto hist_put = [&](int32_t idx, double v) {
        if (st && st->res_hist && idx < st->res_hist_cap) { st->res_hist[idx] = v; if (idx + 1 > hl) hl = idx + 1; }
    };
    hist_put(0, res / bn);
    // flexible CG outer iteration (params.outer): direction, A times it, the
    // previous residual and preconditioned residual; a re-setup restarts it
    const bool fcg = c.p.outer == PCAMG_OUTER_FCG;
    bool restart = true;
    double *fp = c.w_p.p, *fq = c.w_q.p, *frold = c.w_rold.p, *fzold = c.w_cin.p;
    while (k < c.p.max_iter && res / bn > c.p.tol) {
        Hier& h = *c.hist.back();
        cycle(c, h, 1, c.w_r.p, c.w_c.p);
        if (fcg) {
            const double* z = c.w_c.p;
            const double* r = c.w_r.p;
            dot(s, c.n, r, z, partials(c), slot(c, S_FRZ));
            if (restart) {
                copy(s, c.n, z, fp);
                restart = false;
            } else {   // Polak-Ribiere: beta = z.(r - r_old) / (z_old.r_old)
                copy(s, c.n, r, c.w_t1.p);
                axpy(s, c.n, -1.0, frold, c.w_t1.p);
                dot(s, c.n, z, c.w_t1.p, partials(c), slot(c, S_FNUM));
                dot(s, c.n, fzold, frold, partials(c), slot(c, S_FDEN));
                scalar_ops(s, SOP_DIV, slot(c, 0), S_FNUM, S_FDEN, S_FBETA);
                xpby_dev(s, c.n, z, slot(c, S_FBETA), fp);          // p = z + beta p
            }
            spmv_A(c, fp, fq);
            dot(s, c.n, fp, fq, partials(c), slot(c, S_FPQ));
            scalar_ops(s, SOP_PCG_ALPHA, slot(c, 0), S_FRZ, S_FPQ, S_FALPHA);
            axpy_dev(s, c.n, slot(c, S_FALPHA), 1.0, fp, x);         // x += alpha p
            copy(s, c.n, r, frold);
            copy(s, c.n, z, fzold);
        } else {
            axpy(s, c.n, 1.0, c.w_c.p, x);
        }
        remove_mean(c, x);
        fine_residual(c, x, b, c.w_r.p, slot(c, S_NORM2));
        double nres = read_norm(c);
        if (!std::isfinite(nres)) { status = PCAMG_ERR_DIVERGED; res = nres; break; }
        wsum += nres / res;
        ++wcnt;
        res = nres;
        ++k;
        hist_put(k, res / bn);
        if (res / bn <= c.p.tol) break;
        if (wsum / (double)wcnt > c.p.threshold) {
            if (c.p.max_resetups >= 0 && (int32_t)c.hist.size() - re0 >= c.p.max_resetups) break;
            double ts = now_ms();
            rebuild(c, c.w_e.p);
            restart = true;
            if (st && st->rebuilt && k < st->res_hist_cap) st->rebuilt[k] = 1;
            if (c.p.update_mode == PCAMG_UPD_ADD_CORRECTION) {
                axpy(s, c.n, 1.0, c.w_e.p, x);
                remove_mean(c, x);
                fine_residual(c, x, b, c.w_r.p, slot(c, S_NORM2));
                res = read_norm(c);
                hist_put(k, res / bn);
            }
            wsum = 0.0;
            wcnt = 0;
            t_setup += now_ms() - ts;
            if (c.p.max_resetups >= 0 && (int32_t)c.hist.size() - re0 >= c.p.max_resetups) break;
        }
    }
    if (status == PCAMG_OK && !(res / bn <= c.p.tol)) status = PCAMG_ERR_NOT_CONVERGED;
    sync(c);
    prof_resolve(c);
    if (st) {
        st->iters = k;
        st->resetups = (int32_t)c.hist.size() - re0;
        st->levels = c.hist.back()->nlev;
        st->status = status;
        st->rel_res = res / bn;
        double oc = 0.0;
        for (Hier* h : c.hist) oc += h->oc;
        st->oc_mean = oc / (double)c.hist.size();
        st->t_setup_ms = t_setup;
        st->t_solve_ms = now_ms() - t0;
        st->res_hist_len = hl;
        st->t_alg2_ms = c.t_alg2;
        st->t_alg4_ms = c.t_alg4;
        st->cycles = c.ncycles;
        st->wcycles = c.nwcycles;
        st->prof_launches = c.prof_launches;
        st->prof_ms = c.prof_ms;
        st->prof_bytes = (double)c.prof_launches * (12.0 * (double)c.nnz + 28.0 * (double)c.n);
        const double w = c.p.precision == PCAMG_FP32_IR ? 4.0 : 8.0;
        st->cyc_launches = c.cyc_launches;
        st->cyc_ms = c.cyc_ms;
        st->cyc_bytes = (double)c.cyc_launches * ((4.0 + w) * (double)c.nnz + (4.0 + 3.0 * w) * (double)c.n);
        st->gs_sweeps = c.gs_sweeps;
        st->gs_ms = c.gs_ms;
        st->gs_bytes = (double)c.gs_sweeps * ((4.0 + w) * (double)c.nnz + (4.0 + 3.0 * w) * (double)c.n);
    }
    return status;
}

// ---------------------------------------------------------------- several right-hand sides
// The batched V-cycle: the single-vector cycle's steps (gamma = 1:
// pre-smoothing, residual, restriction with the child's fresh start, the
// child, prolongation, post-smoothing; the tail as its dense operator, the
// coarsest level by its pseudo-inverse) on K row-interleaved vectors per
// level. The finest level's vectors belong to the context and a cycle
// continues from its x (x <- x + B_h (b - A x)), so the factors of Alg. 2's
// composite follow one another in place, as in the single-vector composite.
template <class T>
static T* mvb(DBuf<unsigned char>& d) { return reinterpret_cast<T*>(d.p); }

template <class T>
static void mv_ensure(Ctx& c, Hier& h, int K) {
    if (c.mv0_K != K) {
        const size_t bytes = sizeof(T) * (size_t)c.n * K;
        c.mv0_x.alloc(c.mem, bytes);
        c.mv0_b.alloc(c.mem, bytes);
        c.mv0_r.alloc(c.mem, bytes);
        c.mv0_K = K;
    }
    if (h.mv_K == K) return;
    for (int32_t l = 1; l < h.nlev; ++l) {
        Level& L = h.lev[l];
        const size_t bytes = sizeof(T) * (size_t)L.n * K;
        h.mv_x[l].alloc(c.mem, bytes);
        h.mv_b[l].alloc(c.mem, bytes);
        h.mv_r[l].alloc(c.mem, bytes);
        if (L.jac) h.mv_x2[l].alloc(c.mem, bytes); else h.mv_x2[l].free();
    }
    h.mv_K = K;
}

// the level vectors of one batched cycle of h (level 0: the context's)
template <class T>
struct MvVecs {
    T* x[kMaxLevels];
    T* x2[kMaxLevels];
    T* b[kMaxLevels];
    T* r[kMaxLevels];
};

template <class T>
static MvVecs<T> mv_vecs(Ctx& c, Hier& h) {
    MvVecs<T> v;
    for (int32_t l = 0; l < h.nlev; ++l) {
        v.x[l] = l == 0 ? mvb<T>(c.mv0_x) : mvb<T>(h.mv_x[l]);
        v.x2[l] = l == 0 ? nullptr : mvb<T>(h.mv_x2[l]);
        v.b[l] = l == 0 ? mvb<T>(c.mv0_b) : mvb<T>(h.mv_b[l]);
        v.r[l] = l == 0 ? mvb<T>(c.mv0_r) : mvb<T>(h.mv_r[l]);
    }
    return v;
}

template <class T>
static void mv_smooth(Ctx& c, Hier& h, int K, int32_t l, MvVecs<T>& v, bool forward, bool skip_first = false) {
    Level& L = h.lev[l];
    const Csr& A = (l == 0 && L.perm) ? L.Ap : L.A;
    if (L.jac && v.x2[l]) {
        const T* d;
        if constexpr (sizeof(T) == 8) d = L.dl1_64.p; else d = L.dl1_32.p;
        mv_rows<T>(c.stream, 1, K, L.n, nullptr, 0, A, v.x[l], v.b[l], d, v.x2[l]);
        std::swap(v.x[l], v.x2[l]);
        return;
    }
    for (int32_t t = skip_first ? 1 : 0; t < L.ncolour; ++t) {
        const int32_t k = forward ? t : L.ncolour - 1 - t;
        const int32_t beg = L.h_colour_ptr[k], end = L.h_colour_ptr[k + 1];
        if (L.perm)   // colour order: the colour's rows are positions beg..end
            mv_rows<T>(c.stream, 2, K, end - beg, nullptr, beg, A, v.x[l], v.b[l], nullptr, v.x[l]);
        else
            mv_rows<T>(c.stream, 2, K, end - beg, L.colour_rows_v + beg, 0, A, v.x[l], v.b[l], nullptr, v.x[l]);
    }
}

// One visit of level l. Level 0 continues from its x; a coarser level starts
// from zero, or from one l1-Jacobi sweep from zero when `fresh`.
template <class T>
static void mv_level(Ctx& c, Hier& h, int K, int32_t l, bool fresh, MvVecs<T>& v, bool follows = false) {
    cudaStream_t s = c.stream;
    Level& L = h.lev[l];
    const bool dense = l == h.lt && h.tail_op[0].p && h.tail_visits[0] == 1;
    if (dense || l == h.nlev - 1) {
        const T* rhs = v.b[l];
        if (l == 0) {   // the whole hierarchy is one operator: x += M (b - A x)
            mv_rows<T>(s, 0, K, L.n, nullptr, 0, L.perm ? L.Ap : L.A, v.x[0], v.b[0], nullptr, v.r[0]);
            rhs = v.r[0];
        }
        if (dense) mv_dense<T>(s, K, L.n, h.tail_ld, reinterpret_cast<const T*>(h.tail_op[0].p), rhs, v.x[l], l == 0);
        else mv_coarse<T>(s, K, L.n, h.Xinv.p, rhs, v.x[l], l == 0);
        return;
    }
    // `follows` (level 0): a post-sweep of this level just ended with the
    // first colour, from the same b and other colours, so it is not repeated
    for (int32_t k = fresh ? 1 : 0; k < c.p.nu_pre; ++k)
        mv_smooth<T>(c, h, K, l, v, true, follows && l == 0 && k == 0 && !L.jac);
    const Csr& A = (l == 0 && L.perm) ? L.Ap : L.A;
    mv_rows<T>(s, 0, K, L.n, nullptr, 0, A, v.x[l], v.b[l], nullptr, v.r[l]);
    Level& C = h.lev[l + 1];
    const bool child_dense = l + 1 == h.lt && h.tail_op[0].p && h.tail_visits[0] == 1;
    const bool child_fresh = !child_dense && C.jac && c.p.nu_pre >= 1 && l + 1 < h.nlev - 1;
    const T* dc = nullptr;
    if (child_fresh) { if constexpr (sizeof(T) == 8) dc = C.dl1_64.p; else dc = C.dl1_32.p; }
    const T* pv = l == 0 ? LV<T>::pv(L) : nullptr;
    mv_restrict<T>(s, K, L.nc, L.agg_ptr.p, L.perm ? L.memp.p : L.agg_mem.p, pv, v.r[l], v.b[l + 1], v.x[l + 1], dc);
    mv_level<T>(c, h, K, l + 1, child_fresh, v);
    mv_prolong<T>(s, K, prolong_rows(L, c.p.nu_post), L.perm ? L.aggp.p : L.agg.p, pv, v.x[l + 1], v.x[l]);
    for (int32_t k = 0; k < c.p.nu_post; ++k) mv_smooth<T>(c, h, K, l, v, false);
}

// Z = M R for the kr columns of R (column-major n x kr), M Alg. 2's symmetric
// composite of V-cycles over every hierarchy held, z += B_j (r - A z) for
// j = 1..re, re..1 from z = 0; the columns scaled by their fixed scales into
// the finest level's order and back.
template <class T>
static void mv_precond(Ctx& c, int K, int kr, const double* R, double* Z, const double* scale, const double* inv) {
    cudaStream_t s = c.stream;
    const int32_t re = (int32_t)c.hist.size();
    for (Hier* h : c.hist) mv_ensure<T>(c, *h, K);
    Level& L0 = c.hist[0]->lev[0];
    const int* perm = L0.perm ? c.colour_rows0.p : nullptr;
    const int* iperm = L0.perm ? c.iperm0.p : nullptr;
    mv_in<T>(s, K, kr, c.n, perm, R, inv, mvb<T>(c.mv0_b));
    PC_CUDA(cudaMemsetAsync(c.mv0_x.p, 0, sizeof(T) * (size_t)c.n * K, s));
    const bool follow = !L0.jac && L0.ncolour >= 1 && c.hist[0]->lt >= 1 && c.hist[0]->nlev >= 2;
    for (int32_t q = 0; q < 2 * re; ++q) {
        Hier& h = *c.hist[q < re ? q : 2 * re - 1 - q];
        MvVecs<T> v = mv_vecs<T>(c, h);
        mv_level<T>(c, h, K, 0, false, v, follow && q > 0);
        c.ncycles += 1;
    }
    mv_out<T>(s, K, kr, c.n, iperm, mvb<T>(c.mv0_x), scale, Z);
}

// Columns [c0, c0 + kb) of B and X (kb <= 8, run as one batch of K >= kb
// vectors): the outer iteration of params.outer for each column, no re-setup,
// preconditioned by the batched composite.
static pcamg_status solve_multi_block(Ctx& c, int32_t kb, const double* B, double* X, int32_t* iters,
                                      double* rel_res) {
    cudaStream_t s = c.stream;
    const size_t n = (size_t)c.n;
    int K = 1;
    while (K < kb) K <<= 1;
    const bool f32 = c.p.precision == PCAMG_FP32_IR;
    DBuf<double> R, Z, P, Q, Rold, Zold, sc;
    for (DBuf<double>* v : {&R, &Z, &P, &Q, &Rold, &Zold}) v->alloc(c.mem, n * kb);
    sc.alloc(c.mem, 16);
    std::vector<double> bn(kb), res(kb);
    std::vector<int32_t> it(kb, 0);
    std::vector<char> active(kb, 1), restart(kb, 1);
    // per column: its norm, the fixed power-of-two scale of the FP32 cycles
    // (as in a single solve), its mean removed, its residual
    for (int32_t j = 0; j < kb; ++j) {
        dot(s, c.n, B + j * n, B + j * n, partials(c), slot(c, S_NORM2));
        bn[j] = read_norm(c);
        if (!std::isfinite(bn[j]) || !(bn[j] > 0.0)) fail(PCAMG_ERR_INVALID, "a right-hand side is zero or not finite");
        const double rms = bn[j] / std::sqrt((double)c.n);
        const int e = (f32 && rms > 0.0 && std::isfinite(rms)) ? std::ilogb(rms) : 0;
        c.h_red[16 + j] = std::ldexp(1.0, e);
        c.h_red[24 + j] = std::ldexp(1.0, -e);
    }
    PC_CUDA(cudaMemcpyAsync(sc.p, c.h_red + 16, sizeof(double) * 16, cudaMemcpyHostToDevice, s));
    for (int32_t j = 0; j < kb; ++j) {
        remove_mean(c, X + j * n);
        fine_residual(c, X + j * n, B + j * n, R.p + j * n, slot(c, S_NORM2));
        res[j] = read_norm(c);
        if (!std::isfinite(res[j])) fail(PCAMG_ERR_INVALID, "an initial guess is not finite");
        active[j] = res[j] / bn[j] > c.p.tol;
    }
    const bool fcg = c.p.outer == PCAMG_OUTER_FCG;
    pcamg_status status = PCAMG_OK;
    for (int32_t k = 0; k < c.p.max_iter; ++k) {
        bool any = false;
        for (int32_t j = 0; j < kb; ++j) any = any || active[j];
        if (!any) break;
        if (kb == 1) {   // one column: the single-vector composite (graph-captured cycles)
            ScaleGuard sg{c};
            fix_scale(c, bn[0]);
            composite(c, R.p, Z.p);
        } else if (f32) {
            mv_precond<float>(c, K, kb, R.p, Z.p, sc.p, sc.p + 8);
        } else {
            mv_precond<double>(c, K, kb, R.p, Z.p, sc.p, sc.p + 8);
        }
        for (int32_t j = 0; j < kb; ++j) {
            if (!active[j]) continue;
            double* x = X + j * n;
            const double* r = R.p + j * n;
            const double* z = Z.p + j * n;
            if (fcg) {   // the single solve's flexible CG, column j
                double *fp = P.p + j * n, *fq = Q.p + j * n, *frold = Rold.p + j * n, *fzold = Zold.p + j * n;
                dot(s, c.n, r, z, partials(c), slot(c, S_FRZ));
                if (restart[j]) {
                    copy(s, c.n, z, fp);
                    restart[j] = 0;
                } else {
                    copy(s, c.n, r, c.w_t1.p);
                    axpy(s, c.n, -1.0, frold, c.w_t1.p);
                    dot(s, c.n, z, c.w_t1.p, partials(c), slot(c, S_FNUM));
                    dot(s, c.n, fzold, frold, partials(c), slot(c, S_FDEN));
                    scalar_ops(s, SOP_DIV, slot(c, 0), S_FNUM, S_FDEN, S_FBETA);
                    xpby_dev(s, c.n, z, slot(c, S_FBETA), fp);
                }
                spmv_A(c, fp, fq);
                dot(s, c.n, fp, fq, partials(c), slot(c, S_FPQ));
                scalar_ops(s, SOP_PCG_ALPHA, slot(c, 0), S_FRZ, S_FPQ, S_FALPHA);
                axpy_dev(s, c.n, slot(c, S_FALPHA), 1.0, fp, x);
                copy(s, c.n, r, frold);
                copy(s, c.n, z, fzold);
            } else {
                axpy(s, c.n, 1.0, z, x);
            }
            remove_mean(c, x);
            fine_residual(c, x, B + j * n, R.p + j * n, slot(c, S_NORM2));
            const double nres = read_norm(c);
            it[j] += 1;
            if (!std::isfinite(nres)) { status = PCAMG_ERR_DIVERGED; active[j] = 0; res[j] = nres; continue; }
            res[j] = nres;
            if (res[j] / bn[j] <= c.p.tol) active[j] = 0;
        }
    }
    for (int32_t j = 0; j < kb; ++j) {
        if (iters) iters[j] = it[j];
        if (rel_res) rel_res[j] = res[j] / bn[j];
        if (status == PCAMG_OK && !(res[j] / bn[j] <= c.p.tol)) status = PCAMG_ERR_NOT_CONVERGED;
    }
    sync(c);
    return status;
}

pcamg_status solve_multi(Ctx& c, int32_t k, const double* B, double* X, int32_t* iters, double* rel_res) {
    if (k < 1) fail(PCAMG_ERR_INVALID, "no right-hand sides");
    if (c.hist.empty()) fail(PCAMG_ERR_INVALID, "no hierarchy built");
    const bool f32 = c.p.precision == PCAMG_FP32_IR;
    for (Hier* hh : c.hist) {
        if (f32) ensure_tail_op<float>(c, *hh, 1); else ensure_tail_op<double>(c, *hh, 1);
    }
    pcamg_status status = PCAMG_OK;
    const size_t n = (size_t)c.n;
    for (int32_t c0 = 0; c0 < k; c0 += 8) {
        const int32_t kb = std::min<int32_t>(8, k - c0);
        const pcamg_status sb = solve_multi_block(c, kb, B + c0 * n, X + c0 * n, iters ? iters + c0 : nullptr,
                                                  rel_res ? rel_res + c0 : nullptr);
        if (sb == PCAMG_ERR_DIVERGED || (sb != PCAMG_OK && status == PCAMG_OK)) status = sb;
    }
    return status;
}

pcamg_status solve_zero_rhs(Ctx& c, double* x, pcamg_stats* st) {
    cudaStream_t s = c.stream;
    double t0 = now_ms(), t_setup = 0.0;
    int32_t re0 = (int32_t)c.hist.size();
    c.ncycles = 0;
    c.nwcycles = 0;
    if (st && st->rebuilt)
        for (int32_t i = 0; i < st->res_hist_cap; ++i) st->rebuilt[i] = 0;
    double* zero = c.w_t2.p;
    fill(s, c.n, 0.0, zero);
    remove_mean(c, x);
    fine_residual(c, x, zero, c.w_r.p, slot(c, S_NORM2));
    double r0 = read_norm(c), res = r0;
    ScaleGuard sg{c};
    fix_scale(c, r0);
    int32_t k = 0, hl = 0;
    pcamg_status status = PCAMG_OK;
    auto hist_put = [&](int32_t idx, double v) {
        if (st && st->res_hist && idx < st->res_hist_cap) { st->res_hist[idx] = v; if (idx + 1 > hl) hl = idx + 1; }
    };
    if (r0 > 0.0) {
        hist_put(0, 1.0);
        while (k < c.p.max_iter && res / r0 > c.p.tol) {
            cycle(c, *c.hist.back(), 1, c.w_r.p, c.w_c.p);
            axpy(s, c.n, 1.0, c.w_c.p, x);
            remove_mean(c, x);
            fine_residual(c, x, zero, c.w_r.p, slot(c, S_NORM2));
            double nres = read_norm(c);
            if (!std::isfinite(nres)) { status = PCAMG_ERR_DIVERGED; res = nres; break; }
            double conv = nres / res;
            res = nres;
            ++k;
            hist_put(k, res / r0);
            if (res / r0 <= c.p.tol) break;
            if (conv > c.p.threshold) {
                double ts = now_ms();
                // the exact error is the iterate itself: e = x / ||x||
                normalise_orth(c, x, c.w_eh.p);
                Hier* h = build_hierarchy(c, c.w_eh.p);
                c.hist.push_back(h);
                c.last_e = c.w_eh.p;
                t_setup += now_ms() - ts;
                if (st && st->rebuilt && k < st->res_hist_cap) st->rebuilt[k] = 1;
            }
        }
        if (status == PCAMG_OK && !(res / r0 <= c.p.tol)) status = PCAMG_ERR_NOT_CONVERGED;
    }
    sync(c);
    if (st) {
        st->iters = k;
        st->resetups = (int32_t)c.hist.size() - re0;
        st->levels = c.hist.back()->nlev;
        st->status = status;
        st->rel_res = r0 > 0.0 ? res / r0 : 0.0;
        double oc = 0.0;
        for (Hier* h : c.hist) oc += h->oc;
        st->oc_mean = oc / (double)c.hist.size();
        st->t_setup_ms = t_setup;
        st->t_solve_ms = now_ms() - t0;
        st->res_hist_len = hl;
        st->cycles = c.ncycles;
        st->wcycles = c.nwcycles;
    }
    return status;
}

}  // namespace pc
