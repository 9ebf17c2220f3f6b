// Internal declarations of the PC-alphaAMG CUDA library (sm_103a).
// Host code throws pc::Error inside the library; the C ABI layer catches it.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "pcamg.h"

namespace pc {

struct Error {
    pcamg_status status;
    std::string msg;
};

[[noreturn]] void fail(pcamg_status s, const std::string& msg);
void set_global_error(const std::string& msg);   // message for pcamg_last_error(NULL)
void check_cuda(cudaError_t e, const char* what);
// Process-wide count of kernels this library has launched (a graph replay adds
// the number of kernels it holds).
void count_launches(int64_t k);
int64_t launch_count();
bool capturing();
#define PC_CUDA(call) ::pc::check_cuda((call), #call)
#define PC_LAUNCH(what) ::pc::check_cuda(cudaGetLastError(), what)
#define PC_LAUNCHN(what, k) do { ::pc::check_cuda(cudaGetLastError(), what); ::pc::count_launches(k); } while (0)

// Programmatic dependent launch of the cycle kernels. While a cycle graph is
// captured, launch() marks each kernel launch as a programmatic dependent of
// the kernel before it, so it may start while that kernel drains. Such a
// kernel reads only hierarchy data (matrices, aggregates, colour permutations,
// all written before the graph runs) ahead of pdl_wait(), which returns once
// the previous grid has completed and its writes are visible; every block
// reaches pdl_wait() before it exits. pdl_trigger() comes after the wait, so
// at most two grids of the chain are in flight. Outside a programmatic launch
// both instructions do nothing.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// true while a cycle graph is captured and the previous captured node is a
// kernel (a programmatic edge joins two kernels only); consumes the state
bool pdl_next();
void pdl_after_copy();   // the next captured node follows a memset or copy

template <class... P, class... A>
inline void launch(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    const bool pdl = pdl_next();
    cfg.attrs = pdl ? at : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    check_cuda(cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...), "launch");
    count_launches(1);
}

// Counters and flags that many threads of a launch bump: one atomic per warp
// (or per block) instead of one per thread, so a busy launch does not queue
// millions of updates on one address. Every thread of the block must call the
// block forms; the warp forms are called by the lanes active at that point.
__device__ __forceinline__ void warp_count(int* counter, bool pred) {
    const unsigned m = __ballot_sync(__activemask(), pred);
    if (pred && (int)(threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(counter, __popc(m));
}
// slot in a list for the lanes with pred (order between warps is arbitrary)
__device__ __forceinline__ int warp_append(int* counter, bool pred) {
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, pred);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (m && lane == leader) base = atomicAdd(counter, __popc(m));
    base = __shfl_sync(act, base, m ? leader : __ffs(act) - 1);
    return base + __popc(m & ((1u << lane) - 1u));
}
__device__ __forceinline__ void block_count(int* counter, int local) {
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(&s_cnt, local);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd(counter, s_cnt);
}
__device__ __forceinline__ void block_flag(int* flag, int local) {
    if (__syncthreads_or(local) && threadIdx.x == 0) *flag = 1;
}

constexpr int kMaxLevels = 32;
constexpr int kBlock = 256;
constexpr int kNumSMs = 152;

// ---------------------------------------------------------------- memory
// Device allocations are stream ordered on `stream`: from the caller's
// callbacks (pcamg_set_allocator) current when this Mem was made, else from the
// library's per-device pool (freed memory kept cached).
struct Mem {
    cudaStream_t stream = nullptr;
    size_t live = 0, peak = 0;
    pcamg_alloc_fn afn = nullptr;
    pcamg_free_fn ffn = nullptr;
    void* actx = nullptr;
    Mem();
    void* alloc(size_t bytes);
    void release(void* p, size_t bytes);
};

template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    Mem* m = nullptr;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept { *this = static_cast<DBuf&&>(o); }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) { free(); p = o.p; n = o.n; m = o.m; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DBuf() { free(); }
    void alloc(Mem& mem, size_t count) {
        free();
        m = &mem;
        n = count;
        p = static_cast<T*>(mem.alloc(sizeof(T) * (count ? count : 1)));
    }
    void free() {
        if (p && m) m->release(p, sizeof(T) * (n ? n : 1));
        p = nullptr;
        n = 0;
    }
    T* get() const { return p; }
};

struct Csr {
    int32_t n = 0;
    int64_t nnz = 0;
    const int32_t* rowptr = nullptr;  // views (owned elsewhere)
    const int32_t* col = nullptr;
    const double* val = nullptr;
    const float* val32 = nullptr;
    int lpr = 8;  // lanes per row in the sparse kernels (power of two, 2..32)
    // diagonal entries marked: row i stores its diagonal's column as ~i
    // (negative); the streaming kernels decode it (the colour-ordered copy)
    bool dmark = false;
};
int lanes_per_row(int32_t n, int64_t nnz);

// One level of a hierarchy. Level 0 borrows A (and its FP32 copy and colouring)
// from the context.
struct Level {
    int32_t n = 0;
    int64_t nnz = 0;
    DBuf<int32_t> rowptr, col;
    DBuf<double> val;
    DBuf<float> val32;
    Csr A;  // view used by the kernels
    // smoother colouring: rows grouped by colour
    int32_t ncolour = 0;
    DBuf<int32_t> colour, colour_rows;
    std::vector<int32_t> h_colour_ptr;  // ncolour + 1 offsets (host)
    const int32_t* colour_rows_v = nullptr;
    const int32_t* colour_v = nullptr;
    // transfer to the next level
    int32_t nc = 0;
    DBuf<int32_t> agg, agg_ptr, agg_mem;
    DBuf<double> pval;
    DBuf<float> pval32;
    // kept for export when params.keep_setup
    DBuf<int32_t> nbr0, nbr1, tptr, tcol;
    DBuf<double> tw;
    int64_t tnnz = 0;
    int32_t cover_rounds = 0, leftover_rounds = 0;
    // cycle work vectors (sized n); the views are what the cycle uses: a level's
    // own buffers, or for the finest level the context's (shared by all
    // hierarchies: a cycle of one hierarchy can continue from another's result)
    DBuf<double> x64, b64, r64;
    DBuf<float> x32, b32, r32;
    double *x64v = nullptr, *b64v = nullptr, *r64v = nullptr;
    float *x32v = nullptr, *b32v = nullptr, *r32v = nullptr;
    // l1-Jacobi levels above the coarse tail keep a second iterate buffer: a
    // sweep reads one and writes the other (one pass over A); xcur tracks, while
    // a cycle is recorded, which of the two holds x
    DBuf<double> xa64;
    DBuf<float> xa32;
    int xcur = 0;
    DBuf<int32_t> d_cptr;  // colour offsets on the device (levels run by the tail kernel)
    // row-permuted copy (rows grouped by colour) for the streaming smoother
    DBuf<int32_t> gs_ptr, gs_col;
    DBuf<double> gs_val64;
    DBuf<float> gs_val32;
    const int32_t *gs_ptr_v = nullptr, *gs_col_v = nullptr;
    const double* gs_val64_v = nullptr;
    const float* gs_val32_v = nullptr;
    // l1-Jacobi smoothing (small coarse levels): d_i = sum_j |a_ij|
    int32_t jac = 0;
    DBuf<double> dl1_64;
    DBuf<float> dl1_32;
    // finest level in colour order (perm): the cycle's vectors are indexed by
    // position t in the colour-grouped row order (row colour_rows0[t]); Ap is A
    // in that order (the permuted copy with renumbered columns), and the
    // transfer data are restated for it: aggp[t] = agg[row], memp = positions of
    // agg_mem (same order), pvalp[t] = pval[row]
    bool perm = false;
    Csr Ap;
    DBuf<int32_t> aggp, memp;
    DBuf<double> pvalp;
    DBuf<float> pvalp32;
};

// Level view used by the single-block coarse tail (k_tail.cu).
template <class T>
struct TailLevel {
    int n, nc, ncolour, lpr, jac;
    const T* dl1;
    const int *rowptr, *col;
    const T* val;
    const int *cptr, *crows;
    const int *agg, *agg_ptr, *agg_mem;
    const T* pval;
    T *x, *b, *r;
};
template <class T>
void tail_cycle(cudaStream_t s, const TailLevel<T>* lv, int l0, int L, int gamma, int nu_pre,
                int nu_post, const double* Xinv, int fresh);
// The tail's operator N (x = N b for `visits` consecutive visits, the first
// from a zero start), formed column by column; n[l] = unknowns of level l; N
// row-major, row stride ld.
template <class T>
bool tail_operator_fits(const int* n, int l0, int L);
template <class T>
void tail_operator(cudaStream_t s, const TailLevel<T>* lv, const int* n, int l0, int L, int gamma,
                   int nu_pre, int nu_post, const double* Xinv, T* Nout, int ld, int nsm, int visits);
// x = N v, or x += N v (accum)
template <class T>
void tail_gemv(cudaStream_t s, int m, int ld, const T* Nm, const T* v, T* x, bool accum);

struct Hier {
    int32_t nlev = 0;
    Level lev[kMaxLevels];
    int32_t nL = 0;
    DBuf<double> Xinv;   // nL x nL pinned pseudo-inverse of the coarsest matrix
    int32_t npinned = 0;
    double oc = 0.0;
    int32_t lt = -1;                 // first level run by the coarse tail kernel
    DBuf<unsigned char> tail;        // TailLevel<T>[nlev] on the device
    // dense operator of the tail levels per cycle kind (index gamma-1), when
    // params.tail_dense selects it; row-major m x tail_ld, m = lev[lt].n
    DBuf<unsigned char> tail_op[2];
    bool tail_op_tried[2] = {false, false};
    // buffers of the batched cycle (pcamg_solve_multi): per level K
    // row-interleaved vectors x, a second x (l1-Jacobi levels), b and r, in
    // the cycle precision; mv_K = the K they were sized for
    int mv_K = 0;
    DBuf<unsigned char> mv_x[kMaxLevels], mv_x2[kMaxLevels], mv_b[kMaxLevels], mv_r[kMaxLevels];
    // visits of the tail's first level that one product with tail_op[k] stands
    // for: gamma when the parent (level lt - 1) applies it, 1 when lt = 0
    int tail_visits[2] = {1, 1};
    int32_t tail_ld = 0;
    // CUDA graphs of the cycle: 0 V-cycle from zero, 1 W-cycle from zero,
    // 2 V-cycle continuing from the finest level's current x, 3 the same right
    // after another such cycle's post-sweep (its pre-sweep starts at the
    // second colour: the first colour's update would repeat, bit for bit, the
    // last one of that post-sweep)
    cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t graph_kernels[4] = {0, 0, 0, 0};
    // event-record nodes around the finest-level pre-sweep and residual of the
    // V-cycle graphs of kinds 0 and 2 (params.profile bit 1), retargeted to
    // fresh events before each replay
    cudaGraphNode_t prof_node[4][4] = {};   // finest-level pre-sweep start/end, residual start/end
    cudaGraph_t graph_tmpl[4] = {nullptr, nullptr, nullptr, nullptr};   // graphs those nodes belong to
    ~Hier();
};

// A stream owned by the context; declared before every buffer so that it is
// destroyed after them (their frees are enqueued on it).
struct OwnedStream {
    cudaStream_t s = nullptr;
    ~OwnedStream() {
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    }
};

struct Reweighted;

struct Ctx {
    pcamg_params p{};
    OwnedStream own;
    cudaStream_t user = nullptr;    // the caller's stream
    cudaStream_t stream = nullptr;  // where this context's work runs
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    Mem mem;
    int32_t n = 0;
    int64_t nnz = 0;
    DBuf<int32_t> rowptr, col;
    DBuf<double> val;
    DBuf<float> val32;
    // level-0 colouring (A is the same in every hierarchy)
    int32_t ncolour0 = 0;
    DBuf<int32_t> colour0, colour_rows0;
    std::vector<int32_t> h_colour_ptr0;
    DBuf<int32_t> gs_ptr0, gs_col0;   // row-permuted copy of A by colour
    DBuf<double> gs_val0_64;
    DBuf<float> gs_val0_32;
    // finest-level vectors of the batched cycles (K row-interleaved x, b, r;
    // shared by every hierarchy, so each factor of the composite continues
    // from the last), sized for mv0_K vectors in the cycle precision
    int mv0_K = 0;
    DBuf<unsigned char> mv0_x, mv0_b, mv0_r;
    // perm0: the cycles keep the finest level in colour order; gs_col0 then
    // holds positions (iperm0[column]) and iperm0[row] = position of the row
    bool perm0 = false;
    DBuf<int32_t> iperm0;
    std::vector<Hier*> hist;
    // driver work vectors (length n)
    DBuf<double> w_r, w_c, w_e, w_t1, w_t2, w_z, w_p, w_q, w_rold, w_eh, w_ein, w_cin;
    // finest-level cycle vectors shared by every hierarchy (cycle precision)
    DBuf<double> l0_x64, l0_b64, l0_r64;
    DBuf<float> l0_x32, l0_b32, l0_r32;
    DBuf<double> red;     // reduction partials + scalar slots
    int64_t npartials = 4096;
    double* h_red = nullptr;  // pinned host mirror of the scalar slots
    std::string last_error;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int64_t prof_launches = 0;
    double prof_ms = 0.0;
    // timing of the V-cycle's finest-level residual (params.profile bit 1):
    // event pairs recorded around it, resolved when the solve ends
    std::vector<cudaEvent_t> cyc_ev;
    size_t cyc_used = 0;
    cudaEvent_t cyc_tmpl[4] = {nullptr, nullptr, nullptr, nullptr};   // events named in the captured nodes
    int64_t cyc_launches = 0;
    double cyc_ms = 0.0;
    int64_t gs_sweeps = 0;   // finest-level pre-smoothing sweeps timed
    double gs_ms = 0.0;
    int64_t ncycles = 0;
    int64_t nwcycles = 0;
    bool fixed_scale = false;   // FP32 cycle scale set once for the running solve
    int cur_kind = 0;           // cycle graph kind being run or captured
    double t_alg2 = 0.0, t_alg4 = 0.0;
    const double* last_e = nullptr;          // normalised error of the newest hierarchy
    std::unique_ptr<Reweighted> mpnn_cand;   // A^2 candidate pattern for the network's loss
    // the A^2 candidate pattern of Alg. 4 step 2 (row pointers and columns):
    // it depends on A alone, so the first build forms it and later builds copy it
    DBuf<int32_t> cand_ptr, cand_col;
    int64_t cand_nnz = -1;
    DBuf<int64_t> scan_ws;                   // one-pass scan bookkeeping (k_vector.cu)
    ~Ctx();
};

// ---------------------------------------------------------------- kernels (launch wrappers)
// vector ops (k_vector.cu)
int reduce_blocks(int64_t n);
// partial[0..nb) then a second pass writes out[0]; deterministic for fixed n
void dot(cudaStream_t s, int64_t n, const double* x, const double* y, double* partial, double* out);
void sum(cudaStream_t s, int64_t n, const double* x, double* partial, double* out);
void axpy(cudaStream_t s, int64_t n, double a, const double* x, double* y);           // y += a x
void axpy_dev(cudaStream_t s, int64_t n, const double* a, double sign, const double* x, double* y);  // y += sign*(*a) x
void xpby_dev(cudaStream_t s, int64_t n, const double* x, const double* beta, double* y);          // y = x + (*beta) y
void sub_mean(cudaStream_t s, int64_t n, double* x, const double* total);  // x -= total/n
void scale_dev(cudaStream_t s, int64_t n, double* x, const double* num, const double* den);  // x *= num/den
void copy(cudaStream_t s, int64_t n, const double* x, double* y);
void fill(cudaStream_t s, int64_t n, double v, double* y);
void fill_i32(cudaStream_t s, int64_t n, int32_t v, int32_t* y);
void cast_scaled_f32(cudaStream_t s, int64_t n, const double* x, const double* inv_scale, float* y);
void add_scaled_f32(cudaStream_t s, int64_t n, const float* c, const double* scale, double* x);  // x += scale*c
void set_scaled_f32(cudaStream_t s, int64_t n, const float* c, const double* scale, double* x);  // x = scale*c
// y_t = (float)(x_idx(t) * inv); x_t = scale * c_idx(t); y_t = x_idx(t)
void gather_scaled_f32(cudaStream_t s, int64_t n, const int32_t* idx, const double* x, const double* inv, float* y);
void gather_set_scaled_f32(cudaStream_t s, int64_t n, const int32_t* idx, const float* c, const double* scale,
                           double* x);
template <class T>
void gather(cudaStream_t s, int64_t n, const int32_t* idx, const T* x, T* y);
void invert_perm(cudaStream_t s, int32_t n, const int32_t* idx, int32_t* inv);       // inv[idx[t]] = t
void mark_diagonal(cudaStream_t s, int32_t n, const int32_t* ptr, int32_t* col);     // col == i -> ~i in row i
void map_index(cudaStream_t s, int64_t n, const int32_t* map, const int32_t* x, int32_t* y);  // y = map[x]
void cast_f32(cudaStream_t s, int64_t n, const double* x, float* y);
void cast_f64(cudaStream_t s, int64_t n, const float* x, double* y);
void philox_uniform(cudaStream_t s, uint64_t seed, int64_t n, double* out);
void scalar_ops(cudaStream_t s, int op, double* slots, int a, int b, int c);  // small device scalar algebra
// scalar_ops ops
enum { SOP_DIV = 0, SOP_SQRT = 1, SOP_INV_SQRT = 2, SOP_PCG_ALPHA = 3, SOP_NEG_DIV = 4, SOP_INV = 5 };

// sparse level operators (k_spmv.cu)
void residual64(cudaStream_t s, const Csr& A, const double* x, const double* b, double* r,
                double* partial, double* norm2);
void residual32(cudaStream_t s, const Csr& A, const float* x, const float* b, float* r);
void spmv64(cudaStream_t s, const Csr& A, const double* x, double* y);  // y = A x
template <class T>
void gs_colour(cudaStream_t s, const Csr& A, const int32_t* rows, int32_t nrows, const T* b, T* x);
template <class T>
void gs_colour_perm(cudaStream_t s, int32_t beg, int32_t end, const int32_t* rows, const int32_t* pptr,
                    const int32_t* pcol, const T* pval, const T* b, T* x);
template <class T>
void permute_rows(Ctx& c, int32_t n, const int32_t* rows, const int32_t* rowptr, const int32_t* col,
                  const double* val, DBuf<int32_t>& pptr, DBuf<int32_t>& pcol, DBuf<T>& pval);
int residual_partials(int32_t n);
int residual_norm_blocks(int32_t n);   // partials the ||r||^2 launch of residual64 writes
bool use_stream(int32_t rows, int lpr);  // streaming kernels pay off for this launch
template <class T>
void jacobi_update(cudaStream_t s, int32_t n, const T* r, const T* d, T* x);   // x += r / d
// xout = x + (b - A x) / d in one pass (an l1-Jacobi sweep into another buffer)
template <class T>
void jacobi_sweep(cudaStream_t s, const Csr& A, const T* x, const T* b, const T* d, T* xout);
void l1_diagonal(cudaStream_t s, int32_t n, const int32_t* rowptr, const double* val, double* d);
template <class T>
void restrict_agg(cudaStream_t s, int32_t nc, const int32_t* agg_ptr, const int32_t* agg_mem,
                  const T* pval, const T* r, T* bc, T* xc, const T* dc);
template <class T>
void prolong_add(cudaStream_t s, int32_t n, const int32_t* agg, const T* pval, const T* xc, T* x);
template <class T>
void coarse_apply(cudaStream_t s, int32_t m, const double* Xinv, const T* b, T* x);

// setup (k_setup.cu, k_colour.cu, k_dense.cu)
struct Reweighted {  // reweighted graph of one level, rows in column order
    DBuf<int32_t> ptr, col;
    DBuf<double> w;
    int64_t nnz = 0;
};
void build_candidates(Ctx& c, const double* e, Reweighted& out);
int32_t path_cover(Ctx& c, int32_t n, const Reweighted& t, int32_t* nbr0, int32_t* nbr1);
// Alg. 3 on one level: returns nc; fills agg (n), cover of the next level (nc)
int32_t aggregate_level(Ctx& c, int32_t n, const int32_t* nbr0, const int32_t* nbr1,
                        const Reweighted& t, DBuf<int32_t>& agg, DBuf<int32_t>& cnbr0,
                        DBuf<int32_t>& cnbr1, int32_t* rounds);
// MWM aggregation of one level (Section 2.1); returns the number of aggregates
int32_t mwm_aggregate_level(Ctx& c, int32_t n, const int32_t* rowptr, const int32_t* col,
                            const double* val, DBuf<int32_t>& agg, int32_t* rounds_out);
void build_members(Ctx& c, int32_t n, int32_t nc, const int32_t* agg, DBuf<int32_t>& agg_ptr,
                   DBuf<int32_t>& agg_mem);
void build_pval(Ctx& c, int32_t n, int32_t nc, const int32_t* agg_ptr, const int32_t* agg_mem,
                const double* e, DBuf<double>& pval);
// Galerkin: (I,J) sums of (p_u a_uv) p_v over members of I ascending then row order
int64_t galerkin(Ctx& c, int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                 int32_t nc, const int32_t* agg, const int32_t* agg_ptr, const int32_t* agg_mem,
                 const double* pval, bool drop_diag, DBuf<int32_t>& optr, DBuf<int32_t>& ocol,
                 DBuf<double>& oval);
int32_t colour_smoother(Ctx& c, int32_t n, const int32_t* rowptr, const int32_t* col, uint64_t seed,
                        int32_t* colour);
int32_t colour_graph(Ctx& c, int32_t n, const int32_t* rowptr, const int32_t* col, uint64_t seed,
                     int32_t* colour);
void colour_lists(Ctx& c, int32_t n, const int32_t* colour, int32_t ncolour,
                  DBuf<int32_t>& rows, std::vector<int32_t>& h_ptr);
void coarse_factor(Ctx& c, int32_t m, const int32_t* rowptr, const int32_t* col, const double* val,
                   bool force_last, DBuf<double>& Xinv, int32_t* npinned);

// hierarchy + driver (hierarchy.cu, driver.cu)
Hier* build_hierarchy(Ctx& c, const double* e_normalised);
Hier* build_hierarchy_mwm(Ctx& c);   // MWM_setup: boolean UA-AMG hierarchy (Section 2.1)
void cycle(Ctx& c, Hier& h, int gamma, const double* r, double* out);
void smooth_error(Ctx& c, const double* r, double* e);
void start_vector(Ctx& c, double* e);
pcamg_status solve(Ctx& c, const double* b, double* x, pcamg_stats* st);
pcamg_status solve_zero_rhs(Ctx& c, double* x, pcamg_stats* st);
void normalise_orth(Ctx& c, const double* e, double* out);  // (e - mean)/||e - mean||
double* red_partials(Ctx& c);        // reduction partials of the context
double* mpnn_slots(Ctx& c);          // 8 device scalars for the network's reductions
const double* norm_slot(Ctx& c);     // ||e - mean|| of the last normalise_orth

// learned start vector (k_mpnn.cu)
constexpr int kMpnnHidden = 64;
constexpr int kMpnnLayers = 4;
constexpr int kMpnnParams = 64 * 3 + 64 + 4 * (64 * 128 + 64) + 64 + 1;   // 33345
void set_allocator(pcamg_alloc_fn a, pcamg_free_fn f, void* ctx);
void trim_memory();

struct Mpnn;
Mpnn* mpnn_create(const float* h_params);
void mpnn_destroy(Mpnn* m);
void mpnn_set_params(Mpnn& m, const float* h_params);   // also resets the Adam state
void mpnn_get_params(Mpnn& m, float* h_params);
void mpnn_get_grad(Mpnn& m, float* h_grad);
void mpnn_forward(Ctx& c, Mpnn& m, const double* u, double* yhat);
double mpnn_loss_grad(Ctx& c, Mpnn& m, const double* u, const double* target);  // gradient kept in m
void mpnn_adam(Mpnn& m, float lr);

// small helpers
template <class T>
void d2h(Ctx& c, T* host, const T* dev, size_t count);
void sync(Ctx& c);
int64_t read_i64(Ctx& c, const int64_t* dev);
int32_t read_i32(Ctx& c, const int32_t* dev);
// batched kernels (k_multi.cu): K = 1, 2, 4 or 8 row-interleaved vectors.
// mv_rows mode 0: out = b - A x; 1: out = x + (b - A x) / d; 2: Gauss-Seidel on
// rows (rows ? rows[t] : beg + t), out == x
template <class T>
void mv_rows(cudaStream_t s, int mode, int K, int nrows, const int* rows, int beg, const Csr& A, const T* x,
             const T* b, const T* d, T* out);
template <class T>
void mv_restrict(cudaStream_t s, int K, int nc, const int* agg_ptr, const int* mem, const T* pval, const T* r,
                 T* bc, T* xc, const T* dc);
template <class T>
void mv_prolong(cudaStream_t s, int K, int n, const int* agg, const T* pval, const T* xc, T* x);
template <class T>
void mv_dense(cudaStream_t s, int K, int m, int ld, const T* N, const T* v, T* x, bool accum);
template <class T>
void mv_coarse(cudaStream_t s, int K, int m, const double* X, const T* b, T* x, bool accum);
template <class T>
void mv_in(cudaStream_t s, int K, int kr, int n, const int* perm, const double* r, const double* inv, T* v);
template <class T>
void mv_out(cudaStream_t s, int K, int kr, int n, const int* iperm, const T* v, const double* scale, double* z);
// k right-hand sides, column-major n x k (driver.cu)
pcamg_status solve_multi(Ctx& c, int32_t k, const double* B, double* X, int32_t* iters, double* rel_res);
double read_f64(Ctx& c, const double* dev);
// exclusive scan of int32 counts into int32 offsets (out has n+1 entries); returns total
int64_t scan_i32(Ctx& c, const int32_t* in, int32_t* out, int64_t n);
int64_t scan_i64(Ctx& c, const int64_t* in, int64_t* out, int64_t n);
// the same without reading the total back (no host synchronisation)
void scan_i32_device(Ctx& c, const int32_t* in, int32_t* out, int64_t n);

}  // namespace pc
