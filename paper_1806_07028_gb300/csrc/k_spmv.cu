// Sparse level operators of the cycle: residual r = b - A x (with the fused
// ||r||^2 partials), one colour of a Gauss-Seidel sweep, restriction by P^T,
// prolongation by P, and the dense coarsest solve.
//
// Rows are processed by groups of LPR lanes (LPR = power of two >= the mean
// row length, so a warp reads several consecutive rows as one coalesced run of
// column indices and values); each group reduces with warp shuffles.
#include "pcamg_internal.cuh"

namespace pc {

// Lanes cooperating on one row in the sub-warp kernels: enough that each lane
// takes about three entries of an average row (2..32).
int lanes_per_row(int32_t n, int64_t nnz) {
    double avg = n > 0 ? (double)nnz / (double)n : 1.0;
    int l = 2;
    while (l < 32 && 3.0 * l < avg) l <<= 1;
    return l;
}

namespace {

// one rounding per multiply-add, in both precisions
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }

template <int LPR, class T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o, LPR);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// One pass over the rows (no grid-stride loop): every row group is its own
// warp slot, so the whole level's loads are in flight at once.
inline int sparse_grid(int64_t rows, int lpr, int block = kBlock) {
    int64_t threads = rows * lpr;
    int64_t g = (threads + block - 1) / block;
    if (g < 1) g = 1;
    if (g > (int64_t)1 << 30) g = (int64_t)1 << 30;
    return (int)g;
}

// r = b - A x; when partial != null, block b writes sum of r_i^2 of its rows.
// With dl1 given the launch is one l1-Jacobi sweep instead: r receives the new
// iterate x_i + (b_i - sum_j a_ij x_j) / dl1_i (x is not written).
// A lane's first kPre entries of its row (column, value) and the row's dl1 are
// hierarchy data, loaded ahead of pdl_wait(); after it only x and b are read,
// so a cycle launch's dependent chain starts at the x gathers. A lane adds its
// entries in the same order either way.
constexpr int kPre = 2;

template <class T, int LPR>
__global__ void __launch_bounds__(kBlock) k_residual(int n, const int* __restrict__ rowptr,
                                                     const int* __restrict__ col,
                                                     const T* __restrict__ val,
                                                     const T* __restrict__ x,
                                                     const T* __restrict__ b, T* __restrict__ r,
                                                     double* __restrict__ partial,
                                                     const T* __restrict__ dl1 = nullptr) {
    constexpr int RPW = 32 / LPR;
    const int lane = threadIdx.x & 31;
    const int sub = lane % LPR, grp = lane / LPR;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double acc2 = 0.0;
    int64_t row0 = warp * RPW;
    // this group's first row: its hierarchy data before the wait
    int beg = 0, end = 0;
    int pc[kPre];
    T pv[kPre];
    T dr = 1;
    auto prefetch = [&](int64_t row) {
        beg = end = 0;
        dr = 1;
        if (row < n) {
            beg = __ldg(rowptr + row);
            end = __ldg(rowptr + row + 1);
            if (dl1 && sub == 0) dr = __ldg(dl1 + row);
        }
#pragma unroll
        for (int q = 0; q < kPre; ++q) {
            const int k = beg + sub + q * LPR;
            pc[q] = k < end ? __ldg(col + k) : 0;
            pv[q] = k < end ? __ldg(val + k) : T(0);
        }
    };
    prefetch(row0 + grp);
    pdl_wait();
    pdl_trigger();
    for (; row0 < n; row0 += nwarps * RPW) {
        const int64_t row = row0 + grp;
        T s = 0, xr = 0, bv = 0;
        if (row < n) {
            if (sub == 0) {   // issued with the gathers, not after the sum
                bv = __ldg(b + row);
                if (dl1) xr = x[row];
            }
#pragma unroll
            for (int q = 0; q < kPre; ++q)
                if (beg + sub + q * LPR < end) s = fma_t(pv[q], __ldg(x + pc[q]), s);
            for (int k = beg + sub + kPre * LPR; k < end; k += LPR) s = fma_t(__ldg(val + k), __ldg(x + __ldg(col + k)), s);
        }
        s = group_sum<LPR>(s);
        if (sub == 0 && row < n) {
            T rr = bv - s;
            if (dl1) r[row] = xr + rr / dr;
            else r[row] = rr;
            acc2 += (double)rr * (double)rr;
        }
        if (row0 + nwarps * RPW < n) prefetch(row0 + nwarps * RPW + grp);
    }
    if (partial) {
        __shared__ double ws[kBlock / 32];
        acc2 = warp_sum_d(acc2);
        if (lane == 0) ws[threadIdx.x >> 5] = acc2;
        __syncthreads();
        if (threadIdx.x < 32) {
            double v = threadIdx.x < kBlock / 32 ? ws[threadIdx.x] : 0.0;
            v = warp_sum_d(v);
            if (threadIdx.x == 0) partial[blockIdx.x] = v;
        }
    }
}

__global__ void k_finish(int nb, const double* __restrict__ partial, double* __restrict__ out) {
    __shared__ double ws[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
    s = warp_sum_d(s);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
        v = warp_sum_d(v);
        if (threadIdx.x == 0) *out = v;
    }
}

// y = A x
template <int LPR>
__global__ void __launch_bounds__(kBlock) k_spmv(int n, const int* __restrict__ rowptr,
                                                 const int* __restrict__ col,
                                                 const double* __restrict__ val,
                                                 const double* __restrict__ x,
                                                 double* __restrict__ y) {
    constexpr int RPW = 32 / LPR;
    const int lane = threadIdx.x & 31;
    const int sub = lane % LPR, grp = lane / LPR;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row0 = warp * RPW; row0 < n; row0 += nwarps * RPW) {
        int64_t row = row0 + grp;
        double s = 0;
        if (row < n) {
            int beg = __ldg(rowptr + row), end = __ldg(rowptr + row + 1);
            for (int k = beg + sub; k < end; k += LPR) s = fma_t(__ldg(val + k), __ldg(x + __ldg(col + k)), s);
        }
        s = group_sum<LPR>(s);
        if (sub == 0 && row < n) y[row] = s;
    }
}

// One colour of Gauss-Seidel: x_i = (b_i - sum_{j != i} a_ij x_j) / a_ii for the
// listed rows. Rows of one colour share no edge, so they update independently.
template <class T, int LPR>
__global__ void __launch_bounds__(kBlock) k_gs(int nrows, const int* __restrict__ rows,
                                               const int* __restrict__ rowptr,
                                               const int* __restrict__ col,
                                               const T* __restrict__ val,
                                               const T* __restrict__ b, T* __restrict__ x) {
    constexpr int RPW = 32 / LPR;
    const int lane = threadIdx.x & 31;
    const int sub = lane % LPR, grp = lane / LPR;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    pdl_wait();
    pdl_trigger();
    for (int64_t t0 = warp * RPW; t0 < nrows; t0 += nwarps * RPW) {
        int64_t t = t0 + grp;
        T s = 0, d = 0;
        int row = -1;
        if (t < nrows) {
            row = __ldg(rows + t);
            int beg = __ldg(rowptr + row), end = __ldg(rowptr + row + 1);
            for (int k = beg + sub; k < end; k += LPR) {
                int j = __ldg(col + k);
                T a = __ldg(val + k);
                if (j == row) d = a;
                else s = fma_t(a, x[j], s);
            }
        }
        s = group_sum<LPR>(s);
        d = group_sum<LPR>(d);
        if (sub == 0 && t < nrows) x[row] = (__ldg(b + row) - s) / d;
    }
}

// bc_I = sum over members u of aggregate I (ascending) of p_u r_u, and the
// child's start value: zero, or bc_I / d_I when the child begins with an
// l1-Jacobi sweep from zero (x = 0 + (b - A 0) / d = b / d exactly).
template <class T>
__global__ void k_restrict(int nc, const int* __restrict__ agg_ptr, const int* __restrict__ mem,
                           const T* __restrict__ pval, const T* __restrict__ r, T* __restrict__ bc,
                           T* __restrict__ xc, const T* __restrict__ dc) {
    // the aggregate's first two members and their p are hierarchy data, read
    // ahead of the wait (aggregates of paths are mostly pairs)
    const int stride = gridDim.x * blockDim.x;
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    int beg = 0, end = 0, u0 = 0, u1 = 0;
    T p0 = 1, p1 = 1;
    auto prefetch = [&](int J) {
        if (J >= nc) return;
        beg = __ldg(agg_ptr + J);
        end = __ldg(agg_ptr + J + 1);
        u0 = beg < end ? __ldg(mem + beg) : 0;
        u1 = beg + 1 < end ? __ldg(mem + beg + 1) : u0;
        if (pval) { p0 = __ldg(pval + u0); p1 = __ldg(pval + u1); }
    };
    prefetch(I);
    pdl_wait();
    pdl_trigger();
    for (; I < nc; I += stride) {
        T s = 0;
        if (beg < end) s += pval ? p0 * __ldg(r + u0) : __ldg(r + u0);
        if (beg + 1 < end) s += pval ? p1 * __ldg(r + u1) : __ldg(r + u1);
        for (int t = beg + 2; t < end; ++t) {
            int u = __ldg(mem + t);
            s += pval ? __ldg(pval + u) * __ldg(r + u) : __ldg(r + u);
        }
        bc[I] = s;
        if (xc) xc[I] = dc ? s / __ldg(dc + I) : T(0);
        prefetch(I + stride);
    }
}

template <class T>
__global__ void k_prolong(int n, const int* __restrict__ agg, const T* __restrict__ pval,
                          const T* __restrict__ xc, T* __restrict__ x) {
    // agg and p at the row are hierarchy data, read ahead of the wait
    const int stride = gridDim.x * blockDim.x;
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    int a = 0;
    T p = 1;
    if (u < n) { a = __ldg(agg + u); if (pval) p = __ldg(pval + u); }
    pdl_wait();
    pdl_trigger();
    for (; u < n; u += stride) {
        T c = __ldg(xc + a);
        x[u] += pval ? p * c : c;
        if (u + stride < n) { a = __ldg(agg + u + stride); if (pval) p = __ldg(pval + u + stride); }
    }
}

// x = Xinv b, one warp per row (Xinv row-major, FP64)
template <class T>
__global__ void k_coarse_apply(int m, const double* __restrict__ X, const T* __restrict__ b,
                               T* __restrict__ x) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < m; i += nw) {
        double s = 0.0;
        for (int j = lane; j < m; j += 32) s += X[(size_t)i * m + j] * (double)b[j];
        s = warp_sum_d(s);
        if (lane == 0) x[i] = (T)s;
    }
}

// ---- CSR-stream kernels -----------------------------------------------------
// A block owns a tile of kStreamRows consecutive rows. It walks the tile's
// entries in chunks of kStreamChunk: every thread computes products a_k x_col(k)
// for entries of the chunk (coalesced loads of col and val, independent loads of
// x, so many are in flight), stages them in shared memory, and then each thread
// adds the products of its own row in CSR order. A row's sum is therefore taken
// left to right, with one rounding per product and per addition.
constexpr int kStreamRows = 256;
// entries staged per chunk (FP64 stages a value and an x per entry, FP32 one product)
template <class T>
constexpr int kStreamChunk = 2048;
// below this many rows a launch of the streaming kernels would not fill the GPU
constexpr int kStreamMinRows = kNumSMs * kStreamRows * 2;

// Entries [c0, c1) staged in shared memory. FP64: the value a_k into av and
// the gathered x_col(k) into xv, so the row sum can take one fused multiply-add
// per entry (GB300's FP64 rate makes the separate multiply the bottleneck).
// FP32: the product a_k x_col(k) into av (FP32 arithmetic is plentiful and
// half the staging traffic is saved). Each thread first loads kUnroll column
// indices and values (independent, coalesced), then the kUnroll gathered x, so
// many loads are in flight per thread. x is read with ordinary loads when the
// caller writes it in the same kernel (GS).
template <class T>
constexpr int kUnroll = kStreamChunk<T> / kStreamRows;

template <class T>
constexpr int kXv = sizeof(T) == 8 ? kStreamChunk<T> : 1;

// Column indices and values of one chunk, entry c0 + tid + u * kStreamRows in
// slot u, held in registers between their (coalesced, independent) loads and
// the staging.
template <class T>
struct ChunkRegs {
    int cj[kUnroll<T>];
    T cv[kUnroll<T>];
};

template <class T>
__device__ __forceinline__ void load_chunk(int c0, int c1, const int* __restrict__ col, const T* __restrict__ val,
                                           ChunkRegs<T>& R) {
#pragma unroll
    for (int u = 0; u < kUnroll<T>; ++u) {
        const int k = c0 + threadIdx.x + u * kStreamRows;
        R.cj[u] = (k < c1) ? __ldg(col + k) : 0;
        R.cv[u] = (k < c1) ? __ldg(val + k) : T(0);
    }
}

// Stage entries [c0, c1) held in R: gather x_col(k) (ordinary loads: the GS
// kernel writes x) and store value and x (FP64) or their product (FP32), and
// the column (KEEP_COL, GS on a row list) in shared memory.
// DM: diagonal entries are marked (column ~row) and the rows are in place. A
// residual (GS = false) decodes the column; a Gauss-Seidel colour (GS = true)
// stages a zero contribution for the diagonal entry, gathers nothing for it
// and keeps its value in dsm[row - r0] (r0 = the tile's first row), so a row's
// sum is its off-diagonal terms in CSR order, as without the mark.
template <class T, bool KEEP_COL, bool DM = false, bool GS = false>
__device__ __forceinline__ void stage_regs(int c0, int c1, const ChunkRegs<T>& R, const T* x, T* av, T* xv,
                                           int* pc, T* dsm = nullptr, int r0 = 0) {
    T xg[kUnroll<T>];
#pragma unroll
    for (int u = 0; u < kUnroll<T>; ++u) {
        const int k = c0 + threadIdx.x + u * kStreamRows;
        int j = R.cj[u];
        bool on = k < c1;
        if (DM) {
            if (GS) on = on && j >= 0;
            else j = j < 0 ? ~j : j;
        }
        xg[u] = on ? x[j] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kUnroll<T>; ++u) {
        const int k = c0 + threadIdx.x + u * kStreamRows;
        if (k < c1) {
            T a = R.cv[u];
            if (DM && GS && R.cj[u] < 0) {
                dsm[~R.cj[u] - r0] = a;
                a = T(0);
            }
            if constexpr (sizeof(T) == 8) { av[k - c0] = a; xv[k - c0] = xg[u]; }
            else av[k - c0] = a * xg[u];
            if (KEEP_COL) pc[k - c0] = R.cj[u];
        }
    }
}

// add entry k's contribution to s (see stage_regs)
template <class T>
__device__ __forceinline__ T row_add(const T* av, const T* xv, int i, T s) {
    if constexpr (sizeof(T) == 8) return fma_t(av[i], xv[i], s);
    else return s + av[i];
}

// Where a tile's rows live: the tile's entry range [tb, te), this thread's row,
// its entry range [rb, re) and b at that row (loaded early, ahead of use).
template <class T>
struct TileMeta {
    int tb, te, rb, re, row;
    T bv, xv, dv;   // b, and for an l1-Jacobi sweep x and d, at this thread's row
};

// b (and, for an l1-Jacobi sweep (JAC), x and d) at the row are loaded here, early
template <class T, bool PERM, bool WITH_B = true, bool JAC = false>
__device__ __forceinline__ TileMeta<T> tile_meta(int t0, int tend, const int* __restrict__ ptr,
                                                 const int* __restrict__ rows, const T* __restrict__ b,
                                                 const T* x = nullptr, const T* __restrict__ dl1 = nullptr) {
    TileMeta<T> m;
    const int tl = min(t0 + kStreamRows, tend);
    const int t = t0 + threadIdx.x;
    m.tb = __ldg(ptr + t0);
    m.te = __ldg(ptr + tl);
    m.rb = m.re = 0;
    m.row = -1;
    m.bv = m.xv = T(0);
    m.dv = T(1);
    if (t < tend) {
        m.rb = __ldg(ptr + t);
        m.re = __ldg(ptr + t + 1);
        m.row = PERM ? __ldg(rows + t) : t;
        if (WITH_B) {
            m.bv = __ldg(b + m.row);
            if (JAC) { m.xv = x[m.row]; m.dv = __ldg(dl1 + m.row); }
        }
    }
    return m;
}

// A block owns tpb consecutive tiles of kStreamRows rows. While it adds up one
// chunk's rows from shared memory, the loads of the next chunk (of this tile or
// the first of the next tile) and the next tile's row pointers and b are
// already in flight, so the only exposed latency per tile is the x gather.
// The row sums keep the CSR order of each row. Without NORM (the launches
// inside cycle graphs) the first tile's row pointers and chunk (hierarchy
// data) are loaded before pdl_wait(), b and x after it; the NORM form (the
// outer FP64 residual, never a programmatic launch) has no wait.
//   PERM = false: rows t of [0, n) (residual r = b - A x, optional ||r||^2);
//   PERM = true:  permuted rows rows[t] of [beg, end) of one colour, Gauss-Seidel
//                 x_row = (b_row - sum_{j != row} a x_j) / a_row,row.
//   DM:           diagonal entries marked (column ~row), rows in place (rows is
//                 not read); the colour-ordered finest level.
template <class T, bool PERM, bool NORM, bool JAC = false, bool DM = false>
__device__ __forceinline__ void stream_tiles(int beg, int end, int tpb, const int* __restrict__ rows,
                                             const int* __restrict__ ptr, const int* __restrict__ col,
                                             const T* __restrict__ val, const T* x_in, const T* __restrict__ b,
                                             T* out, double* __restrict__ partial,
                                             const T* __restrict__ dl1 = nullptr) {
    constexpr bool KEEP = PERM && !DM;   // GS on a row list finds the diagonal by its column
    __shared__ T av[kStreamChunk<T>];
    __shared__ T xv[kXv<T>];
    __shared__ int pc[KEEP ? kStreamChunk<T> : 1];
    __shared__ T dsm[PERM && DM ? kStreamRows : 1];
    const int ntiles = (end - beg + kStreamRows - 1) / kStreamRows;
    const int tfirst = blockIdx.x * tpb;
    const int tstop = min(ntiles, tfirst + tpb);
    double rr2 = 0.0;
    constexpr bool kPdl = !NORM;
    if (tfirst < tstop) {
        TileMeta<T> M = tile_meta<T, PERM && !DM, !kPdl>(beg + tfirst * kStreamRows, end, ptr, rows, b);
        ChunkRegs<T> R;
        load_chunk<T>(M.tb, min(M.tb + kStreamChunk<T>, M.te), col, val, R);
        if (kPdl) {
            pdl_wait();
            pdl_trigger();
            if (M.row >= 0) {
                M.bv = __ldg(b + M.row);
                if (JAC) { M.xv = x_in[M.row]; M.dv = __ldg(dl1 + M.row); }
            }
        }
        for (int t = tfirst; t < tstop; ++t) {
            TileMeta<T> Mn = M;
            T s = 0, d = 0;
            for (int c0 = M.tb;;) {
                const int c1 = min(c0 + kStreamChunk<T>, M.te);
                stage_regs<T, KEEP, DM, PERM>(c0, c1, R, x_in, av, xv, pc, dsm, beg + t * kStreamRows);
                __syncthreads();
                // R is free again: start the loads the next round needs
                if (c1 < M.te) {
                    load_chunk<T>(c1, min(c1 + kStreamChunk<T>, M.te), col, val, R);
                } else if (t + 1 < tstop) {
                    Mn = tile_meta<T, PERM && !DM, true, JAC>(beg + (t + 1) * kStreamRows, end, ptr, rows, b, x_in, dl1);
                    load_chunk<T>(Mn.tb, min(Mn.tb + kStreamChunk<T>, Mn.te), col, val, R);
                }
                const int kb = max(M.rb, c0), ke = min(M.re, c1);
                for (int k = kb; k < ke; ++k) {
                    if (KEEP && pc[k - c0] == M.row) d = (sizeof(T) == 8) ? av[k - c0] : __ldg(val + k);
                    else s = row_add<T>(av, xv, k - c0, s);
                }
                // the tile's diagonal values are all staged once its last chunk is
                // (read before the barrier: the next tile overwrites them)
                if (PERM && DM && c1 >= M.te && M.row >= 0) d = dsm[M.row - (beg + t * kStreamRows)];
                __syncthreads();
                if (c1 >= M.te) break;
                c0 = c1;
            }
            if (M.row >= 0) {
                if (PERM) {
                    out[M.row] = (M.bv - s) / d;
                } else {
                    const T rr = M.bv - s;
                    if (JAC) out[M.row] = M.xv + rr / M.dv;   // l1-Jacobi sweep
                    else out[M.row] = rr;
                    if (NORM) rr2 = fma((double)rr, (double)rr, rr2);
                }
            }
            M = Mn;
        }
    } else if (kPdl) {
        pdl_wait();
        pdl_trigger();
    }
    if (NORM) {
        __shared__ double ws[kStreamRows / 32];
        rr2 = warp_sum_d(rr2);
        if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = rr2;
        __syncthreads();
        if (threadIdx.x < 32) {
            double v = threadIdx.x < kStreamRows / 32 ? ws[threadIdx.x] : 0.0;
            v = warp_sum_d(v);
            if (threadIdx.x == 0) partial[blockIdx.x] = v;
        }
    }
}

// Tiles per block: pipelining across tiles pays where FP64 arithmetic is the
// long pole (and with the norm it also divides the partial sums); the FP32 and
// Gauss-Seidel launches need every block they can get.
constexpr int kNormTiles = 4;
// tiles per block of a launch over rows [0, n): the host picks the grid
// (stream_grid), every block takes this many consecutive tiles
__device__ __forceinline__ int grid_tiles(int n) {
    const int ntiles = (n + kStreamRows - 1) / kStreamRows;
    return (ntiles + (int)gridDim.x - 1) / (int)gridDim.x;
}
// Tiles per block of the residual and Jacobi launches: pipelining across tiles
// pays where FP64 arithmetic is the long pole, and in FP32 on large levels (a
// block's second tile loads while its first is summed); smaller FP32 levels
// need every block they can get (measured on the 256^3 grid's levels).
template <class T>
inline int stream_tiles_per_block(int64_t rows, bool dmark) {
    if (sizeof(T) == 8 || dmark) return 2;
    return rows >= (3 << 20) ? 2 : 1;
}
template <class T>
inline int stream_grid(int64_t rows, bool dmark) {
    const int64_t nt = (rows + kStreamRows - 1) / kStreamRows;
    const int tpb = stream_tiles_per_block<T>(rows, dmark);
    return (int)std::max<int64_t>(1, (nt + tpb - 1) / tpb);
}
// Gauss-Seidel colours: two tiles per block (the second tile's loads overlap
// the first's sums) at five resident blocks per SM in FP32 (the best of 1-4
// tiles and 5-8 blocks measured on the 256^3 grid)
constexpr int kGsTiles = 2;
template <class T>
constexpr int kGsMinBlocks = sizeof(T) == 8 ? 4 : 5;
// residual launches: five resident blocks per SM in FP32 (the colour-ordered
// finest level's residual: 282 -> 244 us on the 256^3 grid, with two tiles)
template <class T, bool DM>
constexpr int kResMinBlocks = sizeof(T) == 4 ? 5 : 0;

// r_i = b_i - sum_k a_k x_col(k) (fused multiply-adds left to right in FP64);
// partial[block] = sum of r_i^2 of the block's rows when NORM; DM: diagonal
// entries marked (column ~i)
template <class T, bool NORM, bool DM = false>
__global__ void __launch_bounds__(kStreamRows, kResMinBlocks<T, DM>) k_res_stream(int n, const int* __restrict__ rowptr,
                                                             const int* __restrict__ col,
                                                             const T* __restrict__ val,
                                                             const T* __restrict__ x,
                                                             const T* __restrict__ b,
                                                             T* __restrict__ r,
                                                             double* __restrict__ partial) {
    stream_tiles<T, false, NORM, false, DM>(0, n, NORM ? kNormTiles : grid_tiles(n), nullptr, rowptr, col, val, x,
                                            b, r, partial);
}

// One l1-Jacobi sweep into another buffer: xout_i = x_i + (b_i - sum_j a_ij x_j) / dl1_i
template <class T>
__global__ void __launch_bounds__(kStreamRows, 5) k_jac_stream(int n, const int* __restrict__ rowptr,
                                                             const int* __restrict__ col,
                                                             const T* __restrict__ val,
                                                             const T* __restrict__ x,
                                                             const T* __restrict__ b,
                                                             const T* __restrict__ dl1,
                                                             T* __restrict__ xout) {
    stream_tiles<T, false, false, true>(0, n, grid_tiles(n), nullptr, rowptr, col, val, x, b, xout, nullptr, dl1);
}

// One colour of Gauss-Seidel on the row-permuted copy (rows of a colour are
// contiguous there): x_row = (b_row - sum_{j != row} a x_j) / a_row,row.
// DM: the vectors are in the copy's order (row = position, columns are
// positions, the diagonal marked); otherwise rows[t] names the row.
template <class T, bool DM>
__global__ void __launch_bounds__(kStreamRows, kGsMinBlocks<T>) k_gs_stream(int beg, int end, const int* __restrict__ rows,
                                                               const int* __restrict__ pptr,
                                                               const int* __restrict__ pcol,
                                                               const T* __restrict__ pval,
                                                               const T* __restrict__ b, T* __restrict__ x) {
    stream_tiles<T, true, false, false, DM>(beg, end, kGsTiles, rows, pptr, pcol, pval, x, b, x, nullptr);
}

// column of the diagonal entry of row i -> ~i (the rows' own columns are in
// the same numbering as the rows)
__global__ void k_mark_diag(int n, const int* __restrict__ ptr, int* __restrict__ col) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int k = ptr[i]; k < ptr[i + 1]; ++k)
            if (col[k] == i) col[k] = ~i;
}

template <class T>
__global__ void k_jacobi_update(int n, const T* __restrict__ r, const T* __restrict__ d, T* __restrict__ x) {
    pdl_wait();
    pdl_trigger();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        x[i] += r[i] / d[i];
}

// d_i = sum_j |a_ij|, left to right in CSR order
__global__ void k_l1_diagonal(int n, const int* __restrict__ rowptr, const double* __restrict__ val,
                              double* __restrict__ d) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) s += fabs(val[k]);
        d[i] = s;
    }
}

// Row-permuted copy: row t of the copy is row rows[t] of A.
__global__ void k_perm_counts(int n, const int* __restrict__ rows, const int* __restrict__ rowptr,
                              int* __restrict__ cnt) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        int r = rows[t];
        cnt[t] = rowptr[r + 1] - rowptr[r];
    }
}

template <class T>
__global__ void k_perm_fill(int n, const int* __restrict__ rows, const int* __restrict__ rowptr,
                            const int* __restrict__ col, const double* __restrict__ val,
                            const int* __restrict__ pptr, int* __restrict__ pcol, T* __restrict__ pval) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        int r = rows[t], o = pptr[t];
        for (int k = rowptr[r]; k < rowptr[r + 1]; ++k, ++o) {
            pcol[o] = col[k];
            pval[o] = (T)val[k];
        }
    }
}

inline int simple_grid(int64_t n) {
    int64_t g = (n + kBlock - 1) / kBlock;
    if (g < 1) g = 1;
    if (g > (int64_t)kNumSMs * 16) g = kNumSMs * 16;
    return (int)g;
}

}  // namespace

#define PC_LPR_DISPATCH(LPRV, CALL) \
    switch (LPRV) {                  \
        case 2: CALL(2); break;      \
        case 4: CALL(4); break;      \
        case 8: CALL(8); break;      \
        case 16: CALL(16); break;    \
        default: CALL(32); break;    \
    }

// streaming kernels: sparse rows (a tile of 256 rows then fits about one
// chunk) and enough rows to fill the GPU
bool use_stream(int32_t rows, int lpr) { return lpr <= 8 && rows >= kStreamMinRows; }

void residual64(cudaStream_t s, const Csr& A, const double* x, const double* b, double* r,
                double* partial, double* norm2) {
    if (A.dmark) {   // the colour-ordered finest level (always large enough to stream)
        if (norm2 || !use_stream(A.n, A.lpr)) fail(PCAMG_ERR_INVALID, "marked diagonal: streaming residual only");
        const int gt = stream_grid<double>(A.n, true);
        launch(k_res_stream<double, false, true>, gt, kStreamRows, 0, s, A.n, A.rowptr, A.col, A.val, x, b, r,
               (double*)nullptr);
        PC_LAUNCH("residual64");
        return;
    }
    if (use_stream(A.n, A.lpr) || norm2) {
        int g = (A.n + kStreamRows - 1) / kStreamRows;
        if (norm2) {
            const int gn = (g + kNormTiles - 1) / kNormTiles;   // <= residual_partials(n)
            k_res_stream<double, true><<<gn, kStreamRows, 0, s>>>(A.n, A.rowptr, A.col, A.val, x, b, r, partial); ::pc::count_launches(1);
            k_finish<<<1, 1024, 0, s>>>(gn, partial, norm2); ::pc::count_launches(1);
        } else {
            const int gt = stream_grid<double>(A.n, false);
            launch(k_res_stream<double, false>, gt, kStreamRows, 0, s, A.n, A.rowptr, A.col, A.val, x, b, r,
                   (double*)nullptr);
        }
    } else {
        int g = sparse_grid(A.n, A.lpr);
#define CALL(L) launch(k_residual<double, L>, g, kBlock, 0, s, A.n, A.rowptr, A.col, A.val, x, b, r, (double*)nullptr, (const double*)nullptr)
        PC_LPR_DISPATCH(A.lpr, CALL)
#undef CALL
    }
    PC_LAUNCH("residual64");
}

int residual_partials(int32_t n) { return (n + kStreamRows - 1) / kStreamRows; }
int residual_norm_blocks(int32_t n) { return (residual_partials(n) + kNormTiles - 1) / kNormTiles; }

// One l1-Jacobi sweep into another buffer: xout = x + (b - A x) / d, the same
// arithmetic as a residual followed by jacobi_update, in one pass over A.
template <class T>
void jacobi_sweep(cudaStream_t s, const Csr& A, const T* x, const T* b, const T* d, T* xout) {
    const T* val;
    if constexpr (sizeof(T) == 8) val = A.val; else val = A.val32;
    if (use_stream(A.n, A.lpr)) {
        int g = stream_grid<T>(A.n, false);
        launch(k_jac_stream<T>, g, kStreamRows, 0, s, A.n, A.rowptr, A.col, val, x, b, d, xout);
    } else {
        int g = sparse_grid(A.n, A.lpr);
#define CALL(L) launch(k_residual<T, L>, g, kBlock, 0, s, A.n, A.rowptr, A.col, val, x, b, xout, (double*)nullptr, d)
        PC_LPR_DISPATCH(A.lpr, CALL)
#undef CALL
    }
    PC_LAUNCH("jacobi_sweep");
}
template void jacobi_sweep<double>(cudaStream_t, const Csr&, const double*, const double*, const double*, double*);
template void jacobi_sweep<float>(cudaStream_t, const Csr&, const float*, const float*, const float*, float*);

template <class T>
void jacobi_update(cudaStream_t s, int32_t n, const T* r, const T* d, T* x) {
    launch(k_jacobi_update<T>, simple_grid(n), kBlock, 0, s, n, r, d, x);
    PC_LAUNCH("jacobi_update");
}
template void jacobi_update<double>(cudaStream_t, int32_t, const double*, const double*, double*);
template void jacobi_update<float>(cudaStream_t, int32_t, const float*, const float*, float*);

void l1_diagonal(cudaStream_t s, int32_t n, const int32_t* rowptr, const double* val, double* d) {
    k_l1_diagonal<<<simple_grid(n), kBlock, 0, s>>>(n, rowptr, val, d); ::pc::count_launches(1);
    PC_LAUNCH("l1_diagonal");
}

void residual32(cudaStream_t s, const Csr& A, const float* x, const float* b, float* r) {
    if (A.dmark && !use_stream(A.n, A.lpr)) fail(PCAMG_ERR_INVALID, "marked diagonal: streaming residual only");
    if (use_stream(A.n, A.lpr)) {
        const int g = stream_grid<float>(A.n, false);
        const int gdm = stream_grid<float>(A.n, true);
        if (A.dmark)
            launch(k_res_stream<float, false, true>, gdm, kStreamRows, 0, s, A.n, A.rowptr, A.col, A.val32, x, b, r,
                   (double*)nullptr);
        else
            launch(k_res_stream<float, false>, g, kStreamRows, 0, s, A.n, A.rowptr, A.col, A.val32, x, b, r,
                   (double*)nullptr);
    } else {
        int g = sparse_grid(A.n, A.lpr);
#define CALL(L) launch(k_residual<float, L>, g, kBlock, 0, s, A.n, A.rowptr, A.col, A.val32, x, b, r, (double*)nullptr, (const float*)nullptr)
        PC_LPR_DISPATCH(A.lpr, CALL)
#undef CALL
    }
    PC_LAUNCH("residual32");
}

void spmv64(cudaStream_t s, const Csr& A, const double* x, double* y) {
    int g = sparse_grid(A.n, A.lpr);
#define CALL(L) k_spmv<L><<<g, kBlock, 0, s>>>(A.n, A.rowptr, A.col, A.val, x, y)
    PC_LPR_DISPATCH(A.lpr, CALL)
#undef CALL
    count_launches(1);
    PC_LAUNCH("spmv64");
}

template <class T>
void gs_colour(cudaStream_t s, const Csr& A, const int32_t* rows, int32_t nrows, const T* b, T* x) {
    if (nrows <= 0) return;
    int g = sparse_grid(nrows, A.lpr);
    const T* val;
    if constexpr (sizeof(T) == 8) val = A.val; else val = A.val32;
#define CALL(L) launch(k_gs<T, L>, g, kBlock, 0, s, nrows, rows, A.rowptr, A.col, val, b, x)
    PC_LPR_DISPATCH(A.lpr, CALL)
#undef CALL
    PC_LAUNCH("gs_colour");
}

template <class T>
void gs_colour_perm(cudaStream_t s, int32_t beg, int32_t end, const int32_t* rows, const int32_t* pptr,
                    const int32_t* pcol, const T* pval, const T* b, T* x) {
    if (end <= beg) return;
    int g = ((end - beg + kStreamRows - 1) / kStreamRows + kGsTiles - 1) / kGsTiles;
    if (rows) launch(k_gs_stream<T, false>, g, kStreamRows, 0, s, beg, end, rows, pptr, pcol, pval, b, x);
    else launch(k_gs_stream<T, true>, g, kStreamRows, 0, s, beg, end, rows, pptr, pcol, pval, b, x);
    PC_LAUNCH("gs_colour_perm");
}

template <class T>
void permute_rows(Ctx& c, int32_t n, const int32_t* rows, const int32_t* rowptr, const int32_t* col,
                  const double* val, DBuf<int32_t>& pptr, DBuf<int32_t>& pcol, DBuf<T>& pval) {
    cudaStream_t s = c.stream;
    int64_t nnz = 0;
    DBuf<int32_t> cnt;
    cnt.alloc(c.mem, n);
    k_perm_counts<<<simple_grid(n), kBlock, 0, s>>>(n, rows, rowptr, cnt.p); ::pc::count_launches(1);
    pptr.alloc(c.mem, (size_t)n + 1);
    nnz = scan_i32(c, cnt.p, pptr.p, n);
    pcol.alloc(c.mem, nnz);
    pval.alloc(c.mem, nnz);
    k_perm_fill<T><<<simple_grid(n), kBlock, 0, s>>>(n, rows, rowptr, col, val, pptr.p, pcol.p, pval.p); ::pc::count_launches(1);
    PC_LAUNCH("permute_rows");
}

void mark_diagonal(cudaStream_t s, int32_t n, const int32_t* ptr, int32_t* col) {
    k_mark_diag<<<simple_grid(n), kBlock, 0, s>>>(n, ptr, col); ::pc::count_launches(1);
    PC_LAUNCH("mark_diagonal");
}

template <class T>
void restrict_agg(cudaStream_t s, int32_t nc, const int32_t* agg_ptr, const int32_t* agg_mem,
                  const T* pval, const T* r, T* bc, T* xc, const T* dc) {
    launch(k_restrict<T>, simple_grid(nc), kBlock, 0, s, nc, agg_ptr, agg_mem, pval, r, bc, xc, dc);
    PC_LAUNCH("restrict");
}

template <class T>
void prolong_add(cudaStream_t s, int32_t n, const int32_t* agg, const T* pval, const T* xc, T* x) {
    launch(k_prolong<T>, simple_grid(n), kBlock, 0, s, n, agg, pval, xc, x);
    PC_LAUNCH("prolong");
}

template <class T>
void coarse_apply(cudaStream_t s, int32_t m, const double* Xinv, const T* b, T* x) {
    int g = (m * 32 + kBlock - 1) / kBlock;
    if (g > kNumSMs * 4) g = kNumSMs * 4;
    k_coarse_apply<T><<<g, kBlock, 0, s>>>(m, Xinv, b, x); ::pc::count_launches(1);
    PC_LAUNCH("coarse_apply");
}

template void gs_colour<double>(cudaStream_t, const Csr&, const int32_t*, int32_t, const double*, double*);
template void gs_colour_perm<double>(cudaStream_t, int32_t, int32_t, const int32_t*, const int32_t*, const int32_t*, const double*, const double*, double*);
template void gs_colour_perm<float>(cudaStream_t, int32_t, int32_t, const int32_t*, const int32_t*, const int32_t*, const float*, const float*, float*);
template void permute_rows<double>(Ctx&, int32_t, const int32_t*, const int32_t*, const int32_t*, const double*, DBuf<int32_t>&, DBuf<int32_t>&, DBuf<double>&);
template void permute_rows<float>(Ctx&, int32_t, const int32_t*, const int32_t*, const int32_t*, const double*, DBuf<int32_t>&, DBuf<int32_t>&, DBuf<float>&);
template void gs_colour<float>(cudaStream_t, const Csr&, const int32_t*, int32_t, const float*, float*);
template void restrict_agg<double>(cudaStream_t, int32_t, const int32_t*, const int32_t*, const double*, const double*, double*, double*, const double*);
template void restrict_agg<float>(cudaStream_t, int32_t, const int32_t*, const int32_t*, const float*, const float*, float*, float*, const float*);
template void prolong_add<double>(cudaStream_t, int32_t, const int32_t*, const double*, const double*, double*);
template void prolong_add<float>(cudaStream_t, int32_t, const int32_t*, const float*, const float*, float*);
template void coarse_apply<double>(cudaStream_t, int32_t, const double*, const double*, double*);
template void coarse_apply<float>(cudaStream_t, int32_t, const double*, const float*, float*);

}  // namespace pc
