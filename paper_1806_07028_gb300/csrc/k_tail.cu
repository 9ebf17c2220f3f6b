// Coarse tail of the multigrid cycle in one thread-block cluster.
//
// Below a few thousand unknowns a level's work is far smaller than the cost of
// launching its kernels, and a W-cycle visits level l 2^l times. All levels
// from `l0` down to the coarsest therefore run inside one launch of CL thread
// blocks forming a cluster (CL = 8, one block per SM; CL = 1 is the same code
// on a single block): the same steps as the per-level kernels (smoothing, the
// residual, restriction by P^T, the gamma child visits, prolongation by P,
// smoothing, and the dense coarsest solve). Every step splits its rows over
// the blocks; dependent steps are separated by a cluster barrier (release /
// acquire at cluster scope). The recursion is an explicit state machine that
// every thread of every block follows identically, so all barriers are met.
// Vectors written inside the kernel are read with ld.global.cg (from L2,
// coherent across the cluster's SMs); read-only level data use __ldg.
// Small coarse levels are smoothed by l1-Jacobi (two steps per sweep), others
// by colour-ordered Gauss-Seidel (one step per colour).
#include <cooperative_groups.h>

#include "pcamg_internal.cuh"

namespace cg = cooperative_groups;

namespace pc {

namespace {

constexpr int kTailThreads = 1024;
constexpr int kTailWarps = kTailThreads / 32;
constexpr int kTailChunk = 4096;
constexpr int kTailUnroll = kTailChunk / kTailThreads;
constexpr int kTailXs = 2048;
constexpr int kCluster = 8;

template <int CL>
__device__ __forceinline__ void step_sync() {
    if constexpr (CL == 1) __syncthreads();
    else cg::this_cluster().sync();
}

template <int CL>
__device__ __forceinline__ int rank() {
    if constexpr (CL == 1) return 0;
    else return (int)cg::this_cluster().block_rank();
}

// this block's share [lo, hi) of n items
template <int CL>
__device__ __forceinline__ void share(int n, int& lo, int& hi) {
    const int q = rank<CL>();
    lo = (int)(((int64_t)n * q) / CL);
    hi = (int)(((int64_t)n * (q + 1)) / CL);
}

// vectors written inside the kernel: read from L2 when the cluster's blocks
// share them, plainly when they live in this block's shared memory (LOC)
template <bool LOC, class T>
__device__ __forceinline__ T ldv(const T* p) {
    if constexpr (LOC) return *p;
    else return __ldcg(p);
}

__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }

template <class T>
__device__ __forceinline__ T gsum(T v, int lpr) {
    for (int o = lpr >> 1; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o, lpr);
    return v;
}

template <class T, int CL, bool LOC>
__device__ void tail_gs(const TailLevel<T>& L, int k) {
    const int beg = __ldg(L.cptr + k), end = __ldg(L.cptr + k + 1);
    int lo, hi;
    share<CL>(end - beg, lo, hi);
    lo += beg;
    hi += beg;
    const int lpr = L.lpr, rpw = 32 / lpr;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, sub = lane % lpr, grp = lane / lpr;
    T* x = L.x;
    for (int t0 = lo + warp * rpw; t0 < hi; t0 += kTailWarps * rpw) {
        int t = t0 + grp, row = -1;
        T s = 0, d = 0;
        if (t < hi) {
            row = __ldg(L.crows + t);
            int e = __ldg(L.rowptr + row + 1);
            for (int q = __ldg(L.rowptr + row) + sub; q < e; q += lpr) {
                int j = __ldg(L.col + q);
                T a = __ldg(L.val + q);
                if (j == row) d = a;
                else s = fma_t(a, ldv<LOC>(x + j), s);
            }
        }
        s = gsum(s, lpr);
        d = gsum(d, lpr);
        if (sub == 0 && t < hi) x[row] = (ldv<LOC>(L.b + row) - s) / d;
    }
    step_sync<CL>();
}

// r = b - A x for this block's rows: rows in tiles of one per thread; the
// tile's products a x are staged in shared memory in chunks (each thread first
// loads kTailUnroll column indices and values, so many loads are in flight),
// then each thread adds its row's products in CSR order. A small level's x is
// first copied to shared memory so the products need no gathers from L2.
template <class T, int CL, bool LOC>
__device__ void tail_residual(const TailLevel<T>& L, T* prod, T* xs) {
    const T* xg = L.x;
    T* r = L.r;
    const bool staged = !LOC && L.n <= kTailXs;
    if (staged) {
        for (int i = threadIdx.x; i < L.n; i += kTailThreads) xs[i] = ldv<LOC>(xg + i);
        __syncthreads();
    }
    int lo, hi;
    share<CL>(L.n, lo, hi);
    for (int r0 = lo; r0 < hi; r0 += kTailThreads) {
        const int row = r0 + threadIdx.x;
        const int rlast = min(r0 + kTailThreads, hi);
        const int tb = __ldg(L.rowptr + r0), te = __ldg(L.rowptr + rlast);
        int rb = 0, re = 0;
        if (row < hi) { rb = __ldg(L.rowptr + row); re = __ldg(L.rowptr + row + 1); }
        T s = 0;
        for (int c0 = tb; c0 < te; c0 += kTailChunk) {
            const int c1 = min(c0 + kTailChunk, te);
            int cj[kTailUnroll];
            T cv[kTailUnroll];
#pragma unroll
            for (int u = 0; u < kTailUnroll; ++u) {
                const int k = c0 + threadIdx.x + u * kTailThreads;
                cj[u] = (k < c1) ? __ldg(L.col + k) : 0;
                cv[u] = (k < c1) ? __ldg(L.val + k) : T(0);
            }
#pragma unroll
            for (int u = 0; u < kTailUnroll; ++u) {
                const int k = c0 + threadIdx.x + u * kTailThreads;
                if (k < c1) prod[k - c0] = cv[u] * (staged ? xs[cj[u]] : ldv<LOC>(xg + cj[u]));
            }
            __syncthreads();
            const int kb = max(rb, c0), ke = min(re, c1);
            for (int k = kb; k < ke; ++k) s += prod[k - c0];
            __syncthreads();
        }
        if (row < hi) r[row] = ldv<LOC>(L.b + row) - s;
    }
    step_sync<CL>();
}

// l1-Jacobi sweep: x += (b - A x) / d
template <class T, int CL, bool LOC>
__device__ void tail_jacobi(const TailLevel<T>& L, T* prod, T* xs) {
    tail_residual<T, CL, LOC>(L, prod, xs);
    int lo, hi;
    share<CL>(L.n, lo, hi);
    T* x = L.x;
    for (int i = lo + threadIdx.x; i < hi; i += kTailThreads) x[i] = ldv<LOC>(x + i) + ldv<LOC>(L.r + i) / __ldg(L.dl1 + i);
    step_sync<CL>();
}

// Restriction of the residual and the child's start value: zero, or b/d when
// the child begins with an l1-Jacobi sweep from zero.
template <class T, int CL, bool LOC>
__device__ void tail_restrict(const TailLevel<T>& L, const TailLevel<T>& C, bool child_fresh) {
    int lo, hi;
    share<CL>(L.nc, lo, hi);
    T* bc = C.b;
    T* xc = C.x;
    for (int I = lo + threadIdx.x; I < hi; I += kTailThreads) {
        T s = 0;
        int e = __ldg(L.agg_ptr + I + 1);
        for (int t = __ldg(L.agg_ptr + I); t < e; ++t) {
            int u = __ldg(L.agg_mem + t);
            s += L.pval ? __ldg(L.pval + u) * ldv<LOC>(L.r + u) : ldv<LOC>(L.r + u);
        }
        bc[I] = s;
        xc[I] = child_fresh ? s / __ldg(C.dl1 + I) : T(0);
    }
    step_sync<CL>();
}

template <class T, int CL, bool LOC>
__device__ void tail_prolong(const TailLevel<T>& L, const TailLevel<T>& C) {
    int lo, hi;
    share<CL>(L.n, lo, hi);
    T* x = L.x;
    for (int u = lo + threadIdx.x; u < hi; u += kTailThreads) {
        T c = ldv<LOC>(C.x + __ldg(L.agg + u));
        x[u] = ldv<LOC>(x + u) + (L.pval ? __ldg(L.pval + u) * c : c);
    }
    step_sync<CL>();
}

template <class T, int CL, bool LOC>
__device__ void tail_coarse(const TailLevel<T>& L, const double* __restrict__ X) {
    const int m = L.n, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int lo, hi;
    share<CL>(m, lo, hi);
    T* x = L.x;
    for (int i = lo + warp; i < hi; i += kTailWarps) {
        double s = 0.0;
        for (int j = lane; j < m; j += 32) s += __ldg(X + (size_t)i * m + j) * (double)ldv<LOC>(L.b + j);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) x[i] = (T)s;
    }
    step_sync<CL>();
}

template <class T, int CL, bool LOC>
__device__ void tail_body(const TailLevel<T>* __restrict__ lv, int l0, int L, int gamma, int nu_pre,
                          int nu_post, const double* __restrict__ Xinv, int fresh0) {
    __shared__ __align__(16) unsigned char smem[(kTailChunk + kTailXs) * sizeof(T)];
    T* prod = reinterpret_cast<T*>(smem);
    T* xs = prod + kTailChunk;
    int cnt[kMaxLevels];
    int l = l0;
    bool down = true;
    bool fresh = fresh0 != 0;   // x of level l arrives as one Jacobi sweep from zero
    for (;;) {
        if (down) {
            if (l == L - 1) {
                tail_coarse<T, CL, LOC>(lv[l], Xinv);
                down = false;
                if (--l < l0) break;
                continue;
            }
            const TailLevel<T>& V = lv[l];
            for (int s = fresh ? 1 : 0; s < nu_pre; ++s) {
                if (V.jac) tail_jacobi<T, CL, LOC>(V, prod, xs);
                else for (int k = 0; k < V.ncolour; ++k) tail_gs<T, CL, LOC>(V, k);
            }
            const bool cf = lv[l + 1].jac && nu_pre >= 1 && l + 1 < L - 1;
            tail_residual<T, CL, LOC>(V, prod, xs);
            tail_restrict<T, CL, LOC>(V, lv[l + 1], cf);
            cnt[l] = gamma;
            ++l;
            fresh = cf;
        } else {
            if (--cnt[l] > 0) { ++l; down = true; fresh = false; continue; }
            const TailLevel<T>& V = lv[l];
            tail_prolong<T, CL, LOC>(V, lv[l + 1]);
            for (int s = 0; s < nu_post; ++s) {
                if (V.jac) tail_jacobi<T, CL, LOC>(V, prod, xs);
                else for (int k = V.ncolour - 1; k >= 0; --k) tail_gs<T, CL, LOC>(V, k);
            }
            if (l == l0) break;
            --l;
        }
    }
}

template <class T>
__global__ void __cluster_dims__(kCluster, 1, 1) __launch_bounds__(kTailThreads)
    k_tail_cluster(const TailLevel<T>* __restrict__ lv, int l0, int L, int gamma, int nu_pre,
                   int nu_post, const double* __restrict__ Xinv, int fresh) {
    tail_body<T, kCluster, false>(lv, l0, L, gamma, nu_pre, nu_post, Xinv, fresh);
}

// Columns of the tail's linear operator. One visit of the tail levels from a
// zero start is a linear map b -> x of the first tail level (every step --
// l1-Jacobi or Gauss-Seidel sweeps, restriction, the gamma child visits,
// prolongation, the pinned pseudo-inverse -- is linear), so column j of its
// matrix N is the visit applied to the unit vector e_j. Each block takes
// columns j = blockIdx.x, blockIdx.x + gridDim.x, ... and runs the same state
// machine as the cluster kernel on one block, with every level's x, b and r in
// its shared memory; N is stored row-major with row stride ld. With visits > 1
// the column is that many consecutive visits, each continuing from the last
// one's x (a W-cycle's parent visits its child twice with the same b: the two
// visits are one linear map, applied by one product instead of two).
template <class T>
__global__ void __launch_bounds__(kTailThreads, 1)
    k_tail_columns(const TailLevel<T>* __restrict__ lvg, int l0, int L, int gamma, int nu_pre,
                   int nu_post, const double* __restrict__ Xinv, T* __restrict__ Nout, int ld, int visits) {
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ TailLevel<T> lvs[kMaxLevels];
    if (threadIdx.x == 0) {
        T* p = reinterpret_cast<T*>(dyn);
        for (int l = l0; l < L; ++l) {
            lvs[l] = lvg[l];
            const int n = lvs[l].n;
            lvs[l].x = p; p += n;
            lvs[l].b = p; p += n;
            lvs[l].r = p; p += n;
        }
    }
    __syncthreads();
    const int m = lvs[l0].n;
    T* x = lvs[l0].x;
    T* b = lvs[l0].b;
    for (int j = blockIdx.x; j < m; j += gridDim.x) {
        for (int i = threadIdx.x; i < m; i += kTailThreads) {
            b[i] = (i == j) ? T(1) : T(0);
            x[i] = T(0);
        }
        __syncthreads();
        for (int v = 0; v < visits; ++v) tail_body<T, 1, true>(lvs, l0, L, gamma, nu_pre, nu_post, Xinv, 0);
        for (int i = threadIdx.x; i < m; i += kTailThreads) Nout[(size_t)i * ld + j] = x[i];
        __syncthreads();
    }
}

constexpr int kGemvWarpsMax = 32;   // warps (rows) per block at most

template <class T> struct Vec16;
template <> struct Vec16<float> { using V = float4; };
template <> struct Vec16<double> { using V = double2; };

__device__ __forceinline__ float dot16(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
__device__ __forceinline__ double dot16(double2 a, double2 b) { return a.x * b.x + a.y * b.y; }

// x = N v (accum = 0) or x += N v (accum = 1); one warp per row of N, v staged
// in shared memory with zeros up to ld, rows read as 16-byte vectors. N is
// hierarchy data: a lane's first kGemvPre vectors of its row are loaded ahead
// of pdl_wait(), so in a cycle graph they arrive while the previous kernel
// runs; the rest follow kGemvUnroll at a time, all independent.
constexpr int kGemvPre = 8;
constexpr int kGemvUnroll = 8;

template <class T>
__global__ void __launch_bounds__(kGemvWarpsMax * 32)
    k_tail_gemv(int m, int ld, const T* __restrict__ Nm, const T* __restrict__ v, T* __restrict__ x,
                int accum) {
    using V = typename Vec16<T>::V;
    constexpr int W = 16 / sizeof(T);
    extern __shared__ __align__(16) unsigned char dyn[];
    T* vs = reinterpret_cast<T*>(dyn);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * (int)(blockDim.x >> 5) + warp;
    const int nq = ld / W;
    const V* a = reinterpret_cast<const V*>(Nm + (size_t)(row < m ? row : 0) * ld);
    V pre[kGemvPre];
#pragma unroll
    for (int u = 0; u < kGemvPre; ++u) {
        const int q = lane + 32 * u;
        pre[u] = (row < m && q < nq) ? __ldg(a + q) : V{};
    }
    pdl_wait();
    pdl_trigger();
    for (int j = threadIdx.x; j < ld; j += blockDim.x) vs[j] = (j < m) ? v[j] : T(0);
    __syncthreads();
    if (row >= m) return;
    const V* vv = reinterpret_cast<const V*>(vs);
    T s = 0;
#pragma unroll
    for (int u = 0; u < kGemvPre; ++u) {
        const int q = lane + 32 * u;
        if (q < nq) s += dot16(pre[u], vv[q]);
    }
    for (int q0 = lane + 32 * kGemvPre; q0 < nq; q0 += 32 * kGemvUnroll) {
        V t[kGemvUnroll];
#pragma unroll
        for (int u = 0; u < kGemvUnroll; ++u) {
            const int q = q0 + 32 * u;
            t[u] = q < nq ? __ldg(a + q) : V{};
        }
#pragma unroll
        for (int u = 0; u < kGemvUnroll; ++u) {
            const int q = q0 + 32 * u;
            if (q < nq) s += dot16(t[u], vv[q]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) x[row] = accum ? x[row] + s : s;
}

}  // namespace

// dynamic shared memory of k_tail_columns: x, b, r of every tail level
template <class T>
size_t tail_operator_smem(const int* n, int l0, int L) {
    size_t e = 0;
    for (int l = l0; l < L; ++l) e += 3 * (size_t)n[l];
    return e * sizeof(T);
}

template <class T>
bool tail_operator_fits(const int* n, int l0, int L) {
    const size_t stat = (kTailChunk + kTailXs) * sizeof(T) + sizeof(TailLevel<T>) * kMaxLevels;
    return tail_operator_smem<T>(n, l0, L) + stat <= 220 * 1024;
}

template <class T>
void tail_operator(cudaStream_t s, const TailLevel<T>* lv, const int* n, int l0, int L, int gamma,
                   int nu_pre, int nu_post, const double* Xinv, T* Nout, int ld, int nsm, int visits) {
    const size_t dyn = tail_operator_smem<T>(n, l0, L);
    if (!tail_operator_fits<T>(n, l0, L)) fail(PCAMG_ERR_INVALID, "tail operator: levels exceed shared memory");
    PC_CUDA(cudaFuncSetAttribute(k_tail_columns<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    const int m = n[l0];
    const int grid = std::max(1, std::min(m, nsm));
    k_tail_columns<T><<<grid, kTailThreads, dyn, s>>>(lv, l0, L, gamma, nu_pre, nu_post, Xinv, Nout, ld, visits); ::pc::count_launches(1);
    PC_LAUNCH("tail_operator");
}

template <class T>
void tail_gemv(cudaStream_t s, int m, int ld, const T* Nm, const T* v, T* x, bool accum) {
    // rows spread evenly over the SMs: one block per SM with ceil(m / SMs)
    // warps (a warp per row), so no SM takes a second block
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        PC_CUDA(cudaGetDevice(&dev));
        PC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    }
    const int warps = std::max(1, std::min(kGemvWarpsMax, (m + nsm - 1) / nsm));
    const int grid = (m + warps - 1) / warps;
    launch(k_tail_gemv<T>, grid, warps * 32, sizeof(T) * ld, s, m, ld, Nm, v, x, accum ? 1 : 0);
    PC_LAUNCH("tail_gemv");
}

template size_t tail_operator_smem<float>(const int*, int, int);
template size_t tail_operator_smem<double>(const int*, int, int);
template bool tail_operator_fits<float>(const int*, int, int);
template bool tail_operator_fits<double>(const int*, int, int);
template void tail_operator<float>(cudaStream_t, const TailLevel<float>*, const int*, int, int, int, int, int, const double*, float*, int, int, int);
template void tail_operator<double>(cudaStream_t, const TailLevel<double>*, const int*, int, int, int, int, int, const double*, double*, int, int, int);
template void tail_gemv<float>(cudaStream_t, int, int, const float*, const float*, float*, bool);
template void tail_gemv<double>(cudaStream_t, int, int, const double*, const double*, double*, bool);

template <class T>
void tail_cycle(cudaStream_t s, const TailLevel<T>* lv, int l0, int L, int gamma, int nu_pre,
                int nu_post, const double* Xinv, int fresh) {
    k_tail_cluster<T><<<kCluster, kTailThreads, 0, s>>>(lv, l0, L, gamma, nu_pre, nu_post, Xinv, fresh); ::pc::count_launches(1);
    PC_LAUNCH("tail_cycle");
}

template void tail_cycle<double>(cudaStream_t, const TailLevel<double>*, int, int, int, int, int, const double*, int);
template void tail_cycle<float>(cudaStream_t, const TailLevel<float>*, int, int, int, int, int, const double*, int);

}  // namespace pc
