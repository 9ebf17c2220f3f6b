// Coarse tail of the multigrid cycle in one thread block.
//
// Below a few thousand unknowns a level's work is far smaller than the cost of
// launching its kernels, and a W-cycle visits level l 2^l times. All levels
// from `l0` down to the coarsest therefore run inside one 1024-thread block:
// the same steps as the per-level kernels (colour-ordered Gauss-Seidel, the
// residual, restriction by P^T, the gamma child visits, prolongation by P, the
// backward sweep, and the dense coarsest solve), with __syncthreads() between
// dependent steps. The recursion is an explicit state machine that every
// thread follows identically. Vectors written inside the kernel are read with
// ordinary (coherent) loads; only the read-only level data use __ldg. Small
// coarse levels are smoothed by l1-Jacobi (two block-wide phases per sweep),
// others by colour-ordered Gauss-Seidel (one phase per colour).
#include "pcamg_internal.cuh"

namespace pc {

namespace {

constexpr int kTailThreads = 1024;
constexpr int kTailWarps = kTailThreads / 32;

template <class T>
__device__ __forceinline__ T gsum(T v, int lpr) {
    for (int o = lpr >> 1; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o, lpr);
    return v;
}

template <class T>
__device__ void tail_gs(const TailLevel<T>& L, int k) {
    const int beg = __ldg(L.cptr + k), end = __ldg(L.cptr + k + 1);
    const int lpr = L.lpr, rpw = 32 / lpr;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, sub = lane % lpr, grp = lane / lpr;
    T* x = L.x;
    const T* b = L.b;
    for (int t0 = beg + warp * rpw; t0 < end; t0 += kTailWarps * rpw) {
        int t = t0 + grp, row = -1;
        T s = 0, d = 0;
        if (t < end) {
            row = __ldg(L.crows + t);
            int e = __ldg(L.rowptr + row + 1);
            for (int q = __ldg(L.rowptr + row) + sub; q < e; q += lpr) {
                int j = __ldg(L.col + q);
                T a = __ldg(L.val + q);
                if (j == row) d = a;
                else s += a * x[j];
            }
        }
        s = gsum(s, lpr);
        d = gsum(d, lpr);
        if (sub == 0 && t < end) x[row] = (b[row] - s) / d;
    }
    __syncthreads();
}

// r = b - A x, rows in tiles of one per thread; the tile's products a x are
// staged in shared memory in chunks (each thread first loads kTailUnroll
// column indices and values, so many loads are in flight), then each thread
// adds its row's products in CSR order. When the level is small enough, x is
// first copied to shared memory so the products need no gathers from L2.
constexpr int kTailChunk = 4096;
constexpr int kTailUnroll = kTailChunk / kTailThreads;
constexpr int kTailXs = 2048;

template <class T>
__device__ void tail_residual(const TailLevel<T>& L, T* prod, T* xs) {
    const T* xg = L.x;
    const T* b = L.b;
    T* r = L.r;
    const bool staged = L.n <= kTailXs;
    if (staged) {
        for (int i = threadIdx.x; i < L.n; i += kTailThreads) xs[i] = xg[i];
        __syncthreads();
    }
    const T* x = staged ? xs : xg;
    for (int r0 = 0; r0 < L.n; r0 += kTailThreads) {
        const int row = r0 + threadIdx.x;
        const int rlast = min(r0 + kTailThreads, L.n);
        const int tb = __ldg(L.rowptr + r0), te = __ldg(L.rowptr + rlast);
        int rb = 0, re = 0;
        if (row < L.n) { rb = __ldg(L.rowptr + row); re = __ldg(L.rowptr + row + 1); }
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
                if (k < c1) prod[k - c0] = cv[u] * x[cj[u]];
            }
            __syncthreads();
            const int kb = max(rb, c0), ke = min(re, c1);
            for (int k = kb; k < ke; ++k) s += prod[k - c0];
            __syncthreads();
        }
        if (row < L.n) r[row] = b[row] - s;
    }
    __syncthreads();
}

// l1-Jacobi sweep: x += (b - A x) / d
template <class T>
__device__ void tail_jacobi(const TailLevel<T>& L, T* prod, T* xs) {
    tail_residual(L, prod, xs);
    T* x = L.x;
    const T* r = L.r;
    for (int i = threadIdx.x; i < L.n; i += kTailThreads) x[i] += r[i] / __ldg(L.dl1 + i);
    __syncthreads();
}

template <class T>
__device__ void tail_restrict_zero(const TailLevel<T>& L, const TailLevel<T>& C) {
    T* bc = C.b;
    T* xc = C.x;
    const T* r = L.r;
    for (int I = threadIdx.x; I < L.nc; I += kTailThreads) {
        T s = 0;
        int e = __ldg(L.agg_ptr + I + 1);
        for (int t = __ldg(L.agg_ptr + I); t < e; ++t) {
            int u = __ldg(L.agg_mem + t);
            s += L.pval ? __ldg(L.pval + u) * r[u] : r[u];
        }
        bc[I] = s;
        xc[I] = 0;
    }
    __syncthreads();
}

template <class T>
__device__ void tail_prolong(const TailLevel<T>& L, const TailLevel<T>& C) {
    T* x = L.x;
    const T* xc = C.x;
    for (int u = threadIdx.x; u < L.n; u += kTailThreads) {
        T c = xc[__ldg(L.agg + u)];
        x[u] += L.pval ? __ldg(L.pval + u) * c : c;
    }
    __syncthreads();
}

template <class T>
__device__ void tail_coarse(const TailLevel<T>& L, const double* __restrict__ X) {
    const int m = L.n, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T* b = L.b;
    T* x = L.x;
    for (int i = warp; i < m; i += kTailWarps) {
        double s = 0.0;
        for (int j = lane; j < m; j += 32) s += __ldg(X + (size_t)i * m + j) * (double)b[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) x[i] = (T)s;
    }
    __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(kTailThreads) k_tail(const TailLevel<T>* __restrict__ lv, int l0, int L,
                                                       int gamma, int nu_pre, int nu_post,
                                                       const double* __restrict__ Xinv) {
    __shared__ __align__(16) unsigned char smem[(kTailChunk + kTailXs) * sizeof(T)];
    T* prod = reinterpret_cast<T*>(smem);
    T* xs = prod + kTailChunk;
    int cnt[kMaxLevels];
    int l = l0;
    bool down = true;
    for (;;) {
        if (down) {
            if (l == L - 1) {
                tail_coarse(lv[l], Xinv);
                down = false;
                if (--l < l0) break;
                continue;
            }
            const TailLevel<T>& V = lv[l];
            for (int s = 0; s < nu_pre; ++s) {
                if (V.jac) tail_jacobi(V, prod, xs);
                else for (int k = 0; k < V.ncolour; ++k) tail_gs(V, k);
            }
            tail_residual(V, prod, xs);
            tail_restrict_zero(V, lv[l + 1]);
            cnt[l] = gamma;
            ++l;
        } else {
            if (--cnt[l] > 0) { ++l; down = true; continue; }
            const TailLevel<T>& V = lv[l];
            tail_prolong(V, lv[l + 1]);
            for (int s = 0; s < nu_post; ++s) {
                if (V.jac) tail_jacobi(V, prod, xs);
                else for (int k = V.ncolour - 1; k >= 0; --k) tail_gs(V, k);
            }
            if (l == l0) break;
            --l;
        }
    }
}

}  // namespace

template <class T>
void tail_cycle(cudaStream_t s, const TailLevel<T>* lv, int l0, int L, int gamma, int nu_pre,
                int nu_post, const double* Xinv) {
    k_tail<T><<<1, kTailThreads, 0, s>>>(lv, l0, L, gamma, nu_pre, nu_post, Xinv); ::pc::count_launches(1);
    PC_LAUNCH("tail_cycle");
}

template void tail_cycle<double>(cudaStream_t, const TailLevel<double>*, int, int, int, int, int, const double*);
template void tail_cycle<float>(cudaStream_t, const TailLevel<float>*, int, int, int, int, int, const double*);

}  // namespace pc
