// Batched kernels of the multi-right-hand-side solve: one pass over a level's
// matrix serves K vectors. A level's K vectors are stored row-interleaved
// (v[i * K + c]), so a gathered neighbour brings its K values from one
// contiguous run. The steps are those of the single-vector cycle (smoothing,
// residual, restriction, prolongation, the coarse tail as its dense operator,
// the coarsest pseudo-inverse); the row sums use the sub-warp order (LPR lanes
// per row, a shuffle tree), so a column agrees with the single-vector cycle
// to rounding, not bit for bit.
#include "pcamg_internal.cuh"

namespace pc {

namespace {

__device__ __forceinline__ double mfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// sum over the lpr lanes of a row group (lpr a power of two, <= 32)
template <class T>
__device__ __forceinline__ T group_sum_rt(T v, int lpr) {
    for (int o = lpr >> 1; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o, lpr);
    return v;
}

// a row's K values as wide loads and stores (row i starts at i * K, so a row
// of 2, 4 or 8 floats, or 2, 4 or 8 doubles, is 8- or 16-byte aligned)
template <class T, int K>
__device__ __forceinline__ void ldk(const T* p, T (&v)[K]) {
    if constexpr (sizeof(T) == 4 && K % 4 == 0) {
#pragma unroll
        for (int q = 0; q < K / 4; ++q) {
            const float4 w = reinterpret_cast<const float4*>(p)[q];
            v[4 * q] = w.x; v[4 * q + 1] = w.y; v[4 * q + 2] = w.z; v[4 * q + 3] = w.w;
        }
    } else if constexpr (sizeof(T) == 4 && K == 2) {
        const float2 w = *reinterpret_cast<const float2*>(p);
        v[0] = w.x; v[1] = w.y;
    } else if constexpr (sizeof(T) == 8 && K % 2 == 0) {
#pragma unroll
        for (int q = 0; q < K / 2; ++q) {
            const double2 w = reinterpret_cast<const double2*>(p)[q];
            v[2 * q] = w.x; v[2 * q + 1] = w.y;
        }
    } else {
#pragma unroll
        for (int c = 0; c < K; ++c) v[c] = p[c];
    }
}

template <class T, int K>
__device__ __forceinline__ void stk(T* p, const T (&v)[K]) {
    if constexpr (sizeof(T) == 4 && K % 4 == 0) {
#pragma unroll
        for (int q = 0; q < K / 4; ++q)
            reinterpret_cast<float4*>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else if constexpr (sizeof(T) == 4 && K == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    } else if constexpr (sizeof(T) == 8 && K % 2 == 0) {
#pragma unroll
        for (int q = 0; q < K / 2; ++q) reinterpret_cast<double2*>(p)[q] = make_double2(v[2 * q], v[2 * q + 1]);
    } else {
#pragma unroll
        for (int c = 0; c < K; ++c) p[c] = v[c];
    }
}

enum { MV_RES = 0, MV_JAC = 1, MV_GS = 2 };

// Rows t of [0, nrows): row = rows ? rows[t] : beg + t. A row's entries are
// split over lpr lanes (entry k to lane k mod lpr), each lane keeps K sums.
//   MV_RES: out_row = b_row - sum_j a_rj x_j
//   MV_JAC: out_row = x_row + (b_row - sum_j a_rj x_j) / d_row   (out != x)
//   MV_GS:  x_row = (b_row - sum_{j != row} a_rj x_j) / a_row,row (out == x;
//           the rows of one colour)
// A marked diagonal (column ~row) is decoded; in MV_GS the diagonal entry
// (marked, or column == row) gives a_row,row and no product.
template <class T, int K, int MODE>
__global__ void __launch_bounds__(256) k_mv_rows(int nrows, const int* __restrict__ rows, int beg, int lpr,
                                                 const int* __restrict__ rowptr, const int* __restrict__ col,
                                                 const T* __restrict__ val, const T* x, const T* __restrict__ b,
                                                 const T* __restrict__ d, T* out) {
    const int lane = threadIdx.x & 31;
    const int sub = lane & (lpr - 1), grp = lane / lpr, rpw = 32 / lpr;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t0 = warp * rpw; t0 < nrows; t0 += nwarps * rpw) {
        const int64_t t = t0 + grp;
        T s[K];
#pragma unroll
        for (int c = 0; c < K; ++c) s[c] = T(0);
        T dg = T(0);
        int row = -1;
        if (t < nrows) {
            row = rows ? __ldg(rows + t) : beg + (int)t;
            const int e = __ldg(rowptr + row + 1);
            for (int k = __ldg(rowptr + row) + sub; k < e; k += lpr) {
                int j = __ldg(col + k);
                const T a = __ldg(val + k);
                if (MODE == MV_GS && (j < 0 || j == row)) {
                    dg = a;
                    continue;
                }
                if (j < 0) j = ~j;
                T xj[K];
                ldk<T, K>(x + (size_t)j * K, xj);
#pragma unroll
                for (int c = 0; c < K; ++c) s[c] = mfma(a, xj[c], s[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < K; ++c) s[c] = group_sum_rt(s[c], lpr);
        if (MODE == MV_GS) dg = group_sum_rt(dg, lpr);
        if (t < nrows && sub == 0) {
            const size_t o = (size_t)row * K;
            T bv[K], ov[K];
            ldk<T, K>(b + o, bv);
            if (MODE == MV_RES) {
#pragma unroll
                for (int c = 0; c < K; ++c) ov[c] = bv[c] - s[c];
            } else if (MODE == MV_JAC) {
                const T dr = __ldg(d + row);
                T xv[K];
                ldk<T, K>(x + o, xv);
#pragma unroll
                for (int c = 0; c < K; ++c) ov[c] = xv[c] + (bv[c] - s[c]) / dr;
            } else {
#pragma unroll
                for (int c = 0; c < K; ++c) ov[c] = (bv[c] - s[c]) / dg;
            }
            stk<T, K>(out + o, ov);
        }
    }
}

// bc_I = sum over members u of aggregate I (in order) of p_u r_u, K vectors;
// the child's start: zero, or bc_I / dc_I (an l1-Jacobi sweep from zero)
template <class T, int K>
__global__ void k_mv_restrict(int nc, const int* __restrict__ agg_ptr, const int* __restrict__ mem,
                              const T* __restrict__ pval, const T* __restrict__ r, T* __restrict__ bc,
                              T* __restrict__ xc, const T* __restrict__ dc) {
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
        T s[K];
#pragma unroll
        for (int c = 0; c < K; ++c) s[c] = T(0);
        const int e = __ldg(agg_ptr + I + 1);
        for (int t = __ldg(agg_ptr + I); t < e; ++t) {
            const int u = __ldg(mem + t);
            const T p = pval ? __ldg(pval + u) : T(1);
            T ru[K];
            ldk<T, K>(r + (size_t)u * K, ru);
#pragma unroll
            for (int c = 0; c < K; ++c) s[c] += pval ? p * ru[c] : ru[c];
        }
        const T dI = dc ? __ldg(dc + I) : T(1);
        stk<T, K>(bc + (size_t)I * K, s);
        if (xc) {
            T xv[K];
#pragma unroll
            for (int c = 0; c < K; ++c) xv[c] = dc ? s[c] / dI : T(0);
            stk<T, K>(xc + (size_t)I * K, xv);
        }
    }
}

// x_u += p_u xc_agg(u), K vectors
template <class T, int K>
__global__ void k_mv_prolong(int n, const int* __restrict__ agg, const T* __restrict__ pval,
                             const T* __restrict__ xc, T* __restrict__ x) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        T cu[K], xu[K];
        ldk<T, K>(xc + (size_t)__ldg(agg + u) * K, cu);
        ldk<T, K>(x + (size_t)u * K, xu);
        const T p = pval ? __ldg(pval + u) : T(1);
#pragma unroll
        for (int c = 0; c < K; ++c) xu[c] += pval ? p * cu[c] : cu[c];
        stk<T, K>(x + (size_t)u * K, xu);
    }
}

// x = N v for K vectors: a warp per row of N (row-major, stride ld), v staged
// in shared memory
template <class T, int K>
__global__ void k_mv_dense(int m, int ld, const T* __restrict__ N, const T* __restrict__ v, T* __restrict__ x,
                           int accum) {
    extern __shared__ __align__(16) unsigned char mv_dyn[];
    T* vs = reinterpret_cast<T*>(mv_dyn);
    for (int i = threadIdx.x; i < m * K; i += blockDim.x) vs[i] = v[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + warp;
    if (row >= m) return;
    T s[K];
#pragma unroll
    for (int c = 0; c < K; ++c) s[c] = T(0);
    const T* a = N + (size_t)row * ld;
    for (int j = lane; j < m; j += 32) {
        const T aj = __ldg(a + j);
#pragma unroll
        for (int c = 0; c < K; ++c) s[c] = mfma(aj, vs[j * K + c], s[c]);
    }
#pragma unroll
    for (int c = 0; c < K; ++c) {
        T w = s[c];
        for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
        if (lane == 0) x[(size_t)row * K + c] = accum ? x[(size_t)row * K + c] + w : w;
    }
}

// x = X b for K vectors on the coarsest level (X the FP64 pseudo-inverse)
template <class T, int K>
__global__ void k_mv_coarse(int m, const double* __restrict__ X, const T* __restrict__ b, T* __restrict__ x,
                            int accum) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < m; i += nw) {
        double s[K];
#pragma unroll
        for (int c = 0; c < K; ++c) s[c] = 0.0;
        for (int j = lane; j < m; j += 32) {
            const double a = __ldg(X + (size_t)i * m + j);
#pragma unroll
            for (int c = 0; c < K; ++c) s[c] += a * (double)b[(size_t)j * K + c];
        }
#pragma unroll
        for (int c = 0; c < K; ++c) {
            double w = s[c];
            for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
            if (lane == 0) x[(size_t)i * K + c] = accum ? x[(size_t)i * K + c] + (T)w : (T)w;
        }
    }
}

// into the finest level's K vectors: v[i * K + c] = (T)(r[c * n + perm(i)] * inv[c])
// (perm null: the identity; r column-major with leading dimension n; columns
// c >= kr are zero)
template <class T, int K>
__global__ void k_mv_in(int n, int kr, const int* __restrict__ perm, const double* __restrict__ r,
                        const double* __restrict__ inv, T* __restrict__ v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int u = perm ? __ldg(perm + i) : i;
#pragma unroll
        for (int c = 0; c < K; ++c)
            v[(size_t)i * K + c] = c < kr ? (T)(r[(size_t)c * n + u] * inv[c]) : T(0);
    }
}

// out of them: z[c * n + u] = scale[c] * (double)v[iperm(u) * K + c], c < kr
template <class T, int K>
__global__ void k_mv_out(int n, int kr, const int* __restrict__ iperm, const T* __restrict__ v,
                         const double* __restrict__ scale, double* __restrict__ z) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const int i = iperm ? __ldg(iperm + u) : u;
#pragma unroll
        for (int c = 0; c < K; ++c)
            if (c < kr) z[(size_t)c * n + u] = scale[c] * (double)v[(size_t)i * K + c];
    }
}

inline int mv_grid(int64_t threads) {
    int64_t g = (threads + 255) / 256;
    if (g < 1) g = 1;
    if (g > (int64_t)kNumSMs * 32) g = kNumSMs * 32;
    return (int)g;
}

}  // namespace

#define PC_K_DISPATCH(K, CALL)                      \
    switch (K) {                                    \
        case 1: CALL(1); break;                     \
        case 2: CALL(2); break;                     \
        case 4: CALL(4); break;                     \
        case 8: CALL(8); break;                     \
        default: fail(PCAMG_ERR_INVALID, "batch width must be 1, 2, 4 or 8"); \
    }

template <class T>
void mv_rows(cudaStream_t s, int mode, int K, int nrows, const int* rows, int beg, const Csr& A, const T* x,
             const T* b, const T* d, T* out) {
    if (nrows <= 0) return;
    const T* val;
    if constexpr (sizeof(T) == 8) val = A.val; else val = A.val32;
    const int lpr = A.lpr;
    const int g = mv_grid((int64_t)nrows * lpr);
#define CALLM(KK, M) k_mv_rows<T, KK, M><<<g, 256, 0, s>>>(nrows, rows, beg, lpr, A.rowptr, A.col, val, x, b, d, out)
#define CALL(KK)                                             \
    do {                                                     \
        if (mode == 0) CALLM(KK, MV_RES);                    \
        else if (mode == 1) CALLM(KK, MV_JAC);               \
        else CALLM(KK, MV_GS);                               \
    } while (0)
    PC_K_DISPATCH(K, CALL)
#undef CALL
#undef CALLM
    PC_LAUNCHN("mv_rows", 1);
}

template <class T>
void mv_restrict(cudaStream_t s, int K, int nc, const int* agg_ptr, const int* mem, const T* pval, const T* r,
                 T* bc, T* xc, const T* dc) {
#define CALL(KK) k_mv_restrict<T, KK><<<mv_grid(nc), 256, 0, s>>>(nc, agg_ptr, mem, pval, r, bc, xc, dc)
    PC_K_DISPATCH(K, CALL)
#undef CALL
    PC_LAUNCHN("mv_restrict", 1);
}

template <class T>
void mv_prolong(cudaStream_t s, int K, int n, const int* agg, const T* pval, const T* xc, T* x) {
#define CALL(KK) k_mv_prolong<T, KK><<<mv_grid(n), 256, 0, s>>>(n, agg, pval, xc, x)
    PC_K_DISPATCH(K, CALL)
#undef CALL
    PC_LAUNCHN("mv_prolong", 1);
}

template <class T>
void mv_dense(cudaStream_t s, int K, int m, int ld, const T* N, const T* v, T* x, bool accum) {
    const size_t smem = sizeof(T) * (size_t)m * K;
    if (smem > 200 * 1024) fail(PCAMG_ERR_INVALID, "batched tail product: vectors exceed shared memory");
    const int warps = 16;
    const int g = (m + warps - 1) / warps;
#define CALL(KK)                                                                                              \
    do {                                                                                                      \
        PC_CUDA(cudaFuncSetAttribute(k_mv_dense<T, KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        k_mv_dense<T, KK><<<g, warps * 32, smem, s>>>(m, ld, N, v, x, accum ? 1 : 0);                        \
    } while (0)
    PC_K_DISPATCH(K, CALL)
#undef CALL
    PC_LAUNCHN("mv_dense", 1);
}

template <class T>
void mv_coarse(cudaStream_t s, int K, int m, const double* X, const T* b, T* x, bool accum) {
    const int g = std::max(1, std::min(kNumSMs * 4, (m * 32 + 255) / 256));
#define CALL(KK) k_mv_coarse<T, KK><<<g, 256, 0, s>>>(m, X, b, x, accum ? 1 : 0)
    PC_K_DISPATCH(K, CALL)
#undef CALL
    PC_LAUNCHN("mv_coarse", 1);
}

template <class T>
void mv_in(cudaStream_t s, int K, int kr, int n, const int* perm, const double* r, const double* inv, T* v) {
#define CALL(KK) k_mv_in<T, KK><<<mv_grid(n), 256, 0, s>>>(n, kr, perm, r, inv, v)
    PC_K_DISPATCH(K, CALL)
#undef CALL
    PC_LAUNCHN("mv_in", 1);
}

template <class T>
void mv_out(cudaStream_t s, int K, int kr, int n, const int* iperm, const T* v, const double* scale, double* z) {
#define CALL(KK) k_mv_out<T, KK><<<mv_grid(n), 256, 0, s>>>(n, kr, iperm, v, scale, z)
    PC_K_DISPATCH(K, CALL)
#undef CALL
    PC_LAUNCHN("mv_out", 1);
}

#define PC_MV_INST(T)                                                                                          \
    template void mv_rows<T>(cudaStream_t, int, int, int, const int*, int, const Csr&, const T*, const T*,       \
                             const T*, T*);                                                                    \
    template void mv_restrict<T>(cudaStream_t, int, int, const int*, const int*, const T*, const T*, T*, T*,    \
                                 const T*);                                                                    \
    template void mv_prolong<T>(cudaStream_t, int, int, const int*, const T*, const T*, T*);                   \
    template void mv_dense<T>(cudaStream_t, int, int, int, const T*, const T*, T*, bool);                      \
    template void mv_coarse<T>(cudaStream_t, int, int, const double*, const T*, T*, bool);                     \
    template void mv_in<T>(cudaStream_t, int, int, int, const int*, const double*, const double*, T*);          \
    template void mv_out<T>(cudaStream_t, int, int, int, const int*, const T*, const double*, double*);
PC_MV_INST(float)
PC_MV_INST(double)
#undef PC_MV_INST

}  // namespace pc
