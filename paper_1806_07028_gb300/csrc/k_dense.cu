// Coarsest level: dense Cholesky A = L L^T in left-looking order where a pivot
// <= tau * max diag (or the last one, when the chain keeps the constant null
// space) is pinned: its row and column act as the identity with a zero
// right-hand side, so that unknown is 0. The explicit pseudo-inverse X is then
// formed column by column; the coarse solve is the dense product x = X r.
// Every sum runs sequentially in a fixed order with one rounding per operation.
#include "pcamg_internal.cuh"

namespace pc {

namespace {

__global__ void k_dense_assemble(int m, const int* __restrict__ rowptr, const int* __restrict__ col,
                                 const double* __restrict__ val, double* __restrict__ D) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        for (int j = 0; j < m; ++j) D[(size_t)i * m + j] = 0.0;
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) D[(size_t)i * m + col[k]] = val[k];
    }
}

__global__ void __launch_bounds__(1024) k_chol_pinned(int m, const double* __restrict__ D,
                                                      int force_last, double tau,
                                                      double* __restrict__ L, int* __restrict__ pin,
                                                      int* __restrict__ npinned) {
    __shared__ double s_lkk;
    __shared__ int s_pin;
    __shared__ double s_maxd;
    if (threadIdx.x == 0) {
        double md = 0.0;
        for (int i = 0; i < m; ++i) md = fmax(md, D[(size_t)i * m + i]);
        s_maxd = md;
        *npinned = 0;
    }
    for (size_t t = threadIdx.x; t < (size_t)m * m; t += blockDim.x) L[t] = 0.0;
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        if (threadIdx.x == 0) {
            double d = D[(size_t)k * m + k];
            const double* Lk = L + (size_t)k * m;
            int j = 0;
            for (; j + 8 <= k; j += 8) {
                double l[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) l[u] = Lk[j + u];
#pragma unroll
                for (int u = 0; u < 8; ++u) d = __dsub_rn(d, __dmul_rn(l[u], l[u]));
            }
            for (; j < k; ++j) d = __dsub_rn(d, __dmul_rn(Lk[j], Lk[j]));
            int p = (force_last && k == m - 1) || !(d > tau * s_maxd);
            s_pin = p;
            pin[k] = p;
            if (p) { *npinned += 1; s_lkk = 0.0; }
            else { s_lkk = __dsqrt_rn(d); L[(size_t)k * m + k] = s_lkk; }
        }
        __syncthreads();
        if (!s_pin) {
            double lkk = s_lkk;
            const double* Lk = L + (size_t)k * m;
            for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) {
                const double* Li = L + (size_t)i * m;
                double s = D[(size_t)i * m + k];
                int j = 0;
                for (; j + 8 <= k; j += 8) {
                    double a[8], b[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) { a[u] = Li[j + u]; b[u] = Lk[j + u]; }
#pragma unroll
                    for (int u = 0; u < 8; ++u) s = __dsub_rn(s, __dmul_rn(a[u], b[u]));
                }
                for (; j < k; ++j) s = __dsub_rn(s, __dmul_rn(Li[j], Lk[j]));
                L[(size_t)i * m + k] = __ddiv_rn(s, lkk);
            }
        }
        __syncthreads();
    }
}

// Column c of X: forward L y = e_c, backward L^T x = y (y kept in the column).
__global__ void k_chol_inverse(int m, const double* __restrict__ L, const int* __restrict__ pin,
                               double* __restrict__ X) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        for (int i = 0; i < m; ++i) {
            if (pin[i]) { X[(size_t)i * m + c] = 0.0; continue; }
            double s = (i == c) ? 1.0 : 0.0;
            const double* Li = L + (size_t)i * m;
            int j = 0;
            for (; j + 8 <= i; j += 8) {
                double a[8], b[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) { a[u] = Li[j + u]; b[u] = X[(size_t)(j + u) * m + c]; }
#pragma unroll
                for (int u = 0; u < 8; ++u) s = __dsub_rn(s, __dmul_rn(a[u], b[u]));
            }
            for (; j < i; ++j) s = __dsub_rn(s, __dmul_rn(Li[j], X[(size_t)j * m + c]));
            X[(size_t)i * m + c] = __ddiv_rn(s, Li[i]);
        }
        for (int i = m - 1; i >= 0; --i) {
            if (pin[i]) { X[(size_t)i * m + c] = 0.0; continue; }
            double s = X[(size_t)i * m + c];
            int j = i + 1;
            for (; j + 8 <= m; j += 8) {
                double a[8], b[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) { a[u] = L[(size_t)(j + u) * m + i]; b[u] = X[(size_t)(j + u) * m + c]; }
#pragma unroll
                for (int u = 0; u < 8; ++u) s = __dsub_rn(s, __dmul_rn(a[u], b[u]));
            }
            for (; j < m; ++j) s = __dsub_rn(s, __dmul_rn(L[(size_t)j * m + i], X[(size_t)j * m + c]));
            X[(size_t)i * m + c] = __ddiv_rn(s, L[(size_t)i * m + i]);
        }
    }
}

}  // namespace

void coarse_factor(Ctx& c, int32_t m, const int32_t* rowptr, const int32_t* col, const double* val,
                   bool force_last, DBuf<double>& Xinv, int32_t* npinned) {
    cudaStream_t s = c.stream;
    DBuf<double> D, L;
    DBuf<int32_t> pin, np;
    D.alloc(c.mem, (size_t)m * m);
    L.alloc(c.mem, (size_t)m * m);
    pin.alloc(c.mem, m);
    np.alloc(c.mem, 1);
    Xinv.alloc(c.mem, (size_t)m * m);
    int g = (m + kBlock - 1) / kBlock;
    k_dense_assemble<<<g, kBlock, 0, s>>>(m, rowptr, col, val, D.p); ::pc::count_launches(1);
    k_chol_pinned<<<1, 1024, 0, s>>>(m, D.p, force_last ? 1 : 0, 1e-12, L.p, pin.p, np.p); ::pc::count_launches(1);
    k_chol_inverse<<<g, kBlock, 0, s>>>(m, L.p, pin.p, Xinv.p); ::pc::count_launches(1);
    PC_LAUNCH("coarse_factor");
    *npinned = read_i32(c, np.p);
}

}  // namespace pc
