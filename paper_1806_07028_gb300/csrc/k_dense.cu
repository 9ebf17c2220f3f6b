// Coarsest level: dense Cholesky A = L L^T in left-looking order where a pivot
// <= tau * max diag (or the last one, when the chain keeps the constant null
// space) is pinned: its row and column act as the identity with a zero
// right-hand side, so that unknown is 0. The pseudo-inverse is then
// X = L^-T L^-1 restricted to the unpinned unknowns (zero rows and columns for
// pinned ones), formed as Y = L^-1 one column per block and X = Y^T Y; the
// coarse solve is the dense product x = X r.
//
// GB300 executes FP64 at about two lanes per clock per SM, so the work is laid
// out to keep many SMs busy where it is independent (the columns of Y, the
// entries of X) and to keep the one sequential part (the factorisation) free
// of serial reductions: each thread owns one row and accumulates its dot
// products itself.
#include <algorithm>

#include "pcamg_internal.cuh"

namespace pc {

namespace {

constexpr int kInvChunkMax = 32;     // columns of L staged in shared memory per step of Y
constexpr int kInvStageDoubles = 24576;   // 192 KB of staged columns at most

__global__ void k_dense_assemble(int m, const int* __restrict__ rowptr, const int* __restrict__ col,
                                 const double* __restrict__ val, double* __restrict__ D) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        for (int j = 0; j < m; ++j) D[(size_t)i * m + j] = 0.0;
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) D[(size_t)i * m + col[k]] = val[k];
    }
}

// Left-looking pinned Cholesky on one block. L is column-major with leading
// dimension ld (Lc[j * ld + i] = L_ij, zero-initialised), so for a fixed
// column the threads' rows are contiguous. Step k: every thread with a row
// i >= k forms s_i = sum_{j<k} L_ij L_kj; the pivot d = A_kk - s_k decides
// pinning; the rows below get L_ik = (A_ik - s_i) / sqrt(d). Loads of L are
// plain (L1-cached): within one block __syncthreads makes the stores visible.
__global__ void __launch_bounds__(1024) k_chol_pinned(int m, int ld, const double* __restrict__ D,
                                                      int force_last, double tau, double* Lc,
                                                      int* __restrict__ pin, int* __restrict__ npinned) {
    extern __shared__ double sv[];   // s_i of the current step, m entries
    __shared__ double s_lkk, s_maxd;
    __shared__ int s_pin, s_np;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid < 32) {
        double md = 0.0;
        for (int i = tid; i < m; i += 32) md = fmax(md, D[(size_t)i * m + i]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
        if (tid == 0) { s_maxd = md; s_np = 0; }
    }
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        const double* Lk = Lc + k;   // L_kj = Lk[j * ld]
        for (int i = k + tid; i < m; i += nt) {
            const double* Li = Lc + i;
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            int j = 0;
            for (; j + 4 <= k; j += 4) {
                a0 = fma(Li[(size_t)j * ld], Lk[(size_t)j * ld], a0);
                a1 = fma(Li[(size_t)(j + 1) * ld], Lk[(size_t)(j + 1) * ld], a1);
                a2 = fma(Li[(size_t)(j + 2) * ld], Lk[(size_t)(j + 2) * ld], a2);
                a3 = fma(Li[(size_t)(j + 3) * ld], Lk[(size_t)(j + 3) * ld], a3);
            }
            for (; j < k; ++j) a0 = fma(Li[(size_t)j * ld], Lk[(size_t)j * ld], a0);
            sv[i] = (a0 + a1) + (a2 + a3);
        }
        __syncthreads();
        if (tid == 0) {
            const double d = D[(size_t)k * m + k] - sv[k];
            const int p = (force_last && k == m - 1) || !(d > tau * s_maxd);
            pin[k] = p;
            s_pin = p;
            if (p) {
                s_np += 1;
            } else {
                s_lkk = sqrt(d);
                Lc[(size_t)k * ld + k] = s_lkk;
            }
        }
        __syncthreads();
        if (!s_pin) {   // column k of L stays zero for a pinned pivot
            const double lkk = s_lkk;
            for (int i = k + 1 + tid; i < m; i += nt) Lc[(size_t)k * ld + i] = (D[(size_t)i * m + k] - sv[i]) / lkk;
        }
        __syncthreads();
    }
    if (tid == 0) *npinned = s_np;
}

// Column c of Y = L^-1 (pinned rows zero) by forward substitution in
// right-looking form: thread r keeps t_r = delta_rc - sum_{j<i} L_rj y_j; at
// step i the owner of row i finishes y_i = t_i / L_ii and every later row
// subtracts L_ri y_i. Columns of L are staged K at a time. Requires
// m <= blockDim.x. Y is written row-major: Yr[k * ld + c] = Y_kc.
__global__ void __launch_bounds__(1024) k_chol_forward(int m, int ld, int K, const double* __restrict__ Lc,
                                                       const int* __restrict__ pin, double* __restrict__ Yr) {
    extern __shared__ double S[];   // K staged columns, rows [0, m)
    __shared__ double s_y[2];
    const int c = blockIdx.x, r = threadIdx.x;
    double t = (r == c) ? 1.0 : 0.0, y = 0.0;
    for (int i0 = c; i0 < m; i0 += K) {
        const int i1 = min(i0 + K, m);
        for (int q = i0; q < i1; ++q)
            if (r >= i0 && r < m) S[(q - i0) * m + r] = Lc[(size_t)q * ld + r];
        __syncthreads();
        for (int i = i0; i < i1; ++i) {
            if (r == i) {
                y = pin[i] ? 0.0 : t / S[(i - i0) * m + i];
                s_y[i & 1] = y;
            }
            __syncthreads();
            const double yi = s_y[i & 1];
            if (r > i && r < m) t = fma(-S[(i - i0) * m + r], yi, t);
        }
        __syncthreads();
    }
    if (r < m) Yr[(size_t)r * ld + c] = (r >= c) ? y : 0.0;
}

// X = Y^T Y: block i computes row i, thread c the entry sum_{k >= max(i,c)} Y_ki Y_kc.
__global__ void k_xty(int m, int ld, const double* __restrict__ Yr, double* __restrict__ X) {
    const int i = blockIdx.x;
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
        double a0 = 0.0, a1 = 0.0;
        int k = max(i, c);
        for (; k + 2 <= m; k += 2) {
            a0 = fma(__ldg(Yr + (size_t)k * ld + i), __ldg(Yr + (size_t)k * ld + c), a0);
            a1 = fma(__ldg(Yr + (size_t)(k + 1) * ld + i), __ldg(Yr + (size_t)(k + 1) * ld + c), a1);
        }
        if (k < m) a0 = fma(__ldg(Yr + (size_t)k * ld + i), __ldg(Yr + (size_t)k * ld + c), a0);
        X[(size_t)i * m + c] = a0 + a1;
    }
}

// Larger coarsest levels (m > 1024): column c of X by forward and back
// substitution, one thread per column (slow, rare: coarsening stalled).
__global__ void k_chol_inverse_cols(int m, int ld, const double* __restrict__ Lc, const int* __restrict__ pin,
                                    double* __restrict__ X) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        for (int i = 0; i < m; ++i) {
            if (pin[i]) { X[(size_t)i * m + c] = 0.0; continue; }
            double s = (i == c) ? 1.0 : 0.0;
            for (int j = 0; j < i; ++j) s = fma(-__ldg(Lc + (size_t)j * ld + i), X[(size_t)j * m + c], s);
            X[(size_t)i * m + c] = s / __ldg(Lc + (size_t)i * ld + i);
        }
        for (int i = m - 1; i >= 0; --i) {
            if (pin[i]) { X[(size_t)i * m + c] = 0.0; continue; }
            double s = X[(size_t)i * m + c];
            for (int j = i + 1; j < m; ++j) s = fma(-__ldg(Lc + (size_t)i * ld + j), X[(size_t)j * m + c], s);
            X[(size_t)i * m + c] = s / __ldg(Lc + (size_t)i * ld + i);
        }
    }
}

}  // namespace

void coarse_factor(Ctx& c, int32_t m, const int32_t* rowptr, const int32_t* col, const double* val,
                   bool force_last, DBuf<double>& Xinv, int32_t* npinned) {
    cudaStream_t s = c.stream;
    const int ld = (m + 15) / 16 * 16;   // 128-byte columns
    DBuf<double> D, L, Y;
    DBuf<int32_t> pin, np;
    D.alloc(c.mem, (size_t)m * m);
    L.alloc(c.mem, (size_t)m * ld);
    pin.alloc(c.mem, m);
    np.alloc(c.mem, 1);
    Xinv.alloc(c.mem, (size_t)m * m);
    PC_CUDA(cudaMemsetAsync(L.p, 0, sizeof(double) * (size_t)m * ld, s));
    int g = (m + kBlock - 1) / kBlock;
    k_dense_assemble<<<g, kBlock, 0, s>>>(m, rowptr, col, val, D.p); ::pc::count_launches(1);
    const int nt = std::min(1024, (m + 31) / 32 * 32);
    k_chol_pinned<<<1, nt, sizeof(double) * m, s>>>(m, ld, D.p, force_last ? 1 : 0, 1e-12, L.p, pin.p, np.p); ::pc::count_launches(1);
    if (m <= 1024) {
        Y.alloc(c.mem, (size_t)m * ld);
        const int K = std::max(1, std::min(kInvChunkMax, kInvStageDoubles / m));
        const size_t sm = sizeof(double) * (size_t)K * m;
        PC_CUDA(cudaFuncSetAttribute(k_chol_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_chol_forward<<<m, nt, sm, s>>>(m, ld, K, L.p, pin.p, Y.p); ::pc::count_launches(1);
        k_xty<<<m, std::min(256, nt), 0, s>>>(m, ld, Y.p, Xinv.p); ::pc::count_launches(1);
    } else {
        k_chol_inverse_cols<<<(m + 31) / 32, 32, 0, s>>>(m, ld, L.p, pin.p, Xinv.p); ::pc::count_launches(1);
    }
    PC_LAUNCH("coarse_factor");
    *npinned = read_i32(c, np.p);
}

}  // namespace pc
