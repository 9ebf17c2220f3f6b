// Learned start vector: a message-passing network over the graph of A that
// maps per-vertex features to the first test vector of the adaptive method.
// The paper has no learned component; the network, its loss and its training
// are this library's own:
//
//   f_i  = [u_i sqrt(n), log max(deg_i, 1), log max(D_i, tiny)], the last two
//          minus their means over the vertices       (u: relaxed random start)
//   h0   = C(GELU(W_in f + b_in))                                   3 -> 64
//   h'   = C(GELU(W_l [h ; m] + b_l)),  m_i = sum_{j != i} |a_ij| h_j / D_i,   4 layers, 128 -> 64
//   y    = w_out . h + b_out,  y-hat = (y - mean y) / ||y - mean y||
//
// C subtracts every channel's mean over the vertices, so the bfloat16 operands
// carry the variation between vertices, not a common offset. The layer
// kernels store G = GELU(z) in FP32; its column sums are formed next, and the
// following layer subtracts the means while it stages its bfloat16 operand.
//
// Weights are used rounded to bfloat16; the layer products run on the tensor
// cores (tcgen05.mma kind::f16, BF16 operands staged in shared memory, FP32
// accumulators in tensor memory), one CTA per 128-row tile: M = 128 rows,
// N = 64 outputs, K = 128 inputs. The neighbour mean m is formed by the same
// CTA while it stages the tile (a warp per row, 256-byte FP32 feature rows).
// Training (fwd + bwd + Adam) keeps FP32 master weights; the backward products
// dX = dZ W (M = 128 rows, N = 128, K = 64) and dW = X^T dZ (M = 128 inputs,
// N = 64, K = the rows of the CTA's tiles) are tensor-core products as well,
// the dW partials of the CTAs summed in a fixed order.
//
// Loss: for every vertex i over its candidate pairs C(i) (the pattern of A^2
// without i, the pairs Alg. 4 scores), the softmax of -|e_i - e_j| / tau_i of
// the target e is compared with the softmax of -|y_i - y_j| / tau_i of y-hat
// by cross-entropy; tau_i is the standard deviation of |e_i - e_j| over C(i).
// Loss and its gradient in FP64.
//
// Shared-memory operand layout: K-major, no swizzle. A core matrix is 8 rows
// x 16 bytes (8 bf16) stored as 128 contiguous bytes; core matrices adjacent
// in K are 128 bytes apart (leading byte offset), groups of 8 rows are
// (K / 8) * 128 bytes apart (stride byte offset).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "pcamg_internal.cuh"

namespace pc {

namespace {

constexpr int kH = kMpnnHidden;            // 64
constexpr int kTile = 128;                 // rows per tensor-core tile
constexpr int kThr = 256;                  // 8 warps
constexpr int kOffWin = 0, kOffBin = 192, kOffLayer0 = 256, kLayerStride = 8256;
constexpr int kOffWout = 256 + 4 * 8256, kOffBout = kOffWout + 64;
static_assert(kOffBout + 1 == kMpnnParams, "parameter layout");

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) in a K-major operand with K columns
__device__ __forceinline__ uint32_t kmaj(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start, leading / stride byte offsets, the
// fixed 0b001 field at bits 46-48, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* holder, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(holder)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(mbar))
                 : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* m) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(m)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(saddr(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait (about two seconds of SM clock); false when it gave up
__device__ bool mbar_wait(uint64_t* m, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try(m, parity))
        if (clock64() - t0 > (1ll << 32)) return false;
    return true;
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (one row per thread)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// erf by Abramowitz & Stegun, Handbook of Mathematical Functions (1964),
// formula 7.1.26: erf(x) = 1 - (a1 t + ... + a5 t^5) exp(-x^2), t = 1/(1 + p x)
// for x >= 0, odd in x, absolute error <= 1.5e-7 (far below the bfloat16
// operands' resolution). It takes one fast exponential and one fast
// reciprocal; the network evaluates it for every activation, where the
// library erf's instruction count bounded the layer kernels.
__device__ __forceinline__ float erf_as(float x) {
    const float ax = fabsf(x);
    const float t = __fdividef(1.0f, fmaf(0.3275911f, ax, 1.0f));
    float p = 1.061405429f;
    p = fmaf(p, t, -1.453152027f);
    p = fmaf(p, t, 1.421413741f);
    p = fmaf(p, t, -0.284496736f);
    p = fmaf(p, t, 0.254829592f);
    const float y = 1.0f - p * t * __expf(-ax * ax);
    return copysignf(y, x);
}
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erf_as(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.0f + erf_as(x * 0.70710678118654752f)) + x * __expf(-0.5f * x * x) * 0.39894228040143268f;
}

// The MMA issue/commit/wait of one tile: thread 0 issues nk products of K = 16,
// every thread waits; all threads return the same verdict. On a wait that gave
// up the error flag is set and the products in flight get one more bounded wait.
__device__ bool run_mma(uint32_t tmem, uint32_t a0, uint32_t b0, uint32_t lbo, uint32_t sbo_a, uint32_t sbo_b,
                        uint32_t idesc, int nk, bool accumulate, uint64_t* mbar, uint32_t& phase, int* err) {
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc_after();
        for (int kk = 0; kk < nk; ++kk)
            mma_bf16(tmem, sdesc(a0 + kk * 256, lbo, sbo_a), sdesc(b0 + kk * 256, lbo, sbo_b), idesc,
                     (accumulate || kk > 0) ? 1u : 0u);
        mma_commit(mbar);
    }
    __syncwarp();
    const bool mine = mbar_wait(mbar, phase);
    const bool ok = __syncthreads_and(mine) != 0;
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(err, 1);
        if (!mine) mbar_wait(mbar, phase);
    }
    phase ^= 1u;
    tc_after();
    return ok;
}

// ---------------------------------------------------------------- forward
// features (uncentred) and 1/D, one thread per row
__global__ void k_mpnn_feat(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                            const double* __restrict__ val, const double* __restrict__ u, double sqrtn,
                            float* __restrict__ invD, float* __restrict__ F) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int deg = 0;
        double D = 0.0;
        for (int q = rowptr[i]; q < rowptr[i + 1]; ++q)
            if (col[q] != i) { ++deg; D += fabs(val[q]); }
        invD[i] = D > 0.0 ? (float)(1.0 / D) : 0.0f;
        F[3 * i] = (float)(u[i] * sqrtn);
        F[3 * i + 1] = (float)log((double)max(deg, 1));
        F[3 * i + 2] = (float)log(fmax(D, 1e-300));
    }
}

// |a_ij| in FP32, converted once per pass (the layers read it for every
// feature lane; GB300 converts from FP64 at its low FP64 rate)
__global__ void k_abs_f32(int64_t nnz, const double* __restrict__ val, float* __restrict__ aw) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
        aw[k] = (float)fabs(val[k]);
}

// input head: centre features 1 and 2 (fsum: the feature column sums),
// z_in = W_in f + b_in, G0 = GELU(z_in); one thread per row
__global__ void k_mpnn_in(int n, const float* __restrict__ fsum, const float* __restrict__ wq,
                          float* __restrict__ F, float* __restrict__ Zin, float* __restrict__ G0) {
    const float m1 = fsum[1] / (float)n, m2 = fsum[2] / (float)n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float f0 = F[3 * i], f1 = F[3 * i + 1] - m1, f2 = F[3 * i + 2] - m2;
        F[3 * i + 1] = f1;
        F[3 * i + 2] = f2;
        for (int j = 0; j < kH; ++j) {
            float z = wq[kOffBin + j];
            z = fmaf(wq[kOffWin + 3 * j], f0, z);
            z = fmaf(wq[kOffWin + 3 * j + 1], f1, z);
            z = fmaf(wq[kOffWin + 3 * j + 2], f2, z);
            if (Zin) Zin[(size_t)i * kH + j] = z;
            G0[(size_t)i * kH + j] = gelu(z);
        }
    }
}

// One message-passing layer: stage [h | m] of a 128-row tile in bfloat16 --
// h = G - mean G (gsum: column sums of G), m = the weighted neighbour mean of
// G minus the same means -- then Z = [h | m] W^T on the tensor cores, bias,
// and G' = GELU(Z) in FP32. Xout / Zout keep the staged operand and Z for the
// backward pass (null in inference).
__global__ void __launch_bounds__(kThr, 2)
    k_mpnn_layer(int n, const int* __restrict__ rowptr, const int* __restrict__ col, const float* __restrict__ aw,
                 const float* __restrict__ invD, const float* __restrict__ G, const float* __restrict__ gsum,
                 const __nv_bfloat16* __restrict__ Wl, const float* __restrict__ bias,
                 __nv_bfloat16* __restrict__ Xout, float* __restrict__ Zout, float* __restrict__ Gout,
                 int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;              // 128 rows x 128 k, 32 KB
    unsigned char* sB = smem + 32768;      // 64 rows (outputs) x 128 k, 16 KB
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_hold;
    __shared__ float mu[kH];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int idx = threadIdx.x; idx < kH * 16; idx += kThr) {
        const int j = idx >> 4, c8 = idx & 15;
        *reinterpret_cast<uint4*>(sB + kmaj(j, c8 * 8, 128)) =
            *reinterpret_cast<const uint4*>(Wl + (size_t)j * 128 + c8 * 8);
    }
    if (threadIdx.x < kH) mu[threadIdx.x] = gsum[threadIdx.x] / (float)n;
    if (threadIdx.x == 0) mbar_init(&mbar);
    if (warp == 0) tmem_alloc(&tmem_hold, 64);
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = tmem_hold;
    const float mu0 = mu[2 * lane], mu1 = mu[2 * lane + 1];
    uint32_t phase = 0;
    const int ntiles = (n + kTile - 1) / kTile;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int r0 = t * kTile;
        // a warp per row: lane owns features 2 lane, 2 lane + 1 of both halves
        for (int r = warp; r < kTile; r += kThr / 32) {
            const int row = r0 + r;
            float h0 = 0.f, h1 = 0.f, a0 = 0.f, a1 = 0.f;
            if (row < n) {
                const float2 g = *reinterpret_cast<const float2*>(G + (size_t)row * kH + 2 * lane);
                h0 = g.x - mu0;
                h1 = g.y - mu1;
                // eight neighbours per step, their rows loaded before any is used
                // (the diagonal entry and the slots past the row's end add
                // 0 * G[row], which leaves the sums unchanged: the same
                // products in the same order as one neighbour at a time)
                const int e = rowptr[row + 1];
                for (int q = rowptr[row]; q < e; q += 8) {
                    int j[8];
                    float w[8];
                    float2 f[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const bool on = q + u < e;
                        j[u] = on ? col[q + u] : row;
                        w[u] = (!on || j[u] == row) ? 0.f : aw[q + u];
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) f[u] = *reinterpret_cast<const float2*>(G + (size_t)j[u] * kH + 2 * lane);
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        a0 = fmaf(w[u], f[u].x, a0);
                        a1 = fmaf(w[u], f[u].y, a1);
                    }
                }
                const float s = invD[row];
                a0 = a0 * s - mu0;
                a1 = a1 * s - mu1;
            }
            const __nv_bfloat162 hv = __floats2bfloat162_rn(h0, h1), mv = __floats2bfloat162_rn(a0, a1);
            *reinterpret_cast<__nv_bfloat162*>(sA + kmaj(r, 2 * lane, 128)) = hv;
            *reinterpret_cast<__nv_bfloat162*>(sA + kmaj(r, kH + 2 * lane, 128)) = mv;
            if (Xout && row < n) {
                *reinterpret_cast<__nv_bfloat162*>(Xout + (size_t)row * 2 * kH + 2 * lane) = hv;
                *reinterpret_cast<__nv_bfloat162*>(Xout + (size_t)row * 2 * kH + kH + 2 * lane) = mv;
            }
        }
        if (!run_mma(tmem, saddr(sA), saddr(sB), 128, 2048, 2048, idesc_bf16(128, 64), 8, false, &mbar, phase, err))
            break;
        const int quad = warp & 3, half = warp >> 2;
        const int row = r0 + quad * 32 + lane;
        float v[32];
        const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * 32);
        tmem_ld16(ta, v);
        tmem_ld16(ta + 16, v + 16);
        if (row < n) {
#pragma unroll
            for (int c = 0; c < 32; c += 4) {
                const int j = half * 32 + c;
                const float4 z = make_float4(v[c] + bias[j], v[c + 1] + bias[j + 1], v[c + 2] + bias[j + 2],
                                             v[c + 3] + bias[j + 3]);
                if (Zout) *reinterpret_cast<float4*>(Zout + (size_t)row * kH + j) = z;
                *reinterpret_cast<float4*>(Gout + (size_t)row * kH + j) =
                    make_float4(gelu(z.x), gelu(z.y), gelu(z.z), gelu(z.w));
            }
        }
        tc_before();
        __syncthreads();
    }
    tc_before();
    __syncthreads();
    if (warp == 0) tmem_free(tmem, 64);
}

// output head: y_i = w_out . (G_i - mean G) + b_out (FP64 result for the normalisation)
__global__ void k_mpnn_head(int n, const float* __restrict__ G, const float* __restrict__ gsum,
                            const float* __restrict__ wq, double* __restrict__ y) {
    const float inv_n = 1.0f / (float)n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float s = wq[kOffBout];
        const float* g = G + (size_t)i * kH;
        for (int c = 0; c < kH; ++c) s = fmaf(wq[kOffWout + c], g[c] - gsum[c] * inv_n, s);
        y[i] = (double)s;
    }
}

// ---------------------------------------------------------------- loss
// Per row i: tau_i (population standard deviation of |e_i - e_j| over C(i)),
// the log-sum-exps of the target and predicted logits, and the row's
// cross-entropy. One warp per row; tau_i = 0 marks a skipped row.
__global__ void k_loss_rows(int n, const int* __restrict__ cptr, const int* __restrict__ ccol,
                            const double* __restrict__ y, const double* __restrict__ e, double* __restrict__ tau,
                            double* __restrict__ lsep, double* __restrict__ lseq, double* __restrict__ ce) {
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = w0; i < n; i += nw) {
        const int b = cptr[i], en = cptr[i + 1];
        const double ei = e[i], yi = y[i];
        double s = 0.0;
        for (int q = b + lane; q < en; q += 32) s += fabs(ei - e[ccol[q]]);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const int cnt = max(en - b, 1);
        const double mean = s / cnt;
        double v = 0.0;
        for (int q = b + lane; q < en; q += 32) {
            const double d = fabs(ei - e[ccol[q]]) - mean;
            v += d * d;
        }
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const double ti = sqrt(v / cnt);
        double mp = -INFINITY, mq = -INFINITY;
        if (ti > 0.0)
            for (int q = b + lane; q < en; q += 32) {
                const int j = ccol[q];
                mp = fmax(mp, -fabs(ei - e[j]) / ti);
                mq = fmax(mq, -fabs(yi - y[j]) / ti);
            }
        for (int o = 16; o > 0; o >>= 1) {
            mp = fmax(mp, __shfl_xor_sync(0xffffffffu, mp, o));
            mq = fmax(mq, __shfl_xor_sync(0xffffffffu, mq, o));
        }
        double sp = 0.0, sq = 0.0;
        if (ti > 0.0)
            for (int q = b + lane; q < en; q += 32) {
                const int j = ccol[q];
                sp += exp(-fabs(ei - e[j]) / ti - mp);
                sq += exp(-fabs(yi - y[j]) / ti - mq);
            }
        for (int o = 16; o > 0; o >>= 1) {
            sp += __shfl_xor_sync(0xffffffffu, sp, o);
            sq += __shfl_xor_sync(0xffffffffu, sq, o);
        }
        const double lp = mp + log(sp), lq = mq + log(sq);
        double c = 0.0;
        if (ti > 0.0)
            for (int q = b + lane; q < en; q += 32) {
                const int j = ccol[q];
                const double p = exp(-fabs(ei - e[j]) / ti - lp);
                c -= p * (-fabs(yi - y[j]) / ti - lq);
            }
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) {
            tau[i] = ti;
            lsep[i] = ti > 0.0 ? lp : 0.0;
            lseq[i] = ti > 0.0 ? lq : 0.0;
            ce[i] = c;
        }
    }
}

// dL/dy-hat_i = (1/n) sum_{j in C(i)} -sign(y_i - y_j) ((q_ij - p_ij)/tau_i + (q_ji - p_ji)/tau_j)
__global__ void k_loss_grad(int n, const int* __restrict__ cptr, const int* __restrict__ ccol,
                            const double* __restrict__ y, const double* __restrict__ e,
                            const double* __restrict__ tau, const double* __restrict__ lsep,
                            const double* __restrict__ lseq, double* __restrict__ g) {
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    const double inv_n = 1.0 / (double)n;
    for (int i = w0; i < n; i += nw) {
        const double ei = e[i], yi = y[i], ti = tau[i];
        double s = 0.0;
        for (int q = cptr[i] + lane; q < cptr[i + 1]; q += 32) {
            const int j = ccol[q];
            const double d = yi - y[j], de = fabs(ei - e[j]);
            const double sg = (d > 0.0) ? 1.0 : ((d < 0.0) ? -1.0 : 0.0);
            double c = 0.0;
            if (ti > 0.0) c += (exp(-fabs(d) / ti - lseq[i]) - exp(-de / ti - lsep[i])) / ti;
            const double tj = tau[j];
            if (tj > 0.0) c += (exp(-fabs(d) / tj - lseq[j]) - exp(-de / tj - lsep[j])) / tj;
            s -= sg * c;
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) g[i] = s * inv_n;
    }
}

// ---------------------------------------------------------------- backward
// gz = (g - yhat (yhat . g)) / nrm (the mean of gz is removed afterwards)
__global__ void k_norm_back(int n, const double* __restrict__ g, const double* __restrict__ yhat,
                            const double* __restrict__ yg_slot, const double* __restrict__ nrm_slot,
                            double* __restrict__ gz) {
    const double yg = *yg_slot, inv = 1.0 / *nrm_slot;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        gz[i] = (g[i] - yhat[i] * yg) * inv;
}

// dH_4 = dy w_out (FP32 rows)
__global__ void k_head_back(int n, const double* __restrict__ dy, const float* __restrict__ wq,
                            float* __restrict__ dH) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)n * kH;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / kH), c = (int)(t % kH);
        dH[t] = (float)dy[i] * wq[kOffWout + c];
    }
}

// dZ = (dH - mean dH) * GELU'(Z): the centring's backward is the same centring
// (dHsum: column sums of dH); FP32 for the sums, BF16 for the tensor cores
__global__ void k_gelu_back(int n, const float* __restrict__ dH, const float* __restrict__ dHsum,
                            const float* __restrict__ Z, float* __restrict__ dZ, __nv_bfloat16* __restrict__ dZb) {
    const int64_t m = (int64_t)n * kH;
    const float inv_n = 1.0f / (float)n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
        const float v = (dH[t] - dHsum[t % kH] * inv_n) * gelu_grad(Z[t]);
        dZ[t] = v;
        if (dZb) dZb[t] = __float2bfloat16_rn(v);
    }
}

// dX = dZ W for a 128-row tile: columns [0, 64) go to dHs (the self half),
// [64, 128) to dM. A = dZ (M = rows, K = 64), B[c][j] = W[j][c] (N = 128, K = 64).
__global__ void __launch_bounds__(kThr, 2)
    k_mpnn_dx(int n, const __nv_bfloat16* __restrict__ dZ, const __nv_bfloat16* __restrict__ Wl,
              float* __restrict__ dHs, float* __restrict__ dM, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;            // 128 x 64, 16 KB
    unsigned char* sB = smem + 16384;    // 128 x 64, 16 KB
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_hold;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int idx = threadIdx.x; idx < kH * 128; idx += kThr) {
        const int j = idx >> 7, c = idx & 127;   // W[j][c] -> B(c, j)
        *reinterpret_cast<__nv_bfloat16*>(sB + kmaj(c, j, 64)) = Wl[idx];
    }
    if (threadIdx.x == 0) mbar_init(&mbar);
    if (warp == 0) tmem_alloc(&tmem_hold, 128);
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = tmem_hold;
    uint32_t phase = 0;
    const int ntiles = (n + kTile - 1) / kTile;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int r0 = t * kTile;
        for (int idx = threadIdx.x; idx < kTile * 8; idx += kThr) {
            const int r = idx >> 3, k8 = idx & 7, row = r0 + r;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (row < n) v = *reinterpret_cast<const uint4*>(dZ + (size_t)row * kH + k8 * 8);
            *reinterpret_cast<uint4*>(sA + kmaj(r, k8 * 8, 64)) = v;
        }
        if (!run_mma(tmem, saddr(sA), saddr(sB), 128, 1024, 1024, idesc_bf16(128, 128), 4, false, &mbar, phase,
                     err))
            break;
        const int quad = warp & 3, half = warp >> 2;
        const int row = r0 + quad * 32 + lane;
        float* out = half ? dM : dHs;
        const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * 64);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float v[16];
            tmem_ld16(ta + q * 16, v);
            if (row < n) {
                float4* o = reinterpret_cast<float4*>(out + (size_t)row * kH + q * 16);
#pragma unroll
                for (int u = 0; u < 4; ++u) o[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
            }
        }
        tc_before();
        __syncthreads();
    }
    tc_before();
    __syncthreads();
    if (warp == 0) tmem_free(tmem, 128);
}

// dH_prev_i = dHs_i + sum_{k != i} |a_ik| dM_k / D_k (the neighbour mean's
// transpose on the symmetric pattern); a warp per row, two features per lane
__global__ void k_nbr_back(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                           const float* __restrict__ aw, const float* __restrict__ invD,
                           const float* __restrict__ dHs, const float* __restrict__ dM, float* __restrict__ dH) {
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = w0; i < n; i += nw) {
        float2 a = *reinterpret_cast<const float2*>(dHs + (size_t)i * kH + 2 * lane);
        const int e = rowptr[i + 1];
        int q = rowptr[i];
        for (; q + 4 <= e; q += 4) {
            int k[4];
            float w[4];
            float2 m[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) k[u] = col[q + u];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                w[u] = (k[u] == i) ? 0.f : aw[q + u] * invD[k[u]];
                m[u] = *reinterpret_cast<const float2*>(dM + (size_t)k[u] * kH + 2 * lane);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a.x = fmaf(w[u], m[u].x, a.x);
                a.y = fmaf(w[u], m[u].y, a.y);
            }
        }
        for (; q < e; ++q) {
            const int k = col[q];
            if (k == i) continue;
            const float w = aw[q] * invD[k];
            const float2 m = *reinterpret_cast<const float2*>(dM + (size_t)k * kH + 2 * lane);
            a.x = fmaf(w, m.x, a.x);
            a.y = fmaf(w, m.y, a.y);
        }
        *reinterpret_cast<float2*>(dH + (size_t)i * kH + 2 * lane) = a;
    }
}

// dW^T partial of this CTA over its row tiles: A(c, r) = X[r][c] with X the
// staged [h | m] operand (M = 128 inputs, K = rows), B(j, r) = dZ[r][j]
// (N = 64). Partial written as part[cta][j][c] (FP32).
__global__ void __launch_bounds__(kThr, 1)
    k_mpnn_dw(int n, const __nv_bfloat16* __restrict__ X, const __nv_bfloat16* __restrict__ dZ,
              float* __restrict__ part, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;            // 128 inputs x 128 rows, 32 KB
    unsigned char* sB = smem + 32768;    // 64 outputs x 128 rows, 16 KB
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_hold;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) mbar_init(&mbar);
    if (warp == 0) tmem_alloc(&tmem_hold, 64);
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = tmem_hold;
    uint32_t phase = 0;
    bool any = false, ok = true;
    const int ntiles = (n + kTile - 1) / kTile;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int r0 = t * kTile;
        for (int idx = threadIdx.x; idx < kTile * 64; idx += kThr) {
            const int r = idx >> 6, c2 = (idx & 63) * 2, row = r0 + r;   // two inputs per step
            __nv_bfloat162 x = __floats2bfloat162_rn(0.f, 0.f), g = x;
            if (row < n) {
                x = *reinterpret_cast<const __nv_bfloat162*>(X + (size_t)row * 2 * kH + c2);
                if (c2 < kH) g = *reinterpret_cast<const __nv_bfloat162*>(dZ + (size_t)row * kH + c2);
            }
            *reinterpret_cast<__nv_bfloat16*>(sA + kmaj(c2, r, 128)) = x.x;
            *reinterpret_cast<__nv_bfloat16*>(sA + kmaj(c2 + 1, r, 128)) = x.y;
            if (c2 < kH) {
                *reinterpret_cast<__nv_bfloat16*>(sB + kmaj(c2, r, 128)) = g.x;
                *reinterpret_cast<__nv_bfloat16*>(sB + kmaj(c2 + 1, r, 128)) = g.y;
            }
        }
        ok = run_mma(tmem, saddr(sA), saddr(sB), 128, 2048, 2048, idesc_bf16(128, 64), 8, any, &mbar, phase, err);
        if (!ok) break;
        any = true;
        tc_before();
        __syncthreads();
    }
    // epilogue: TMEM lane c holds input c; columns are the outputs j
    const int quad = warp & 3, half = warp >> 2;
    const int c = quad * 32 + lane;
    float* dst = part + (size_t)blockIdx.x * kH * 128;
    if (ok && any) {
        tc_after();
        const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * 32);
        float v[32];
        tmem_ld16(ta, v);
        tmem_ld16(ta + 16, v + 16);
#pragma unroll
        for (int q = 0; q < 32; ++q) dst[(size_t)(half * 32 + q) * 128 + c] = v[q];
    } else {
        for (int q = 0; q < 32; ++q) dst[(size_t)(half * 32 + q) * 128 + c] = 0.f;
    }
    tc_before();
    __syncthreads();
    if (warp == 0) tmem_free(tmem, 64);
}

// out[k] = sum over the partial rows b of part[b][k]: block k, its threads
// take b = tid, tid + 256, ... and a fixed tree combines them (FP64).
constexpr int kSumThreads = 256;
__global__ void __launch_bounds__(kSumThreads) k_sum_parts(int nb, int K, const float* __restrict__ part,
                                                         float* __restrict__ out) {
    __shared__ double ws[kSumThreads / 32];
    const int k = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += kSumThreads) s += (double)part[(size_t)b * K + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kSumThreads / 32; ++w) t += ws[w];
        out[k] = (float)t;
    }
}

// Column sums of small per-row products into block partials (rows split in
// chunks of kSumRows; a thread per output column):
//   mode 0: plain sums         out[j]      = sum_i X[i][j]                  (K = 64)
//   mode 1: output head        out[c]      = sum_i dy_i (G_i[c] - mean G[c]), out[64] = sum_i dy_i (K = 65)
//   mode 2: input head         out[3j + k] = sum_i dZ[i][j] F[i][k], out[192 + j] = sum_i dZ[i][j]  (K = 256)
//   mode 3: features           out[k]      = sum_i F[i][k]                  (K = 3)
constexpr int kSumRows = 512;
__global__ void k_colsums(int n, int mode, const float* __restrict__ dZ, const double* __restrict__ dy,
                          const float* __restrict__ G, const float* __restrict__ gsum, const float* __restrict__ F,
                          float* __restrict__ part, int K) {
    const int b = blockIdx.x;
    const int i0 = b * kSumRows, i1 = min(n, i0 + kSumRows);
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        if (mode == 0 || mode == 3) {     // plain sums: FP32 within the block, four chains
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            const float* X = (mode == 0) ? dZ : F;
            const int ld = (mode == 0) ? kH : 3;
            int i = i0;
            for (; i + 4 <= i1; i += 4) {
                a0 += X[(size_t)i * ld + k];
                a1 += X[(size_t)(i + 1) * ld + k];
                a2 += X[(size_t)(i + 2) * ld + k];
                a3 += X[(size_t)(i + 3) * ld + k];
            }
            for (; i < i1; ++i) a0 += X[(size_t)i * ld + k];
            part[(size_t)b * K + k] = (a0 + a1) + (a2 + a3);
            continue;
        }
        double s = 0.0;
        const double mu = (mode == 1 && k < kH) ? (double)gsum[k] / (double)n : 0.0;
        for (int i = i0; i < i1; ++i) {
            if (mode == 1) s += (k < kH) ? dy[i] * ((double)G[(size_t)i * kH + k] - mu) : dy[i];
            else if (k < 192) s += (double)dZ[(size_t)i * kH + k / 3] * F[3 * i + k % 3];
            else s += dZ[(size_t)i * kH + (k - 192)];
        }
        part[(size_t)b * K + k] = (float)s;
    }
}

// Adam on the FP32 master weights, then the bfloat16-rounded working copies
__global__ void k_adam(int np, float lr, float c1, float c2, const float* __restrict__ g, float* __restrict__ w,
                       float* __restrict__ m, float* __restrict__ v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float vi = 0.999f * v[i] + 0.001f * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    }
}

__global__ void k_round_params(int np, const float* __restrict__ w, float* __restrict__ wq,
                               __nv_bfloat16* __restrict__ wl) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        const __nv_bfloat16 b = __float2bfloat16_rn(w[i]);
        wq[i] = __bfloat162float(b);
        const int o = i - kOffLayer0;
        if (o >= 0 && o < 4 * kLayerStride && (o % kLayerStride) < kH * 128)
            wl[(o / kLayerStride) * kH * 128 + (o % kLayerStride)] = b;
    }
}

int grid_for(int64_t work, int block = 256) {
    int64_t g = (work + block - 1) / block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, kNumSMs * 8));
}

}  // namespace

// ---------------------------------------------------------------- host side
struct Mpnn {
    Mem mem;   // the legacy default stream: the network's calls are synchronous
    DBuf<float> w_, m_, v_, g_, wq_;
    DBuf<__nv_bfloat16> wl_;
    float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr, *wq = nullptr;
    __nv_bfloat16* wl = nullptr;
    int64_t t = 0;
};

static void mpnn_refresh(Mpnn& M) {
    k_round_params<<<grid_for(kMpnnParams), 256>>>(kMpnnParams, M.w, M.wq, M.wl); ::pc::count_launches(1);
    PC_LAUNCH("mpnn_round");
}

Mpnn* mpnn_create(const float* h_params) {
    std::unique_ptr<Mpnn> M(new Mpnn());
    const size_t nb = kMpnnParams;
    M->w_.alloc(M->mem, nb); M->m_.alloc(M->mem, nb); M->v_.alloc(M->mem, nb);
    M->g_.alloc(M->mem, nb); M->wq_.alloc(M->mem, nb);
    M->wl_.alloc(M->mem, (size_t)4 * kH * 128);
    M->w = M->w_.p; M->m = M->m_.p; M->v = M->v_.p; M->g = M->g_.p; M->wq = M->wq_.p; M->wl = M->wl_.p;
    PC_CUDA(cudaMemsetAsync(M->g, 0, sizeof(float) * nb, nullptr));
    mpnn_set_params(*M, h_params);
    return M.release();
}

void mpnn_destroy(Mpnn* M) {
    if (!M) return;
    cudaDeviceSynchronize();   // the network's buffers may still be read by queued work
    delete M;
}

void mpnn_set_params(Mpnn& M, const float* h) {
    const size_t b = sizeof(float) * kMpnnParams;
    PC_CUDA(cudaMemcpy(M.w, h, b, cudaMemcpyHostToDevice));
    PC_CUDA(cudaMemset(M.m, 0, b));
    PC_CUDA(cudaMemset(M.v, 0, b));
    M.t = 0;
    mpnn_refresh(M);
    PC_CUDA(cudaDeviceSynchronize());
}

void mpnn_get_params(Mpnn& M, float* h) {
    PC_CUDA(cudaMemcpy(h, M.w, sizeof(float) * kMpnnParams, cudaMemcpyDeviceToHost));
}

void mpnn_get_grad(Mpnn& M, float* h) {
    PC_CUDA(cudaMemcpy(h, M.g, sizeof(float) * kMpnnParams, cudaMemcpyDeviceToHost));
}

// Activations of one pass over a graph; the training caches only when needed.
struct MpnnWork {
    DBuf<float> aw, invD, F, Zin, Z, G, gsum, dH, dHs, dM, dZ, part, hsum;
    DBuf<__nv_bfloat16> X, dZb;
    DBuf<double> y, tau, lsep, lseq, ce, gy, gz;
    DBuf<int32_t> err;
};

static void check_err(Ctx& c, const int32_t* err) {
    if (read_i32(c, err)) fail(PCAMG_ERR_CUDA, "mpnn: a tensor-core wait gave up");
}

static void set_smem(const void* fn, int bytes) {
    PC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
}

static int sum_blocks(int n) { return (n + kSumRows - 1) / kSumRows; }

// column sums of an FP32 [n x 64] matrix into out[64] (fixed order)
static void colsum64(cudaStream_t s, int n, const float* X, float* part, float* out) {
    const int nb = sum_blocks(n);
    k_colsums<<<nb, 64, 0, s>>>(n, 0, X, nullptr, nullptr, nullptr, nullptr, part, kH); ::pc::count_launches(1);
    k_sum_parts<<<kH, kSumThreads, 0, s>>>(nb, kH, part, out); ::pc::count_launches(1);
}

// forward; train = keep X_l, Z_l, every G_l, F and Z_in for the backward pass
static void forward(Ctx& c, Mpnn& P, const double* u, double* yhat, MpnnWork& w, bool train) {
    cudaStream_t s = c.stream;
    const int n = c.n;
    const int L = kMpnnLayers;
    const size_t nh = (size_t)n * kH;
    const int nb = sum_blocks(n);
    w.err.alloc(c.mem, 1);
    PC_CUDA(cudaMemsetAsync(w.err.p, 0, sizeof(int32_t), s));
    w.invD.alloc(c.mem, n);
    w.aw.alloc(c.mem, c.nnz);
    k_abs_f32<<<grid_for(c.nnz), 256, 0, s>>>(c.nnz, c.val.p, w.aw.p); ::pc::count_launches(1);
    w.F.alloc(c.mem, (size_t)n * 3);
    w.G.alloc(c.mem, train ? nh * (L + 1) : nh * 2);
    w.gsum.alloc(c.mem, (size_t)kH * (L + 1));
    w.part.alloc(c.mem, (size_t)nb * 256);
    if (train) {
        w.Zin.alloc(c.mem, nh);
        w.Z.alloc(c.mem, nh * L);
        w.X.alloc(c.mem, nh * 2 * L);
    }
    w.y.alloc(c.mem, n);
    k_mpnn_feat<<<grid_for(n), 256, 0, s>>>(n, c.rowptr.p, c.col.p, c.val.p, u, std::sqrt((double)n), w.invD.p, w.F.p);
    ::pc::count_launches(1);
    // column sums of the features, for centring the two degree features
    k_colsums<<<nb, 64, 0, s>>>(n, 3, nullptr, nullptr, nullptr, nullptr, w.F.p, w.part.p, 3); ::pc::count_launches(1);
    k_sum_parts<<<3, kSumThreads, 0, s>>>(nb, 3, w.part.p, w.gsum.p); ::pc::count_launches(1);
    k_mpnn_in<<<grid_for(n), 256, 0, s>>>(n, w.gsum.p, P.wq, w.F.p, train ? w.Zin.p : nullptr, w.G.p);
    ::pc::count_launches(1);
    auto Gl = [&](int l) { return w.G.p + (train ? (size_t)l : (size_t)(l & 1)) * nh; };
    colsum64(s, n, Gl(0), w.part.p, w.gsum.p);
    const int smem = 49152;
    set_smem((const void*)k_mpnn_layer, smem);
    const int ntiles = (n + kTile - 1) / kTile;
    const int grid = std::max(1, std::min(ntiles, 2 * kNumSMs));
    for (int l = 0; l < L; ++l) {
        k_mpnn_layer<<<grid, kThr, smem, s>>>(n, c.rowptr.p, c.col.p, w.aw.p, w.invD.p, Gl(l), w.gsum.p + l * kH,
                                              P.wl + (size_t)l * kH * 128,
                                              P.wq + kOffLayer0 + l * kLayerStride + kH * 128,
                                              train ? w.X.p + (size_t)l * nh * 2 : nullptr,
                                              train ? w.Z.p + l * nh : nullptr, Gl(l + 1), w.err.p);
        ::pc::count_launches(1);
        colsum64(s, n, Gl(l + 1), w.part.p, w.gsum.p + (l + 1) * kH);
    }
    k_mpnn_head<<<grid_for(n), 256, 0, s>>>(n, Gl(L), w.gsum.p + L * kH, P.wq, w.y.p); ::pc::count_launches(1);
    PC_LAUNCH("mpnn_forward");
    normalise_orth(c, w.y.p, yhat);
    check_err(c, w.err.p);
}

void mpnn_forward(Ctx& c, Mpnn& P, const double* u, double* yhat) {
    MpnnWork w;
    forward(c, P, u, yhat, w, false);
    sync(c);
}

double mpnn_loss_grad(Ctx& c, Mpnn& P, const double* u, const double* target) {
    cudaStream_t s = c.stream;
    const int n = c.n;
    const int L = kMpnnLayers;
    const size_t nh = (size_t)n * kH;
    if (!c.mpnn_cand) {
        c.mpnn_cand.reset(new Reweighted());
        build_candidates(c, target, *c.mpnn_cand);
    }
    const Reweighted& cand = *c.mpnn_cand;
    MpnnWork w;
    DBuf<double> yhat;
    yhat.alloc(c.mem, n);
    forward(c, P, u, yhat.p, w, true);
    // loss and dL/dy-hat
    w.tau.alloc(c.mem, n);
    w.lsep.alloc(c.mem, n);
    w.lseq.alloc(c.mem, n);
    w.ce.alloc(c.mem, n);
    w.gy.alloc(c.mem, n);
    w.gz.alloc(c.mem, n);
    const int gw = grid_for((int64_t)n * 32);
    k_loss_rows<<<gw, 256, 0, s>>>(n, cand.ptr.p, cand.col.p, yhat.p, target, w.tau.p, w.lsep.p, w.lseq.p, w.ce.p);
    ::pc::count_launches(1);
    k_loss_grad<<<gw, 256, 0, s>>>(n, cand.ptr.p, cand.col.p, yhat.p, target, w.tau.p, w.lsep.p, w.lseq.p, w.gy.p);
    ::pc::count_launches(1);
    PC_LAUNCH("mpnn_loss");
    double* sl = mpnn_slots(c);
    // ||y - mean y|| of the forward normalisation, before other reductions
    copy(s, 1, norm_slot(c), sl + 2);
    sum(s, n, w.ce.p, red_partials(c), sl + 0);
    // back through y-hat = (y - mean y) / ||y - mean y||
    dot(s, n, yhat.p, w.gy.p, red_partials(c), sl + 1);
    k_norm_back<<<grid_for(n), 256, 0, s>>>(n, w.gy.p, yhat.p, sl + 1, sl + 2, w.gz.p); ::pc::count_launches(1);
    sum(s, n, w.gz.p, red_partials(c), sl + 3);
    sub_mean(s, n, w.gz.p, sl + 3);           // gz is now dL/dy
    // output head
    w.dH.alloc(c.mem, nh);
    w.dHs.alloc(c.mem, nh);
    w.dM.alloc(c.mem, nh);
    w.dZ.alloc(c.mem, nh);
    w.dZb.alloc(c.mem, nh);
    w.hsum.alloc(c.mem, kH);
    const int nb = sum_blocks(n);
    const int ntiles = (n + kTile - 1) / kTile;
    const int gdw = std::max(1, std::min(ntiles, kNumSMs));
    DBuf<float> wpart;
    wpart.alloc(c.mem, (size_t)gdw * kH * 128);
    k_colsums<<<nb, 128, 0, s>>>(n, 1, nullptr, w.gz.p, w.G.p + (size_t)L * nh, w.gsum.p + L * kH, nullptr,
                                 w.part.p, 65);
    ::pc::count_launches(1);
    k_sum_parts<<<65, kSumThreads, 0, s>>>(nb, 65, w.part.p, P.g + kOffWout); ::pc::count_launches(1);
    k_head_back<<<grid_for((int64_t)nh), 256, 0, s>>>(n, w.gz.p, P.wq, w.dH.p); ::pc::count_launches(1);
    set_smem((const void*)k_mpnn_dx, 32768);
    set_smem((const void*)k_mpnn_dw, 49152);
    const int gdx = std::max(1, std::min(ntiles, 2 * kNumSMs));
    for (int l = L - 1; l >= 0; --l) {
        float* gW = P.g + kOffLayer0 + l * kLayerStride;
        colsum64(s, n, w.dH.p, w.part.p, w.hsum.p);
        k_gelu_back<<<grid_for((int64_t)nh), 256, 0, s>>>(n, w.dH.p, w.hsum.p, w.Z.p + l * nh, w.dZ.p, w.dZb.p);
        ::pc::count_launches(1);
        colsum64(s, n, w.dZ.p, w.part.p, gW + kH * 128);
        k_mpnn_dw<<<gdw, kThr, 49152, s>>>(n, w.X.p + (size_t)l * nh * 2, w.dZb.p, wpart.p, w.err.p);
        ::pc::count_launches(1);
        k_sum_parts<<<kH * 128, kSumThreads, 0, s>>>(gdw, kH * 128, wpart.p, gW); ::pc::count_launches(1);
        k_mpnn_dx<<<gdx, kThr, 32768, s>>>(n, w.dZb.p, P.wl + (size_t)l * kH * 128, w.dHs.p, w.dM.p, w.err.p);
        ::pc::count_launches(1);
        k_nbr_back<<<grid_for((int64_t)n * 32), 256, 0, s>>>(n, c.rowptr.p, c.col.p, w.aw.p, w.invD.p, w.dHs.p,
                                                            w.dM.p, w.dH.p);
        ::pc::count_launches(1);
    }
    // input head
    colsum64(s, n, w.dH.p, w.part.p, w.hsum.p);
    k_gelu_back<<<grid_for((int64_t)nh), 256, 0, s>>>(n, w.dH.p, w.hsum.p, w.Zin.p, w.dZ.p, nullptr);
    ::pc::count_launches(1);
    k_colsums<<<nb, 256, 0, s>>>(n, 2, w.dZ.p, nullptr, nullptr, nullptr, w.F.p, w.part.p, 256);
    ::pc::count_launches(1);
    k_sum_parts<<<256, kSumThreads, 0, s>>>(nb, 256, w.part.p, P.g + kOffWin); ::pc::count_launches(1);
    PC_LAUNCH("mpnn_backward");
    check_err(c, w.err.p);
    double L0 = 0.0;
    PC_CUDA(cudaMemcpyAsync(&L0, sl + 0, sizeof(double), cudaMemcpyDeviceToHost, s));
    sync(c);
    return L0 / (double)n;
}

void mpnn_adam(Mpnn& P, float lr) {
    P.t += 1;
    const float c1 = 1.0f - std::pow(0.9f, (float)P.t), c2 = 1.0f - std::pow(0.999f, (float)P.t);
    k_adam<<<grid_for(kMpnnParams), 256>>>(kMpnnParams, lr, c1, c2, P.g, P.w, P.m, P.v);
    ::pc::count_launches(1);
    mpnn_refresh(P);
    PC_CUDA(cudaDeviceSynchronize());
}

}  // namespace pc
