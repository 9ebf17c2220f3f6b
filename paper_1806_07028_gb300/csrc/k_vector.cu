// Vector kernels: deterministic reductions, axpy-type updates, precision casts,
// scans and the Philox4x64-10 generator (Salmon et al., SC'11).
#include "pcamg_internal.cuh"

namespace pc {

namespace {

constexpr int kRedBlock = 256;
constexpr int kRedMaxBlocks = 1024;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block sum in a fixed tree: warp shuffles, then warp 0 over the warp sums.
__device__ double block_sum(double v) {
    __shared__ double ws[32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? ws[threadIdx.x] : 0.0;
    if (wid == 0) v = warp_sum(v);
    __syncthreads();
    return v;  // valid in thread 0
}

// Per-block partial of sum x_i y_i (or sum x_i): four independent loads and
// fused multiply-adds per step (GB300's FP64 rate, not HBM, bounds these
// loops), accumulated in a fixed order.
template <bool HAS_Y>
__global__ void k_dot_partial(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                              double* __restrict__ partial) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    const int64_t st = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; i + 3 * st < n; i += 4 * st) {
        const double a0 = x[i], a1 = x[i + st], a2 = x[i + 2 * st], a3 = x[i + 3 * st];
        if constexpr (HAS_Y) {
            s0 = fma(a0, y[i], s0);
            s1 = fma(a1, y[i + st], s1);
            s2 = fma(a2, y[i + 2 * st], s2);
            s3 = fma(a3, y[i + 3 * st], s3);
        } else {
            s0 += a0; s1 += a1; s2 += a2; s3 += a3;
        }
    }
    for (; i < n; i += st) s0 = HAS_Y ? fma(x[i], y[i], s0) : s0 + x[i];
    double s = (s0 + s1) + (s2 + s3);
    s = block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_finish_sum(int nb, const double* __restrict__ partial, double* __restrict__ out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
    s = block_sum(s);
    if (threadIdx.x == 0) *out = s;
}

__global__ void k_axpy(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}

__global__ void k_axpy_dev(int64_t n, const double* __restrict__ a, double sign, const double* __restrict__ x,
                           double* __restrict__ y) {
    double aa = sign * (*a);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += aa * x[i];
}

__global__ void k_xpby_dev(int64_t n, const double* __restrict__ x, const double* __restrict__ beta,
                           double* __restrict__ y) {
    double b = *beta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = x[i] + b * y[i];
}

__global__ void k_sub_mean(int64_t n, double* __restrict__ x, const double* __restrict__ total) {
    double m = (*total) / (double)n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] -= m;
}

__global__ void k_scale_dev(int64_t n, double* __restrict__ x, const double* __restrict__ num,
                            const double* __restrict__ den) {
    double f = (num ? *num : 1.0) / (*den);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] *= f;
}

__global__ void k_copy(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = x[i];
}

__global__ void k_fill(int64_t n, double v, double* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = v;
}

__global__ void k_fill_i32(int64_t n, int32_t v, int32_t* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = v;
}

// Four elements per thread and step with 16-byte loads and stores when every
// pointer is 16-byte aligned (the remainder, or unaligned data, one at a time):
// more bytes in flight per thread on these pure streaming passes.
__global__ void k_cast_scaled_f32(int64_t n, const double* __restrict__ x, const double* __restrict__ inv,
                                  float* __restrict__ y) {
    double f = inv ? *inv : 1.0;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
    int64_t head = 0;
    if ((((uintptr_t)x | (uintptr_t)y) & 15) == 0) {
        head = n & ~(int64_t)3;
        for (int64_t q = t0; 4 * q < head; q += st) {
            const double2 a = reinterpret_cast<const double2*>(x)[2 * q];
            const double2 b = reinterpret_cast<const double2*>(x)[2 * q + 1];
            reinterpret_cast<float4*>(y)[q] = make_float4((float)(a.x * f), (float)(a.y * f),
                                                         (float)(b.x * f), (float)(b.y * f));
        }
    }
    for (int64_t i = head + t0; i < n; i += st) y[i] = (float)(x[i] * f);
}

__global__ void k_add_scaled_f32(int64_t n, const float* __restrict__ c, const double* __restrict__ sc,
                                 double* __restrict__ x) {
    double f = *sc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += f * (double)c[i];
}

// gathers through an index: y_t = x_idx(t) (scaled and rounded to float, or
// copied), for moving vectors between the row order and the finest level's
// colour order; the writes are coalesced
__global__ void k_gather_scaled_f32(int64_t n, const int* __restrict__ idx, const double* __restrict__ x,
                                    const double* __restrict__ inv, float* __restrict__ y) {
    const double f = inv ? *inv : 1.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)(x[__ldg(idx + i)] * f);
}

__global__ void k_gather_set_scaled_f32(int64_t n, const int* __restrict__ idx, const float* __restrict__ c,
                                        const double* __restrict__ sc, double* __restrict__ x) {
    const double f = *sc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = f * (double)c[__ldg(idx + i)];
}

template <class T>
__global__ void k_gather(int64_t n, const int* __restrict__ idx, const T* __restrict__ x, T* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = x[__ldg(idx + i)];
}

// inv[idx[t]] = t
__global__ void k_invert_perm(int n, const int* __restrict__ idx, int* __restrict__ inv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) inv[__ldg(idx + i)] = i;
}

// y[k] = map[x[k]] (indices renamed in place when y == x)
__global__ void k_map_index(int64_t n, const int* __restrict__ map, const int* x, int* y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = __ldg(map + x[i]);
}

__global__ void k_set_scaled_f32(int64_t n, const float* __restrict__ c, const double* __restrict__ sc,
                                 double* __restrict__ x) {
    double f = *sc;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
    int64_t head = 0;
    if ((((uintptr_t)x | (uintptr_t)c) & 15) == 0) {
        head = n & ~(int64_t)3;
        for (int64_t q = t0; 4 * q < head; q += st) {
            const float4 a = reinterpret_cast<const float4*>(c)[q];
            reinterpret_cast<double2*>(x)[2 * q] = make_double2(f * (double)a.x, f * (double)a.y);
            reinterpret_cast<double2*>(x)[2 * q + 1] = make_double2(f * (double)a.z, f * (double)a.w);
        }
    }
    for (int64_t i = head + t0; i < n; i += st) x[i] = f * (double)c[i];
}

__global__ void k_cast_f64(int64_t n, const float* __restrict__ x, double* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (double)x[i];
}

// Philox4x64-10 from its published definition: per round, words 0 and 2 are
// multiplied by two odd 64-bit constants; the high halves are xored with words
// 1 and 3 and the round key; the key advances by two Weyl increments.
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += W0; k1 += W1; }
        uint64_t lo0 = M0 * c[0], hi0 = __umul64hi(M0, c[0]);
        uint64_t lo1 = M1 * c[2], hi1 = __umul64hi(M1, c[2]);
        uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

__global__ void k_philox_uniform(uint64_t seed, int64_t n, double* __restrict__ out) {
    // one thread per block of four outputs
    int64_t nb = (n + 3) >> 2;
    for (int64_t blk = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; blk < nb; blk += (int64_t)gridDim.x * blockDim.x) {
        uint64_t c[4] = {(uint64_t)blk, 0, 0, 0};
        philox4x64_10(c, seed, 0);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            int64_t i = blk * 4 + w;
            if (i < n) out[i] = __dsub_rn(ldexp((double)(c[w] >> 11), -52), 1.0);
        }
    }
}

// Small scalar algebra on device slots so that Krylov steps need no host trip.
__global__ void k_scalar(int op, double* s, int a, int b, int c) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    switch (op) {
        case SOP_DIV: s[c] = (s[b] != 0.0) ? s[a] / s[b] : 0.0; break;
        case SOP_SQRT: s[c] = sqrt(s[a]); break;
        case SOP_INV_SQRT: s[c] = (s[a] > 0.0) ? 1.0 / sqrt(s[a]) : 0.0; break;
        case SOP_PCG_ALPHA: s[c] = (s[a] > 0.0 && s[b] > 0.0) ? s[a] / s[b] : 0.0; break;
        case SOP_NEG_DIV: s[c] = (s[b] != 0.0) ? -s[a] / s[b] : 0.0; break;
        case SOP_INV: s[c] = (s[a] != 0.0) ? 1.0 / s[a] : 0.0; break;
        default: break;
    }
}

// ---- scan: one pass over tiles of 1024 (256 threads x 4) -----------------
// Decoupled look-back (Merrill and Garland, "Single-pass Parallel Prefix Scan
// with Decoupled Look-back", 2016). Tiles take tickets in launch order; a tile
// publishes its sum, then its inclusive prefix once it has added up its
// predecessors' published words, nearest first, back to the first prefix. A
// state word holds the status in its top two bits (0 nothing yet, 1 sum, 2
// prefix) and a value below 2^62 (the scanned values are counts, never
// negative). The word itself carries the value, so relaxed loads and stores
// suffice. Predecessors took their tickets earlier and are running or done, so
// the wait ends; it is bounded all the same (about two seconds of SM clock),
// after which the tile sets ws[kScanErr] and leaves its outputs unwritten.
constexpr int kScanErr = 0, kScanTicket = 1, kScanTotal = 2, kScanHead = 3;
constexpr uint64_t kScanSum = 1ull << 62, kScanPrefix = 2ull << 62, kScanVal = (1ull << 62) - 1;

__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <class TI, class TO>
__global__ void __launch_bounds__(256) k_scan(int64_t n, const TI* __restrict__ in, TO* __restrict__ out,
                                              uint64_t* ws) {
    __shared__ int64_t wsum[8];
    __shared__ int64_t s_excl;
    __shared__ int64_t s_tile;
    __shared__ int s_ok;
    if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(ws + kScanTicket), 1ull);
    __syncthreads();
    const int64_t tile = s_tile;
    uint64_t* state = ws + kScanHead;
    const int64_t base = tile * 1024 + threadIdx.x * 4;
    int64_t v[4];
    int64_t t = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t i = base + k;
        v[k] = (i < n) ? (int64_t)in[i] : 0;
        t += v[k];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = t;   // inclusive warp scan of the thread sums
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const int64_t w = lane < 8 ? wsum[lane] : 0;
        int64_t wi = w;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        const int64_t agg = __shfl_sync(0xffffffffu, wi, 7);   // the tile's sum
        if (lane < 8) wsum[lane] = wi - w;                       // exclusive warp offsets
        int64_t excl = 0;
        bool ok = true;
        if (tile == 0) {
            if (lane == 0) st_relaxed(state, kScanPrefix | (uint64_t)agg);
        } else {
            if (lane == 0) st_relaxed(state + tile, kScanSum | (uint64_t)agg);
            const long long t0 = clock64();
            for (int64_t j = tile - 1;;) {   // window j, j-1, .., j-31
                const int64_t idx = j - lane;
                uint64_t word;
                for (;;) {   // both exits are warp-uniform
                    word = idx >= 0 ? ld_relaxed(state + idx) : kScanPrefix;
                    if (__all_sync(0xffffffffu, (word >> 62) != 0)) break;
                    if (__any_sync(0xffffffffu, clock64() - t0 > (1ll << 32))) { ok = false; break; }
                }
                if (!ok) break;
                const unsigned pre = __ballot_sync(0xffffffffu, (word >> 62) == 2);
                const int first = pre ? __ffs(pre) - 1 : 31;   // nearest prefix, or the whole window
                int64_t part = lane <= first ? (int64_t)(word & kScanVal) : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                excl += part;
                if (pre) break;
                j -= 32;
            }
            if (lane == 0) {
                if (ok) st_relaxed(state + tile, kScanPrefix | (uint64_t)(excl + agg));
                else atomicExch(reinterpret_cast<unsigned long long*>(ws + kScanErr), 1ull);
            }
        }
        if (lane == 0) {
            s_excl = excl;
            s_ok = ok ? 1 : 0;
            if (ok && (tile + 1) * 1024 >= n) {   // the last tile holds the total
                out[n] = (TO)(excl + agg);
                ws[kScanTotal] = (uint64_t)(excl + agg);
            }
        }
    }
    __syncthreads();
    if (!s_ok) return;
    int64_t run = s_excl + wsum[wid] + inc - t;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t i = base + k;
        if (i < n) out[i] = (TO)run;
        run += v[k];
    }
}

inline int grid_for(int64_t n, int per_block = kBlock) {
    int64_t g = (n + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > (int64_t)kNumSMs * 16) g = kNumSMs * 16;
    return (int)g;
}

}  // namespace

int reduce_blocks(int64_t n) {
    int64_t g = (n + 4 * kRedBlock - 1) / (4 * kRedBlock);
    if (g < 1) g = 1;
    if (g > kRedMaxBlocks) g = kRedMaxBlocks;
    return (int)g;
}

void dot(cudaStream_t s, int64_t n, const double* x, const double* y, double* partial, double* out) {
    int nb = reduce_blocks(n);
    if (y) k_dot_partial<true><<<nb, kRedBlock, 0, s>>>(n, x, y, partial);
    else k_dot_partial<false><<<nb, kRedBlock, 0, s>>>(n, x, nullptr, partial);
    ::pc::count_launches(1);
    k_finish_sum<<<1, 1024, 0, s>>>(nb, partial, out); ::pc::count_launches(1);
    PC_LAUNCH("dot");
}

void sum(cudaStream_t s, int64_t n, const double* x, double* partial, double* out) {
    dot(s, n, x, nullptr, partial, out);
}

void axpy(cudaStream_t s, int64_t n, double a, const double* x, double* y) {
    k_axpy<<<grid_for(n), kBlock, 0, s>>>(n, a, x, y); ::pc::count_launches(1);
    PC_LAUNCH("axpy");
}
void axpy_dev(cudaStream_t s, int64_t n, const double* a, double sign, const double* x, double* y) {
    k_axpy_dev<<<grid_for(n), kBlock, 0, s>>>(n, a, sign, x, y); ::pc::count_launches(1);
    PC_LAUNCH("axpy_dev");
}
void xpby_dev(cudaStream_t s, int64_t n, const double* x, const double* beta, double* y) {
    k_xpby_dev<<<grid_for(n), kBlock, 0, s>>>(n, x, beta, y); ::pc::count_launches(1);
    PC_LAUNCH("xpby_dev");
}
void sub_mean(cudaStream_t s, int64_t n, double* x, const double* total) {
    k_sub_mean<<<grid_for(n), kBlock, 0, s>>>(n, x, total); ::pc::count_launches(1);
    PC_LAUNCH("sub_mean");
}
void scale_dev(cudaStream_t s, int64_t n, double* x, const double* num, const double* den) {
    k_scale_dev<<<grid_for(n), kBlock, 0, s>>>(n, x, num, den); ::pc::count_launches(1);
    PC_LAUNCH("scale_dev");
}
void copy(cudaStream_t s, int64_t n, const double* x, double* y) {
    k_copy<<<grid_for(n), kBlock, 0, s>>>(n, x, y); ::pc::count_launches(1);
    PC_LAUNCH("copy");
}
void fill(cudaStream_t s, int64_t n, double v, double* y) {
    k_fill<<<grid_for(n), kBlock, 0, s>>>(n, v, y); ::pc::count_launches(1);
    PC_LAUNCH("fill");
}
void fill_i32(cudaStream_t s, int64_t n, int32_t v, int32_t* y) {
    k_fill_i32<<<grid_for(n), kBlock, 0, s>>>(n, v, y); ::pc::count_launches(1);
    PC_LAUNCH("fill_i32");
}
void cast_scaled_f32(cudaStream_t s, int64_t n, const double* x, const double* inv, float* y) {
    k_cast_scaled_f32<<<grid_for((n + 3) / 4), kBlock, 0, s>>>(n, x, inv, y); ::pc::count_launches(1);
    PC_LAUNCH("cast_scaled_f32");
}
void cast_f32(cudaStream_t s, int64_t n, const double* x, float* y) { cast_scaled_f32(s, n, x, nullptr, y); }
void add_scaled_f32(cudaStream_t s, int64_t n, const float* c, const double* scale, double* x) {
    k_add_scaled_f32<<<grid_for(n), kBlock, 0, s>>>(n, c, scale, x); ::pc::count_launches(1);
    PC_LAUNCH("add_scaled_f32");
}
void set_scaled_f32(cudaStream_t s, int64_t n, const float* c, const double* scale, double* x) {
    k_set_scaled_f32<<<grid_for((n + 3) / 4), kBlock, 0, s>>>(n, c, scale, x); ::pc::count_launches(1);
    PC_LAUNCH("set_scaled_f32");
}
void gather_scaled_f32(cudaStream_t s, int64_t n, const int32_t* idx, const double* x, const double* inv, float* y) {
    k_gather_scaled_f32<<<grid_for(n), kBlock, 0, s>>>(n, idx, x, inv, y); ::pc::count_launches(1);
    PC_LAUNCH("gather_scaled_f32");
}
void gather_set_scaled_f32(cudaStream_t s, int64_t n, const int32_t* idx, const float* c, const double* scale,
                           double* x) {
    k_gather_set_scaled_f32<<<grid_for(n), kBlock, 0, s>>>(n, idx, c, scale, x); ::pc::count_launches(1);
    PC_LAUNCH("gather_set_scaled_f32");
}
template <class T>
void gather(cudaStream_t s, int64_t n, const int32_t* idx, const T* x, T* y) {
    k_gather<T><<<grid_for(n), kBlock, 0, s>>>(n, idx, x, y); ::pc::count_launches(1);
    PC_LAUNCH("gather");
}
template void gather<double>(cudaStream_t, int64_t, const int32_t*, const double*, double*);
template void gather<float>(cudaStream_t, int64_t, const int32_t*, const float*, float*);
template void gather<int32_t>(cudaStream_t, int64_t, const int32_t*, const int32_t*, int32_t*);
void invert_perm(cudaStream_t s, int32_t n, const int32_t* idx, int32_t* inv) {
    k_invert_perm<<<grid_for(n), kBlock, 0, s>>>(n, idx, inv); ::pc::count_launches(1);
    PC_LAUNCH("invert_perm");
}
void map_index(cudaStream_t s, int64_t n, const int32_t* map, const int32_t* x, int32_t* y) {
    k_map_index<<<grid_for(n), kBlock, 0, s>>>(n, map, x, y); ::pc::count_launches(1);
    PC_LAUNCH("map_index");
}
void cast_f64(cudaStream_t s, int64_t n, const float* x, double* y) {
    k_cast_f64<<<grid_for(n), kBlock, 0, s>>>(n, x, y); ::pc::count_launches(1);
    PC_LAUNCH("cast_f64");
}
void philox_uniform(cudaStream_t s, uint64_t seed, int64_t n, double* out) {
    k_philox_uniform<<<grid_for((n + 3) / 4), kBlock, 0, s>>>(seed, n, out); ::pc::count_launches(1);
    PC_LAUNCH("philox_uniform");
}
void scalar_ops(cudaStream_t s, int op, double* slots, int a, int b, int c) {
    k_scalar<<<1, 32, 0, s>>>(op, slots, a, b, c); ::pc::count_launches(1);
    PC_LAUNCH("scalar_ops");
}

// Exclusive scan of non-negative counts; out[n] receives the total. The
// bookkeeping words live in the context: [err, ticket, total, tile states..];
// the error word persists, so a wait that gave up in a scan whose total is not
// read is reported by the next scan that reads one.
template <class TI, class TO>
static int64_t scan_impl(Ctx& c, const TI* in, TO* out, int64_t n, bool read_total = true) {
    const int64_t ntiles = std::max<int64_t>(1, (n + 1023) / 1024);
    const size_t words = (size_t)(kScanHead + ntiles);
    if (c.scan_ws.n < words) {
        DBuf<int64_t> grown;
        grown.alloc(c.mem, std::max(words, (size_t)4096));
        PC_CUDA(cudaMemsetAsync(grown.p, 0, sizeof(int64_t) * grown.n, c.stream));
        if (c.scan_ws.p)
            PC_CUDA(cudaMemcpyAsync(grown.p, c.scan_ws.p, sizeof(int64_t), cudaMemcpyDeviceToDevice, c.stream));
        c.scan_ws = std::move(grown);
    }
    PC_CUDA(cudaMemsetAsync(c.scan_ws.p + kScanTicket, 0, sizeof(int64_t) * (words - kScanTicket), c.stream));
    k_scan<TI, TO><<<(unsigned)ntiles, 256, 0, c.stream>>>(n, in, out, reinterpret_cast<uint64_t*>(c.scan_ws.p));
    ::pc::count_launches(1);
    PC_LAUNCH("scan");
    if (!read_total) return -1;
    int64_t h[kScanHead];
    d2h(c, h, c.scan_ws.p, kScanHead);
    if (h[kScanErr]) fail(PCAMG_ERR_CUDA, "scan: a look-back wait gave up");
    return h[kScanTotal];
}

int64_t scan_i32(Ctx& c, const int32_t* in, int32_t* out, int64_t n) {
    return scan_impl<int32_t, int32_t>(c, in, out, n);
}
void scan_i32_device(Ctx& c, const int32_t* in, int32_t* out, int64_t n) {
    scan_impl<int32_t, int32_t>(c, in, out, n, false);
}
int64_t scan_i64(Ctx& c, const int64_t* in, int64_t* out, int64_t n) {
    return scan_impl<int64_t, int64_t>(c, in, out, n);
}

}  // namespace pc
