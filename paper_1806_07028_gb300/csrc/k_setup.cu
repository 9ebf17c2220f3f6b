// Setup kernels of PathCoverAMG_setup (Alg. 4):
//  * row products: the A^2 pattern (Alg. 4 step 2) and the Galerkin products
//    P^T A P and B^T A~ B (Alg. 4 steps 7 and 9) share one engine that, for each
//    output row, enumerates contributions in a fixed order, merges equal column
//    keys by summing in that order, and writes the row sorted by column;
//  * the path cover (Alg. 1) as locally-dominant rounds over paths;
//  * list ranking of the paths, matching along them and leftover handling
//    (Alg. 3), aggregate numbering, members, P values and path shortening.
// Every integer result is deterministic and independent of thread scheduling.
#include <utility>
#include <algorithm>
#include <climits>
#include <type_traits>
#include <cstring>

#include "net24.cuh"
#include "pcamg_internal.cuh"

namespace pc {

namespace {

constexpr int kBlockCap = 2048;       // contributions a block-per-row product stages in smem
constexpr int kOrderWarpCap = 256;    // candidates a warp orders in shared memory
constexpr uint32_t kSkip = 0xffffffffu;

inline int grid1(int64_t n, int block = kBlock) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > (int64_t)kNumSMs * 32) g = kNumSMs * 32;
    return (int)g;
}

inline int grid_warps(int64_t rows) {
    int64_t g = (rows + 7) / 8;
    if (g < 1) g = 1;
    if (g > (int64_t)kNumSMs * 64) g = kNumSMs * 64;
    return (int)g;
}

#define FOR_EACH(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// ---------------------------------------------------------------- small sorting network
// The comparators of the 24-position network (net24.cuh) applied to two
// register arrays: the keys and what moves with them.

// (w descending, column ascending): the proposal order of a row's candidates
__device__ __forceinline__ bool order_before(uint64_t w1, int c1, uint64_t w2, int c2) {
    return (w1 > w2) || (w1 == w2 && c1 < c2);
}
// proposal order: weight bits and column move together
template <int a, int c>
__device__ __forceinline__ void net_cswap(uint64_t (&kw)[kNet24], int (&kc)[kNet24]) {
    const bool sw = order_before(kw[c], kc[c], kw[a], kc[a]);
    const uint64_t wa = kw[a], wc = kw[c];
    const int ca = kc[a], cc = kc[c];
    kw[a] = sw ? wc : wa; kw[c] = sw ? wa : wc;
    kc[a] = sw ? cc : ca; kc[c] = sw ? ca : cc;
}
// row products: ascending 32-bit keys, each with its value
template <int a, int c>
__device__ __forceinline__ void net_cswap(uint32_t (&key)[kNet24], double (&val)[kNet24]) {
    const bool sw = key[c] < key[a];
    const uint32_t ka = key[a], kc = key[c];
    const double va = val[a], vc = val[c];
    key[a] = sw ? kc : ka; key[c] = sw ? ka : kc;
    val[a] = sw ? vc : va; val[c] = sw ? va : vc;
}
template <class K, class V, int... Q>
__device__ __forceinline__ void net24_apply(K (&k)[kNet24], V (&v)[kNet24], std::integer_sequence<int, Q...>) {
    (net_cswap<net24(Q, true), net24(Q, false)>(k, v), ...);
}

// ---------------------------------------------------------------- row products
// Row u of the A^2 pattern: for j in row u of A (A holds its diagonal), for v in
// row j: key v, skipping v == u.
struct CandSrc {
    const int* __restrict__ rowptr;
    const int* __restrict__ col;
    __device__ int nmem(int r) const { return rowptr[r + 1] - rowptr[r]; }
    __device__ int mem_row(int r, int t) const { return col[rowptr[r] + t]; }
    __device__ int mbase(int r) const { return rowptr[r]; }
    __device__ int mem_at(int base, int t) const { return col[base + t]; }
    __device__ int in_beg(int j) const { return rowptr[j]; }
    __device__ int in_end(int j) const { return rowptr[j + 1]; }
    __device__ void kv(int r, int, int k, uint32_t& key, double& v) const {
        int c = col[k];
        key = (c == r) ? kSkip : (uint32_t)c;
        v = 0.0;
    }
};

// Row I of P^T A P: members u of aggregate I ascending, then row u of A in
// order; key agg(v), value (p_u a_uv) p_v (p = 1 when pval is null).
struct GalSrc {
    const int* __restrict__ agg_ptr;
    const int* __restrict__ mem;
    const int* __restrict__ rowptr;
    const int* __restrict__ col;
    const double* __restrict__ val;
    const double* __restrict__ pval;
    const int* __restrict__ agg;
    int drop_diag;
    __device__ int nmem(int r) const { return agg_ptr[r + 1] - agg_ptr[r]; }
    __device__ int mem_row(int r, int t) const { return mem[agg_ptr[r] + t]; }
    __device__ int mbase(int r) const { return agg_ptr[r]; }
    __device__ int mem_at(int base, int t) const { return mem[base + t]; }
    __device__ int in_beg(int u) const { return rowptr[u]; }
    __device__ int in_end(int u) const { return rowptr[u + 1]; }
    __device__ void kv(int r, int u, int k, uint32_t& key, double& v) const {
        int c = col[k];
        int J = agg[c];
        key = (drop_diag && J == r) ? kSkip : (uint32_t)J;
        v = pval ? __dmul_rn(__dmul_rn(pval[u], val[k]), pval[c]) : val[k];
    }
};

// Warp per row. The row's contributions are numbered e = 0..total-1 in their
// fixed order (member rows one after another), and every output entry is the
// sum of one column's contributions taken in that order. A row of more than
// 32 contributions whose columns all fit 24 bits is merged through a per-warp
// hash table keyed by column (twice as many slots as the padded contribution
// count): each round of 32 contributions groups equal columns (a warp match),
// the group's first lane adds the column with the group's size, the distinct
// columns are then sorted, each column's contributions are given consecutive
// positions in contribution order, and one lane per column adds them up.
// Shorter or wider rows sort (column, e) keys of all contributions instead
// (bitonic, padded to a power of two) and the first lane of each run of equal
// columns adds the run. Rows with more than kWarpMembers member rows or
// kWarpCap contributions are flagged for the block kernels. (A warp's scratch
// is 3.2 KB, so the block's eight warps fit eight times per SM; the rare
// longer rows take the block kernels.)
constexpr int kWarpCap = 128;
constexpr int kWarpMembers = 64;
constexpr int kWarpsPerBlock = 8;
constexpr int kHashSlots = 256;              // at most twice kWarpCap: never more than half full
constexpr uint32_t kHashEmpty = 0xffffffffu;
constexpr uint16_t kNoSlot = 0xffffu;
static_assert(kHashSlots == 2 * kWarpCap && kHashSlots == 256, "slot numbers are 8 bits");

struct MemberInfo {
    int pre[kWarpMembers + 1];   // prefix of the member rows' lengths
    int row[kWarpMembers];
    int beg[kWarpMembers];       // first input entry of each member row
};

struct alignas(16) WarpScratch {
    union {
        uint64_t key[kWarpCap];        // wide rows: the sorted keys
        uint32_t hash[kHashSlots];     // narrow rows: column << 8 | count, later a column's next position
    };
    double val[kWarpCap];              // value of contribution e
    union {
        MemberInfo m;                  // while the contributions are staged
        uint32_t dist[kWarpCap + 1];   // narrow rows, afterwards: distinct columns (column << 8 | slot),
                                       // then the columns' first merged positions
    };
    uint16_t slot[kWarpCap];           // narrow rows: table slot of contribution e (kNoSlot: skipped)
    uint8_t ord[kWarpCap];             // narrow rows: the contribution at each merged position
};

// Ascending bitonic sort of 32*R 64-bit keys held in registers: key i lives in
// lane i % 32, register i / 32. Partners closer than 32 positions are exchanged
// by warp shuffles, farther ones inside the thread.
template <int R>
__device__ __forceinline__ void sort_keys_regs(uint64_t (&key)[R], int lane) {
#pragma unroll
    for (int k = 2; k <= 32 * R; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int rp = r ^ (j >> 5);
                    if (rp > r) {
                        const bool up = ((lane + 32 * r) & k) == 0;
                        if ((key[r] > key[rp]) == up) { const uint64_t t = key[r]; key[r] = key[rp]; key[rp] = t; }
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint64_t pk = __shfl_xor_sync(0xffffffffu, key[r], j);
                    const bool up = ((lane + 32 * r) & k) == 0;
                    const bool lower = (lane & j) == 0;
                    // the lower position keeps the smaller key when up, the larger when down
                    const bool take = (lower == up) ? (pk < key[r]) : (pk > key[r]);
                    if (take) key[r] = pk;
                }
            }
        }
    }
}

// The same network on 32-bit keys (one shuffle and one integer compare per
// exchange instead of two and a 64-bit compare).
template <int R>
__device__ __forceinline__ void sort_keys_regs32(uint32_t (&key)[R], int lane) {
#pragma unroll
    for (int k = 2; k <= 32 * R; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int rp = r ^ (j >> 5);
                    if (rp > r) {
                        const bool up = ((lane + 32 * r) & k) == 0;
                        if ((key[r] > key[rp]) == up) { const uint32_t t = key[r]; key[r] = key[rp]; key[rp] = t; }
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint32_t pk = __shfl_xor_sync(0xffffffffu, key[r], j);
                    const bool up = ((lane + 32 * r) & k) == 0;
                    const bool lower = (lane & j) == 0;
                    const bool take = (lower == up) ? (pk < key[r]) : (pk > key[r]);
                    if (take) key[r] = pk;
                }
            }
        }
    }
}

// Contribution e of the row (e < total): its column key (kSkip when dropped)
// and value, from the member row t with pre[t] <= e < pre[t + 1].
template <class Src>
__device__ __forceinline__ void contribution(int r, int nm, int e, const Src& src, const WarpScratch& W,
                                             uint32_t& kk, double& v) {
    int lo = 0, hi = nm - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (W.m.pre[mid] <= e) lo = mid; else hi = mid - 1;
    }
    const int j = W.m.row[lo];
    const int k = W.m.beg[lo] + (e - W.m.pre[lo]);
    src.kv(r, j, k, kk, v);
}

// Stage the contributions as keys (column, e) in registers and values in
// W.val[e], sort the keys and store them in W.key as (column << 32 | e) in
// sorted order. Keys of skipped contributions and of the padding are ~0 and
// sort last. NARROW (every column below 2^24, at most 32 contributions) packs
// a key into 32 bits, column << 8 | e; the order is the same.
template <int R, bool NARROW, class Src>
__device__ __forceinline__ void stage_sort_keys(int lane, int r, int nm, int total, const Src& src,
                                                WarpScratch& W) {
    using K = typename std::conditional<NARROW, uint32_t, uint64_t>::type;
    constexpr K kPad = NARROW ? (K)0xffffffffu : (K)~0ull;
    K key[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int e = lane + 32 * q;
        key[q] = kPad;
        double v = 0.0;
        if (e < total) {
            uint32_t kk;
            contribution(r, nm, e, src, W, kk, v);
            if (kk != kSkip) key[q] = NARROW ? (K)((kk << 8) | (uint32_t)e) : (K)(((uint64_t)kk << 32) | (uint64_t)e);
        }
        W.val[e] = v;
    }
    if constexpr (NARROW) {
        sort_keys_regs32<R>(key, lane);
#pragma unroll
        for (int q = 0; q < R; ++q)
            W.key[lane + 32 * q] = (key[q] == kPad) ? ~0ull
                                                    : (((uint64_t)(key[q] >> 8) << 32) | (uint64_t)(key[q] & 255u));
    } else {
        sort_keys_regs<R>(key, lane);
#pragma unroll
        for (int q = 0; q < R; ++q) W.key[lane + 32 * q] = key[q];
    }
}

// Narrow rows (every column below 2^24), first half: stage the contributions
// (values in W.val[e]) and count each column's contributions in the hash
// table, W.hash[slot] = column << 8 | count (a count is at most kWarpCap, so it
// never reaches the column bits). Lanes of one round with the same column form
// one group; the group's first lane adds the column with the group's size, so
// the table takes one atomic per distinct column and round. Returns the number
// of distinct columns D, listed unsorted in W.dist[0..D) as column << 8 | slot,
// and leaves each contribution's slot in W.slot[e].
template <class Src>
__device__ __forceinline__ int hash_stage(int lane, int r, int nm, int total, int hbits, const Src& src,
                                          WarpScratch& W) {
    const int nslots = 1 << hbits;   // twice the padded contribution count, 128 or 256
    uint4* h4 = reinterpret_cast<uint4*>(W.hash);
    const uint4 empty = make_uint4(kHashEmpty, kHashEmpty, kHashEmpty, kHashEmpty);
    for (int t = lane; t < nslots / 4; t += 32) h4[t] = empty;
    __syncwarp();
    for (int e0 = 0; e0 < total; e0 += 32) {
        const int e = e0 + lane;
        uint32_t kk = kSkip;
        if (e < total) {
            double v;
            contribution(r, nm, e, src, W, kk, v);
            W.val[e] = v;
        }
        const unsigned grp = __match_any_sync(0xffffffffu, kk);
        const int lead = __ffs(grp) - 1;
        int sl = kNoSlot;
        if (kk != kSkip && lane == lead) {
            const uint32_t n = (uint32_t)__popc(grp);
            uint32_t h = (kk * 2654435761u) >> (32 - hbits);   // multiplicative hash
            // at most nslots / 2 columns: a free or matching slot is always
            // found within the bound
            for (int probe = 0; probe < nslots; ++probe, h = (h + 1) & (uint32_t)(nslots - 1)) {
                const uint32_t old = atomicCAS(&W.hash[h], kHashEmpty, (kk << 8) | n);
                if (old == kHashEmpty) { sl = (int)h; break; }
                if ((old >> 8) == kk) { atomicAdd(&W.hash[h], n); sl = (int)h; break; }
            }
        }
        sl = __shfl_sync(0xffffffffu, sl, lead);
        if (e < total) W.slot[e] = (kk != kSkip) ? (uint16_t)sl : kNoSlot;
        __syncwarp();
    }
    // the member lists are no longer read: W.dist takes their place
    int D = 0;
    for (int h = lane; h < nslots; h += 32) {
        const uint32_t w = W.hash[h];
        const bool used = w != kHashEmpty;
        const unsigned b = __ballot_sync(0xffffffffu, used);
        if (used) W.dist[D + __popc(b & ((1u << lane) - 1u))] = (w & 0xffffff00u) | (uint32_t)h;
        D += __popc(b);
    }
    __syncwarp();
    return D;
}

// Narrow rows, second half (D distinct columns, D <= 32 * R): sort the
// distinct columns, give column i the merged positions W.dist[i] ..
// W.dist[i + 1] - 1 (in column order), place each contribution at its
// column's next position, round by round and lane by lane, i.e. in
// contribution order, and let lane i add column i's values in that order.
// Writes the row's D entries at ocol/oval[o ..].
template <int R>
__device__ __forceinline__ void hash_emit(int lane, int total, int D, WarpScratch& W, int64_t o,
                                          int* __restrict__ ocol, double* __restrict__ oval) {
    uint32_t key[R];
#pragma unroll
    for (int q = 0; q < R; ++q) key[q] = (lane + 32 * q < D) ? W.dist[lane + 32 * q] : 0xffffffffu;
    sort_keys_regs32<R>(key, lane);
    __syncwarp();   // every lane has read W.dist: it now takes the columns' first positions
    int carry = 0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int i = lane + 32 * q;
        const uint32_t sl = key[q] & 255u;
        const int c = (i < D) ? (int)(W.hash[sl] & 255u) : 0;
        int inc = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += y;
        }
        __syncwarp();
        if (i < D) { W.hash[sl] = (uint32_t)(carry + inc - c); W.dist[i] = (uint32_t)(carry + inc - c); }
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) W.dist[D] = (uint32_t)carry;
    __syncwarp();
    for (int e0 = 0; e0 < total; e0 += 32) {
        const int e = e0 + lane;
        const uint32_t sl = (e < total) ? W.slot[e] : kNoSlot;
        const unsigned grp = __match_any_sync(0xffffffffu, sl);
        uint32_t base = 0;
        if (sl != kNoSlot) {
            base = W.hash[sl];
            W.ord[base + __popc(grp & ((1u << lane) - 1u))] = (uint8_t)e;
        }
        __syncwarp();
        if (sl != kNoSlot && lane == __ffs(grp) - 1) W.hash[sl] = base + (uint32_t)__popc(grp);
        __syncwarp();
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int i = lane + 32 * q;
        if (i < D) {
            const int b = (int)W.dist[i], en = (int)W.dist[i + 1];
            double sum = W.val[W.ord[b]];
            for (int t = b + 1; t < en; ++t) sum = __dadd_rn(sum, W.val[W.ord[t]]);
            ocol[o + i] = (int)(key[q] >> 8);
            if (oval) oval[o + i] = sum;
        }
    }
}

// Rows of at most kThreadProdCap contributions from at most kThreadProdCap
// member rows (every coarse row of P^T A P at a 3D 7-point grid's finest level:
// two or three members of seven entries), a thread per row, into the one-pass
// layout at tptr[r] (count in cnt, long flag cleared); every other row is
// listed in wrows for the warp kernel. Columns must fit 24 bits (nrows <= 2^24). The contributions are numbered in their
// fixed order (member rows one after another, each in CSR order) and keyed
// column << 8 | e (columns below 2^24), sorted with their values by the
// 24-position network, and each run of equal columns is added up in order:
// the warp kernel's sums, bit for bit.
constexpr int kThreadProdCap = kNet24;
constexpr int64_t kThreadProdMean = 20;   // largest mean contributions per row for the thread kernel
template <class Src>
__global__ void __launch_bounds__(kBlock) k_rowprod_thread(int nrows, Src src, int* __restrict__ cnt,
                                                           unsigned char* __restrict__ is_long,
                                                           int* __restrict__ ocol, double* __restrict__ oval,
                                                           const int64_t* __restrict__ tptr,
                                                           int* __restrict__ wrows, int* __restrict__ wcount) {
    constexpr uint32_t kPad = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;   // a multiple of 32: w0 is warp-uniform
    for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; w0 < nrows; w0 += stride) {
        const int64_t r64 = w0 + lane;
        bool mine = false;
        int r = 0, base = 0, nm = 0, total = 0;
        if (r64 < nrows) {
            r = (int)r64;
            base = src.mbase(r);
            nm = src.nmem(r);
            if (nm <= kThreadProdCap) {
                for (int t = 0; t < nm && total <= kThreadProdCap; ++t) {
                    const int j = src.mem_at(base, t);
                    total += src.in_end(j) - src.in_beg(j);
                }
                mine = total <= kThreadProdCap;
            }
        }
        // the other rows are listed for the warp kernel (one atomic per warp)
        const unsigned other = __ballot_sync(0xffffffffu, r64 < nrows && !mine);
        if (other) {
            int b = 0;
            if (lane == 0) b = atomicAdd(wcount, __popc(other));
            b = __shfl_sync(0xffffffffu, b, 0);
            if ((other >> lane) & 1u) wrows[b + __popc(other & ((1u << lane) - 1u))] = r;
        }
        if (!mine) continue;
        uint32_t key[kNet24];
        double val[kNet24];
        int t = -1, k = 0, kend = 0, j = 0;
#pragma unroll
        for (int e = 0; e < kNet24; ++e) {
            key[e] = kPad;
            val[e] = 0.0;
            if (e < total) {
                while (k == kend) {   // the next member row with entries left (e < total: one exists)
                    ++t;
                    j = src.mem_at(base, t);
                    k = src.in_beg(j);
                    kend = src.in_end(j);
                }
                uint32_t kk;
                double v;
                src.kv(r, j, k, kk, v);
                ++k;
                if (kk != kSkip) { key[e] = (kk << 8) | (uint32_t)e; val[e] = v; }
            }
        }
        net24_apply(key, val, std::make_integer_sequence<int, kNet24Size>{});
        const int64_t o = tptr[r];
        int D = 0;
        uint32_t cur = kPad;
        double sum = 0.0;
#pragma unroll
        for (int e = 0; e < kNet24; ++e) {
            if (key[e] != kPad) {
                const uint32_t c = key[e] >> 8;
                if (c != cur) {
                    if (cur != kPad) {
                        ocol[o + D] = (int)cur;
                        if (oval) oval[o + D] = sum;
                        ++D;
                    }
                    cur = c;
                    sum = val[e];
                } else {
                    sum = __dadd_rn(sum, val[e]);
                }
            }
        }
        if (cur != kPad) {
            ocol[o + D] = (int)cur;
            if (oval) oval[o + D] = sum;
            ++D;
        }
        cnt[r] = D;
        is_long[r] = 0;
    }
}

// MODE 0: count the row's distinct columns (cnt) and flag long rows;
// MODE 1: write the row at optr[r] (counts known);
// MODE 2: both at once -- count, flag, and write the row at tptr[r] of a
//         temporary layout sized by each row's contribution count (compacted
//         afterwards), so the sort-reduce runs once.
// (eight blocks of eight warps per SM: a row's merge is a long chain of
// dependent shuffles, shared-memory atomics and compares, so resident warps
// are what hides it)
template <class Src, int MODE>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 8) k_rowprod_warp(
        int nrows, Src src, int* __restrict__ cnt, unsigned char* __restrict__ is_long,
        int* __restrict__ long_list, int* __restrict__ long_count, const int* __restrict__ optr,
        int* __restrict__ ocol, double* __restrict__ oval, const int64_t* __restrict__ tptr,
        const int* __restrict__ rows = nullptr, const int* __restrict__ rcount = nullptr) {
    constexpr bool FILL = MODE != 0;
    constexpr bool COUNT = MODE != 1;
    __shared__ WarpScratch ws_all[kWarpsPerBlock];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    WarpScratch& W = ws_all[wib];
    const bool narrow = nrows <= (1 << 24);   // every column fits 24 bits
    const int64_t gw = (int64_t)blockIdx.x * kWarpsPerBlock + wib;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerBlock;
    // Software pipeline over the warp's rows r, r + nw, r + 2 nw, ...: each
    // step issues the member range of the row three steps ahead, the member
    // rows of the row two steps ahead and the entry ranges of the next row's
    // member rows (lane t: member t < 32), each from data that arrived a step
    // earlier, so a row's member data are in registers when its turn comes.
    struct Stage {
        int base = 0, nm = 0, mr = 0, mb = 0, len = 0;
    };
    auto s1 = [&](int64_t rr, Stage& q) {
        q = Stage();
        if (rr < nrows) { q.base = src.mbase((int)rr); q.nm = src.nmem((int)rr); }
    };
    auto s2 = [&](Stage& q) { if (lane < q.nm && lane < 32) q.mr = src.mem_at(q.base, lane); };
    auto s3 = [&](Stage& q) {
        if (lane < q.nm && lane < 32) { q.mb = src.in_beg(q.mr); q.len = src.in_end(q.mr) - q.mb; }
    };
    // the rows: all of them, or those listed (rows[0 .. *rcount))
    const int64_t m = rows ? (int64_t)*rcount : (int64_t)nrows;
    auto row_at = [&](int64_t q) -> int64_t { return q < m ? (rows ? (int64_t)rows[q] : q) : (int64_t)nrows; };
    Stage p1, p2, p3;
    s1(row_at(gw), p3); s2(p3); s3(p3);
    s1(row_at(gw + nw), p2); s2(p2);
    s1(row_at(gw + 2 * nw), p1);
    for (int64_t q64 = gw; q64 < m; q64 += nw) {
        const int r = (int)row_at(q64);
        const Stage cur = p3;
        p3 = p2; s3(p3);
        p2 = p1; s2(p2);
        s1(row_at(q64 + 3 * nw), p1);
        if (MODE == 1 && is_long[r]) continue;
        const int nm = cur.nm;
        bool over = nm > kWarpMembers;
        int total = 0;
        if (!over) {
            // member rows and the prefix of their lengths
            const int len = cur.len, mr = cur.mr, mb = cur.mb;
            int inc = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            total = __shfl_sync(0xffffffffu, inc, 31);
            if (lane < nm) { W.m.pre[lane + 1] = inc; W.m.row[lane] = mr; W.m.beg[lane] = mb; }
            if (nm > 32) {
                int len2 = 0, mr2 = 0, mb2 = 0;
                if (lane + 32 < nm) { mr2 = src.mem_at(cur.base, lane + 32); mb2 = src.in_beg(mr2); len2 = src.in_end(mr2) - mb2; }
                int inc2 = len2;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int y = __shfl_up_sync(0xffffffffu, inc2, o);
                    if (lane >= o) inc2 += y;
                }
                if (lane + 32 < nm) { W.m.pre[lane + 33] = total + inc2; W.m.row[lane + 32] = mr2; W.m.beg[lane + 32] = mb2; }
                total += __shfl_sync(0xffffffffu, inc2, 31);
            }
            if (lane == 0) W.m.pre[0] = 0;
            over = total > kWarpCap;
        }
        if (!over && narrow && total > 32) {
            // columns of a square product are row numbers, below nrows
            __syncwarp();
            const int64_t o = (MODE == 1) ? (int64_t)optr[r] : (MODE == 2 ? tptr[r] : 0);
            const int D = hash_stage(lane, r, nm, total, total > 64 ? 8 : 7, src, W);
            if (FILL && D > 0) {
                if (D <= 32) hash_emit<1>(lane, total, D, W, o, ocol, oval);
                else if (D <= 64) hash_emit<2>(lane, total, D, W, o, ocol, oval);
                else hash_emit<4>(lane, total, D, W, o, ocol, oval);
            }
            if (COUNT && lane == 0) { cnt[r] = D; is_long[r] = 0; }
        } else if (!over) {
            __syncwarp();
            int P = 32;
            while (P < total) P <<= 1;
            if (narrow && P == 32) stage_sort_keys<1, true>(lane, r, nm, total, src, W);
            else if (P == 32) stage_sort_keys<1, false>(lane, r, nm, total, src, W);
            else if (P == 64) stage_sort_keys<2, false>(lane, r, nm, total, src, W);
            else stage_sort_keys<4, false>(lane, r, nm, total, src, W);
            __syncwarp();
            // runs of equal columns
            int carry = 0;
            const int64_t o = (MODE == 1) ? (int64_t)optr[r] : (MODE == 2 ? tptr[r] : 0);
            for (int e0 = 0; e0 < P; e0 += 32) {
                const int e = e0 + lane;
                const uint64_t ke = W.key[e];
                const bool start = ke != ~0ull && (e == 0 || (W.key[e - 1] >> 32) != (ke >> 32));
                const unsigned ball = __ballot_sync(0xffffffffu, start);
                if (FILL && start) {
                    const uint32_t c = (uint32_t)(ke >> 32);
                    double sum = W.val[(uint32_t)ke];
                    for (int q = e + 1; q < P; ++q) {
                        const uint64_t kq = W.key[q];
                        if (kq == ~0ull || (uint32_t)(kq >> 32) != c) break;
                        sum = __dadd_rn(sum, W.val[(uint32_t)kq]);
                    }
                    const int64_t idx = o + carry + __popc(ball & ((1u << lane) - 1u));
                    ocol[idx] = (int)c;
                    if (oval) oval[idx] = sum;
                }
                carry += __popc(ball);
            }
            if (COUNT && lane == 0) { cnt[r] = carry; is_long[r] = 0; }
        }
        if (over && COUNT && lane == 0) {
            is_long[r] = 1;
            cnt[r] = 0;
            long_list[atomicAdd(long_count, 1)] = r;
        }
        __syncwarp();
    }
}

// Contribution count of every row a one-pass kernel takes (the warp kernel,
// or the shared-memory block kernel up to kBlockCap contributions; 0 for the
// larger rows): the temporary layout of the one-pass product.
template <class Src>
__global__ void k_rowprod_ubrow(int nrows, Src src, int64_t* __restrict__ ub) {
    FOR_EACH(r64, nrows) {
        const int r = (int)r64;
        const int nm = src.nmem(r);
        int64_t s = 0;
        for (int t = 0; t < nm && s <= kBlockCap; ++t) {
            const int j = src.mem_row(r, t);
            s += src.in_end(j) - src.in_beg(j);
        }
        ub[r] = (s <= kBlockCap) ? s : 0;
    }
}

// Copy the rows written in the temporary layout to their final place. A warp
// takes 32 consecutive rows: their counts and offsets are one coalesced load
// per lane, then the rows' first 32 entries are copied eight rows at a time
// (loads of the eight issued before their stores), longer rows' remainders
// after them.
__global__ void k_rowprod_compact(int nrows, const unsigned char* __restrict__ is_long, const int* __restrict__ cnt,
                                  const int64_t* __restrict__ tptr, const int* __restrict__ tcol,
                                  const double* __restrict__ tval, const int* __restrict__ optr,
                                  int* __restrict__ ocol, double* __restrict__ oval) {
    constexpr int kGroup = 8;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r0 = w0 * 32; r0 < nrows; r0 += nw * 32) {
        const int64_t r = r0 + lane;
        int m = 0, o = 0;
        int64_t t = 0;
        if (r < nrows && !is_long[r]) { m = cnt[r]; t = tptr[r]; o = optr[r]; }
        for (int j0 = 0; j0 < 32; j0 += kGroup) {
            int cv[kGroup];
            double vv[kGroup];
            int mj[kGroup], oj[kGroup];
#pragma unroll
            for (int u = 0; u < kGroup; ++u) {
                mj[u] = __shfl_sync(0xffffffffu, m, j0 + u);
                oj[u] = __shfl_sync(0xffffffffu, o, j0 + u);
                const int64_t tj = __shfl_sync(0xffffffffu, t, j0 + u);
                const bool on = lane < mj[u];
                cv[u] = on ? tcol[tj + lane] : 0;
                vv[u] = (on && oval) ? tval[tj + lane] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < kGroup; ++u) {
                if (lane < mj[u]) {
                    ocol[oj[u] + lane] = cv[u];
                    if (oval) oval[oj[u] + lane] = vv[u];
                }
            }
        }
        // entries beyond the first 32 of long rows
        unsigned longer = __ballot_sync(0xffffffffu, m > 32);
        while (longer) {
            const int j = __ffs(longer) - 1;
            longer &= longer - 1;
            const int mj = __shfl_sync(0xffffffffu, m, j);
            const int oj = __shfl_sync(0xffffffffu, o, j);
            const int64_t tj = __shfl_sync(0xffffffffu, t, j);
            for (int q = 32 + lane; q < mj; q += 32) {
                ocol[oj + q] = tcol[tj + q];
                if (oval) oval[oj + q] = tval[tj + q];
            }
        }
    }
}

// Split the rows the warp kernel left: up to kBlockCap contributions to the
// shared-memory block kernel (list B), larger to the global-memory one (list
// C, with their contribution counts). A row's result does not depend on the
// order of the lists.
template <class Src>
__global__ void k_rowprod_split(int nlong, const int* __restrict__ rows, Src src, int* __restrict__ listB,
                                int* __restrict__ listC, int64_t* __restrict__ ubC, int* __restrict__ counts) {
    FOR_EACH(i, nlong) {
        const int r = rows[i];
        int64_t s = 0;
        const int nm = src.nmem(r);
        for (int t = 0; t < nm; ++t) {
            const int j = src.mem_row(r, t);
            s += src.in_end(j) - src.in_beg(j);
        }
        if (s <= kBlockCap) {
            listB[atomicAdd(&counts[0], 1)] = r;
        } else {
            const int k = atomicAdd(&counts[1], 1);
            listC[k] = r;
            ubC[k] = s;
        }
    }
}

template <class Src>
__global__ void k_rowprod_ub(int nlong, const int* __restrict__ rows, Src src, int64_t* __restrict__ ub) {
    FOR_EACH(i, nlong) {
        int r = rows[i];
        int64_t s = 0;
        int nm = src.nmem(r);
        for (int t = 0; t < nm; ++t) {
            int j = src.mem_row(r, t);
            s += src.in_end(j) - src.in_beg(j);
        }
        ub[i] = s;
    }
}

__device__ __forceinline__ int64_t next_pow2(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Ascending bitonic sort of P (power of two) 64-bit keys by one block.
__device__ void block_bitonic_u64(uint64_t* keys, int64_t P) {
    for (int64_t k = 2; k <= P; k <<= 1) {
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
                int64_t ixj = i ^ j;
                if (ixj > i) {
                    uint64_t a = keys[i], b = keys[ixj];
                    bool up = (i & k) == 0;
                    if ((a > b) == up) { keys[i] = b; keys[ixj] = a; }
                }
            }
            __syncthreads();
        }
    }
}

// Block-wide exclusive scan of 0/1 flags given per thread in chunks; returns
// the prefix for this thread's item and the chunk total.
__device__ int block_excl_scan(int flag, int* total) {
    __shared__ int ws[32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = flag;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) ws[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        int w = lane < nw ? ws[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) ws[lane] = wi - w;
        if (lane == nw - 1) ws[31] = wi;
    }
    __syncthreads();
    int res = ws[wid] + inc - flag;
    *total = ws[31];
    __syncthreads();
    return res;
}

// Block per long row: stage (key << 32 | seq) and values by sequence number,
// sort, then each run of equal keys is summed in sequence order.
// MODE as for the warp kernel: 0 count, 1 fill at optr[r], 2 count and write
// at tptr[r] of the temporary layout (clearing the row's long flag).
template <class Src, int MODE, bool GLOBAL>
__global__ void k_rowprod_block(const int* __restrict__ rows, Src src, int* __restrict__ cnt,
                                const int* __restrict__ optr, int* __restrict__ ocol,
                                double* __restrict__ oval, uint64_t* __restrict__ gkeys,
                                double* __restrict__ gvals, const int64_t* __restrict__ goff,
                                const int64_t* __restrict__ tptr, unsigned char* __restrict__ is_long) {
    constexpr bool FILL = MODE != 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int r = rows[blockIdx.x];
    uint64_t* keys;
    double* vals;
    if (GLOBAL) {
        keys = gkeys + goff[blockIdx.x];
        vals = gvals + goff[blockIdx.x];
    } else {
        keys = reinterpret_cast<uint64_t*>(smem_raw);
        vals = reinterpret_cast<double*>(smem_raw + sizeof(uint64_t) * kBlockCap);
    }
    int64_t base = 0;
    int nm = src.nmem(r);
    for (int t = 0; t < nm; ++t) {
        int j = src.mem_row(r, t);
        int b = src.in_beg(j), e = src.in_end(j);
        for (int k = b + threadIdx.x; k < e; k += blockDim.x) {
            uint32_t key;
            double v;
            src.kv(r, j, k, key, v);
            int64_t seq = base + (k - b);
            keys[seq] = (key == kSkip) ? ~0ull : (((uint64_t)key << 32) | (uint64_t)seq);
            vals[seq] = v;
        }
        base += e - b;
    }
    int64_t P = next_pow2(base);
    for (int64_t i = base + threadIdx.x; i < P; i += blockDim.x) keys[i] = ~0ull;
    __syncthreads();
    block_bitonic_u64(keys, P);
    // run starts
    int carry = 0;
    for (int64_t c0 = 0; c0 < base; c0 += blockDim.x) {
        int64_t p = c0 + threadIdx.x;
        int flag = 0;
        if (p < base) {
            uint64_t kp = keys[p];
            flag = (kp != ~0ull) && (p == 0 || (keys[p - 1] >> 32) != (kp >> 32));
        }
        int tot;
        int pre = block_excl_scan(flag, &tot);
        if (FILL && flag) {
            uint64_t kp = keys[p];
            uint32_t kk = (uint32_t)(kp >> 32);
            double s = vals[(uint32_t)kp];
            for (int64_t q = p + 1; q < base; ++q) {
                uint64_t kq = keys[q];
                if ((uint32_t)(kq >> 32) != kk || kq == ~0ull) break;
                s = __dadd_rn(s, vals[(uint32_t)kq]);
            }
            const int64_t o = (MODE == 1 ? (int64_t)optr[r] : tptr[r]) + carry + pre;
            ocol[o] = (int)kk;
            if (oval) oval[o] = s;
        }
        carry += tot;
    }
    if (MODE != 1 && threadIdx.x == 0) cnt[r] = carry;
    if (MODE == 2 && threadIdx.x == 0) is_long[r] = 0;
}

// ---------------------------------------------------------------- weights
__global__ void k_maxabs(int64_t n, const double* __restrict__ x, double* __restrict__ out) {
    __shared__ double ws[32];
    double m = 0.0;
    FOR_EACH(i, n) m = fmax(m, fabs(x[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) out[blockIdx.x] = v;
    }
}

__global__ void k_delta(int nb, const double* __restrict__ part, double* __restrict__ delta) {
    double m = 0.0;
    for (int i = 0; i < nb; ++i) m = fmax(m, part[i]);
    double d = ldexp(m, -52);
    *delta = (d == 0.0) ? 1.0 : d;
}

// w_uv = 1 / max(|e_u - e_v|, delta)  (Alg. 4 step 2 with the tie cap)
__global__ void k_weights(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                          const double* __restrict__ e, const double* __restrict__ delta,
                          double* __restrict__ w) {
    double dl = *delta;
    FOR_EACH(u64, n) {
        int u = (int)u64;
        double eu = e[u];
        for (int k = ptr[u]; k < ptr[u + 1]; ++k) {
            double d = fabs(__dsub_rn(eu, e[col[k]]));
            if (d < dl) d = dl;
            w[k] = __ddiv_rn(1.0, d);
        }
    }
}

// ---------------------------------------------------------------- edge order
// Edge (a,b,w) before (c,d,x): heavier first, then smaller min id, then smaller max id.
__device__ __forceinline__ bool edge_before(double w1, int a1, int b1, double w2, int a2, int b2) {
    if (w1 != w2) return w1 > w2;
    int lo1 = min(a1, b1), lo2 = min(a2, b2);
    if (lo1 != lo2) return lo1 < lo2;
    return max(a1, b1) < max(a2, b2);
}

// Each row re-ordered by (w desc, column asc): the order in which a vertex
// proposes its edges.
// Class of every row for the proposal ordering: 0 = up to kOrderThreadCap
// candidates, sorted by one thread; 1 = up to kOrderWarpCap, sorted by a warp;
// 2 = longer, listed for a block each.
constexpr int kOrderThreadCap = kNet24;   // every interior row of a 3D 7-point grid's A^2 pattern
// Class-1 rows are listed (in no particular order: each is sorted on its own)
// for the warp kernel, one atomic per warp; class-2 rows for the block kernel.
__global__ void k_order_rows_classify(int n, const int* __restrict__ ptr, unsigned char* __restrict__ cls,
                                      int* __restrict__ mid_list, int* __restrict__ mid_count,
                                      int* __restrict__ long_list, int* __restrict__ long_count) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;   // a multiple of 32: w0 is warp-uniform
    for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; w0 < n; w0 += stride) {
        const int64_t u64 = w0 + lane;
        bool mid = false;
        if (u64 < n) {
            const int u = (int)u64;
            const int len = ptr[u + 1] - ptr[u];
            const bool big = len > kOrderWarpCap;
            mid = !big && len > kOrderThreadCap;
            cls[u] = big ? 2 : (mid ? 1 : 0);
            if (big) long_list[atomicAdd(long_count, 1)] = u;
        }
        const unsigned m = __ballot_sync(0xffffffffu, mid);
        if (m) {
            int b = 0;
            if (lane == 0) b = atomicAdd(mid_count, __popc(m));
            b = __shfl_sync(0xffffffffu, b, 0);
            if (mid) mid_list[b + __popc(m & ((1u << lane) - 1u))] = (int)u64;
        }
    }
}

// Warp per row for rows of up to kOrderWarpCap entries (class 1), sorted in
// the order (w descending, column ascending) by a bitonic network held in
// registers: element i of the padded row lives in lane i % 32, register i / 32;
// partners closer than 32 positions are exchanged by warp shuffles, farther
// ones inside the thread. Weights are positive, so their IEEE bit patterns
// compare as unsigned integers exactly as the doubles do; the sort compares
// bits on the integer pipe (GB300's FP64 pipe issues a comparison at a small
// fraction of the integer rate). Padding entries (bits 0, column INT_MAX) sort
// last. Columns are distinct within a row, so the order is strict and the
// result unique (order_before).

// Thread per row for rows of up to kOrderThreadCap entries (class 0), sorted
// by the 24-position network in registers (every comparator puts the element
// that comes first, order_before, at its lower position; padding entries come
// last). A row's loads are all issued before the network starts; neighbouring
// threads hold neighbouring rows, so a warp's loads and stores cover one
// contiguous stretch of the arrays.
__global__ void __launch_bounds__(kBlock)
    k_order_rows_thread(int n, const unsigned char* __restrict__ cls, const int* __restrict__ ptr,
                        const int* __restrict__ col, const double* __restrict__ w, int* __restrict__ scol,
                        double* __restrict__ sw) {
    FOR_EACH(u64, n) {
        const int u = (int)u64;
        if (cls[u] != 0) continue;
        const int b = ptr[u], len = ptr[u + 1] - b;
        uint64_t kw[kOrderThreadCap];
        int kc[kOrderThreadCap];
#pragma unroll
        for (int i = 0; i < kOrderThreadCap; ++i) {
            kw[i] = 0ull;
            kc[i] = INT_MAX;
            if (i < len) {
                kw[i] = (uint64_t)__double_as_longlong(__ldg(w + b + i));
                kc[i] = __ldg(col + b + i);
            }
        }
        net24_apply(kw, kc, std::make_integer_sequence<int, kNet24Size>{});
#pragma unroll
        for (int i = 0; i < kOrderThreadCap; ++i) {
            if (i < len) {
                scol[b + i] = kc[i];
                sw[b + i] = __longlong_as_double((long long)kw[i]);
            }
        }
    }
}

template <int R>
__device__ __forceinline__ void order_row_regs(int lane, int b, int len, const int* __restrict__ col,
                                               const double* __restrict__ w, int* __restrict__ scol,
                                               double* __restrict__ sw) {
    uint64_t kw[R];
    int kc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = lane + 32 * r;
        kw[r] = (i < len) ? (uint64_t)__double_as_longlong(w[b + i]) : 0ull;
        kc[r] = (i < len) ? col[b + i] : INT_MAX;
    }
#pragma unroll
    for (int k = 2; k <= 32 * R; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {   // partner in register r ^ (j / 32) of the same lane
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int rp = r ^ (j >> 5);
                    if (rp > r) {
                        const int i = lane + 32 * r;
                        const bool up = (i & k) == 0;
                        // ascending in "before" order when up: position r first
                        const bool swap = up ? order_before(kw[rp], kc[rp], kw[r], kc[r])
                                             : order_before(kw[r], kc[r], kw[rp], kc[rp]);
                        if (swap) {
                            const uint64_t tw = kw[r]; kw[r] = kw[rp]; kw[rp] = tw;
                            const int tc = kc[r]; kc[r] = kc[rp]; kc[rp] = tc;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint64_t pw = __shfl_xor_sync(0xffffffffu, kw[r], j);
                    const int pc = __shfl_xor_sync(0xffffffffu, kc[r], j);
                    const int i = lane + 32 * r;
                    const bool up = (i & k) == 0;
                    const bool lower = (lane & j) == 0;
                    const bool pb = order_before(pw, pc, kw[r], kc[r]);   // partner first?
                    const bool mb = order_before(kw[r], kc[r], pw, pc);   // me first?
                    // the lower position keeps the earlier element when up, the later when down
                    const bool take = (lower == up) ? pb : mb;
                    if (take) { kw[r] = pw; kc[r] = pc; }
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = lane + 32 * r;
        if (i < len) { scol[b + i] = kc[r]; sw[b + i] = __longlong_as_double((long long)kw[r]); }
    }
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_order_rows_warp(const int* __restrict__ rows, const int* __restrict__ count, const int* __restrict__ ptr,
                      const int* __restrict__ col, const double* __restrict__ w, int* __restrict__ scol,
                      double* __restrict__ sw) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int m = *count;
    for (int64_t i = (int64_t)blockIdx.x * kWarpsPerBlock + wib; i < m; i += (int64_t)gridDim.x * kWarpsPerBlock) {
        const int u = rows[i];
        const int b = ptr[u], len = ptr[u + 1] - b;
        if (len <= 1) {
            if (len == 1 && lane == 0) { scol[b] = col[b]; sw[b] = w[b]; }
        } else if (len <= 32) {
            order_row_regs<1>(lane, b, len, col, w, scol, sw);
        } else if (len <= 64) {
            order_row_regs<2>(lane, b, len, col, w, scol, sw);
        } else if (len <= 128) {
            order_row_regs<4>(lane, b, len, col, w, scol, sw);
        } else {
            order_row_regs<8>(lane, b, len, col, w, scol, sw);
        }
    }
}

__global__ void k_row_lengths(int m, const int* __restrict__ rows, const int* __restrict__ ptr, int* __restrict__ len) {
    FOR_EACH(i, m) len[i] = ptr[rows[i] + 1] - ptr[rows[i]];
}

__global__ void k_order_rows_block(const int* __restrict__ rows, const int* __restrict__ ptr,
                                   const int* __restrict__ col, const double* __restrict__ w,
                                   int* __restrict__ scol, double* __restrict__ sw,
                                   uint32_t* __restrict__ gidx, const int64_t* __restrict__ goff) {
    int u = rows[blockIdx.x];
    int b = ptr[u], len = ptr[u + 1] - b;
    uint32_t* idx = gidx + goff[blockIdx.x];
    int64_t P = next_pow2(len);
    for (int64_t i = threadIdx.x; i < P; i += blockDim.x) idx[i] = (i < len) ? (uint32_t)i : 0xffffffffu;
    __syncthreads();
    for (int64_t k = 2; k <= P; k <<= 1) {
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
                int64_t ixj = i ^ j;
                if (ixj > i) {
                    uint32_t a = idx[i], c2 = idx[ixj];
                    // "a after c2" in the (w desc, col asc) order; sentinels last
                    bool a_gt;
                    if (a == 0xffffffffu) a_gt = (c2 != 0xffffffffu);
                    else if (c2 == 0xffffffffu) a_gt = false;
                    else {
                        double wa = w[b + a], wc = w[b + c2];
                        a_gt = (wa < wc) || (wa == wc && col[b + a] > col[b + c2]);
                    }
                    bool up = (i & k) == 0;
                    if (a_gt == up) { idx[i] = c2; idx[ixj] = a; }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        scol[b + i] = col[b + idx[i]];
        sw[b + i] = w[b + idx[i]];
    }
}

// ---------------------------------------------------------------- path cover rounds
__global__ void k_cover_init(int n, const int* __restrict__ ptr, int* deg, int* oe, int* cptr,
                             int* nbr0, int* nbr1) {
    FOR_EACH(u, n) {
        deg[u] = 0; oe[u] = (int)u; cptr[u] = ptr[u]; nbr0[u] = -1; nbr1[u] = -1;
    }
}

// The rounds run over a list of live vertices: endpoints (degree < 2) that
// still had a proposal when the list was last compacted. Degrees only grow and
// eligibility is only lost, so a vertex that dropped out never proposes again,
// and its proposal slot stays -1.
__global__ void k_cover_iota(int n, int* __restrict__ list, int* __restrict__ cnt) {
    FOR_EACH(u, n) list[u] = (int)u;
    if (blockIdx.x == 0 && threadIdx.x == 0) *cnt = n;
}

__global__ void k_cover_compact(const int* __restrict__ list, const int* __restrict__ cnt,
                                const int* __restrict__ deg, const int* __restrict__ bv,
                                int* __restrict__ out, int* __restrict__ ocnt) {
    const int m = *cnt;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int u = list[i];
        const bool keep = deg[u] < 2 && bv[u] >= 0;
        const int slot = warp_append(ocnt, keep);
        if (keep) out[slot] = u;
    }
}

#define FOR_LIST(u, list, cnt) \
    for (int i_ = blockIdx.x * blockDim.x + threadIdx.x, m_ = *(cnt); i_ < m_; i_ += gridDim.x * blockDim.x) \
        for (int u = (list)[i_], once_ = 1; once_; once_ = 0)

// 1. each endpoint advances to its best eligible edge (ineligible edges stay so)
__global__ void k_cover_best(const int* __restrict__ list, const int* __restrict__ cnt,
                             const int* __restrict__ ptr, const int* __restrict__ scol,
                             const int* __restrict__ deg, const int* __restrict__ oe,
                             int* __restrict__ cptr, int* __restrict__ bv) {
    FOR_LIST(u, list, cnt) {
        if (deg[u] >= 2) continue;
        int p = cptr[u], e = ptr[u + 1], o = oe[u];
        while (p < e) {
            int v = scol[p];
            if (deg[v] >= 2 || o == v) ++p; else break;
        }
        cptr[u] = p;
        bv[u] = (p < e) ? scol[p] : -1;
    }
}

// 2. each path keeps the better proposal of its two endpoints (both live
// endpoints of a path compute the same choice; either may be the one listed)
__global__ void k_cover_choose(const int* __restrict__ list, const int* __restrict__ cnt,
                               const int* __restrict__ deg, const int* __restrict__ oe,
                               const int* __restrict__ cptr, const int* __restrict__ bv,
                               const double* __restrict__ sw, int* __restrict__ cf,
                               int* __restrict__ ct) {
    FOR_LIST(u, list, cnt) {
        if (deg[u] >= 2) continue;
        int o = oe[u];
        int x = -1, y = -1;
        double wx = 0.0;
        if (bv[u] >= 0) { x = u; y = bv[u]; wx = sw[cptr[u]]; }
        if (o != u && bv[o] >= 0) {
            double wo = sw[cptr[o]];
            if (x < 0 || edge_before(wo, o, bv[o], wx, x, y)) { x = o; y = bv[o]; }
        }
        cf[u] = x; ct[u] = y; cf[o] = x; ct[o] = y;
    }
}

// 3. an edge chosen by both of its paths joins them
__global__ void k_cover_accept(const int* __restrict__ list, const int* __restrict__ cnt,
                               int* __restrict__ deg, int* __restrict__ oe,
                               const int* __restrict__ cf, const int* __restrict__ ct,
                               int* __restrict__ nbr0, int* __restrict__ nbr1,
                               int* __restrict__ counter) {
    int added = 0;
    FOR_LIST(u, list, cnt) {
        if (cf[u] != u) continue;
        int y = ct[u];
        if (y < 0 || y < u) continue;
        if (deg[u] >= 2) continue;
        if (cf[y] != y || ct[y] != u) continue;
        int a = oe[u], b = oe[y];
        oe[a] = b;
        oe[b] = a;
        if (nbr0[u] < 0) nbr0[u] = y; else nbr1[u] = y;
        if (nbr0[y] < 0) nbr0[y] = u; else nbr1[y] = u;
        deg[u] += 1;
        deg[y] += 1;
        ++added;
    }
    block_count(counter, added);
}

__global__ void k_canonical(int n, int* __restrict__ nbr0, int* __restrict__ nbr1) {
    FOR_EACH(u, n) {
        int a = nbr0[u], b = nbr1[u];
        if (a >= 0 && b >= 0 && b < a) { nbr0[u] = b; nbr1[u] = a; }
        else if (a < 0 && b >= 0) { nbr0[u] = b; nbr1[u] = -1; }
    }
}

// ---------------------------------------------------------------- list ranking
// Half-edge h = 2u+k points from u to nbr_k(u). Its successor continues away
// from u at the head. Pointer jumping gives each half-edge the path end it
// reaches and the number of edges to it.
// List ranking state of half-edge h = 2u + k (u's k-th cover neighbour): the
// half-edge it jumps to (-1 at the path's end), the distance covered and the
// end vertex reached, in one 16-byte record so that a jump gathers one sector.
__global__ void k_rank_init(int n, const int* __restrict__ nbr0, const int* __restrict__ nbr1,
                            int4* __restrict__ st) {
    FOR_EACH(u64, n) {
        int u = (int)u64;
        for (int k = 0; k < 2; ++k) {
            int h = 2 * u + k;
            int v = k ? nbr1[u] : nbr0[u];
            if (v < 0) { st[h] = make_int4(-1, 0, -1, 0); continue; }
            int w0 = nbr0[v], w1 = nbr1[v];
            int w = (w0 >= 0 && w0 != u) ? w0 : ((w1 >= 0 && w1 != u) ? w1 : -1);
            st[h] = make_int4((w < 0) ? -1 : (2 * v + (w0 == w ? 0 : 1)), 1, v, 0);
        }
    }
}

// one pointer jump: (jmp, dist, endv) of h <- (jmp[j], dist[h] + dist[j], endv[j]), j = jmp[h]
__global__ void k_rank_jump(int nh, const int4* __restrict__ st, int4* __restrict__ st2,
                            int* __restrict__ active) {
    int more = 0;
    FOR_EACH(h, nh) {
        const int4 a = st[h];
        if (a.x >= 0) {
            const int4 b = st[a.x];
            st2[h] = make_int4(b.x, a.y + b.y, b.z, 0);
            if (b.x >= 0) more = 1;
        } else {
            st2[h] = a;
        }
    }
    block_flag(active, more);
}

// Positions from the canonical end (the endpoint with the smaller id), then the
// matching along the path: positions (0,1), (2,3), ... form aggregates named
// by their first vertex; links to the previous and next matched pair of the
// same path are kept for path shortening.
__global__ void k_pair(int n, const int* __restrict__ nbr0, const int* __restrict__ nbr1,
                       const int4* __restrict__ st,
                       int* __restrict__ lab, int* __restrict__ size, int* __restrict__ sprev,
                       int* __restrict__ snext, unsigned char* __restrict__ ishead) {
    FOR_EACH(u64, n) {
        int u = (int)u64;
        int a = nbr0[u], b = nbr1[u];
        int deg = (a >= 0) + (b >= 0);
        ishead[u] = 0;
        sprev[u] = -1;
        snext[u] = -1;
        if (deg == 0) continue;
        int L, pos, toward = -1, away = -1;
        if (deg == 1) {
            const int4 h0 = st[2 * u];
            int E = h0.z, d = h0.y;
            L = d + 1;
            if (u < E) { pos = 0; away = a; }
            else { pos = d; toward = a; }
        } else {
            const int4 h0 = st[2 * u], h1 = st[2 * u + 1];
            int E0 = h0.z, d0 = h0.y, E1 = h1.z, d1 = h1.y;
            L = d0 + d1 + 1;
            if (E0 < E1) { pos = d0; toward = a; away = b; }
            else { pos = d1; toward = b; away = a; }
        }
        if ((pos & 1) || pos + 1 >= L) continue;
        // u heads the pair (u, away)
        int q = away;
        lab[u] = u;
        lab[q] = u;
        size[u] = 2;
        ishead[u] = 1;
        if (pos + 3 < L) {
            int q0 = nbr0[q], q1 = nbr1[q];
            snext[u] = (q0 != u) ? q0 : q1;
        }
        if (pos >= 2) {
            int t0 = nbr0[toward], t1 = nbr1[toward];
            sprev[u] = (t0 != u) ? t0 : t1;
        }
    }
}

// ---------------------------------------------------------------- leftovers
// best(u): heaviest reweighted edge at u, ties to the smaller neighbour id
__global__ void k_best(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                       const double* __restrict__ w, int* __restrict__ best,
                       int* __restrict__ lab, int* __restrict__ size) {
    FOR_EACH(u64, n) {
        int u = (int)u64;
        // positive weights: their bit patterns order as the values do
        int bb = -1;
        uint64_t bw = 0;
        for (int k = ptr[u]; k < ptr[u + 1]; ++k) {
            const uint64_t x = (uint64_t)__double_as_longlong(w[k]);
            const int c = col[k];
            if (bb < 0 || x > bw || (x == bw && c < bb)) { bb = c; bw = x; }
        }
        best[u] = bb;
        if (bb < 0 && lab[u] < 0) { lab[u] = u; size[u] = 1; }
    }
}

// state at the start of a round: 0 aggregated, 1 waiting (best unaggregated),
// 2 joiner of aggregate jg[u] (best aggregated)
__global__ void k_left_classify(int n, const int* __restrict__ lab, const int* __restrict__ best,
                                int* __restrict__ st, int* __restrict__ jg, int* __restrict__ gcnt,
                                int* __restrict__ nleft) {
    int left = 0;
    FOR_EACH(u64, n) {
        int u = (int)u64;
        if (lab[u] >= 0) { st[u] = 0; continue; }
        ++left;
        int v = best[u];
        int g = lab[v];
        if (g >= 0) { st[u] = 2; jg[u] = g; atomicAdd(gcnt + g, 1); }
        else st[u] = 1;
    }
    block_count(nleft, left);
}

// case 1: mutual best pairs among the waiting vertices
__global__ void k_left_case1(int n, const int* __restrict__ st, const int* __restrict__ best,
                             int* __restrict__ lab, int* __restrict__ size) {
    FOR_EACH(u64, n) {
        int u = (int)u64;
        if (st[u] != 1) continue;
        int v = best[u];
        if (v > u && st[v] == 1 && best[v] == u) {
            lab[u] = u;
            lab[v] = u;
            size[u] = 2;
        }
    }
}

__global__ void k_left_fill(int n, const int* __restrict__ st, const int* __restrict__ jg,
                            const int* __restrict__ goff, int* __restrict__ gfill,
                            int* __restrict__ list) {
    FOR_EACH(u64, n) {
        int u = (int)u64;
        if (st[u] != 2) continue;
        int g = jg[u];
        list[goff[g] + atomicAdd(gfill + g, 1)] = u;
    }
}

// cases 2/3: the joiners of one aggregate, in ascending order, one at a time
__device__ __forceinline__ void left_apply(int u, int v, int* lab, int* size) {
    int h = lab[v];
    if (h < 0) {
        lab[u] = u; lab[v] = u; size[u] = 2;
    } else if (size[h] == 2) {
        lab[u] = h; size[h] = 3;
    } else {
        lab[v] = u; size[h] -= 1; lab[u] = u; size[u] = 2;
    }
}

__global__ void k_left_join(int n, const int* __restrict__ goff, int* __restrict__ list,
                            const int* __restrict__ best, int* __restrict__ lab,
                            int* __restrict__ size) {
    FOR_EACH(g64, n) {
        int g = (int)g64;
        int b = goff[g], e = goff[g + 1];
        if (b == e) continue;
        for (int i = b + 1; i < e; ++i) {  // insertion sort (few joiners)
            int x = list[i], j = i;
            while (j > b && list[j - 1] > x) { list[j] = list[j - 1]; --j; }
            list[j] = x;
        }
        for (int i = b; i < e; ++i) {
            int u = list[i];
            left_apply(u, best[u], lab, size);
        }
    }
}

// after the round cap: the paper's sequential loop, ascending order
__global__ void k_left_tail(int n, const int* __restrict__ best, int* __restrict__ lab,
                            int* __restrict__ size) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int u = 0; u < n; ++u)
        if (lab[u] < 0) left_apply(u, best[u], lab, size);
}

// ---------------------------------------------------------------- numbering
__global__ void k_minmem(int n, const int* __restrict__ lab, int* __restrict__ minmem) {
    FOR_EACH(u, n) atomicMin(minmem + lab[u], (int)u);
}

__global__ void k_isfirst(int n, const int* __restrict__ lab, const int* __restrict__ minmem,
                          int* __restrict__ flag) {
    FOR_EACH(u, n) flag[u] = (minmem[lab[u]] == (int)u) ? 1 : 0;
}

__global__ void k_agg_ids(int n, const int* __restrict__ lab, const int* __restrict__ minmem,
                          const int* __restrict__ cidat, int* __restrict__ agg) {
    FOR_EACH(u, n) agg[u] = cidat[minmem[lab[u]]];
}

// ---------------------------------------------------------------- MWM (Section 2.1)
// Heaviest-first matching on the weighted adjacency of A_l (edge {u,v} weighs
// -a_uv > 0) as locally-dominant rounds: every free vertex points at its best
// free neighbour in the order of Alg. 1 (weight descending, then the smaller
// end, then the larger end); two vertices pointing at each other are matched.
// Each round matches the best free edge overall, and a matched edge is one the
// sequential heaviest-first pass over sorted edges also takes, so the rounds
// give that matching. Weights compare through their bit patterns (positive).
__device__ __forceinline__ bool mwm_before(uint64_t w1, int a1, int b1, uint64_t w2, int a2, int b2) {
    if (w1 != w2) return w1 > w2;
    const int lo1 = min(a1, b1), lo2 = min(a2, b2);
    if (lo1 != lo2) return lo1 < lo2;
    return max(a1, b1) < max(a2, b2);
}

__device__ __forceinline__ uint64_t neg_bits(double a) { return (uint64_t)__double_as_longlong(-a); }

__global__ void k_mwm_best(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                           const double* __restrict__ val, const int* __restrict__ mate,
                           int* __restrict__ best) {
    FOR_EACH(v64, n) {
        const int v = (int)v64;
        int b = -1;
        uint64_t bw = 0;
        if (mate[v] < 0) {
            for (int k = rowptr[v]; k < rowptr[v + 1]; ++k) {
                const int u = col[k];
                if (u == v || mate[u] >= 0) continue;
                const uint64_t w = neg_bits(val[k]);
                if (b < 0 || mwm_before(w, v, u, bw, v, b)) { b = u; bw = w; }
            }
        }
        best[v] = b;
    }
}

__global__ void k_mwm_accept(int n, const int* __restrict__ best, int* __restrict__ mate,
                             int* __restrict__ counter) {
    int matched = 0;
    FOR_EACH(v64, n) {
        const int v = (int)v64;
        const int u = best[v];
        if (u >= 0 && best[u] == v) {
            mate[v] = u;
            if (v < u) ++matched;
        }
    }
    block_count(counter, matched);
}

// pair label = the pair's smaller vertex; a free vertex (all its neighbours are
// matched once the rounds end) takes the label of its heaviest neighbour's pair;
// a vertex without neighbours labels itself
__global__ void k_mwm_label(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                            const double* __restrict__ val, const int* __restrict__ mate,
                            int* __restrict__ lab) {
    FOR_EACH(v64, n) {
        const int v = (int)v64;
        const int m = mate[v];
        if (m >= 0) { lab[v] = min(v, m); continue; }
        int b = -1;
        uint64_t bw = 0;
        for (int k = rowptr[v]; k < rowptr[v + 1]; ++k) {
            const int u = col[k];
            if (u == v) continue;
            const uint64_t w = neg_bits(val[k]);
            if (b < 0 || mwm_before(w, v, u, bw, v, b)) { b = u; bw = w; }
        }
        lab[v] = (b < 0) ? v : min(b, mate[b]);
    }
}

// coarse cover: matched pair k of a path is joined to pairs k-1 and k+1
__global__ void k_shorten(int n, const unsigned char* __restrict__ ishead,
                          const int* __restrict__ sprev, const int* __restrict__ snext,
                          const int* __restrict__ minmem, const int* __restrict__ cidat,
                          int* __restrict__ cn0, int* __restrict__ cn1) {
    FOR_EACH(u64, n) {
        int h = (int)u64;
        if (!ishead[h]) continue;
        int I = cidat[minmem[h]];
        int a = sprev[h] >= 0 ? cidat[minmem[sprev[h]]] : -1;
        int b = snext[h] >= 0 ? cidat[minmem[snext[h]]] : -1;
        if (a >= 0 && b >= 0) { cn0[I] = min(a, b); cn1[I] = max(a, b); }
        else if (a >= 0) { cn0[I] = a; cn1[I] = -1; }
        else if (b >= 0) { cn0[I] = b; cn1[I] = -1; }
    }
}

__global__ void k_count_agg(int n, const int* __restrict__ agg, int* __restrict__ cnt) {
    FOR_EACH(u, n) atomicAdd(cnt + agg[u], 1);
}

__global__ void k_fill_members(int n, const int* __restrict__ agg, const int* __restrict__ aptr,
                               int* __restrict__ fillc, int* __restrict__ mem) {
    FOR_EACH(u, n) {
        int I = agg[u];
        mem[aptr[I] + atomicAdd(fillc + I, 1)] = (int)u;
    }
}

__global__ void k_sort_members(int nc, const int* __restrict__ aptr, int* __restrict__ mem) {
    FOR_EACH(I, nc) {
        int b = aptr[I], e = aptr[I + 1];
        for (int i = b + 1; i < e; ++i) {
            int x = mem[i], j = i;
            while (j > b && mem[j - 1] > x) { mem[j] = mem[j - 1]; --j; }
            mem[j] = x;
        }
    }
}

// P_1 carries e: (P_1)_uI = e_u; an aggregate where e vanishes uses 1
__global__ void k_pval(int nc, const int* __restrict__ aptr, const int* __restrict__ mem,
                       const double* __restrict__ e, double* __restrict__ pval) {
    FOR_EACH(I, nc) {
        int b = aptr[I], en = aptr[I + 1];
        bool zero = true;
        for (int t = b; t < en; ++t) if (e[mem[t]] != 0.0) zero = false;
        for (int t = b; t < en; ++t) pval[mem[t]] = zero ? 1.0 : e[mem[t]];
    }
}

}  // namespace

// ---------------------------------------------------------------- host side
template <class Src>
static void row_product(Ctx& c, int32_t nrows, const Src& src, DBuf<int32_t>& optr,
                        DBuf<int32_t>& ocol, DBuf<double>* oval, int64_t* nnz_out) {
    cudaStream_t s = c.stream;
    DBuf<int32_t> cnt, long_list, long_count;
    DBuf<unsigned char> is_long;
    cnt.alloc(c.mem, nrows);
    long_list.alloc(c.mem, nrows);
    long_count.alloc(c.mem, 1);
    is_long.alloc(c.mem, nrows);
    PC_CUDA(cudaMemsetAsync(long_count.p, 0, sizeof(int32_t), s));
    // one pass of the warp kernel into a temporary layout sized by the rows'
    // contribution counts
    DBuf<int64_t> ubr, tptr;
    DBuf<int32_t> tcol;
    DBuf<double> tval;
    ubr.alloc(c.mem, nrows);
    tptr.alloc(c.mem, (size_t)nrows + 1);
    k_rowprod_ubrow<Src><<<grid1(nrows), kBlock, 0, s>>>(nrows, src, ubr.p); ::pc::count_launches(1);
    const int64_t tot_ub = scan_i64(c, ubr.p, tptr.p, nrows);
    tcol.alloc(c.mem, std::max<int64_t>(tot_ub, 1));
    if (oval) tval.alloc(c.mem, std::max<int64_t>(tot_ub, 1));
    // Short rows a thread each (columns in 24 bits), the others listed for the
    // warp kernel, where the rows are short on average: the thread kernel is
    // faster where nearly every row qualifies (the 256^3 grid's finest two
    // levels, 13.8 and 18.9 contributions per row on average) and slower where
    // half or fewer do (24.8 at the next level: the listing and the warp
    // kernel's scattered row order cost more than the thread rows save).
    // Either way the rows get the same entries, bit for bit.
    const bool use_thread = nrows <= (1 << 24) && tot_ub <= kThreadProdMean * (int64_t)nrows;
    DBuf<int32_t> wrows, wcount;
    if (use_thread) {
        wrows.alloc(c.mem, nrows);
        wcount.alloc(c.mem, 1);
        PC_CUDA(cudaMemsetAsync(wcount.p, 0, sizeof(int32_t), s));
        k_rowprod_thread<Src><<<grid1(nrows), kBlock, 0, s>>>(nrows, src, cnt.p, is_long.p, tcol.p,
                                                              oval ? tval.p : nullptr, tptr.p, wrows.p, wcount.p);
        ::pc::count_launches(1);
        PC_LAUNCH("rowprod_thread(once)");
    }
    k_rowprod_warp<Src, 2><<<grid_warps(nrows), kWarpsPerBlock * 32, 0, s>>>(
        nrows, src, cnt.p, is_long.p, long_list.p, long_count.p, nullptr, tcol.p, oval ? tval.p : nullptr, tptr.p,
        use_thread ? wrows.p : nullptr, use_thread ? wcount.p : nullptr);
    ::pc::count_launches(1);
    PC_LAUNCH("rowprod_warp(once)");
    int32_t nlong = read_i32(c, long_count.p);
    int32_t nB = 0, nC = 0;
    DBuf<int32_t> dB, dC;
    DBuf<int64_t> offC;
    DBuf<uint64_t> gkeys;
    DBuf<double> gvals;
    if (nlong > 0) {
        DBuf<int32_t> counts;
        DBuf<int64_t> ubC;
        counts.alloc(c.mem, 2);
        dB.alloc(c.mem, nlong);
        dC.alloc(c.mem, nlong);
        ubC.alloc(c.mem, nlong);
        PC_CUDA(cudaMemsetAsync(counts.p, 0, sizeof(int32_t) * 2, s));
        k_rowprod_split<Src><<<grid1(nlong), kBlock, 0, s>>>(nlong, long_list.p, src, dB.p, dC.p, ubC.p, counts.p);
        ::pc::count_launches(1);
        PC_LAUNCH("rowprod_split");
        int32_t hc[2] = {0, 0};
        d2h(c, hc, counts.p, 2);
        nB = hc[0];
        nC = hc[1];
        if (nB > 0) {   // one pass, into the temporary layout
            size_t smem = kBlockCap * (sizeof(uint64_t) + sizeof(double));
            k_rowprod_block<Src, 2, false><<<(unsigned)nB, kBlock, smem, s>>>(
                dB.p, src, cnt.p, nullptr, tcol.p, oval ? tval.p : nullptr, nullptr, nullptr, nullptr, tptr.p, is_long.p);
            ::pc::count_launches(1);
            PC_LAUNCH("rowprod_block(once)");
        }
        if (nC > 0) {   // rare: staging in global memory, count then fill
            std::vector<int64_t> hub(nC), hoff(nC);
            d2h(c, hub.data(), ubC.p, nC);
            int64_t totC = 0;
            for (int32_t i = 0; i < nC; ++i) {
                if (hub[i] >= (int64_t)1 << 31) fail(PCAMG_ERR_INVALID, "row product: a row has 2^31 or more contributions");
                hoff[i] = totC;
                int64_t P = 1;
                while (P < hub[i]) P <<= 1;
                totC += P;
            }
            offC.alloc(c.mem, nC);
            gkeys.alloc(c.mem, totC);
            gvals.alloc(c.mem, totC);
            PC_CUDA(cudaMemcpyAsync(offC.p, hoff.data(), sizeof(int64_t) * nC, cudaMemcpyHostToDevice, s));
            k_rowprod_block<Src, 0, true><<<(unsigned)nC, kBlock, 0, s>>>(
                dC.p, src, cnt.p, nullptr, nullptr, nullptr, gkeys.p, gvals.p, offC.p, nullptr, nullptr); ::pc::count_launches(1);
            PC_LAUNCH("rowprod_global(count)");
        }
    }
    optr.alloc(c.mem, (size_t)nrows + 1);
    int64_t total = scan_i32(c, cnt.p, optr.p, nrows);
    if (total >= ((int64_t)1 << 31)) fail(PCAMG_ERR_INVALID, "row product: result has 2^31 or more entries");
    ocol.alloc(c.mem, total);
    double* ov = nullptr;
    if (oval) { oval->alloc(c.mem, total); ov = oval->p; }
    const int gcompact = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)nrows + 255) / 256, (int64_t)kNumSMs * 16));
    k_rowprod_compact<<<gcompact, kWarpsPerBlock * 32, 0, s>>>(nrows, is_long.p, cnt.p, tptr.p, tcol.p,
                                                                         oval ? tval.p : nullptr, optr.p, ocol.p, ov);
    ::pc::count_launches(1);
    PC_LAUNCH("rowprod_compact");
    if (nC > 0) {
        k_rowprod_block<Src, 1, true><<<(unsigned)nC, kBlock, 0, s>>>(
            dC.p, src, nullptr, optr.p, ocol.p, ov, gkeys.p, gvals.p, offC.p, nullptr, nullptr); ::pc::count_launches(1);
        PC_LAUNCH("rowprod_global(fill)");
    }
    *nnz_out = total;
    sync(c);
}

void build_candidates(Ctx& c, const double* e, Reweighted& out) {
    // the A^2 pattern depends on A alone: formed by the first build, copied
    // for the later ones (only the weights follow the new e)
    if (c.cand_nnz < 0) {
        CandSrc src{c.rowptr.p, c.col.p};
        row_product(c, c.n, src, c.cand_ptr, c.cand_col, nullptr, &c.cand_nnz);
    }
    out.nnz = c.cand_nnz;
    out.ptr.alloc(c.mem, (size_t)c.n + 1);
    out.col.alloc(c.mem, (size_t)out.nnz);
    PC_CUDA(cudaMemcpyAsync(out.ptr.p, c.cand_ptr.p, sizeof(int32_t) * ((size_t)c.n + 1), cudaMemcpyDeviceToDevice,
                            c.stream));
    PC_CUDA(cudaMemcpyAsync(out.col.p, c.cand_col.p, sizeof(int32_t) * (size_t)out.nnz, cudaMemcpyDeviceToDevice,
                            c.stream));
    out.w.alloc(c.mem, out.nnz);
    int nb = 256;
    DBuf<double> part;
    part.alloc(c.mem, nb + 1);
    k_maxabs<<<nb, kBlock, 0, c.stream>>>(c.n, e, part.p); ::pc::count_launches(1);
    k_delta<<<1, 1, 0, c.stream>>>(nb, part.p, part.p + nb); ::pc::count_launches(1);
    k_weights<<<grid1(c.n), kBlock, 0, c.stream>>>(c.n, out.ptr.p, out.col.p, e, part.p + nb, out.w.p); ::pc::count_launches(1);
    PC_LAUNCH("weights");
    sync(c);
}

int32_t path_cover(Ctx& c, int32_t n, const Reweighted& t, int32_t* nbr0, int32_t* nbr1) {
    cudaStream_t s = c.stream;
    // rows in proposal order
    DBuf<int32_t> scol, long_list, long_count, mid_list;
    DBuf<double> sw;
    DBuf<unsigned char> is_long;
    scol.alloc(c.mem, t.nnz);
    sw.alloc(c.mem, t.nnz);
    long_list.alloc(c.mem, n);
    mid_list.alloc(c.mem, n);
    long_count.alloc(c.mem, 2);   // [0] class-2 rows, [1] class-1 rows
    is_long.alloc(c.mem, n);
    PC_CUDA(cudaMemsetAsync(long_count.p, 0, 2 * sizeof(int32_t), s));
    k_order_rows_classify<<<grid1(n), kBlock, 0, s>>>(n, t.ptr.p, is_long.p, mid_list.p, long_count.p + 1,
                                                      long_list.p, long_count.p);
    ::pc::count_launches(1);
    PC_LAUNCH("order_rows");
    k_order_rows_thread<<<grid1(n), kBlock, 0, s>>>(n, is_long.p, t.ptr.p, t.col.p, t.w.p, scol.p, sw.p);
    ::pc::count_launches(1);
    PC_LAUNCH("order_rows_thread");
    k_order_rows_warp<<<grid_warps(n), kWarpsPerBlock * 32, 0, s>>>(mid_list.p, long_count.p + 1, t.ptr.p,
                                                                     t.col.p, t.w.p, scol.p, sw.p);
    ::pc::count_launches(1);
    PC_LAUNCH("order_rows_warp");
    const int32_t nbig = read_i32(c, long_count.p);
    if (nbig > 0) {   // rare: rows longer than kOrderWarpCap, a block each
        std::vector<int32_t> big(nbig), hl(nbig);
        d2h(c, big.data(), long_list.p, nbig);
        DBuf<int32_t> dlen;
        dlen.alloc(c.mem, nbig);
        k_row_lengths<<<grid1(nbig), kBlock, 0, s>>>(nbig, long_list.p, t.ptr.p, dlen.p); ::pc::count_launches(1);
        d2h(c, hl.data(), dlen.p, nbig);
        std::vector<int64_t> off(nbig);
        int64_t tot = 0;
        for (int32_t i = 0; i < nbig; ++i) {
            int64_t len = hl[i], P = 1;
            while (P < len) P <<= 1;
            off[i] = tot;
            tot += P;
        }
        DBuf<int32_t> drows;
        DBuf<int64_t> doff;
        DBuf<uint32_t> gidx;
        drows.alloc(c.mem, nbig);
        doff.alloc(c.mem, nbig);
        gidx.alloc(c.mem, tot);
        PC_CUDA(cudaMemcpyAsync(drows.p, big.data(), sizeof(int32_t) * nbig, cudaMemcpyHostToDevice, s));
        PC_CUDA(cudaMemcpyAsync(doff.p, off.data(), sizeof(int64_t) * nbig, cudaMemcpyHostToDevice, s));
        k_order_rows_block<<<nbig, kBlock, 0, s>>>(drows.p, t.ptr.p, t.col.p, t.w.p, scol.p, sw.p, gidx.p, doff.p); ::pc::count_launches(1);
        PC_LAUNCH("order_rows_block");
        sync(c);
    }
    DBuf<int32_t> deg, oe, cptr, bv, cf, ct, counters;
    deg.alloc(c.mem, n); oe.alloc(c.mem, n); cptr.alloc(c.mem, n); bv.alloc(c.mem, n);
    cf.alloc(c.mem, n); ct.alloc(c.mem, n);
    const int kBatchMax = 64;
    counters.alloc(c.mem, kBatchMax);
    k_cover_init<<<grid1(n), kBlock, 0, s>>>(n, t.ptr.p, deg.p, oe.p, cptr.p, nbr0, nbr1); ::pc::count_launches(1);
    fill_i32(s, n, -1, cf.p);
    int32_t rounds = 0, batch = 4;
    std::vector<int32_t> hc(kBatchMax);
    DBuf<int32_t> la, lb, lcnt;
    la.alloc(c.mem, n); lb.alloc(c.mem, n); lcnt.alloc(c.mem, 2);
    k_cover_iota<<<grid1(n), kBlock, 0, s>>>(n, la.p, lcnt.p); ::pc::count_launches(1);
    int32_t *list = la.p, *spare = lb.p, *cnt = lcnt.p, *scnt = lcnt.p + 1;
    const int lgrid = kNumSMs * 8;
    for (;;) {
        PC_CUDA(cudaMemsetAsync(counters.p, 0, sizeof(int32_t) * batch, s));
        for (int r = 0; r < batch; ++r) {
            k_cover_best<<<lgrid, kBlock, 0, s>>>(list, cnt, t.ptr.p, scol.p, deg.p, oe.p, cptr.p, bv.p); ::pc::count_launches(1);
            k_cover_choose<<<lgrid, kBlock, 0, s>>>(list, cnt, deg.p, oe.p, cptr.p, bv.p, sw.p, cf.p, ct.p); ::pc::count_launches(1);
            k_cover_accept<<<lgrid, kBlock, 0, s>>>(list, cnt, deg.p, oe.p, cf.p, ct.p, nbr0, nbr1, counters.p + r); ::pc::count_launches(1);
        }
        // drop the vertices that can no longer propose
        PC_CUDA(cudaMemsetAsync(scnt, 0, sizeof(int32_t), s));
        k_cover_compact<<<lgrid, kBlock, 0, s>>>(list, cnt, deg.p, bv.p, spare, scnt); ::pc::count_launches(1);
        std::swap(list, spare);
        std::swap(cnt, scnt);
        PC_LAUNCH("cover rounds");
        d2h(c, hc.data(), counters.p, batch);
        bool done = false;
        for (int r = 0; r < batch; ++r) {
            ++rounds;
            if (hc[r] == 0) { done = true; break; }
        }
        if (done) break;
        const int64_t cap = c.p.max_cover_rounds > 0 ? (int64_t)c.p.max_cover_rounds : (int64_t)n + 1;
        if (rounds > cap) fail(PCAMG_ERR_ROUND_CAP, "path cover rounds exceeded their cap");
        batch = std::min(batch * 2, kBatchMax);
    }
    // rounds that added edges (the last round found none)
    if (c.p.max_cover_rounds > 0 && rounds - 1 > c.p.max_cover_rounds)
        fail(PCAMG_ERR_ROUND_CAP, "path cover rounds exceeded their cap");
    k_canonical<<<grid1(n), kBlock, 0, s>>>(n, nbr0, nbr1); ::pc::count_launches(1);
    PC_LAUNCH("canonical");
    sync(c);
    return rounds;
}

int32_t aggregate_level(Ctx& c, int32_t n, const int32_t* nbr0, const int32_t* nbr1,
                        const Reweighted& t, DBuf<int32_t>& agg, DBuf<int32_t>& cnbr0,
                        DBuf<int32_t>& cnbr1, int32_t* rounds_out) {
    cudaStream_t s = c.stream;
    int64_t nh = 2 * (int64_t)n;
    DBuf<int4> rk[2];
    DBuf<int32_t> active;
    for (int k = 0; k < 2; ++k) rk[k].alloc(c.mem, nh);
    active.alloc(c.mem, 1);
    k_rank_init<<<grid1(n), kBlock, 0, s>>>(n, nbr0, nbr1, rk[0].p); ::pc::count_launches(1);
    PC_LAUNCH("rank_init");
    // pointer jumping: the active flag is read every 4 rounds (rounds after the
    // last jump copy their input)
    int cur = 0;
    for (int it = 0;; it += 4) {
        PC_CUDA(cudaMemsetAsync(active.p, 0, sizeof(int32_t), s));
        for (int k = 0; k < 4; ++k) {
            k_rank_jump<<<grid1(nh), kBlock, 0, s>>>((int)nh, rk[cur].p, rk[1 - cur].p, active.p); ::pc::count_launches(1);
            cur = 1 - cur;
        }
        PC_LAUNCH("rank_jump");
        if (read_i32(c, active.p) == 0) break;
        if (it > 40) fail(PCAMG_ERR_ROUND_CAP, "list ranking did not finish");
    }
    DBuf<int32_t> lab, size, sprev, snext, best, st, jg, gcnt, goff, gfill, list, nleft;
    DBuf<unsigned char> ishead;
    lab.alloc(c.mem, n); size.alloc(c.mem, n); sprev.alloc(c.mem, n); snext.alloc(c.mem, n);
    best.alloc(c.mem, n); st.alloc(c.mem, n); jg.alloc(c.mem, n); gcnt.alloc(c.mem, n);
    goff.alloc(c.mem, (size_t)n + 1); gfill.alloc(c.mem, n); list.alloc(c.mem, n); nleft.alloc(c.mem, 1);
    ishead.alloc(c.mem, n);
    fill_i32(s, n, -1, lab.p);
    fill_i32(s, n, 0, size.p);
    k_pair<<<grid1(n), kBlock, 0, s>>>(n, nbr0, nbr1, rk[cur].p, lab.p, size.p,
                                       sprev.p, snext.p, ishead.p); ::pc::count_launches(1);
    k_best<<<grid1(n), kBlock, 0, s>>>(n, t.ptr.p, t.col.p, t.w.p, best.p, lab.p, size.p); ::pc::count_launches(1);
    PC_LAUNCH("pair/best");
    // Leftover rounds are launched in batches and their leftover counts read
    // once per batch: a round that finds no leftover vertex changes nothing
    // (every vertex is classified 0, so no pair, joiner or list entry arises),
    // so rounds past the last productive one are harmless no-ops. The rounds
    // counted are those that found leftovers, as in a round-by-round loop.
    int32_t rounds = 0, batch = 2;
    constexpr int kLeftBatchMax = 16;
    DBuf<int32_t> nl;
    nl.alloc(c.mem, kLeftBatchMax);
    int32_t hn[kLeftBatchMax];
    for (;;) {
        const int B = std::min(batch, c.p.round_cap - rounds);
        if (B <= 0) {   // cap reached: the paper's sequential loop finishes if needed
            PC_CUDA(cudaMemsetAsync(gcnt.p, 0, sizeof(int32_t) * n, s));
            PC_CUDA(cudaMemsetAsync(nleft.p, 0, sizeof(int32_t), s));
            k_left_classify<<<grid1(n), kBlock, 0, s>>>(n, lab.p, best.p, st.p, jg.p, gcnt.p, nleft.p); ::pc::count_launches(1);
            PC_LAUNCH("left_classify");
            if (read_i32(c, nleft.p) == 0) break;
            k_left_tail<<<1, 1, 0, s>>>(n, best.p, lab.p, size.p); ::pc::count_launches(1);
            PC_LAUNCH("left_tail");
            ++rounds;
            break;
        }
        PC_CUDA(cudaMemsetAsync(nl.p, 0, sizeof(int32_t) * B, s));
        for (int r = 0; r < B; ++r) {
            PC_CUDA(cudaMemsetAsync(gcnt.p, 0, sizeof(int32_t) * n, s));
            k_left_classify<<<grid1(n), kBlock, 0, s>>>(n, lab.p, best.p, st.p, jg.p, gcnt.p, nl.p + r); ::pc::count_launches(1);
            k_left_case1<<<grid1(n), kBlock, 0, s>>>(n, st.p, best.p, lab.p, size.p); ::pc::count_launches(1);
            scan_i32_device(c, gcnt.p, goff.p, n);
            PC_CUDA(cudaMemsetAsync(gfill.p, 0, sizeof(int32_t) * n, s));
            k_left_fill<<<grid1(n), kBlock, 0, s>>>(n, st.p, jg.p, goff.p, gfill.p, list.p); ::pc::count_launches(1);
            k_left_join<<<grid1(n), kBlock, 0, s>>>(n, goff.p, list.p, best.p, lab.p, size.p); ::pc::count_launches(1);
            PC_LAUNCH("left_round");
        }
        d2h(c, hn, nl.p, B);
        int j = 0;
        while (j < B && hn[j] > 0) ++j;
        rounds += j;
        if (j < B) break;
        batch = std::min(batch * 2, kLeftBatchMax);
    }
    // numbering by smallest member
    DBuf<int32_t> minmem, flag, cidat;
    minmem.alloc(c.mem, n); flag.alloc(c.mem, n); cidat.alloc(c.mem, (size_t)n + 1);
    fill_i32(s, n, 0x7fffffff, minmem.p);
    k_minmem<<<grid1(n), kBlock, 0, s>>>(n, lab.p, minmem.p); ::pc::count_launches(1);
    k_isfirst<<<grid1(n), kBlock, 0, s>>>(n, lab.p, minmem.p, flag.p); ::pc::count_launches(1);
    PC_LAUNCH("numbering");
    int32_t nc = (int32_t)scan_i32(c, flag.p, cidat.p, n);
    agg.alloc(c.mem, n);
    k_agg_ids<<<grid1(n), kBlock, 0, s>>>(n, lab.p, minmem.p, cidat.p, agg.p); ::pc::count_launches(1);
    cnbr0.alloc(c.mem, nc);
    cnbr1.alloc(c.mem, nc);
    fill_i32(s, nc, -1, cnbr0.p);
    fill_i32(s, nc, -1, cnbr1.p);
    k_shorten<<<grid1(n), kBlock, 0, s>>>(n, ishead.p, sprev.p, snext.p, minmem.p, cidat.p, cnbr0.p, cnbr1.p); ::pc::count_launches(1);
    PC_LAUNCH("agg/shorten");
    sync(c);
    if (rounds_out) *rounds_out = rounds;
    return nc;
}

int32_t mwm_aggregate_level(Ctx& c, int32_t n, const int32_t* rowptr, const int32_t* col,
                            const double* val, DBuf<int32_t>& agg, int32_t* rounds_out) {
    cudaStream_t s = c.stream;
    DBuf<int32_t> mate, best, counters, lab, minmem, flag, cidat;
    mate.alloc(c.mem, n); best.alloc(c.mem, n); lab.alloc(c.mem, n);
    const int kBatchMax = 64;
    counters.alloc(c.mem, kBatchMax);
    fill_i32(s, n, -1, mate.p);
    int32_t rounds = 0, batch = 4;
    int32_t hc[kBatchMax];
    // rounds in batches; a round after the last productive one matches nothing
    for (;;) {
        PC_CUDA(cudaMemsetAsync(counters.p, 0, sizeof(int32_t) * batch, s));
        for (int r = 0; r < batch; ++r) {
            k_mwm_best<<<grid1(n), kBlock, 0, s>>>(n, rowptr, col, val, mate.p, best.p); ::pc::count_launches(1);
            k_mwm_accept<<<grid1(n), kBlock, 0, s>>>(n, best.p, mate.p, counters.p + r); ::pc::count_launches(1);
        }
        PC_LAUNCH("mwm rounds");
        d2h(c, hc, counters.p, batch);
        bool done = false;
        for (int r = 0; r < batch; ++r) {
            ++rounds;
            if (hc[r] == 0) { done = true; break; }
        }
        if (done) break;
        if (rounds > n + 1) fail(PCAMG_ERR_ROUND_CAP, "matching rounds exceeded n");
        batch = std::min(batch * 2, kBatchMax);
    }
    k_mwm_label<<<grid1(n), kBlock, 0, s>>>(n, rowptr, col, val, mate.p, lab.p); ::pc::count_launches(1);
    minmem.alloc(c.mem, n); flag.alloc(c.mem, n); cidat.alloc(c.mem, (size_t)n + 1);
    fill_i32(s, n, 0x7fffffff, minmem.p);
    k_minmem<<<grid1(n), kBlock, 0, s>>>(n, lab.p, minmem.p); ::pc::count_launches(1);
    k_isfirst<<<grid1(n), kBlock, 0, s>>>(n, lab.p, minmem.p, flag.p); ::pc::count_launches(1);
    PC_LAUNCH("mwm numbering");
    const int32_t nc = (int32_t)scan_i32(c, flag.p, cidat.p, n);
    agg.alloc(c.mem, n);
    k_agg_ids<<<grid1(n), kBlock, 0, s>>>(n, lab.p, minmem.p, cidat.p, agg.p); ::pc::count_launches(1);
    PC_LAUNCH("mwm ids");
    if (rounds_out) *rounds_out = rounds;
    return nc;
}

void build_members(Ctx& c, int32_t n, int32_t nc, const int32_t* agg, DBuf<int32_t>& agg_ptr,
                   DBuf<int32_t>& agg_mem) {
    cudaStream_t s = c.stream;
    DBuf<int32_t> cnt, fillc;
    cnt.alloc(c.mem, nc);
    fillc.alloc(c.mem, nc);
    PC_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * nc, s));
    PC_CUDA(cudaMemsetAsync(fillc.p, 0, sizeof(int32_t) * nc, s));
    k_count_agg<<<grid1(n), kBlock, 0, s>>>(n, agg, cnt.p); ::pc::count_launches(1);
    agg_ptr.alloc(c.mem, (size_t)nc + 1);
    scan_i32(c, cnt.p, agg_ptr.p, nc);
    agg_mem.alloc(c.mem, n);
    k_fill_members<<<grid1(n), kBlock, 0, s>>>(n, agg, agg_ptr.p, fillc.p, agg_mem.p); ::pc::count_launches(1);
    k_sort_members<<<grid1(nc), kBlock, 0, s>>>(nc, agg_ptr.p, agg_mem.p); ::pc::count_launches(1);
    PC_LAUNCH("members");
}

void build_pval(Ctx& c, int32_t n, int32_t nc, const int32_t* agg_ptr, const int32_t* agg_mem,
                const double* e, DBuf<double>& pval) {
    pval.alloc(c.mem, n);
    k_pval<<<grid1(nc), kBlock, 0, c.stream>>>(nc, agg_ptr, agg_mem, e, pval.p); ::pc::count_launches(1);
    PC_LAUNCH("pval");
}

int64_t galerkin(Ctx& c, int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                 int32_t nc, const int32_t* agg, const int32_t* agg_ptr, const int32_t* agg_mem,
                 const double* pval, bool drop_diag, DBuf<int32_t>& optr, DBuf<int32_t>& ocol,
                 DBuf<double>& oval) {
    (void)n;
    GalSrc src{agg_ptr, agg_mem, rowptr, col, val, pval, agg, drop_diag ? 1 : 0};
    int64_t nnz = 0;
    row_product(c, nc, src, optr, ocol, &oval, &nnz);
    return nnz;
}

}  // namespace pc
