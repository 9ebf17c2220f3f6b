// Smoother colouring. A connected bipartite graph is coloured by the parity of
// the breadth-first distance from vertex 0 (two colours). Otherwise:
// Jones-Plassmann rounds with priorities
// (splitmix64(seed ^ i), i). In a round every uncoloured vertex whose priority
// beats all its uncoloured neighbours takes the smallest colour not used by its
// already coloured neighbours; such winners are never adjacent, so a round's
// assignments are independent. The colour classes are independent sets, which
// makes a multicolour Gauss-Seidel sweep deterministic and parallel.
#include <algorithm>
#include <vector>

#include "pcamg_internal.cuh"

namespace pc {

namespace {

#define FOR_EACH(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

inline int gridc(int64_t n) {
    int64_t g = (n + kBlock - 1) / kBlock;
    if (g < 1) g = 1;
    if (g > (int64_t)kNumSMs * 32) g = kNumSMs * 32;
    return (int)g;
}

// SplitMix64 output function (Steele, Lea, Flood 2014).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_colour_round(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                               uint64_t seed, const int* __restrict__ cin, int* __restrict__ cout,
                               int* __restrict__ left, int* __restrict__ maxc) {
    int nleft = 0, cmax = -1;
    FOR_EACH(v64, n) {
        int v = (int)v64;
        int cv = cin[v];
        if (cv >= 0) { cout[v] = cv; continue; }
        uint64_t hv = splitmix64(seed ^ (uint64_t)(int64_t)v);
        int beg = rowptr[v], end = rowptr[v + 1];
        bool win = true;
        for (int k = beg; k < end && win; ++k) {
            int u = col[k];
            if (u == v || cin[u] >= 0) continue;
            uint64_t hu = splitmix64(seed ^ (uint64_t)(int64_t)u);
            if (hu > hv || (hu == hv && u > v)) win = false;
        }
        if (!win) { cout[v] = -1; ++nleft; continue; }
        uint64_t mask = 0;
        for (int k = beg; k < end; ++k) {
            int u = col[k];
            int cu = cin[u];
            if (u != v && cu >= 0 && cu < 64) mask |= 1ull << cu;
        }
        int c;
        if (~mask != 0ull) {
            c = __ffsll((long long)~mask) - 1;
        } else {
            c = 64;
            for (;;) {  // rare: 64 or more colours around v
                bool used = false;
                for (int k = beg; k < end; ++k) {
                    int u = col[k];
                    if (u != v && cin[u] == c) { used = true; break; }
                }
                if (!used) break;
                ++c;
            }
        }
        cout[v] = c;
        cmax = max(cmax, c);
    }
    block_count(left, nleft);
    // largest colour of the block, one atomic per block
    __shared__ int s_max;
    if (threadIdx.x == 0) s_max = -1;
    __syncthreads();
    for (int o = 16; o > 0; o >>= 1) cmax = max(cmax, __shfl_down_sync(0xffffffffu, cmax, o));
    if ((threadIdx.x & 31) == 0 && cmax >= 0) atomicMax(&s_max, cmax);
    __syncthreads();
    if (threadIdx.x == 0 && s_max >= 0) atomicMax(maxc, s_max);
}

// One breadth-first level from vertex 0 over its frontier (the vertices at
// distance d, listed by the previous level): every frontier vertex claims its
// unlabelled neighbours for distance d + 1 (one claimant wins each, by
// compare-and-swap, and lists it for the next level). An edge between two
// vertices at distance d means an odd cycle; distances d are final before this
// launch and it writes only d + 1, so the test is race free. The lists' order
// depends on scheduling; the distances do not.
__global__ void k_bfs_level(const int* __restrict__ rowptr, const int* __restrict__ col, int d,
                            const int* __restrict__ qin, const int* __restrict__ nin,
                            int* __restrict__ qout, int* __restrict__ nout, int* __restrict__ dist,
                            int* __restrict__ odd) {
    const int m = *nin;
    int o = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int v = qin[i];
        for (int k = rowptr[v]; k < rowptr[v + 1]; ++k) {
            const int u = col[k];
            if (u == v) continue;
            const int du = dist[u];
            if (du == d) o = 1;
            else if (du < 0 && atomicCAS(dist + u, -1, d + 1) == -1) qout[atomicAdd(nout, 1)] = u;
        }
    }
    block_flag(odd, o);
}

__global__ void k_parity_colour(int n, const int* __restrict__ dist, int* __restrict__ colour,
                                int* __restrict__ unreached) {
    FOR_EACH(v, n) {
        const int d = dist[v];
        colour[v] = d & 1;
        if (d < 0) *unreached = 1;
    }
}

__global__ void k_colour_count(int n, const int* __restrict__ colour, int* __restrict__ cnt) {
    FOR_EACH(v, n) atomicAdd(cnt + colour[v], 1);
}

// Rows of each colour into its segment. Within a warp, lanes of equal colour
// take consecutive slots with one atomic per colour, so segments fill in
// nearly ascending row order (the order inside a colour does not change the
// sweep: rows of one colour are independent).
__global__ void k_colour_place(int n, const int* __restrict__ colour, const int* __restrict__ base,
                               int* __restrict__ cursor, int* __restrict__ rows) {
    for (int64_t v0 = blockIdx.x * (int64_t)blockDim.x; v0 < n; v0 += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = v0 + threadIdx.x;
        int c = (v < n) ? colour[v] : -1;
        unsigned peers = __match_any_sync(0xffffffffu, c);
        int lane = threadIdx.x & 31;
        int leader = __ffs(peers) - 1;
        int rank = __popc(peers & ((1u << lane) - 1u));
        int off = 0;
        if (lane == leader && c >= 0) off = atomicAdd(cursor + c, __popc(peers));
        off = __shfl_sync(0xffffffffu, off, leader);
        if (c >= 0) rows[base[c] + off + rank] = (int)v;
    }
}

}  // namespace

int32_t colour_graph(Ctx& c, int32_t n, const int32_t* rowptr, const int32_t* col, uint64_t seed,
                     int32_t* colour) {
    cudaStream_t s = c.stream;
    DBuf<int32_t> tmp, left, maxc;
    tmp.alloc(c.mem, n);
    left.alloc(c.mem, 1);
    maxc.alloc(c.mem, 1);
    fill_i32(s, n, -1, colour);
    PC_CUDA(cudaMemsetAsync(maxc.p, 0, sizeof(int32_t), s));
    int32_t* a = colour;
    int32_t* b = tmp.p;
    // rounds in batches; a round after the last one changes nothing
    const int kBatch = 4;
    DBuf<int32_t> lefts;
    lefts.alloc(c.mem, kBatch);
    int32_t hl[kBatch];
    for (int round = 0;;) {
        PC_CUDA(cudaMemsetAsync(lefts.p, 0, sizeof(int32_t) * kBatch, s));
        for (int k = 0; k < kBatch; ++k) {
            k_colour_round<<<gridc(n), kBlock, 0, s>>>(n, rowptr, col, seed, a, b, lefts.p + k, maxc.p); ::pc::count_launches(1);
            int32_t* t = a; a = b; b = t;
        }
        PC_LAUNCH("colour_round");
        d2h(c, hl, lefts.p, kBatch);
        round += kBatch;
        if (hl[kBatch - 1] == 0) break;
        if (round > n + kBatch) fail(PCAMG_ERR_ROUND_CAP, "colouring rounds exceeded n");
    }
    (void)left;
    if (a != colour) PC_CUDA(cudaMemcpyAsync(colour, a, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    int32_t nc = read_i32(c, maxc.p) + 1;
    return nc;
}

// Smoother colouring: a connected bipartite graph gets the parity of each
// vertex's breadth-first distance from vertex 0 (two colours); any other graph
// the Jones-Plassmann colouring. Levels run in batches with one read of their
// flags per batch (a level past the last labels nothing); an odd cycle ends the
// search early.
int32_t colour_smoother(Ctx& c, int32_t n, const int32_t* rowptr, const int32_t* col, uint64_t seed,
                        int32_t* colour) {
    cudaStream_t s = c.stream;
    if (n < 2) return colour_graph(c, n, rowptr, col, seed, colour);
    constexpr int kMaxBatch = 64;
    DBuf<int32_t> dist, q0, q1, cnt;
    dist.alloc(c.mem, n);
    q0.alloc(c.mem, n);
    q1.alloc(c.mem, n);
    cnt.alloc(c.mem, kMaxBatch + 3);   // [frontier sizes of the batch's levels..., odd, unreached]
    fill_i32(s, n, -1, dist.p);
    PC_CUDA(cudaMemsetAsync(dist.p, 0, sizeof(int32_t), s));   // vertex 0 at distance 0
    PC_CUDA(cudaMemsetAsync(q0.p, 0, sizeof(int32_t), s));     // frontier of level 0: {0}
    int32_t* odd = cnt.p + kMaxBatch + 1;
    int32_t* unreached = cnt.p + kMaxBatch + 2;
    PC_CUDA(cudaMemsetAsync(odd, 0, sizeof(int32_t) * 2, s));
    const int one = 1;
    int32_t h[kMaxBatch + 2];
    bool bipartite = true;
    int32_t* qa = q0.p;
    int32_t* qb = q1.p;
    for (int d = 0, batch = 8;; batch = std::min(batch * 2, kMaxBatch)) {
        // cnt[0] = size of level d's frontier (carried over), cnt[1..batch] filled here
        if (d == 0) PC_CUDA(cudaMemcpyAsync(cnt.p, &one, sizeof(int32_t), cudaMemcpyHostToDevice, s));
        PC_CUDA(cudaMemsetAsync(cnt.p + 1, 0, sizeof(int32_t) * batch, s));
        const int grid = kNumSMs * 4;
        for (int k = 0; k < batch; ++k) {
            k_bfs_level<<<grid, kBlock, 0, s>>>(rowptr, col, d + k, qa, cnt.p + k, qb, cnt.p + k + 1,
                                                dist.p, odd);
            ::pc::count_launches(1);
            int32_t* t = qa; qa = qb; qb = t;
        }
        PC_LAUNCH("bfs_level");
        d2h(c, h, cnt.p, batch + 1);
        d2h(c, h + batch + 1, odd, 1);
        d += batch;
        if (h[batch + 1]) { bipartite = false; break; }
        if (h[batch] == 0) break;
        // the last level's frontier size starts the next batch
        PC_CUDA(cudaMemcpyAsync(cnt.p, cnt.p + batch, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        if (d > n + batch) fail(PCAMG_ERR_ROUND_CAP, "breadth-first levels exceeded n");
    }
    if (bipartite) {
        k_parity_colour<<<gridc(n), kBlock, 0, s>>>(n, dist.p, colour, unreached); ::pc::count_launches(1);
        PC_LAUNCH("parity_colour");
        if (read_i32(c, unreached) == 0) return 2;
    }
    return colour_graph(c, n, rowptr, col, seed, colour);
}

// Rows grouped by colour (segments in colour order).
void colour_lists(Ctx& c, int32_t n, const int32_t* colour, int32_t ncolour,
                  DBuf<int32_t>& rows, std::vector<int32_t>& h_ptr) {
    cudaStream_t s = c.stream;
    rows.alloc(c.mem, n);
    DBuf<int32_t> cnt, base, cursor;
    cnt.alloc(c.mem, ncolour);
    base.alloc(c.mem, ncolour);
    cursor.alloc(c.mem, ncolour);
    PC_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * ncolour, s));
    PC_CUDA(cudaMemsetAsync(cursor.p, 0, sizeof(int32_t) * ncolour, s));
    k_colour_count<<<gridc(n), kBlock, 0, s>>>(n, colour, cnt.p); ::pc::count_launches(1);
    PC_LAUNCH("colour_count");
    std::vector<int32_t> hc(ncolour);
    d2h(c, hc.data(), cnt.p, ncolour);
    h_ptr.assign((size_t)ncolour + 1, 0);
    for (int32_t k = 0; k < ncolour; ++k) h_ptr[k + 1] = h_ptr[k] + hc[k];
    PC_CUDA(cudaMemcpyAsync(base.p, h_ptr.data(), sizeof(int32_t) * ncolour, cudaMemcpyHostToDevice, s));
    k_colour_place<<<gridc(n), kBlock, 0, s>>>(n, colour, base.p, cursor.p, rows.p); ::pc::count_launches(1);
    PC_LAUNCH("colour_place");
    sync(c);
}

}  // namespace pc
