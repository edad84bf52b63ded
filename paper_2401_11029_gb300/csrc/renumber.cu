// Vertex renumbering on the device (cflr_load_graph).
//
// The order is the breadth-first order of the edges taken as undirected that
// a one-thread queue search gives: components in the order of their smallest
// vertex, each searched from that vertex, the neighbours of a vertex in edge
// order (the edge index, then its source side before its destination side;
// the two entries a self-loop gives are the same vertex).  Consecutive ids
// then go to vertices that reach one another, so a closure row falls into
// few 32-bit words of the tile lists.
//
// Steps: an undirected adjacency (CSR) whose lists hold (edge index << 32 |
// neighbour) and are sorted; connected components by hooking the larger of
// two roots under the smaller and pointer jumping, so every component's root
// is its smallest vertex; a breadth-first search from all roots at once.  In
// level L the frontier is sorted by root and, within a root, by the order of
// the search.  An unseen neighbour v goes to the frontier vertex that reaches
// it first in that order: the smallest key (frontier position << 32 | list
// position) that claims it.  Each frontier vertex then writes the vertices it
// won, in list order, at a scanned offset, so the next frontier keeps the
// order the queue search would give it.  A vertex's final position is its
// component's offset, plus the vertices of its component in earlier levels,
// plus its rank in its component's part of its level; per-root tables of the
// frontier segments (first, end, earlier count), kept for two levels, give
// both without a pass of their own.
#include "kernels.cuh"

#include <mutex>

namespace cflr {

namespace {

constexpr uint32_t RN_UNSEEN = 0xFFFFFFFFu;

inline int rn_grid(unsigned long long items, int per_block, int sms, int mult) {
    unsigned long long g = (items + per_block - 1) / per_block;
    const unsigned long long cap = (unsigned long long)sms * mult;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

// Degrees of the undirected graph (a self-loop counts twice) and the largest.
__global__ void k_rn_degree(const uint32_t *src, const uint32_t *dst, unsigned long long m,
                            uint32_t *deg) {
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (unsigned long long)gridDim.x * blockDim.x) {
        atomicAdd(&deg[src[e]], 1u);
        atomicAdd(&deg[dst[e]], 1u);
    }
}

__global__ void k_rn_max(const uint32_t *deg, uint32_t n, uint32_t *out) {
    uint32_t mx = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        mx = max(mx, deg[v]);
    mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

// Adjacency entries (edge << 32 | neighbour), in any order within a list.
__global__ void k_rn_fill(const uint32_t *src, const uint32_t *dst, unsigned long long m,
                          unsigned long long *cur, unsigned long long *adj) {
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t s = src[e], d = dst[e];
        adj[atomicAdd(&cur[s], 1ull)] = (e << 32) | d;
        adj[atomicAdd(&cur[d], 1ull)] = (e << 32) | s;
    }
}

// Sort the lists of up to 32 entries in registers (a warp per list); longer
// ones are listed for k_rn_sort_big.
__global__ void __launch_bounds__(256) k_rn_sort_small(const unsigned long long *off, uint32_t n,
                                                       unsigned long long *adj, uint32_t *big,
                                                       uint32_t *big_n) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < n; v += warps) {
        const unsigned long long a = off[v], d = off[v + 1] - a;
        if (d <= 1) continue;
        if (d > 32) {
            if (lane == 0) big[atomicAdd(big_n, 1u)] = v;
            continue;
        }
        unsigned long long x = (unsigned long long)lane < d ? adj[a + lane] : ~0ull;
#pragma unroll
        for (uint32_t k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, x, j);
                const bool up = (lane & k) == 0, lower = (lane & j) == 0;
                x = (lower == up) ? min(x, y) : max(x, y);
            }
        }
        if ((unsigned long long)lane < d) adj[a + lane] = x;
    }
}

// Sort the listed longer lists, a CTA each, by a bitonic sort of P entries in
// shared memory (P: the next power of two, at most the launch's size).
__global__ void __launch_bounds__(256) k_rn_sort_big(const unsigned long long *off,
                                                     unsigned long long *adj, const uint32_t *big,
                                                     const uint32_t *big_n) {
    extern __shared__ unsigned long long sk[];
    const uint32_t nb = *big_n;
    for (uint32_t r = blockIdx.x; r < nb; r += gridDim.x) {
        const uint32_t v = big[r];
        const unsigned long long a = off[v];
        const uint32_t d = (uint32_t)(off[v + 1] - a);
        uint32_t P = 64;
        while (P < d) P <<= 1;
        for (uint32_t t = threadIdx.x; t < P; t += blockDim.x) sk[t] = t < d ? adj[a + t] : ~0ull;
        __syncthreads();
        for (uint32_t k = 2; k <= P; k <<= 1) {
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                for (uint32_t q = threadIdx.x; q < P / 2; q += blockDim.x) {
                    const uint32_t t = ((q & ~(j - 1)) << 1) | (q & (j - 1));
                    const unsigned long long x = sk[t], y = sk[t | j];
                    const bool up = (t & k) == 0;
                    if ((x > y) == up) {
                        sk[t] = y;
                        sk[t | j] = x;
                    }
                }
                __syncthreads();
            }
        }
        for (uint32_t t = threadIdx.x; t < d; t += blockDim.x) adj[a + t] = sk[t];
        __syncthreads();
    }
}

__global__ void k_rn_init(uint32_t n, uint32_t *parent, uint32_t *lvl, unsigned long long *key,
                          uint32_t *iperm) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        parent[v] = v;
        lvl[v] = RN_UNSEEN;
        key[v] = ~0ull;
        iperm[v] = RN_UNSEEN;
    }
}

// Pointer jumping: every vertex to its root (parents always have smaller
// ids, so the chains end).  *more is set when a chain was left unfinished.
__global__ void k_rn_compress(uint32_t *parent, uint32_t n, unsigned *more) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint32_t x = parent[v];
        for (int it = 0; it < 4096 && parent[x] != x; it++) x = parent[x];
        if (parent[x] != x) *more = 1;
        parent[v] = x;
    }
}

// Hooking: for an edge between two components, the larger root goes under
// the smaller (a root that another edge hooked in the same pass may lose that
// link; its edge then hooks again in the next pass).
__global__ void k_rn_hook(const uint32_t *src, const uint32_t *dst, unsigned long long m,
                          uint32_t *parent, unsigned *more) {
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t ru = parent[src[e]], rv = parent[dst[e]];
        if (ru != rv) {
            atomicMin(&parent[max(ru, rv)], min(ru, rv));
            *more = 1;
        }
    }
}

// Component sizes (by root) and the root flags.
__global__ void k_rn_count(const uint32_t *parent, uint32_t n, uint32_t *cnt, uint32_t *is_root) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        atomicAdd(&cnt[parent[v]], 1u);
        is_root[v] = parent[v] == v ? 1u : 0u;
    }
}

// Level 0: the roots in id order, each first in its component.
__global__ void k_rn_roots(const uint32_t *parent, uint32_t n, const unsigned long long *roff,
                           const unsigned long long *comp_off, uint32_t *F, uint32_t *lvl,
                           uint32_t *sf, uint32_t *se, uint32_t *pc, uint32_t *perm,
                           uint32_t *iperm) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (parent[v] != v) continue;
        const uint32_t q = (uint32_t)roff[v];
        F[q] = v;
        lvl[v] = 0;
        sf[v] = q;
        se[v] = q + 1;
        pc[v] = 0;
        const uint32_t pos = (uint32_t)comp_off[v];
        iperm[pos] = v;
        perm[v] = pos;
    }
}

// Claims of one level: every unseen neighbour takes the smallest key.
__global__ void __launch_bounds__(256) k_rn_claim(const uint32_t *F, uint32_t fsize,
                                                  const unsigned long long *off,
                                                  const unsigned long long *adj,
                                                  const uint32_t *lvl, unsigned long long *key) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < fsize; q += warps) {
        const uint32_t u = F[q];
        const unsigned long long a = off[u], b = off[u + 1];
        for (unsigned long long j = a + lane; j < b; j += 32) {
            const uint32_t v = (uint32_t)adj[j];
            if (lvl[v] == RN_UNSEEN)
                atomicMin(&key[v], ((unsigned long long)q << 32) | (uint32_t)(j - a));
        }
    }
}

// The vertices each frontier vertex won.
__global__ void __launch_bounds__(256) k_rn_won(const uint32_t *F, uint32_t fsize,
                                                const unsigned long long *off,
                                                const unsigned long long *adj,
                                                const uint32_t *lvl,
                                                const unsigned long long *key, uint32_t *won) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < fsize; q += warps) {
        const uint32_t u = F[q];
        const unsigned long long a = off[u], b = off[u + 1];
        uint32_t c = 0;
        for (unsigned long long j = a + lane; j < b; j += 32) {
            const uint32_t v = (uint32_t)adj[j];
            c += lvl[v] == RN_UNSEEN &&
                 key[v] == (((unsigned long long)q << 32) | (uint32_t)(j - a));
        }
        c = __reduce_add_sync(0xFFFFFFFFu, c);
        if (lane == 0) won[q] = c;
    }
}

// The next frontier (won vertices in list order from woff[q]) and the final
// positions of its vertices; the segment-start warp of each root carries the
// root's segment table to the next level.
__global__ void __launch_bounds__(256) k_rn_write(
    const uint32_t *F, uint32_t fsize, const unsigned long long *off,
    const unsigned long long *adj, uint32_t *lvl, const unsigned long long *key,
    const unsigned long long *woff, uint32_t *F2, uint32_t level, const uint32_t *parent,
    const unsigned long long *comp_off, const uint32_t *sf, const uint32_t *se,
    const uint32_t *pc, uint32_t *sf2, uint32_t *se2, uint32_t *pc2, uint32_t *perm,
    uint32_t *iperm, uint32_t n) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < fsize; q += warps) {
        const uint32_t u = F[q], r = parent[u];
        const uint32_t s0 = sf[r], s1 = se[r];
        const unsigned long long wbase = woff[s0];
        if (q == s0 && lane == 0) {
            sf2[r] = (uint32_t)wbase;
            se2[r] = (uint32_t)woff[s1];
            pc2[r] = pc[r] + (s1 - s0);
        }
        // first final position of the root's vertices of the next level
        const unsigned long long pos0 = comp_off[r] + pc[r] + (s1 - s0);
        unsigned long long t = woff[q];
        const unsigned long long a = off[u], b = off[u + 1];
        for (unsigned long long jb = a; jb < b; jb += 32) {
            const unsigned long long j = jb + lane;
            uint32_t v = 0;
            bool w = false;
            if (j < b) {
                v = (uint32_t)adj[j];
                w = lvl[v] == RN_UNSEEN &&
                    key[v] == (((unsigned long long)q << 32) | (uint32_t)(j - a));
            }
            const unsigned m = __ballot_sync(0xFFFFFFFFu, w);
            if (w) {
                // (positions stay below n whenever the component counts are
                // right; k_rn_check reports a position left unwritten)
                const unsigned long long tt = t + __popc(m & ((1u << lane) - 1));
                const unsigned long long pos = pos0 + (tt - wbase);
                lvl[v] = level + 1;
                if (tt < n) F2[tt] = v;
                if (pos < n) {
                    iperm[pos] = v;
                    perm[v] = (uint32_t)pos;
                }
            }
            t += __popc(m);
        }
    }
}

// *bad = 1 unless perm and iperm are inverse permutations of 0..n-1.
__global__ void k_rn_check(const uint32_t *perm, const uint32_t *iperm, uint32_t n,
                           unsigned *bad) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint32_t v = iperm[k];
        if (v >= n || perm[v] != k) *bad = 1;
    }
}

}  // namespace

void launch_rn_adjacency(const uint32_t *src, const uint32_t *dst, unsigned long long m,
                         uint32_t n, uint32_t *deg, uint32_t *max_deg, int sms, cudaStream_t st) {
    cudaMemsetAsync(deg, 0, (size_t)n * 4, st);
    cudaMemsetAsync(max_deg, 0, 4, st);
    if (m) k_rn_degree<<<rn_grid(m, 256, sms, 8), 256, 0, st>>>(src, dst, m, deg);
    if (n) k_rn_max<<<rn_grid(n, 256, sms, 4), 256, 0, st>>>(deg, n, max_deg);
}

void launch_rn_fill(const uint32_t *src, const uint32_t *dst, unsigned long long m, uint32_t n,
                    const unsigned long long *off, unsigned long long *cur,
                    unsigned long long *adj, uint32_t *big, uint32_t *big_n, uint32_t max_deg,
                    int sms, cudaStream_t st) {
    cudaMemcpyAsync(cur, off, (size_t)n * 8, cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(big_n, 0, 4, st);
    if (m) k_rn_fill<<<rn_grid(m, 256, sms, 8), 256, 0, st>>>(src, dst, m, cur, adj);
    if (!n) return;
    k_rn_sort_small<<<rn_grid(n, 8, sms, 16), 256, 0, st>>>(off, n, adj, big, big_n);
    if (max_deg > 32) {
        uint32_t P = 64;
        while (P < max_deg) P <<= 1;
        static std::mutex mu;
        static bool done[64] = {};
        int dev = 0;
        cudaGetDevice(&dev);
        {
            std::lock_guard<std::mutex> lock(mu);
            if (dev >= 0 && dev < 64 && !done[dev]) {
                cudaFuncSetAttribute(k_rn_sort_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(RENUM_LIST_MAX * 8));
                done[dev] = true;
            }
        }
        k_rn_sort_big<<<sms * 2, 256, (size_t)P * 8, st>>>(off, adj, big, big_n);
    }
}

void launch_rn_init(uint32_t n, uint32_t *parent, uint32_t *lvl, unsigned long long *key,
                    uint32_t *iperm, int sms, cudaStream_t st) {
    if (n) k_rn_init<<<rn_grid(n, 256, sms, 4), 256, 0, st>>>(n, parent, lvl, key, iperm);
}

void launch_rn_cc_pass(const uint32_t *src, const uint32_t *dst, unsigned long long m,
                       uint32_t n, uint32_t *parent, unsigned *more, int sms, cudaStream_t st) {
    cudaMemsetAsync(more, 0, 4, st);
    if (n) k_rn_compress<<<rn_grid(n, 256, sms, 4), 256, 0, st>>>(parent, n, more);
    if (m) k_rn_hook<<<rn_grid(m, 256, sms, 8), 256, 0, st>>>(src, dst, m, parent, more);
}

void launch_rn_count(const uint32_t *parent, uint32_t n, uint32_t *cnt, uint32_t *is_root,
                     int sms, cudaStream_t st) {
    cudaMemsetAsync(cnt, 0, (size_t)n * 4, st);
    if (n) k_rn_count<<<rn_grid(n, 256, sms, 4), 256, 0, st>>>(parent, n, cnt, is_root);
}

void launch_rn_roots(const uint32_t *parent, uint32_t n, const unsigned long long *roff,
                     const unsigned long long *comp_off, uint32_t *F, uint32_t *lvl, uint32_t *sf,
                     uint32_t *se, uint32_t *pc, uint32_t *perm, uint32_t *iperm, int sms,
                     cudaStream_t st) {
    if (n)
        k_rn_roots<<<rn_grid(n, 256, sms, 4), 256, 0, st>>>(parent, n, roff, comp_off, F, lvl, sf,
                                                             se, pc, perm, iperm);
}

void launch_rn_claim(const uint32_t *F, uint32_t fsize, const unsigned long long *off,
                     const unsigned long long *adj, const uint32_t *lvl, unsigned long long *key,
                     uint32_t *won, int sms, cudaStream_t st) {
    if (!fsize) return;
    const int g = rn_grid(fsize, 8, sms, 16);
    k_rn_claim<<<g, 256, 0, st>>>(F, fsize, off, adj, lvl, key);
    k_rn_won<<<g, 256, 0, st>>>(F, fsize, off, adj, lvl, key, won);
}

void launch_rn_write(const uint32_t *F, uint32_t fsize, const unsigned long long *off,
                     const unsigned long long *adj, uint32_t *lvl, const unsigned long long *key,
                     const unsigned long long *woff, uint32_t *F2, uint32_t level,
                     const uint32_t *parent, const unsigned long long *comp_off,
                     const uint32_t *sf, const uint32_t *se, const uint32_t *pc, uint32_t *sf2,
                     uint32_t *se2, uint32_t *pc2, uint32_t *perm, uint32_t *iperm, uint32_t n,
                     int sms, cudaStream_t st) {
    if (!fsize) return;
    k_rn_write<<<rn_grid(fsize, 8, sms, 16), 256, 0, st>>>(F, fsize, off, adj, lvl, key, woff, F2,
                                                          level, parent, comp_off, sf, se, pc,
                                                          sf2, se2, pc2, perm, iperm, n);
}

void launch_rn_check(const uint32_t *perm, const uint32_t *iperm, uint32_t n, unsigned *bad,
                     int sms, cudaStream_t st) {
    cudaMemsetAsync(bad, 0, 4, st);
    if (n) k_rn_check<<<rn_grid(n, 256, sms, 4), 256, 0, st>>>(perm, iperm, n, bad);
}

}  // namespace cflr
