// CUDA kernels of the CFL-reachability closure loop (sm_103a).
//
// One closure iteration of Algorithm 1 with optimisation 1 is, for every
// production c -> a b,  T_c = (dA . B) u (A_old . dB),  dC = T_c \ M_c,
// M_c <- M_c u dC  (paper Sec. 3, optimisations 1 and 2).  The kernels below
// split it into:
//   k_symbolic   work list: one group per (production or indexed family,
//                delta row) with its product steps (referenced tiles),
//                binned by the shared memory its accumulator needs
//   k_spgemm_*   the boolean products of a group with the mask fused:
//                a shared-memory set of the mask row plus the products;
//                a product is emitted only when the set did not hold it
//   k_commit     dedupe across groups into the per-non-terminal hash set;
//                the winners are the new pairs dC, counted per row
//   k_reset_dnew / k_capacity / k_capacity_big / k_scatter / k_pack
//                the union M_c u dC in the row and column forms: rows are
//                lists of 32-bit tiles with slack; a row that lacks room
//                moves (folding its tiles), the new pairs are appended and
//                packed into tiles, so a union touches only the rows that
//                grow (the role optimisation 3 plays)
// All work is integer; the result does not depend on thread timing.
#include "kernels.cuh"

#include <algorithm>
#include <cstdio>
#include <mutex>

namespace cflr {

#define FULL_MASK 0xFFFFFFFFu

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

// 64-bit mixer (the MurmurHash3 64-bit finaliser).
__device__ __forceinline__ unsigned long long hmix(unsigned long long k);
// Home slot of a pair key (i << 32 | j) in a pair set: the 32 columns of one
// 32-bit word of a row share an aligned block of 32 slots, so the pairs one
// tile emits land in one or two cache lines.
__device__ __forceinline__ unsigned long long pair_home(unsigned long long key,
                                                        unsigned long long m) {
    return ((hmix(key >> 5) << 5) | (key & 31)) & m;
}
__device__ __forceinline__ unsigned long long hmix(unsigned long long k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

// Position of the n-th (from 0) set bit of m; m has more than n set bits.
__device__ __forceinline__ uint32_t select_bit(uint32_t m, uint32_t n) {
    uint32_t pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const uint32_t c = __popc(m & ((1u << w) - 1));
        if (n >= c) {
            n -= c;
            m >>= w;
            pos += w;
        }
    }
    return pos;
}

// A row descriptor of `slot` that lies inside its instance's pool (checked
// builds; always true otherwise): 16-byte aligned, tiles within the capacity,
// tile and entry sections within the pool.
__device__ __forceinline__ bool row_in_pool(const SlotTab &S, uint32_t slot, uint4 d,
                                            unsigned *err) {
#if defined(CFLR_CHECKED)
    const unsigned long long end = (unsigned long long)d.x + tile_words(d.z) +
                                   (d.z ? entry_cap(d) : 0ull);
    return CFLR_CHECK((d.x & 3u) == 0 && d.y <= d.z && end <= S.pool_cap[S.inst[slot]], err);
#else
    return true;
#endif
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t t = __shfl_up_sync(FULL_MASK, v, d);
        if (lane >= d) v += t;
    }
    return v;
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(FULL_MASK, v, d);
    return v;
}

// Accumulators of one output row.  Products arrive as 32-bit tiles (word w,
// bits b: the columns 32w + i for every set bit i of b); a single column v is
// the one-bit tile (v >> 5, 1 << (v & 31)).  ins() adds a tile and returns
// the bits that were not present yet.  Nearly every product is already
// present (masked or repeated), so a tile is tested with a plain
// shared-memory read first and the atomic runs only when a bit is missing.

// Open-addressing table of 2^lg slots (word, bits), interleaved so that
// one 16-byte store clears two slots (clear_table); the caller keeps the
// load <= 1/2.
struct HashAcc {
    uint32_t *tab;
    int lg;
    unsigned *err;     // gets OVF_FULL if a probe sequence finds the table full
    __device__ __forceinline__ uint32_t ins(uint32_t w, uint32_t b) const {
        const uint32_t m = (1u << lg) - 1;
        uint32_t s = (w * 2654435761u) >> (32 - lg);
        // at most one pass over the table (the callers keep it at most half
        // full, so the pass always ends early)
        for (uint32_t p = 0;; p++) {
            if (p > m) {
                atomicOr(err, OVF_FULL);
                return 0;
            }
            const uint32_t cur = ((volatile uint32_t *)tab)[2 * s];
            if (cur == w) break;
            if (cur == EMPTY32) {
                const uint32_t old = atomicCAS(&tab[2 * s], EMPTY32, w);
                if (old == EMPTY32 || old == w) break;
            }
            s = (s + 1) & m;
        }
        const uint32_t ob = ((volatile uint32_t *)tab)[2 * s + 1];
        if ((ob & b) == b) return 0;
        return b & ~atomicOr(&tab[2 * s + 1], b);
    }
    __device__ __forceinline__ void set(uint32_t w, uint32_t b) const { ins(w, b); }
};

// Empty all 2^lg slots of a table (16-byte aligned, lg >= 1); thread tid of nth.
__device__ __forceinline__ void clear_table(uint32_t *tab, uint32_t lg, uint32_t tid,
                                            uint32_t nth) {
    uint4 *t4 = reinterpret_cast<uint4 *>(tab);
    for (uint32_t s = tid; s < (1u << lg) / 2; s += nth)
        t4[s] = make_uint4(EMPTY32, 0u, EMPTY32, 0u);
}

// n-bit bitmap of the row (bin 3).
struct BitmapAcc {
    uint32_t *bm;
#if defined(CFLR_CHECKED)
    uint32_t words;     // the row's words (checked builds)
    unsigned *err;
#endif
    __device__ __forceinline__ uint32_t ins(uint32_t w, uint32_t b) const {
#if defined(CFLR_CHECKED)
        if (!CFLR_CHECK(w < words, err)) return 0;
#endif
        const uint32_t ob = ((volatile uint32_t *)bm)[w];
        if ((ob & b) == b) return 0;
        return b & ~atomicOr(&bm[w], b);
    }
    // bits whose newness nobody asks (the mask row): one atomic, no read
    __device__ __forceinline__ void set(uint32_t w, uint32_t b) const {
#if defined(CFLR_CHECKED)
        if (!CFLR_CHECK(w < words, err)) return;
#endif
        atomicOr(&bm[w], b);
    }
};

// Whether a pair set holds `key`; a probe sequence that passes over the
// whole table (a full set: k_check keeps every set at most half full) ends
// with OVF_FULL in *err.
__device__ __forceinline__ bool htab_contains(const unsigned long long *tab,
                                              unsigned long long m, unsigned long long key,
                                              unsigned *err) {
    unsigned long long h = pair_home(key, m);
    for (unsigned long long p = 0; p <= m; p++) {
        unsigned long long v = tab[h];
        if (v == key) return true;
        if (v == EMPTY_KEY) return false;
        h = (h + 1) & m;
    }
    atomicOr(err, OVF_FULL);
    return false;
}

// Warp-collective append of flagged keys to the candidate buffer.  All 32
// lanes must call it.  Returns (in every lane) the number appended.
__device__ __forceinline__ uint32_t emit_candidates(bool flag, unsigned long long key,
                                                    uint32_t slot, const WorkBufs &W,
                                                    int lane, uint2 wit) {
    const unsigned m = __ballot_sync(FULL_MASK, flag);
    if (!m) return 0;
    const uint32_t cnt = __popc(m);
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&W.cnt->cand, (unsigned long long)cnt);
    base = __shfl_sync(FULL_MASK, base, 0);
    if (flag) {
        unsigned long long pos = base + __popc(m & ((1u << lane) - 1));
        if (pos < W.cand_cap) {
            W.cand_key[pos] = key;
            W.cand_slot[pos] = slot;
            if (W.cand_wit) W.cand_wit[pos] = wit;
        }
    }
    if (lane == 0 && base + cnt > W.cand_cap) atomicOr(&W.cnt->overflow, OVF_CAND);
    return cnt;
}

// A warp's reservation in the candidate buffer: entries [pos, end) are its
// own.  The product kernels reserve CAND_CHUNK entries (or more) at a time,
// so most emits take no atomic on the shared count; what a warp leaves
// unused when it ends is marked empty (slot EMPTY32) for the commit.
struct CandChunk {
    unsigned long long pos, end;
};
constexpr unsigned long long CAND_CHUNK = 64;

// Warp-collective: mark the rest of the warp's reservation empty.
__device__ __forceinline__ void release_chunk(const WorkBufs &W, const CandChunk &ck, int lane) {
    if (ck.pos >= ck.end) return;
    for (unsigned long long q = ck.pos + lane; q < ck.end; q += 32)
        if (q < W.cand_cap) W.cand_slot[q] = EMPTY32;
    if (lane == 0) atomicAdd(&W.cnt->holes, ck.end - ck.pos);
}

// Exclusive scan over the 256 threads of a block; `total` gets the block sum.
__device__ __forceinline__ unsigned long long block_excl_scan256(unsigned long long v,
                                                                 unsigned long long *sh,
                                                                 unsigned long long &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        unsigned long long t = __shfl_up_sync(FULL_MASK, x, d);
        if (lane >= d) x += t;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long y = lane < 8 ? sh[lane] : 0;
#pragma unroll
        for (int d = 1; d < 8; d <<= 1) {
            unsigned long long t = __shfl_up_sync(FULL_MASK, y, d);
            if (lane >= d) y += t;
        }
        if (lane < 8) sh[8 + lane] = y;
    }
    __syncthreads();
    total = sh[15];
    const unsigned long long before = (w ? sh[8 + w - 1] : 0ull) + x - v;
    __syncthreads();
    return before;
}

// ---------------------------------------------------------------------------
// k_symbolic: groups of this iteration, binned by shared-memory need
// ---------------------------------------------------------------------------

constexpr int SYM_BUF = 16;   // per-warp staging of groups before one atomic

// Product steps (referenced tiles) of one use and their bytes, over the
// delta entries q0, q0 + qstep, ... (pool[dstart + q], q < d): each entry k
// references row k of slot g in orientation o, counted only when the row's
// occupancy bit says it is non-empty.
struct Work {
    unsigned long long f, fb;
};

__device__ __forceinline__ Work gathered_work(const SlotTab &S, uint32_t g, uint32_t o, uint32_t n,
                                              const uint32_t *pool, uint32_t dstart, uint32_t d,
                                              uint32_t q0, uint32_t qstep, unsigned *err) {
    const uint4 *dg = S.desc[g] + (size_t)o * n;
    const uint32_t *oc = S.occ[g];
    const uint32_t ow = S.occ_w[g], lx = S.local[g];
    const uint32_t bit = 1u << (lx & 31);
    Work w{0, 0};
    if (qstep == 1) {
        // one lane over all entries: four entries' loads in flight together
        for (uint32_t q = q0; q < d; q += 4) {
            uint32_t k[4], ob[4];
            uint4 gd[4];
#pragma unroll
            for (int t = 0; t < 4; t++) {
                k[t] = q + t < d ? pool[dstart + q + t] : 0u;
                if (!CFLR_CHECK(k[t] < n, err)) k[t] = 0;
            }
#pragma unroll
            for (int t = 0; t < 4; t++)
                ob[t] = q + t < d ? oc[((size_t)o * n + k[t]) * ow + (lx >> 5)] & bit : 0u;
#pragma unroll
            for (int t = 0; t < 4; t++) gd[t] = ob[t] ? dg[k[t]] : make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int t = 0; t < 4; t++) {
                if (!ob[t]) continue;
                const uint32_t nt = gd[t].y - (o ? (gd[t].w & DLAST_MASK) : 0u);
                w.f += nt;
                w.fb += 16ull + 8ull * nt;
            }
        }
        return w;
    }
    for (uint32_t q = q0; q < d; q += qstep) {
        const uint32_t k = pool[dstart + q];
        if (!CFLR_CHECK(k < n, err)) continue;
        if (oc[((size_t)o * n + k) * ow + (lx >> 5)] & bit) {
            // column form (o = 1): A_old, the tiles before the last merge's
            const uint4 gd = dg[k];
            const uint32_t nt = gd.y - (o ? (gd.w & DLAST_MASK) : 0u);
            w.f += nt;
            w.fb += 16ull + 8ull * nt;
        }
    }
    return w;
}

// The same for a family on its shared operand's delta (optimisation 4): the
// members reference the consecutive slots g0 .. g0+F-1, whose occupancy bits
// are consecutive, so a few words per entry say which members have a row.
__device__ __forceinline__ Work family_work(const SlotTab &S, uint32_t g0, uint32_t F, uint32_t o,
                                            uint32_t n, const uint32_t *pool, uint32_t dstart,
                                            uint32_t d, uint32_t q0, uint32_t qstep,
                                            unsigned *err) {
    const uint32_t *oc = S.occ[g0];
    const uint32_t ow = S.occ_w[g0], lx0 = S.local[g0];
    Work w{0, 0};
    if (qstep == 32 && F >= 16 && d <= 32) {
        // a whole warp on a short delta (lane q0 of 32): the lanes take the
        // members of each entry in turn, so the members' descriptors load
        // together instead of one after another on the entry's lane
        for (uint32_t q = 0; q < d; q++) {
            const uint32_t k = pool[dstart + q];
            if (!CFLR_CHECK(k < n, err)) continue;
            const uint32_t *ok = oc + ((size_t)o * n + k) * ow;
            for (uint32_t i = q0; i < F; i += 32) {
                const uint32_t x = lx0 + i;
                if ((ok[x >> 5] >> (x & 31)) & 1u) {
                    const uint4 gd = S.desc[g0 + i][(size_t)o * n + k];
                    const uint32_t nt = gd.y - (o ? (gd.w & DLAST_MASK) : 0u);
                    w.f += nt;
                    w.fb += 16ull + 8ull * nt;
                }
            }
        }
        return w;
    }
    for (uint32_t q = q0; q < d; q += qstep) {
        const uint32_t k = pool[dstart + q];
        if (!CFLR_CHECK(k < n, err)) continue;
        const uint32_t *ok = oc + ((size_t)o * n + k) * ow;
        for (uint32_t wi = lx0 >> 5; wi <= (lx0 + F - 1) >> 5; wi++) {
            const uint32_t lo = wi * 32;
            uint32_t m = ok[wi];
            if (lx0 > lo) m &= ~0u << (lx0 - lo);
            if (lx0 + F < lo + 32) m &= (1u << (lx0 + F - lo)) - 1;
            while (m) {
                // up to four members' descriptors in flight together
                uint4 gd[4];
                uint32_t cnt = 0;
#pragma unroll
                for (int t = 0; t < 4; t++) {
                    gd[t] = make_uint4(0, 0, 0, 0);
                    if (m) {
                        const uint32_t i = lo + (__ffs(m) - 1) - lx0;
                        m &= m - 1;
                        gd[t] = S.desc[g0 + i][(size_t)o * n + k];
                        cnt++;
                    }
                }
#pragma unroll
                for (int t = 0; t < 4; t++) {
                    const uint32_t nt = gd[t].y - (o ? (gd[t].w & DLAST_MASK) : 0u);
                    w.f += nt;
                    w.fb += 8ull * nt;
                }
                w.fb += 16ull * cnt;
            }
        }
    }
    return w;
}

// Per-member product steps of a family on one delta row (thread tid of nth
// working on it; members' gathered slots g0 .. g0+F-1, F <= 64): mf[i] and
// mc[i] (zeroed by the caller, shared by the nth threads) get the tiles and
// the referenced rows of member i.  Threads take the entries, four at a
// time; the (entry, member) pairs whose occupancy bit is set are taken
// FM_BATCH at a time across a lane's entries, their descriptors loading
// together.
// The members' descriptor arrays follow one another (the slots of one
// instance are consecutive, 2n descriptors each), so member i's row k of
// orientation o is S.desc[g0][(2i + o) n + k].
constexpr int FM_BATCH = 4;

__device__ __forceinline__ void family_members(const SlotTab &S, uint32_t g0, uint32_t F,
                                               uint32_t o, uint32_t n, const uint32_t *pool,
                                               uint32_t dstart, uint32_t d, uint32_t tid,
                                               uint32_t nth, unsigned long long *mf,
                                               uint32_t *mc, unsigned *err) {
    const uint32_t *oc = S.occ[g0];
    const uint4 *dg = S.desc[g0];
    const uint32_t ow = S.occ_w[g0], lx0 = S.local[g0];
    const uint32_t w0 = lx0 >> 5, sh = lx0 & 31, wlast = (lx0 + F - 1) >> 5;
    const unsigned long long fmask = F == 64 ? ~0ull : (1ull << F) - 1;
    const size_t oo = (size_t)o * n;
    for (uint32_t qb = 0; qb < d; qb += nth * 4) {
        uint32_t k[4];
        unsigned long long m[4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const uint32_t q = qb + nth * t + tid;
            k[t] = q < d ? pool[dstart + q] : 0u;
            if (!CFLR_CHECK(k[t] < n, err)) k[t] = d;   // skipped below
        }
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const uint32_t q = qb + nth * t + tid;
            m[t] = 0;
            if (q < d && k[t] < n) {
                const uint32_t *ok = oc + (oo + k[t]) * ow + w0;
                const uint32_t x0 = ok[0];
                const uint32_t x1 = w0 + 1 <= wlast ? ok[1] : 0u;
                const uint32_t x2 = w0 + 2 <= wlast ? ok[2] : 0u;
                const unsigned long long lo64 = ((unsigned long long)x1 << 32) | x0;
                m[t] = ((lo64 >> sh) | (sh ? (unsigned long long)x2 << (64 - sh) : 0ull)) & fmask;
            }
        }
        while (m[0] | m[1] | m[2] | m[3]) {
            uint32_t mi[FM_BATCH], mk[FM_BATCH];
            uint4 gd[FM_BATCH];
#pragma unroll
            for (int j = 0; j < FM_BATCH; j++) {
                // the lowest pair left in the first entry with pairs left
                const int t = m[0] ? 0 : m[1] ? 1 : m[2] ? 2 : m[3] ? 3 : 4;
                const unsigned long long cur = t == 0 ? m[0] : t == 1 ? m[1] : t == 2 ? m[2]
                                                                                  : m[3];
                mi[j] = t < 4 ? (uint32_t)(__ffsll((long long)cur) - 1) : EMPTY32;
                mk[j] = t == 0 ? k[0] : t == 1 ? k[1] : t == 2 ? k[2] : k[3];
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (t == u) m[u] &= m[u] - 1;
            }
#pragma unroll
            for (int j = 0; j < FM_BATCH; j++)
                gd[j] = mi[j] != EMPTY32 ? dg[(size_t)(2 * mi[j]) * n + oo + mk[j]]
                                         : make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int j = 0; j < FM_BATCH; j++) {
                if (mi[j] == EMPTY32) continue;
                const uint32_t nt = gd[j].y - (o ? (gd[j].w & DLAST_MASK) : 0u);
                atomicAdd(&mf[mi[j]], (unsigned long long)nt);
                atomicAdd(&mc[mi[j]], 1u);
            }
        }
    }
}

__device__ __forceinline__ Work warp_sum(Work w) {
    w.f = warp_sum64(w.f);
    w.fb = warp_sum64(w.fb);
    return w;
}

// prod_only >= 0 restricts the work list to one production (the plain form).
// Mode 0: a warp per touched row; a row whose delta has more than SYM_BIG_D
// entries, or more than SYM_MIN_D entries and more than SYM_BIG_W descriptor
// reads (entries times the members of its uses, a use of one production
// counting as one), is listed for mode 1 (while the list has room) instead.
// Mode 1: a CTA per listed row, its threads sharing the entries (a long
// delta row on one warp would hold the launch up long after the other warps
// finish).
constexpr uint32_t SYM_BIG_D = 1024, SYM_MIN_D = 64, SYM_BIG_W = 32768;

__global__ void __launch_bounds__(256, 4) k_symbolic(SlotTab S, ProdTab P, WorkBufs W,
                                                     int prod_only, Tuning T, int mode) {
    __shared__ Work red[8];
    __shared__ unsigned long long mem_f[8][64];   // per-member sums of a family (a warp's)
    __shared__ uint32_t mem_c[8][64];
    __shared__ uint2 stage[8][N_BINS][SYM_BUF];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int par = *W.parity;
    const unsigned long long n_in = W.touched_n[par];
    const uint2 *t_in = W.touched[par];
    int fill[N_BINS] = {0, 0, 0, 0};
    unsigned long long bytes[N_BINS] = {0, 0, 0, 0};
    unsigned long long flops = 0, sym_bytes = 0;
    unsigned long long flops3 = 0, mask3 = 0;   // the bitmap bin's product and mask tiles

    auto flush = [&](int b) {   // lane 0 only
        unsigned long long pos = atomicAdd(&W.cnt->groups[b], (unsigned long long)fill[b]);
        for (int q = 0; q < fill[b]; q++) {
            if (pos + q < W.group_cap[b]) W.groups[b][pos + q] = stage[wib][b][q];
        }
        if (pos + fill[b] > W.group_cap[b]) atomicOr(&W.cnt->overflow, OVF_GROUPS);
        fill[b] = 0;
    };
    auto append = [&](int b, uint2 grp) {   // one group, any lane
        const unsigned long long pos = atomicAdd(&W.cnt->groups[b], 1ull);
        if (pos < W.group_cap[b]) W.groups[b][pos] = grp;
        else atomicOr(&W.cnt->overflow, OVF_GROUPS);
    };
    // warp-collective: each lane's group (bin b >= 0) appended, one atomic
    // per bin
    auto append_lanes = [&](int b, uint2 grp) {
#pragma unroll
        for (int bb = 0; bb < N_BINS; bb++) {
            const unsigned m = __ballot_sync(FULL_MASK, b == bb);
            if (!m) continue;
            const int leader = __ffs(m) - 1;
            unsigned long long pos = 0;
            if (lane == leader) pos = atomicAdd(&W.cnt->groups[bb], (unsigned long long)__popc(m));
            pos = __shfl_sync(FULL_MASK, pos, leader);
            if (b == bb) {
                pos += __popc(m & ((1u << lane) - 1));
                if (pos < W.group_cap[bb]) W.groups[bb][pos] = grp;
                else atomicOr(&W.cnt->overflow, OVF_GROUPS);
            }
        }
    };

    // classify one group of f product steps: mode, bin and table size;
    // returns the bin and fills the group record.  Groups of a family whose
    // members write different non-terminals probe their pair sets (there is
    // no single mask row) and stay in the hash bins (force_probe).
    bool acct = true;   // whether this lane adds the group's work and bytes
    auto classify = [&](uint32_t code, uint32_t part, uint32_t idx, uint32_t d, uint32_t mlen,
                        unsigned long long mbytes, unsigned long long f,
                        unsigned long long fbytes, bool force_probe, uint2 &grp) -> int {
        const bool probe =
            force_probe || (unsigned long long)mlen > (unsigned long long)T.probe_ratio * f;
        const unsigned long long need = probe ? f : f + mlen;
        const int b = need <= T.limit[0] ? 0 : need <= T.limit[1] ? 1 : need <= T.limit[2] ? 2 : 3;
        // table of the smallest power of two >= 2*need slots (>= 32)
        uint32_t lg = 5;
        while (b < 3 && (1ull << lg) < 2 * need) lg++;
        grp = make_uint2(((code >> 2) << 8) | (lg << 3) | (probe ? MODE_PROBE : 0u) | part, idx);
        // algorithmic bytes: the delta entries (4 B each), the descriptor
        // (16 B) and tiles (8 B each) of every referenced row, and the mask
        // row's descriptor and tiles when it is loaded
        if (acct) {
            bytes[b] += 4ull * d + fbytes + (probe ? 0ull : mbytes + 16ull);
            sym_bytes += 20ull * d + 40ull;
            flops += f;
            if (b == 3) {
                flops3 += f;
                mask3 += probe ? 0ull : mlen;
            }
        }
        return b;
    };

    // the groups of one use on delta row (o, idx); lanes q0 (step qstep)
    // share the delta entries, `sum` reduces over them, and `emit` takes
    // each group (called on every lane that shares the use)
    auto use_groups = [&](uint32_t code, uint32_t o, uint32_t n, uint32_t idx,
                          const uint32_t *pool, uint32_t dstart, uint32_t d, uint32_t q0,
                          uint32_t qstep, auto sum, auto emit) {
        const uint32_t part = code & 3;
        const size_t r = (size_t)o * n + idx;
        if (part == PART_F) {
            const uint4 fm = P.fam[code >> 2];
            const uint32_t *mp = P.fam_prod + fm.x;
            const uint4 pr0 = P.prod[mp[0]];
            const uint32_t g0 = (fm.w == PART_A) ? pr0.z : pr0.y;
            auto member_slot = [&](uint32_t i) {
                const uint4 pr = P.prod[mp[i]];
                return (fm.w == PART_A) ? pr.z : pr.y;
            };
            if ((fm.z & FAM_CONSEC) && (qstep == 32 || qstep == 256) && fm.y <= 64) {
                // a whole warp (or CTA) on the use: per-member sums first,
                // then the family's group, or one group per member
                const bool cta = qstep == 256;
                auto group_sync = [&]() {
                    if (cta) __syncthreads();
                    else __syncwarp();
                };
                unsigned long long *mf = mem_f[cta ? 0 : wib];
                uint32_t *mc = mem_c[cta ? 0 : wib];
                for (uint32_t i = q0; i < fm.y; i += qstep) {
                    mf[i] = 0;
                    mc[i] = 0;
                }
                group_sync();
                family_members(S, g0, fm.y, o, n, pool, dstart, d, q0, qstep, mf, mc,
                               &W.cnt->overflow);
                group_sync();
                Work wt{0, 0};
                for (uint32_t i = q0; i < fm.y; i += qstep) {
                    wt.f += mf[i];
                    wt.fb += 16ull * mc[i] + 8ull * mf[i];
                }
                const Work wk = sum(wt);
                if (wk.f) {
                    uint2 grp;
                    if (fm.z & FAM_CSHARED) {   // every member writes c: one mask row
                        const uint32_t mt = S.desc[pr0.x][r].y;
                        emit(classify(code, PART_F, idx, d, mt, 8ull * mt, wk.f, wk.fb, false,
                                      grp),
                             grp);
                    } else if (wk.f <= T.limit[2]) {
                        emit(classify(code, PART_F, idx, d, 0, 0, wk.f, wk.fb, true, grp), grp);
                    } else {
                        // too large for a hash bin: one group per member,
                        // the threads taking the members
                        const bool keep_acct = acct;
                        acct = true;
                        for (uint32_t i0 = 0; i0 < fm.y; i0 += qstep) {
                            const uint32_t i = i0 + q0;
                            int b = -1;
                            uint2 mg = make_uint2(0, 0);
                            if (i < fm.y && mf[i]) {
                                const uint32_t mt = S.desc[P.prod[mp[i]].x][r].y;
                                b = classify((mp[i] << 2) | fm.w, fm.w, idx, d, mt, 8ull * mt,
                                             mf[i], 16ull * mc[i] + 8ull * mf[i], false, mg);
                            }
                            if (cta) {
                                if (b >= 0) append(b, mg);
                            } else {
                                append_lanes(b, mg);
                            }
                        }
                        acct = keep_acct;
                    }
                }
                group_sync();
                return;
            }
            Work wk{0, 0};
            if (fm.z & FAM_CONSEC) {
                wk = family_work(S, g0, fm.y, o, n, pool, dstart, d, q0, qstep,
                                 &W.cnt->overflow);
            } else {
                for (uint32_t i = 0; i < fm.y; i++) {
                    const Work wi = gathered_work(S, member_slot(i), o, n, pool, dstart, d, q0,
                                                  qstep, &W.cnt->overflow);
                    wk.f += wi.f;
                    wk.fb += wi.fb;
                }
            }
            wk = sum(wk);
            if (wk.f == 0) return;
            uint2 grp;
            if (fm.z & FAM_CSHARED) {   // every member writes c: one mask row
                const uint32_t mt = S.desc[pr0.x][r].y;
                emit(classify(code, PART_F, idx, d, mt, 8ull * mt, wk.f, wk.fb, false, grp), grp);
            } else if (wk.f <= T.limit[2]) {
                emit(classify(code, PART_F, idx, d, 0, 0, wk.f, wk.fb, true, grp), grp);
            } else if (qstep == 32) {
                // too large for a hash bin: one group per member; with a
                // whole warp on the use, the lanes take the members (each
                // lane counts its member's products over all entries)
                const bool keep_acct = acct;
                acct = true;
                for (uint32_t i0 = 0; i0 < fm.y; i0 += 32) {
                    const uint32_t i = i0 + q0;
                    int b = -1;
                    uint2 mg = make_uint2(0, 0);
                    if (i < fm.y) {
                        const uint4 pr = P.prod[mp[i]];
                        const uint32_t mt = S.desc[pr.x][r].y;
                        const Work wi = gathered_work(S, (fm.w == PART_A) ? pr.z : pr.y, o, n,
                                                      pool, dstart, d, 0, 1, &W.cnt->overflow);
                        if (wi.f)
                            b = classify((mp[i] << 2) | fm.w, fm.w, idx, d, mt, 8ull * mt, wi.f,
                                         wi.fb, false, mg);
                    }
                    append_lanes(b, mg);
                }
                acct = keep_acct;
            } else {               // too large for a hash bin: one group per member
                for (uint32_t i = 0; i < fm.y; i++) {
                    const Work wi = sum(gathered_work(S, member_slot(i), o, n, pool, dstart, d,
                                                      q0, qstep, &W.cnt->overflow));
                    if (wi.f == 0) continue;
                    const uint32_t mt = S.desc[P.prod[mp[i]].x][r].y;
                    emit(classify((mp[i] << 2) | fm.w, fm.w, idx, d, mt, 8ull * mt, wi.f, wi.fb,
                                  false, grp),
                         grp);
                }
            }
            return;
        }
        const uint4 pr = P.prod[code >> 2];
        const uint32_t mt = S.desc[pr.x][r].y;
        Work wk{0, 0};
        if (part == PART_U) {
            wk.f = d;
            wk.fb = 4ull * d;
        } else {
            // gathered rows: b's row form (PART_A) or a's column form (PART_B)
            wk = sum(gathered_work(S, (part == PART_A) ? pr.z : pr.y, o, n, pool, dstart, d, q0,
                                   qstep, &W.cnt->overflow));
        }
        if (wk.f == 0) return;
        uint2 grp;
        emit(classify(code, part, idx, d, mt, 8ull * mt, wk.f, wk.fb, false, grp), grp);
    };

    if (mode == 1) {
        // a CTA per long delta row: the threads share its entries, sums over
        // the CTA, thread 0 classifies and appends
        const unsigned long long n_big = min(W.cnt->big_n, W.big_cap);
        auto block_sum = [&](Work w) {
            w = warp_sum(w);
            __syncthreads();                 // red[] free from the last sum
            if (lane == 0) red[wib] = w;
            __syncthreads();
            Work t{0, 0};
#pragma unroll
            for (int q = 0; q < 8; q++) {
                t.f += red[q].f;
                t.fb += red[q].fb;
            }
            return t;
        };
        acct = threadIdx.x == 0;
        for (unsigned long long e = blockIdx.x; e < n_big; e += gridDim.x) {
            const uint2 t = W.big_rows[e];
            const uint32_t xo = t.x, idx = t.y, slot = xo >> 1, o = xo & 1;
            const uint32_t n = S.n[slot];
            const uint4 dsc = S.desc[slot][(size_t)o * n + idx];
            const uint32_t d = S.dn[slot][(size_t)o * n + idx].x;
            const uint32_t dstart = dsc.x + tile_words(dsc.z);
            const uint32_t *pool = S.pool[slot];
            for (uint32_t u = P.use_off[xo]; u < P.use_off[xo + 1]; u++) {
                const uint32_t code = P.use_code[u];
                if (prod_only >= 0 && (code >> 2) != (uint32_t)prod_only) continue;
                use_groups(code, o, n, idx, pool, dstart, d, threadIdx.x, 256, block_sum,
                           [&](int bb, uint2 g) {
                               if (threadIdx.x == 0) append(bb, g);
                           });
            }
        }
    }
    // a warp per touched row, at a stride: rows the same merge touched lie
    // together in the list and often cost alike (claiming runs of rows from
    // a cursor was measured slower, more so the longer the runs)
    for (unsigned long long e = (unsigned long long)blockIdx.x * 8 + wib; mode == 0 && e < n_in;
         e += (unsigned long long)gridDim.x * 8) {
        const uint2 t = t_in[e];
        const uint32_t xo = t.x, idx = t.y, slot = xo >> 1, o = xo & 1;
        const uint32_t n = S.n[slot];
        const uint4 dsc = S.desc[slot][(size_t)o * n + idx];
        const uint32_t d = S.dn[slot][(size_t)o * n + idx].x;
        const uint32_t dstart = dsc.x + tile_words(dsc.z);
        const uint32_t *pool = S.pool[slot];
        const uint32_t u0 = P.use_off[xo], u1 = P.use_off[xo + 1];
        bool big = d > SYM_BIG_D;
        if (!big && d > SYM_MIN_D) {
            uint32_t w = 0;
            for (uint32_t u = u0 + lane; u < u1; u += 32) {
                const uint32_t code = P.use_code[u];
                w += (code & 3) == PART_F ? P.fam[code >> 2].y : 1u;
            }
            big = (unsigned long long)__reduce_add_sync(FULL_MASK, w) * d > SYM_BIG_W;
        }
        if (big && u1 > u0) {
            // listed for the CTA pass when there is room, else done here
            unsigned long long pos = 0;
            if (lane == 0) pos = atomicAdd(&W.cnt->big_n, 1ull);
            pos = __shfl_sync(FULL_MASK, pos, 0);
            if (pos < W.big_cap) {
                if (lane == 0) W.big_rows[pos] = t;
                continue;
            }
        }
        if (u1 - u0 >= 32 && d <= 16) {
            // many productions read this row, each with few products: one
            // lane per use, groups appended with one atomic per bin
            for (uint32_t ub = u0; ub < u1; ub += 32) {
                const uint32_t u = ub + lane;
                int b = -1;
                uint2 grp = make_uint2(0, 0);
                if (u < u1) {
                    const uint32_t code = P.use_code[u];
                    if (prod_only < 0 || (code >> 2) == (uint32_t)prod_only) {
                        acct = true;
                        // a use yields at most one group, except a split
                        // family, whose member groups are appended at once
                        bool one = true;
                        use_groups(code, o, n, idx, pool, dstart, d, 0, 1,
                                   [](Work w) { return w; },
                                   [&](int bb, uint2 g) {
                                       if (one && b < 0) {
                                           b = bb;
                                           grp = g;
                                       } else {
                                           append(bb, g);
                                       }
                                       one = false;
                                   });
                    }
                }
                append_lanes(b, grp);
            }
            continue;
        }
        for (uint32_t u = u0; u < u1; u++) {
            const uint32_t code = P.use_code[u];
            if (prod_only >= 0 && (code >> 2) != (uint32_t)prod_only) continue;
            // the warp shares the delta entries; lane 0 stages and counts
            // the groups
            acct = lane == 0;
            use_groups(code, o, n, idx, pool, dstart, d, lane, 32,
                       [](Work w) { return warp_sum(w); },
                       [&](int bb, uint2 g) {
                           if (lane == 0) {
                               stage[wib][bb][fill[bb]++] = g;
                               if (fill[bb] == SYM_BUF) flush(bb);
                           }
                       });
        }
    }
    // every lane may hold byte and work counts (lane-per-use mode)
    for (int b = 0; b < N_BINS; b++) bytes[b] = warp_sum64(bytes[b]);
    flops = warp_sum64(flops);
    sym_bytes = warp_sum64(sym_bytes);
    flops3 = warp_sum64(flops3);
    mask3 = warp_sum64(mask3);
    if (lane == 0) {
        for (int b = 0; b < N_BINS; b++) {
            if (fill[b]) flush(b);
            if (bytes[b]) atomicAdd(&W.cnt->bytes_bin[b], bytes[b]);
        }
        if (flops) atomicAdd(&W.cnt->flops, flops);
        if (flops3) atomicAdd(&W.cnt->tiles_bin3[0], flops3);
        if (mask3) atomicAdd(&W.cnt->tiles_bin3[1], mask3);
        if (sym_bytes) atomicAdd(&W.cnt->bytes_sym, sym_bytes);
    }
}

// Group code layout: prod << 8 | log2(table slots) << 3 | probe bit (MODE_PROBE) | part,
// or family << 8 | ... | PART_F for a family's block product.
struct GroupInfo {
    uint32_t part, c, a, b, idx, n, o, lg;
    bool probe;
    // family groups: member i is production P.fam_prod[first + i]; `tagged`
    // when the members write different non-terminals (accumulator keys
    // carry the member); `consec` when the slots of their other operand are
    // consecutive.  A plain group has first = its production.
    bool fam, tagged, consec;
    uint32_t first, F;
};

constexpr uint32_t TAG_SHIFT = 21;   // member << TAG_SHIFT | word (words < 2^21)

__device__ __forceinline__ GroupInfo decode_group(const ProdTab &P, const SlotTab &S,
                                                  uint2 g) {
    GroupInfo gi;
    gi.probe = (g.x & MODE_PROBE) != 0;
    gi.lg = (g.x >> 3) & 31;
    gi.part = g.x & 3;
    gi.fam = gi.part == PART_F;
    gi.tagged = false;
    gi.consec = false;
    gi.first = g.x >> 8;
    gi.F = 1;
    uint32_t p0 = gi.first;
    if (gi.fam) {
        const uint4 fm = P.fam[g.x >> 8];
        gi.part = fm.w;
        gi.first = fm.x;
        gi.F = fm.y;
        gi.tagged = (fm.z & FAM_CSHARED) == 0;
        gi.consec = (fm.z & FAM_CONSEC) != 0;
        p0 = P.fam_prod[fm.x];
    }
    const uint4 pr = P.prod[p0];
    gi.c = pr.x; gi.a = pr.y; gi.b = pr.z;
    gi.idx = g.y;
    gi.n = S.n[gi.c];
    gi.o = (gi.part == PART_B) ? 1u : 0u;
    return gi;
}

// The delta of a group: the entries the last merge added to a's row form
// (PART_A, PART_U) or b's column form; returns {pool offset, count}.  A
// family's shared operand is its members' a (PART_A) or b (PART_B).
__device__ __forceinline__ uint2 owner_delta(const SlotTab &S, const GroupInfo &gi,
                                             unsigned *err) {
    const uint32_t x = (gi.part == PART_B) ? gi.b : gi.a;
    const size_t r = (size_t)gi.o * gi.n + gi.idx;
    const uint4 dsc = S.desc[x][r];
    const uint32_t d = S.dn[x][r].x;
    if (!CFLR_CHECK(gi.idx < gi.n, err) || !row_in_pool(S, x, dsc, err) ||
        !CFLR_CHECK(d <= (dsc.z ? entry_cap(dsc) : 0u), err))
        return make_uint2(0, 0);
    return make_uint2(dsc.x + tile_words(dsc.z), d);
}

__device__ __forceinline__ unsigned long long group_key(const GroupInfo &gi, uint32_t v) {
    // row groups produce (idx, v); column groups produce (v, idx)
    return gi.o ? (((unsigned long long)v << 32) | gi.idx)
                : (((unsigned long long)gi.idx << 32) | v);
}

// Expand the products of a group's delta entries into the accumulator
// `acc` and emit the ones that are new (warp-collective).  Each delta entry
// k gathers row k of the other operand as a list of tiles: all of b's row k
// for dA . B, and for A_old . dB the tiles of a's column k that precede the
// last merge's (dn.y of them, at the end of the list).
//   Plain groups: warp `warp_id` of `nwarps` takes an even share of the
// entries, 32 consecutive ones at a time (lane l the l-th).
//   Family groups (optimisation 4): when the members' gathered slots are
// consecutive, the same shares of the entries, each entry's members found
// from its occupancy bits; otherwise warp `warp_id` takes the (entry, member)
// items warp_id*32 + l of every block of nwarps*32.  A member's row counts
// only when its occupancy bit is set.  Tagged families key the accumulator
// by member and word, and emit to each member's non-terminal.
// The 32 tile lists the lanes hold are walked together as one packed
// sequence of 16-byte tile pairs (see `walk`).  Returns the emitted count.

// TAGS false: the caller never gets a tagged family group (the bitmap bin:
// a tagged family stays within bin 2's limit or splits into its members), so
// the member tags are not carried through the walk.  PACKED: walk the lanes'
// tile lists as one packed sequence (walk_packed) rather than list by list
// (walk_lists); WALK_U: 16-byte tile-pair loads each lane of the packed walk
// has in flight.
template <bool WIT, bool TAGS, bool PACKED, int WALK_U, class Acc>
__device__ __forceinline__ uint32_t expand_rows(const SlotTab &S, const ProdTab &P,
                                                const WorkBufs &W, const GroupInfo &gi,
                                                uint2 own, uint32_t warp_id, uint32_t nwarps,
                                                int lane, const Acc &acc, CandChunk &ck) {
    // the packed walk emits two windows' tiles per reservation
    static_assert(!PACKED || WALK_U % 2 == 0, "the packed walk needs an even depth");
    const uint32_t dstart = own.x, d = own.y;
    const uint32_t *pool = S.pool[gi.c];
    const size_t oo = (size_t)gi.o * gi.n;
    const uint32_t g0 = (gi.part == PART_A) ? gi.b : gi.a;   // gathered slot (member 0)
    const uint4 *dg = (gi.part == PART_U) ? nullptr : S.desc[g0] + oo;
    uint32_t emitted = 0;
    // the derivation step new pairs record (single-path semantics): the
    // production's operands, or the unit production's one, and the middle
    // vertex k (the delta entry whose gathered row gave the pair)
    auto witness = [&](uint32_t tag, uint32_t k) -> uint2 {
        if (gi.part == PART_U) return make_uint2(WIT_UNIT | S.local[gi.a], 0);
        const uint4 pr = gi.fam ? P.prod[P.fam_prod[gi.first + tag]] : make_uint4(0, gi.a, gi.b, 0);
        return make_uint2(WIT_BINARY | (S.local[pr.y] << 15) | S.local[pr.z], k);
    };
    // the new bits n[i] of word wd[i] (i < 4) of member tag (any number per
    // lane), one reservation in the candidate buffer for all of them; nearly
    // every product is already present, so callers vote first
    auto emit_bits = [&](uint32_t n0, uint32_t wd0, uint32_t n1, uint32_t wd1, uint32_t n2,
                         uint32_t wd2, uint32_t n3, uint32_t wd3, uint32_t tag, uint32_t k) {
        const uint32_t slot = TAGS && gi.tagged ? P.prod[P.fam_prod[gi.first + tag]].x : gi.c;
        if (gi.probe && (n0 | n1 | n2 | n3)) {
            const unsigned long long *ht = S.htab[slot];
            const unsigned long long hm = S.hmask[slot];
            auto absent = [&](uint32_t nb, uint32_t wd) {
                uint32_t keep = 0;
                for (uint32_t r = nb; r; r &= r - 1) {
                    const uint32_t i = __ffs(r) - 1;
                    if (!htab_contains(ht, hm, group_key(gi, wd * 32 + i), &W.cnt->overflow))
                        keep |= 1u << i;
                }
                return keep;
            };
            n0 = absent(n0, wd0);
            n1 = absent(n1, wd1);
            n2 = absent(n2, wd2);
            n3 = absent(n3, wd3);
        }
        const uint32_t cnt = __popc(n0) + __popc(n1) + __popc(n2) + __popc(n3);
        const uint32_t incl = warp_incl_scan(cnt, lane);
        const uint32_t total = __shfl_sync(FULL_MASK, incl, 31);
        if (!total) return;
        // the warp's q-th new entry goes to the rest of its reservation,
        // then to a new one of at least CAND_CHUNK entries
        const unsigned long long rem = ck.end - ck.pos;
        unsigned long long nbase = 0;
        if (total > rem) {
            const unsigned long long take = max((unsigned long long)total - rem, CAND_CHUNK);
            if (lane == 0) {
                nbase = atomicAdd(&W.cnt->cand, take);
                if (nbase + take > W.cand_cap) atomicOr(&W.cnt->overflow, OVF_CAND);
            }
            nbase = __shfl_sync(FULL_MASK, nbase, 0);
            ck.end = nbase + take;
        }
        unsigned long long q = incl - cnt;
        const unsigned long long cpos = ck.pos;
        ck.pos = total > rem ? nbase + (total - rem) : ck.pos + total;
        uint2 wit = make_uint2(0, 0);
        if constexpr (WIT) {
            if (cnt) wit = witness(tag, k);
        }
        auto put = [&](uint32_t nb, uint32_t wd) {
            for (uint32_t r = nb; r; r &= r - 1, q++) {
                const unsigned long long pos = q < rem ? cpos + q : nbase + (q - rem);
                if (pos < W.cand_cap) {
                    W.cand_key[pos] = group_key(gi, wd * 32 + (__ffs(r) - 1));
                    W.cand_slot[pos] = slot;
                    if constexpr (WIT) W.cand_wit[pos] = wit;
                }
            }
        };
        put(n0, wd0);
        put(n1, wd1);
        put(n2, wd2);
        put(n3, wd3);
        // the members' candidate counts (k_check sizes their pair sets)
        if (TAGS && gi.tagged && cnt) atomicAdd(&S.cand[slot], (unsigned long long)cnt);
        emitted += total;
    };
    auto key_of = [&](uint32_t wd, uint32_t tag) {
        return TAGS && gi.tagged ? (tag << TAG_SHIFT) | wd : wd;
    };
    // two tiles (w.x, w.y) and (w.z, w.w) of member tag, gathered through
    // delta entry k, nv of them valid
    auto consume_tiles = [&](uint4 w, uint32_t nv, uint32_t tag, uint32_t k) {
        const uint32_t n0 = nv > 0 ? acc.ins(key_of(w.x, tag), w.y) : 0u;
        const uint32_t n1 = nv > 1 ? acc.ins(key_of(w.z, tag), w.w) : 0u;
        if (__any_sync(FULL_MASK, (n0 | n1) != 0)) emit_bits(n0, w.x, n1, w.z, 0u, 0u, 0u, 0u, tag, k);
    };
    // The tile lists held by the lanes (toff, tn; member tag; delta entry k),
    // one at a time: a list of 32 or more tiles is walked by the whole warp
    // (16-byte loads, two in flight per lane), shorter ones are packed 32
    // tiles per step with a per-lane search of the owning list.  Cheaper
    // than the packed walk below when a group has few, short lists (its
    // fixed cost per call is lower): the warp bins use it.
    auto walk_lists = [&](uint32_t toff, uint32_t tn, uint32_t tag, uint32_t k) {
        // long tile lists: the warp strides over one list at a time
        unsigned lm = __ballot_sync(FULL_MASK, tn >= 32);
        while (lm) {
            const int l = __ffs(lm) - 1;
            lm &= lm - 1;
            const uint32_t *tl = pool + __shfl_sync(FULL_MASK, toff, l);
            const uint32_t T = __shfl_sync(FULL_MASK, tn, l);
            const uint32_t ltag = __shfl_sync(FULL_MASK, tag, l);
            const uint32_t lk = WIT ? __shfl_sync(FULL_MASK, k, l) : 0u;
            for (uint32_t qb = 0; qb < T; qb += 128) {
                uint4 w[2];
                uint32_t nv[2];
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const uint32_t q = qb + 64 * h + 2 * lane;
                    w[h] = make_uint4(0, 0, 0, 0);
                    nv[h] = 0;
                    if (q + 2 <= T) {
                        w[h] = *reinterpret_cast<const uint4 *>(tl + 2 * q);
                        nv[h] = 2;
                    } else if (q < T) {
                        const uint2 t = *reinterpret_cast<const uint2 *>(tl + 2 * q);
                        w[h].x = t.x;
                        w[h].y = t.y;
                        nv[h] = 1;
                    }
                }
                // four tiles per lane, one vote and one reservation
                const uint32_t n0 = nv[0] > 0 ? acc.ins(key_of(w[0].x, ltag), w[0].y) : 0u;
                const uint32_t n1 = nv[0] > 1 ? acc.ins(key_of(w[0].z, ltag), w[0].w) : 0u;
                const uint32_t n2 = nv[1] > 0 ? acc.ins(key_of(w[1].x, ltag), w[1].y) : 0u;
                const uint32_t n3 = nv[1] > 1 ? acc.ins(key_of(w[1].z, ltag), w[1].w) : 0u;
                if (__any_sync(FULL_MASK, (n0 | n1 | n2 | n3) != 0))
                    emit_bits(n0, w[0].x, n1, w[0].z, n2, w[1].x, n3, w[1].z, ltag, lk);
            }
        }
        // short tile lists: packed, 32 tiles per step
        const uint32_t stn = tn < 32 ? tn : 0;
        const uint32_t incl = warp_incl_scan(stn, lane);
        const uint32_t total = __shfl_sync(FULL_MASK, incl, 31);
        for (uint32_t fb = 0; fb < total; fb += 32) {
            const uint32_t f = fb + lane;
            int lo = 0, hi = 31;
#pragma unroll
            for (int st = 0; st < 5; st++) {     // first lane whose inclusive sum > f
                const int mid = (lo + hi) >> 1;
                const uint32_t v = __shfl_sync(FULL_MASK, incl, mid);
                if (f < v) hi = mid; else lo = mid + 1;
            }
            const int owner = lo > 31 ? 31 : lo;
            const uint32_t o_toff = __shfl_sync(FULL_MASK, toff, owner);
            const uint32_t o_incl = __shfl_sync(FULL_MASK, incl, owner);
            const uint32_t o_len = __shfl_sync(FULL_MASK, stn, owner);
            const uint32_t o_tag = __shfl_sync(FULL_MASK, tag, owner);
            const uint32_t o_kk = WIT ? __shfl_sync(FULL_MASK, k, owner) : 0u;
            uint4 w = make_uint4(0, 0, 0, 0);
            uint32_t nv = 0;
            if (f < total) {
                const uint2 t = *reinterpret_cast<const uint2 *>(
                    pool + o_toff + 2 * (f - (o_incl - o_len)));
                w.x = t.x;
                w.y = t.y;
                nv = 1;
            }
            consume_tiles(w, nv, o_tag, o_kk);
        }
    };
    // The tile lists held by the lanes (toff, tn; member tag; delta entry k),
    // walked as one sequence of 16-byte tile pairs: the lists with tiles are
    // moved to the front lanes, list l owns the pairs [excl_l, incl_l) of the
    // sequence, and each lane loads the pair at its position in WALK_U
    // windows of 32 positions at a time (all loads in flight before any is
    // used).  The owner of position p is the number of lists that end at or
    // before p: the lists that end before the window (a ballot) plus those
    // that end inside it (one bit each, OR-reduced over the warp).  Segments
    // start on 16-byte boundaries and a tile section holds an even number of
    // tiles, so a pair never leaves its segment; the second tile of a list's
    // last pair is ignored when the list has an odd count.
    auto walk_packed = [&](uint32_t toff, uint32_t tn, uint32_t tag, uint32_t k) {
        const unsigned nz = __ballot_sync(FULL_MASK, tn != 0);
        if (!nz) return;
        const uint32_t cnt = __popc(nz);
        const uint32_t src = (uint32_t)lane < cnt ? select_bit(nz, (uint32_t)lane) : 0u;
        toff = __shfl_sync(FULL_MASK, toff, src);
        tn = __shfl_sync(FULL_MASK, tn, src);
        if (TAGS || WIT) tag = __shfl_sync(FULL_MASK, tag, src);
        if (WIT) k = __shfl_sync(FULL_MASK, k, src);
        if ((uint32_t)lane >= cnt) tn = 0;
        const uint32_t np = (tn + 1) >> 1;
        const uint32_t incl = warp_incl_scan(np, lane);
        const uint32_t excl = incl - np;
        const uint32_t total = __shfl_sync(FULL_MASK, incl, 31);
        const uint32_t le = FULL_MASK >> (31 - lane);
        for (uint32_t b = 0; b < total; b += 32 * WALK_U) {
            uint4 w[WALK_U];
            uint32_t nv[WALK_U], tg[WALK_U], kk[WALK_U];
#pragma unroll
            for (int u = 0; u < WALK_U; u++) {
                w[u] = make_uint4(0, 0, 0, 0);
                nv[u] = tg[u] = kk[u] = 0;
                const uint32_t bu = b + 32 * u, p = bu + lane;
                if (bu >= total) continue;          // uniform: the last windows may be empty
                const uint32_t first = __popc(__ballot_sync(FULL_MASK, incl <= bu));
                const uint32_t ends =
                    __reduce_or_sync(FULL_MASK, (incl > bu && incl - bu < 32) ? 1u << (incl - bu) : 0u);
                const uint32_t own = min(first + __popc(ends & le), 31u);
                const uint32_t o_toff = __shfl_sync(FULL_MASK, toff, own);
                const uint32_t o_excl = __shfl_sync(FULL_MASK, excl, own);
                const uint32_t o_tn = __shfl_sync(FULL_MASK, tn, own);
                tg[u] = (TAGS || WIT) ? __shfl_sync(FULL_MASK, tag, own) : 0u;
                kk[u] = WIT ? __shfl_sync(FULL_MASK, k, own) : 0u;
                if (p < total) {
                    const uint32_t rel = p - o_excl;
                    nv[u] = min(2u, o_tn - 2 * rel);
                    w[u] = *reinterpret_cast<const uint4 *>(pool + o_toff + 4 * rel);
                }
            }
            uint32_t nb[2 * WALK_U], any = 0;
#pragma unroll
            for (int u = 0; u < WALK_U; u++) {
                nb[2 * u] = nv[u] > 0 ? acc.ins(key_of(w[u].x, tg[u]), w[u].y) : 0u;
                nb[2 * u + 1] = nv[u] > 1 ? acc.ins(key_of(w[u].z, tg[u]), w[u].w) : 0u;
                any |= nb[2 * u] | nb[2 * u + 1];
            }
            // nearly every product is already present: one vote, then the
            // new bits go out four tiles per reservation (with tags or
            // witnesses, one window's pair at a time)
            if (__any_sync(FULL_MASK, any != 0)) {
                if constexpr (!TAGS && !WIT) {
#pragma unroll
                    for (int u = 0; u < WALK_U; u += 2)
                        emit_bits(nb[2 * u], w[u].x, nb[2 * u + 1], w[u].z, nb[2 * u + 2],
                                  w[u + 1].x, nb[2 * u + 3], w[u + 1].z, 0u, 0u);
                } else {
#pragma unroll
                    for (int u = 0; u < WALK_U; u++)
                        emit_bits(nb[2 * u], w[u].x, nb[2 * u + 1], w[u].z, 0u, 0u, 0u, 0u, tg[u],
                                  kk[u]);
                }
            }
        }
    };
    auto walk = [&](uint32_t toff, uint32_t tn, uint32_t tag, uint32_t k) {
        if constexpr (PACKED) walk_packed(toff, tn, tag, k);
        else walk_lists(toff, tn, tag, k);
    };
    if (gi.part == PART_U) {        // c -> a: the delta entries themselves
        for (uint32_t cb = warp_id; cb < d; cb += nwarps * 32) {
            const uint32_t e = cb + lane * nwarps;
            uint32_t nb = 0, wd = 0;
            if (e < d) {
                const uint32_t v = pool[dstart + e];
                if (CFLR_CHECK(v < gi.n, &W.cnt->overflow)) {
                    wd = v >> 5;
                    nb = acc.ins(wd, 1u << (v & 31));
                }
            }
            if (__any_sync(FULL_MASK, nb != 0)) emit_bits(nb, wd, 0u, 0u, 0u, 0u, 0u, 0u, 0, 0);
        }
        return emitted;
    }
    if (gi.fam && gi.consec && gi.F <= 64) {
        // the (entry, member) pairs whose member has a row, packed 32 per
        // step: lane l takes entry l of a block of 32, its members' occupancy
        // bits become a 64-bit mask, and a warp scan numbers the pairs
        const uint32_t *oc = S.occ[g0];
        const uint32_t ow = S.occ_w[g0], lx0 = S.local[g0];
        const uint32_t w0 = lx0 >> 5, sh = lx0 & 31, wlast = (lx0 + gi.F - 1) >> 5;
        const unsigned long long fmask = gi.F == 64 ? ~0ull : (1ull << gi.F) - 1;
        const uint32_t lo_e = (uint32_t)((unsigned long long)d * warp_id / nwarps);
        const uint32_t hi_e = (uint32_t)((unsigned long long)d * (warp_id + 1) / nwarps);
        for (uint32_t cb = lo_e; cb < hi_e; cb += 32) {
            const uint32_t e = cb + lane;
            uint32_t k = 0, mlo = 0, mhi = 0;
            if (e < hi_e) {
                k = pool[dstart + e];
                if (!CFLR_CHECK(k < gi.n, &W.cnt->overflow)) k = 0;
                const uint32_t *ok = oc + (oo + k) * ow + w0;
                const uint32_t x0 = ok[0];
                const uint32_t x1 = w0 + 1 <= wlast ? ok[1] : 0u;
                const uint32_t x2 = w0 + 2 <= wlast ? ok[2] : 0u;
                const unsigned long long lo64 = ((unsigned long long)x1 << 32) | x0;
                const unsigned long long m64 =
                    ((lo64 >> sh) | (sh ? (unsigned long long)x2 << (64 - sh) : 0ull)) & fmask;
                mlo = (uint32_t)m64;
                mhi = (uint32_t)(m64 >> 32);
            }
            const uint32_t cnt = __popc(mlo) + __popc(mhi);
            const uint32_t incl = warp_incl_scan(cnt, lane);
            const uint32_t total = __shfl_sync(FULL_MASK, incl, 31);
            for (uint32_t fb = 0; fb < total; fb += 32) {
                const uint32_t f = fb + lane;
                int lo = 0, hi = 31;
#pragma unroll
                for (int st = 0; st < 5; st++) {     // first lane whose inclusive sum > f
                    const int mid = (lo + hi) >> 1;
                    const uint32_t v = __shfl_sync(FULL_MASK, incl, mid);
                    if (f < v) hi = mid; else lo = mid + 1;
                }
                const int owner = lo > 31 ? 31 : lo;
                const uint32_t o_k = __shfl_sync(FULL_MASK, k, owner);
                const uint32_t o_lo = __shfl_sync(FULL_MASK, mlo, owner);
                const uint32_t o_hi = __shfl_sync(FULL_MASK, mhi, owner);
                const uint32_t o_incl = __shfl_sync(FULL_MASK, incl, owner);
                const uint32_t o_cnt = __shfl_sync(FULL_MASK, cnt, owner);
                uint32_t toff = 0, tn = 0, tag = 0;
                if (f < total) {
                    const uint32_t nth = f - (o_incl - o_cnt), plo = __popc(o_lo);
                    tag = nth < plo ? select_bit(o_lo, nth) : 32 + select_bit(o_hi, nth - plo);
                    const uint4 gd = S.desc[g0 + tag][oo + o_k];
                    if (row_in_pool(S, g0 + tag, gd, &W.cnt->overflow)) {
                        toff = gd.x;
                        tn = gd.y - (gi.o ? (gd.w & DLAST_MASK) : 0u);
                    }
                }
                walk(toff, tn, tag, o_k);
            }
        }
        return emitted;
    }
    if (gi.fam) {
        // any family: the (entry, member) pairs numbered entry * F + member,
        // 32 per warp step; a member's row counts when its occupancy bit is set
        const unsigned long long items = (unsigned long long)d * gi.F;
        for (unsigned long long ib = (unsigned long long)warp_id * 32; ib < items;
             ib += (unsigned long long)nwarps * 32) {
            const unsigned long long it = ib + lane;
            uint32_t toff = 0, tn = 0, tag = 0, k = 0;
            if (it < items) {
                const uint32_t e = (uint32_t)(it / gi.F), i = (uint32_t)(it - (unsigned long long)e * gi.F);
                k = pool[dstart + e];
                const uint4 pr = P.prod[P.fam_prod[gi.first + i]];
                const uint32_t gs = (gi.part == PART_A) ? pr.z : pr.y;
                const uint32_t lx = S.local[gs];
                if (CFLR_CHECK(k < gi.n, &W.cnt->overflow) &&
                    ((S.occ[gs][(oo + k) * S.occ_w[gs] + (lx >> 5)] >> (lx & 31)) & 1u)) {
                    const uint4 gd = S.desc[gs][oo + k];
                    if (row_in_pool(S, gs, gd, &W.cnt->overflow)) {
                        toff = gd.x;
                        tn = gd.y - (gi.o ? (gd.w & DLAST_MASK) : 0u);
                        tag = i;
                    }
                }
            }
            walk(toff, tn, tag, k);
        }
        return emitted;
    }
    // an even share of the entries per warp, in runs of 32 (coalesced)
    const uint32_t lo_e = (uint32_t)((unsigned long long)d * warp_id / nwarps);
    const uint32_t hi_e = (uint32_t)((unsigned long long)d * (warp_id + 1) / nwarps);
    for (uint32_t cb = lo_e; cb < hi_e; cb += 32) {
        const uint32_t e = cb + lane;
        uint32_t toff = 0, tn = 0, k = 0;
        if (e < hi_e) {
            k = pool[dstart + e];
            if (CFLR_CHECK(k < gi.n, &W.cnt->overflow)) {
                const uint4 gd = dg[k];
                if (row_in_pool(S, g0, gd, &W.cnt->overflow)) {
                    toff = gd.x;
                    tn = gd.y - (gi.o ? (gd.w & DLAST_MASK) : 0u);   // A_old for A . dB
                }
            }
        }
        walk(toff, tn, 0, k);
    }
    return emitted;
}

// Load the mask row (the output row of c as it stands) into the accumulator:
// thread tid of nth takes every nth tile.
template <class Acc>
__device__ __forceinline__ void preload_mask(const SlotTab &S, const GroupInfo &gi,
                                             const Acc &acc, uint32_t tid, uint32_t nth,
                                             unsigned *err) {
    const uint4 md = S.desc[gi.c][(size_t)gi.o * gi.n + gi.idx];
    if (!row_in_pool(S, gi.c, md, err)) return;
    const uint32_t *tl = S.pool[gi.c] + md.x;
    // tile pairs (a tile section holds an even number of tiles)
    for (uint32_t q = tid; 2 * q < md.y; q += nth) {
        const uint4 t = *reinterpret_cast<const uint4 *>(tl + 4 * q);
        acc.set(t.x, t.y);
        if (2 * q + 1 < md.y) acc.set(t.z, t.w);
    }
}

// Bins 0 and 1: one warp per group, a private shared-memory table per warp
// (2^LG words and their bits).
template <int LG, int WARPS, bool WIT>
__global__ void __launch_bounds__(WARPS * 32, WARPS == 8 ? 4 : 3) k_spgemm_warp(SlotTab S, ProdTab P, WorkBufs W,
                                                            int bin) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t *tab = smem + (size_t)wib * (2u << LG);
    const unsigned long long n_groups =
        min(W.cnt->groups[bin], W.group_cap[bin]);
    const unsigned long long nw = (unsigned long long)gridDim.x * WARPS;
    CandChunk ck{0, 0};
    unsigned long long bytes = 0;
    for (unsigned long long g = (unsigned long long)blockIdx.x * WARPS + wib; g < n_groups;
         g += nw) {
        const GroupInfo gi = decode_group(P, S, W.groups[bin][g]);
        const int lg = min((int)gi.lg, LG);
        clear_table(tab, lg, lane, 32);
        __syncwarp();
        const HashAcc acc{tab, lg, &W.cnt->overflow};
        if (!gi.probe) {
            preload_mask(S, gi, acc, lane, 32, &W.cnt->overflow);
            __syncwarp();
        }
        const uint2 own = owner_delta(S, gi, &W.cnt->overflow);
        const uint32_t e =
            expand_rows<WIT, true, false, 2>(S, P, W, gi, own, 0, 1, lane, acc, ck);
        if (lane == 0 && e) {
            if (!gi.tagged) atomicAdd(&S.cand[gi.c], (unsigned long long)e);
            bytes += 12ull * e;
        }
        __syncwarp();
    }
    release_chunk(W, ck, lane);
    if (lane == 0 && bytes) atomicAdd(&W.cnt->bytes_bin[bin], bytes);
}

// Bin 2: one CTA per group sharing a 2^LG-word shared-memory table.
template <int LG, bool WIT>
__global__ void __launch_bounds__(256, LG == 12 ? 4 : 3) k_spgemm_cta(SlotTab S, ProdTab P, WorkBufs W, int bin) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ uint32_t emitted_sh;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    __shared__ unsigned long long next_sh[2];
    const unsigned long long n_groups = min(W.cnt->groups[bin], W.group_cap[bin]);
    CandChunk ck{0, 0};
    unsigned long long bytes = 0;
    // groups are claimed one at a time from a cursor (their sizes vary a
    // lot), the next one while the current one starts
    if (threadIdx.x == 0) next_sh[0] = atomicAdd(&W.cnt->claim[bin], 1ull);
    __syncthreads();
    unsigned long long g = next_sh[0];
    for (uint32_t q = 1; g < n_groups; q ^= 1) {
        const GroupInfo gi = decode_group(P, S, W.groups[bin][g]);
        const int lg = min((int)gi.lg, LG);
        clear_table(smem, lg, threadIdx.x, blockDim.x);
        if (threadIdx.x == 0) {
            emitted_sh = 0;
            next_sh[q] = atomicAdd(&W.cnt->claim[bin], 1ull);
        }
        __syncthreads();
        const HashAcc acc{smem, lg, &W.cnt->overflow};
        if (!gi.probe) preload_mask(S, gi, acc, threadIdx.x, blockDim.x, &W.cnt->overflow);
        __syncthreads();
        const uint2 own = owner_delta(S, gi, &W.cnt->overflow);
        const uint32_t e = expand_rows<WIT, true, true, 2>(S, P, W, gi, own, wib,
                                                            blockDim.x >> 5, lane, acc, ck);
        if (lane == 0 && e) atomicAdd(&emitted_sh, e);
        __syncthreads();
        if (threadIdx.x == 0 && emitted_sh) {
            if (!gi.tagged) atomicAdd(&S.cand[gi.c], (unsigned long long)emitted_sh);
            bytes += 12ull * emitted_sh;
        }
        g = next_sh[q];
    }
    release_chunk(W, ck, lane);
    if (threadIdx.x == 0 && bytes) atomicAdd(&W.cnt->bytes_bin[bin], bytes);
}

// Bin 3: one CTA per group with an n-bit bitmap of the output row (shared
// memory when it fits, else a per-CTA slice of global scratch).  In mask mode
// the mask row's bits are set first; in probe mode new bits are checked
// against the non-terminal's hash set instead.
template <bool WIT, int GPC>
__global__ void __launch_bounds__(256, 4) k_spgemm_bitmap(SlotTab S, ProdTab P, WorkBufs W,
                                                          int bin, int use_smem,
                                                          uint32_t bm_stride) {
    // GPC groups at a time: each half (quarter, ...) of the CTA has its own
    // bitmap and its own named barrier, so a short group does not hold the
    // others up and twice the groups are in flight per SM
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ uint32_t emitted_sh[GPC];
    constexpr int TPG = 256 / GPC;                    // threads per group
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int part = threadIdx.x / TPG, ptid = threadIdx.x % TPG;
    auto psync = [&]() {
        if (GPC == 1) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(part + 1), "r"(TPG) : "memory");
    };
    const unsigned long long n_groups = min(W.cnt->groups[bin], W.group_cap[bin]);
    uint32_t *bm = use_smem ? smem + (size_t)part * bm_stride
                            : W.bitmap_scratch + ((size_t)blockIdx.x * GPC + part) * W.bitmap_words;
#if defined(CFLR_CHECKED)
    BitmapAcc acc{bm, 0u, &W.cnt->overflow};
#else
    const BitmapAcc acc{bm};
#endif
    CandChunk ck{0, 0};
    unsigned long long bytes = 0;
    // each part claims groups one at a time from a cursor (their sizes vary
    // a lot), the next one while the current one starts
    __shared__ unsigned long long next_sh[GPC][2];
    if (ptid == 0) next_sh[part][0] = atomicAdd(&W.cnt->claim[bin], 1ull);
    psync();
    unsigned long long g = next_sh[part][0];
    for (uint32_t q = 1; g < n_groups; q ^= 1) {
        const GroupInfo gi = decode_group(P, S, W.groups[bin][g]);
        const uint32_t words = (gi.n + 31) >> 5;
#if defined(CFLR_CHECKED)
        acc.words = words;
#endif
        if (use_smem) {   // 16-byte stores: the stride is a multiple of four words
            uint4 *b4 = reinterpret_cast<uint4 *>(bm);
            for (uint32_t s = ptid; s < (words + 3) >> 2; s += TPG) b4[s] = make_uint4(0, 0, 0, 0);
        } else {
            for (uint32_t s = ptid; s < words; s += TPG) bm[s] = 0;
        }
        if (ptid == 0) {
            emitted_sh[part] = 0;
            next_sh[part][q] = atomicAdd(&W.cnt->claim[bin], 1ull);
        }
        psync();
        if (!gi.probe) preload_mask(S, gi, acc, ptid, TPG, &W.cnt->overflow);
        psync();
        const uint2 own = owner_delta(S, gi, &W.cnt->overflow);
        const uint32_t e = expand_rows<WIT, false, true, 4>(S, P, W, gi, own, wib % (8 / GPC), 8 / GPC,
                                                     lane, acc, ck);
        if (lane == 0 && e) atomicAdd(&emitted_sh[part], e);
        psync();
        if (ptid == 0 && emitted_sh[part]) {
            if (!gi.tagged) atomicAdd(&S.cand[gi.c], (unsigned long long)emitted_sh[part]);
            bytes += 12ull * emitted_sh[part];
        }
        g = next_sh[part][q];
    }
    release_chunk(W, ck, lane);
    if (ptid == 0 && bytes) atomicAdd(&W.cnt->bytes_bin[bin], bytes);
}

// ---------------------------------------------------------------------------
// k_commit: global dedupe of candidates into the per-slot pair sets
// ---------------------------------------------------------------------------

// The commit stages a CTA's new pairs and touched rows in shared memory and
// reserves their room in the global lists with one atomic per list per
// round: per-warp atomics on those few counters serialise at the L2 (every
// warp of the grid hits the same addresses).
constexpr uint32_t COMMIT_ROUND = 512;    // candidates a CTA takes per round
constexpr uint32_t COMMIT_SLOTS = 1024;   // per-slot counts kept in shared memory

__global__ void __launch_bounds__(256) k_commit(SlotTab S, WorkBufs W, uint32_t n_slots) {
    __shared__ unsigned long long st_key[COMMIT_ROUND];
    __shared__ uint32_t st_slot[COMMIT_ROUND];
    __shared__ uint2 st_touch[2 * COMMIT_ROUND];
    __shared__ uint32_t slot_new[COMMIT_SLOTS];
    __shared__ uint32_t n_new, n_touch;
    __shared__ unsigned long long base_new, base_touch;
    __shared__ unsigned stop;
    // one read for the CTA (this kernel's own threads may set OVF_FULL, and
    // every thread must take the same path to the barriers below)
    if (threadIdx.x == 0) stop = W.cnt->overflow & OVF_STOP;
    __syncthreads();
    if (stop) return;                          // the iteration is re-run after a growth
    const int lane = threadIdx.x & 31;
    const int par = *W.parity;
    unsigned long long *out_n = &W.touched_n[par ^ 1];
    uint2 *t_out = W.touched[par ^ 1];
    const unsigned long long nc = min(W.cnt->cand, W.cand_cap);
    const bool hist = n_slots <= COMMIT_SLOTS;
    for (uint32_t s = threadIdx.x; s < COMMIT_SLOTS; s += blockDim.x) slot_new[s] = 0;
    if (threadIdx.x == 0) n_new = n_touch = 0;
    __syncthreads();
    for (unsigned long long r0 = (unsigned long long)blockIdx.x * COMMIT_ROUND; r0 < nc;
         r0 += (unsigned long long)gridDim.x * COMMIT_ROUND) {
        for (uint32_t q = 0; q < COMMIT_ROUND; q += blockDim.x) {
            const unsigned long long t = r0 + q + threadIdx.x;
            bool isnew = false;
            unsigned long long key = 0;
            uint32_t slot = EMPTY32;
            if (t < nc) slot = W.cand_slot[t];
            if (slot != EMPTY32) {            // not an unused reserved entry
                key = W.cand_key[t];
                if (!CFLR_CHECK((key >> 32) < S.n[slot] && (uint32_t)key < S.n[slot],
                                &W.cnt->overflow))
                    slot = EMPTY32;
            }
            if (slot != EMPTY32) {
                unsigned long long *tab = S.htab[slot];
                const unsigned long long m = S.hmask[slot];
                unsigned long long h = pair_home(key, m);
                bool placed = false;
                // at most one pass over the set (k_check keeps it half full)
                for (unsigned long long p = 0; p <= m; p++) {
                    unsigned long long v = tab[h];
                    if (v == key) {
                        placed = true;
                        break;
                    }
                    if (v == EMPTY_KEY) {
                        v = atomicCAS(&tab[h], EMPTY_KEY, key);
                        if (v == EMPTY_KEY) {
                            isnew = placed = true;
                            if (W.cand_wit && S.hval[slot]) S.hval[slot][h] = W.cand_wit[t];
                            break;
                        }
                        if (v == key) {
                            placed = true;
                            break;
                        }
                    }
                    h = (h + 1) & m;
                }
                if (!placed) atomicOr(&W.cnt->overflow, OVF_FULL);
            }
            // count the new pair in its row of each form, and list a row the
            // first time it gets one (the rows the merge appends to)
            bool first_r = false, first_c = false;
            const uint32_t i = (uint32_t)(key >> 32), j = (uint32_t)key;
            if (isnew) {
                uint2 *dn = S.dn[slot];
                first_r = atomicAdd(&dn[i].x, 1u) == 0;
                first_c = atomicAdd(&dn[(size_t)S.n[slot] + j].x, 1u) == 0;
                if (hist) atomicAdd(&slot_new[slot], 1u);
                else atomicAdd(&S.delta[slot], 1ull);
            }
            // stage the warp's new pairs and first-touched rows (one shared
            // atomic per warp and list)
            const unsigned m = __ballot_sync(FULL_MASK, isnew);
            if (m) {
                uint32_t p0 = 0;
                if (lane == 0) p0 = atomicAdd(&n_new, (uint32_t)__popc(m));
                p0 = __shfl_sync(FULL_MASK, p0, 0);
                if (isnew) {
                    const uint32_t p = p0 + __popc(m & ((1u << lane) - 1));
                    st_key[p] = key;
                    st_slot[p] = slot;
                }
                const unsigned fr = __ballot_sync(FULL_MASK, first_r);
                const unsigned fc = __ballot_sync(FULL_MASK, first_c);
                if (fr | fc) {
                    uint32_t q0 = 0;
                    if (lane == 0) q0 = atomicAdd(&n_touch, (uint32_t)(__popc(fr) + __popc(fc)));
                    q0 = __shfl_sync(FULL_MASK, q0, 0);
                    const unsigned below = (1u << lane) - 1;
                    if (first_r) st_touch[q0 + __popc(fr & below)] = make_uint2(slot * 2, i);
                    if (first_c)
                        st_touch[q0 + __popc(fr) + __popc(fc & below)] = make_uint2(slot * 2 + 1, j);
                }
            }
        }
        __syncthreads();
        const uint32_t nn = n_new, nt = n_touch;
        if (threadIdx.x == 0) {
            base_new = nn ? atomicAdd(&W.cnt->delta, (unsigned long long)nn) : 0;
            base_touch = nt ? atomicAdd(out_n, (unsigned long long)nt) : 0;
        }
        __syncthreads();
        // new pairs <= candidates <= the delta buffer's capacity
        for (uint32_t q = threadIdx.x; q < nn; q += blockDim.x) {
            W.delta_key[base_new + q] = st_key[q];
            W.delta_slot[base_new + q] = st_slot[q];
        }
        for (uint32_t q = threadIdx.x; q < nt; q += blockDim.x) {
            const unsigned long long tp = base_touch + q;
            if (tp < W.touched_cap) t_out[tp] = st_touch[q];
            else atomicOr(&W.cnt->overflow, OVF_TOUCHED);
        }
        __syncthreads();
        if (threadIdx.x == 0) n_new = n_touch = 0;
        __syncthreads();
    }
    if (hist) {
        for (uint32_t s = threadIdx.x; s < n_slots; s += blockDim.x)
            if (slot_new[s]) atomicAdd(&S.delta[s], (unsigned long long)slot_new[s]);
    }
}

// ---------------------------------------------------------------------------
// merge: M <- M u dC in the row and column forms
// ---------------------------------------------------------------------------

// Rows that received entries in the previous merge stop being "new".
__global__ void k_reset_dnew(SlotTab S, WorkBufs W) {
    if (W.cnt->overflow & OVF_STOP) return;
    const int par = *W.parity;
    const unsigned long long n_in = W.touched_n[par];
    const uint2 *t_in = W.touched[par];
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
         e < n_in; e += (unsigned long long)gridDim.x * blockDim.x) {
        const uint2 t = t_in[e];
        const uint32_t slot = t.x >> 1, o = t.x & 1;
        const size_t r = (size_t)o * S.n[slot] + t.y;
        S.dn[slot][r] = make_uint2(0, 0);
        S.desc[slot][r].w &= ~DLAST_MASK;
    }
}

constexpr uint32_t TILE_WARP_MAX = 256;   // tiles one warp folds (k_capacity, k_pack)

// Capacities of a moved row: its folded tiles plus room to append as many
// tiles again (at least twice this merge's entries), and a power of two of
// at least twice this merge's entries (desc.w keeps its log2); a row that
// keeps growing moves a logarithmic number of times.
__device__ __forceinline__ uint32_t tile_cap_after_move(uint32_t tiles, uint32_t incoming) {
    return tiles + max(max(2u * incoming, tiles), 8u);
}
__device__ __forceinline__ uint32_t entry_log_after_move(uint32_t incoming) {
    uint32_t lg = 3;
    while ((1u << lg) < 2u * incoming) lg++;
    return lg;
}

// Deduplicate `cnt` tiles (word, bits), read through get(q), in a warp's
// shared-memory table of 2^lg >= 2*cnt slots and write one tile per word to
// out; returns the number written (warp-collective, all lanes).
template <class Get>
__device__ __forceinline__ uint32_t warp_fold_tiles(uint32_t *tab, uint32_t cnt, Get get,
                                                    uint32_t *out, int lane, unsigned *err) {
    uint32_t lg = 5;
    while ((1u << lg) < 2 * cnt) lg++;
    clear_table(tab, lg, lane, 32);
    __syncwarp();
    const HashAcc acc{tab, (int)lg, err};
    for (uint32_t q = lane; q < cnt; q += 32) {
        const uint2 t = get(q);
        acc.ins(t.x, t.y);
    }
    __syncwarp();
    uint32_t base = 0;
    for (uint32_t sb = 0; sb < (1u << lg); sb += 32) {
        const uint32_t s = sb + lane;
        const uint2 sl = reinterpret_cast<const uint2 *>(tab)[s];
        const bool has = sl.x != EMPTY32;
        const unsigned m = __ballot_sync(FULL_MASK, has);
        if (has) reinterpret_cast<uint2 *>(out)[base + __popc(m & ((1u << lane) - 1))] = sl;
        base += __popc(m);
    }
    __syncwarp();
    return base;
}

// Make room for every listed row: its new entries (dn.x) in the entry area
// and as many tiles at the end of its tile list.  A row without that room
// moves to a new segment with its tiles folded to one per word; rows of more
// than TILE_WARP_MAX tiles are left to k_capacity_big.  Also sets the
// occupancy bit of a row's first entries and clears the append cursors.
// Idempotent: after a pool overflow the host grows the pool and runs it again.
__global__ void __launch_bounds__(256) k_capacity(SlotTab S, InstTab I, WorkBufs W) {
    __shared__ __align__(16) uint32_t tabs[8][4 * TILE_WARP_MAX];   // a table per warp
    if (W.cnt->overflow & OVF_STOP) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t *tab = tabs[wib];
    const int par = *W.parity;
    const uint2 *t_out = W.touched[par ^ 1];
    const unsigned long long n_t = min(W.touched_n[par ^ 1], W.touched_cap);
    const unsigned long long nw = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    unsigned long long moved = 0;           // tile bytes read and written (lane 0)
    for (unsigned long long e = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + wib;
         e < n_t; e += nw) {
        const uint2 t = t_out[e];
        const uint32_t slot = t.x >> 1, o = t.x & 1;
        const size_t r = (size_t)o * S.n[slot] + t.y;
        uint4 *dp = &S.desc[slot][r];
        const uint4 dsc = *dp;
        const uint32_t w = S.dn[slot][r].x;
        if (lane == 0) {
            S.dn[slot][r].y = 0;
            if (dsc.y == 0) {                 // the row gets its first entries
                const uint32_t lx = S.local[slot];
                atomicOr(&S.occ[slot][r * S.occ_w[slot] + (lx >> 5)], 1u << (lx & 31));
            }
        }
        if ((unsigned long long)dsc.y + w <= dsc.z && w <= entry_cap(dsc)) continue;
        if (dsc.y > TILE_WARP_MAX) continue;
        if (!row_in_pool(S, slot, dsc, &W.cnt->overflow)) continue;
        uint32_t *pool = S.pool[slot];
        // fold into the table first (the count sizes the new segment) ...
        uint32_t lg = 5;
        while ((1u << lg) < 2 * dsc.y) lg++;
        clear_table(tab, lg, lane, 32);
        __syncwarp();
        const HashAcc acc{tab, (int)lg, &W.cnt->overflow};
        for (uint32_t q = lane; q < dsc.y; q += 32) {
            const uint2 tl = *reinterpret_cast<const uint2 *>(pool + dsc.x + 2 * q);
            acc.ins(tl.x, tl.y);
        }
        __syncwarp();
        uint32_t D = 0;
        for (uint32_t s = lane; s < (1u << lg); s += 32) D += tab[2 * s] != EMPTY32;
        for (int dd = 16; dd > 0; dd >>= 1) D += __shfl_xor_sync(FULL_MASK, D, dd);
        const uint32_t tcap = tile_cap_after_move(D, w), elog = entry_log_after_move(w);
        const unsigned long long size = (unsigned long long)tile_words(tcap) + (1ull << elog);
        const uint32_t inst = S.inst[slot];
        unsigned long long off = 0;
        if (lane == 0) {
            off = atomicAdd(&I.pool_top[inst], size);
            if (off + size > I.pool_cap[inst]) {
                atomicOr(&W.cnt->overflow, OVF_POOL);
                off = ~0ull;
            }
        }
        off = __shfl_sync(FULL_MASK, off, 0);
        if (off == ~0ull) {
            __syncwarp();
            continue;
        }
        // ... then write the table's words as the new tile list
        uint32_t *np = pool + off;
        uint32_t base = 0;
        for (uint32_t sb = 0; sb < (1u << lg); sb += 32) {
            const uint2 sl = reinterpret_cast<const uint2 *>(tab)[sb + lane];
            const bool has = sl.x != EMPTY32;
            const unsigned m = __ballot_sync(FULL_MASK, has);
            if (has) reinterpret_cast<uint2 *>(np)[base + __popc(m & ((1u << lane) - 1))] = sl;
            base += __popc(m);
        }
        __syncwarp();
        if (lane == 0) {
            *dp = make_uint4((uint32_t)off, D, tcap, elog << ELOG_SHIFT);
            moved += 8ull * (dsc.y + D);
        }
        __syncwarp();
    }
    if (lane == 0 && moved) atomicAdd(&W.cnt->bytes_move[0], moved);
}

// The rows k_capacity leaves (more than TILE_WARP_MAX tiles): the CTA lists
// the large rows among 256 touched rows at a time, then folds each through
// an n-bit bitmap in shared memory (its tiles come out in word order).
// Without room for the bitmap (use_smem 0) the tiles are copied as they are.
// Idempotent like k_capacity.
__global__ void __launch_bounds__(256) k_capacity_big(SlotTab S, InstTab I, WorkBufs W,
                                                      int use_smem) {
    extern __shared__ uint32_t bm[];
    __shared__ uint32_t list[256];
    __shared__ uint32_t list_n;
    __shared__ unsigned long long sh[16];
    __shared__ unsigned long long off_sh;
    if (W.cnt->overflow & OVF_STOP) return;
    const int par = *W.parity;
    const uint2 *t_out = W.touched[par ^ 1];
    const unsigned long long n_t = min(W.touched_n[par ^ 1], W.touched_cap);
    unsigned long long moved = 0;           // tile bytes read and written (thread 0)
    for (unsigned long long cb = (unsigned long long)blockIdx.x * 256; cb < n_t;
         cb += (unsigned long long)gridDim.x * 256) {
        if (threadIdx.x == 0) list_n = 0;
        __syncthreads();
        const unsigned long long e = cb + threadIdx.x;
        if (e < n_t) {
            const uint2 t = t_out[e];
            const uint32_t slot = t.x >> 1, o = t.x & 1;
            const size_t r = (size_t)o * S.n[slot] + t.y;
            const uint4 dsc = S.desc[slot][r];
            const uint32_t w = S.dn[slot][r].x;
            if (((unsigned long long)dsc.y + w > dsc.z || w > entry_cap(dsc)) &&
                dsc.y > TILE_WARP_MAX)
                list[atomicAdd(&list_n, 1u)] = threadIdx.x;
        }
        __syncthreads();
        const uint32_t ln = list_n;
        for (uint32_t li = 0; li < ln; li++) {
            const uint2 t = t_out[cb + list[li]];
            const uint32_t slot = t.x >> 1, o = t.x & 1;
            const uint32_t n = S.n[slot];
            const size_t r = (size_t)o * n + t.y;
            uint4 *dp = &S.desc[slot][r];
            const uint4 dsc = *dp;
            const uint32_t w = S.dn[slot][r].x;
            uint32_t *pool = S.pool[slot];
            const uint32_t words = (n + 31) >> 5;
            const uint32_t per = (words + blockDim.x - 1) / blockDim.x;
            const uint32_t w0 = min(words, threadIdx.x * per), w1 = min(words, w0 + per);
            uint32_t cnt = 0;
            if (use_smem) {
                for (uint32_t q = threadIdx.x; q < words; q += blockDim.x) bm[q] = 0;
                __syncthreads();
                for (uint32_t q = threadIdx.x; q < dsc.y; q += blockDim.x) {
                    const uint2 tl = *reinterpret_cast<const uint2 *>(pool + dsc.x + 2 * q);
                    atomicOr(&bm[tl.x], tl.y);
                }
                __syncthreads();
                for (uint32_t q = w0; q < w1; q++) cnt += bm[q] != 0;
            }
            unsigned long long D = 0;
            const unsigned long long before = block_excl_scan256(cnt, sh, D);
            const uint32_t ntn = use_smem ? (uint32_t)D : dsc.y;
            const uint32_t tcap = tile_cap_after_move(ntn, w), elog = entry_log_after_move(w);
            const unsigned long long size = (unsigned long long)tile_words(tcap) + (1ull << elog);
            if (threadIdx.x == 0) {
                unsigned long long off = atomicAdd(&I.pool_top[S.inst[slot]], size);
                if (off + size > I.pool_cap[S.inst[slot]]) {
                    atomicOr(&W.cnt->overflow, OVF_POOL);
                    off = ~0ull;
                }
                off_sh = off;
            }
            __syncthreads();
            const unsigned long long off = off_sh;
            if (off != ~0ull) {
                uint32_t *np = pool + off;
                if (use_smem) {
                    unsigned long long pos = before;
                    for (uint32_t q = w0; q < w1; q++) {
                        const uint32_t b = bm[q];
                        if (b) {
                            np[2 * pos] = q;
                            np[2 * pos + 1] = b;
                            pos++;
                        }
                    }
                } else {
                    for (uint32_t q = threadIdx.x; q < 2 * dsc.y; q += blockDim.x)
                        np[q] = pool[dsc.x + q];
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    *dp = make_uint4((uint32_t)off, ntn, tcap, elog << ELOG_SHIFT);
                    moved += 8ull * (dsc.y + ntn);
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0 && moved) atomicAdd(&W.cnt->bytes_move[1], moved);
}

// Append the new pairs as single entries: (i, j) goes to the entry area of
// row i of the row form and of row j of the column form.
__global__ void __launch_bounds__(256) k_scatter(SlotTab S, WorkBufs W) {
    if (W.cnt->overflow & (OVF_STOP | OVF_POOL)) return;
    const unsigned long long nd = W.cnt->delta;
    for (unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
         t < nd; t += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long key = W.delta_key[t];
        const uint32_t slot = W.delta_slot[t];
        const uint32_t i = (uint32_t)(key >> 32), j = (uint32_t)key;
        const uint4 *dsc = S.desc[slot];
        uint2 *dn = S.dn[slot];
        uint32_t *pool = S.pool[slot];
        const uint32_t n = S.n[slot];
        const uint4 dr = dsc[i];
        const uint32_t pr = atomicAdd(&dn[i].y, 1u);
        if (row_in_pool(S, slot, dr, &W.cnt->overflow) &&
            CFLR_CHECK(dr.z && pr < entry_cap(dr), &W.cnt->overflow))
            pool[(size_t)dr.x + tile_words(dr.z) + pr] = j;
        const uint4 dc = dsc[(size_t)n + j];
        const uint32_t pc = atomicAdd(&dn[(size_t)n + j].y, 1u);
        if (row_in_pool(S, slot, dc, &W.cnt->overflow) &&
            CFLR_CHECK(dc.z && pc < entry_cap(dc), &W.cnt->overflow))
            pool[(size_t)dc.x + tile_words(dc.z) + pc] = i;
    }
}

// Pack every appended row's new entries into tiles (one per word, 256
// entries at a time) at the end of its tile list.  The new pairs are not in
// the row yet, so the tiles of a row never share a set bit; a word may get a
// second tile, until the row's next move folds them.
__global__ void __launch_bounds__(256) k_pack(SlotTab S, WorkBufs W) {
    __shared__ __align__(16) uint32_t tabs[8][4 * TILE_WARP_MAX];
    if (W.cnt->overflow & (OVF_STOP | OVF_POOL)) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t *tab = tabs[wib];
    const int par = *W.parity;
    const uint2 *t_out = W.touched[par ^ 1];
    const unsigned long long n_t = min(W.touched_n[par ^ 1], W.touched_cap);
    const unsigned long long nw = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long e = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + wib;
         e < n_t; e += nw) {
        const uint2 t = t_out[e];
        const uint32_t slot = t.x >> 1, o = t.x & 1;
        const size_t r = (size_t)o * S.n[slot] + t.y;
        uint4 *dp = &S.desc[slot][r];
        const uint4 dsc = *dp;
        const uint32_t w = S.dn[slot][r].x;
        if (!row_in_pool(S, slot, dsc, &W.cnt->overflow) ||
            !CFLR_CHECK(w <= entry_cap(dsc) && dsc.y + w <= dsc.z, &W.cnt->overflow))
            continue;
        const uint32_t *ent = S.pool[slot] + dsc.x + tile_words(dsc.z);
        uint32_t *tl = S.pool[slot] + dsc.x;
        if (w == 1) {                  // one new pair: one tile, no table
            if (lane == 0) {
                const uint32_t v = ent[0];
                reinterpret_cast<uint2 *>(tl)[dsc.y] = make_uint2(v >> 5, 1u << (v & 31));
                dp->y = dsc.y + 1;
                dp->w = (dsc.w & ~DLAST_MASK) | 1u;
            }
            __syncwarp();
            continue;
        }
        uint32_t nt = dsc.y;
        for (uint32_t c0 = 0; c0 < w; c0 += TILE_WARP_MAX) {
            const uint32_t cnt = min(TILE_WARP_MAX, w - c0);
            nt += warp_fold_tiles(tab, cnt,
                                  [&](uint32_t q) {
                                      const uint32_t v = ent[c0 + q];
                                      return make_uint2(v >> 5, 1u << (v & 31));
                                  },
                                  tl + 2 * nt, lane, &W.cnt->overflow);
        }
        if (lane == 0) {
            dp->y = nt;
            // the delta's tiles (a count beyond the field falls back to
            // gathering all of A, a superset of A_old with the same union)
            const uint32_t dl = nt - dsc.y;
            dp->w = (dsc.w & ~DLAST_MASK) | (dl <= DLAST_MASK ? dl : 0u);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// iteration frame (device-side checks; lets the loop run inside a CUDA graph)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_iter_begin(SlotTab S, InstTab I, WorkBufs W,
                                                    uint32_t n_slots, uint32_t n_inst) {
    const int par = *W.parity;
    if (threadIdx.x == 0) {
        *W.cnt = Counters{};
        W.touched_n[par ^ 1] = 0;
    }
    for (uint32_t s = threadIdx.x; s < n_slots; s += blockDim.x) {
        S.cand[s] = 0;
        S.delta[s] = 0;
    }
    for (uint32_t k = threadIdx.x; k < n_inst; k += blockDim.x) I.delta[k] = 0;
}

// Before the commit: stop the iteration if a buffer overflowed or if some
// pair set could pass half full with this iteration's candidates.
__global__ void __launch_bounds__(256) k_check(SlotTab S, WorkBufs W, uint32_t n_slots,
                                               int growth) {
    if (!growth) return;               // sets kept at their size (a test setting)
    bool grow = false;
    for (uint32_t s = threadIdx.x; s < n_slots; s += blockDim.x)
        grow |= 2 * (S.nnz[s] + S.cand[s]) > S.hmask[s] + 1;
    if (__syncthreads_or(grow) && threadIdx.x == 0) atomicOr(&W.cnt->overflow, OVF_HASH);
}

// After the merge: add the new pairs to the counts, advance every
// instance's iteration count, flip the touched-list parity and decide
// whether the closure loop goes on (Algorithm 1: while M is changing).
__global__ void __launch_bounds__(256) k_iter_end(SlotTab S, InstTab I, WorkBufs W, LoopCtl *ctl,
                                                  uint32_t n_slots, uint32_t n_inst,
                                                  int count_iteration,
                                                  cudaGraphConditionalHandle handle,
                                                  int in_graph) {
    const unsigned flags = W.cnt->overflow & (OVF_STOP | OVF_POOL);
    if (flags) {                        // the host grows a buffer and finishes the iteration
        if (threadIdx.x == 0) {
            ctl->status = flags;
            if (in_graph) cudaGraphSetConditional(handle, 0);
        }
        return;
    }
    for (uint32_t s = threadIdx.x; s < n_slots; s += blockDim.x) {
        const unsigned long long d = S.delta[s];
        S.nnz[s] += d;
        if (d) atomicAdd(&I.delta[S.inst[s]], d);
    }
    __syncthreads();
    int finished = 0;                   // some instance reached its fixpoint now
    if (count_iteration) {
        for (uint32_t k = threadIdx.x; k < n_inst; k += blockDim.x) {
            if (I.active[k]) {
                I.iters[k] += 1;
                if (I.delta[k] == 0) finished = 1;
            }
            I.active[k] = I.delta[k] > 0 ? 1u : 0u;
        }
    }
    finished = __syncthreads_or(finished);
    if (threadIdx.x == 0) {
        const unsigned long long total = W.cnt->delta;
        const int par = *W.parity;
        if (count_iteration) {
            ctl->total_flops += W.cnt->flops;
            ctl->total_cand += W.cnt->cand - W.cnt->holes;
            ctl->total_delta += total;
            ctl->total_touched_in += W.touched_n[par];
            ctl->total_touched_out += W.touched_n[par ^ 1];
            for (int b = 0; b < N_BINS; b++) {
                ctl->bytes_bin[b] += W.cnt->bytes_bin[b];
                ctl->total_groups[b] += min(W.cnt->groups[b], W.group_cap[b]);
            }
            ctl->bytes_sym += W.cnt->bytes_sym;
            ctl->tiles_bin3[0] += W.cnt->tiles_bin3[0];
            ctl->tiles_bin3[1] += W.cnt->tiles_bin3[1];
            ctl->bytes_move[0] += W.cnt->bytes_move[0];
            ctl->bytes_move[1] += W.cnt->bytes_move[1];
        }
        *W.parity = par ^ 1;
        ctl->status = 0;
        ctl->last_delta = total;
        if (count_iteration) ctl->iter += 1;
        const bool more = total > 0 && ctl->iter < ctl->limit &&
                          !(ctl->stop_on_converge && finished);
        if (in_graph) cudaGraphSetConditional(handle, more ? 1u : 0u);
    }
}

// ---------------------------------------------------------------------------
// initialisation (Algorithm 1, terminal initialisation) and maintenance
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_init_edges(const uint32_t *src, const uint32_t *lab,
                                                    const uint32_t *dst,
                                                    unsigned long long n_edges,
                                                    const uint32_t *term_off,
                                                    const uint32_t *term_slot,
                                                    uint32_t n_terms, WorkBufs W) {
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x +
                                   (threadIdx.x & ~31u);
         base < n_edges; base += stride) {
        const unsigned long long e = base + lane;
        uint32_t q0 = 0, q1 = 0, l = 0;
        unsigned long long key = 0;
        if (e < n_edges) {
            l = lab[e];
            if (l < n_terms) { q0 = term_off[l]; q1 = term_off[l + 1]; }
            key = ((unsigned long long)src[e] << 32) | dst[e];
        }
        // every terminal maps to few non-terminals: emit one round per target
        uint32_t rounds = q1 - q0;
        for (int d = 16; d > 0; d >>= 1) rounds = max(rounds, __shfl_xor_sync(FULL_MASK, rounds, d));
        for (uint32_t r = 0; r < rounds; r++) {
            const bool f = q0 + r < q1;
            const uint32_t slot = f ? term_slot[q0 + r] : 0;
            emit_candidates(f, key, slot, W, lane, make_uint2(WIT_EDGE | (l & WIT_PAYLOAD), 0));
        }
    }
}

__global__ void k_init_eps(uint32_t slot, uint32_t n, WorkBufs W) {
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x +
                                   (threadIdx.x & ~31u);
         base < n; base += stride) {
        const unsigned long long i = base + lane;
        emit_candidates(i < n, (i << 32) | i, slot, W, lane, make_uint2(WIT_EPS, 0));
    }
}

__global__ void k_rehash(const unsigned long long *old_tab, const uint2 *old_val,
                         unsigned long long old_cap, unsigned long long *new_tab,
                         uint2 *new_val, unsigned long long new_cap, unsigned *err) {
    const unsigned long long m = new_cap - 1;
    for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
         s < old_cap; s += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long key = old_tab[s];
        if (key == EMPTY_KEY) continue;
        unsigned long long h = pair_home(key, m);
        unsigned long long p = 0;     // one pass at most (the new set is at most 1/4 full)
        while (atomicCAS(&new_tab[h], EMPTY_KEY, key) != EMPTY_KEY && ++p <= m) h = (h + 1) & m;
        if (p > m) {
            atomicOr(err, OVF_FULL);
            continue;
        }
        if (new_val) new_val[h] = old_val[s];
    }
}

// The recorded derivation step of one pair (single thread): {~0, ~0} when
// the pair is not in the set.
__global__ void k_witness_lookup(const unsigned long long *tab, const uint2 *val,
                                 unsigned long long m, unsigned long long key, uint2 *out) {
    unsigned long long h = pair_home(key, m);
    for (unsigned long long probes = 0; probes <= m; probes++) {
        const unsigned long long v = tab[h];
        if (v == key) {
            *out = val[h];
            return;
        }
        if (v == EMPTY_KEY) break;
        h = (h + 1) & m;
    }
    *out = make_uint2(EMPTY32, EMPTY32);
}

__global__ void k_fill_u64(unsigned long long *p, unsigned long long count,
                           unsigned long long v) {
    for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
         s < count; s += (unsigned long long)gridDim.x * blockDim.x)
        p[s] = v;
}

// Split a batch's touched list back into per-instance lists with local
// slot ids: first count the entries of every instance, then scatter.
// (Lanes of one instance add their entries with one atomic per warp: the
// rows of an instance lie together in the list.)
__global__ void k_touched_count(const uint2 *in, unsigned long long n, const uint32_t *slot_inst,
                                unsigned long long *cnt) {
    const int lane = threadIdx.x & 31;
    for (unsigned long long b = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
         b < n; b += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long s = b + lane;
        const uint32_t k = s < n ? slot_inst[in[s].x >> 1] : EMPTY32;
        const unsigned same = __match_any_sync(FULL_MASK, k);
        if (k != EMPTY32 && lane == __ffs(same) - 1)
            atomicAdd(&cnt[k], (unsigned long long)__popc(same));
    }
}

__global__ void k_touched_split(const uint2 *in, unsigned long long n, const uint32_t *slot_inst,
                                const uint32_t *inst_base, uint2 *const *out,
                                unsigned long long *cursor) {
    const int lane = threadIdx.x & 31;
    for (unsigned long long b = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
         b < n; b += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long s = b + lane;
        uint2 t = make_uint2(0, 0);
        uint32_t k = EMPTY32;
        if (s < n) {
            t = in[s];
            k = slot_inst[t.x >> 1];
        }
        const unsigned same = __match_any_sync(FULL_MASK, k);
        const int leader = __ffs(same) - 1;
        unsigned long long pos = 0;
        if (k != EMPTY32 && lane == leader) pos = atomicAdd(&cursor[k], (unsigned long long)__popc(same));
        pos = __shfl_sync(FULL_MASK, pos, leader);
        if (k != EMPTY32) {
            pos += __popc(same & ((1u << lane) - 1));
            out[k][pos] = make_uint2(t.x - 2 * inst_base[k], t.y);
        }
    }
}

__global__ void k_remap_touched(const uint2 *in, unsigned long long n, uint32_t slot_base,
                                uint2 *out) {
    for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
         s < n; s += (unsigned long long)gridDim.x * blockDim.x) {
        const uint2 t = in[s];
        out[s] = make_uint2(t.x + 2 * slot_base, t.y);
    }
}

// ---------------------------------------------------------------------------
// extraction: rows of the row form, each sorted, written in row order
// ---------------------------------------------------------------------------

// Extraction walks the rows in the caller's vertex order: row i of the
// output is stored row perm[i], and a stored column v is the caller's
// vertex iperm[v] (both null when the vertices were kept in input order).
__device__ __forceinline__ uint32_t stored_row(const uint32_t *perm, uint32_t i) {
    return perm ? perm[i] : i;
}

// Pairs in a row: the set bits of its tiles (no two tiles share a bit).
__global__ void k_row_lengths(const uint4 *desc, const uint32_t *pool, uint32_t n,
                              const uint32_t *perm, uint32_t *len) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint4 d = desc[stored_row(perm, i)];
        const uint32_t *tl = pool + d.x;
        uint32_t c = 0;
        for (uint32_t q = 0; q < d.y; q++) c += __popc(tl[2 * q + 1]);
        len[i] = c;
    }
}

// Renumber vertex ids in place: a[e] <- perm[a[e]].
__global__ void k_permute_ids(uint32_t *a, unsigned long long m, const uint32_t *perm) {
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (unsigned long long)gridDim.x * blockDim.x)
        a[e] = perm[a[e]];
}

constexpr int EXTRACT_WARP_MAX = 1024;
constexpr uint32_t EXTRACT_BATCH = 4;   // rows a warp takes per claim

// Write one row of len <= EXTRACT_WARP_MAX pairs (warp-collective): its
// nt tiles tl decoded into the warp's shared buffer s, the columns turned
// into caller ids, sorted, and written as (src, column) pairs from o on.
__device__ __forceinline__ void extract_row_warp(const uint32_t *tl, uint32_t nt, uint32_t len,
                                                 uint32_t src, const uint32_t *iperm,
                                                 unsigned long long o, uint32_t *out_src,
                                                 uint32_t *out_dst, uint32_t *s, int lane) {
    // each lane decodes one tile per round at its scan position
    uint32_t base = 0;
    for (uint32_t qb = 0; qb < nt; qb += 32) {
        const uint32_t q = qb + lane;
        const uint32_t w = q < nt ? tl[2 * q] : 0, b = q < nt ? tl[2 * q + 1] : 0;
        const uint32_t c = __popc(b);
        const uint32_t incl = warp_incl_scan(c, lane);
        uint32_t pos = base + incl - c;
        for (uint32_t rb = b; rb; rb &= rb - 1) s[pos++] = w * 32 + (__ffs(rb) - 1);
        base += __shfl_sync(FULL_MASK, incl, 31);
    }
    __syncwarp();
    // caller ids: one gather per entry, the whole warp's loads in
    // flight together (per tile they would wait one after another)
    if (iperm) {
#pragma unroll 4
        for (uint32_t t = lane; t < len; t += 32) s[t] = iperm[s[t]];
    }
    __syncwarp();
    if (len <= 32) {
        // bitonic network over the lanes: in each block of k lanes
        // (ascending when lane & k is clear) the lower lane of every
        // pair j apart keeps the minimum
        uint32_t v = (uint32_t)lane < len ? s[lane] : EMPTY32;
#pragma unroll
        for (uint32_t k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                const uint32_t u = __shfl_xor_sync(FULL_MASK, v, j);
                const bool up = (lane & k) == 0, lower = (lane & j) == 0;
                v = (lower == up) ? min(v, u) : max(v, u);
            }
        }
        if ((uint32_t)lane < len) {
            out_src[o + lane] = src;
            out_dst[o + lane] = v;
        }
        __syncwarp();
        return;
    }
    uint32_t P = 64;
    while (P < len) P <<= 1;
    for (uint32_t t = len + lane; t < P; t += 32) s[t] = EMPTY32;
    __syncwarp();
    // bitonic sort of P entries: every lane takes whole pairs (t, t + jj),
    // t the q-th index with bit jj clear
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t jj = k >> 1; jj > 0; jj >>= 1) {
            for (uint32_t q = lane; q < P / 2; q += 32) {
                const uint32_t t = ((q & ~(jj - 1)) << 1) | (q & (jj - 1));
                const uint32_t a = s[t], b = s[t | jj];
                const bool up = (t & k) == 0;
                if ((a > b) == up) {
                    s[t] = b;
                    s[t | jj] = a;
                }
            }
            __syncwarp();
        }
    }
    for (uint32_t t = lane; t < len; t += 32) {
        out_src[o + t] = src;
        out_dst[o + t] = s[t];
    }
    __syncwarp();
}

// One warp per row: rows up to 32 entries are sorted in registers (one entry
// per lane), longer ones up to 1024 entries by a bitonic sort in shared
// memory; longer rows are listed for k_extract_big.  Warps claim rows
// EXTRACT_BATCH at a time from cursor[1] (zeroed by the launcher), so a few
// long rows do not leave one warp running after the others; cursor[0]
// counts the listed long rows.
__global__ void __launch_bounds__(256) k_extract_small(const uint4 *desc, const uint32_t *pool,
                                                       uint32_t n, const uint32_t *perm,
                                                       const uint32_t *iperm,
                                                       const unsigned long long *row_out,
                                                       uint32_t *out_src, uint32_t *out_dst,
                                                       uint32_t *big_rows,
                                                       uint32_t *cursor) {
    __shared__ uint32_t sbuf[8][EXTRACT_WARP_MAX];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t *s = sbuf[wib];
    for (;;) {
        uint32_t i0 = 0;
        if (lane == 0) i0 = atomicAdd(&cursor[1], EXTRACT_BATCH);
        i0 = __shfl_sync(FULL_MASK, i0, 0);
        if (i0 >= n) break;
        for (uint32_t i = i0; i < min(n, i0 + EXTRACT_BATCH); i++) {
            const uint4 d = desc[stored_row(perm, i)];
            const uint32_t nt = d.y;
            const uint32_t *tl = pool + d.x;
            uint32_t len = 0;
            for (uint32_t q = lane; q < nt; q += 32) len += __popc(tl[2 * q + 1]);
            for (int dd = 16; dd > 0; dd >>= 1) len += __shfl_xor_sync(FULL_MASK, len, dd);
            if (len == 0) continue;
            if (len > EXTRACT_WARP_MAX) {
                if (lane == 0) big_rows[atomicAdd(&cursor[0], 1u)] = i;
                continue;
            }
            extract_row_warp(tl, nt, len, i, iperm, row_out[i], out_src, out_dst, s, lane);
        }
    }
}

// One long row by the whole CTA (CTA-collective): its columns marked in an
// n-bit bitmap bm (caller ids), then the set bits written in increasing
// order as (src, column) pairs from o on.  scan: 256 words of shared memory.
__device__ __forceinline__ void extract_row_cta(const uint32_t *tl, uint32_t ntiles, uint32_t n,
                                                uint32_t src, const uint32_t *iperm,
                                                unsigned long long o, uint32_t *out_src,
                                                uint32_t *out_dst, uint32_t *bm,
                                                uint32_t *scan) {
    const uint32_t words = (n + 31) >> 5;
    const uint32_t per = (words + blockDim.x - 1) / blockDim.x;
    for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) bm[w] = 0;
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < ntiles; q += blockDim.x) {
        const uint32_t w = tl[2 * q];
        // four bits of the tile at a time, their gathers in flight together
        for (uint32_t rb = tl[2 * q + 1]; rb;) {
            uint32_t v[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                v[u] = rb ? w * 32 + (__ffs(rb) - 1) : EMPTY32;
                rb &= rb - 1;
            }
            if (iperm) {
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (v[u] != EMPTY32) v[u] = iperm[v[u]];
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (v[u] != EMPTY32) atomicOr(&bm[v[u] >> 5], 1u << (v[u] & 31));
        }
    }
    __syncthreads();
    const uint32_t w0 = threadIdx.x * per, w1 = min(words, w0 + per);
    uint32_t cnt = 0;
    for (uint32_t w = w0; w < w1; w++) cnt += __popc(bm[w]);
    scan[threadIdx.x] = cnt;
    __syncthreads();
    for (uint32_t off = 1; off < blockDim.x; off <<= 1) {
        const uint32_t v = threadIdx.x >= off ? scan[threadIdx.x - off] : 0;
        __syncthreads();
        scan[threadIdx.x] += v;
        __syncthreads();
    }
    o += scan[threadIdx.x] - cnt;
    for (uint32_t w = w0; w < w1; w++) {
        uint32_t bits = bm[w];
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            out_src[o] = src;
            out_dst[o] = w * 32 + b;
            o++;
        }
    }
    __syncthreads();
}

// One CTA per long row listed by k_extract_small.
__global__ void __launch_bounds__(256) k_extract_big(const uint4 *desc, const uint32_t *pool,
                                                     uint32_t n, const uint32_t *perm,
                                                     const uint32_t *iperm,
                                                     const unsigned long long *row_out,
                                                     uint32_t *out_src, uint32_t *out_dst,
                                                     const uint32_t *big_rows,
                                                     const uint32_t *big_count,
                                                     uint32_t *gbitmap, int use_smem) {
    extern __shared__ uint32_t smem[];
    __shared__ uint32_t scan[256];
    const uint32_t words = (n + 31) >> 5;
    uint32_t *bm = use_smem ? smem : gbitmap + (size_t)blockIdx.x * words;
    const uint32_t nb = *big_count;
    for (uint32_t r = blockIdx.x; r < nb; r += gridDim.x) {
        const uint32_t i = big_rows[r];
        const uint4 d = desc[stored_row(perm, i)];
        extract_row_cta(pool + d.x, d.y, n, i, iperm, row_out[i], out_src, out_dst, bm, scan);
    }
}

// ---------------------------------------------------------------------------
// Extraction of a list of non-terminals, one after another (the pairs of
// several non-terminals in one call).  The rows of every listed
// non-terminal, in caller order, are cut into units of rows; the units
// follow the list order, so the exclusive scan of their pair counts is each
// unit's first output position; within a unit the rows follow one another.
// Rows of more than EXTRACT_WARP_MAX pairs are listed (row, k, output
// position) for a CTA each.
// ---------------------------------------------------------------------------

__device__ __forceinline__ const uint4 *list_desc(const ExtractList &L, uint32_t k) {
    return L.desc + (size_t)L.nts[k] * 2 * L.n;   // row form of nts[k]
}

// The listed non-terminal k owning unit u, and the unit's rows [r0, r1).
__device__ __forceinline__ uint32_t unit_rows(const ExtractList &L, unsigned long long u,
                                              uint32_t &r0, uint32_t &r1) {
    uint32_t lo = 0, hi = L.count;          // unit_first[lo] <= u < unit_first[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (L.unit_first[mid] <= u) lo = mid;
        else hi = mid;
    }
    const uint32_t R = L.rows_per[lo];
    const unsigned long long a = (u - L.unit_first[lo]) * R;
    r0 = (uint32_t)min(a, (unsigned long long)L.n);
    r1 = (uint32_t)min(a + R, (unsigned long long)L.n);
    return lo;
}

// Pairs of every unit (a warp per unit, its lanes over the rows).
__global__ void __launch_bounds__(256) k_unit_lengths(ExtractList L,
                                                      unsigned long long *unit_len) {
    const int lane = threadIdx.x & 31;
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long u = (unsigned long long)blockIdx.x * (blockDim.x >> 5) +
                                (threadIdx.x >> 5);
         u < L.units; u += warps) {
        uint32_t r0, r1;
        const uint4 *dk = list_desc(L, unit_rows(L, u, r0, r1));
        unsigned long long len = 0;
        for (uint32_t i = r0 + lane; i < r1; i += 32) {
            const uint4 d = dk[stored_row(L.perm, i)];
            const uint32_t *tl = L.pool + d.x;
            uint32_t c32 = 0;
            for (uint32_t q = 0; q < d.y; q++) c32 += __popc(tl[2 * q + 1]);
            len += c32;
        }
        len = warp_sum64(len);
        if (lane == 0) unit_len[u] = len;
    }
}

// The rows of every unit (a warp per unit, units claimed from cursor[1]):
// the lanes read 32 rows' descriptors at once and the warp takes the
// non-empty ones in order.  cursor[0] counts the listed long rows.
__global__ void __launch_bounds__(256) k_extract_units(ExtractList L,
                                                       const unsigned long long *unit_off,
                                                       uint32_t *out_src, uint32_t *out_dst,
                                                       uint4 *big, unsigned long long big_cap,
                                                       unsigned long long *cursor,
                                                       unsigned *err) {
    __shared__ uint32_t sbuf[8][EXTRACT_WARP_MAX];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t *s = sbuf[wib];
    for (;;) {
        unsigned long long u = 0;
        if (lane == 0) u = L.u_begin + atomicAdd(&cursor[1], 1ull);
        u = __shfl_sync(FULL_MASK, u, 0);
        if (u >= L.u_end) break;
        uint32_t r0, r1;
        const uint32_t k = unit_rows(L, u, r0, r1);
        const uint4 *dk = list_desc(L, k);
        unsigned long long o = unit_off[u];     // absolute; written at o - L.base
        for (uint32_t rb = r0; rb < r1; rb += 32) {
            const uint32_t i = rb + lane;
            const uint4 d = i < r1 ? dk[stored_row(L.perm, i)] : make_uint4(0, 0, 0, 0);
            for (unsigned m = __ballot_sync(FULL_MASK, d.y != 0); m; m &= m - 1) {
                const int l = __ffs(m) - 1;
                const uint32_t nt = __shfl_sync(FULL_MASK, d.y, l);
                const uint32_t *tl = L.pool + __shfl_sync(FULL_MASK, d.x, l);
                uint32_t len = 0;
                for (uint32_t q = lane; q < nt; q += 32) len += __popc(tl[2 * q + 1]);
                len = __reduce_add_sync(FULL_MASK, len);
                if (len == 0) continue;
                if (o + len > L.limit) {
                    // more pairs than the pair sets count: nothing is written
                    // past the caller's arrays
                    if (lane == 0) atomicOr(err, 2u);
                } else if (len > EXTRACT_WARP_MAX) {
                    if (lane == 0) {
                        const unsigned long long pos = atomicAdd(&cursor[0], 1ull);
                        const unsigned long long ro = o - L.base;
                        if (pos < big_cap)
                            big[pos] = make_uint4(rb + l, k, (uint32_t)ro, (uint32_t)(ro >> 32));
                        else
                            atomicOr(err, 1u);
                    }
                } else {
                    extract_row_warp(tl, nt, len, rb + l, L.iperm, o - L.base, out_src, out_dst,
                                     s, lane);
                }
                o += len;
            }
        }
    }
}

// One CTA per long row listed by k_extract_units.
__global__ void __launch_bounds__(256) k_extract_units_big(ExtractList L, uint32_t *out_src,
                                                           uint32_t *out_dst, const uint4 *big,
                                                           unsigned long long big_cap,
                                                           const unsigned long long *cursor,
                                                           uint32_t *gbitmap, int use_smem) {
    extern __shared__ uint32_t smem[];
    __shared__ uint32_t scan[256];
    const uint32_t words = (L.n + 31) >> 5;
    uint32_t *bm = use_smem ? smem : gbitmap + (size_t)blockIdx.x * words;
    const unsigned long long nb = min(cursor[0], big_cap);
    for (unsigned long long r = blockIdx.x; r < nb; r += gridDim.x) {
        const uint4 e = big[r];
        const uint4 d = list_desc(L, e.y)[stored_row(L.perm, e.x)];
        extract_row_cta(L.pool + d.x, d.y, L.n, e.x, L.iperm,
                        ((unsigned long long)e.w << 32) | e.z, out_src, out_dst, bm, scan);
    }
}

// ---------------------------------------------------------------------------
// exclusive scan of uint32 or uint64 counts into uint64 offsets (three
// phases; in place when in == out)
// ---------------------------------------------------------------------------

constexpr uint32_t SCAN_TILE = 1024;   // 256 threads x 4 elements

template <typename T>
__global__ void __launch_bounds__(256) k_scan_reduce(const T *in, unsigned long long n,
                                                     unsigned long long *bsum) {
    __shared__ unsigned long long sh[16];
    const unsigned long long base = (unsigned long long)blockIdx.x * SCAN_TILE + threadIdx.x * 4;
    unsigned long long v = 0;
#pragma unroll
    for (int q = 0; q < 4; q++)
        if (base + q < n) v += in[base + q];
    unsigned long long total;
    block_excl_scan256(v, sh, total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(256) k_scan_top(unsigned long long *bsum, uint32_t nb,
                                                  unsigned long long *grand) {
    __shared__ unsigned long long sh[16];
    unsigned long long carry = 0;
    for (uint32_t b0 = 0; b0 < nb; b0 += 256) {
        const uint32_t i = b0 + threadIdx.x;
        const unsigned long long v = i < nb ? bsum[i] : 0;
        unsigned long long total;
        const unsigned long long ex = block_excl_scan256(v, sh, total);
        if (i < nb) bsum[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0 && grand) *grand = carry;
}

template <typename T>
__global__ void __launch_bounds__(256) k_scan_down(const T *in, unsigned long long n,
                                                   const unsigned long long *bsum,
                                                   unsigned long long *out) {
    __shared__ unsigned long long sh[16];
    const unsigned long long base = (unsigned long long)blockIdx.x * SCAN_TILE + threadIdx.x * 4;
    T x[4];
    unsigned long long v = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        x[q] = base + q < n ? in[base + q] : 0;
        v += x[q];
    }
    unsigned long long total;
    unsigned long long acc = bsum[blockIdx.x] + block_excl_scan256(v, sh, total);
#pragma unroll
    for (int q = 0; q < 4; q++) {
        if (base + q < n) out[base + q] = acc;
        acc += x[q];
    }
}

void launch_exclusive_scan(const uint32_t *in, uint32_t n, unsigned long long *out,
                           unsigned long long *bsum, unsigned long long *grand, cudaStream_t st) {
    if (!n) return;
    const uint32_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    k_scan_reduce<uint32_t><<<nb, 256, 0, st>>>(in, n, bsum);
    k_scan_top<<<1, 256, 0, st>>>(bsum, nb, grand);
    k_scan_down<uint32_t><<<nb, 256, 0, st>>>(in, n, bsum, out);
}

void launch_exclusive_scan64(unsigned long long *in_out, unsigned long long n,
                             unsigned long long *bsum, unsigned long long *grand,
                             cudaStream_t st) {
    if (!n) return;
    const unsigned long long nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    k_scan_reduce<unsigned long long><<<(unsigned)nb, 256, 0, st>>>(in_out, n, bsum);
    k_scan_top<<<1, 256, 0, st>>>(bsum, (uint32_t)nb, grand);
    k_scan_down<unsigned long long><<<(unsigned)nb, 256, 0, st>>>(in_out, n, bsum, in_out);
}

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------

static inline int grid_for(unsigned long long work, int per_block, int sms, int mult) {
    unsigned long long g = (work + per_block - 1) / per_block;
    const unsigned long long cap = (unsigned long long)sms * mult;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

// tables of words and bits: 2 x 4 bytes per slot
constexpr size_t BIN0_SMEM = 8 * 2 * 256 * 4;    // 8 warps x 256 slots
constexpr size_t BIN1_SMEM = 4 * 2 * 2048 * 4;   // 4 warps x 2048 slots
constexpr size_t BIN1S_SMEM = 8 * 2 * 1024 * 4;  // 8 warps x 1024 slots (limit <= 512)
constexpr size_t BIN2_SMEM = 2 * 8192 * 4;
constexpr size_t BIN2S_SMEM = 2 * 4096 * 4;       // limit <= 2048
constexpr size_t SMEM_BITMAP_MAX = 200 * 1024;

static void set_smem_attrs();
void prepare_launch_attributes() { set_smem_attrs(); }

template <bool WIT>
static void set_bin_smem_attrs() {
    cudaFuncSetAttribute(k_spgemm_warp<11, 4, WIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)BIN1_SMEM);
    cudaFuncSetAttribute(k_spgemm_cta<13, WIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)BIN2_SMEM);
    cudaFuncSetAttribute(k_spgemm_warp<10, 8, WIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)BIN1S_SMEM);
    cudaFuncSetAttribute(k_spgemm_bitmap<WIT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)SMEM_BITMAP_MAX);
    cudaFuncSetAttribute(k_spgemm_bitmap<WIT, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)SMEM_BITMAP_MAX);
}

// cudaFuncSetAttribute applies to the device current at the call, so the
// limits are set once per device (under a lock: contexts on several host
// threads may launch at the same time).
static void set_smem_attrs() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return;
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 64 && done[dev]) return;
    if (dev < 64) done[dev] = true;
    set_bin_smem_attrs<false>();
    set_bin_smem_attrs<true>();
    cudaFuncSetAttribute(k_extract_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)SMEM_BITMAP_MAX);
    cudaFuncSetAttribute(k_extract_units_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)SMEM_BITMAP_MAX);
    cudaFuncSetAttribute(k_capacity_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)SMEM_BITMAP_MAX);
}

void launch_symbolic(const SlotTab &S, const ProdTab &P, const WorkBufs &W, int prod_only,
                     const Tuning &T, int sms, cudaStream_t st) {
    k_symbolic<<<sms * 8, 256, 0, st>>>(S, P, W, prod_only, T, 0);
    k_symbolic<<<sms * 4, 256, 0, st>>>(S, P, W, prod_only, T, 1);
}

// The product bins, with the witness plumbing compiled in only when the
// batch records witnesses (it costs registers).
template <bool WIT>
static void launch_bin(int bin, const SlotTab &S, const ProdTab &P, const WorkBufs &W,
                       uint32_t max_n, const Tuning &T, int sms, cudaStream_t st) {
    switch (bin) {
    case 0:
        k_spgemm_warp<8, 8, WIT><<<sms * T.ctas_per_sm[0], 256, BIN0_SMEM, st>>>(S, P, W, 0);
        break;
    case 1:   // the smaller table when the limit allows it: more warps per SM
        if (T.limit[1] <= 512)
            k_spgemm_warp<10, 8, WIT><<<sms * T.ctas_per_sm[1], 256, BIN1S_SMEM, st>>>(S, P, W, 1);
        else
            k_spgemm_warp<11, 4, WIT><<<sms * T.ctas_per_sm[1], 128, BIN1_SMEM, st>>>(S, P, W, 1);
        break;
    case 2:
        if (T.limit[2] <= 2048)
            k_spgemm_cta<12, WIT><<<sms * T.ctas_per_sm[2], 256, BIN2S_SMEM, st>>>(S, P, W, 2);
        else
            k_spgemm_cta<13, WIT><<<sms * T.ctas_per_sm[2], 256, BIN2_SMEM, st>>>(S, P, W, 2);
        break;
    default: {
        // bitmap words rounded to 16 bytes; two groups per CTA when four CTAs
        // of two bitmaps fit the shared memory (then registers, not shared
        // memory, bound the CTAs per SM either way)
        const uint32_t words = ((max_n + 31) / 32 + 3) & ~3u;
        const size_t bm_bytes = (size_t)words * 4;
        const bool sm = bm_bytes <= SMEM_BITMAP_MAX;
        const bool two = sm && 8 * (bm_bytes + 512) <= 220 * 1024;
        int per_sm = sm ? (int)((220 * 1024) / ((two ? 2 : 1) * bm_bytes + 1024)) : 4;
        per_sm = per_sm < 1 ? 1 : (per_sm > (int)T.ctas_per_sm[3] ? (int)T.ctas_per_sm[3] : per_sm);
        if (two)
            k_spgemm_bitmap<WIT, 2><<<sms * per_sm, 256, 2 * bm_bytes, st>>>(S, P, W, 3, 1, words);
        else
            k_spgemm_bitmap<WIT, 1><<<sms * per_sm, 256, sm ? bm_bytes : 0, st>>>(S, P, W, 3,
                                                                                 sm ? 1 : 0, words);
        break;
    }
    }
}

void launch_spgemm(int bin, const SlotTab &S, const ProdTab &P, const WorkBufs &W,
                   uint32_t max_n, const Tuning &T, int sms, cudaStream_t st) {
    set_smem_attrs();
    if (W.cand_wit) launch_bin<true>(bin, S, P, W, max_n, T, sms, st);
    else launch_bin<false>(bin, S, P, W, max_n, T, sms, st);
}

void launch_commit(const SlotTab &S, const WorkBufs &W, uint32_t n_slots, int sms,
                   cudaStream_t st) {
    k_commit<<<sms * 8, 256, 0, st>>>(S, W, n_slots);
}

void launch_iter_begin(const SlotTab &S, const InstTab &I, const WorkBufs &W, uint32_t n_slots,
                       uint32_t n_inst, cudaStream_t st) {
    k_iter_begin<<<1, 256, 0, st>>>(S, I, W, n_slots, n_inst);
}

void launch_check(const SlotTab &S, const WorkBufs &W, uint32_t n_slots, bool growth,
                  cudaStream_t st) {
    k_check<<<1, 256, 0, st>>>(S, W, n_slots, growth ? 1 : 0);
}

void launch_iter_end(const SlotTab &S, const InstTab &I, const WorkBufs &W, LoopCtl *ctl,
                     uint32_t n_slots, uint32_t n_inst, bool count_iteration,
                     cudaGraphConditionalHandle handle, bool in_graph, cudaStream_t st) {
    k_iter_end<<<1, 256, 0, st>>>(S, I, W, ctl, n_slots, n_inst, count_iteration ? 1 : 0, handle,
                                  in_graph ? 1 : 0);
}

void launch_reset_dnew(const SlotTab &S, const WorkBufs &W, int sms, cudaStream_t st) {
    k_reset_dnew<<<sms * 4, 256, 0, st>>>(S, W);
}


void launch_capacity(const SlotTab &S, const InstTab &I, const WorkBufs &W, int sms,
                     cudaStream_t st) {
    k_capacity<<<sms * 8, 256, 0, st>>>(S, I, W);
}

void launch_capacity_big(const SlotTab &S, const InstTab &I, const WorkBufs &W, uint32_t max_n,
                         int sms, cudaStream_t st) {
    set_smem_attrs();
    const size_t bm_bytes = (size_t)((max_n + 31) / 32) * 4;
    const bool sm = bm_bytes <= SMEM_BITMAP_MAX;
    int per_sm = sm ? (int)((220 * 1024) / (bm_bytes + 3072)) : 8;
    per_sm = per_sm < 1 ? 1 : (per_sm > 8 ? 8 : per_sm);
    k_capacity_big<<<sms * per_sm, 256, sm ? bm_bytes : 0, st>>>(S, I, W, sm ? 1 : 0);
}

void launch_scatter(const SlotTab &S, const WorkBufs &W, int sms, cudaStream_t st) {
    k_scatter<<<sms * 8, 256, 0, st>>>(S, W);
}

void launch_pack(const SlotTab &S, const WorkBufs &W, int sms, cudaStream_t st) {
    k_pack<<<sms * 8, 256, 0, st>>>(S, W);
}

void launch_init_edges(const uint32_t *src, const uint32_t *lab, const uint32_t *dst,
                       unsigned long long n_edges, const uint32_t *term_off,
                       const uint32_t *term_slot, uint32_t n_terms, const WorkBufs &W,
                       int sms, cudaStream_t st) {
    if (!n_edges) return;
    k_init_edges<<<grid_for(n_edges, 256, sms, 8), 256, 0, st>>>(src, lab, dst, n_edges,
                                                                  term_off, term_slot, n_terms, W);
}

void launch_init_eps(uint32_t slot, uint32_t n, const WorkBufs &W, int sms, cudaStream_t st) {
    if (!n) return;
    k_init_eps<<<grid_for(n, 256, sms, 8), 256, 0, st>>>(slot, n, W);
}

void launch_rehash(const unsigned long long *old_tab, const uint2 *old_val,
                   unsigned long long old_cap, unsigned long long *new_tab, uint2 *new_val,
                   unsigned long long new_cap, unsigned *err, int sms, cudaStream_t st) {
    k_rehash<<<grid_for(old_cap, 256, sms, 8), 256, 0, st>>>(old_tab, old_val, old_cap, new_tab,
                                                              new_val, new_cap, err);
}

void launch_witness_lookup(const unsigned long long *tab, const uint2 *val,
                           unsigned long long mask, unsigned long long key, uint2 *out,
                           cudaStream_t st) {
    k_witness_lookup<<<1, 1, 0, st>>>(tab, val, mask, key, out);
}

void launch_fill_u64(unsigned long long *p, unsigned long long count, unsigned long long v,
                     int sms, cudaStream_t st) {
    if (!count) return;
    k_fill_u64<<<grid_for(count, 256, sms, 8), 256, 0, st>>>(p, count, v);
}

void launch_remap_touched(const uint2 *in, unsigned long long n, uint32_t slot_base,
                          uint2 *out, cudaStream_t st) {
    if (!n) return;
    k_remap_touched<<<grid_for(n, 256, 152, 8), 256, 0, st>>>(in, n, slot_base, out);
}

void launch_touched_count(const uint2 *in, unsigned long long n, const uint32_t *slot_inst,
                          unsigned long long *cnt, cudaStream_t st) {
    if (!n) return;
    k_touched_count<<<grid_for(n, 256, 152, 8), 256, 0, st>>>(in, n, slot_inst, cnt);
}

void launch_touched_split(const uint2 *in, unsigned long long n, const uint32_t *slot_inst,
                          const uint32_t *inst_base, uint2 *const *out,
                          unsigned long long *cursor, cudaStream_t st) {
    if (!n) return;
    k_touched_split<<<grid_for(n, 256, 152, 8), 256, 0, st>>>(in, n, slot_inst, inst_base, out,
                                                              cursor);
}

void launch_permute_ids(uint32_t *a, unsigned long long m, const uint32_t *perm, int sms,
                        cudaStream_t st) {
    if (!m) return;
    k_permute_ids<<<grid_for(m, 256, sms, 8), 256, 0, st>>>(a, m, perm);
}

void launch_row_lengths(const uint4 *desc, const uint32_t *pool, uint32_t n,
                        const uint32_t *perm, uint32_t *len, cudaStream_t st) {
    if (!n) return;
    k_row_lengths<<<grid_for(n, 256, 152, 8), 256, 0, st>>>(desc, pool, n, perm, len);
}

void extract_plan(uint32_t count, uint32_t n, const uint64_t *pairs, int sms,
                  uint32_t *rows_per, unsigned long long *unit_first) {
    const unsigned long long target = (unsigned long long)sms * 64 * 8;   // resident warps x 8
    unsigned long long total = 0;
    for (uint32_t k = 0; k < count; k++) total += pairs[k];
    const unsigned long long share = std::max<unsigned long long>(256, total / target);
    unit_first[0] = 0;
    for (uint32_t k = 0; k < count; k++) {
        unsigned long long u = std::max<unsigned long long>(((unsigned long long)n + 4095) / 4096,
                                                            (pairs[k] + share - 1) / share);
        u = std::max<unsigned long long>(1, std::min<unsigned long long>(u, n));
        const uint32_t R = (uint32_t)(((unsigned long long)n + u - 1) / u);
        rows_per[k] = std::max<uint32_t>(R, 1);
        unit_first[k + 1] = unit_first[k] + ((unsigned long long)n + rows_per[k] - 1) / rows_per[k];
    }
}

void launch_extract_count(const ExtractList &L, unsigned long long *units,
                          unsigned long long *bsum, unsigned long long *total, int sms,
                          cudaStream_t st) {
    const unsigned long long nu = L.units;
    if (!nu || !L.n) return;
    k_unit_lengths<<<grid_for(nu, 8, sms, 8), 256, 0, st>>>(L, units);
    launch_exclusive_scan64(units, nu, bsum, total, st);
}

void launch_extract_write(const ExtractList &L, uint32_t *out_src, uint32_t *out_dst,
                          const unsigned long long *units, uint4 *big,
                          unsigned long long big_cap, unsigned long long *cursor,
                          uint32_t *bitmap, unsigned *err, int sms, cudaStream_t st) {
    const unsigned long long nu = L.u_end > L.u_begin ? L.u_end - L.u_begin : 0;
    if (!nu || !L.n) return;
    set_smem_attrs();
    cudaMemsetAsync(cursor, 0, 2 * sizeof(unsigned long long), st);
    k_extract_units<<<grid_for(nu, 8, sms, 8), 256, 0, st>>>(L, units, out_src, out_dst, big,
                                                             big_cap, cursor, err);
    const size_t bm_bytes = (size_t)((L.n + 31) / 32) * 4;
    const bool sm = bm_bytes <= SMEM_BITMAP_MAX;
    k_extract_units_big<<<sms * 4, 256, sm ? bm_bytes : 0, st>>>(L, out_src, out_dst, big,
                                                                 big_cap, cursor, bitmap,
                                                                 sm ? 1 : 0);
}

void launch_extract(const uint4 *desc, const uint32_t *pool, uint32_t n, const uint32_t *perm,
                    const uint32_t *iperm, const unsigned long long *row_out, uint32_t *out_src,
                    uint32_t *out_dst, uint32_t *big_rows, uint32_t *big_count,
                    uint32_t *bitmap, int sms, cudaStream_t st) {
    if (!n) return;
    set_smem_attrs();
    cudaMemsetAsync(big_count, 0, 2 * sizeof(uint32_t), st);   // long-row count, row cursor
    k_extract_small<<<grid_for(n, 8, sms, 8), 256, 0, st>>>(desc, pool, n, perm, iperm,
                                                            row_out, out_src, out_dst, big_rows,
                                                            big_count);
    const size_t bm_bytes = (size_t)((n + 31) / 32) * 4;
    const bool sm = bm_bytes <= SMEM_BITMAP_MAX;
    k_extract_big<<<sms * 4, 256, sm ? bm_bytes : 0, st>>>(desc, pool, n, perm, iperm,
                                                           row_out, out_src, out_dst, big_rows,
                                                           big_count, bitmap, sm ? 1 : 0);
}

}  // namespace cflr
