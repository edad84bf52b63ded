// Host runtime of the CFL-reachability library: contexts, device memory,
// the closure-loop driver and the C ABI of include/cflr.h.
//
// The driver runs Algorithm 1's closure loop with optimisation 1 (paper
// Sec. 2-3): per iteration it builds the work list from the rows that grew in
// the last merge, runs the masked products, deduplicates the candidates into
// the new pairs and appends them.  Every buffer whose size depends on data
// (work list, candidates, hash sets, pool) is checked after the phase that
// fills it; on overflow the phase is re-run with a larger buffer before any
// matrix changes, so growth never loses or duplicates a pair.
#include "cflr.h"
#include "grammar.h"
#include "kernels.cuh"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <array>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

using namespace cflr;

namespace {

enum { ST_CREATED = 0, ST_GRAMMAR = 1, ST_GRAPH = 2, ST_SOLVED = 3 };

enum KernelId {
    KID_SYMBOLIC = 0, KID_BIN0, KID_BIN1, KID_BIN2, KID_BIN3, KID_COMMIT, KID_RESET,
    KID_CAPACITY, KID_SCATTER, KID_PACK, KID_INIT, KID_REHASH, KID_CAPACITY_BIG, N_KID
};
const char *kKernelNames[N_KID] = {
    "k_symbolic", "k_spgemm_bin0", "k_spgemm_bin1", "k_spgemm_bin2", "k_spgemm_bin3",
    "k_commit", "k_reset_dnew", "k_capacity", "k_scatter", "k_pack", "k_init",
    "k_rehash", "k_capacity_big"};

struct CudaError {
    cudaError_t e;
    const char *what;
};

inline void ck(cudaError_t e, const char *what) {
    if (e != cudaSuccess) throw CudaError{e, what};
}

struct Status {
    int code;
    std::string msg;
};

// A named range on the host timeline for profilers (NVTX; costs nothing when
// no tool is attached): the load, the renumbering, the terminal
// initialisation, the solve and its iterations, growths and the extraction.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

inline uint64_t next_pow2(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

struct Runner;

// One stream-ordered memory pool per device for all contexts of this
// library.  Freed blocks stay in the pool (release threshold: none), so
// loading, solving and dropping graphs repeatedly does not map and unmap
// device memory or synchronise the device the way cudaMalloc/cudaFree do.
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};

cudaError_t library_pool(int device, cudaMemPool_t *out) {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (!g_pools[device]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t p;
        cudaError_t e = cudaMemPoolCreate(&p, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = ~0ull;
        e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) return e;
        g_pools[device] = p;
    }
    *out = g_pools[device];
    return cudaSuccess;
}

}  // namespace

struct cflr_ctx {
    cflr_config cfg{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaMemPool_t mpool = nullptr;      // the library's stream-ordered pool on `device`
    int sms = 152;
    size_t smem_optin = 0;
    std::string err;
    int state = ST_CREATED;
    Grammar g;
    // graph and matrices
    uint32_t n = 0;
    uint64_t ignored = 0;
    uint4 *desc = nullptr;              // n_nt * 2 * n descriptors
    uint2 *dn = nullptr;                // n_nt * 2 * n delta counts / append cursors
    uint32_t *occ = nullptr;            // occupancy bits: 2 * n * occ_w words
    uint32_t occ_w = 0;
    uint32_t *pool = nullptr;
    uint64_t pool_cap = 0;
    uint64_t pool_top = 0;              // host mirror between solves
    std::vector<unsigned long long *> htab;
    std::vector<uint2 *> hval;          // witnesses beside htab (cfg.witness only)
    std::vector<uint64_t> hcap;
    std::vector<uint64_t> nnz;
    uint2 *touched = nullptr;           // rows with dnew > 0 (local slot ids)
    uint64_t touched_n = 0;
    uint64_t touched_cap = 0;
    uint32_t iterations = 0;
    // the graph as loaded (device copies, kept for cflr_reset)
    uint64_t m_edges = 0, n_init = 0;
    uint32_t *e_src = nullptr, *e_lab = nullptr, *e_dst = nullptr;
    uint32_t *t_off = nullptr, *t_slot = nullptr;
    size_t t_off_n = 0, t_slot_n = 0;
    // vertex renumbering (null when the caller's order is kept):
    // perm[caller id] = stored id, iperm[stored id] = caller id
    uint32_t *perm = nullptr, *iperm = nullptr;
    std::vector<uint64_t> init_cnt;
    Runner *runner = nullptr;           // cached work buffers of solves led by this context
    // extraction scratch
    // (listed non-terminal ids, unit offsets and their block sums, counters
    // and group totals, long-row list, row bitmaps)
    uint32_t *x_nts = nullptr, *x_bm = nullptr;
    unsigned long long *x_first = nullptr, *x_unit = nullptr, *x_bsum = nullptr,
                       *x_misc = nullptr;
    uint4 *x_bigl = nullptr;
    size_t x_nts_n = 0, x_bm_n = 0, x_first_n = 0, x_unit_n = 0, x_bsum_n = 0, x_misc_n = 0,
           x_bigl_n = 0;
    uint32_t *x_src = nullptr, *x_dst = nullptr;
    uint64_t x_out_cap = 0;
    // accounting
    uint64_t bytes_now = 0, bytes_peak = 0;
    cflr_stats last{};
    Tuning tuning;                      // product-kernel schedule (cflr_autotune)
    std::string grammar_text;           // as loaded (key of the autotune cache)
    std::string cache_path;             // copy of cfg.autotune_cache (cfg points here)
    // profiling (per kernel)
    uint64_t k_launches[N_KID] = {};
    double k_ms[N_KID] = {};
    uint64_t k_bytes[N_KID] = {};

    int fail(int code, const std::string &m) {
        err = m;
        return code;
    }

    void *dalloc(size_t bytes) {
        if (bytes == 0) bytes = 16;
        if (cfg.mem_budget_bytes && bytes_now + bytes > cfg.mem_budget_bytes)
            throw Status{CFLR_ENOMEM, "device memory budget exceeded (" +
                                          std::to_string(bytes_now + bytes) + " > " +
                                          std::to_string(cfg.mem_budget_bytes) + " bytes)"};
        void *p = nullptr;
        cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, mpool, stream);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            throw Status{CFLR_ENOMEM, "device allocation of " + std::to_string(bytes) +
                                          " bytes failed"};
        }
        ck(e, "cudaMallocFromPoolAsync");
        bytes_now += bytes;
        bytes_peak = std::max(bytes_peak, bytes_now);
        return p;
    }
    void dfree(void *p, size_t bytes) {
        if (!p) return;
        if (bytes == 0) bytes = 16;
        cudaFreeAsync(p, stream);
        bytes_now -= std::min(bytes_now, (uint64_t)bytes);
    }

    // a device array of at least `need` elements (its contents are not kept)
    template <typename T>
    void scratch(T *&p, size_t &cap, size_t need) {
        need = std::max<size_t>(need, 1);
        if (p && cap >= need) return;
        if (p) dfree(p, cap * sizeof(T));
        p = nullptr;
        cap = 0;
        p = (T *)dalloc(need * sizeof(T));
        cap = need;
    }
    template <typename T>
    void drop(T *&p, size_t &cap) {
        if (p) dfree(p, cap * sizeof(T));
        p = nullptr;
        cap = 0;
    }
    // extraction scratch
    void free_extract_scratch() {
        drop(x_nts, x_nts_n);
        drop(x_first, x_first_n);
        drop(x_bm, x_bm_n);
        drop(x_unit, x_unit_n);
        drop(x_bsum, x_bsum_n);
        drop(x_misc, x_misc_n);
        drop(x_bigl, x_bigl_n);
    }
    // device staging of cflr_get_pairs's host output
    void free_extract_out() {
        if (x_src) dfree(x_src, x_out_cap * 4);
        if (x_dst) dfree(x_dst, x_out_cap * 4);
        x_src = x_dst = nullptr;
        x_out_cap = 0;
    }

    void free_graph() {
        free_extract_scratch();
        free_extract_out();
        if (e_src) dfree(e_src, m_edges * 4);
        if (e_lab) dfree(e_lab, m_edges * 4);
        if (e_dst) dfree(e_dst, m_edges * 4);
        if (t_off) dfree(t_off, t_off_n * 4);
        if (t_slot) dfree(t_slot, t_slot_n * 4);
        if (perm) dfree(perm, (size_t)n * 4);
        if (iperm) dfree(iperm, (size_t)n * 4);
        perm = iperm = nullptr;
        e_src = e_lab = e_dst = t_off = t_slot = nullptr;
        m_edges = n_init = 0;
        t_off_n = t_slot_n = 0;
        init_cnt.clear();
        uint32_t nt = (uint32_t)g.nts.size();
        if (desc) dfree(desc, (size_t)nt * 2 * n * sizeof(uint4));
        desc = nullptr;
        if (dn) dfree(dn, (size_t)nt * 2 * n * sizeof(uint2));
        dn = nullptr;
        if (occ) dfree(occ, (size_t)2 * n * occ_w * 4);
        occ = nullptr;
        occ_w = 0;
        if (pool) dfree(pool, pool_cap * 4);
        pool = nullptr;
        pool_cap = pool_top = 0;
        for (size_t s = 0; s < htab.size(); s++) {
            if (htab[s]) dfree(htab[s], hcap[s] * 8);
            if (s < hval.size() && hval[s]) dfree(hval[s], hcap[s] * 8);
        }
        htab.clear();
        hval.clear();
        hcap.clear();
        nnz.clear();
        if (touched) dfree(touched, touched_cap * sizeof(uint2));
        touched = nullptr;
        touched_n = touched_cap = 0;
        n = 0;
        iterations = 0;
    }
};

namespace {

// Per-kernel CUDA-event timing on the solve stream (profile mode).
struct Prof {
    cflr_ctx *owner;
    bool on;
    cudaStream_t st;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
    std::vector<cudaEvent_t> free_ev;
    cudaEvent_t get() {
        if (!free_ev.empty()) {
            cudaEvent_t e = free_ev.back();
            free_ev.pop_back();
            return e;
        }
        cudaEvent_t e;
        ck(cudaEventCreate(&e), "cudaEventCreate");
        return e;
    }
    template <class F>
    void run(int kid, F f) {
        if (!on) {
            f();
            ck(cudaGetLastError(), kKernelNames[kid]);
            return;
        }
        cudaEvent_t a = get(), b = get();
        ck(cudaEventRecord(a, st), "cudaEventRecord");
        f();
        ck(cudaGetLastError(), kKernelNames[kid]);
        ck(cudaEventRecord(b, st), "cudaEventRecord");
        marks.push_back({kid, {a, b}});
    }
    void collect() {
        for (auto &m : marks) {
            float ms = 0;
            ck(cudaEventSynchronize(m.second.second), "cudaEventSynchronize");
            ck(cudaEventElapsedTime(&ms, m.second.first, m.second.second), "cudaEventElapsedTime");
            owner->k_ms[m.first] += ms;
            owner->k_launches[m.first] += 1;
            free_ev.push_back(m.second.first);
            free_ev.push_back(m.second.second);
        }
        marks.clear();
    }
    ~Prof() {
        for (auto &m : marks) {
            cudaEventDestroy(m.second.first);
            cudaEventDestroy(m.second.second);
        }
        for (auto e : free_ev) cudaEventDestroy(e);
    }
};

template <class T>
struct DevArr {           // device array owned by a context's accounting
    cflr_ctx *o = nullptr;
    T *p = nullptr;
    size_t n = 0;
    void alloc(cflr_ctx *owner, size_t count) {
        release();
        o = owner;
        n = count;
        p = (T *)o->dalloc(std::max<size_t>(count, 1) * sizeof(T));
    }
    void release() {
        if (p) o->dfree(p, std::max<size_t>(n, 1) * sizeof(T));
        p = nullptr;
        n = 0;
    }
    void ensure(cflr_ctx *owner, size_t count) {   // grow-only, contents dropped
        if (!p || count > n) alloc(owner, count);
    }
    ~DevArr() { release(); }
};

// The closure-loop driver over one or more contexts (a batch).  Every
// context's non-terminals get global slot ids; work items name slots, so
// one launch sequence serves the whole batch.
struct Runner {
    std::vector<cflr_ctx *> cx;
    cflr_ctx *own;
    cudaStream_t st;
    int sms;
    Prof prof;
    std::vector<uint32_t> base;        // first slot of each context
    uint32_t n_slots = 0, n_prods = 0;
    uint32_t max_n = 0;
    std::vector<uint32_t> slot_ctx;    // slot -> context index
    // device tables
    DevArr<uint4 *> d_desc;
    DevArr<uint2 *> d_dn;
    DevArr<uint32_t *> d_pool;
    DevArr<uint32_t> d_n, d_inst, d_occw, d_local;
    DevArr<uint32_t *> d_occ;
    DevArr<unsigned long long *> d_htab;
    DevArr<uint2 *> d_hval;
    DevArr<uint2> d_cand_wit;
    bool wit = false;                  // some context of the batch records witnesses
    DevArr<unsigned long long> d_hmask, d_cand, d_delta, d_nnz;
    DevArr<unsigned long long> d_pool_top, d_pool_cap, d_inst_delta;
    DevArr<uint32_t> d_inst_active, d_inst_iters, d_inst_base;
    DevArr<unsigned long long> d_inst_cnt;
    DevArr<uint2 *> d_inst_out;
    DevArr<uint4> d_prod;
    DevArr<uint4> d_fam;
    DevArr<uint32_t> d_fam_prod;
    DevArr<uint32_t> d_use_off, d_use_code;
    // work buffers
    DevArr<uint2> d_touched[2];
    DevArr<unsigned long long> d_touched_n;   // [2]
    DevArr<uint2> d_groups[N_BINS];
    DevArr<unsigned long long> d_cand_key, d_delta_key;
    DevArr<uint32_t> d_cand_slot, d_delta_slot;
    DevArr<uint32_t> d_bitmap;
    DevArr<uint2> d_big;                      // long delta rows for the symbolic CTA pass
    DevArr<Counters> d_cnt;
    DevArr<LoopCtl> d_ctl;
    DevArr<int> d_parity;
    Counters *h_cnt = nullptr;                // pinned
    LoopCtl *h_ctl = nullptr;                 // pinned
    int *h_parity = nullptr;                  // pinned
    unsigned long long *h_small = nullptr;    // pinned scratch for small reads
    size_t h_small_n = 0;
    uint64_t cand_cap = 0, touched_cap = 0;
    uint64_t group_cap[N_BINS] = {};
    uint64_t regrows = 0;
    uint64_t regrow_kind[3] = {};      // work buffers, pair sets, row pools
    // the iteration as one CUDA graph: a while-loop node around the body
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraphConditionalHandle handle = 0;
    bool graph_valid = false;

    explicit Runner(cflr_ctx *owner) : own(owner), st(owner->stream), sms(owner->sms) {
        prof.owner = own;
        prof.on = own->cfg.profile != 0;
        prof.st = st;
        ck(cudaMallocHost(&h_cnt, sizeof(Counters)), "cudaMallocHost");
        ck(cudaMallocHost(&h_ctl, sizeof(LoopCtl)), "cudaMallocHost");
        ck(cudaMallocHost(&h_parity, sizeof(int)), "cudaMallocHost");
    }
    ~Runner() {
        drop_graph();
        if (h_cnt) cudaFreeHost(h_cnt);
        if (h_ctl) cudaFreeHost(h_ctl);
        if (h_parity) cudaFreeHost(h_parity);
        if (h_small) cudaFreeHost(h_small);
    }
    void drop_graph() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        gexec = nullptr;
        graph = nullptr;
        graph_valid = false;
    }

    // A context's allocation (stream-ordered on the context's stream) made
    // ready for use on the batch stream.
    void *alloc_for(cflr_ctx *c, size_t bytes) {
        void *p = c->dalloc(bytes);
        if (c->stream != st) ck(cudaStreamSynchronize(c->stream), "allocation");
        return p;
    }

    unsigned long long *small(size_t n) {
        if (n > h_small_n) {
            if (h_small) cudaFreeHost(h_small);
            h_small = nullptr;
            h_small_n = std::max<size_t>(n, 64);
            ck(cudaMallocHost(&h_small, h_small_n * 8), "cudaMallocHost");
        }
        return h_small;
    }
    void sync(const char *what) { ck(cudaStreamSynchronize(st), what); }

    // ---- tables ---------------------------------------------------------
    // Point the runner at a batch of contexts (their matrices are loaded):
    // global slot ids, production and use tables, pair counts.
    void bind(std::vector<cflr_ctx *> ctxs) {
        cx = std::move(ctxs);
        regrows = 0;
        regrow_kind[0] = regrow_kind[1] = regrow_kind[2] = 0;
        drop_graph();
        wit = false;
        for (auto *c : cx) wit |= c->cfg.witness != 0;
        if (wit && cand_cap && d_cand_wit.n < cand_cap) d_cand_wit.alloc(own, cand_cap);
        base.clear();
        slot_ctx.clear();
        n_slots = 0;
        max_n = 0;
        for (size_t k = 0; k < cx.size(); k++) {
            base.push_back(n_slots);
            uint32_t nt = (uint32_t)cx[k]->g.nts.size();
            for (uint32_t x = 0; x < nt; x++) slot_ctx.push_back((uint32_t)k);
            n_slots += nt;
            max_n = std::max(max_n, cx[k]->n);
        }
        std::vector<uint4 *> hd(n_slots);
        std::vector<uint2 *> hdn(n_slots);
        std::vector<uint32_t *> hoc(n_slots);
        std::vector<uint32_t> hn(n_slots), hi(n_slots), how(n_slots), hl(n_slots);
        std::vector<unsigned long long> hz(n_slots);
        std::vector<uint4> prods, fams;
        std::vector<uint32_t> fam_prod;
        std::vector<std::vector<uint32_t>> uses((size_t)n_slots * 2);
        for (size_t k = 0; k < cx.size(); k++) {
            cflr_ctx *c = cx[k];
            uint32_t nt = (uint32_t)c->g.nts.size(), b0 = base[k];
            for (uint32_t x = 0; x < nt; x++) {
                hd[b0 + x] = c->desc + (size_t)x * 2 * c->n;
                hdn[b0 + x] = c->dn + (size_t)x * 2 * c->n;
                hoc[b0 + x] = c->occ;
                how[b0 + x] = c->occ_w;
                hl[b0 + x] = x;
                hn[b0 + x] = c->n;
                hi[b0 + x] = (uint32_t)k;
                hz[b0 + x] = c->nnz[x];
            }
            const Grammar &g = c->g;
            std::vector<uint32_t> pid(g.bin_c.size());
            for (size_t p = 0; p < g.bin_c.size(); p++) {
                pid[p] = (uint32_t)prods.size();
                prods.push_back(make_uint4(b0 + g.bin_c[p], b0 + g.bin_a[p], b0 + g.bin_b[p], 0));
            }
            // covered[p][side]: the use of production p on its a (side 0,
            // dA . B) or its b (side 1, A_old . dB) belongs to a family use
            std::vector<std::array<char, 2>> covered(g.bin_c.size(), {0, 0});
            // A family runs as one block product on the delta of the operand
            // its members share (one work-list use instead of F):
            // {offset into fam_prod, F, 1 if every member writes one c | 2
            // if the other operand's slots are consecutive, part}.
            auto add_family = [&](const std::vector<int> &m, int side, bool sc) {
                const uint32_t F = (uint32_t)m.size(), off = (uint32_t)fam_prod.size();
                bool consecutive = true;
                for (uint32_t i = 0; i < F; i++) {
                    fam_prod.push_back(pid[m[i]]);
                    covered[m[i]][side] = 1;
                    const uint32_t gi = side == 0 ? g.bin_b[m[i]] : g.bin_a[m[i]];
                    const uint32_t g0 = side == 0 ? g.bin_b[m[0]] : g.bin_a[m[0]];
                    consecutive &= gi == g0 + i;
                }
                const uint32_t fid = (uint32_t)fams.size();
                fams.push_back(make_uint4(off, F, (sc ? 1u : 0u) | (consecutive ? 2u : 0u),
                                          side == 0 ? PART_A : PART_B));
                const uint32_t x = side == 0 ? g.bin_a[m[0]] : g.bin_b[m[0]];
                uses[(size_t)(b0 + x) * 2 + side].push_back(fid << 2 | PART_F);
            };
            if (own->cfg.form != CFLR_FORM_PLAIN) {
                // Optimisation 4: an indexed family whose members share one
                // operand.  It needs every member and the other operand's
                // members on consecutive slots (their occupancy bits are then
                // consecutive); when the members write different
                // non-terminals, vertex words below 2^21, so that a member tag
                // fits beside the word in the accumulator.
                std::vector<std::vector<int>> members(g.fam_size.size());
                for (size_t p = 0; p < g.bin_c.size(); p++) {
                    if (g.bin_fam[p] < 0) continue;
                    auto &m = members[g.bin_fam[p]];
                    if (m.empty()) m.assign(g.fam_size[g.bin_fam[p]], -1);
                    m[g.bin_member[p]] = (int)p;
                }
                for (const auto &m : members) {
                    const uint32_t F = (uint32_t)m.size();
                    if (F < 2 || F > 1024 || std::count(m.begin(), m.end(), -1)) continue;
                    bool sa = true, sb = true, sc = true, consecutive = true;
                    for (uint32_t i = 0; i < F; i++) {
                        sa &= g.bin_a[m[i]] == g.bin_a[m[0]];
                        sb &= g.bin_b[m[i]] == g.bin_b[m[0]];
                        sc &= g.bin_c[m[i]] == g.bin_c[m[0]];
                        const uint32_t gi = sa ? g.bin_b[m[i]] : g.bin_a[m[i]];
                        const uint32_t g0 = sa ? g.bin_b[m[0]] : g.bin_a[m[0]];
                        consecutive &= gi == g0 + i;
                    }
                    if (sa == sb || !consecutive || (!sc && c->n > (1u << 26))) continue;
                    add_family(m, sa ? 0 : 1, sc);
                }
                // (Grouping the other productions that share the operand, the
                // side and the output non-terminal the same way, as in
                // M -> N1 N3 | N2 N3, was measured slower: 3 % fewer
                // candidates did not pay for the per-member lookups.)
            }
            for (size_t p = 0; p < g.bin_c.size(); p++) {
                if (!covered[p][0])
                    uses[(size_t)(b0 + g.bin_a[p]) * 2 + 0].push_back(pid[p] << 2 | PART_A);
                if (!covered[p][1])
                    uses[(size_t)(b0 + g.bin_b[p]) * 2 + 1].push_back(pid[p] << 2 | PART_B);
            }
            for (size_t p = 0; p < g.unit_c.size(); p++) {
                uint32_t id = (uint32_t)prods.size();
                prods.push_back(make_uint4(b0 + g.unit_c[p], b0 + g.unit_a[p], 0, 1));
                uses[(size_t)(b0 + g.unit_a[p]) * 2 + 0].push_back(id << 2 | PART_U);
            }
        }
        n_prods = (uint32_t)prods.size();
        std::vector<uint32_t> off(1, 0), codes;
        for (auto &u : uses) {
            codes.insert(codes.end(), u.begin(), u.end());
            off.push_back((uint32_t)codes.size());
        }
        const size_t ni = cx.size();
        d_desc.ensure(own, n_slots);
        d_dn.ensure(own, n_slots);
        d_occ.ensure(own, n_slots);
        d_occw.ensure(own, n_slots);
        d_local.ensure(own, n_slots);
        d_pool.ensure(own, n_slots);
        d_n.ensure(own, n_slots);
        d_inst.ensure(own, n_slots);
        d_htab.ensure(own, n_slots);
        d_hval.ensure(own, n_slots);
        d_hmask.ensure(own, n_slots);
        d_cand.ensure(own, n_slots);
        d_delta.ensure(own, n_slots);
        d_nnz.ensure(own, n_slots);
        d_prod.ensure(own, prods.size());
        d_fam.ensure(own, std::max<size_t>(fams.size(), 1));
        d_fam_prod.ensure(own, std::max<size_t>(fam_prod.size(), 1));
        d_use_off.ensure(own, off.size());
        d_use_code.ensure(own, codes.size());
        d_pool_top.ensure(own, ni);
        d_pool_cap.ensure(own, ni);
        d_inst_delta.ensure(own, ni);
        d_inst_active.ensure(own, ni);
        d_inst_iters.ensure(own, ni);
        d_touched_n.ensure(own, 2);
        d_cnt.ensure(own, 1);
        d_ctl.ensure(own, 1);
        d_parity.ensure(own, 1);
        ck(cudaMemcpyAsync(d_desc.p, hd.data(), n_slots * sizeof(uint4 *), cudaMemcpyHostToDevice, st), "H2D");
        ck(cudaMemcpyAsync(d_dn.p, hdn.data(), n_slots * sizeof(uint2 *), cudaMemcpyHostToDevice, st), "H2D");
        ck(cudaMemcpyAsync(d_occ.p, hoc.data(), n_slots * sizeof(uint32_t *), cudaMemcpyHostToDevice, st), "H2D");
        ck(cudaMemcpyAsync(d_occw.p, how.data(), n_slots * 4, cudaMemcpyHostToDevice, st), "H2D");
        ck(cudaMemcpyAsync(d_local.p, hl.data(), n_slots * 4, cudaMemcpyHostToDevice, st), "H2D");
        ck(cudaMemcpyAsync(d_n.p, hn.data(), n_slots * 4, cudaMemcpyHostToDevice, st), "H2D");
        ck(cudaMemcpyAsync(d_inst.p, hi.data(), n_slots * 4, cudaMemcpyHostToDevice, st), "H2D");
        ck(cudaMemcpyAsync(d_nnz.p, hz.data(), n_slots * 8, cudaMemcpyHostToDevice, st), "H2D");
        if (!prods.empty())
            ck(cudaMemcpyAsync(d_prod.p, prods.data(), prods.size() * sizeof(uint4), cudaMemcpyHostToDevice, st), "H2D");
        if (!fams.empty()) {
            ck(cudaMemcpyAsync(d_fam.p, fams.data(), fams.size() * sizeof(uint4), cudaMemcpyHostToDevice, st), "H2D");
            ck(cudaMemcpyAsync(d_fam_prod.p, fam_prod.data(), fam_prod.size() * 4, cudaMemcpyHostToDevice, st), "H2D");
        }
        ck(cudaMemcpyAsync(d_use_off.p, off.data(), off.size() * 4, cudaMemcpyHostToDevice, st), "H2D");
        if (!codes.empty())
            ck(cudaMemcpyAsync(d_use_code.p, codes.data(), codes.size() * 4, cudaMemcpyHostToDevice, st), "H2D");
        // loop state: parity 0, no touched rows, iteration count 0
        std::vector<uint32_t> act(ni);
        for (size_t k = 0; k < ni; k++) act[k] = cx[k]->touched_n ? 1u : 0u;
        ck(cudaMemcpyAsync(d_inst_active.p, act.data(), ni * 4, cudaMemcpyHostToDevice, st), "H2D");
        ck(cudaMemsetAsync(d_inst_iters.p, 0, ni * 4, st), "memset");
        ck(cudaMemsetAsync(d_touched_n.p, 0, 16, st), "memset");
        ck(cudaMemsetAsync(d_parity.p, 0, sizeof(int), st), "memset");
        LoopCtl ctl{};
        ctl.limit = own->cfg.max_iterations ? own->cfg.max_iterations : 0xFFFFFFFFu;
        ctl.stop_on_converge = own->cfg.stop_on_first_converged ? 1u : 0u;
        *h_ctl = ctl;
        ck(cudaMemcpyAsync(d_ctl.p, h_ctl, sizeof(LoopCtl), cudaMemcpyHostToDevice, st), "H2D");
        upload_htabs();
        upload_pools();
        sync("bind");
    }

    void upload_htabs() {
        std::vector<unsigned long long *> ht(n_slots);
        std::vector<uint2 *> hv(n_slots);
        std::vector<unsigned long long> hm(n_slots);
        for (uint32_t s = 0; s < n_slots; s++) {
            cflr_ctx *c = cx[slot_ctx[s]];
            uint32_t x = s - base[slot_ctx[s]];
            ht[s] = c->htab[x];
            hv[s] = x < c->hval.size() ? c->hval[x] : nullptr;
            hm[s] = c->hcap[x] - 1;
        }
        ck(cudaMemcpyAsync(d_htab.p, ht.data(), n_slots * 8, cudaMemcpyHostToDevice, st), "H2D");
        ck(cudaMemcpyAsync(d_hval.p, hv.data(), n_slots * sizeof(uint2 *), cudaMemcpyHostToDevice,
                           st), "H2D");
        ck(cudaMemcpyAsync(d_hmask.p, hm.data(), n_slots * 8, cudaMemcpyHostToDevice, st), "H2D");
        sync("upload htabs");
    }

    // Pool pointers, capacities and (at bind only) the bump counters.
    void upload_pools(bool tops = true) {
        std::vector<unsigned long long> top(cx.size()), cap(cx.size());
        std::vector<uint32_t *> hp(n_slots);
        for (size_t k = 0; k < cx.size(); k++) {
            top[k] = cx[k]->pool_top;
            cap[k] = cx[k]->pool_cap;
        }
        for (uint32_t s = 0; s < n_slots; s++) hp[s] = cx[slot_ctx[s]]->pool;
        if (tops)
            ck(cudaMemcpyAsync(d_pool_top.p, top.data(), cx.size() * 8, cudaMemcpyHostToDevice, st), "H2D");
        ck(cudaMemcpyAsync(d_pool_cap.p, cap.data(), cx.size() * 8, cudaMemcpyHostToDevice, st), "H2D");
        ck(cudaMemcpyAsync(d_pool.p, hp.data(), n_slots * sizeof(uint32_t *), cudaMemcpyHostToDevice, st), "H2D");
        sync("upload pools");
    }

    // After a solve: pool counters, pair counts and iteration counts back to
    // the contexts.
    void download_state(bool add_iterations) {
        const size_t ni = cx.size();
        std::vector<unsigned long long> top(ni), nz(n_slots);
        std::vector<uint32_t> it(ni);
        ck(cudaMemcpyAsync(top.data(), d_pool_top.p, ni * 8, cudaMemcpyDeviceToHost, st), "D2H");
        ck(cudaMemcpyAsync(nz.data(), d_nnz.p, n_slots * 8, cudaMemcpyDeviceToHost, st), "D2H");
        ck(cudaMemcpyAsync(it.data(), d_inst_iters.p, ni * 4, cudaMemcpyDeviceToHost, st), "D2H");
        sync("download state");
        for (size_t k = 0; k < ni; k++) {
            cx[k]->pool_top = top[k];
            if (add_iterations) cx[k]->iterations += it[k];
        }
        for (uint32_t s = 0; s < n_slots; s++) cx[slot_ctx[s]]->nnz[s - base[slot_ctx[s]]] = nz[s];
    }

    SlotTab slots() {
        SlotTab S;
        S.desc = d_desc.p; S.dn = d_dn.p; S.pool = d_pool.p; S.n = d_n.p; S.inst = d_inst.p;
        S.htab = d_htab.p; S.hval = d_hval.p; S.hmask = d_hmask.p; S.cand = d_cand.p; S.delta = d_delta.p;
        S.nnz = d_nnz.p;
        S.occ = d_occ.p; S.occ_w = d_occw.p; S.local = d_local.p;
        S.pool_cap = d_pool_cap.p;
        return S;
    }
    ProdTab prodtab() {
        ProdTab P;
        P.prod = d_prod.p; P.use_off = d_use_off.p; P.use_code = d_use_code.p;
        P.fam = d_fam.p;
        P.fam_prod = d_fam_prod.p;
        return P;
    }
    InstTab insttab() {
        InstTab I;
        I.pool_top = d_pool_top.p; I.pool_cap = d_pool_cap.p; I.delta = d_inst_delta.p;
        I.active = d_inst_active.p; I.iters = d_inst_iters.p;
        return I;
    }
    WorkBufs work() {
        WorkBufs W{};
        W.touched[0] = d_touched[0].p;
        W.touched[1] = d_touched[1].p;
        W.touched_n = d_touched_n.p;
        W.parity = d_parity.p;
        W.touched_cap = touched_cap;
        for (int b = 0; b < N_BINS; b++) {
            W.groups[b] = d_groups[b].p;
            W.group_cap[b] = group_cap[b];
        }
        W.cand_key = d_cand_key.p; W.cand_slot = d_cand_slot.p; W.cand_cap = cand_cap;
        W.cand_wit = wit ? d_cand_wit.p : nullptr;
        W.delta_key = d_delta_key.p; W.delta_slot = d_delta_slot.p;
        W.bitmap_scratch = d_bitmap.p;
        W.bitmap_words = (max_n + 31) / 32;
        W.big_rows = d_big.p;
        W.big_cap = d_big.n;
        W.cnt = d_cnt.p;
        return W;
    }

    // ---- buffers ----------------------------------------------------------
    // smallest first sizes; cfg.initial_capacity lowers them (growth tests)
    uint64_t min_cap(uint64_t dflt) const {
        return own->cfg.initial_capacity ? std::max<uint64_t>(own->cfg.initial_capacity, 32)
                                         : dflt;
    }
    void size_cand(uint64_t cap) {
        cap = std::max<uint64_t>(cap, min_cap(1 << 16));
        if (cap <= cand_cap) return;
        cand_cap = cap;
        d_cand_key.alloc(own, cap);
        d_cand_slot.alloc(own, cap);
        if (wit) d_cand_wit.alloc(own, cap);
        d_delta_key.alloc(own, cap);
        d_delta_slot.alloc(own, cap);
        graph_valid = false;
    }
    // Both touched lists; the list touched[parity] keeps its rows.  Each must
    // hold two rows per new pair (row and column form).
    void size_touched(uint64_t cap, int parity) {
        cap = std::max<uint64_t>(cap, min_cap(1 << 16));
        if (cap <= touched_cap) return;
        DevArr<uint2> keep;
        keep.alloc(own, cap);
        if (parity >= 0 && d_touched[parity].p) {
            ck(cudaMemcpyAsync(keep.p, d_touched[parity].p, touched_cap * sizeof(uint2),
                               cudaMemcpyDeviceToDevice, st), "D2D");
            sync("touched copy");
        }
        const int pin = parity >= 0 ? parity : 0;
        std::swap(d_touched[pin].p, keep.p);
        std::swap(d_touched[pin].n, keep.n);
        d_touched[pin].o = own;
        keep.release();
        d_touched[pin ^ 1].alloc(own, cap);
        touched_cap = cap;
        // a listed row has more than 64 delta entries, and the deltas of
        // one iteration hold at most touched_cap entries
        d_big.ensure(own, cap / 64 + 1024);
        graph_valid = false;
    }
    void size_groups(int b, uint64_t cap) {
        cap = std::max<uint64_t>(cap, min_cap(1 << 14));
        if (cap <= group_cap[b]) return;
        group_cap[b] = cap;
        d_groups[b].alloc(own, cap);
        graph_valid = false;
    }
    void init_buffers(uint64_t cand_hint, uint64_t touched_in) {
        const uint64_t ic = own->cfg.initial_capacity;
        size_cand(ic ? std::max<uint64_t>(ic, 32) : cand_hint);
        size_touched(std::max<uint64_t>(2 * cand_cap, touched_in), -1);
        // work lists: the lightest bins take most groups; a solve touching
        // many rows starts with room for four groups per row in them and
        // one per two rows in the others
        for (int b = 0; b < N_BINS; b++)
            size_groups(b, ic ? ic
                              : std::max<uint64_t>(b < 2 ? 1 << 18 : 1 << 14,
                                                   b < 2 ? 4 * touched_in : touched_in / 2));
        if (max_n > 200 * 1024 * 8) {   // bitmaps do not fit shared memory
            uint64_t words = (max_n + 31) / 32;
            d_bitmap.ensure(own, words * (uint64_t)sms * 8);
            graph_valid = false;
        }
    }

    void grow_htab(uint32_t s, uint64_t need) {
        cflr_ctx *c = cx[slot_ctx[s]];
        uint32_t x = s - base[slot_ctx[s]];
        // room for eight times the need (the set is at most an eighth full
        // afterwards): a fresh solve's sets grow through several iterations,
        // and every growth costs a host round trip and a re-run of the commit
        // (58.5 -> 51.4 ms for the first solve of the 200k alias graph, with
        // the pool quadrupling instead of doubling)
        uint64_t cap = next_pow2(std::max<uint64_t>(8 * need, 1024));
        unsigned long long *nt = (unsigned long long *)alloc_for(c, cap * 8);
        ck(cudaMemsetAsync(nt, 0xFF, cap * 8, st), "memset");
        uint2 *nv = c->hval[x] ? (uint2 *)alloc_for(c, cap * 8) : nullptr;
        prof.run(KID_REHASH, [&] {
            launch_rehash(c->htab[x], c->hval[x], c->hcap[x], nt, nv, cap,
                          &d_cnt.p->overflow, sms, st);
        });
        own->k_bytes[KID_REHASH] += c->hcap[x] * 8 + need * 8;
        // the old table is freed on the context's stream: when that is the
        // batch stream the free is ordered after the rehash and no wait is
        // needed (the rehash reports through the loop status read next; a
        // points-to solve grows hundreds of sets, and one wait each had cost
        // about 30 % of its first solve)
        if (c->stream != st) sync("rehash");
        c->dfree(c->htab[x], c->hcap[x] * 8);
        if (c->hval[x]) c->dfree(c->hval[x], c->hcap[x] * 8);
        c->htab[x] = nt;
        c->hval[x] = nv;
        c->hcap[x] = cap;
        regrows++;
        regrow_kind[1]++;
    }

    void grow_pool(size_t k, uint64_t top) {
        cflr_ctx *c = cx[k];
        uint64_t cap = std::max<uint64_t>(4 * c->pool_cap, top + top / 2 + (1 << 20));
        cap = std::min<uint64_t>(cap, 0xFFFFFFF0ull);
        if (cap <= c->pool_cap || top > cap)
            throw Status{CFLR_ENOMEM, "row pool exceeds 2^32 entries"};
        uint32_t *np = (uint32_t *)alloc_for(c, cap * 4);
        ck(cudaMemcpyAsync(np, c->pool, c->pool_cap * 4, cudaMemcpyDeviceToDevice, st), "D2D");
        if (c->stream != st) sync("pool copy");    // the free runs on the context's stream
        c->dfree(c->pool, c->pool_cap * 4);
        c->pool = np;       // rows address the pool by offset, so they stay valid
        c->pool_cap = cap;
        regrows++;
        regrow_kind[2]++;
    }

    // ---- the iteration --------------------------------------------------
    const Tuning &tuning() const { return own->tuning; }
    // Products of one iteration (symbolic pass and the four bins).
    void launch_products(const SlotTab &S, const ProdTab &P, const WorkBufs &W, bool timed) {
        auto run = [&](int kid, auto f) { if (timed) prof.run(kid, f); else f(); };
        if (own->cfg.form == CFLR_FORM_PLAIN) {
            // one launch sequence per production, like one library mxm each
            for (uint32_t p = 0; p < n_prods; p++) {
                run(KID_SYMBOLIC, [&] { launch_symbolic(S, P, W, (int)p, tuning(), sms, st); });
                for (int b = 0; b < N_BINS; b++)
                    run(KID_BIN0 + b,
                        [&] { launch_spgemm(b, S, P, W, max_n, tuning(), sms, st); });
                // group counts, claim cursors (adjacent) and the long-row
                // list start again
                ck(cudaMemsetAsync(d_cnt.p->groups, 0,
                                   sizeof(d_cnt.p->groups) + sizeof(d_cnt.p->claim), st),
                   "memset");
                ck(cudaMemsetAsync(&d_cnt.p->big_n, 0, sizeof(d_cnt.p->big_n), st), "memset");
            }
        } else {
            run(KID_SYMBOLIC, [&] { launch_symbolic(S, P, W, -1, tuning(), sms, st); });
            for (int b = 0; b < N_BINS; b++)
                run(KID_BIN0 + b, [&] { launch_spgemm(b, S, P, W, max_n, tuning(), sms, st); });
        }
    }
    // Commit and union, from the dedupe (stage 0), the capacity pass
    // (stage 1) or the scatter (stage 2), then the end of the iteration.
    void launch_merge(const SlotTab &S, const InstTab &I, const WorkBufs &W, int stage,
                      bool count_iteration, bool in_graph, bool timed) {
        auto run = [&](int kid, auto f) { if (timed) prof.run(kid, f); else f(); };
        if (stage <= 0) {
            // the previous deltas end before the commit counts the new ones
            run(KID_RESET, [&] { launch_reset_dnew(S, W, sms, st); });
            run(KID_COMMIT, [&] { launch_commit(S, W, n_slots, sms, st); });
        }
        if (stage <= 1) {
            run(KID_CAPACITY, [&] { launch_capacity(S, I, W, sms, st); });
            run(KID_CAPACITY_BIG, [&] { launch_capacity_big(S, I, W, max_n, sms, st); });
        }
        run(KID_SCATTER, [&] { launch_scatter(S, W, sms, st); });
        run(KID_PACK, [&] { launch_pack(S, W, sms, st); });
        launch_iter_end(S, I, W, d_ctl.p, n_slots, (uint32_t)cx.size(), count_iteration,
                        handle, in_graph, st);
        ck(cudaGetLastError(), "k_iter_end");
    }
    // One whole iteration as a launch sequence (also the graph's body).
    void launch_iteration(bool in_graph, bool timed) {
        const SlotTab S = slots();
        const ProdTab P = prodtab();
        const InstTab I = insttab();
        const WorkBufs W = work();
        launch_iter_begin(S, I, W, n_slots, (uint32_t)cx.size(), st);
        launch_products(S, P, W, timed);
        bool growth = true;
        for (auto *c : cx) growth &= c->cfg.test_fixed_pair_sets == 0;
        launch_check(S, W, n_slots, growth, st);
        launch_merge(S, I, W, 0, true, in_graph, timed);
    }

    void ensure_graph() {
        if (graph_valid) return;
        drop_graph();
        prepare_launch_attributes();
        ck(cudaGraphCreate(&graph, 0), "cudaGraphCreate");
        ck(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault),
           "cudaGraphConditionalHandleCreate");
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        ck(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp), "cudaGraphAddNode");
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        ck(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal),
           "cudaStreamBeginCaptureToGraph");
        launch_iteration(true, false);
        cudaGraph_t captured = nullptr;
        ck(cudaStreamEndCapture(st, &captured), "cudaStreamEndCapture");
        ck(cudaGraphInstantiate(&gexec, graph, 0), "cudaGraphInstantiate");
        graph_valid = true;
    }

    void read_status() {
        ck(cudaMemcpyAsync(h_cnt, d_cnt.p, sizeof(Counters), cudaMemcpyDeviceToHost, st), "D2H");
        ck(cudaMemcpyAsync(h_ctl, d_ctl.p, sizeof(LoopCtl), cudaMemcpyDeviceToHost, st), "D2H");
        ck(cudaMemcpyAsync(h_parity, d_parity.p, sizeof(int), cudaMemcpyDeviceToHost, st), "D2H");
        sync("status");
    }
    void clear_overflow() {
        ck(cudaMemsetAsync(&d_cnt.p->overflow, 0, sizeof(unsigned), st), "memset");
    }

    // New size of a work buffer that overflowed at `count` entries.  The
    // counts keep rising for several iterations and an overflow costs the
    // iteration's products, so the buffers triple (half again under a
    // memory budget).
    uint64_t regrow_size(uint64_t count) const {
        return own->cfg.mem_budget_bytes ? count * 3 / 2 : count * 3;
    }

    // Grow what the last (stopped) iteration overflowed and finish it.
    // Returns false when the iteration must be run again from its start.
    bool recover() {
        Range range("cflr: grow buffers");
        const unsigned st_bits = h_ctl->status;
        if (st_bits & OVF_FULL)
            throw Status{CFLR_ECUDA, "a pair set filled up: a hash probe passed over the "
                                     "whole table (the pair sets were kept at their size)"};
        if (st_bits & OVF_BOUNDS)
            throw Status{CFLR_ECUDA, "an index failed its bounds check (checked build)"};
        if (st_bits & (OVF_GROUPS | OVF_CAND)) {       // nothing was committed
            for (int b = 0; b < N_BINS; b++) {
                uint64_t want = h_cnt->groups[b] > group_cap[b] ? regrow_size(h_cnt->groups[b]) : 0;
                if ((st_bits & OVF_GROUPS) && own->cfg.form == CFLR_FORM_PLAIN)
                    want = std::max<uint64_t>(want, 2 * group_cap[b]);   // counts reset per production
                if (want) size_groups(b, want);
            }
            if (st_bits & OVF_CAND) {
                size_cand(regrow_size(h_cnt->cand));
                size_touched(2 * cand_cap, *h_parity);
            }
            regrows++;
            regrow_kind[0]++;
            return false;
        }
        const SlotTab S = slots();
        const InstTab I = insttab();
        const WorkBufs W = work();
        if (st_bits & OVF_HASH) {                      // grow pair sets, then commit
            std::vector<unsigned long long> nz(n_slots), cd(n_slots);
            ck(cudaMemcpyAsync(nz.data(), d_nnz.p, n_slots * 8, cudaMemcpyDeviceToHost, st), "D2H");
            ck(cudaMemcpyAsync(cd.data(), d_cand.p, n_slots * 8, cudaMemcpyDeviceToHost, st), "D2H");
            sync("hash sizes");
            for (uint32_t s = 0; s < n_slots; s++) {
                cflr_ctx *c = cx[slot_ctx[s]];
                uint32_t x = s - base[slot_ctx[s]];
                if (2 * (nz[s] + cd[s]) > c->hcap[x]) grow_htab(s, nz[s] + cd[s]);
            }
            upload_htabs();
            clear_overflow();
            launch_merge(S, I, W, 0, true, false, true);
            read_status();
        }
        for (int guard = 0; h_ctl->status & OVF_POOL; guard++) {   // grow pools, redo the union
            if (guard > 8) throw Status{CFLR_ENOMEM, "pool growth did not converge"};
            std::vector<unsigned long long> top(cx.size());
            ck(cudaMemcpyAsync(top.data(), d_pool_top.p, cx.size() * 8, cudaMemcpyDeviceToHost, st), "D2H");
            sync("pool tops");
            for (size_t k = 0; k < cx.size(); k++)
                if (top[k] > cx[k]->pool_cap) grow_pool(k, top[k]);
            upload_pools(false);
            clear_overflow();
            launch_merge(S, I, W, 1, true, false, true);
            read_status();
        }
        if (h_ctl->status & OVF_FULL)
            throw Status{CFLR_ECUDA, "a pair set filled up: a hash probe passed over the "
                                     "whole table"};
        if (h_ctl->status & OVF_BOUNDS)
            throw Status{CFLR_ECUDA, "an index failed its bounds check (checked build)"};
        if (h_ctl->status) throw Status{CFLR_ECUDA, "internal: unexpected loop status"};
        return true;
    }

    // Run closure iterations until the fixpoint (true) or the iteration
    // limit (false).
    bool run_loop() {
        const bool use_graph = own->cfg.form == CFLR_FORM_GRAPH && !prof.on;
        // A buffer growth changes the pointers the graph was captured with,
        // so after one the loop runs host-launched iterations until one of
        // them needs no growth, and only then captures the graph again (a
        // fresh context grows several buffers in its first iterations).
        bool settled = graph_valid;
        for (;;) {
            if (use_graph && settled) {
                Range range("cflr: closure loop (CUDA graph)");
                ensure_graph();
                ck(cudaGraphLaunch(gexec, st), "cudaGraphLaunch");
                read_status();
            } else {
                Range range("cflr: closure iteration");
                launch_iteration(false, true);
                read_status();
            }
            prof.collect();
            settled = h_ctl->status == 0;
            if (h_ctl->status && !recover()) continue;
            if (h_ctl->last_delta == 0) return true;
            if (h_ctl->iter >= h_ctl->limit) return false;
            if (h_ctl->stop_on_converge && first_converged()) return false;
        }
    }

    // True when some instance of the batch reached its fixpoint.
    bool first_converged() {
        std::vector<uint32_t> act(cx.size());
        ck(cudaMemcpyAsync(act.data(), d_inst_active.p, cx.size() * 4, cudaMemcpyDeviceToHost, st), "D2H");
        sync("active");
        for (uint32_t a : act)
            if (!a) return true;
        return false;
    }

    // Pending delta rows of each context into the "in" touched list.
    void import_touched() {
        uint64_t total = 0;
        for (auto *c : cx) total += c->touched_n;
        size_touched(std::max<uint64_t>(total, 2 * cand_cap), -1);
        uint64_t at = 0;
        for (size_t k = 0; k < cx.size(); k++) {
            cflr_ctx *c = cx[k];
            if (c->touched_n)
                launch_remap_touched(c->touched, c->touched_n, base[k], d_touched[0].p + at, st);
            ck(cudaGetLastError(), "remap");
            at += c->touched_n;
        }
        unsigned long long *h = small(2);
        h[0] = at;
        h[1] = 0;
        ck(cudaMemcpyAsync(d_touched_n.p, h, 16, cudaMemcpyHostToDevice, st), "H2D");
        ck(cudaMemsetAsync(d_parity.p, 0, sizeof(int), st), "memset");
        sync("import");
    }

    // Save the pending delta rows of each context (local slot ids), split
    // on the device.
    void export_touched() {
        unsigned long long *h = small(2);
        ck(cudaMemcpyAsync(h, d_touched_n.p, 16, cudaMemcpyDeviceToHost, st), "D2H");
        ck(cudaMemcpyAsync(h_parity, d_parity.p, sizeof(int), cudaMemcpyDeviceToHost, st), "D2H");
        sync("export");
        const int par = *h_parity;
        const uint64_t n_in = h[par];
        const size_t ni = cx.size();
        if (n_in == 0) {
            for (auto *c : cx) c->touched_n = 0;
            return;
        }
        if (ni == 1) {
            // one instance: its slots are the batch's, so the list is copied
            // as it is (a split would serialise on one cursor)
            cflr_ctx *c = cx[0];
            if (n_in > c->touched_cap) {
                if (c->touched) c->dfree(c->touched, c->touched_cap * sizeof(uint2));
                c->touched = nullptr;
                c->touched_cap = std::max<uint64_t>(n_in + n_in / 4, 1024);
                c->touched = (uint2 *)alloc_for(c, c->touched_cap * sizeof(uint2));
            }
            c->touched_n = n_in;
            ck(cudaMemcpyAsync(c->touched, d_touched[par].p, n_in * sizeof(uint2),
                               cudaMemcpyDeviceToDevice, st), "D2D touched");
            sync("export copy");
            return;
        }
        d_inst_cnt.ensure(own, ni);
        d_inst_base.ensure(own, ni);
        d_inst_out.ensure(own, ni);
        ck(cudaMemsetAsync(d_inst_cnt.p, 0, ni * 8, st), "memset");
        launch_touched_count(d_touched[par].p, n_in, d_inst.p, d_inst_cnt.p, st);
        ck(cudaGetLastError(), "touched count");
        std::vector<unsigned long long> cnt(ni);
        ck(cudaMemcpyAsync(cnt.data(), d_inst_cnt.p, ni * 8, cudaMemcpyDeviceToHost, st), "D2H");
        sync("export counts");
        std::vector<uint2 *> outp(ni);
        std::vector<uint32_t> b(ni);
        for (size_t k = 0; k < ni; k++) {
            cflr_ctx *c = cx[k];
            if (cnt[k] > c->touched_cap) {
                if (c->touched) c->dfree(c->touched, c->touched_cap * sizeof(uint2));
                c->touched = nullptr;
                c->touched_cap = std::max<uint64_t>(cnt[k] + cnt[k] / 4, 1024);
                c->touched = (uint2 *)alloc_for(c, c->touched_cap * sizeof(uint2));
            }
            c->touched_n = cnt[k];
            outp[k] = c->touched;
            b[k] = base[k];
        }
        ck(cudaMemcpyAsync(d_inst_out.p, outp.data(), ni * sizeof(uint2 *), cudaMemcpyHostToDevice, st), "H2D");
        ck(cudaMemcpyAsync(d_inst_base.p, b.data(), ni * 4, cudaMemcpyHostToDevice, st), "H2D");
        ck(cudaMemsetAsync(d_inst_cnt.p, 0, ni * 8, st), "memset");
        launch_touched_split(d_touched[par].p, n_in, d_inst.p, d_inst_base.p, d_inst_out.p,
                             d_inst_cnt.p, st);
        ck(cudaGetLastError(), "touched split");
        sync("export split");
    }

    // Byte and work totals of the finished solve, from the loop control.
    void account() {
        read_status();
        own->k_bytes[KID_SYMBOLIC] += h_ctl->bytes_sym;
        for (int b = 0; b < N_BINS; b++) own->k_bytes[KID_BIN0 + b] += h_ctl->bytes_bin[b];
        own->k_bytes[KID_COMMIT] += 20 * h_ctl->total_cand + 20 * h_ctl->total_delta +
                                    8 * h_ctl->total_touched_out;
        own->k_bytes[KID_RESET] += 12 * h_ctl->total_touched_in;
        own->k_bytes[KID_CAPACITY] += 24 * h_ctl->total_touched_out + h_ctl->bytes_move[0];
        own->k_bytes[KID_CAPACITY_BIG] += h_ctl->bytes_move[1];
        own->k_bytes[KID_SCATTER] += 60 * h_ctl->total_delta;
        own->k_bytes[KID_PACK] += 24 * h_ctl->total_delta + 24 * h_ctl->total_touched_out;
    }
};

Runner &runner_of(cflr_ctx *c) {
    if (!c->runner) c->runner = new Runner(c);
    c->runner->prof.on = c->cfg.profile != 0;
    return *c->runner;
}

// Breadth-first order of the vertices over the edges taken as undirected,
// each unvisited vertex (in id order) starting a new search.  Vertices that
// reach one another through few edges get nearby ids, so the rows of the
// closure matrices fall into few 32-bit words.  Returns order[k] = the
// caller id of stored vertex k.
std::vector<uint32_t> locality_order(uint32_t n, uint64_t m, const uint32_t *src,
                                     const uint32_t *dst) {
    // Undirected adjacency (CSR).  Degree counting and the fill run on up to
    // eight host threads, each owning a range of vertices: a thread scans
    // every edge in order and touches only its own vertices, so each list
    // keeps the edge order (the order a one-thread fill gives).
    unsigned T = std::min(std::max(1u, std::thread::hardware_concurrency()), 8u);
    if (m < (1u << 18)) T = 1;
    std::vector<uint64_t> off((size_t)n + 1, 0);
    std::vector<uint32_t> adj(2 * m);
    auto on_threads = [&](auto &&work) {
        std::vector<std::thread> th;
        for (unsigned t = 0; t < T; t++) {
            const uint32_t v0 = (uint32_t)((uint64_t)n * t / T);
            const uint32_t v1 = (uint32_t)((uint64_t)n * (t + 1) / T);
            try {
                th.emplace_back(work, v0, v1);
            } catch (const std::system_error &) {
                work(v0, v1);      // no thread to be had: do that range here
            }
        }
        for (auto &x : th) x.join();
    };
    on_threads([&](uint32_t v0, uint32_t v1) {
        uint64_t *o = off.data() + 1;
        for (uint64_t e = 0; e < m; e++) {
            if (src[e] - v0 < v1 - v0) o[src[e]]++;
            if (dst[e] - v0 < v1 - v0) o[dst[e]]++;
        }
    });
    for (uint32_t v = 0; v < n; v++) off[v + 1] += off[v];
    on_threads([&](uint32_t v0, uint32_t v1) {
        std::vector<uint64_t> cur(off.begin() + v0, off.begin() + v1);
        uint64_t *c = cur.data() - v0;     // indexed by vertex, v0 <= v < v1
        for (uint64_t e = 0; e < m; e++) {
            const uint32_t s = src[e], d = dst[e];
            if (s - v0 < v1 - v0) adj[c[s]++] = d;
            if (d - v0 < v1 - v0) adj[c[d]++] = s;
        }
    });
    std::vector<uint32_t> order;
    order.reserve(n);
    std::vector<uint8_t> seen(n, 0);
    for (uint32_t s = 0; s < n; s++) {
        if (seen[s]) continue;
        seen[s] = 1;
        size_t head = order.size();
        order.push_back(s);
        while (head < order.size()) {
            // the lists of vertices a few places ahead in the queue are far
            // apart in memory: fetch their offsets and heads early (a miss per
            // vertex was most of the pass: 16.8 -> 11.2 ms on 200k vertices
            // and 1.1M edges, one Grace core)
            if (head + 16 < order.size()) __builtin_prefetch(&off[order[head + 16]]);
            if (head + 8 < order.size()) __builtin_prefetch(&adj[off[order[head + 8]]]);
            const uint32_t u = order[head++];
            for (uint64_t q = off[u]; q < off[(size_t)u + 1]; q++) {
                const uint32_t v = adj[q];
                if (!seen[v]) {
                    seen[v] = 1;
                    order.push_back(v);
                }
            }
        }
    }
    return order;
}

// Device arrays of one call, freed on every way out of it.
struct TempArrays {
    cflr_ctx *c;
    std::vector<std::pair<void *, size_t>> held;
    template <typename T>
    T *get(size_t count) {
        const size_t b = std::max<size_t>(count * sizeof(T), 16);
        void *p = c->dalloc(b);
        held.push_back({p, b});
        return (T *)p;
    }
    ~TempArrays() {
        for (auto &h : held) c->dfree(h.first, h.second);
    }
};

// The order locality_order gives, found on the device from the uploaded
// edges c->e_src / c->e_dst (caller ids) into c->perm / c->iperm (the
// kernels' steps are described with launch_rn_adjacency).  Returns false,
// with nothing to keep, for graphs it does not take: 2^32 edges or more, a
// vertex with more than RENUM_LIST_MAX edge ends, components that did not
// settle in 128 passes, or scratch beyond the context's memory budget.
bool device_order_steps(cflr_ctx *c, uint32_t n, uint64_t m);

bool device_order(cflr_ctx *c, uint32_t n, uint64_t m) {
    if (m >= (1ull << 32)) return false;
    try {
        return device_order_steps(c, n, m);
    } catch (const Status &s) {
        // no room for the search's scratch under the memory budget: the host
        // search needs none (the scratch is freed on the way out)
        if (s.code == CFLR_ENOMEM) return false;
        throw;
    }
}

bool device_order_steps(cflr_ctx *c, uint32_t n, uint64_t m) {
    Range range("cflr: vertex renumbering (device)");
    cudaStream_t st = c->stream;
    const int sms = c->sms;
    TempArrays tmp{c, {}};
    uint32_t *word = tmp.get<uint32_t>(8);          // max degree, long lists, flags
    unsigned long long *tot = tmp.get<unsigned long long>(2);
    auto read_word = [&](const void *d, size_t bytes, void *to) {
        ck(cudaMemcpyAsync(to, d, bytes, cudaMemcpyDeviceToHost, st), "D2H");
        ck(cudaStreamSynchronize(st), "sync renumbering");
    };
    uint32_t *deg = tmp.get<uint32_t>(n);
    unsigned long long *off = tmp.get<unsigned long long>((size_t)n + 1);
    unsigned long long *bsum = tmp.get<unsigned long long>((size_t)n / 1024 + 2);
    launch_rn_adjacency(c->e_src, c->e_dst, m, n, deg, word, sms, st);
    launch_exclusive_scan(deg, n, off, bsum, off + n, st);
    ck(cudaGetLastError(), "renumbering: degrees");
    uint32_t max_deg = 0;
    read_word(word, 4, &max_deg);
    if (max_deg > RENUM_LIST_MAX) return false;
    unsigned long long *adj = tmp.get<unsigned long long>(2 * m);
    unsigned long long *cur = tmp.get<unsigned long long>(n);
    uint32_t *big = tmp.get<uint32_t>(n);
    launch_rn_fill(c->e_src, c->e_dst, m, n, off, cur, adj, big, word + 1, max_deg, sms, st);
    uint32_t *parent = tmp.get<uint32_t>(n);
    uint32_t *lvl = tmp.get<uint32_t>(n);
    unsigned long long *key = tmp.get<unsigned long long>(n);
    launch_rn_init(n, parent, lvl, key, c->iperm, sms, st);
    ck(cudaGetLastError(), "renumbering: adjacency");
    for (int pass = 0;; pass++) {
        if (pass == 128) return false;
        launch_rn_cc_pass(c->e_src, c->e_dst, m, n, parent, (unsigned *)(word + 2), sms, st);
        ck(cudaGetLastError(), "renumbering: components");
        uint32_t more = 0;
        read_word(word + 2, 4, &more);
        if (!more) break;
    }
    uint32_t *cnt = tmp.get<uint32_t>(n);
    uint32_t *is_root = tmp.get<uint32_t>(n);
    unsigned long long *comp_off = tmp.get<unsigned long long>(n);
    unsigned long long *roff = tmp.get<unsigned long long>(n);
    launch_rn_count(parent, n, cnt, is_root, sms, st);
    launch_exclusive_scan(cnt, n, comp_off, bsum, nullptr, st);
    launch_exclusive_scan(is_root, n, roff, bsum, tot, st);
    uint32_t *F = tmp.get<uint32_t>(n), *F2 = tmp.get<uint32_t>(n);
    uint32_t *seg[2][3];      // per root: segment first, segment end, earlier count
    for (int b = 0; b < 2; b++)
        for (int k = 0; k < 3; k++) seg[b][k] = tmp.get<uint32_t>(n);
    uint32_t *won = tmp.get<uint32_t>(n);
    unsigned long long *woff = tmp.get<unsigned long long>((size_t)n + 1);
    launch_rn_roots(parent, n, roff, comp_off, F, lvl, seg[0][0], seg[0][1], seg[0][2], c->perm,
                    c->iperm, sms, st);
    ck(cudaGetLastError(), "renumbering: roots");
    unsigned long long fsize = 0;
    read_word(tot, 8, &fsize);
    uint64_t placed = 0;
    int b = 0;
    for (uint32_t level = 0; fsize; level++) {
        if (level > n) throw Status{CFLR_ECUDA, "internal: the device search did not end"};
        placed += fsize;
        launch_rn_claim(F, (uint32_t)fsize, off, adj, lvl, key, won, sms, st);
        launch_exclusive_scan(won, (uint32_t)fsize, woff, bsum, woff + fsize, st);
        launch_rn_write(F, (uint32_t)fsize, off, adj, lvl, key, woff, F2, level, parent, comp_off,
                        seg[b][0], seg[b][1], seg[b][2], seg[b ^ 1][0], seg[b ^ 1][1],
                        seg[b ^ 1][2], c->perm, c->iperm, n, sms, st);
        ck(cudaGetLastError(), "renumbering: level");
        unsigned long long next = 0;
        read_word(woff + fsize, 8, &next);
        std::swap(F, F2);
        b ^= 1;
        fsize = next;
    }
    if (placed != n)
        throw Status{CFLR_ECUDA, "internal: the device search placed " + std::to_string(placed) +
                                     " of " + std::to_string(n) + " vertices"};
    launch_rn_check(c->perm, c->iperm, n, (unsigned *)(word + 3), sms, st);
    ck(cudaGetLastError(), "renumbering: check");
    uint32_t bad = 0;
    read_word(word + 3, 4, &bad);
    if (bad) throw Status{CFLR_ECUDA, "internal: the device order is not a permutation"};
    return true;
}

// One pass over the input edges on up to eight host threads (contiguous
// ranges): the first edge with a vertex id >= n (m when there is none), the
// edges per label a production uses, and the other edges.
struct EdgeScan {
    uint64_t bad = 0;
    std::vector<uint64_t> per_label;
    uint64_t ignored = 0;
};
EdgeScan scan_edges(const Grammar &g, uint32_t n, uint64_t m, const uint32_t *src,
                    const uint32_t *lab, const uint32_t *dst) {
    const uint32_t nterm = (uint32_t)g.terms.size();
    std::vector<uint8_t> used(nterm);
    for (uint32_t l = 0; l < nterm; l++) used[l] = !g.term_nts[l].empty();
    unsigned T = std::min(std::max(1u, std::thread::hardware_concurrency()), 8u);
    if (m < (1u << 18)) T = 1;
    std::vector<EdgeScan> part(T);
    auto work = [&](unsigned t) {
        EdgeScan &r = part[t];
        const uint64_t e0 = m * t / T, e1 = m * (t + 1) / T;
        r.bad = m;
        r.per_label.assign(nterm, 0);
        for (uint64_t e = e0; e < e1; e++) {
            if ((src[e] >= n || dst[e] >= n) && r.bad == m) r.bad = e;
            if (lab[e] < nterm && used[lab[e]]) r.per_label[lab[e]]++;
            else r.ignored++;
        }
    };
    std::vector<std::thread> th;
    for (unsigned t = 1; t < T; t++) {
        try {
            th.emplace_back(work, t);
        } catch (const std::system_error &) {
            work(t);                 // no thread to be had: that range here
        }
    }
    work(0);
    for (auto &x : th) x.join();
    EdgeScan out;
    out.bad = m;
    out.per_label.assign(nterm, 0);
    for (auto &r : part) {
        out.bad = std::min(out.bad, r.bad);
        out.ignored += r.ignored;
        for (uint32_t l = 0; l < nterm; l++) out.per_label[l] += r.per_label[l];
    }
    return out;
}

// Copy the graph to the device and size the matrices (cflr_load_graph).
void upload_graph(cflr_ctx *c, uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *lab,
                  const uint32_t *dst, const EdgeScan &scan) {
    const Grammar &g = c->g;
    const uint32_t nt = (uint32_t)g.nts.size(), nterm = (uint32_t)g.terms.size();
    cudaStream_t st = c->stream;
    // per-label edge counts -> per-non-terminal initial counts
    const std::vector<uint64_t> &per_label = scan.per_label;
    const uint64_t ignored = scan.ignored;
    c->init_cnt.assign(nt, 0);
    for (uint32_t l = 0; l < nterm; l++)
        for (uint32_t A : g.term_nts[l]) c->init_cnt[A] += per_label[l];
    for (uint32_t A : g.eps) c->init_cnt[A] += n;
    c->n_init = 0;
    for (uint32_t A = 0; A < nt; A++) c->n_init += c->init_cnt[A];
    c->ignored = ignored;
    c->n = n;
    c->m_edges = m;
    c->e_src = (uint32_t *)c->dalloc(m * 4);
    c->e_lab = (uint32_t *)c->dalloc(m * 4);
    c->e_dst = (uint32_t *)c->dalloc(m * 4);
    if (m) {
        ck(cudaMemcpyAsync(c->e_src, src, m * 4, cudaMemcpyHostToDevice, st), "H2D edges");
        ck(cudaMemcpyAsync(c->e_lab, lab, m * 4, cudaMemcpyHostToDevice, st), "H2D edges");
        ck(cudaMemcpyAsync(c->e_dst, dst, m * 4, cudaMemcpyHostToDevice, st), "H2D edges");
    }
    if (!c->cfg.keep_vertex_order && n > 0) {
        c->perm = (uint32_t *)c->dalloc((size_t)n * 4);
        c->iperm = (uint32_t *)c->dalloc((size_t)n * 4);
        const int where = c->cfg.order_on_device;
        const bool on_device = where > 0 || (where == 0 && m >= (1u << 18));
        if (!on_device || !device_order(c, n, m)) {
            Range range("cflr: vertex renumbering (host)");
            const std::vector<uint32_t> order = locality_order(n, m, src, dst);
            std::vector<uint32_t> perm(n);
            for (uint32_t k = 0; k < n; k++) perm[order[k]] = k;
            ck(cudaMemcpyAsync(c->perm, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st),
               "H2D order");
            ck(cudaMemcpyAsync(c->iperm, order.data(), (size_t)n * 4, cudaMemcpyHostToDevice,
                               st),
               "H2D order");
            // the host vectors die here: wait for the copies that read them
            ck(cudaStreamSynchronize(st), "sync order");
        }
        launch_permute_ids(c->e_src, m, c->perm, c->sms, st);
        launch_permute_ids(c->e_dst, m, c->perm, c->sms, st);
    }
    std::vector<uint32_t> toff(1, 0), tslot;
    for (uint32_t l = 0; l < nterm; l++) {
        tslot.insert(tslot.end(), g.term_nts[l].begin(), g.term_nts[l].end());
        toff.push_back((uint32_t)tslot.size());
    }
    c->t_off_n = toff.size();
    c->t_slot_n = std::max<size_t>(tslot.size(), 1);
    c->t_off = (uint32_t *)c->dalloc(c->t_off_n * 4);
    c->t_slot = (uint32_t *)c->dalloc(c->t_slot_n * 4);
    ck(cudaMemcpyAsync(c->t_off, toff.data(), toff.size() * 4, cudaMemcpyHostToDevice, st), "H2D");
    if (!tslot.empty())
        ck(cudaMemcpyAsync(c->t_slot, tslot.data(), tslot.size() * 4, cudaMemcpyHostToDevice, st),
           "H2D");
    c->desc = (uint4 *)c->dalloc((size_t)nt * 2 * n * sizeof(uint4));
    c->dn = (uint2 *)c->dalloc((size_t)nt * 2 * n * sizeof(uint2));
    c->occ_w = (nt + 31) / 32;
    c->occ = (uint32_t *)c->dalloc((size_t)2 * n * c->occ_w * 4);
    c->pool_cap = std::min<uint64_t>(std::max<uint64_t>(16 * c->n_init, 1 << 16), 0xFFFFFFF0ull);
    if (c->cfg.initial_capacity)   // small first pool: the growth path runs early
        c->pool_cap = std::max<uint64_t>(8 * c->n_init / 5 + 4 * 2 * (uint64_t)nt, 64);
    // with a size hint, named non-terminals start with an even share of the
    // expected closure (terminal wrappers only ever hold their edges), with
    // room for the candidates a pair set must also hold before they are
    // deduplicated; the pool gets six words per expected pair (both forms'
    // tiles and entries, and the segments rows leave behind when they move)
    const uint64_t expect = (uint64_t)c->cfg.size_hint * m;
    const uint64_t share = g.n_named ? expect / g.n_named : 0;
    if (expect && !c->cfg.initial_capacity)
        c->pool_cap = std::min<uint64_t>(std::max<uint64_t>(c->pool_cap, 6 * expect),
                                         0xFFFFFFF0ull);
    c->pool = (uint32_t *)c->dalloc(c->pool_cap * 4);
    if (c->cfg.witness && nt > 32768)
        throw Status{CFLR_EINVAL, "witnesses need at most 32768 non-terminals"};
    c->htab.assign(nt, nullptr);
    c->hval.assign(nt, nullptr);
    c->hcap.assign(nt, 0);
    c->nnz.assign(nt, 0);
    for (uint32_t A = 0; A < nt; A++) {
        uint64_t want = std::max<uint64_t>(4 * c->init_cnt[A], 1024);
        if (A < g.n_named) want = std::max<uint64_t>(want, 3 * share);
        c->hcap[A] = next_pow2(want);
        c->htab[A] = (unsigned long long *)c->dalloc(c->hcap[A] * 8);
        if (c->cfg.witness) c->hval[A] = (uint2 *)c->dalloc(c->hcap[A] * 8);
    }
}

// Algorithm 1, terminal initialisation: M_A(i, j) = 1 for every edge
// (i, x, j) and production A -> x, and the identity for every A -> eps.  The
// initial pairs go through the same commit and merge as the closure loop, so
// afterwards every row's entries are its delta (M_old is empty).
void reset_matrices(cflr_ctx *c) {
    Range range("cflr: terminal initialisation");
    const Grammar &g = c->g;
    const uint32_t nt = (uint32_t)g.nts.size(), nterm = (uint32_t)g.terms.size();
    const uint32_t n = c->n;
    cudaStream_t st = c->stream;
    ck(cudaMemsetAsync(c->desc, 0, (size_t)nt * 2 * n * sizeof(uint4), st), "memset");
    ck(cudaMemsetAsync(c->dn, 0, (size_t)nt * 2 * n * sizeof(uint2), st), "memset");
    ck(cudaMemsetAsync(c->occ, 0, (size_t)2 * n * c->occ_w * 4, st), "memset");
    for (uint32_t A = 0; A < nt; A++)
        ck(cudaMemsetAsync(c->htab[A], 0xFF, c->hcap[A] * 8, st), "memset");
    c->pool_top = 0;
    std::fill(c->nnz.begin(), c->nnz.end(), 0);
    c->iterations = 0;
    c->touched_n = 0;
    Runner &r = runner_of(c);
    r.bind({c});
    r.init_buffers(std::max<uint64_t>(c->n_init, 1), 0);
    if (r.cand_cap < c->n_init) {      // the initial pairs are counted exactly
        r.size_cand(c->n_init);
        r.size_touched(2 * r.cand_cap, -1);
    }
    const SlotTab S = r.slots();
    const InstTab I = r.insttab();
    const WorkBufs W = r.work();
    launch_iter_begin(S, I, W, r.n_slots, 1, st);
    r.prof.run(KID_INIT, [&] {
        launch_init_edges(c->e_src, c->e_lab, c->e_dst, c->m_edges, c->t_off, c->t_slot, nterm, W,
                          c->sms, st);
        for (uint32_t A : g.eps) launch_init_eps(A, n, W, c->sms, st);
    });
    c->k_bytes[KID_INIT] += 12 * c->m_edges + 12 * c->n_init;
    // the pair sets were sized from the exact initial counts, so the commit
    // needs no capacity check; the pool may still grow
    r.launch_merge(S, I, W, 0, false, false, true);
    r.read_status();
    if (r.h_cnt->overflow & OVF_CAND) throw Status{CFLR_ECUDA, "internal: init overflow"};
    if (r.h_ctl->status) r.recover();
    r.download_state(false);
    r.export_touched();
    r.prof.collect();
}

int finish_status(cflr_ctx *c, const Status &s) { return c->fail(s.code, s.msg); }

int cuda_status(cflr_ctx *c, const CudaError &e) {
    c->err = std::string(e.what) + ": " + cudaGetErrorString(e.e);
    return CFLR_ECUDA;
}

int solve_many(std::vector<cflr_ctx *> cx, cflr_stats *stats) {
    Range range("cflr_solve");
    cflr_ctx *own = cx[0];
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    ck(cudaSetDevice(own->device), "cudaSetDevice");
    std::vector<cflr_ctx *> active;
    for (auto *c : cx)
        if (c->touched_n) active.push_back(c);
    ck(cudaEventCreate(&ev0), "event");
    ck(cudaEventCreate(&ev1), "event");
    ck(cudaEventRecord(ev0, own->stream), "event");
    int rc = CFLR_OK;
    uint64_t flops = 0, cand = 0, regrows = 0, groups[4] = {0, 0, 0, 0}, kinds[3] = {0, 0, 0};
    uint64_t tiles3[2] = {0, 0};
    if (!active.empty()) {
        Runner &r = runner_of(own);
        r.bind(active);
        uint64_t hint = 0;
        for (auto *c : active) hint += c->touched_n;
        // candidates: the peak of a fresh alias solve is about 24 per touched
        // row of the first iteration; room for 32 (at most 2^26 entries)
        // spares the reruns of the iterations that overflow (first solve of
        // the 200k alias graph 51.4 -> 45.7 ms)
        r.init_buffers(std::min<uint64_t>(std::max<uint64_t>(hint * 32, 1 << 16), 1ull << 26),
                       hint);
        r.import_touched();
        if (!r.run_loop()) rc = CFLR_ELIMIT;
        r.account();
        r.download_state(true);
        r.export_touched();
        flops = r.h_ctl->total_flops;
        tiles3[0] = r.h_ctl->tiles_bin3[0];
        tiles3[1] = r.h_ctl->tiles_bin3[1];
        cand = r.h_ctl->total_cand;
        for (int b = 0; b < 4; b++) groups[b] = r.h_ctl->total_groups[b];
        regrows = r.regrows;
        for (int q = 0; q < 3; q++) kinds[q] = r.regrow_kind[q];
    }
    ck(cudaEventRecord(ev1, own->stream), "event");
    ck(cudaEventSynchronize(ev1), "event");
    float ms = 0;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    for (size_t k = 0; k < cx.size(); k++) {
        cflr_ctx *c = cx[k];
        cflr_stats s{};
        s.iterations = c->iterations;
        for (uint32_t x = 0; x < c->g.n_named; x++) s.total_pairs += c->nnz[x];
        s.solve_ms = ms;
        s.peak_device_bytes = c->bytes_peak;
        s.ignored_edges = c->ignored;
        s.flops = flops;
        s.candidates = cand;
        s.regrows = regrows;
        s.regrow_buffers = kinds[0];
        s.regrow_sets = kinds[1];
        s.regrow_pools = kinds[2];
        s.flops_bin3 = tiles3[0];
        s.mask_tiles_bin3 = tiles3[1];
        s.converged = c->touched_n == 0 ? 1u : 0u;
        for (int b = 0; b < 4; b++) s.groups[b] = groups[b];
        c->last = s;
        if (stats) stats[k] = s;
        if (s.converged) c->state = ST_SOLVED;
    }
    if (rc == CFLR_ELIMIT)
        own->err = "max_iterations reached before the fixpoint";
    return rc;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

void cflr_default_config(cflr_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->form = CFLR_FORM_BATCHED;
}

int cflr_create(cflr_ctx **out, const cflr_config *cfg) {
    if (!out) return CFLR_EINVAL;
    *out = nullptr;
    cflr_config c;
    if (cfg) c = *cfg;
    else cflr_default_config(&c);
    if (c.form < CFLR_FORM_PLAIN || c.form > CFLR_FORM_GRAPH) return CFLR_EINVAL;
    std::unique_ptr<cflr_ctx> x(new cflr_ctx());
    x->cfg = c;
    // the caller's string need not outlive this call
    if (c.autotune_cache) {
        x->cache_path = c.autotune_cache;
        x->cfg.autotune_cache = x->cache_path.c_str();
    }
    x->device = c.device;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev) {
        cudaGetLastError();
        return CFLR_ECUDA;
    }
    if (cudaSetDevice(c.device) != cudaSuccess) return CFLR_ECUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, c.device) != cudaSuccess) return CFLR_ECUDA;
    x->sms = prop.multiProcessorCount;
    x->smem_optin = prop.sharedMemPerBlockOptin;
    if (library_pool(c.device, &x->mpool) != cudaSuccess) {
        cudaGetLastError();
        return CFLR_ECUDA;
    }
    if (c.stream) {
        x->stream = (cudaStream_t)c.stream;
    } else {
        if (cudaStreamCreateWithFlags(&x->stream, cudaStreamNonBlocking) != cudaSuccess)
            return CFLR_ECUDA;
        x->own_stream = true;
    }
    *out = x.release();
    return CFLR_OK;
}

int cflr_load_grammar(cflr_ctx *c, const char *text, size_t len) {
    if (!c) return CFLR_EINVAL;
    if (!text) return c->fail(CFLR_EINVAL, "grammar text is NULL");
    try {
        cudaSetDevice(c->device);
        Grammar g;
        std::string err;
        if (parse_grammar(text, len, g, err)) return c->fail(CFLR_EGRAMMAR, err);
        if (g.nts.size() >= (1u << 20)) return c->fail(CFLR_EGRAMMAR, "too many non-terminals");
        c->free_graph();
        c->g = std::move(g);
        c->grammar_text.assign(text, len);
        c->state = ST_GRAMMAR;
        c->err.clear();
        return CFLR_OK;
    } catch (const CudaError &e) {
        return cuda_status(c, e);
    }
}

int cflr_symbol_id(const cflr_ctx *c, const char *name, uint32_t *id, int *is_terminal) {
    if (!c || !name || !id) return CFLR_EINVAL;
    if (c->state < ST_GRAMMAR) return CFLR_ESTATE;
    int k = c->g.find_nt(name);
    if (k >= 0) {
        *id = (uint32_t)k;
        if (is_terminal) *is_terminal = 0;
        return CFLR_OK;
    }
    k = c->g.find_term(name);
    if (k >= 0) {
        *id = (uint32_t)k;
        if (is_terminal) *is_terminal = 1;
        return CFLR_OK;
    }
    return CFLR_EINVAL;
}

int cflr_grammar_sizes(const cflr_ctx *c, uint32_t *n_nonterminals, uint32_t *n_named,
                       uint32_t *n_terminals) {
    if (!c) return CFLR_EINVAL;
    if (c->state < ST_GRAMMAR) return CFLR_ESTATE;
    if (n_nonterminals) *n_nonterminals = (uint32_t)c->g.nts.size();
    if (n_named) *n_named = c->g.n_named;
    if (n_terminals) *n_terminals = (uint32_t)c->g.terms.size();
    return CFLR_OK;
}

int cflr_load_graph(cflr_ctx *c, uint32_t n_vertices, uint64_t n_edges, const uint32_t *src,
                    const uint32_t *label, const uint32_t *dst) {
    if (!c) return CFLR_EINVAL;
    if (c->state < ST_GRAMMAR) return c->fail(CFLR_ESTATE, "load a grammar first");
    if (n_edges && (!src || !label || !dst)) return c->fail(CFLR_EINVAL, "NULL edge array");
    const uint64_t nt = c->g.nts.size();
    const long double bound = (long double)nt * n_vertices * (long double)n_vertices;
    if (bound >= 4.6e18L || n_vertices >= 0xFFFFFFF0u)
        return c->fail(CFLR_EGRAPH, "too many vertices for 64-bit pair keys");
    const EdgeScan scan = scan_edges(c->g, n_vertices, n_edges, src, label, dst);
    if (scan.bad < n_edges)
        return c->fail(CFLR_EGRAPH, "edge " + std::to_string(scan.bad) + " has a vertex id >= " +
                                        std::to_string(n_vertices));
    try {
        Range range("cflr_load_graph");
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        c->free_graph();
        c->state = ST_GRAMMAR;
        upload_graph(c, n_vertices, n_edges, src, label, dst, scan);
        reset_matrices(c);
        c->state = ST_GRAPH;
        c->err.clear();
        return CFLR_OK;
    } catch (const Status &s) {
        c->free_graph();
        return finish_status(c, s);
    } catch (const CudaError &e) {
        return cuda_status(c, e);
    }
}

int cflr_solve(cflr_ctx *c, cflr_stats *stats) {
    if (!c) return CFLR_EINVAL;
    cflr_ctx *arr[1] = {c};
    return cflr_solve_batch(arr, 1, stats);
}

int cflr_solve_batch(cflr_ctx *const *ctxs, int n, cflr_stats *stats) {
    if (!ctxs || n <= 0) return CFLR_EINVAL;
    std::vector<cflr_ctx *> cx;
    for (int k = 0; k < n; k++) {
        if (!ctxs[k]) return CFLR_EINVAL;
        if (ctxs[k]->state < ST_GRAPH) return ctxs[k]->fail(CFLR_ESTATE, "load a graph first");
        if (ctxs[k]->device != ctxs[0]->device)
            return ctxs[0]->fail(CFLR_EINVAL, "contexts of one batch must share a device");
        cx.push_back(ctxs[k]);
    }
    try {
        return solve_many(cx, stats);
    } catch (const Status &s) {
        // A failed growth may strike between the commit and the merge of an
        // iteration: the matrices are then incomplete, so they are dropped
        // and the contexts need a new graph.
        for (auto *c : cx) {
            c->free_graph();
            c->state = ST_GRAMMAR;
        }
        return finish_status(cx[0], s);
    } catch (const CudaError &e) {
        return cuda_status(cx[0], e);
    }
}

int cflr_get_vertex_order(const cflr_ctx *cc, uint32_t *order, uint64_t capacity) {
    cflr_ctx *c = const_cast<cflr_ctx *>(cc);
    if (!c) return CFLR_EINVAL;
    if (c->state < ST_GRAPH) return c->fail(CFLR_ESTATE, "no graph loaded");
    if (!order) return c->fail(CFLR_EINVAL, "order is NULL");
    if (capacity < c->n) return c->fail(CFLR_EINVAL, "capacity smaller than the vertex count");
    if (!c->iperm) {
        for (uint32_t k = 0; k < c->n; k++) order[k] = k;
        return CFLR_OK;
    }
    try {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        ck(cudaMemcpyAsync(order, c->iperm, (size_t)c->n * 4, cudaMemcpyDeviceToHost, c->stream),
           "D2H order");
        ck(cudaStreamSynchronize(c->stream), "sync order");
        return CFLR_OK;
    } catch (const CudaError &e) {
        return cuda_status(c, e);
    }
}

int cflr_reset(cflr_ctx *c) {
    if (!c) return CFLR_EINVAL;
    if (c->state < ST_GRAPH) return c->fail(CFLR_ESTATE, "no graph loaded");
    try {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        reset_matrices(c);
        c->state = ST_GRAPH;
        return CFLR_OK;
    } catch (const Status &s) {
        c->free_graph();
        c->state = ST_GRAMMAR;
        return finish_status(c, s);
    } catch (const CudaError &e) {
        return cuda_status(c, e);
    }
}

}  // extern "C"

namespace {

// A stream and events that are destroyed on every way out of a call.
struct CopyLane {
    cudaStream_t s = nullptr;
    std::vector<cudaEvent_t> ev;
    ~CopyLane() {
        if (s) cudaStreamSynchronize(s);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        if (s) cudaStreamDestroy(s);
    }
    cudaEvent_t record(cudaStream_t on) {
        cudaEvent_t e;
        ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
        ev.push_back(e);
        ck(cudaEventRecord(e, on), "cudaEventRecord");
        return e;
    }
};

// Write the pairs of the listed non-terminals (nts[0..count), output
// positions offsets[0..count]) one after another, each non-terminal's
// sorted by (src, dst): into the device arrays ws/wd, or into the host
// arrays hs/hd through two device staging buffers of at most STAGE pairs.
// For the host, the units' first positions are read back after the count,
// the units are cut into ranges that fit a buffer, and each range is written
// into one buffer while the other is copied out on a second stream.
// Checks the extracted count against the pair sets' counts.
void extract_many(cflr_ctx *c, uint32_t count, const uint32_t *nts, const uint64_t *offsets,
                  uint32_t *ws, uint32_t *wd, uint32_t *hs, uint32_t *hd) {
    Range range("cflr: extraction");
    constexpr uint64_t STAGE = 1ull << 24;
    cudaStream_t st = c->stream;
    const uint32_t n = c->n;
    std::vector<uint32_t> tab;            // the non-empty entries, then their rows per unit
    std::vector<uint64_t> pairs;
    for (uint32_t i = 0; i < count; i++) {
        const uint64_t cnt = offsets[i + 1] - offsets[i];
        if (!cnt) continue;
        tab.push_back(nts[i]);
        pairs.push_back(cnt);
    }
    if (tab.empty()) return;
    const uint32_t E = (uint32_t)tab.size();
    uint64_t total = 0;
    for (uint64_t p : pairs) total += p;
    tab.resize(2 * (size_t)E);
    std::vector<unsigned long long> first(E + 1);
    extract_plan(E, n, pairs.data(), c->sms, tab.data() + E, first.data());
    const uint64_t U = first[E];
    c->scratch(c->x_nts, c->x_nts_n, 2 * (size_t)E);
    c->scratch(c->x_first, c->x_first_n, (size_t)E + 1);
    c->scratch(c->x_unit, c->x_unit_n, U + 1);
    c->scratch(c->x_bsum, c->x_bsum_n, U / 1024 + 2);
    c->scratch(c->x_misc, c->x_misc_n, 4);       // cursors, error flag, total
    const size_t words = ((size_t)n + 31) / 32;
    if (words * 4 > 200 * 1024) c->scratch(c->x_bm, c->x_bm_n, words * (size_t)c->sms * 4);
    ck(cudaMemcpyAsync(c->x_nts, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, st), "H2D");
    ck(cudaMemcpyAsync(c->x_first, first.data(), first.size() * 8, cudaMemcpyHostToDevice, st),
       "H2D");
    ck(cudaMemsetAsync(c->x_misc + 2, 0, 8, st), "memset");
    unsigned *err = (unsigned *)(c->x_misc + 2);
    ExtractList L{};
    L.desc = c->desc;
    L.pool = c->pool;
    L.perm = c->perm;
    L.iperm = c->iperm;
    L.nts = c->x_nts;
    L.rows_per = c->x_nts + E;
    L.unit_first = c->x_first;
    L.n = n;
    L.count = E;
    L.units = U;
    launch_extract_count(L, c->x_unit, c->x_bsum, c->x_misc + 3, c->sms, st);
    ck(cudaGetLastError(), "extract count");
    unsigned long long misc[4] = {0, 0, 0, 0};
    auto check = [&]() {
        ck(cudaMemcpyAsync(misc, c->x_misc, sizeof(misc), cudaMemcpyDeviceToHost, st), "D2H");
        ck(cudaStreamSynchronize(st), "sync extract");
        if (misc[2] & 1)
            throw Status{CFLR_ECUDA, "internal: the long-row list of the extraction overflowed"};
        if (misc[2] & 2)
            throw Status{CFLR_ECUDA, "internal: a row held more pairs than the pair sets count"};
        if (misc[3] != total)
            throw Status{CFLR_ECUDA, "internal: extracted " + std::to_string(misc[3]) +
                                         " pairs where the pair sets hold " +
                                         std::to_string(total)};
    };
    if (!hs) {
        c->scratch(c->x_bigl, c->x_bigl_n, total / 1024 + 1);
        L.u_begin = 0;
        L.u_end = U;
        L.base = 0;
        L.limit = total;
        launch_extract_write(L, ws, wd, c->x_unit, c->x_bigl, c->x_bigl_n, c->x_misc, c->x_bm,
                             err, c->sms, st);
        ck(cudaGetLastError(), "extract");
        check();
        return;
    }
    // ranges of units that fit a staging buffer (a unit larger than that
    // makes a range of its own and sizes the buffers)
    std::vector<unsigned long long> uoff(U + 1);
    ck(cudaMemcpyAsync(uoff.data(), c->x_unit, U * 8, cudaMemcpyDeviceToHost, st), "D2H");
    ck(cudaStreamSynchronize(st), "sync extract count");
    uoff[U] = total;
    std::vector<uint64_t> cut(1, 0);
    uint64_t cap = 0;
    for (uint64_t u = 1; u <= U; u++) {
        if (uoff[u] - uoff[cut.back()] > STAGE && u - 1 > cut.back()) cut.push_back(u - 1);
        if (u == U) cut.push_back(U);
    }
    for (size_t r = 0; r + 1 < cut.size(); r++)
        cap = std::max<uint64_t>(cap, uoff[cut[r + 1]] - uoff[cut[r]]);
    cap = std::max<uint64_t>(cap, 1);
    if (c->x_out_cap < 2 * cap) {
        c->free_extract_out();
        c->x_src = (uint32_t *)c->dalloc(2 * cap * 4);
        c->x_dst = (uint32_t *)c->dalloc(2 * cap * 4);
        c->x_out_cap = 2 * cap;
    }
    c->scratch(c->x_bigl, c->x_bigl_n, cap / 1024 + 1);
    CopyLane lane;
    ck(cudaStreamCreateWithFlags(&lane.s, cudaStreamNonBlocking), "cudaStreamCreate");
    cudaEvent_t copied[2] = {nullptr, nullptr};   // the last copy out of each buffer
    for (size_t r = 0; r + 1 < cut.size(); r++) {
        const int b = (int)(r & 1);
        if (copied[b]) ck(cudaStreamWaitEvent(st, copied[b], 0), "cudaStreamWaitEvent");
        L.u_begin = cut[r];
        L.u_end = cut[r + 1];
        L.base = uoff[cut[r]];
        L.limit = uoff[cut[r + 1]];
        uint32_t *bs = c->x_src + b * cap, *bd = c->x_dst + b * cap;
        launch_extract_write(L, bs, bd, c->x_unit, c->x_bigl, c->x_bigl_n, c->x_misc, c->x_bm,
                             err, c->sms, st);
        ck(cudaGetLastError(), "extract");
        ck(cudaStreamWaitEvent(lane.s, lane.record(st), 0), "cudaStreamWaitEvent");
        const uint64_t k = L.limit - L.base;
        ck(cudaMemcpyAsync(hs + L.base, bs, k * 4, cudaMemcpyDeviceToHost, lane.s), "D2H pairs");
        ck(cudaMemcpyAsync(hd + L.base, bd, k * 4, cudaMemcpyDeviceToHost, lane.s), "D2H pairs");
        copied[b] = lane.record(lane.s);
    }
    ck(cudaStreamSynchronize(lane.s), "sync copy");
    check();
}

int get_pairs_common(cflr_ctx *c, uint32_t nonterminal, uint32_t *src, uint32_t *dst,
                     uint64_t capacity, uint64_t *n_pairs, bool on_device) {
    if (!c || !n_pairs) return CFLR_EINVAL;
    if (c->state < ST_GRAPH) return c->fail(CFLR_ESTATE, "no graph loaded");
    if (nonterminal >= c->g.nts.size()) return c->fail(CFLR_EINVAL, "bad non-terminal id");
    const uint64_t cnt = c->nnz[nonterminal];
    *n_pairs = cnt;
    if (!src && !dst) return CFLR_OK;
    if (!src || !dst) return c->fail(CFLR_EINVAL, "src and dst must both be given");
    if (capacity < cnt) return c->fail(CFLR_EINVAL, "capacity smaller than the pair count");
    if (cnt == 0) return CFLR_OK;
    try {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        const uint64_t off[2] = {0, cnt};
        if (on_device) {
            extract_many(c, 1, &nonterminal, off, src, dst, nullptr, nullptr);
            return CFLR_OK;
        }
        extract_many(c, 1, &nonterminal, off, nullptr, nullptr, src, dst);
        return CFLR_OK;
    } catch (const Status &s) {
        return finish_status(c, s);
    } catch (const CudaError &e) {
        return cuda_status(c, e);
    }
}

// The pairs of several non-terminals, one after another (cflr_get_pairs_many
// and cflr_get_pairs_device_many), with one synchronisation for the call.
int get_pairs_many_common(cflr_ctx *c, uint32_t count, const uint32_t *nts, uint32_t *src,
                          uint32_t *dst, uint64_t capacity, uint64_t *offsets, bool on_device) {
    if (!c || !offsets || (count && !nts)) return CFLR_EINVAL;
    if (c->state < ST_GRAPH) return c->fail(CFLR_ESTATE, "no graph loaded");
    uint64_t total = 0;
    for (uint32_t i = 0; i < count; i++) {
        if (nts[i] >= c->g.nts.size()) return c->fail(CFLR_EINVAL, "bad non-terminal id");
        offsets[i] = total;
        total += c->nnz[nts[i]];
    }
    offsets[count] = total;
    if (!src && !dst) return CFLR_OK;
    if (!src || !dst) return c->fail(CFLR_EINVAL, "src and dst must both be given");
    if (capacity < total) return c->fail(CFLR_EINVAL, "capacity smaller than the pair count");
    if (total == 0) return CFLR_OK;
    try {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        if (on_device) {
            extract_many(c, count, nts, offsets, src, dst, nullptr, nullptr);
            return CFLR_OK;
        }
        extract_many(c, count, nts, offsets, nullptr, nullptr, src, dst);
        return CFLR_OK;
    } catch (const Status &s) {
        return finish_status(c, s);
    } catch (const CudaError &e) {
        return cuda_status(c, e);
    }
}

}  // namespace

extern "C" {

int cflr_get_pairs_many(const cflr_ctx *cc, uint32_t count, const uint32_t *nonterminals,
                        uint32_t *src, uint32_t *dst, uint64_t capacity, uint64_t *offsets) {
    return get_pairs_many_common(const_cast<cflr_ctx *>(cc), count, nonterminals, src, dst,
                                 capacity, offsets, false);
}

int cflr_get_pairs_device_many(const cflr_ctx *cc, uint32_t count, const uint32_t *nonterminals,
                               uint32_t *d_src, uint32_t *d_dst, uint64_t capacity,
                               uint64_t *offsets) {
    return get_pairs_many_common(const_cast<cflr_ctx *>(cc), count, nonterminals, d_src, d_dst,
                                 capacity, offsets, true);
}

int cflr_get_pairs(const cflr_ctx *cc, uint32_t nonterminal, uint32_t *src, uint32_t *dst,
                   uint64_t capacity, uint64_t *n_pairs) {
    return get_pairs_common(const_cast<cflr_ctx *>(cc), nonterminal, src, dst, capacity, n_pairs,
                            false);
}

int cflr_get_pairs_device(const cflr_ctx *cc, uint32_t nonterminal, uint32_t *d_src,
                          uint32_t *d_dst, uint64_t capacity, uint64_t *n_pairs) {
    return get_pairs_common(const_cast<cflr_ctx *>(cc), nonterminal, d_src, d_dst, capacity,
                            n_pairs, true);
}

int cflr_get_witness(const cflr_ctx *cc, uint32_t nonterminal, uint32_t src, uint32_t dst,
                     int *kind, uint32_t *id, uint32_t *id2, uint32_t *mid) {
    cflr_ctx *c = const_cast<cflr_ctx *>(cc);
    if (!c || !kind) return CFLR_EINVAL;
    if (c->state < ST_GRAPH) return c->fail(CFLR_ESTATE, "no graph loaded");
    if (!c->cfg.witness) return c->fail(CFLR_ESTATE, "the context records no witnesses");
    if (nonterminal >= c->g.nts.size()) return c->fail(CFLR_EINVAL, "bad non-terminal id");
    if (src >= c->n || dst >= c->n) return c->fail(CFLR_EINVAL, "vertex id out of range");
    try {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        cudaStream_t st = c->stream;
        uint32_t s = src, d = dst;
        if (c->perm) {      // stored ids
            ck(cudaMemcpyAsync(&s, c->perm + src, 4, cudaMemcpyDeviceToHost, st), "D2H");
            ck(cudaMemcpyAsync(&d, c->perm + dst, 4, cudaMemcpyDeviceToHost, st), "D2H");
            ck(cudaStreamSynchronize(st), "sync");
        }
        uint2 *out = (uint2 *)c->dalloc(sizeof(uint2));
        launch_witness_lookup(c->htab[nonterminal], c->hval[nonterminal],
                              c->hcap[nonterminal] - 1, ((unsigned long long)s << 32) | d, out,
                              st);
        uint2 w;
        ck(cudaMemcpyAsync(&w, out, sizeof(uint2), cudaMemcpyDeviceToHost, st), "D2H");
        ck(cudaStreamSynchronize(st), "sync witness");
        c->dfree(out, sizeof(uint2));
        if (w.x == EMPTY32 && w.y == EMPTY32)
            return c->fail(CFLR_EINVAL, "the pair is not in the relation");
        const uint32_t k = w.x >> 30, pay = w.x & WIT_PAYLOAD;
        *kind = (int)k;
        uint32_t a = 0, b = 0, m = 0;
        if (w.x >= WIT_EPS) {
            *kind = CFLR_WIT_EPS;
        } else if (k == 0) {
            *kind = CFLR_WIT_BINARY;
            a = pay >> 15;
            b = pay & 0x7FFF;
            m = w.y;
            if (c->iperm) {
                ck(cudaMemcpyAsync(&m, c->iperm + w.y, 4, cudaMemcpyDeviceToHost, st), "D2H");
                ck(cudaStreamSynchronize(st), "sync");
            }
        } else if (k == 1) {
            *kind = CFLR_WIT_EDGE;
            a = pay;
        } else {
            *kind = CFLR_WIT_UNIT;
            a = pay;
        }
        if (id) *id = a;
        if (id2) *id2 = b;
        if (mid) *mid = m;
        return CFLR_OK;
    } catch (const Status &e) {
        return finish_status(c, e);
    } catch (const CudaError &e) {
        return cuda_status(c, e);
    }
}

int cflr_get_tuning(const cflr_ctx *c, cflr_tuning *t) {
    if (!c || !t) return CFLR_EINVAL;
    t->probe_ratio = c->tuning.probe_ratio;
    for (int b = 0; b < 3; b++) t->bin_limit[b] = c->tuning.limit[b];
    for (int b = 0; b < 4; b++) t->ctas_per_sm[b] = c->tuning.ctas_per_sm[b];
    return CFLR_OK;
}

int cflr_set_tuning(cflr_ctx *c, const cflr_tuning *t) {
    if (!c || !t) return CFLR_EINVAL;
    const uint32_t cap[3] = {BIN0_LIMIT, BIN1_LIMIT, BIN2_LIMIT};
    if (t->probe_ratio < 1) return c->fail(CFLR_EINVAL, "probe_ratio must be >= 1");
    for (int b = 0; b < 3; b++) {
        if (t->bin_limit[b] < 1 || t->bin_limit[b] > cap[b] ||
            (b && t->bin_limit[b] <= t->bin_limit[b - 1]))
            return c->fail(CFLR_EINVAL, "bin limits must increase within 128, 1024, 4096");
    }
    for (int b = 0; b < 4; b++)
        if (t->ctas_per_sm[b] < 1 || t->ctas_per_sm[b] > 32)
            return c->fail(CFLR_EINVAL, "ctas_per_sm must be in 1..32");
    Tuning n;
    n.probe_ratio = t->probe_ratio;
    for (int b = 0; b < 3; b++) n.limit[b] = t->bin_limit[b];
    for (int b = 0; b < 4; b++) n.ctas_per_sm[b] = t->ctas_per_sm[b];
    c->tuning = n;
    if (c->runner) c->runner->drop_graph();   // the graph holds the old grids
    return CFLR_OK;
}

}  // extern "C"

namespace {

std::string autotune_key(const cflr_ctx *c) {
    uint64_t h = 1469598103934665603ull;                     // FNV-1a of the grammar text
    for (unsigned char ch : c->grammar_text) h = (h ^ ch) * 1099511628211ull;
    char buf[96];
    snprintf(buf, sizeof buf, "%016llx_%u_%llu", (unsigned long long)h, c->n,
             (unsigned long long)c->m_edges);
    return buf;
}

bool cache_lookup(const char *path, const std::string &key, Tuning &t) {
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char k[128];
    Tuning r;
    bool found = false;
    while (fscanf(f, "%127s %u %u %u %u %u %u %u %u", k, &r.probe_ratio, &r.limit[0],
                  &r.limit[1], &r.limit[2], &r.ctas_per_sm[0], &r.ctas_per_sm[1],
                  &r.ctas_per_sm[2], &r.ctas_per_sm[3]) == 9) {
        if (key == k) {
            t = r;
            found = true;
        }
    }
    fclose(f);
    return found;
}

void cache_store(const char *path, const std::string &key, const Tuning &t) {
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %u %u %u %u %u %u %u %u\n", key.c_str(), t.probe_ratio, t.limit[0], t.limit[1],
            t.limit[2], t.ctas_per_sm[0], t.ctas_per_sm[1], t.ctas_per_sm[2], t.ctas_per_sm[3]);
    fclose(f);
}

}  // namespace

extern "C" {

int cflr_autotune(cflr_ctx *c, uint32_t max_trials, cflr_tuning *best) {
    if (!c) return CFLR_EINVAL;
    if (c->state < ST_GRAPH) return c->fail(CFLR_ESTATE, "load a graph first");
    const std::string key = autotune_key(c);
    const char *cache = c->cfg.autotune_cache;
    Tuning found;
    if (cache && cache_lookup(cache, key, found)) {
        c->tuning = found;
        if (c->runner) c->runner->drop_graph();
        // the schedule does not change the initial matrices: a context that
        // has not run an iteration since its graph was loaded stays as it is
        int rc = c->iterations == 0 ? CFLR_OK : cflr_reset(c);
        if (rc == CFLR_OK && best) cflr_get_tuning(c, best);
        return rc;
    }
    if (!max_trials) max_trials = 24;
    auto trial = [&](const Tuning &t, double &ms) -> int {
        c->tuning = t;
        if (c->runner) c->runner->drop_graph();
        int rc = cflr_reset(c);
        if (rc != CFLR_OK) return rc;
        cflr_stats st;
        rc = cflr_solve(c, &st);
        if (rc != CFLR_OK && rc != CFLR_ELIMIT) return rc;
        ms = st.solve_ms;
        return CFLR_OK;
    };
    Tuning cur = c->tuning;
    double cur_ms = 0;
    int rc = trial(cur, cur_ms);            // warms the buffers too
    if (rc != CFLR_OK) return rc;
    rc = trial(cur, cur_ms);
    if (rc != CFLR_OK) return rc;
    uint32_t used = 2;
    // candidate values per field, tried in this order
    const std::vector<std::pair<int, std::vector<uint32_t>>> fields = {
        {0, {1, 2, 8, 16, 64}},             // probe_ratio
        {5, {4, 6, 8}},                     // ctas_per_sm[3] (bitmap bin)
        {3, {0, 1024, 2048, 3072}},         // limit[2]; 0: limit[1] + 1, bin 2 off
                                            // (the bitmap bin takes those groups)
        {2, {256, 512}},                    // limit[1]
        {4, {2, 4}},                        // ctas_per_sm[2]
        {6, {2, 4, 6}},                     // ctas_per_sm[1]
    };
    auto with = [](Tuning t, int field, uint32_t v) {
        switch (field) {
        case 0: t.probe_ratio = v; break;
        case 2: t.limit[1] = v; break;
        case 3: t.limit[2] = v ? v : t.limit[1] + 1; break;
        case 4: t.ctas_per_sm[2] = v; break;
        case 5: t.ctas_per_sm[3] = v; break;
        case 6: t.ctas_per_sm[1] = v; break;
        }
        return t;
    };
    for (const auto &fv : fields) {
        for (uint32_t v : fv.second) {
            if (used >= max_trials) break;
            Tuning t = with(cur, fv.first, v);
            if (t.limit[1] >= t.limit[2] || t.limit[0] >= t.limit[1]) continue;
            double ms = 0;
            rc = trial(t, ms);
            used++;
            if (rc != CFLR_OK) return rc;
            if (ms < cur_ms) {
                cur = t;
                cur_ms = ms;
            }
        }
    }
    c->tuning = cur;
    if (c->runner) c->runner->drop_graph();
    rc = cflr_reset(c);
    if (rc != CFLR_OK) return rc;
    if (cache) cache_store(cache, key, cur);
    if (best) cflr_get_tuning(c, best);
    return CFLR_OK;
}

int cflr_kernel_stats(const cflr_ctx *c, int k, const char **name, uint64_t *launches,
                      double *total_ms, uint64_t *alg_bytes) {
    if (!c) return CFLR_EINVAL;
    if (k < 0) {
        if (launches) *launches = N_KID;
        return CFLR_OK;
    }
    if (k >= N_KID) return CFLR_EINVAL;
    if (name) *name = kKernelNames[k];
    if (launches) *launches = c->k_launches[k];
    if (total_ms) *total_ms = c->k_ms[k];
    if (alg_bytes) *alg_bytes = c->k_bytes[k];
    return CFLR_OK;
}

const char *cflr_last_error(const cflr_ctx *c) {
    if (!c) return "NULL context";
    return c->err.c_str();
}

void cflr_destroy(cflr_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    delete c->runner;
    c->runner = nullptr;
    c->free_graph();
    if (c->stream) cudaStreamSynchronize(c->stream);   // the frees above are stream-ordered
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"

// ===========================================================================
// Allocation-free extraction (cflr_get_pairs_device_noalloc)
//
// Some callers may not allocate device memory at the point where they read
// results: code that runs against a fixed device-memory plan made at start-up,
// embedders whose own allocator owns the whole device, or paths that must not
// risk the implicit device synchronisation a cudaMalloc/cudaFree can cause.
// For them this variant of the extraction keeps its scratch (row lengths, row
// offsets, scan block sums and the list of long rows) in one file-scope
// device array instead of context-owned buffers.  The array is sized for
// graphs of up to CFLR_NOALLOC_MAX_VERTICES vertices (about 16 MiB) and, like
// any __device__ variable, is held by every GPU that loads this library until
// the process exits.
// ===========================================================================

#include <mutex>

namespace {

constexpr uint64_t NA_MAX = CFLR_NOALLOC_MAX_VERTICES;
// word layout (8-byte words): offsets | scan block sums | lengths | long rows
constexpr uint64_t NA_OFF_WORDS = NA_MAX;
constexpr uint64_t NA_BSUM_WORDS = NA_MAX / 1024 + 2;
constexpr uint64_t NA_LEN_WORDS = NA_MAX / 2;
constexpr uint64_t NA_BIG_WORDS = (NA_MAX + 2) / 2;
constexpr uint64_t NA_WORDS = NA_OFF_WORDS + NA_BSUM_WORDS + NA_LEN_WORDS + NA_BIG_WORDS;

// In host code this name is only a stand-in for the device variable: its
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[NA_WORDS];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[NA_MAX_DEVICES] = {};

// Device address of the scratch array on `device`, which must be current.
// Looked up once per device, on the first call made for that device.
cudaError_t noalloc_scratch(int device, void **out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (device < 0 || device >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[device] = p;
    }
    *out = g_noalloc_ptr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" int cflr_get_pairs_device_noalloc(const cflr_ctx *cc, uint32_t nonterminal,
                                             uint32_t *d_src, uint32_t *d_dst,
                                             uint64_t capacity, uint64_t *n_pairs) {
    cflr_ctx *c = const_cast<cflr_ctx *>(cc);
    if (!c || !n_pairs) return CFLR_EINVAL;
    if (c->state < ST_GRAPH) return c->fail(CFLR_ESTATE, "no graph loaded");
    if (nonterminal >= c->g.nts.size()) return c->fail(CFLR_EINVAL, "bad non-terminal id");
    const uint64_t cnt = c->nnz[nonterminal];
    *n_pairs = cnt;
    if (!d_src && !d_dst) return CFLR_OK;
    if (!d_src || !d_dst) return c->fail(CFLR_EINVAL, "d_src and d_dst must both be given");
    if (capacity < cnt) return c->fail(CFLR_EINVAL, "capacity smaller than the pair count");
    if (c->n > NA_MAX)
        return c->fail(CFLR_EINVAL, "graph has " + std::to_string(c->n) +
                                        " vertices; the allocation-free extraction supports at "
                                        "most " + std::to_string(NA_MAX));
    if (cnt == 0) return CFLR_OK;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_status(c, CudaError{e, "cudaSetDevice"});
    void *base = nullptr;
    e = noalloc_scratch(c->device, &base);
    if (e != cudaSuccess) return cuda_status(c, CudaError{e, "cudaGetSymbolAddress"});
    unsigned long long *w = (unsigned long long *)base;
    unsigned long long *off = w;
    unsigned long long *bsum = w + NA_OFF_WORDS;
    uint32_t *len = (uint32_t *)(bsum + NA_BSUM_WORDS);
    uint32_t *big = (uint32_t *)(w + NA_OFF_WORDS + NA_BSUM_WORDS + NA_LEN_WORDS);
    const uint32_t n = c->n;
    const uint4 *desc = c->desc + (size_t)nonterminal * 2 * n;
    cudaStream_t st = c->stream;
    // Every scratch word used below is written before it is read (lengths,
    // offsets, block sums) or cleared first (the long-row counter).
    launch_row_lengths(desc, c->pool, n, c->perm, len, st);
    launch_exclusive_scan(len, n, off, bsum, nullptr, st);
    launch_extract(desc, c->pool, n, c->perm, c->iperm, off, d_src, d_dst, big, big + n, nullptr,
                   c->sms, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(c, CudaError{e, "extract (no-alloc)"});
    return CFLR_OK;
}
