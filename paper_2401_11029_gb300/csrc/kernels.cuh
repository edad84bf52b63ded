// Device data layout and kernel entry points of the CFL-r closure loop.
//
// Layout in HBM (one "slot" = one non-terminal of one solved instance):
//   desc[s]     uint4 per row and orientation, 2*n entries per slot:
//                 [0, n)  row form    (row i -> the j with M(i, j))
//                 [n, 2n) column form (column j -> the i with M(i, j))
//               The row is a list of 32-bit tiles (word w, bits b: the
//               columns 32w + i for every set bit i of b) at pool[.x ..],
//               followed by an area of single entries:
//               .x = offset of the row segment in the instance pool
//                    (a multiple of 4 words, so loads of 16 bytes align)
//               .y = tiles in use; they hold every pair of the row, and no
//                    two tiles share a set bit
//               .z = tile capacity; the entry area starts at
//                    .x + tile_words(.z)
//               .w = log2 of the entry capacity << ELOG_SHIFT | the tiles
//                    the last merge appended (they hold the delta; the tiles
//                    before them are M_old)
//   dn[s]       uint2 per row and orientation: .x = pairs the last merge
//               added to the row (its delta for optimisation 1, kept as
//               single entries in the entry area), .y = append cursor
//   pool        uint32 arena of row segments; rows grow by relocation,
//               and a relocation folds the tiles (one tile per word).
//   htab[s]     open-addressing set of 64-bit keys (i << 32 | j): every pair
//               of M_s, used for the complement mask and for deduplication.
// Work items refer to slots, so one launch covers many instances.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cflr {

constexpr uint32_t PART_A = 0;      // dA . B     : row groups of a's delta
constexpr uint32_t PART_B = 1;      // A_old . dB : column groups of b's delta
constexpr uint32_t PART_U = 2;      // c -> a     : row groups of a's delta
constexpr uint32_t PART_F = 3;      // a family of productions on its shared
                                    // operand's delta (optimisation 4)
constexpr uint32_t MODE_PROBE = 4;  // group code bit: mask by probing htab[c]
                                    // group code: prod << 8 | lg << 3 | probe | part
constexpr unsigned long long EMPTY_KEY = ~0ull;
constexpr uint32_t EMPTY32 = 0xFFFFFFFFu;

constexpr int N_BINS = 4;
// Bin limits on a group's smem need (mask entries + products); a bin's table
// holds twice its limit so the load factor stays <= 1/2.
constexpr uint32_t BIN0_LIMIT = 128;    // warp per group, 256-slot table
constexpr uint32_t BIN1_LIMIT = 1024;   // warp per group, 2048-slot table
constexpr uint32_t BIN2_LIMIT = 4096;   // CTA per group, 8192-slot table
                                        // bin 3: CTA per group, n-bit bitmap
constexpr uint32_t PROBE_RATIO = 4;     // probe when mask_len > PROBE_RATIO*flops

// Run-time schedule of the product kernels (picked by cflr_autotune).
struct Tuning {
    uint32_t probe_ratio = PROBE_RATIO;          // see PROBE_RATIO
    uint32_t limit[3] = {BIN0_LIMIT, BIN1_LIMIT, BIN2_LIMIT};   // need bounds of bins 0-2
    uint32_t ctas_per_sm[4] = {8, 3, 3, 8};      // grids (bin 3: upper bound)
};

// desc.w: log2 of the entry capacity << ELOG_SHIFT | the number of tiles the
// last merge appended (DLAST_MASK)
constexpr uint32_t ELOG_SHIFT = 27;
constexpr uint32_t DLAST_MASK = (1u << ELOG_SHIFT) - 1;
__host__ __device__ __forceinline__ uint32_t entry_cap(uint4 desc) {
    return 1u << (desc.w >> ELOG_SHIFT);
}

// pool words of a row's tile section (a multiple of 4, so both the tiles and
// the single entries after them start on 16-byte boundaries)
__host__ __device__ __forceinline__ uint32_t tile_words(uint32_t tiles) {
    return (2 * tiles + 3) & ~3u;
}

// Derivation step of a pair (single-path semantics), kept beside its key in
// the pair set when witnesses are on: .x = kind | payload, .y = the middle
// vertex (stored id) of a binary step.  Payloads: local ids a << 15 | b
// (binary), a (unit), the label (edge).
constexpr uint32_t WIT_BINARY = 0u << 30, WIT_EDGE = 1u << 30, WIT_UNIT = 2u << 30,
                   WIT_EPS = 3u << 30, WIT_PAYLOAD = (1u << 30) - 1;

struct SlotTab {              // per slot (device arrays, length n_slots)
    uint4 **desc;             // row descriptors (2*n per slot)
    uint2 **dn;               // delta counts and append cursors (2*n per slot)
    uint32_t **pool;          // instance pool of the slot
    uint32_t *n;              // vertices of the slot's instance
    uint32_t *inst;           // instance index of the slot
    unsigned long long **htab;
    uint2 **hval;                   // witnesses beside htab's keys (null: off)
    unsigned long long *hmask;      // capacity - 1
    unsigned long long *cand;       // candidates emitted for the slot (iteration)
    unsigned long long *delta;      // new pairs of the slot (iteration)
    unsigned long long *nnz;        // pairs of the slot so far
    // occupancy: occ[s][(o*n + k)*occ_w[s] + local[s]/32] has bit local[s]%32
    // set once row k of orientation o of slot s is non-empty (one bit per
    // non-terminal of the instance, all of a vertex's bits in one line)
    uint32_t **occ;
    uint32_t *occ_w;                // words per vertex and orientation
    uint32_t *local;                // non-terminal id of the slot in its instance
    const unsigned long long *pool_cap;   // pool words of each instance (index: inst)
};

struct InstTab {              // per instance
    unsigned long long *pool_top;   // entries in use (device counters)
    unsigned long long *pool_cap;
    unsigned long long *delta;      // new pairs of the instance (iteration)
    uint32_t *active;               // 1 while the instance still has delta rows
    uint32_t *iters;                // closure iterations the instance has run
};

// Closure-loop control in device memory (one per batch).
struct LoopCtl {
    uint32_t iter;                  // iterations finished since the solve began
    uint32_t limit;                 // stop after this many (0xFFFFFFFF = none)
    uint32_t status;                // overflow bits that stopped the last iteration
    uint32_t stop_on_converge;      // stop once some instance reaches its fixpoint
    unsigned long long last_delta;  // new pairs of the last finished iteration
    // totals over the finished iterations (work and algorithmic bytes)
    unsigned long long total_flops, total_cand, total_delta;
    unsigned long long total_touched_in, total_touched_out;
    unsigned long long bytes_bin[N_BINS];
    unsigned long long bytes_sym;
    unsigned long long total_groups[N_BINS];
    unsigned long long bytes_move[2];
    unsigned long long tiles_bin3[2];
};

struct ProdTab {              // global production table of the batch
    const uint4 *prod;        // {c_slot, a_slot, b_slot, kind(0 binary, 1 unit)}
    const uint32_t *use_off;  // per slot*2+o: offsets into use_code
    const uint32_t *use_code; // prod << 2 | part, or family << 2 | PART_F
    // families run as one block product (optimisation 4):
    // {offset into fam_prod, members F, flags, part of the shared operand
    // (PART_A: a shared, PART_B: b shared)}; member i is production
    // fam_prod[offset + i].  Flags: FAM_CSHARED when every member writes the
    // same c, FAM_CONSEC when the slots of the members' other operand are
    // consecutive (so are their occupancy bits)
    const uint4 *fam;
    const uint32_t *fam_prod;
};
constexpr uint32_t FAM_CSHARED = 1, FAM_CONSEC = 2;

struct Counters {
    unsigned long long groups[N_BINS];
    unsigned long long claim[N_BINS];   // next group of the bin to take (CTA-level bins)
    unsigned long long cand;
    unsigned long long delta;
    unsigned long long flops;
    unsigned long long bytes_bin[N_BINS];
    unsigned long long bytes_sym;
    unsigned long long holes;       // reserved candidate entries left unused
    unsigned long long big_n;       // delta rows listed for the CTA pass of k_symbolic
    unsigned long long bytes_move[2];   // tile bytes read and written by moved rows
                                        // (k_capacity, k_capacity_big)
    unsigned long long tiles_bin3[2];   // product and mask tiles of the bitmap bin
    unsigned int overflow;          // OVF_* bits
    unsigned int pad;
};

constexpr unsigned OVF_GROUPS = 1u;    // work list overflow        (before the commit)
constexpr unsigned OVF_CAND = 2u;      // candidate buffer overflow (before the commit)
constexpr unsigned OVF_POOL = 4u;      // row pool exhausted        (inside the merge)
constexpr unsigned OVF_TOUCHED = 8u;   // touched list overflow (cannot happen: sized 2x)
constexpr unsigned OVF_HASH = 16u;     // a pair set would pass half full (before the commit)
constexpr unsigned OVF_FULL = 32u;     // a probe sequence passed over a whole hash table
                                       // (cannot happen while sets stay half full): fatal
constexpr unsigned OVF_BOUNDS = 64u;   // an index failed its bounds check (checked
                                       // builds only; the access was skipped): fatal
constexpr unsigned OVF_PRE = OVF_GROUPS | OVF_CAND | OVF_HASH;   // iteration not committed
constexpr unsigned OVF_STOP = OVF_PRE | OVF_FULL | OVF_BOUNDS;   // the merge kernels do nothing

// Checked builds (CFLR_CHECKED defined; libcflr_checked.so) test the indices
// that come from data (vertex ids read from rows, tile-list segments against
// the pool, accumulator words against the row width, pair keys) before they
// are used; a failed test sets OVF_BOUNDS in *err and the access is skipped,
// so a layout bug ends the solve with CFLR_ECUDA instead of reading or
// writing out of bounds.  In normal builds the tests compile to nothing.
#if defined(CFLR_CHECKED)
#define CFLR_CHECK(cond, err) ((cond) ? true : (atomicOr((err), OVF_BOUNDS), false))
#else
#define CFLR_CHECK(cond, err) true
#endif

struct WorkBufs {
    // touched rows {slot*2+o, idx}: touched[*parity] lists the rows whose
    // dnew > 0 (this iteration's deltas, "in"); touched[*parity ^ 1] gets the
    // rows the current merge appends to ("out").  The end-of-iteration
    // kernel flips the parity, so the same launch sequence serves every
    // iteration (and can be captured once in a CUDA graph).
    uint2 *touched[2];
    unsigned long long *touched_n;     // [2], device counts
    int *parity;                       // device
    unsigned long long touched_cap;
    uint2 *groups[N_BINS]; unsigned long long group_cap[N_BINS];   // {code, idx}
    unsigned long long *cand_key; uint32_t *cand_slot; unsigned long long cand_cap;
    uint2 *cand_wit;                   // witness of each candidate (null: off)
    unsigned long long *delta_key; uint32_t *delta_slot;
    uint32_t *bitmap_scratch; unsigned long long bitmap_words;  // per CTA, global
    uint2 *big_rows; unsigned long long big_cap;   // long delta rows (k_symbolic)
    Counters *cnt;
};

// ---- launch wrappers (kernels.cu) -------------------------------------
// Set the kernels' shared-memory limits (done by the first launch anyway;
// call it before capturing launches into a graph).
void prepare_launch_attributes();
void launch_symbolic(const SlotTab &S, const ProdTab &P, const WorkBufs &W, int prod_only,
                     const Tuning &T, int sms, cudaStream_t st);
void launch_spgemm(int bin, const SlotTab &S, const ProdTab &P, const WorkBufs &W,
                   uint32_t max_n, const Tuning &T, int sms, cudaStream_t st);
void launch_commit(const SlotTab &S, const WorkBufs &W, uint32_t n_slots, int sms,
                   cudaStream_t st);
// Iteration frame: zero the per-iteration counters; check the pre-commit
// conditions (buffer overflow, pair-set load); finish the iteration (pair
// counts, per-instance iteration counts, parity flip, loop condition).
void launch_iter_begin(const SlotTab &S, const InstTab &I, const WorkBufs &W, uint32_t n_slots,
                       uint32_t n_inst, cudaStream_t st);
// growth false (a test setting): never stop for a pair set's load, so a set
// may fill up (the capped probes then report OVF_FULL)
void launch_check(const SlotTab &S, const WorkBufs &W, uint32_t n_slots, bool growth,
                  cudaStream_t st);
void launch_iter_end(const SlotTab &S, const InstTab &I, const WorkBufs &W, LoopCtl *ctl,
                     uint32_t n_slots, uint32_t n_inst, bool count_iteration,
                     cudaGraphConditionalHandle handle, bool in_graph, cudaStream_t st);
void launch_reset_dnew(const SlotTab &S, const WorkBufs &W, int sms, cudaStream_t st);
// Room for every row the merge appends to (its new entries, and as many
// tiles again): rows that must grow move to a new segment with their tiles
// folded to one per word (one warp per row up to TILE_WARP_MAX tiles, then
// one CTA per row with an n-bit shared-memory bitmap for max_n up to the
// shared-memory limit, else copied as they are).
void launch_capacity(const SlotTab &S, const InstTab &I, const WorkBufs &W, int sms,
                     cudaStream_t st);
void launch_capacity_big(const SlotTab &S, const InstTab &I, const WorkBufs &W, uint32_t max_n,
                         int sms, cudaStream_t st);
void launch_scatter(const SlotTab &S, const WorkBufs &W, int sms, cudaStream_t st);
// Pack every appended row's new entries into tiles at the end of its tile list.
void launch_pack(const SlotTab &S, const WorkBufs &W, int sms, cudaStream_t st);

void launch_init_edges(const uint32_t *src, const uint32_t *lab, const uint32_t *dst,
                       unsigned long long n_edges, const uint32_t *term_off,
                       const uint32_t *term_slot, uint32_t n_terms, const WorkBufs &W,
                       int sms, cudaStream_t st);
void launch_init_eps(uint32_t slot, uint32_t n, const WorkBufs &W, int sms, cudaStream_t st);
// Move a pair set (and its witnesses, when val pointers are non-null) into
// a larger table; a key that finds no free slot in one pass sets OVF_FULL in
// *err.
void launch_rehash(const unsigned long long *old_tab, const uint2 *old_val,
                   unsigned long long old_cap, unsigned long long *new_tab, uint2 *new_val,
                   unsigned long long new_cap, unsigned *err, int sms, cudaStream_t st);
// The witness of pair `key` in a pair set of capacity mask + 1, written to
// *out ({~0, ~0} when the pair is absent).
void launch_witness_lookup(const unsigned long long *tab, const uint2 *val,
                           unsigned long long mask, unsigned long long key, uint2 *out,
                           cudaStream_t st);
void launch_fill_u64(unsigned long long *p, unsigned long long count, unsigned long long v,
                     int sms, cudaStream_t st);
void launch_remap_touched(const uint2 *in, unsigned long long n, uint32_t slot_base,
                          uint2 *out, cudaStream_t st);
// Per-instance split of a batch touched list (counts, then scatter with
// local slot ids); slot_inst maps a slot to its instance.
void launch_touched_count(const uint2 *in, unsigned long long n, const uint32_t *slot_inst,
                          unsigned long long *cnt, cudaStream_t st);
void launch_touched_split(const uint2 *in, unsigned long long n, const uint32_t *slot_inst,
                          const uint32_t *inst_base, uint2 *const *out,
                          unsigned long long *cursor, cudaStream_t st);

// out[i] = in[0] + ... + in[i-1]; bsum: ceil(n/1024) scratch; grand (nullable)
// receives the total.
void launch_exclusive_scan(const uint32_t *in, uint32_t n, unsigned long long *out,
                           unsigned long long *bsum, unsigned long long *grand, cudaStream_t st);

// Extraction of one non-terminal's pairs, sorted by (src, dst), in the
// caller's vertex ids, with caller-provided scratch (the allocation-free
// read-out; the other read-outs use the list extraction below): perm maps a
// caller id to its stored row, iperm a stored id back (both null when the
// vertices kept their input order).
void launch_row_lengths(const uint4 *desc, const uint32_t *pool, uint32_t n,
                        const uint32_t *perm, uint32_t *len, cudaStream_t st);
// big_rows: scratch of n uint32 followed by two counters (big_count points
// at the first: the long-row count, then the row cursor); bitmap: scratch of
// sms*4*ceil(n/32) words used when a row bitmap does not fit shared memory.
void launch_extract(const uint4 *desc, const uint32_t *pool, uint32_t n, const uint32_t *perm,
                    const uint32_t *iperm, const unsigned long long *row_out, uint32_t *out_src,
                    uint32_t *out_dst, uint32_t *big_rows, uint32_t *big_count,
                    uint32_t *bitmap, int sms, cudaStream_t st);

// Extraction of a list of non-terminals, one after another (each
// non-terminal's pairs sorted by (src, dst)).  The rows of listed
// non-terminal k are cut into units of rows_per[k] rows, units unit_first[k]
// .. unit_first[k + 1] - 1; every listed one is non-empty.  All tables are on
// the device.
// launch_extract_count: units (units + 1 words) receives every unit's first
// output position (an exclusive scan of the units' pair counts in list
// order), *total the pair count; bsum: units / 1024 + 2 words.
// launch_extract_write: the rows of units u_begin .. u_end - 1, a pair at
// output position o written at out_src / out_dst[o - base]; a row that
// would end past position `limit` is not written (bit 1 of *err).  Long rows
// are listed in big (big_cap entries: the range's pairs / 1024 + 1 always
// suffice; an overflow sets bit 0 of *err); cursor: two words; bitmap as for
// launch_extract.
struct ExtractList {
    const uint4 *desc;                  // every non-terminal's descriptors, 2 n each
    const uint32_t *pool;
    const uint32_t *perm, *iperm;
    const uint32_t *nts;                // listed non-terminal ids (count)
    const uint32_t *rows_per;           // rows per unit of each (count)
    const unsigned long long *unit_first;   // first unit of each (count + 1)
    uint32_t n, count;
    unsigned long long units;           // unit_first[count]
    unsigned long long u_begin, u_end;  // units written by launch_extract_write
    unsigned long long base, limit;     // output positions: written at o - base, o < limit
};
// Units of listed non-terminals with pairs[k] pairs each, n rows: about
// eight units per resident warp in all, each with a like share of the pairs
// and at most 4096 rows.  Fills rows_per and unit_first (count + 1).
void extract_plan(uint32_t count, uint32_t n, const uint64_t *pairs, int sms,
                  uint32_t *rows_per, unsigned long long *unit_first);
void launch_extract_count(const ExtractList &L, unsigned long long *units,
                          unsigned long long *bsum, unsigned long long *total, int sms,
                          cudaStream_t st);
void launch_extract_write(const ExtractList &L, uint32_t *out_src, uint32_t *out_dst,
                          const unsigned long long *units, uint4 *big,
                          unsigned long long big_cap, unsigned long long *cursor,
                          uint32_t *bitmap, unsigned *err, int sms, cudaStream_t st);

// Vertex renumbering on the device (renumber.cu): the breadth-first order of
// the undirected edges a one-thread queue search gives.  The host runs, in
// this order: launch_rn_adjacency (degrees deg[n], the largest into
// *max_deg), an exclusive scan of deg into off[0..n], launch_rn_fill (the
// adjacency lists adj[off[v] ..] of (edge << 32 | neighbour), sorted; every
// list at most RENUM_LIST_MAX long; cur: n words, big: n words, big_n: one),
// launch_rn_init, launch_rn_cc_pass until *more stays 0, launch_rn_count,
// scans of cnt (component offsets) and is_root (root offsets, the root count
// as total), launch_rn_roots (level 0), then per level launch_rn_claim, a
// scan of won into woff[0..fsize], launch_rn_write (the next frontier into
// F2, the next segment tables, perm and iperm), until the frontier is empty;
// launch_rn_check sets *bad unless perm and iperm are inverse permutations.
constexpr uint32_t RENUM_LIST_MAX = 8192;
void launch_rn_adjacency(const uint32_t *src, const uint32_t *dst, unsigned long long m,
                         uint32_t n, uint32_t *deg, uint32_t *max_deg, int sms, cudaStream_t st);
void launch_rn_fill(const uint32_t *src, const uint32_t *dst, unsigned long long m, uint32_t n,
                    const unsigned long long *off, unsigned long long *cur,
                    unsigned long long *adj, uint32_t *big, uint32_t *big_n, uint32_t max_deg,
                    int sms, cudaStream_t st);
void launch_rn_init(uint32_t n, uint32_t *parent, uint32_t *lvl, unsigned long long *key,
                    uint32_t *iperm, int sms, cudaStream_t st);
void launch_rn_cc_pass(const uint32_t *src, const uint32_t *dst, unsigned long long m,
                       uint32_t n, uint32_t *parent, unsigned *more, int sms, cudaStream_t st);
void launch_rn_count(const uint32_t *parent, uint32_t n, uint32_t *cnt, uint32_t *is_root,
                     int sms, cudaStream_t st);
void launch_rn_roots(const uint32_t *parent, uint32_t n, const unsigned long long *roff,
                     const unsigned long long *comp_off, uint32_t *F, uint32_t *lvl, uint32_t *sf,
                     uint32_t *se, uint32_t *pc, uint32_t *perm, uint32_t *iperm, int sms,
                     cudaStream_t st);
void launch_rn_claim(const uint32_t *F, uint32_t fsize, const unsigned long long *off,
                     const unsigned long long *adj, const uint32_t *lvl, unsigned long long *key,
                     uint32_t *won, int sms, cudaStream_t st);
void launch_rn_write(const uint32_t *F, uint32_t fsize, const unsigned long long *off,
                     const unsigned long long *adj, uint32_t *lvl, const unsigned long long *key,
                     const unsigned long long *woff, uint32_t *F2, uint32_t level,
                     const uint32_t *parent, const unsigned long long *comp_off,
                     const uint32_t *sf, const uint32_t *se, const uint32_t *pc, uint32_t *sf2,
                     uint32_t *se2, uint32_t *pc2, uint32_t *perm, uint32_t *iperm, uint32_t n,
                     int sms, cudaStream_t st);
void launch_rn_check(const uint32_t *perm, const uint32_t *iperm, uint32_t n, unsigned *bad,
                     int sms, cudaStream_t st);

// a[e] <- perm[a[e]] for e < m (vertex renumbering of the loaded edges)
void launch_permute_ids(uint32_t *a, unsigned long long m, const uint32_t *perm, int sms,
                        cudaStream_t st);

}  // namespace cflr
