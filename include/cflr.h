/*
 * cflr.h - C ABI of the GB300 CFL-reachability solver.
 *
 * Problem (paper Sec. 2, Algorithm 1 "Data"/"Result"): given a context-free
 * grammar Gr = (N, Sigma, P, S) in weak Chomsky normal form and a graph
 * G = (V, E) whose edges carry terminal labels, compute for every
 * non-terminal X the boolean |V| x |V| matrix
 *     M_X(i, j) = 1  iff  some path i -> j has a label word derivable from X.
 * The solver keeps one sparse boolean matrix per non-terminal (Algorithm 1,
 * storage comment) and runs the closure loop of Algorithm 1 in the
 * semi-naive form of optimisation 1:  every production c -> a b adds
 * (dA . B) u (A_old . dB) to M_c, minus what M_c already holds, until no
 * iteration adds a pair.  All device work runs in this library's own CUDA
 * kernels for sm_103a; the arithmetic is boolean/integer and exact.
 *
 * Conventions for every entry point:
 *   - The return value is a status: CFLR_OK (0) or a negative CFLR_E* code.
 *     On error, cflr_last_error() describes it; the context stays usable
 *     unless the code is CFLR_ECUDA (the CUDA context itself failed).
 *   - Input buffers are host memory owned by the caller and are copied before
 *     the call returns.  The context owns all device memory it allocates and
 *     frees it in cflr_destroy().  Output buffers are host memory owned by
 *     the caller.
 *   - Call order: cflr_create -> cflr_load_grammar -> cflr_load_graph ->
 *     cflr_solve -> cflr_get_pairs (any number of times).  Loading a new
 *     graph discards the previous matrices; loading a new grammar discards
 *     the graph.  Calls out of order return CFLR_ESTATE.
 *   - A context belongs to one host thread at a time.  Contexts on different
 *     streams may solve concurrently.
 */
#ifndef CFLR_H
#define CFLR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    CFLR_OK = 0,
    CFLR_EINVAL = -1,    /* bad argument (NULL pointer, size, capacity too small) */
    CFLR_EGRAMMAR = -2,  /* grammar text is malformed or not in WCNF            */
    CFLR_EGRAPH = -3,    /* vertex id out of range, or too many vertices        */
    CFLR_ENOMEM = -4,    /* device memory exhausted or over mem_budget_bytes    */
    CFLR_ECUDA = -5,     /* a CUDA runtime call failed                          */
    CFLR_ELIMIT = -6,    /* max_iterations reached before the fixpoint          */
    CFLR_ESTATE = -7,    /* call out of order                                   */
    CFLR_ETIMEOUT = -8   /* a bounded device-side wait gave up                  */
};

/* Execution forms of the closure loop (all give identical pair sets). */
enum {
    CFLR_FORM_PLAIN = 0,    /* one launch sequence per production per iteration,
                               the shape of one library mxm per production      */
    CFLR_FORM_BATCHED = 1,  /* every production of an iteration in one launch
                               sequence; the host checks convergence each time  */
    CFLR_FORM_GRAPH = 2     /* the batched iteration captured in a CUDA graph and
                               repeated on the device until no pair is added    */
};

typedef struct cflr_ctx cflr_ctx;

typedef struct {
    int device;                 /* CUDA device ordinal                              */
    void *stream;               /* cudaStream_t to run on; NULL = a private stream  */
    uint64_t mem_budget_bytes;  /* cap on device bytes this context may hold; 0 = none.
                                   A work buffer that overflows triples without a
                                   budget and grows by half under one              */
    uint32_t max_iterations;    /* stop with CFLR_ELIMIT after this many; 0 = none  */
    int form;                   /* CFLR_FORM_*                                      */
    int profile;                /* nonzero: time every kernel launch with CUDA events
                                   on the solve stream (see cflr_kernel_stats)      */
    const char *autotune_cache; /* path of the cflr_autotune cache file, or NULL;
                                   cflr_create copies the string                    */
    uint32_t initial_capacity;  /* entries of the first work buffers; 0 = sized from
                                   the input.  Small values exercise the growth
                                   paths (every phase re-runs after a growth).      */
    uint32_t size_hint;         /* expected pairs per input edge of the finished
                                   closure over all non-terminals (0 = unknown): the
                                   pair sets start with room for an even share of it
                                   (three slots per expected pair) and the row pool
                                   with six words per expected pair, so a fresh
                                   graph grows them rarely                          */
    int stop_on_first_converged;/* nonzero: a batch led by this context stops after
                                   the first iteration in which some context reaches
                                   its fixpoint (CFLR_ELIMIT while others remain), so
                                   a server can retire and admit between iterations  */
    int keep_vertex_order;      /* nonzero: store vertex v as row v.  0 (default):
                                   the library renumbers the vertices internally in
                                   breadth-first order of the undirected input edges,
                                   so a row's entries fall into few 32-bit words (the
                                   bit-packed tiles of the row storage); results
                                   always use the caller's ids                      */
    int witness;                /* nonzero: keep one derivation step for every pair
                                   (single-path semantics, see cflr_get_witness);
                                   costs 8 more bytes per pair-set slot and per
                                   candidate, and needs at most 32768
                                   non-terminals                                    */
    int test_fixed_pair_sets;   /* testing only: nonzero keeps every pair set at its
                                   first size.  A set that fills up then stops the
                                   solve: its hash probes are capped at one pass over
                                   the table and report the full set, cflr_solve
                                   returns CFLR_ECUDA and the context needs a new
                                   graph (it stays usable)                          */
    int order_on_device;        /* where the breadth-first vertex order is found
                                   (unless keep_vertex_order): 0 (default) on the
                                   GPU for graphs of at least 2^18 edges, on the
                                   host below that; 1 on the GPU; -1 on the host.
                                   Both give the same order.  The GPU search needs
                                   fewer than 2^32 edges and no vertex with more
                                   than 8192 edge ends; other graphs are ordered on
                                   the host whatever this says                      */
} cflr_config;

typedef struct {
    uint32_t iterations;        /* closure iterations run (the last one adds nothing) */
    uint64_t total_pairs;       /* sum of pairs over the non-terminals named in the
                                   grammar text (terminal wrappers excluded)        */
    double solve_ms;            /* device time of cflr_solve (CUDA events)          */
    uint64_t peak_device_bytes; /* high-water mark of this context's device memory  */
    uint64_t ignored_edges;     /* edges whose label no production uses             */
    uint64_t flops;             /* product steps: every referenced 32-bit tile is one
                                   step that ORs up to 32 pairs into an accumulator */
    uint64_t candidates;        /* pairs the products emitted after the mask        */
    uint64_t regrows;           /* buffer growths that re-ran a phase               */
    uint32_t converged;         /* 1 when the context has reached its fixpoint      */
    uint64_t groups[4];         /* work-list groups run by each product bin         */
    uint64_t regrow_buffers;    /* of regrows: work buffers (work list, candidates)  */
    uint64_t regrow_sets;       /* of regrows: pair sets (hash tables) moved          */
    uint64_t regrow_pools;      /* of regrows: row pools moved                       */
    uint64_t flops_bin3;        /* of flops: product steps of the bitmap bin (3)     */
    uint64_t mask_tiles_bin3;   /* mask-row tiles the bitmap bin's groups loaded     */
} cflr_stats;

/* Schedule of the product kernels.  Each (production, delta row) group goes
 * to the first bin whose limit holds its accumulator need (mask entries plus
 * products, or products alone when it probes the pair set instead of
 * loading the mask row, which it does when mask_len > probe_ratio *
 * products); bin 3 takes the rest with an n-bit bitmap.  Limits must
 * increase and stay within 128, 1024 and 4096 (the bins' table sizes). */
typedef struct {
    uint32_t probe_ratio;       /* >= 1                                             */
    uint32_t bin_limit[3];      /* accumulator need bounds of bins 0, 1, 2          */
    uint32_t ctas_per_sm[4];    /* grid of each bin in CTAs per SM (1..32); for bin 3
                                   an upper bound under the shared-memory limit     */
} cflr_tuning;

/* Default configuration: device 0, private stream, no budget, no iteration
 * limit, CFLR_FORM_BATCHED, profiling off. */
void cflr_default_config(cflr_config *cfg);

/* Create a context on cfg->device (cfg NULL = defaults).  *out receives the
 * context; nothing is allocated on the device until a graph is loaded.
 * Errors: CFLR_EINVAL (out NULL, bad form), CFLR_ECUDA (device unusable). */
int cflr_create(cflr_ctx **out, const cflr_config *cfg);

/* Load a grammar (paper Sec. 2, WCNF definition) from text of len bytes.
 * Format: one production per line, "LHS -> X Y", "LHS -> x", "LHS -> eps"
 * or "LHS -> X" (unit production); "|" separates alternatives; "#" starts a
 * comment.  A symbol is a non-terminal iff it is the left-hand side of some
 * production; all other symbols are terminals (edge labels).  A directive
 * "%index v lo hi" makes each production mentioning "_{v}" stand for one copy
 * per value lo..hi (the indexed non-terminals of the paper's appendix B).
 * A terminal inside a binary production is replaced by a fresh non-terminal
 * named "<x>" with the single production "<x> -> x".
 * Errors: CFLR_EINVAL (NULL text), CFLR_EGRAMMAR (malformed; see
 * cflr_last_error for the line). */
int cflr_load_grammar(cflr_ctx *c, const char *text, size_t len);

/* Look up a symbol of the loaded grammar.  Non-terminal ids are 0..nt-1 in
 * order of first appearance as a left-hand side, wrappers "<x>" last;
 * terminal ids are 0..t-1 in order of first appearance.
 * Errors: CFLR_ESTATE (no grammar), CFLR_EINVAL (unknown name). */
int cflr_symbol_id(const cflr_ctx *c, const char *name, uint32_t *id, int *is_terminal);

/* Number of non-terminals (wrappers included), of those named in the text,
 * and of terminals. */
int cflr_grammar_sizes(const cflr_ctx *c, uint32_t *n_nonterminals, uint32_t *n_named,
                       uint32_t *n_terminals);

/* Load a graph: n_vertices vertices with ids 0..n_vertices-1 (the paper's
 * 1..n shifted by one) and n_edges edges src[e] --label[e]--> dst[e], all
 * host arrays of uint32.  Labels are terminal ids from cflr_symbol_id; a
 * label id that is not a terminal of the grammar is legal, adds nothing
 * (Algorithm 1 initialisation with the empty set) and is counted in
 * cflr_stats.ignored_edges.  Duplicate edges are harmless.  The edges are
 * copied to the device and turned into the initial matrices (Algorithm 1,
 * terminal initialisation; the identity for every A -> eps).
 * Errors: CFLR_ESTATE (no grammar), CFLR_EINVAL (NULL arrays with
 * n_edges > 0), CFLR_EGRAPH (an id >= n_vertices, or n_vertices too large for
 * the packed 64-bit pair keys: n_nonterminals * n_vertices^2 >= 2^62),
 * CFLR_ENOMEM, CFLR_ECUDA. */
int cflr_load_graph(cflr_ctx *c, uint32_t n_vertices, uint64_t n_edges,
                    const uint32_t *src, const uint32_t *label, const uint32_t *dst);

/* Run the closure loop of Algorithm 1 with optimisation 1 to its fixpoint.
 * Blocks until the device finishes.  stats may be NULL.  Solving again
 * without a new graph is a no-op that reports the same pairs.
 * Errors: CFLR_ESTATE (no graph), CFLR_ELIMIT (max_iterations reached; the
 * matrices hold every pair found so far and a further cflr_solve continues
 * from there), CFLR_ENOMEM (the matrices are dropped: load a graph again),
 * CFLR_ECUDA. */
int cflr_solve(cflr_ctx *c, cflr_stats *stats);

/* Copy the pairs of non-terminal `nonterminal` into host arrays src/dst,
 * sorted by (src, dst).  *n_pairs receives the count.  With src == dst ==
 * NULL only the count is returned.  If capacity < count, nothing is copied,
 * *n_pairs holds the count and CFLR_EINVAL is returned.
 * Errors: CFLR_ESTATE (not solved), CFLR_EINVAL (bad id, capacity). */
int cflr_get_pairs(const cflr_ctx *c, uint32_t nonterminal, uint32_t *src, uint32_t *dst,
                   uint64_t capacity, uint64_t *n_pairs);

/* As cflr_get_pairs, but d_src/d_dst are device pointers (on this context's
 * device) owned by the caller; the pairs never leave the GPU.  The call
 * returns after the copy has finished on the context's stream. */
int cflr_get_pairs_device(const cflr_ctx *c, uint32_t nonterminal, uint32_t *d_src,
                          uint32_t *d_dst, uint64_t capacity, uint64_t *n_pairs);

/* The pairs of several non-terminals in one call (the result of Algorithm 1
 * for each of them, as cflr_get_pairs gives it).  nonterminals[0..count)
 * (host array; an id may repeat) are written one after another into the host
 * arrays src/dst, each non-terminal's pairs sorted by (src, dst).
 * offsets (host array of count + 1 entries, required) receives where the
 * pairs of nonterminals[i] start, and offsets[count] the total.  With
 * src == dst == NULL only offsets are filled.  If capacity < total, nothing is
 * copied, offsets are filled and CFLR_EINVAL is returned.  All listed
 * non-terminals are extracted together (not one call's work per
 * non-terminal): the pairs pass through two device staging buffers of at
 * most 16 Mi pairs, each copied to the host while the next range is written.
 * The call waits for the device twice: after counting and at the end.
 * Errors: CFLR_ESTATE (no graph), CFLR_EINVAL (NULL offsets, a bad id,
 * capacity), CFLR_ENOMEM, CFLR_ECUDA. */
int cflr_get_pairs_many(const cflr_ctx *c, uint32_t count, const uint32_t *nonterminals,
                        uint32_t *src, uint32_t *dst, uint64_t capacity, uint64_t *offsets);

/* As cflr_get_pairs_many, but d_src/d_dst are device pointers (on this
 * context's device) owned by the caller; offsets stays a host array.  No
 * staging: the kernels write the caller's arrays, and the call waits for the
 * device once, after the last pair has been written on the context's
 * stream. */
int cflr_get_pairs_device_many(const cflr_ctx *c, uint32_t count, const uint32_t *nonterminals,
                               uint32_t *d_src, uint32_t *d_dst, uint64_t capacity,
                               uint64_t *offsets);

/* Kinds of a derivation step (cflr_get_witness). */
enum {
    CFLR_WIT_BINARY = 0,  /* nonterminal -> A B: (src, mid) in A, (mid, dst) in B    */
    CFLR_WIT_EDGE = 1,    /* nonterminal -> x: an edge src --x--> dst (id = label)   */
    CFLR_WIT_UNIT = 2,    /* nonterminal -> A: (src, dst) in A (id = A)              */
    CFLR_WIT_EPS = 3      /* nonterminal -> eps: src == dst                          */
};

/* Single-path semantics (the paper's closing remarks: its optimisations carry
 * over by changing the semiring).  With cfg.witness set, every pair keeps the
 * first derivation step the closure found for it: *kind is a CFLR_WIT_*
 * value, *id and *id2 the non-terminal ids A and B (CFLR_WIT_BINARY), A
 * (CFLR_WIT_UNIT) or the label (CFLR_WIT_EDGE), and *mid the middle vertex
 * of a binary step.  The steps of a pair refer only to pairs found in
 * earlier iterations, so following them down to edges always ends, and
 * gives a path from src to dst whose label word the non-terminal derives.
 * Pointers other than kind may be NULL.  Errors: CFLR_ESTATE (no graph, or
 * the context was created without cfg.witness), CFLR_EINVAL (a bad id, or
 * (src, dst) not in the relation), CFLR_ECUDA. */
int cflr_get_witness(const cflr_ctx *c, uint32_t nonterminal, uint32_t src, uint32_t dst,
                     int *kind, uint32_t *id, uint32_t *id2, uint32_t *mid);

/* Largest graph (vertices) cflr_get_pairs_device_noalloc accepts. */
#define CFLR_NOALLOC_MAX_VERTICES 1048576u

/* As cflr_get_pairs_device, but allocates no device memory.  (The paper has
 * no counterpart; this serves callers that may not allocate when they read
 * results: code that runs against a fixed device-memory plan made at
 * start-up, embedders whose own allocator owns the whole device, and paths
 * that must not risk the device synchronisation cudaMalloc/cudaFree can
 * cause.)  Its scratch lives in one static device array of about 16 MiB
 * inside this library, which every GPU that loads the library holds until
 * the process exits.
 *   - Graphs with more than CFLR_NOALLOC_MAX_VERTICES vertices are rejected
 *     with CFLR_EINVAL; nothing is launched.
 *   - The first call for a device looks up the array's device address on
 *     that device (cudaGetSymbolAddress); make that first call before any
 *     stream capture.  The address is kept for the life of the process: a
 *     cudaDeviceReset destroys the array (and every context of this library
 *     on that device), and this entry point must not be called for that
 *     device afterwards.
 *   - All calls share the one array per device: calls whose work overlaps
 *     on the GPU (other host threads, or contexts on other streams) race and
 *     may return wrong pairs.  Serialise them.
 *   - Arguments, output format and other errors as cflr_get_pairs_device. */
int cflr_get_pairs_device_noalloc(const cflr_ctx *c, uint32_t nonterminal, uint32_t *d_src,
                                  uint32_t *d_dst, uint64_t capacity, uint64_t *n_pairs);

/* The vertex order the context stores the loaded graph in: order[k]
 * receives the caller's id of the vertex stored as row k (the identity with
 * keep_vertex_order).  order is a host array of at least n_vertices entries
 * (capacity).  The order only places rows in memory; results never depend
 * on it.  Errors: CFLR_ESTATE (no graph), CFLR_EINVAL (NULL order, capacity
 * below the vertex count), CFLR_ECUDA. */
int cflr_get_vertex_order(const cflr_ctx *c, uint32_t *order, uint64_t capacity);

/* Restore the matrices of the loaded graph to Algorithm 1's terminal
 * initialisation, from the copy of the edges cflr_load_graph keeps on the
 * device (no host transfer).  Device buffers grown by earlier solves are
 * kept, so a reset-solve cycle allocates nothing in steady state.
 * Errors: CFLR_ESTATE (no graph), CFLR_ENOMEM, CFLR_ECUDA. */
int cflr_reset(cflr_ctx *c);

/* Solve n independent contexts together: each closure iteration runs the
 * products of all unfinished contexts in one launch sequence.  Every
 * context must hold a loaded graph and use the same device and stream as
 * ctxs[0].  stats (nullable) is an array of n.  Results are identical to
 * solving each context alone.  The iteration limit and the work buffers are
 * those of ctxs[0], which may be a context whose solve has already finished
 * (it then only lends its buffers): with max_iterations = 1 every call
 * advances each unfinished context by one closure iteration, and contexts
 * may join or leave between calls (continuous batching).  stats[k].converged
 * tells which contexts are done; the call returns CFLR_ELIMIT while any is
 * not.
 * Errors: as cflr_solve; CFLR_EINVAL for n <= 0 or mixed devices. */
int cflr_solve_batch(cflr_ctx *const *ctxs, int n, cflr_stats *stats);

/* Per-kernel timing of the last solve when cfg.profile was set: for kernel
 * index k (0..count-1) its name, launches, total device milliseconds (CUDA
 * events on the solve stream) and algorithmic bytes moved (the bytes the
 * method must read and write, counted by the kernels themselves).
 * cflr_kernel_stats(c, -1, ...) returns the number of kernels in *launches. */
int cflr_kernel_stats(const cflr_ctx *c, int k, const char **name, uint64_t *launches,
                      double *total_ms, uint64_t *alg_bytes);

/* Read or set the product-kernel schedule of a context (also used for
 * batches it leads).  Errors: CFLR_EINVAL (NULL, or a schedule outside the
 * limits above). */
int cflr_get_tuning(const cflr_ctx *c, cflr_tuning *t);
int cflr_set_tuning(cflr_ctx *c, const cflr_tuning *t);

/* Pick the schedule for the loaded graph by measurement: starting from the
 * current one, try candidate values of each field in turn (coordinate
 * descent), timing a reset-and-solve of the loaded graph for each, and keep
 * the fastest.  At most max_trials solves (0 = 24).  When cfg.autotune_cache
 * names a file, a schedule stored there for the same grammar text and graph
 * size is used without measuring, and a measured one is added to it.
 * Afterwards the matrices are back at the terminal initialisation (as after
 * cflr_reset) and *best (nullable) holds the schedule now in use.
 * Errors: CFLR_ESTATE (no graph), and those of cflr_solve. */
int cflr_autotune(cflr_ctx *c, uint32_t max_trials, cflr_tuning *best);

/* Description of the last error on this context (never NULL). */
const char *cflr_last_error(const cflr_ctx *c);

/* Free every device and host resource of the context.  NULL is a no-op. */
void cflr_destroy(cflr_ctx *c);

#ifdef __cplusplus
}
#endif

#endif /* CFLR_H */
