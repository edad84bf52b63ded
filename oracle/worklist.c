/*
 * CFL-reachability oracle: a single-threaded worklist solver in plain C.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file's library.  It shares
 * no code, header, table or helper with the CUDA library.
 *
 * What it computes (the paper's problem statement, Algorithm 1, "Result"):
 * for every non-terminal X the set
 *     R_X = { (i, j) | some path i -> j has a label word w with X =>* w }.
 * The method of the paper (Algorithm 1 with optimisations 1-5) reaches exactly
 * this set (Sec. 4: the optimisations preserve the answers), and it is the
 * least fixpoint of the productions, so any schedule that applies them until
 * nothing changes gives the same result.  This file applies them pair by pair
 * (the classic dynamic-transitive-closure worklist), which is the plainest way
 * to reach the least fixpoint:
 *
 *   seed   (u, A, v) for every edge (u, x, v) and every production A -> x
 *          (Algorithm 1, terminal initialisation);
 *          (i, A, i) for every vertex i and every production A -> eps;
 *   pop    (u, A, v) and apply every production in which A occurs:
 *            C -> A B : for every w with (v, B, w) known, add (u, C, w)
 *            C -> B A : for every w with (w, B, u) known, add (w, C, v)
 *            C -> A   : add (u, C, v)           (unit production)
 *   "add"  inserts into R_C and pushes the triple only when it is new;
 *   stop   when the worklist is empty.
 *
 * The grammar arrives already in weak Chomsky normal form (Sec. 2, WCNF
 * definition) with terminals of binary productions wrapped by the caller.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define EMPTY_KEY UINT64_MAX

typedef struct {
    uint64_t *keys;
    uint64_t cap;   /* power of two */
    uint64_t size;
} pairset;

typedef struct {
    uint32_t *v;
    uint32_t len, cap;
} vec32;

typedef struct {
    uint32_t c, other;
} use_t;

typedef struct {
    uint32_t n, n_nt;
    pairset *R;        /* R[X]: the pairs of non-terminal X                    */
    vec32 **out;       /* out[X][u]: all v with (u, X, v); only if X is read so */
    vec32 **in;        /* in[X][v]:  all u with (u, X, v); only if X is read so */
    /* productions indexed by the non-terminal that was just derived */
    uint32_t *left_off, *right_off, *unit_off;   /* n_nt + 1 offsets each */
    use_t *left_use;   /* A -> (C, B) for every C -> A B */
    use_t *right_use;  /* A -> (C, B) for every C -> B A */
    uint32_t *unit_use;/* A -> C      for every C -> A   */
    uint32_t *wl;      /* worklist of (u, X, v) triples */
    uint64_t wl_len, wl_cap;
    uint64_t pops, joins;
    int oom;
} oracle_state;

static uint64_t mix64(uint64_t x) {
    x ^= x >> 30; x *= 0xBF58476D1CE4E5B9ULL;
    x ^= x >> 27; x *= 0x94D049BB133111EBULL;
    x ^= x >> 31;
    return x;
}

static int set_init(pairset *s, uint64_t cap) {
    s->cap = cap; s->size = 0;
    s->keys = (uint64_t *)malloc(cap * sizeof(uint64_t));
    if (!s->keys) return -1;
    memset(s->keys, 0xFF, cap * sizeof(uint64_t));
    return 0;
}

static int set_insert_raw(uint64_t *keys, uint64_t cap, uint64_t key) {
    uint64_t m = cap - 1, h = mix64(key) & m;
    for (;;) {
        if (keys[h] == key) return 0;
        if (keys[h] == EMPTY_KEY) { keys[h] = key; return 1; }
        h = (h + 1) & m;
    }
}

/* 1 if key was new, 0 if present, -1 on allocation failure */
static int set_insert(pairset *s, uint64_t key) {
    if (2 * (s->size + 1) > s->cap) {
        pairset t;
        if (set_init(&t, s->cap * 2)) return -1;
        for (uint64_t i = 0; i < s->cap; i++)
            if (s->keys[i] != EMPTY_KEY) set_insert_raw(t.keys, t.cap, s->keys[i]);
        free(s->keys);
        s->keys = t.keys; s->cap = t.cap;
    }
    int r = set_insert_raw(s->keys, s->cap, key);
    s->size += (uint64_t)r;
    return r;
}

static int vec_push(vec32 *a, uint32_t x) {
    if (a->len == a->cap) {
        uint32_t nc = a->cap ? a->cap * 2 : 4;
        uint32_t *p = (uint32_t *)realloc(a->v, (size_t)nc * sizeof(uint32_t));
        if (!p) return -1;
        a->v = p; a->cap = nc;
    }
    a->v[a->len++] = x;
    return 0;
}

static void add(oracle_state *st, uint32_t u, uint32_t X, uint32_t v) {
    int r = set_insert(&st->R[X], ((uint64_t)u << 32) | v);
    if (r < 0) { st->oom = 1; return; }
    if (r == 0) return;
    if (st->out[X] && vec_push(&st->out[X][u], v)) { st->oom = 1; return; }
    if (st->in[X] && vec_push(&st->in[X][v], u)) { st->oom = 1; return; }
    if (st->wl_len + 3 > st->wl_cap) {
        uint64_t nc = st->wl_cap ? st->wl_cap * 2 : 3 * 4096;
        uint32_t *p = (uint32_t *)realloc(st->wl, nc * sizeof(uint32_t));
        if (!p) { st->oom = 1; return; }
        st->wl = p; st->wl_cap = nc;
    }
    st->wl[st->wl_len++] = u;
    st->wl[st->wl_len++] = X;
    st->wl[st->wl_len++] = v;
}

void oracle_free(oracle_state *st);

/*
 * Solve one instance.
 *   n        number of vertices (ids 0 .. n-1)
 *   n_nt     number of non-terminals (ids 0 .. n_nt-1)
 *   binary   3*n_bin ids (c, a, b) for productions c -> a b
 *   unit     2*n_unit ids (c, a) for productions c -> a
 *   eps      n_eps ids A for productions A -> eps
 *   init     3*n_init triples (u, A, v): the terminal initialisation
 * Returns a state to read results from, or NULL when memory ran out.
 */
oracle_state *oracle_solve(uint32_t n, uint32_t n_nt,
                           uint32_t n_bin, const uint32_t *binary,
                           uint32_t n_unit, const uint32_t *unit,
                           uint32_t n_eps, const uint32_t *eps,
                           uint64_t n_init, const uint32_t *init) {
    oracle_state *st = (oracle_state *)calloc(1, sizeof(oracle_state));
    if (!st) return NULL;
    st->n = n; st->n_nt = n_nt;
    st->R = (pairset *)calloc(n_nt, sizeof(pairset));
    st->out = (vec32 **)calloc(n_nt, sizeof(vec32 *));
    st->in = (vec32 **)calloc(n_nt, sizeof(vec32 *));
    st->left_off = (uint32_t *)calloc(n_nt + 1, sizeof(uint32_t));
    st->right_off = (uint32_t *)calloc(n_nt + 1, sizeof(uint32_t));
    st->unit_off = (uint32_t *)calloc(n_nt + 1, sizeof(uint32_t));
    st->left_use = (use_t *)malloc((n_bin + 1) * sizeof(use_t));
    st->right_use = (use_t *)malloc((n_bin + 1) * sizeof(use_t));
    st->unit_use = (uint32_t *)malloc((n_unit + 1) * sizeof(uint32_t));
    if (!st->R || !st->out || !st->in || !st->left_off || !st->right_off ||
        !st->unit_off || !st->left_use || !st->right_use || !st->unit_use) {
        oracle_free(st); return NULL;
    }
    for (uint32_t X = 0; X < n_nt; X++)
        if (set_init(&st->R[X], 16)) { oracle_free(st); return NULL; }

    /* Index productions by each operand; allocate the adjacency a production reads. */
    for (uint32_t p = 0; p < n_bin; p++) {
        uint32_t a = binary[3 * p + 1], b = binary[3 * p + 2];
        st->left_off[a + 1]++;
        st->right_off[b + 1]++;
        if (!st->out[b]) st->out[b] = (vec32 *)calloc(n ? n : 1, sizeof(vec32));
        if (!st->in[a]) st->in[a] = (vec32 *)calloc(n ? n : 1, sizeof(vec32));
        if (!st->out[b] || !st->in[a]) { oracle_free(st); return NULL; }
    }
    for (uint32_t p = 0; p < n_unit; p++) st->unit_off[unit[2 * p + 1] + 1]++;
    for (uint32_t X = 0; X < n_nt; X++) {
        st->left_off[X + 1] += st->left_off[X];
        st->right_off[X + 1] += st->right_off[X];
        st->unit_off[X + 1] += st->unit_off[X];
    }
    {
        uint32_t *fl = (uint32_t *)calloc(n_nt + 1, sizeof(uint32_t));
        uint32_t *fr = (uint32_t *)calloc(n_nt + 1, sizeof(uint32_t));
        uint32_t *fu = (uint32_t *)calloc(n_nt + 1, sizeof(uint32_t));
        if (!fl || !fr || !fu) { free(fl); free(fr); free(fu); oracle_free(st); return NULL; }
        for (uint32_t p = 0; p < n_bin; p++) {
            uint32_t c = binary[3 * p], a = binary[3 * p + 1], b = binary[3 * p + 2];
            use_t ul = {c, b}, ur = {c, a};
            st->left_use[st->left_off[a] + fl[a]++] = ul;
            st->right_use[st->right_off[b] + fr[b]++] = ur;
        }
        for (uint32_t p = 0; p < n_unit; p++) {
            uint32_t c = unit[2 * p], a = unit[2 * p + 1];
            st->unit_use[st->unit_off[a] + fu[a]++] = c;
        }
        free(fl); free(fr); free(fu);
    }

    for (uint64_t e = 0; e < n_init && !st->oom; e++)
        add(st, init[3 * e], init[3 * e + 1], init[3 * e + 2]);
    for (uint32_t k = 0; k < n_eps && !st->oom; k++)
        for (uint32_t i = 0; i < n && !st->oom; i++) add(st, i, eps[k], i);

    while (st->wl_len && !st->oom) {
        st->wl_len -= 3;
        uint32_t u = st->wl[st->wl_len], A = st->wl[st->wl_len + 1], v = st->wl[st->wl_len + 2];
        st->pops++;
        /* C -> A B : (u,A,v) (v,B,w) gives (u,C,w) */
        for (uint32_t q = st->left_off[A]; q < st->left_off[A + 1]; q++) {
            uint32_t C = st->left_use[q].c, B = st->left_use[q].other;
            vec32 *lst = &st->out[B][v];
            for (uint32_t t = 0; t < lst->len && !st->oom; t++) {  /* lst may grow */
                st->joins++;
                add(st, u, C, lst->v[t]);
            }
        }
        /* C -> B A : (w,B,u) (u,A,v) gives (w,C,v) */
        for (uint32_t q = st->right_off[A]; q < st->right_off[A + 1]; q++) {
            uint32_t C = st->right_use[q].c, B = st->right_use[q].other;
            vec32 *lst = &st->in[B][u];
            for (uint32_t t = 0; t < lst->len && !st->oom; t++) {
                st->joins++;
                add(st, lst->v[t], C, v);
            }
        }
        /* C -> A : (u,A,v) gives (u,C,v) */
        for (uint32_t q = st->unit_off[A]; q < st->unit_off[A + 1]; q++)
            add(st, u, st->unit_use[q], v);
    }
    if (st->oom) { oracle_free(st); return NULL; }
    return st;
}

uint64_t oracle_count(const oracle_state *st, uint32_t X) {
    return X < st->n_nt ? st->R[X].size : 0;
}

/* Copy the pairs of X as keys (src << 32 | dst), in no particular order. */
uint64_t oracle_keys(const oracle_state *st, uint32_t X, uint64_t *out) {
    if (X >= st->n_nt) return 0;
    uint64_t k = 0;
    const pairset *s = &st->R[X];
    for (uint64_t i = 0; i < s->cap; i++)
        if (s->keys[i] != EMPTY_KEY) out[k++] = s->keys[i];
    return k;
}

uint64_t oracle_pops(const oracle_state *st) { return st->pops; }
uint64_t oracle_joins(const oracle_state *st) { return st->joins; }

void oracle_free(oracle_state *st) {
    if (!st) return;
    for (uint32_t X = 0; X < st->n_nt; X++) {
        if (st->R) free(st->R[X].keys);
        if (st->out && st->out[X]) {
            for (uint32_t i = 0; i < st->n; i++) free(st->out[X][i].v);
            free(st->out[X]);
        }
        if (st->in && st->in[X]) {
            for (uint32_t i = 0; i < st->n; i++) free(st->in[X][i].v);
            free(st->in[X]);
        }
    }
    free(st->R); free(st->out); free(st->in);
    free(st->left_off); free(st->right_off); free(st->unit_off);
    free(st->left_use); free(st->right_use); free(st->unit_use);
    free(st->wl);
    free(st);
}
