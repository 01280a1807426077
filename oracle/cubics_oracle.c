/*
 * CUBICS oracle: a plain, slow, obviously-correct CPU reference for the solver's hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg may load this library.  It shares no code, header, table or helper with the
 * CUDA path: domains here are arrays of byte flags (one byte per value of [lo_i, hi_i]),
 * never bitsets, and all arithmetic is done in int64.
 *
 * What it computes (arxiv 1909.09213):
 *   - the CSP triple (X, D, C) and the notion of solution, Section 1.1;
 *   - the solver's three operations, Section 1.1: domain reduction (assign a variable one
 *     of its values), constraint propagation (remove values that occur in no solution),
 *     backtracking (restore domains at a dead end, record solutions);
 *   - propagation of every constraint to a common fixpoint before each labeling step,
 *     Section 2.1 / 2.2.
 * The paper does not fix the strength of each propagator, the branching heuristic or the
 * node accounting; this file uses the following readings:
 *   ne       x != y + c: when one side is fixed, remove the value it forbids on the other;
 *   lin_le   sum a_i x_i <= b: bounds reasoning with floor/ceil division (mathematical
 *            rounding, not C truncation); repeated variables are merged, zero terms dropped;
 *   alldiff  value elimination from fixed members, failure when two members share a fixed
 *            value or when the union of the domains has fewer values than members;
 *   alldiff_bc  (the stronger propagation of Section 4, second direction) bounds
 *            consistency on the interval relaxation: a bound v of member i stays when the
 *            other members can take pairwise distinct values, all different from v, each
 *            within its own [min, max]; unsupported bounds are removed until all are
 *            supported (holes are kept);
 *   table    full arc consistency on a binary relation;
 *   search   d-way branching on the first-fail variable (smallest domain, ties to the lowest
 *            index), values in ascending order; every fixpoint call is one node, every
 *            failed fixpoint one fail;
 *   hash     h = 0x9E3779B97F4A7C15, then h = splitmix64(h ^ (i << 32 | (u32)value_i)) for
 *            i = 0..n-1; a solution set is summarised by (count, sum of h, xor of h).
 * Parity is pinned by the tests in tests/test_oracle*.py (worked example of Section 1.1,
 * published N-queens counts, brute-force enumeration, fixpoint order-independence).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n;
    const int32_t *lo, *hi;
    int32_t n_ne;
    const int32_t *ne_x, *ne_y, *ne_c;
    int32_t n_lin;
    const int32_t *lin_start, *lin_coef, *lin_var, *lin_rhs;
    int32_t n_ad;
    const int32_t *ad_start, *ad_var;
    int32_t n_tab;
    const int32_t *tab_x, *tab_y;
    const int64_t *tab_off;          /* byte offset of table t's matrix in tab_allowed */
    const uint8_t *tab_allowed;      /* row a - lo_x, column b - lo_y, row-major */
    int32_t n_adb;                   /* bounds-consistent alldifferent groups */
    const int32_t *adb_start, *adb_var;
} oracle_model;

typedef struct {
    int64_t nodes, fails, solutions, stored;
    uint64_t hash_sum, hash_xor;
    int64_t evals[4];                /* propagator evaluations: ne, lin, alldiff, table */
    double work_bytes;               /* algorithmic bytes (FIFO fixpoint, see oracle_solve) */
    int32_t status;                  /* 1 SAT, 0 UNSAT, -5 node limit hit */
    int32_t max_depth;
} oracle_stats;

enum { K_NE = 0, K_LIN = 1, K_AD = 2, K_TAB = 3 };

/* ------------------------------------------------------------------ domains */

typedef struct {
    const oracle_model *m;
    int64_t *off;      /* first flag of variable i */
    int64_t total;     /* number of flags */
} layout;

static void layout_init(layout *L, const oracle_model *m) {
    L->m = m;
    L->off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m->n + 1));
    L->total = 0;
    for (int i = 0; i < m->n; i++) {
        L->off[i] = L->total;
        L->total += (int64_t)m->hi[i] - m->lo[i] + 1;
    }
    L->off[m->n] = L->total;
}

static void layout_free(layout *L) { free(L->off); }

static int64_t dsize(const layout *L, const uint8_t *d, int i) {
    int64_t c = 0;
    for (int64_t k = L->off[i]; k < L->off[i + 1]; k++) c += d[k] != 0;
    return c;
}

static int has(const layout *L, const uint8_t *d, int i, int64_t v) {
    if (v < L->m->lo[i] || v > L->m->hi[i]) return 0;
    return d[L->off[i] + (v - L->m->lo[i])] != 0;
}

/* removes v from D(i); returns 1 if it was there */
static int drop(const layout *L, uint8_t *d, int i, int64_t v) {
    if (!has(L, d, i, v)) return 0;
    d[L->off[i] + (v - L->m->lo[i])] = 0;
    return 1;
}

static int64_t dmin(const layout *L, const uint8_t *d, int i) {
    for (int64_t v = L->m->lo[i]; v <= L->m->hi[i]; v++)
        if (has(L, d, i, v)) return v;
    return INT64_MAX;
}

static int64_t dmax(const layout *L, const uint8_t *d, int i) {
    for (int64_t v = L->m->hi[i]; v >= L->m->lo[i]; v--)
        if (has(L, d, i, v)) return v;
    return INT64_MIN;
}

/* the single value of D(i) when |D(i)| == 1 */
static int fixed_value(const layout *L, const uint8_t *d, int i, int64_t *v) {
    if (dsize(L, d, i) != 1) return 0;
    *v = dmin(L, d, i);
    return 1;
}

/* ------------------------------------------------------------------ propagators
 * Each returns -1 when a domain became empty (failure), 1 when a domain changed, 0 else.
 * `changed` (if not NULL) receives a flag per variable whose domain shrank.            */

static int mark(uint8_t *changed, int i) { if (changed) changed[i] = 1; return 1; }

static int prop_ne(const layout *L, uint8_t *d, int k, uint8_t *changed) {
    const oracle_model *m = L->m;
    int x = m->ne_x[k], y = m->ne_y[k];
    int64_t c = m->ne_c[k], v;
    int ch = 0;
    if (y < 0) {                                     /* x != c */
        if (drop(L, d, x, c)) ch = mark(changed, x);
    } else {
        if (fixed_value(L, d, y, &v) && drop(L, d, x, v + c)) ch = mark(changed, x);
        if (fixed_value(L, d, x, &v) && drop(L, d, y, v - c)) ch = mark(changed, y);
    }
    if (dsize(L, d, x) == 0 || (y >= 0 && dsize(L, d, y) == 0)) return -1;
    return ch;
}

static int64_t floor_div(int64_t q, int64_t a) {
    int64_t t = q / a;
    if ((q % a != 0) && ((q < 0) != (a < 0))) t -= 1;
    return t;
}

static int64_t ceil_div(int64_t q, int64_t a) { return -floor_div(-q, a); }

/* merged coefficient of the first occurrence of term t's variable in row r; 0 for repeats */
static int64_t merged_coef(const oracle_model *m, int r, int t) {
    int v = m->lin_var[t];
    for (int s = m->lin_start[r]; s < t; s++)
        if (m->lin_var[s] == v) return 0;
    int64_t a = 0;
    for (int s = t; s < m->lin_start[r + 1]; s++)
        if (m->lin_var[s] == v) a += m->lin_coef[s];
    return a;
}

static int prop_lin(const layout *L, uint8_t *d, int r, uint8_t *changed) {
    const oracle_model *m = L->m;
    int b0 = m->lin_start[r], b1 = m->lin_start[r + 1];
    int64_t smin = 0;
    for (int t = b0; t < b1; t++) {
        int64_t a = merged_coef(m, r, t);
        if (a == 0) continue;
        int i = m->lin_var[t];
        if (dsize(L, d, i) == 0) return -1;
        smin += a > 0 ? a * dmin(L, d, i) : a * dmax(L, d, i);
    }
    if (smin > m->lin_rhs[r]) return -1;             /* also covers rows with no terms */
    int ch = 0;
    for (int t = b0; t < b1; t++) {
        int64_t a = merged_coef(m, r, t);
        if (a == 0) continue;
        int i = m->lin_var[t];
        int64_t own = a > 0 ? a * dmin(L, d, i) : a * dmax(L, d, i);
        int64_t slack = (int64_t)m->lin_rhs[r] - (smin - own);
        for (int64_t v = m->lo[i]; v <= m->hi[i]; v++) {
            int keep = a > 0 ? v <= floor_div(slack, a) : v >= ceil_div(slack, a);
            if (!keep && drop(L, d, i, v)) ch = mark(changed, i);
        }
        if (dsize(L, d, i) == 0) return -1;
    }
    return ch;
}

static int prop_alldiff(const layout *L, uint8_t *d, int g, uint8_t *changed) {
    const oracle_model *m = L->m;
    int b0 = m->ad_start[g], b1 = m->ad_start[g + 1];
    int ch = 0;
    for (int s = b0; s < b1; s++) {
        int64_t v;
        if (!fixed_value(L, d, m->ad_var[s], &v)) continue;
        for (int t = b0; t < b1; t++) {
            if (t == s) continue;
            int j = m->ad_var[t];
            if (drop(L, d, j, v)) ch = mark(changed, j);
            if (dsize(L, d, j) == 0) return -1;
        }
    }
    /* pigeonhole: the members need k distinct values */
    int64_t lo = INT64_MAX, hi = INT64_MIN;
    for (int s = b0; s < b1; s++) {
        int i = m->ad_var[s];
        if (m->lo[i] < lo) lo = m->lo[i];
        if (m->hi[i] > hi) hi = m->hi[i];
    }
    int64_t uni = 0;
    for (int64_t v = lo; v <= hi; v++) {
        int any = 0;
        for (int s = b0; s < b1; s++) any |= has(L, d, m->ad_var[s], v);
        uni += any;
    }
    if (uni < (int64_t)(b1 - b0)) return -1;
    return ch;
}

/* Augmenting path from member j (Kuhn's bipartite matching): owner[v - base] is the member
 * holding value v, -1 when free, -2 when reserved for the member whose bound is tested. */
static int bc_augment(int j, const int64_t *lo, const int64_t *hi, int64_t base, int32_t *owner,
                      uint8_t *seen) {
    for (int64_t v = lo[j]; v <= hi[j]; v++) {
        int64_t x = v - base;
        if (seen[x] || owner[x] == -2) continue;
        seen[x] = 1;
        if (owner[x] < 0 || bc_augment(owner[x], lo, hi, base, owner, seen)) {
            owner[x] = j;
            return 1;
        }
    }
    return 0;
}

/* v is a supported value for member i: the other k - 1 members can be matched to distinct
 * values other than v inside their intervals (Hall's marriage condition) */
static int bc_supported(int k, const int64_t *lo, const int64_t *hi, int i, int64_t v,
                        int64_t base, int64_t span, int32_t *owner, uint8_t *seen) {
    for (int64_t x = 0; x < span; x++) owner[x] = -1;
    owner[v - base] = -2;
    for (int j = 0; j < k; j++) {
        if (j == i) continue;
        memset(seen, 0, (size_t)span);
        if (!bc_augment(j, lo, hi, base, owner, seen)) return 0;
    }
    return 1;
}

static int prop_alldiff_bc(const layout *L, uint8_t *d, int g, uint8_t *changed) {
    const oracle_model *m = L->m;
    int b0 = m->adb_start[g], b1 = m->adb_start[g + 1], k = b1 - b0;
    if (k == 0) return 0;
    int64_t base = INT64_MAX, top = INT64_MIN;
    for (int s = b0; s < b1; s++) {
        int i = m->adb_var[s];
        if (m->lo[i] < base) base = m->lo[i];
        if (m->hi[i] > top) top = m->hi[i];
    }
    int64_t span = top - base + 1;
    int64_t *lo = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    int64_t *hi = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    int32_t *owner = (int32_t *)malloc(sizeof(int32_t) * (size_t)span);
    uint8_t *seen = (uint8_t *)malloc((size_t)span);
    int ch = 0, res = 0;
    for (int again = 1; again && res == 0;) {
        again = 0;
        for (int s = 0; s < k; s++) {
            int i = m->adb_var[b0 + s];
            if (dsize(L, d, i) == 0) { res = -1; break; }
            lo[s] = dmin(L, d, i);
            hi[s] = dmax(L, d, i);
        }
        for (int s = 0; s < k && res == 0; s++) {
            int i = m->adb_var[b0 + s];
            for (int side = 0; side < 2 && res == 0; side++) {
                for (;;) {
                    if (dsize(L, d, i) == 0) { res = -1; break; }
                    lo[s] = dmin(L, d, i);
                    hi[s] = dmax(L, d, i);
                    int64_t v = side == 0 ? lo[s] : hi[s];
                    if (bc_supported(k, lo, hi, s, v, base, span, owner, seen)) break;
                    drop(L, d, i, v);
                    ch = mark(changed, i);
                    again = 1;
                }
            }
        }
    }
    free(lo); free(hi); free(owner); free(seen);
    return res < 0 ? -1 : ch;
}

static int allowed(const oracle_model *m, int t, int64_t a, int64_t b) {
    int x = m->tab_x[t], y = m->tab_y[t];
    int64_t sy = (int64_t)m->hi[y] - m->lo[y] + 1;
    return m->tab_allowed[m->tab_off[t] + (a - m->lo[x]) * sy + (b - m->lo[y])] != 0;
}

static int prop_table(const layout *L, uint8_t *d, int t, uint8_t *changed) {
    const oracle_model *m = L->m;
    int x = m->tab_x[t], y = m->tab_y[t];
    int ch = 0;
    for (int64_t a = m->lo[x]; a <= m->hi[x]; a++) {
        if (!has(L, d, x, a)) continue;
        int support = 0;
        for (int64_t b = m->lo[y]; b <= m->hi[y] && !support; b++)
            support = has(L, d, y, b) && allowed(m, t, a, b);
        if (!support && drop(L, d, x, a)) ch = mark(changed, x);
    }
    for (int64_t b = m->lo[y]; b <= m->hi[y]; b++) {
        if (!has(L, d, y, b)) continue;
        int support = 0;
        for (int64_t a = m->lo[x]; a <= m->hi[x] && !support; a++)
            support = has(L, d, x, a) && allowed(m, t, a, b);
        if (!support && drop(L, d, y, b)) ch = mark(changed, y);
    }
    if (dsize(L, d, x) == 0 || dsize(L, d, y) == 0) return -1;
    return ch;
}

/* ------------------------------------------------------------------ fixpoints */

static int n_props(const oracle_model *m) {
    return m->n_ne + m->n_lin + m->n_ad + m->n_tab + m->n_adb;
}

/* propagator p in the global numbering ne..., lin..., alldiff..., table..., alldiff_bc...
 * (alldiff_bc evaluations are counted with the alldiff ones) */
static int apply(const layout *L, uint8_t *d, int p, uint8_t *changed, int *kind) {
    const oracle_model *m = L->m;
    if (p < m->n_ne) { *kind = K_NE; return prop_ne(L, d, p, changed); }
    p -= m->n_ne;
    if (p < m->n_lin) { *kind = K_LIN; return prop_lin(L, d, p, changed); }
    p -= m->n_lin;
    if (p < m->n_ad) { *kind = K_AD; return prop_alldiff(L, d, p, changed); }
    p -= m->n_ad;
    if (p < m->n_tab) { *kind = K_TAB; return prop_table(L, d, p, changed); }
    p -= m->n_tab;
    *kind = K_AD;
    return prop_alldiff_bc(L, d, p, changed);
}

static int in_scope(const oracle_model *m, int p, int var) {
    if (p < m->n_ne) return m->ne_x[p] == var || m->ne_y[p] == var;
    p -= m->n_ne;
    if (p < m->n_lin) {
        for (int t = m->lin_start[p]; t < m->lin_start[p + 1]; t++)
            if (m->lin_var[t] == var) return 1;
        return 0;
    }
    p -= m->n_lin;
    if (p < m->n_ad) {
        for (int t = m->ad_start[p]; t < m->ad_start[p + 1]; t++)
            if (m->ad_var[t] == var) return 1;
        return 0;
    }
    p -= m->n_ad;
    if (p < m->n_tab) return m->tab_x[p] == var || m->tab_y[p] == var;
    p -= m->n_tab;
    for (int t = m->adb_start[p]; t < m->adb_start[p + 1]; t++)
        if (m->adb_var[t] == var) return 1;
    return 0;
}

static int any_empty(const layout *L, const uint8_t *d) {
    for (int i = 0; i < L->m->n; i++)
        if (dsize(L, d, i) == 0) return 1;
    return 0;
}

/* variant 0: sweep every propagator in declaration order until a sweep changes nothing */
static int fix_sweep(const layout *L, uint8_t *d, oracle_stats *st) {
    int P = n_props(L->m), kind;
    if (any_empty(L, d)) return 1;
    for (;;) {
        int ch = 0;
        for (int p = 0; p < P; p++) {
            int r = apply(L, d, p, NULL, &kind);
            if (st) st->evals[kind]++;
            if (r < 0) return 1;
            ch |= r;
        }
        if (!ch) return 0;
    }
}

/* tiny xorshift for the random-order variant (test infrastructure only) */
static uint64_t rnd_next(uint64_t *s) {
    uint64_t x = *s;
    x ^= x << 13; x ^= x >> 7; x ^= x << 17;
    *s = x;
    return x;
}

/* variant 2: each sweep visits the propagators in a fresh random order */
static int fix_random(const layout *L, uint8_t *d, uint64_t *rs) {
    int P = n_props(L->m), kind;
    int *ord = (int *)malloc(sizeof(int) * (size_t)(P + 1));
    int res = 0;
    if (any_empty(L, d)) { free(ord); return 1; }
    for (int p = 0; p < P; p++) ord[p] = p;
    for (;;) {
        for (int p = P - 1; p > 0; p--) {
            int q = (int)(rnd_next(rs) % (uint64_t)(p + 1));
            int tmp = ord[p]; ord[p] = ord[q]; ord[q] = tmp;
        }
        int ch = 0;
        for (int p = 0; p < P && res == 0; p++) {
            int r = apply(L, d, ord[p], NULL, &kind);
            if (r < 0) res = 1;
            else ch |= r;
        }
        if (res || !ch) break;
    }
    free(ord);
    return res;
}

/* Algorithmic bytes of one propagator evaluation over W-word bitset domains (the work a
 * bitset implementation must at least move): ne 12 B; table 4 (|D(x)| + 2) per direction;
 * lin 4 W (2k + changed terms); alldiff 4 W 2k.  Sizes are taken before the evaluation. */
static double eval_bytes(const layout *L, const uint8_t *d, int p, int W, int nchanged) {
    const oracle_model *m = L->m;
    if (p < m->n_ne) return 12.0;
    p -= m->n_ne;
    if (p < m->n_lin) {
        int k = m->lin_start[p + 1] - m->lin_start[p];
        return 4.0 * W * (2.0 * k + nchanged);
    }
    p -= m->n_lin;
    if (p < m->n_ad) {
        int k = m->ad_start[p + 1] - m->ad_start[p];
        return 4.0 * W * 2.0 * k;
    }
    p -= m->n_ad;
    if (p < m->n_tab)
        return 4.0 * ((double)dsize(L, d, m->tab_x[p]) + 2.0) + 4.0 * ((double)dsize(L, d, m->tab_y[p]) + 2.0);
    p -= m->n_tab;
    return 4.0 * W * 2.0 * (double)(m->adb_start[p + 1] - m->adb_start[p]);
}

/* variant 1: FIFO queue of propagators woken by the variables whose domain changed.
 * `wake` lists the initially changed variables (NULL = every propagator starts queued). */
static int fix_fifo(const layout *L, uint8_t *d, const uint8_t *wake, oracle_stats *st, int W) {
    const oracle_model *m = L->m;
    int P = n_props(m), kind, res = 0;
    int *q = (int *)malloc(sizeof(int) * (size_t)(P + 1));
    uint8_t *inq = (uint8_t *)calloc((size_t)P + 1, 1);
    uint8_t *chg = (uint8_t *)calloc((size_t)m->n + 1, 1);
    int head = 0, cnt = 0;
    if (any_empty(L, d)) res = 1;
    for (int p = 0; p < P && !res; p++) {
        int woke = wake == NULL;
        for (int i = 0; i < m->n && !woke; i++) woke = wake[i] && in_scope(m, p, i);
        if (woke) { q[(head + cnt) % P] = p; cnt++; inq[p] = 1; }
    }
    while (cnt > 0 && !res) {
        int p = q[head];
        head = (head + 1) % P;
        cnt--;
        inq[p] = 0;
        memset(chg, 0, (size_t)m->n);
        double before = (W > 0 && st) ? eval_bytes(L, d, p, W, 0) : 0.0;
        int r = apply(L, d, p, chg, &kind);
        if (st) {
            st->evals[kind]++;
            if (W > 0) {
                int nch = 0;
                for (int i = 0; i < m->n; i++) nch += chg[i];
                st->work_bytes += before + (kind == K_LIN ? 4.0 * W * nch : 0.0);
            }
        }
        if (r < 0) { res = 1; break; }
        for (int i = 0; i < m->n; i++) {
            if (!chg[i]) continue;
            for (int s = 0; s < P; s++)
                if (!inq[s] && in_scope(m, s, i)) { q[(head + cnt) % P] = s; cnt++; inq[s] = 1; }
        }
    }
    free(q); free(inq); free(chg);
    return res;
}

/* ------------------------------------------------------------------ hashing */

uint64_t oracle_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t oracle_solution_hash(int32_t n, const int32_t *values) {
    uint64_t h = 0x9E3779B97F4A7C15ull;
    for (int i = 0; i < n; i++)
        h = oracle_splitmix64(h ^ (((uint64_t)(uint32_t)i << 32) | (uint64_t)(uint32_t)values[i]));
    return h;
}

/* ------------------------------------------------------------------ search */

typedef struct {
    const layout *L;
    int32_t mode, variant, W;
    int64_t cap, node_limit;
    int32_t *sols;
    oracle_stats *st;
    int stop;
    uint64_t rs;
} search_ctx;

static int fixpoint(search_ctx *c, uint8_t *d, const uint8_t *wake) {
    switch (c->variant) {
    case 1: return fix_fifo(c->L, d, wake, c->st, c->W);
    case 2: return fix_random(c->L, d, &c->rs);
    default: return fix_sweep(c->L, d, c->st);
    }
}

static void record(search_ctx *c, const uint8_t *d) {
    const layout *L = c->L;
    int n = L->m->n;
    int32_t *vals = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    for (int i = 0; i < n; i++) vals[i] = (int32_t)dmin(L, d, i);
    uint64_t h = oracle_solution_hash(n, vals);
    c->st->solutions++;
    c->st->hash_sum += h;
    c->st->hash_xor ^= h;
    if (c->st->stored < c->cap) {
        memcpy(c->sols + c->st->stored * n, vals, sizeof(int32_t) * (size_t)n);
        c->st->stored++;
    }
    free(vals);
    if (c->mode == 1) c->stop = 1;
}

/* one node: propagate d (a fresh copy owned by this call), then label and recurse */
static void node(search_ctx *c, uint8_t *d, const uint8_t *wake, int depth) {
    const layout *L = c->L;
    const oracle_model *m = L->m;
    if (c->node_limit > 0 && c->st->nodes >= c->node_limit) { c->stop = 2; return; }
    c->st->nodes++;
    if (depth > c->st->max_depth) c->st->max_depth = depth;
    if (fixpoint(c, d, wake)) { c->st->fails++; return; }
    int best = -1;
    int64_t bsize = 0;
    for (int i = 0; i < m->n; i++) {                 /* first-fail, lowest index on ties */
        int64_t s = dsize(L, d, i);
        if (s > 1 && (best < 0 || s < bsize)) { best = i; bsize = s; }
    }
    if (best < 0) { record(c, d); return; }
    uint8_t *child = (uint8_t *)malloc((size_t)L->total + 1);
    uint8_t *w = (uint8_t *)calloc((size_t)m->n + 1, 1);
    w[best] = 1;
    for (int64_t v = m->lo[best]; v <= m->hi[best] && !c->stop; v++) {
        if (!has(L, d, best, v)) continue;
        memcpy(child, d, (size_t)L->total);
        for (int64_t u = m->lo[best]; u <= m->hi[best]; u++)
            if (u != v) drop(L, child, best, u);
        node(c, child, w, depth + 1);
    }
    free(child);
    free(w);
}

static uint8_t *initial_domains(const layout *L, const uint8_t *dom0) {
    uint8_t *d = (uint8_t *)malloc((size_t)L->total + 1);
    if (dom0) memcpy(d, dom0, (size_t)L->total);
    else memset(d, 1, (size_t)L->total);
    return d;
}

/*
 * Search from domains dom0 (NULL = the full ranges).  mode 0 counts all solutions, mode 1
 * stops at the first.  Up to `cap` solutions are written to sols (cap * n values).
 * variant selects the fixpoint loop: 0 sweep, 1 FIFO (also accumulates work_bytes with W
 * words per domain when W > 0), 2 random order.  node_limit 0 = none.
 * Returns st->status: 1 SAT, 0 UNSAT, -5 when the node limit stopped the search.
 */
int oracle_solve(const oracle_model *m, const uint8_t *dom0, int32_t mode, int64_t cap,
                 int32_t *sols, int32_t variant, int64_t node_limit, int32_t W,
                 uint64_t seed, oracle_stats *st) {
    layout L;
    layout_init(&L, m);
    memset(st, 0, sizeof(*st));
    search_ctx c = {&L, mode, variant, W, cap, node_limit, sols, st, 0, seed | 1};
    uint8_t *d = initial_domains(&L, dom0);
    node(&c, d, NULL, 0);
    free(d);
    layout_free(&L);
    st->status = c.stop == 2 ? -5 : (st->solutions > 0 ? 1 : 0);
    return st->status;
}

/* one fixpoint from dom (updated in place); returns 1 when failed */
int oracle_propagate(const oracle_model *m, uint8_t *dom, int32_t variant, uint64_t seed,
                     oracle_stats *st) {
    layout L;
    layout_init(&L, m);
    oracle_stats local;
    memset(&local, 0, sizeof(local));
    search_ctx c = {&L, 0, variant, 0, 0, 0, NULL, st ? st : &local, 0, seed | 1};
    int r = fixpoint(&c, dom, NULL);
    layout_free(&L);
    return r;
}

/* ------------------------------------------------------------------ definitions */

/* 1 when `values` satisfies every domain and every constraint's defining relation */
int oracle_check_solution(const oracle_model *m, const uint8_t *dom0, const int32_t *values) {
    layout L;
    layout_init(&L, m);
    int ok = 1;
    for (int i = 0; i < m->n && ok; i++) {
        if (values[i] < m->lo[i] || values[i] > m->hi[i]) ok = 0;
        else if (dom0 && !dom0[L.off[i] + (values[i] - m->lo[i])]) ok = 0;
    }
    for (int k = 0; k < m->n_ne && ok; k++) {
        int64_t rhs = m->ne_y[k] < 0 ? m->ne_c[k] : (int64_t)values[m->ne_y[k]] + m->ne_c[k];
        if ((int64_t)values[m->ne_x[k]] == rhs) ok = 0;
    }
    for (int r = 0; r < m->n_lin && ok; r++) {
        int64_t s = 0;
        for (int t = m->lin_start[r]; t < m->lin_start[r + 1]; t++)
            s += (int64_t)m->lin_coef[t] * values[m->lin_var[t]];
        if (s > m->lin_rhs[r]) ok = 0;
    }
    for (int g = 0; g < m->n_ad && ok; g++)
        for (int s = m->ad_start[g]; s < m->ad_start[g + 1]; s++)
            for (int t = s + 1; t < m->ad_start[g + 1]; t++)
                if (values[m->ad_var[s]] == values[m->ad_var[t]]) ok = 0;
    for (int t = 0; t < m->n_tab && ok; t++)
        if (!allowed(m, t, values[m->tab_x[t]], values[m->tab_y[t]])) ok = 0;
    for (int g = 0; g < m->n_adb && ok; g++)
        for (int s = m->adb_start[g]; s < m->adb_start[g + 1]; s++)
            for (int t = s + 1; t < m->adb_start[g + 1]; t++)
                if (values[m->adb_var[s]] == values[m->adb_var[t]]) ok = 0;
    layout_free(&L);
    return ok;
}

/* Enumerate every assignment of prod D_i (odometer order) and keep those satisfying every
 * relation.  Returns the number of solutions; fills hash sum/xor and up to cap solutions. */
int64_t oracle_brute_force(const oracle_model *m, const uint8_t *dom0, int64_t cap, int32_t *sols,
                           uint64_t *hsum, uint64_t *hxor) {
    int n = m->n;
    int32_t *v = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int64_t count = 0;
    *hsum = 0;
    *hxor = 0;
    for (int i = 0; i < n; i++) v[i] = m->lo[i];
    for (;;) {
        if (oracle_check_solution(m, dom0, v)) {
            uint64_t h = oracle_solution_hash(n, v);
            if (count < cap) memcpy(sols + count * n, v, sizeof(int32_t) * (size_t)n);
            count++;
            *hsum += h;
            *hxor ^= h;
        }
        int i = n - 1;
        while (i >= 0 && v[i] == m->hi[i]) { v[i] = m->lo[i]; i--; }
        if (i < 0) break;
        v[i]++;
    }
    free(v);
    return count;
}
