/*
 * Reference oracle, plain C: the paper's projected transfer matrix modulo one
 * prime p < 2^31 (Sec. 3.1-3.3 for the operators, Sec. 3.5 for the modular
 * arithmetic).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
 * CPU-baseline legs of bench.py.  It shares no code with the CUDA library.
 *
 * Deliberately plain: states are canonical label arrays kept in a hash map
 * (the "standard hashing" alternative the paper mentions in Sec. 3.4, so no
 * ranking is involved), and every per-site factor is applied to each state by
 * running the single-edge operators of the paper in order on a small list of
 * terms:
 *   J_{a,b}  identity if a~b, else join the two blocks, times w;
 *   H_{a,b} = 1 - J_{a,b}                (v = -1);
 *   D_i      make i a singleton;
 *   V_i = -w + D_i                       (v = -1);
 *   P_{a,b}  drop the state if a~b, eq. (projector).
 * Square:     T_i = prod_{j!=i} P V_i H_{i,i+1},  T_m = prod_j P V_m   (T_sq_proj)
 * Triangular: T_i = prod_j P V_i H_{i-1,i} H_{i,i+1}                   (Sec. 3.3)
 * Last row:   T_i^last = prod_{j>i} P D_i H_{i,i+1}, T_m^last = D_m   (T_last_i)
 * Multiplying by w is a shift of the coefficient array; coefficients above
 * w^D are dropped (Sec. 3.5).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXM 24
#define OR_MAXTERMS 64

typedef struct { uint8_t lab[OR_MAXM]; } part_t;

typedef struct { part_t s; int coef; int shift; } term_t;

typedef struct {
    int m, D1;
    size_t cap, n;
    part_t *keys;
    uint8_t *used;
    uint32_t *vals; /* cap * D1 */
} vec_t;

static void canon(part_t *s, int m) {
    int map[256];
    for (int k = 0; k < 256; k++) map[k] = -1;
    int next = 0;
    for (int i = 0; i < m; i++) {
        int x = s->lab[i];
        if (map[x] < 0) map[x] = next++;
        s->lab[i] = (uint8_t)map[x];
    }
}

static uint64_t hash_part(const part_t *s, int m) {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < m; i++) { h ^= s->lab[i]; h *= 1099511628211ull; }
    return h;
}

static int vec_init(vec_t *v, int m, int D1, size_t cap) {
    size_t c = 64;
    while (c < 2 * cap) c <<= 1;
    v->m = m; v->D1 = D1; v->cap = c; v->n = 0;
    v->keys = (part_t *)malloc(c * sizeof(part_t));
    v->used = (uint8_t *)calloc(c, 1);
    v->vals = (uint32_t *)malloc(c * (size_t)D1 * sizeof(uint32_t));
    return (v->keys && v->used && v->vals) ? 0 : -1;
}

static void vec_free(vec_t *v) {
    free(v->keys); free(v->used); free(v->vals);
    v->keys = NULL; v->used = NULL; v->vals = NULL;
}

static uint32_t *vec_slot(vec_t *v, const part_t *s);

static int vec_grow(vec_t *v) {
    vec_t nv;
    if (vec_init(&nv, v->m, v->D1, v->cap)) return -1;
    for (size_t k = 0; k < v->cap; k++) {
        if (!v->used[k]) continue;
        uint32_t *dst = vec_slot(&nv, &v->keys[k]);
        memcpy(dst, v->vals + k * v->D1, v->D1 * sizeof(uint32_t));
    }
    vec_free(v);
    *v = nv;
    return 0;
}

/* Slot of state s, created (zero polynomial) if absent. */
static uint32_t *vec_slot(vec_t *v, const part_t *s) {
    if (2 * (v->n + 1) > v->cap) {
        if (vec_grow(v)) return NULL;
    }
    size_t mask = v->cap - 1, k = hash_part(s, v->m) & mask;
    while (v->used[k]) {
        if (memcmp(v->keys[k].lab, s->lab, v->m) == 0) return v->vals + k * v->D1;
        k = (k + 1) & mask;
    }
    v->used[k] = 1;
    v->keys[k] = *s;
    v->n++;
    uint32_t *p = v->vals + k * v->D1;
    memset(p, 0, v->D1 * sizeof(uint32_t));
    return p;
}

/* ---------------------------------------------------------------- operators */

static void join(part_t *s, int m, int a, int b) {
    uint8_t la = s->lab[a], lb = s->lab[b];
    for (int i = 0; i < m; i++) if (s->lab[i] == lb) s->lab[i] = la;
    canon(s, m);
}

static void detach(part_t *s, int m, int i) {
    s->lab[i] = 255;
    canon(s, m);
}

static int op_H(term_t *t, int n, int m, int a, int b, term_t *out) {
    int k = 0;
    for (int j = 0; j < n; j++) {
        out[k++] = t[j];
        term_t u = t[j];
        u.coef = -u.coef;
        if (u.s.lab[a] != u.s.lab[b]) { join(&u.s, m, a, b); u.shift += 1; }
        out[k++] = u;
    }
    return k;
}

static int op_V(term_t *t, int n, int m, int i, term_t *out) {
    int k = 0;
    for (int j = 0; j < n; j++) {
        term_t u = t[j];
        detach(&u.s, m, i);
        out[k++] = u;
        term_t x = t[j];
        x.coef = -x.coef;
        x.shift += 1;
        out[k++] = x;
    }
    return k;
}

static int op_D(term_t *t, int n, int m, int i, term_t *out) {
    for (int j = 0; j < n; j++) { out[j] = t[j]; detach(&out[j].s, m, i); }
    return n;
}

static int op_P(term_t *t, int n, int a, int b) {
    int k = 0;
    for (int j = 0; j < n; j++) if (t[j].s.lab[a] != t[j].s.lab[b]) t[k++] = t[j];
    return k;
}

/* kind: 0 = square T_i, 1 = triangular T_i, 2 = T_i^last */
static int site_terms(int kind, int m, int i, const part_t *s, term_t *res) {
    term_t a[OR_MAXTERMS], b[OR_MAXTERMS];
    int n = 1;
    a[0].s = *s; a[0].coef = 1; a[0].shift = 0;
    if (kind == 0) {
        if (i < m - 1) { n = op_H(a, n, m, i, i + 1, b); memcpy(a, b, n * sizeof(term_t)); }
        n = op_V(a, n, m, i, b);
        for (int j = 0; j + 1 < m; j++) if (j != i || i == m - 1) n = op_P(b, n, j, j + 1);
    } else if (kind == 1) {
        if (i < m - 1) { n = op_H(a, n, m, i, i + 1, b); memcpy(a, b, n * sizeof(term_t)); }
        if (i > 0) { n = op_H(a, n, m, i - 1, i, b); memcpy(a, b, n * sizeof(term_t)); }
        n = op_V(a, n, m, i, b);
        for (int j = 0; j + 1 < m; j++) n = op_P(b, n, j, j + 1);
    } else {
        if (i < m - 1) { n = op_H(a, n, m, i, i + 1, b); memcpy(a, b, n * sizeof(term_t)); }
        n = op_D(a, n, m, i, b);
        for (int j = i + 1; j + 1 < m; j++) n = op_P(b, n, j, j + 1);
    }
    memcpy(res, b, n * sizeof(term_t));
    return n;
}

static int apply_site(int kind, int m, int i, vec_t *src, vec_t *dst, uint32_t p) {
    int D1 = src->D1;
    term_t terms[OR_MAXTERMS];
    for (size_t k = 0; k < src->cap; k++) {
        if (!src->used[k]) continue;
        const uint32_t *x = src->vals + k * D1;
        int nt = site_terms(kind, m, i, &src->keys[k], terms);
        for (int t = 0; t < nt; t++) {
            if (terms[t].shift >= D1) continue;
            uint32_t *y = vec_slot(dst, &terms[t].s);
            if (!y) return -1;
            uint64_t c = (uint64_t)(((int64_t)terms[t].coef % (int64_t)p + (int64_t)p) % (int64_t)p);
            for (int d = terms[t].shift; d < D1; d++)
                y[d] = (uint32_t)((y[d] + c * x[d - terms[t].shift]) % p);
        }
    }
    return 0;
}

/*
 * P~ of the L x s rectangle modulo p, coefficients w^0..w^D, for every s in
 * heights[] (ascending), out = [n_heights][D+1].  lattice 0 = square,
 * 1 = triangular.  Returns 0, or -1 on bad arguments / allocation failure.
 */
int oracle_ptilde_heights(int lattice, int L, const int *heights, int n_heights,
                          int D, uint32_t p, uint32_t *out) {
    if (L < 1 || L > OR_MAXM || D < 0 || n_heights < 1 || (lattice != 0 && lattice != 1)) return -1;
    int D1 = D + 1;
    vec_t cur, nxt;
    if (vec_init(&cur, L, D1, 16)) return -1;
    part_t e0;
    for (int i = 0; i < L; i++) e0.lab[i] = (uint8_t)i;
    uint32_t *x = vec_slot(&cur, &e0);
    x[0] = 1 % p;
    int h = 1;
    for (int q = 0; q < n_heights; q++) {
        if (heights[q] < h) { vec_free(&cur); return -1; }
        while (h < heights[q]) {
            for (int i = 0; i < L; i++) {
                if (vec_init(&nxt, L, D1, cur.n * 2)) { vec_free(&cur); return -1; }
                if (apply_site(lattice, L, i, &cur, &nxt, p)) { vec_free(&cur); vec_free(&nxt); return -1; }
                vec_free(&cur);
                cur = nxt;
            }
            h++;
        }
        /* read-out on a copy: T_last, then the e0 coefficient */
        vec_t r;
        if (vec_init(&r, L, D1, cur.n)) { vec_free(&cur); return -1; }
        for (size_t k = 0; k < cur.cap; k++)
            if (cur.used[k]) memcpy(vec_slot(&r, &cur.keys[k]), cur.vals + k * D1, D1 * sizeof(uint32_t));
        for (int i = 0; i < L; i++) {
            if (vec_init(&nxt, L, D1, r.n)) { vec_free(&r); vec_free(&cur); return -1; }
            apply_site(2, L, i, &r, &nxt, p);
            vec_free(&r);
            r = nxt;
        }
        uint32_t *y = vec_slot(&r, &e0);
        memcpy(out + (size_t)q * D1, y, D1 * sizeof(uint32_t));
        vec_free(&r);
    }
    vec_free(&cur);
    return 0;
}
