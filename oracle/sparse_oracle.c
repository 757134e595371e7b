/*
 * sparse_oracle.c -- plain, slow, FP64 CPU oracle of the same propagation on
 * a sparse representation: a stabilizer (or an observable) is held as its
 * list of terms lambda * P, the (lambda, string) pairs of Sec. II-B, so that
 * the number of qubits is not limited by a 4^n vector (n <= 32 here).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load this library.  It shares no
 * code, header, table or constant with the CUDA library, nor with
 * pauli_oracle.c: the rules below are restated from the paper on their own, so
 * that agreement with the dense oracle is a check of both.
 *
 * Keys: the base-4 index of Sec. III-B (Example 2), qubit 0 the most
 * significant digit, I, X, Y, Z = 0, 1, 2, 3, in a uint64 (n <= 32).
 *
 * One gate maps every term by the gate's rule on its own letters:
 *   H, S, R_x, R_y, R_z: Table I applied to the one-hot weight vector of the
 *     term's letter on the gate's wire (w = lambda * e_letter);
 *   CX(control, target): the map_CX letter-pair list of Sec. III-C, first
 *     letter = control, the minus sign of XZ <-> YY applied both ways;
 *   the other gates are the same compositions as in the dense oracle:
 *     Z = S S, X = H Z H, Y = Z X, S^dagger = S S S, CZ(a,b) = H_b CX(a,b) H_b;
 *   inverse rotation: (cos, -sin).
 * Images of weight exactly zero are dropped (they contribute nothing).  After
 * a rotation the images are sorted by key and equal keys are summed (at most
 * two images meet, so the order of the sum does not matter); sums that are
 * exactly zero are dropped.  A Clifford gate maps each nonzero term to one
 * nonzero term and distinct strings to distinct strings, so its images need
 * no merge.
 *
 * <0^n| O |0^n> = sum of the coefficients of the strings of I and Z only
 * (Sec. II-A readout), summed in key order.
 *
 * Build: with pauli_oracle.c, gcc -O2 -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint8_t op, q0, q1, flags;
    int32_t param;
} sp_gate;

enum { SP_H = 0, SP_S = 1, SP_SDG = 2, SP_X = 3, SP_Y = 4, SP_Z = 5,
       SP_CX = 6, SP_CZ = 7, SP_RX = 8, SP_RY = 9, SP_RZ = 10, SP_NUM_OPS = 11 };

enum { L_I = 0, L_X = 1, L_Y = 2, L_Z = 3 };

typedef struct {
    int64_t len, cap;
    uint64_t *key;
    double *val;
} term_list;

/* letter of qubit q (qubit 0 = most significant base-4 digit) */
static int letter(uint64_t key, int n, int q) {
    return (int)((key >> (2 * (n - 1 - q))) & 3u);
}

static uint64_t with_letter(uint64_t key, int n, int q, int a) {
    const int sh = 2 * (n - 1 - q);
    return (key & ~((uint64_t)3u << sh)) | ((uint64_t)a << sh);
}

static int reserve(term_list *t, int64_t need) {
    if (need <= t->cap) return 0;
    int64_t cap = t->cap ? t->cap : 16;
    while (cap < need) cap *= 2;
    uint64_t *k = (uint64_t *)realloc(t->key, (size_t)cap * sizeof(uint64_t));
    if (!k) return -1;
    t->key = k;
    double *v = (double *)realloc(t->val, (size_t)cap * sizeof(double));
    if (!v) return -1;
    t->val = v;
    t->cap = cap;
    return 0;
}

static int push(term_list *t, uint64_t k, double v) {
    if (reserve(t, t->len + 1)) return -1;
    t->key[t->len] = k;
    t->val[t->len] = v;
    t->len++;
    return 0;
}

/* ---------------- sort by key, sum equal keys, drop exact zeros ---------------- */

typedef struct {
    uint64_t k;
    double v;
} kv;

static int kv_cmp(const void *a, const void *b) {
    const uint64_t x = ((const kv *)a)->k, y = ((const kv *)b)->k;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static int merge(term_list *t) {
    if (t->len == 0) return 0;
    kv *tmp = (kv *)malloc((size_t)t->len * sizeof(kv));
    if (!tmp) return -1;
    for (int64_t i = 0; i < t->len; ++i) {
        tmp[i].k = t->key[i];
        tmp[i].v = t->val[i];
    }
    qsort(tmp, (size_t)t->len, sizeof(kv), kv_cmp);
    int64_t out = 0;
    for (int64_t i = 0; i < t->len;) {
        int64_t j = i;
        double acc = 0.0;
        while (j < t->len && tmp[j].k == tmp[i].k) acc += tmp[j++].v;
        if (acc != 0.0) {
            t->key[out] = tmp[i].k;
            t->val[out] = acc;
            out++;
        }
        i = j;
    }
    t->len = out;
    free(tmp);
    return 0;
}

/* ---------------- Table I on one term ---------------- */

enum { ROW_H, ROW_S, ROW_RX, ROW_RY, ROW_RZ };

/* Table I rows on w = [w_I, w_X, w_Y, w_Z]; c = cos(theta), s = sin(theta). */
static void row_image(int row, double c, double s, const double w[4], double o[4]) {
    o[0] = w[0];
    switch (row) {
    case ROW_H:  o[1] = w[3]; o[2] = -w[2]; o[3] = w[1]; break;
    case ROW_S:  o[1] = -w[2]; o[2] = w[1]; o[3] = w[3]; break;
    case ROW_RX: o[1] = w[1]; o[2] = w[2] * c - w[3] * s; o[3] = w[2] * s + w[3] * c; break;
    case ROW_RY: o[1] = w[1] * c + w[3] * s; o[2] = w[2]; o[3] = w[3] * c - w[1] * s; break;
    case ROW_RZ: o[1] = w[1] * c - w[2] * s; o[2] = w[2] * c + w[1] * s; o[3] = w[3]; break;
    }
}

/*
 * One Table I row on wire q over the list.  A term lambda * P with letter a
 * on wire q has weight vector lambda * e_a there; each nonzero image weight b
 * gives the term with letter b.  Only a rotation can give two images.
 */
static int apply_row(term_list *t, int n, int q, int row, double c, double s) {
    term_list out = {0, 0, NULL, NULL};
    for (int64_t i = 0; i < t->len; ++i) {
        double w[4] = {0.0, 0.0, 0.0, 0.0}, o[4];
        const int a = letter(t->key[i], n, q);
        w[a] = t->val[i];
        row_image(row, c, s, w, o);
        for (int b = 0; b < 4; ++b) {
            /* images of weight exactly zero contribute nothing */
            if (o[b] == 0.0) continue;
            if (push(&out, with_letter(t->key[i], n, q, b), o[b])) return -1;
        }
    }
    free(t->key);
    free(t->val);
    *t = out;
    if (row == ROW_RX || row == ROW_RY || row == ROW_RZ) return merge(t);
    return 0;
}

/* ---------------- CX letter pairs (Sec. III-C) ---------------- */

/* (control, target) letters -> image letters and sign, as listed in the paper. */
static void cx_image(int a, int b, int *a2, int *b2, double *sg) {
    static const struct { char in[3]; char out[4]; } list[16] = {
        {"II", "II"}, {"IX", "IX"}, {"ZI", "ZI"}, {"ZX", "ZX"},
        {"XI", "XX"}, {"XX", "XI"}, {"IY", "ZY"}, {"ZY", "IY"},
        {"YI", "YX"}, {"YX", "YI"}, {"IZ", "ZZ"}, {"ZZ", "IZ"},
        {"XY", "YZ"}, {"YZ", "XY"}, {"XZ", "-YY"}, {"YY", "-XZ"},
    };
    static const char letters[] = "IXYZ";
    for (int r = 0; r < 16; ++r) {
        if (list[r].in[0] != letters[a] || list[r].in[1] != letters[b]) continue;
        const char *img = list[r].out;
        *sg = 1.0;
        if (*img == '-') { *sg = -1.0; ++img; }
        *a2 = (int)(strchr(letters, img[0]) - letters);
        *b2 = (int)(strchr(letters, img[1]) - letters);
        return;
    }
}

static void apply_cx(term_list *t, int n, int c, int tq) {
    for (int64_t i = 0; i < t->len; ++i) {
        int a2, b2;
        double sg;
        cx_image(letter(t->key[i], n, c), letter(t->key[i], n, tq), &a2, &b2, &sg);
        t->key[i] = with_letter(with_letter(t->key[i], n, c, a2), n, tq, b2);
        t->val[i] *= sg;
    }
}

/* ---------------- gates ---------------- */

static int apply_gate(term_list *t, int n, const sp_gate *g, double c, double s, int inverse) {
    const int q = g->q0;
    int rc = 0;
    switch (g->op) {
    case SP_H: rc = apply_row(t, n, q, ROW_H, 0, 0); break;
    case SP_S:
    case SP_SDG: {
        /* S once, or S^dagger = S S S; inversion swaps the two */
        const int times = ((g->op == SP_S) != (inverse != 0)) ? 1 : 3;
        for (int r = 0; r < times && !rc; ++r) rc = apply_row(t, n, q, ROW_S, 0, 0);
        break;
    }
    case SP_Z:
        rc = apply_row(t, n, q, ROW_S, 0, 0);
        if (!rc) rc = apply_row(t, n, q, ROW_S, 0, 0);
        break;
    case SP_X: {
        const sp_gate z = {SP_Z, g->q0, 0, 0, -1};
        rc = apply_row(t, n, q, ROW_H, 0, 0);
        if (!rc) rc = apply_gate(t, n, &z, 0, 0, 0);
        if (!rc) rc = apply_row(t, n, q, ROW_H, 0, 0);
        break;
    }
    case SP_Y: {
        const sp_gate x = {SP_X, g->q0, 0, 0, -1}, z = {SP_Z, g->q0, 0, 0, -1};
        rc = apply_gate(t, n, &x, 0, 0, 0);
        if (!rc) rc = apply_gate(t, n, &z, 0, 0, 0);
        break;
    }
    case SP_CX: apply_cx(t, n, g->q0, g->q1); break;
    case SP_CZ:
        rc = apply_row(t, n, g->q1, ROW_H, 0, 0);
        if (!rc) apply_cx(t, n, g->q0, g->q1);
        if (!rc) rc = apply_row(t, n, g->q1, ROW_H, 0, 0);
        break;
    case SP_RX: rc = apply_row(t, n, q, ROW_RX, c, inverse ? -s : s); break;
    case SP_RY: rc = apply_row(t, n, q, ROW_RY, c, inverse ? -s : s); break;
    case SP_RZ: rc = apply_row(t, n, q, ROW_RZ, c, inverse ? -s : s); break;
    }
    return rc;
}

static int valid(int n, int64_t m, const sp_gate *gates, int64_t n_params) {
    if (n < 1 || n > 32 || m < 0) return 0;
    for (int64_t i = 0; i < m; ++i) {
        const sp_gate *g = &gates[i];
        if (g->op >= SP_NUM_OPS || g->q0 >= n) return 0;
        if ((g->op == SP_CX || g->op == SP_CZ) && (g->q1 >= n || g->q1 == g->q0)) return 0;
        if (g->op >= SP_RX && (g->param < 0 || g->param >= n_params)) return 0;
    }
    return 1;
}

/*
 * Propagates the list (keys_in, vals_in) through the circuit: forward
 * (P -> U P U^dagger, gates in order) or, with backward != 0, backward
 * (P -> U^dagger P U, reverse order, inverse gates).  The result is written in
 * key order.  Returns 0; -1 for an invalid circuit or n; -2 when the result
 * has more than cap_out terms (n_out then holds the count); -3 out of memory.
 */
int orc_sparse_propagate(int n, int64_t m, const sp_gate *gates, const double *thetas,
                         int64_t n_params, int backward, int64_t n_in, const uint64_t *keys_in,
                         const double *vals_in, int64_t cap_out, uint64_t *keys_out,
                         double *vals_out, int64_t *n_out) {
    if (!valid(n, m, gates, n_params) || n_in < 0) return -1;
    const uint64_t lim = n == 32 ? ~(uint64_t)0 : (((uint64_t)1 << (2 * n)) - 1);
    term_list t = {0, 0, NULL, NULL};
    for (int64_t i = 0; i < n_in; ++i) {
        if (keys_in[i] > lim) return -1;
        if (push(&t, keys_in[i], vals_in[i])) return -3;
    }
    int rc = merge(&t);
    for (int64_t k = 0; k < m && !rc; ++k) {
        const int64_t i = backward ? m - 1 - k : k;
        const sp_gate *g = &gates[i];
        double c = 0.0, s = 0.0;
        if (g->op >= SP_RX) {
            c = cos(thetas[g->param]);
            s = sin(thetas[g->param]);
        }
        rc = apply_gate(&t, n, g, c, s, backward);
    }
    if (!rc) rc = merge(&t);
    if (rc) {
        free(t.key);
        free(t.val);
        return -3;
    }
    *n_out = t.len;
    if (t.len > cap_out) rc = -2;
    else
        for (int64_t i = 0; i < t.len; ++i) {
            keys_out[i] = t.key[i];
            vals_out[i] = t.val[i];
        }
    free(t.key);
    free(t.val);
    return rc;
}

/* Sum of the coefficients of the strings made of I and Z only, in list order. */
double orc_sparse_sum_xfree(int n, int64_t len, const uint64_t *keys, const double *vals) {
    double acc = 0.0;
    for (int64_t i = 0; i < len; ++i) {
        int xfree = 1;
        for (int q = 0; q < n; ++q) {
            const int a = letter(keys[i], n, q);
            if (a == L_X || a == L_Y) xfree = 0;
        }
        if (xfree) acc += vals[i];
    }
    return acc;
}

/* <0^n| U^dagger O U |0^n> by backward propagation of O's terms. */
int orc_sparse_expect(int n, int64_t m, const sp_gate *gates, const double *thetas,
                      int64_t n_params, int64_t n_terms, const uint64_t *keys,
                      const double *vals, double *out) {
    if (!valid(n, m, gates, n_params) || n_terms < 0) return -1;
    const uint64_t lim = n == 32 ? ~(uint64_t)0 : (((uint64_t)1 << (2 * n)) - 1);
    term_list t = {0, 0, NULL, NULL};
    for (int64_t i = 0; i < n_terms; ++i) {
        if (keys[i] > lim) return -1;
        if (push(&t, keys[i], vals[i])) return -3;
    }
    int rc = merge(&t);
    for (int64_t k = m - 1; k >= 0 && !rc; --k) {
        const sp_gate *g = &gates[k];
        double c = 0.0, s = 0.0;
        if (g->op >= SP_RX) {
            c = cos(thetas[g->param]);
            s = sin(thetas[g->param]);
        }
        rc = apply_gate(&t, n, g, c, s, 1);
    }
    if (!rc) rc = merge(&t);
    if (!rc) *out = orc_sparse_sum_xfree(n, t.len, t.key, t.val);
    free(t.key);
    free(t.val);
    return rc ? -3 : 0;
}
