/*
 * pauli_oracle.c -- plain, slow, FP64 CPU oracle for the Pauli-coefficient
 * propagation of arXiv 2502.10685 ("Parallelizing the stabilizer formalism for
 * quantum machine learning applications").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load this library.  It shares no
 * code, header, table or constant with the CUDA library and includes none of
 * its files; the gate-record layout below is the public interface restated.
 *
 * What it computes (Sec. II-A, Eq. (1)): the stabilizer generators of |0^n>
 * are Z_k = I^(k) Z I^(n-k-1); a circuit g_1..g_m maps each to
 * U Z_k U^dagger with U = g_m ... g_1, applied one gate at a time.  Each
 * generator is held as the dense vector of its 4^n Pauli coefficients.
 *
 * Encoding (Sec. III-B, Example 2): the string p_0 p_1 ... p_{n-1} has index
 * sum_j d_j 4^(n-1-j) with I=0, X=1, Y=2, Z=3; qubit 0 is the most significant
 * base-4 digit ("XYZ" -> 27).
 *
 * Gate rules, applied literally:
 *   H, S, R_x, R_y, R_z: the rows of Table I on w = [w0,w1,w2,w3], the
 *     coefficients of I, X, Y, Z on the gate's wire.
 *   CX(control, target): the letter-pair list of Sec. III-C (map_CX), first
 *     letter = control, with the minus sign on XZ <-> YY applied both ways.
 *   Gates the paper does not list are compositions of those rules, each an
 *   identity of conjugation maps (global phases cancel in g P g^dagger):
 *     Z = S S,  X = H Z H,  Y = Z X (X first),  S^dagger = S S S,
 *     CZ(a,b) = H_b CX(a,b) H_b.
 *   Inverse rotation: R(theta)^-1 = R(-theta), i.e. (cos, -sin).
 * Observables evolve backward (U^dagger O U): reverse gate order, inverse
 * gates.  <0^n| O |0^n> is the sum of the coefficients of the strings made of
 * I and Z only (Sec. II-A readout, <0|I|0> = <0|Z|0> = 1, <0|X|0> = <0|Y|0> = 0).
 * Parameter-shift gradient (Sec. I, 2m evaluations): each gate that reads
 * slot j contributes (f(theta_g + pi/2) - f(theta_g - pi/2)) / 2.
 * flatten()/expand (Eq. (5), Examples 3 and 4): each term's n x 4 weight
 * rows are Kronecker-multiplied (qubit 0 outermost) and the terms summed.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so the
 * arithmetic is exactly the sequence written here).  Sums are sequential.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Gate record: the public 8-byte layout {u8 op, u8 q0, u8 q1, u8 flags, i32 param}. */
typedef struct {
    uint8_t op, q0, q1, flags;
    int32_t param;
} orc_gate;

/* Opcodes of the public interface, restated. */
enum {
    ORC_H = 0, ORC_S = 1, ORC_SDG = 2, ORC_X = 3, ORC_Y = 4, ORC_Z = 5,
    ORC_CX = 6, ORC_CZ = 7, ORC_RX = 8, ORC_RY = 9, ORC_RZ = 10,
    ORC_NUM_OPS = 11
};

/* Table I rows. */
enum { ROW_H, ROW_S, ROW_RX, ROW_RY, ROW_RZ };

#define ORC_OK 0
#define ORC_EINVAL (-1)

static int64_t pow4(int k) { return (int64_t)1 << (2 * k); }

/* base-4 digit of qubit q in index idx (qubit 0 most significant) */
static int digit(int64_t idx, int n, int q) {
    return (int)((idx / pow4(n - 1 - q)) % 4);
}

/* ---------------- encoding (Sec. III-B) ---------------- */

static int letter_value(char ch) {
    switch (ch) {
    case 'I': return 0;
    case 'X': return 1;
    case 'Y': return 2;
    case 'Z': return 3;
    default: return -1;
    }
}

/* stringToIndex(): "XYZ" -> 1*16 + 2*4 + 3 = 27.  Returns -1 on a bad letter. */
int64_t orc_string_to_index(const char *s) {
    int64_t idx = 0;
    for (const char *p = s; *p; ++p) {
        int d = letter_value(*p);
        if (d < 0) return -1;
        idx = idx * 4 + d;
    }
    return idx;
}

/* indexToString(): needs n; writes n letters and a terminating NUL. */
void orc_index_to_string(int n, int64_t idx, char *out) {
    static const char letters[4] = {'I', 'X', 'Y', 'Z'};
    for (int q = 0; q < n; ++q) out[q] = letters[digit(idx, n, q)];
    out[n] = '\0';
}

/* ---------------- Table I ---------------- */

/* One row of Table I applied to w = [w0, w1, w2, w3]; c = cos(theta), s = sin(theta). */
static void table1_row(int row, double c, double s, const double w[4], double out[4]) {
    switch (row) {
    case ROW_H:  /* [w0, w3, -w2, w1] */
        out[0] = w[0]; out[1] = w[3]; out[2] = -w[2]; out[3] = w[1];
        break;
    case ROW_S:  /* [w0, -w2, w1, w3] */
        out[0] = w[0]; out[1] = -w[2]; out[2] = w[1]; out[3] = w[3];
        break;
    case ROW_RX: /* [w0, w1, w2 c - w3 s, w2 s + w3 c] */
        out[0] = w[0]; out[1] = w[1];
        out[2] = w[2] * c - w[3] * s;
        out[3] = w[2] * s + w[3] * c;
        break;
    case ROW_RY: /* [w0, w1 c + w3 s, w2, w3 c - w1 s] */
        out[0] = w[0];
        out[1] = w[1] * c + w[3] * s;
        out[2] = w[2];
        out[3] = w[3] * c - w[1] * s;
        break;
    case ROW_RZ: /* [w0, w1 c - w2 s, w2 c + w1 s, w3] */
        out[0] = w[0];
        out[1] = w[1] * c - w[2] * s;
        out[2] = w[2] * c + w[1] * s;
        out[3] = w[3];
        break;
    }
}

/* map_non-CX of one gate on wire q over the whole dense vector. */
static void apply_row(int n, int q, int row, double c, double s, double *v) {
    int64_t stride = pow4(n - 1 - q);
    int64_t N = pow4(n);
    for (int64_t i = 0; i < N; ++i) {
        if (digit(i, n, q) != 0) continue;
        double w[4], o[4];
        for (int a = 0; a < 4; ++a) w[a] = v[i + a * stride];
        table1_row(row, c, s, w, o);
        for (int a = 0; a < 4; ++a) v[i + a * stride] = o[a];
    }
}

/* ---------------- CX rule list (Sec. III-C) ---------------- */

/* Letter pairs (control, target) -> image, as printed; '-' marks the sign. */
static const char *const cx_rules[16] = {
    "II>II", "IX>IX", "ZI>ZI", "ZX>ZX",
    "XI>XX", "XX>XI", "IY>ZY", "ZY>IY",
    "YI>YX", "YX>YI", "IZ>ZZ", "ZZ>IZ",
    "XY>YZ", "YZ>XY", "XZ>-YY", "YY>-XZ",
};

static int cx_dst[4][4][2];
static double cx_sign[4][4];
static int cx_ready = 0;

static void cx_build(void) {
    if (cx_ready) return;
    for (int r = 0; r < 16; ++r) {
        const char *rule = cx_rules[r];
        int a = letter_value(rule[0]), b = letter_value(rule[1]);
        const char *img = rule + 3;
        double sg = 1.0;
        if (*img == '-') { sg = -1.0; ++img; }
        cx_dst[a][b][0] = letter_value(img[0]);
        cx_dst[a][b][1] = letter_value(img[1]);
        cx_sign[a][b] = sg;
    }
    cx_ready = 1;
}

/* map_CX over the whole vector; tmp is scratch of 4^n doubles. */
static void apply_cx(int n, int c, int t, double *v, double *tmp) {
    cx_build();
    int64_t N = pow4(n);
    int64_t sc = pow4(n - 1 - c), st = pow4(n - 1 - t);
    for (int64_t i = 0; i < N; ++i) tmp[i] = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        int a = digit(i, n, c), b = digit(i, n, t);
        int64_t j = i - a * sc - b * st + cx_dst[a][b][0] * sc + cx_dst[a][b][1] * st;
        tmp[j] = cx_sign[a][b] * v[i];
    }
    memcpy(v, tmp, (size_t)N * sizeof(double));
}

/* ---------------- gates ---------------- */

static int valid_gate(int n, const orc_gate *g, int64_t n_params) {
    if (g->op >= ORC_NUM_OPS) return 0;
    if (g->q0 >= n) return 0;
    if (g->op == ORC_CX || g->op == ORC_CZ) {
        if (g->q1 >= n || g->q1 == g->q0) return 0;
    }
    if (g->op >= ORC_RX) {
        if (g->param < 0 || g->param >= n_params) return 0;
    }
    return 1;
}

/*
 * Conjugation by one gate (forward map P -> g P g^dagger), or by its inverse
 * when inverse != 0.  c, s are cos/sin of the rotation angle (ignored for
 * Clifford gates).
 */
void orc_apply_gate_cs(int n, int op, int q0, int q1, double c, double s, int inverse,
                       double *v, double *tmp) {
    switch (op) {
    case ORC_H: apply_row(n, q0, ROW_H, 0, 0, v); break;
    case ORC_S:   /* S, or S^dagger = S S S when inverted */
        for (int r = 0; r < (inverse ? 3 : 1); ++r) apply_row(n, q0, ROW_S, 0, 0, v);
        break;
    case ORC_SDG: /* S^dagger = S S S, or S when inverted */
        for (int r = 0; r < (inverse ? 1 : 3); ++r) apply_row(n, q0, ROW_S, 0, 0, v);
        break;
    case ORC_Z:
        apply_row(n, q0, ROW_S, 0, 0, v); apply_row(n, q0, ROW_S, 0, 0, v);
        break;
    case ORC_X:
        apply_row(n, q0, ROW_H, 0, 0, v);
        apply_row(n, q0, ROW_S, 0, 0, v); apply_row(n, q0, ROW_S, 0, 0, v);
        apply_row(n, q0, ROW_H, 0, 0, v);
        break;
    case ORC_Y:
        orc_apply_gate_cs(n, ORC_X, q0, 0, 0, 0, 0, v, tmp);
        orc_apply_gate_cs(n, ORC_Z, q0, 0, 0, 0, 0, v, tmp);
        break;
    case ORC_CX: apply_cx(n, q0, q1, v, tmp); break;
    case ORC_CZ:
        apply_row(n, q1, ROW_H, 0, 0, v);
        apply_cx(n, q0, q1, v, tmp);
        apply_row(n, q1, ROW_H, 0, 0, v);
        break;
    case ORC_RX: apply_row(n, q0, ROW_RX, c, inverse ? -s : s, v); break;
    case ORC_RY: apply_row(n, q0, ROW_RY, c, inverse ? -s : s, v); break;
    case ORC_RZ: apply_row(n, q0, ROW_RZ, c, inverse ? -s : s, v); break;
    }
}

static void gate_cs(const orc_gate *g, const double *thetas, double shift, double *c, double *s) {
    *c = 0.0; *s = 0.0;
    if (g->op >= ORC_RX) {
        double th = thetas[g->param] + shift;
        *c = cos(th);
        *s = sin(th);
    }
}

/* Validate a gate list; returns ORC_OK or ORC_EINVAL. */
int orc_validate(int n, int64_t m, const orc_gate *gates, int64_t n_params) {
    if (n < 1 || n > 12 || m < 0) return ORC_EINVAL;
    for (int64_t i = 0; i < m; ++i)
        if (!valid_gate(n, &gates[i], n_params)) return ORC_EINVAL;
    return ORC_OK;
}

/*
 * Forward propagation (Eq. (1)): v <- U v U^dagger gate by gate, in order.
 * shift_gate >= 0 adds `shift` to that one gate's angle (parameter shift).
 */
static int forward_impl(int n, int64_t m, const orc_gate *gates, const double *thetas,
                        int64_t n_params, int64_t shift_gate, double shift, double *v) {
    if (orc_validate(n, m, gates, n_params) != ORC_OK) return ORC_EINVAL;
    double *tmp = (double *)malloc((size_t)pow4(n) * sizeof(double));
    if (!tmp) return ORC_EINVAL;
    for (int64_t i = 0; i < m; ++i) {
        double c, s;
        gate_cs(&gates[i], thetas, i == shift_gate ? shift : 0.0, &c, &s);
        orc_apply_gate_cs(n, gates[i].op, gates[i].q0, gates[i].q1, c, s, 0, v, tmp);
    }
    free(tmp);
    return ORC_OK;
}

/* Backward propagation: v <- U^dagger v U (reverse order, inverse gates). */
static int backward_impl(int n, int64_t m, const orc_gate *gates, const double *thetas,
                         int64_t n_params, int64_t shift_gate, double shift, double *v) {
    if (orc_validate(n, m, gates, n_params) != ORC_OK) return ORC_EINVAL;
    double *tmp = (double *)malloc((size_t)pow4(n) * sizeof(double));
    if (!tmp) return ORC_EINVAL;
    for (int64_t i = m - 1; i >= 0; --i) {
        double c, s;
        gate_cs(&gates[i], thetas, i == shift_gate ? shift : 0.0, &c, &s);
        orc_apply_gate_cs(n, gates[i].op, gates[i].q0, gates[i].q1, c, s, 1, v, tmp);
    }
    free(tmp);
    return ORC_OK;
}

int orc_forward(int n, int64_t m, const orc_gate *gates, const double *thetas, int64_t n_params,
                double *v) {
    return forward_impl(n, m, gates, thetas, n_params, -1, 0.0, v);
}

int orc_backward(int n, int64_t m, const orc_gate *gates, const double *thetas, int64_t n_params,
                 double *v) {
    return backward_impl(n, m, gates, thetas, n_params, -1, 0.0, v);
}

/* Generator Z_k of |0^n> (Eq. (1)): coefficient 1 at the string I..Z..I. */
void orc_init_generator(int n, int k, double *v) {
    int64_t N = pow4(n);
    for (int64_t i = 0; i < N; ++i) v[i] = 0.0;
    v[3 * pow4(n - 1 - k)] = 1.0;
}

/* All n evolved generators, out = n x 4^n. */
int orc_generators(int n, int64_t m, const orc_gate *gates, const double *thetas,
                   int64_t n_params, double *out) {
    int64_t N = pow4(n);
    for (int k = 0; k < n; ++k) {
        orc_init_generator(n, k, out + k * N);
        int rc = orc_forward(n, m, gates, thetas, n_params, out + k * N);
        if (rc != ORC_OK) return rc;
    }
    return ORC_OK;
}

/* <0^n| P |0^n> summed with weights v: the strings with digits in {I, Z} only. */
double orc_sum_xfree(int n, const double *v) {
    int64_t N = pow4(n);
    double acc = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        int ok = 1;
        for (int q = 0; q < n; ++q) {
            int d = digit(i, n, q);
            if (d == 1 || d == 2) { ok = 0; break; }
        }
        if (ok) acc += v[i];
    }
    return acc;
}

static int expect_impl(int n, int64_t m, const orc_gate *gates, const double *thetas,
                       int64_t n_params, const double *O, int64_t shift_gate, double shift,
                       double *out) {
    int64_t N = pow4(n);
    double *v = (double *)malloc((size_t)N * sizeof(double));
    if (!v) return ORC_EINVAL;
    memcpy(v, O, (size_t)N * sizeof(double));
    int rc = backward_impl(n, m, gates, thetas, n_params, shift_gate, shift, v);
    if (rc == ORC_OK) *out = orc_sum_xfree(n, v);
    free(v);
    return rc;
}

/* <0^n| U^dagger O U |0^n>, O given as a dense 4^n coefficient vector. */
int orc_expect(int n, int64_t m, const orc_gate *gates, const double *thetas, int64_t n_params,
               const double *O, double *out) {
    return expect_impl(n, m, gates, thetas, n_params, O, -1, 0.0, out);
}

/* Parameter-shift gradient d<O>/d theta_j for every slot j (Sec. I). */
int orc_psr_grad(int n, int64_t m, const orc_gate *gates, const double *thetas, int64_t n_params,
                 const double *O, double *grads) {
    const double half_pi = 1.5707963267948966;
    if (orc_validate(n, m, gates, n_params) != ORC_OK) return ORC_EINVAL;
    for (int64_t j = 0; j < n_params; ++j) grads[j] = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        if (gates[i].op < ORC_RX) continue;
        double fp, fm;
        int rc = expect_impl(n, m, gates, thetas, n_params, O, i, half_pi, &fp);
        if (rc == ORC_OK) rc = expect_impl(n, m, gates, thetas, n_params, O, i, -half_pi, &fm);
        if (rc != ORC_OK) return rc;
        grads[gates[i].param] += (fp - fm) / 2.0;
    }
    return ORC_OK;
}

/* Gradient of the single gate occurrence i (used to sample large cases). */
int orc_psr_grad_gate(int n, int64_t m, const orc_gate *gates, const double *thetas,
                      int64_t n_params, const double *O, int64_t i, double *grad) {
    const double half_pi = 1.5707963267948966;
    if (i < 0 || i >= m || gates[i].op < ORC_RX) return ORC_EINVAL;
    double fp, fm;
    int rc = expect_impl(n, m, gates, thetas, n_params, O, i, half_pi, &fp);
    if (rc == ORC_OK) rc = expect_impl(n, m, gates, thetas, n_params, O, i, -half_pi, &fm);
    if (rc == ORC_OK) *grad = (fp - fm) / 2.0;
    return rc;
}

/*
 * flatten()/expand of Eq. (5): W holds n_terms x n x 4 weights; out (4^n) is
 * the sum over terms of the Kronecker product of the term's n rows, qubit 0
 * outermost, so out[sum_j d_j 4^(n-1-j)] += prod_j W[t][j][d_j].
 */
void orc_expand(int n, int n_terms, const double *W, double *out) {
    int64_t N = pow4(n);
    for (int64_t i = 0; i < N; ++i) out[i] = 0.0;
    for (int t = 0; t < n_terms; ++t) {
        for (int64_t i = 0; i < N; ++i) {
            double p = 1.0;
            for (int q = 0; q < n; ++q) p *= W[((int64_t)t * n + q) * 4 + digit(i, n, q)];
            out[i] += p;
        }
    }
}

/* map_non-CX of one Table I row on a single weight vector w (Eq. (4)). */
void orc_map_noncx(int op, double c, double s, const double w[4], double out[4]) {
    int row = op == ORC_H ? ROW_H : op == ORC_S ? ROW_S : op == ORC_RX ? ROW_RX
            : op == ORC_RY ? ROW_RY : ROW_RZ;
    table1_row(row, c, s, w, out);
}

int orc_num_ops(void) { return ORC_NUM_OPS; }

/* ---------------- density matrix (Sec. III-D decoding, Sec. IV-C, Eq. (3)) ----------------
 *
 * rho = 2^-n sum_P r_P P, where r is the forward-evolved coefficient vector of
 * 2^n |0><0| = sum over strings of I and Z (Eq. (3) with the state's own Pauli
 * weights).  Each string P is decoded as in Sec. III-D: every row a of P has a
 * single nonzero entry, at the column b obtained by flipping the qubits that
 * carry X or Y, with the value prod_q <a_q| p_q |b_q> (I, X, Y, Z 2x2 entries).
 * Rows and columns index basis states with qubit 0 as the most significant bit.
 * out_re / out_im: 2^n x 2^n, row-major. */
int orc_density_matrix(int n, int64_t m, const orc_gate *gates, const double *thetas,
                       int64_t n_params, double *out_re, double *out_im) {
    if (n < 1 || n > 10) return ORC_EINVAL;
    const int64_t N = pow4(n), D = (int64_t)1 << n;
    double *r = (double *)malloc((size_t)N * sizeof(double));
    if (!r) return ORC_EINVAL;
    for (int64_t i = 0; i < N; ++i) {
        int xfree = 1;
        for (int q = 0; q < n; ++q) {
            int d = digit(i, n, q);
            if (d == 1 || d == 2) { xfree = 0; break; }
        }
        r[i] = xfree ? 1.0 : 0.0;
    }
    int rc = orc_forward(n, m, gates, thetas, n_params, r);
    if (rc != ORC_OK) { free(r); return rc; }
    /* 2x2 entries <a|p|b> of I, X, Y, Z as (re, im) */
    static const double pre[4][2][2] = {{{1, 0}, {0, 1}}, {{0, 1}, {1, 0}}, {{0, 0}, {0, 0}},
                                        {{1, 0}, {0, -1}}};
    static const double pim[4][2][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}, {{0, -1}, {1, 0}},
                                        {{0, 0}, {0, 0}}};
    for (int64_t k = 0; k < D * D; ++k) { out_re[k] = 0.0; out_im[k] = 0.0; }
    const double scale = 1.0 / (double)D;
    for (int64_t i = 0; i < N; ++i) {
        if (r[i] == 0.0) continue;
        int64_t flip = 0;
        for (int q = 0; q < n; ++q) {
            int d = digit(i, n, q);
            if (d == 1 || d == 2) flip |= (int64_t)1 << (n - 1 - q);
        }
        for (int64_t a = 0; a < D; ++a) {
            int64_t b = a ^ flip;
            double vr = 1.0, vi = 0.0;
            for (int q = 0; q < n; ++q) {
                int d = digit(i, n, q);
                int aq = (int)((a >> (n - 1 - q)) & 1), bq = (int)((b >> (n - 1 - q)) & 1);
                double er = pre[d][aq][bq], ei = pim[d][aq][bq];
                double tr = vr * er - vi * ei, ti = vr * ei + vi * er;
                vr = tr; vi = ti;
            }
            out_re[a * D + b] += scale * r[i] * vr;
            out_im[a * D + b] += scale * r[i] * vi;
        }
    }
    free(r);
    return ORC_OK;
}
