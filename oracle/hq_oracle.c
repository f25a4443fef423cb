/*
 * hq_oracle.c -- CPU oracle for the state-vector path (TEST INFRASTRUCTURE).
 *
 * Plain, slow, obviously-correct complex128 reference of what the GPU path
 * computes.  It is used only by the tests, by the bench's CPU-baseline leg and
 * by the smoke check; the product never links or calls it.  It shares no code
 * with the CUDA path.
 *
 * Conventions (HybridQ, arXiv 2111.06868):
 *   - Sec. 2 "Gates": a MatrixGate is a dense 2^k x 2^k matrix on k qubits.
 *     Local basis index r = sum_j r_j 2^(k-1-j): qubits[0] is the local MSB.
 *   - Sec. 2.2 (Grover oracle printout): qubit q is axis q of the C-order
 *     (2,)*n tensor, i.e. bit (n-1-q) of the flat amplitude index.
 *   - Sec. 4.1: initial-state tokens '0' '1' '+' '-' build a product state.
 *   - Sec. 4.2: the state-vector engine applies each (fused) gate as a
 *     matrix-vector product on the groups of 2^k amplitudes that differ only in
 *     the target bits.  The oracle applies the gates one by one, unfused: the
 *     method (fusion + any kernel) reaches exactly U_G...U_1 |psi0> up to
 *     rounding, and that product is the definition written out here.
 *   - Expectation <psi|P|psi> of a Pauli string: P applied factor by factor as
 *     1-qubit gates, then the inner product summed serially in double.
 *   - Gradients (not in the paper; the method is the adjoint reverse sweep of
 *     Jones & Gacon, arXiv 2009.02823): the derivative of E = <psi|H|psi> with
 *     respect to rotation angles, by (a) the adjoint sweep and (b) the
 *     parameter-shift rule, exact for R_P(t) = exp(-i t P / 2).
 *
 * Memory layout: a state is 2^n interleaved (re, im) doubles; matrices are
 * row-major interleaved complex128.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define OR_MAXK 6

/* bit position of qubit q in an n-qubit flat index (Sec. 2.2 ordering) */
static int64_t qubit_bit(int n, int q) { return (int64_t)1 << (n - 1 - q); }

/* psi = kron over qubits 0..n-1 of the one-qubit token states (Sec. 4.1) */
void or_state_init(int n, const char *tokens, double *psi_out)
{
    cplx *psi = (cplx *)psi_out;
    const double s = 1.0 / sqrt(2.0);
    int64_t dim = (int64_t)1 << n;
    for (int64_t x = 0; x < dim; ++x) {
        cplx a = 1.0;
        for (int q = 0; q < n; ++q) {
            int bit = (x & qubit_bit(n, q)) != 0;
            char t = tokens ? tokens[q] : '0';
            cplx f = 0.0;
            if (t == '0') f = bit ? 0.0 : 1.0;
            else if (t == '1') f = bit ? 1.0 : 0.0;
            else if (t == '+') f = s;
            else if (t == '-') f = bit ? -s : s;
            a *= f;
        }
        psi[x] = a;
    }
}

/*
 * psi <- (M on qubits) psi.  For every base index x with all target bits zero,
 * gather v[r] = psi[x + off(r)], compute w = M v, scatter w back.
 */
void or_apply_gate(int n, double *psi_io, int k, const int *qubits, const double *mat)
{
    cplx *psi = (cplx *)psi_io;
    const cplx *M = (const cplx *)mat;
    int K = 1 << k;
    int64_t dim = (int64_t)1 << n, tmask = 0;
    int64_t off[1 << OR_MAXK];
    for (int j = 0; j < k; ++j) tmask |= qubit_bit(n, qubits[j]);
    for (int r = 0; r < K; ++r) {
        off[r] = 0;
        for (int j = 0; j < k; ++j)
            if ((r >> (k - 1 - j)) & 1) off[r] += qubit_bit(n, qubits[j]);
    }
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < dim; ++x) {
        if (x & tmask) continue;
        cplx v[1 << OR_MAXK], w[1 << OR_MAXK];
        for (int c = 0; c < K; ++c) v[c] = psi[x + off[c]];
        for (int r = 0; r < K; ++r) {
            cplx acc = 0.0;
            for (int c = 0; c < K; ++c) acc += M[r * K + c] * v[c];
            w[r] = acc;
        }
        for (int r = 0; r < K; ++r) psi[x + off[r]] = w[r];
    }
}

/* R_P(t) = cos(t/2) I - i sin(t/2) P, P in {X, Y, Z}; writes 2x2 complex */
static void rotation_matrix(char axis, double t, cplx *m)
{
    double c = cos(0.5 * t), s = sin(0.5 * t);
    if (axis == 'X') { m[0] = c; m[1] = -I * s; m[2] = -I * s; m[3] = c; }
    else if (axis == 'Y') { m[0] = c; m[1] = -s; m[2] = s; m[3] = c; }
    else { m[0] = c - I * s; m[1] = 0; m[2] = 0; m[3] = c + I * s; }
}

/* d R_P(t) / dt = -(1/2) sin(t/2) I - (i/2) cos(t/2) P */
static void rotation_derivative(char axis, double t, cplx *m)
{
    double c = cos(0.5 * t), s = sin(0.5 * t);
    cplx P[4];
    if (axis == 'X') { P[0] = 0; P[1] = 1; P[2] = 1; P[3] = 0; }
    else if (axis == 'Y') { P[0] = 0; P[1] = -I; P[2] = I; P[3] = 0; }
    else { P[0] = 1; P[1] = 0; P[2] = 0; P[3] = -1; }
    for (int i = 0; i < 4; ++i) m[i] = -0.5 * I * c * P[i];
    m[0] += -0.5 * s;
    m[3] += -0.5 * s;
}

/*
 * A circuit, as flat arrays (G gates):
 *   k[g], qubits[g*6 + j], kind[g] (0 = fixed matrix at mats + 2*off[g] doubles,
 *   1 = rotation about axis[g] by theta[param[g]]).
 */
typedef struct {
    int G;
    const int *k, *qubits, *kind, *axis, *param;
    const double *mats;
    const int64_t *off;
} circ_t;

static void gate_matrix(const circ_t *c, int g, const double *theta, int dagger, cplx *out)
{
    int K = 1 << c->k[g];
    cplx tmp[1 << (2 * OR_MAXK)];
    const cplx *src;
    if (c->kind[g] == 0) {
        src = (const cplx *)(c->mats) + c->off[g];
    } else {
        rotation_matrix((char)c->axis[g], theta[c->param[g]], tmp);
        src = tmp;
    }
    for (int r = 0; r < K; ++r)
        for (int col = 0; col < K; ++col)
            out[r * K + col] = dagger ? conj(src[col * K + r]) : src[r * K + col];
}

static void apply_circuit_range(int n, cplx *psi, const circ_t *c, const double *theta, int g0, int g1)
{
    static cplx m[1 << (2 * OR_MAXK)];
    for (int g = g0; g < g1; ++g) {
        gate_matrix(c, g, theta, 0, m);
        or_apply_gate(n, (double *)psi, c->k[g], c->qubits + 6 * g, (const double *)m);
    }
}

void or_apply_circuit(int n, double *psi, int G, const int *k, const int *qubits, const int *kind,
                      const int *axis, const int *param, const double *mats, const int64_t *off,
                      const double *theta)
{
    circ_t c = {G, k, qubits, kind, axis, param, mats, off};
    apply_circuit_range(n, (cplx *)psi, &c, theta, 0, G);
}

/*
 * Pauli sums: T terms; term t has coeff[t], len[t] factors, factor j acting on
 * qubit tq[t*8 + j] with operator top[t*8 + j] in {'X','Y','Z'}.
 */
static void apply_pauli_string(int n, cplx *v, int len, const int *q, const char *op)
{
    static const cplx X[4] = {0, 1, 1, 0};
    static const cplx Y[4] = {0, -I, I, 0};
    static const cplx Z[4] = {1, 0, 0, -1};
    for (int j = 0; j < len; ++j) {
        const cplx *m = op[j] == 'X' ? X : op[j] == 'Y' ? Y : Z;
        or_apply_gate(n, (double *)v, 1, &q[j], (const double *)m);
    }
}

static cplx inner(int64_t dim, const cplx *a, const cplx *b)
{
    cplx s = 0.0;
    for (int64_t x = 0; x < dim; ++x) s += conj(a[x]) * b[x];
    return s;
}

/* out = H psi */
static void apply_hamiltonian(int n, const cplx *psi, cplx *out, cplx *tmp, int T, const double *coeff,
                              const int *len, const int *tq, const char *top)
{
    int64_t dim = (int64_t)1 << n;
    memset(out, 0, sizeof(cplx) * dim);
    for (int t = 0; t < T; ++t) {
        memcpy(tmp, psi, sizeof(cplx) * dim);
        apply_pauli_string(n, tmp, len[t], tq + 8 * t, top + 8 * t);
        for (int64_t x = 0; x < dim; ++x) out[x] += coeff[t] * tmp[x];
    }
}

/* E = sum_t coeff_t <psi| P_t |psi>  (real part; P_t Hermitian) */
double or_expectation(int n, const double *psi_in, int T, const double *coeff, const int *len,
                      const int *tq, const char *top)
{
    int64_t dim = (int64_t)1 << n;
    const cplx *psi = (const cplx *)psi_in;
    cplx *tmp = malloc(sizeof(cplx) * dim);
    double e = 0.0;
    for (int t = 0; t < T; ++t) {
        memcpy(tmp, psi, sizeof(cplx) * dim);
        apply_pauli_string(n, tmp, len[t], tq + 8 * t, top + 8 * t);
        e += coeff[t] * creal(inner(dim, psi, tmp));
    }
    free(tmp);
    return e;
}

/* ||psi||^2 summed serially */
double or_norm2(int n, const double *psi_in)
{
    int64_t dim = (int64_t)1 << n;
    const cplx *psi = (const cplx *)psi_in;
    double s = 0.0;
    for (int64_t x = 0; x < dim; ++x) s += creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
    return s;
}

/* E(theta) for a parametrised circuit from the token state */
double or_energy(int n, const char *tokens, int G, const int *k, const int *qubits, const int *kind,
                 const int *axis, const int *param, const double *mats, const int64_t *off,
                 const double *theta, int T, const double *coeff, const int *len, const int *tq,
                 const char *top)
{
    int64_t dim = (int64_t)1 << n;
    double *psi = malloc(sizeof(cplx) * dim);
    or_state_init(n, tokens, psi);
    or_apply_circuit(n, psi, G, k, qubits, kind, axis, param, mats, off, theta);
    double e = or_expectation(n, psi, T, coeff, len, tq, top);
    free(psi);
    return e;
}

/*
 * Adjoint reverse sweep (Jones & Gacon): psi_G = U_G..U_1 psi_0, lambda = H psi_G,
 * phi = psi_G; for g = G..1: phi <- U_g^+ phi; if g is a rotation,
 * grad[param_g] += 2 Re <lambda| dU_g phi>; lambda <- U_g^+ lambda.
 * Returns E; grad has P entries (zeroed here).
 */
double or_adjoint_grad(int n, const char *tokens, int G, const int *k, const int *qubits, const int *kind,
                       const int *axis, const int *param, const double *mats, const int64_t *off,
                       const double *theta, int P, int T, const double *coeff, const int *len,
                       const int *tq, const char *top, double *grad)
{
    circ_t c = {G, k, qubits, kind, axis, param, mats, off};
    int64_t dim = (int64_t)1 << n;
    cplx *phi = malloc(sizeof(cplx) * dim);
    cplx *lam = malloc(sizeof(cplx) * dim);
    cplx *mu = malloc(sizeof(cplx) * dim);
    static cplx m[1 << (2 * OR_MAXK)];
    or_state_init(n, tokens, (double *)phi);
    apply_circuit_range(n, phi, &c, theta, 0, G);
    apply_hamiltonian(n, phi, lam, mu, T, coeff, len, tq, top);
    double e = creal(inner(dim, phi, lam));
    for (int p = 0; p < P; ++p) grad[p] = 0.0;
    for (int g = G - 1; g >= 0; --g) {
        gate_matrix(&c, g, theta, 1, m);
        or_apply_gate(n, (double *)phi, k[g], qubits + 6 * g, (const double *)m);
        if (kind[g] == 1) {
            cplx d[4];
            rotation_derivative((char)axis[g], theta[param[g]], d);
            memcpy(mu, phi, sizeof(cplx) * dim);
            or_apply_gate(n, (double *)mu, 1, qubits + 6 * g, (const double *)d);
            grad[param[g]] += 2.0 * creal(inner(dim, lam, mu));
        }
        or_apply_gate(n, (double *)lam, k[g], qubits + 6 * g, (const double *)m);
    }
    free(phi);
    free(lam);
    free(mu);
    return e;
}

/*
 * Parameter-shift gradient: for each rotation occurrence g with parameter p,
 * dE/dp += [E(theta_g + pi/2) - E(theta_g - pi/2)] / 2, shifting that
 * occurrence only (exact for exp(-i t P/2)).
 */
void or_param_shift_grad(int n, const char *tokens, int G, const int *k, const int *qubits, const int *kind,
                         const int *axis, const int *param, const double *mats, const int64_t *off,
                         const double *theta, int P, int T, const double *coeff, const int *len,
                         const int *tq, const char *top, double *grad)
{
    /* each occurrence gets its own parameter slot so that only it is shifted */
    int *pocc = malloc(sizeof(int) * (G > 0 ? G : 1));
    double *th = malloc(sizeof(double) * (G > 0 ? G : 1));
    for (int g = 0; g < G; ++g) {
        pocc[g] = g;
        th[g] = kind[g] == 1 ? theta[param[g]] : 0.0;
    }
    for (int p = 0; p < P; ++p) grad[p] = 0.0;
    for (int g = 0; g < G; ++g) {
        if (kind[g] != 1) continue;
        double t0 = th[g];
        th[g] = t0 + M_PI / 2;
        double ep = or_energy(n, tokens, G, k, qubits, kind, axis, pocc, mats, off, th, T, coeff, len, tq, top);
        th[g] = t0 - M_PI / 2;
        double em = or_energy(n, tokens, G, k, qubits, kind, axis, pocc, mats, off, th, T, coeff, len, tq, top);
        th[g] = t0;
        grad[param[g]] += 0.5 * (ep - em);
    }
    free(pocc);
    free(th);
}

/*
 * Matrix of a gate sequence restricted to the qubit list `bq` (kb qubits):
 * column c = the sequence applied to basis state |c> of a kb-qubit register,
 * where gate qubits are renamed to their position in bq.  Mirrors the
 * "matrix(circuit)" utility of Sec. 3.1.  out: 2^kb x 2^kb row-major.
 */
void or_sequence_matrix(int kb, const int *bq, int G, const int *k, const int *qubits, const double *mats,
                        const int64_t *off, double *out)
{
    int K = 1 << kb;
    cplx *col = malloc(sizeof(cplx) * K);
    cplx *o = (cplx *)out;
    for (int c = 0; c < K; ++c) {
        for (int r = 0; r < K; ++r) col[r] = (r == c) ? 1.0 : 0.0;
        for (int g = 0; g < G; ++g) {
            int lq[OR_MAXK];
            for (int j = 0; j < k[g]; ++j) {
                lq[j] = -1;
                for (int i = 0; i < kb; ++i)
                    if (bq[i] == qubits[6 * g + j]) lq[j] = i;
            }
            or_apply_gate(kb, (double *)col, k[g], lq, mats + 2 * off[g]);
        }
        for (int r = 0; r < K; ++r) o[r * K + c] = col[r];
    }
    free(col);
}

void or_set_threads(int t);
#ifdef _OPENMP
#include <omp.h>
void or_set_threads(int t) { omp_set_num_threads(t); }
int or_max_threads(void) { return omp_get_max_threads(); }
#else
void or_set_threads(int t) { (void)t; }
int or_max_threads(void) { return 1; }
#endif
