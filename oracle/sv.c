/*
 * Oracle: plain, slow, obviously-correct CPU complex128 state-vector simulator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library; the product path never
 * does.  It shares no code with the CUDA library: gate matrices, gate
 * application, Pauli expectations and gradients are all written out here from
 * their definitions.
 *
 * What it computes (paper: Sec. I.B "Primitives" -- circuits of rx/ry/rzz/h/cx
 * gates on |0..0>, expectation_ps of Pauli strings, the TFIM energy
 * H = -sum Z_i Z_j - g sum X_i, value_and_grad of the energy):
 *   - psi in C^(2^n), bit q of the index is qubit q;
 *   - every gate applied unfused, in list order, by gathering the 2^k
 *     amplitudes of each index class and multiplying by the 2^k x 2^k matrix;
 *   - <psi|P|psi> = sum_x conj(psi[x ^ m]) i^{#Y} (-1)^{popc(x & z)} psi[x];
 *   - (H psi)[y] = sum_j c_j i^{#Y_j} (-1)^{popc((y ^ m_j) & z_j)} psi[y ^ m_j];
 *   - dE/dtheta by the two-term parameter-shift rule (the "2k circuit
 *     evaluations" the paper contrasts with reverse-mode AD in Sec. I.B), and
 *     by central finite differences;
 *   - Born probabilities of a subset of qubits (the QML readout of Sec. VII.B)
 *     and single-qubit projective measurements (the MIPT trajectories of
 *     Sec. VII.C, the shadow snapshots of Sec. VII.A).
 * Gate conventions: R_P(t) = exp(-i t P / 2) (RX, RY, RZ, RZZ, and RP for any
 * Pauli word P on 1..5 qubits, word digit j = 2 bits of mat_off, 0 I, 1 X, 2 Y, 3 Z); 2-qubit local index
 * r = 2*bit(q[0]) + bit(q[1]); CX(control, target); CP(phi) = diag(1,1,1,e^{i phi}).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cx;

/* One record of the flat gate-list input format (56 bytes). */
typedef struct {
    uint16_t op;
    uint8_t nq;
    uint8_t pad;
    int32_t q[5];
    int32_t param;
    double scale;
    double angle0;
    int64_t mat_off;
} og_gate;

enum {
    O_I = 0, O_X, O_Y, O_Z, O_H, O_S, O_T, O_RX, O_RY, O_RZ,
    O_CX, O_CZ, O_CP, O_SWAP, O_RZZ, O_U1, O_U2, O_UK, O_RP
};

#define OK 0
#define EBAD 1

static int op_qubits(const og_gate* g) {
    switch (g->op) {
    case O_I: case O_X: case O_Y: case O_Z: case O_H: case O_S: case O_T:
    case O_RX: case O_RY: case O_RZ: case O_U1:
        return 1;
    case O_CX: case O_CZ: case O_CP: case O_SWAP: case O_RZZ: case O_U2:
        return 2;
    case O_UK: case O_RP:
        return g->nq;
    default:
        return -1;
    }
}

static double gate_angle(const og_gate* g, const double* params, double extra) {
    double a = g->angle0 + extra;
    if (g->param >= 0) a += g->scale * params[g->param];
    return a;
}

/* Fill M (2^k x 2^k, row-major) with the gate's matrix in its own local order. */
static int gate_matrix(const og_gate* g, const double* pool, const double* params,
                       double extra, cx* M, int* k_out) {
    int k = op_qubits(g);
    if (k < 1 || k > 5) return EBAD;
    int d = 1 << k;
    for (int i = 0; i < d * d; ++i) M[i] = 0.0;
    const double r2 = 1.0 / sqrt(2.0);
    double th, c, s;
    switch (g->op) {
    case O_I: M[0] = 1; M[3] = 1; break;
    case O_X: M[1] = 1; M[2] = 1; break;
    case O_Y: M[1] = -I; M[2] = I; break;
    case O_Z: M[0] = 1; M[3] = -1; break;
    case O_H: M[0] = r2; M[1] = r2; M[2] = r2; M[3] = -r2; break;
    case O_S: M[0] = 1; M[3] = I; break;
    case O_T: M[0] = 1; M[3] = cexp(I * M_PI / 4.0); break;
    case O_RX:
        th = gate_angle(g, params, extra); c = cos(th / 2); s = sin(th / 2);
        M[0] = c; M[1] = -I * s; M[2] = -I * s; M[3] = c; break;
    case O_RY:
        th = gate_angle(g, params, extra); c = cos(th / 2); s = sin(th / 2);
        M[0] = c; M[1] = -s; M[2] = s; M[3] = c; break;
    case O_RZ:
        th = gate_angle(g, params, extra);
        M[0] = cexp(-I * th / 2); M[3] = cexp(I * th / 2); break;
    case O_CX:  /* control q[0] (MSB of r), target q[1] */
        M[0 * 4 + 0] = 1; M[1 * 4 + 1] = 1; M[2 * 4 + 3] = 1; M[3 * 4 + 2] = 1; break;
    case O_CZ:
        M[0] = 1; M[5] = 1; M[10] = 1; M[15] = -1; break;
    case O_CP:
        th = gate_angle(g, params, extra);
        M[0] = 1; M[5] = 1; M[10] = 1; M[15] = cexp(I * th); break;
    case O_SWAP:
        M[0 * 4 + 0] = 1; M[1 * 4 + 2] = 1; M[2 * 4 + 1] = 1; M[3 * 4 + 3] = 1; break;
    case O_RZZ:  /* exp(-i th Z(x)Z / 2): Z(x)Z = diag(1,-1,-1,1) */
        th = gate_angle(g, params, extra);
        M[0] = cexp(-I * th / 2); M[5] = cexp(I * th / 2);
        M[10] = cexp(I * th / 2); M[15] = cexp(-I * th / 2); break;
    case O_RP: {  /* exp(-i th P / 2), P = sigma_{w_0} (x) ... (x) sigma_{w_{k-1}}, q[0] first */
        th = gate_angle(g, params, extra); c = cos(th / 2); s = sin(th / 2);
        /* P[r][col] = prod_j sigma_{w_j}[bit_j(r)][bit_j(col)], bit_j = bit k-1-j */
        static const double complex sig[4][2][2] = {
            {{1, 0}, {0, 1}}, {{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
        for (int r = 0; r < d; ++r)
            for (int col = 0; col < d; ++col) {
                cx pv = 1.0;
                for (int j = 0; j < k; ++j) {
                    const int w = (int)((g->mat_off >> (2 * j)) & 3);
                    pv *= sig[w][(r >> (k - 1 - j)) & 1][(col >> (k - 1 - j)) & 1];
                }
                M[r * d + col] = (r == col ? c : 0.0) - I * s * pv;
            }
        break;
    }
    case O_U1: case O_U2: case O_UK:
        if (g->mat_off < 0) return EBAD;
        for (int i = 0; i < d * d; ++i)
            M[i] = pool[2 * (g->mat_off + i)] + I * pool[2 * (g->mat_off + i) + 1];
        break;
    default:
        return EBAD;
    }
    *k_out = k;
    return OK;
}

/* Apply one k-qubit matrix to psi by definition. */
static void apply_matrix(int n, cx* psi, const int32_t* q, int k, const cx* M) {
    const int64_t N = (int64_t)1 << n;
    const int d = 1 << k;
    int64_t qmask = 0;
    for (int j = 0; j < k; ++j) qmask |= (int64_t)1 << q[j];
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < N; ++x) {
        if (x & qmask) continue; /* one representative per index class */
        int64_t idx[32];
        cx v[32], w[32];
        for (int r = 0; r < d; ++r) {
            int64_t y = x;
            for (int j = 0; j < k; ++j)
                if ((r >> (k - 1 - j)) & 1) y |= (int64_t)1 << q[j];
            idx[r] = y;
            v[r] = psi[y];
        }
        for (int r = 0; r < d; ++r) {
            cx acc = 0;
            for (int s = 0; s < d; ++s) acc += M[r * d + s] * v[s];
            w[r] = acc;
        }
        for (int r = 0; r < d; ++r) psi[idx[r]] = w[r];
    }
}

static int check_gate(int n, const og_gate* g, int P, int64_t n_mat) {
    int k = op_qubits(g);
    if (k < 1 || k > 5) return EBAD;
    for (int j = 0; j < k; ++j) {
        if (g->q[j] < 0 || g->q[j] >= n) return EBAD;
        for (int i = 0; i < j; ++i)
            if (g->q[i] == g->q[j]) return EBAD;
    }
    if (g->param >= P) return EBAD;
    if (g->op == O_RP && (g->mat_off < 0 || g->mat_off >= (1LL << (2 * k)))) return EBAD;
    if ((g->op == O_U1 || g->op == O_U2 || g->op == O_UK) &&
        (g->mat_off < 0 || g->mat_off + (1LL << (2 * k)) > n_mat))
        return EBAD;
    return OK;
}

/* Apply ops[0..n_ops) in order; if shift_gate >= 0 that gate's angle gets +shift. */
static int apply_ops(int n, cx* psi, const og_gate* ops, int64_t n_ops,
                     const double* pool, int64_t n_mat, const double* params, int P,
                     int64_t shift_gate, double shift) {
    cx M[1024];
    for (int64_t i = 0; i < n_ops; ++i) {
        int k;
        if (check_gate(n, &ops[i], P, n_mat)) return EBAD;
        if (gate_matrix(&ops[i], pool, params, i == shift_gate ? shift : 0.0, M, &k))
            return EBAD;
        apply_matrix(n, psi, ops[i].q, k, M);
    }
    return OK;
}

int orc_apply(int n, double* psi_ri, const og_gate* ops, int64_t n_ops,
              const double* pool, int64_t n_mat, const double* params, int P) {
    return apply_ops(n, (cx*)psi_ri, ops, n_ops, pool, n_mat, params, P, -1, 0.0);
}

/* The full 2^k x 2^k matrix of one gate (for tests of the gate formulas). */
int orc_gate_matrix(const og_gate* g, const double* pool, const double* params,
                    double* out_ri) {
    int k;
    return gate_matrix(g, pool, params, 0.0, (cx*)out_ri, &k);
}

static cx ipow(int e) {
    switch (e & 3) {
    case 0: return 1;
    case 1: return I;
    case 2: return -1;
    default: return -I;
    }
}

static int popc64(uint64_t v) {
    int c = 0;
    while (v) { v &= v - 1; ++c; }
    return c;
}

/* <psi|P|psi> for one Pauli string. */
static cx expect_one(int n, const cx* psi, uint64_t xm, uint64_t zm) {
    const int64_t N = (int64_t)1 << n;
    const cx ph = ipow(popc64(xm & zm));
    long double sr = 0, si = 0;
    for (int64_t x = 0; x < N; ++x) {
        cx t = conj(psi[x ^ (int64_t)xm]) * psi[x];
        if (popc64((uint64_t)x & zm) & 1) t = -t;
        sr += creal(t);
        si += cimag(t);
    }
    cx s = (double)sr + I * (double)si;
    return ph * s;
}

int orc_expect(int n, const double* psi_ri, const uint64_t* xm, const uint64_t* zm,
               int64_t T, double* out_re, double* out_im) {
    const uint64_t lim = (n >= 64) ? ~0ULL : ((1ULL << n) - 1);
    for (int64_t t = 0; t < T; ++t)
        if ((xm[t] & ~lim) || (zm[t] & ~lim)) return EBAD;
#pragma omp parallel for schedule(dynamic)
    for (int64_t t = 0; t < T; ++t) {
        cx e = expect_one(n, (const cx*)psi_ri, xm[t], zm[t]);
        out_re[t] = creal(e);
        out_im[t] = cimag(e);
    }
    return OK;
}

/* lambda = H psi with H = sum_t coeff[t] P_t. */
int orc_hamiltonian_apply(int n, const double* psi_ri, const uint64_t* xm, const uint64_t* zm,
                          const double* coeff, int64_t T, double* out_ri) {
    const int64_t N = (int64_t)1 << n;
    const cx* psi = (const cx*)psi_ri;
    cx* out = (cx*)out_ri;
#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < N; ++y) {
        cx acc = 0;
        for (int64_t t = 0; t < T; ++t) {
            int64_t x = y ^ (int64_t)xm[t];
            cx v = ipow(popc64(xm[t] & zm[t])) * psi[x];
            if (popc64((uint64_t)x & zm[t]) & 1) v = -v;
            acc += coeff[t] * v;
        }
        out[y] = acc;
    }
    return OK;
}

static double energy_of(int n, const cx* psi, const uint64_t* xm, const uint64_t* zm,
                        const double* coeff, int64_t T) {
    long double e = 0;
    for (int64_t t = 0; t < T; ++t) e += coeff[t] * creal(expect_one(n, psi, xm[t], zm[t]));
    return (double)e;
}

/* E(theta) = <psi(theta)|H|psi(theta)>, psi(theta) = U(theta)|0..0>. */
static int energy_eval(int n, const og_gate* ops, int64_t n_ops, const double* pool,
                       int64_t n_mat, const double* params, int P, const uint64_t* xm,
                       const uint64_t* zm, const double* coeff, int64_t T,
                       int64_t shift_gate, double shift, double* E, cx* work) {
    const int64_t N = (int64_t)1 << n;
    for (int64_t x = 0; x < N; ++x) work[x] = 0;
    work[0] = 1;
    if (apply_ops(n, work, ops, n_ops, pool, n_mat, params, P, shift_gate, shift)) return EBAD;
    *E = energy_of(n, work, xm, zm, coeff, T);
    return OK;
}

int orc_energy(int n, const og_gate* ops, int64_t n_ops, const double* pool, int64_t n_mat,
               const double* params, int P, const uint64_t* xm, const uint64_t* zm,
               const double* coeff, int64_t T, double* E) {
    cx* work = (cx*)malloc(sizeof(cx) * ((size_t)1 << n));
    if (!work) return EBAD;
    int rc = energy_eval(n, ops, n_ops, pool, n_mat, params, P, xm, zm, coeff, T, -1, 0.0, E, work);
    free(work);
    return rc;
}

static int shiftable(int op) {
    return op == O_RX || op == O_RY || op == O_RZ || op == O_RZZ || op == O_CP || op == O_RP;
}

/*
 * Parameter-shift gradient: every parameterised gate has a generator with
 * eigenvalues +-1/2 (up to a global phase for CP), so
 * dE/d(angle_g) = [E(angle_g + pi/2) - E(angle_g - pi/2)] / 2, and
 * dE/dtheta_p = sum over gates g reading p of scale_g * dE/d(angle_g).
 * Runs the shifted evaluations in parallel, one state per thread.
 */
int orc_grad_param_shift(int n, const og_gate* ops, int64_t n_ops, const double* pool,
                         int64_t n_mat, const double* params, int P, const uint64_t* xm,
                         const uint64_t* zm, const double* coeff, int64_t T, double* grad) {
    for (int p = 0; p < P; ++p) grad[p] = 0.0;
    for (int64_t i = 0; i < n_ops; ++i) {
        if (check_gate(n, &ops[i], P, n_mat)) return EBAD;
        if (ops[i].param >= 0 && !shiftable(ops[i].op)) return EBAD;
    }
    double* dg = (double*)calloc((size_t)(n_ops > 0 ? n_ops : 1), sizeof(double));
    int bad = 0;
#pragma omp parallel
    {
        cx* work = (cx*)malloc(sizeof(cx) * ((size_t)1 << n));
#pragma omp for schedule(dynamic)
        for (int64_t i = 0; i < n_ops; ++i) {
            if (ops[i].param < 0) continue;
            double ep, em;
            int r1 = energy_eval(n, ops, n_ops, pool, n_mat, params, P, xm, zm, coeff, T,
                                 i, M_PI / 2, &ep, work);
            int r2 = energy_eval(n, ops, n_ops, pool, n_mat, params, P, xm, zm, coeff, T,
                                 i, -M_PI / 2, &em, work);
            if (r1 || r2) bad = 1;
            dg[i] = 0.5 * (ep - em);
        }
        free(work);
    }
    for (int64_t i = 0; i < n_ops; ++i)
        if (ops[i].param >= 0) grad[ops[i].param] += ops[i].scale * dg[i];
    free(dg);
    return bad ? EBAD : OK;
}

/* Central finite differences in theta with step h. */
int orc_grad_fd(int n, const og_gate* ops, int64_t n_ops, const double* pool, int64_t n_mat,
                const double* params, int P, const uint64_t* xm, const uint64_t* zm,
                const double* coeff, int64_t T, double h, double* grad) {
    int bad = 0;
#pragma omp parallel
    {
        cx* work = (cx*)malloc(sizeof(cx) * ((size_t)1 << n));
        double* th = (double*)malloc(sizeof(double) * (size_t)(P > 0 ? P : 1));
        memcpy(th, params, sizeof(double) * (size_t)P);
#pragma omp for schedule(dynamic)
        for (int p = 0; p < P; ++p) {
            double ep, em;
            th[p] = params[p] + h;
            int r1 = energy_eval(n, ops, n_ops, pool, n_mat, th, P, xm, zm, coeff, T, -1, 0, &ep, work);
            th[p] = params[p] - h;
            int r2 = energy_eval(n, ops, n_ops, pool, n_mat, th, P, xm, zm, coeff, T, -1, 0, &em, work);
            th[p] = params[p];
            if (r1 || r2) bad = 1;
            grad[p] = (ep - em) / (2 * h);
        }
        free(th);
        free(work);
    }
    return bad ? EBAD : OK;
}

/* Born probabilities of measuring qubits q[0..k-1] in the computational basis:
 * out[j] = sum of |psi[x]|^2 over the x whose bits at q[0..k-1] spell j, with
 * q[0] the most significant bit of j (the diagonal of the reduced density
 * matrix of those qubits). */
int orc_marginal_probs(int n, const double* psi_ri, const int32_t* q, int k, double* out) {
    const int64_t N = (int64_t)1 << n;
    const cx* psi = (const cx*)psi_ri;
    if (k < 1 || k > 20) return EBAD;
    for (int i = 0; i < k; ++i) {
        if (q[i] < 0 || q[i] >= n) return EBAD;
        for (int j = 0; j < i; ++j)
            if (q[j] == q[i]) return EBAD;
    }
    long double* acc = (long double*)calloc((size_t)1 << k, sizeof(long double));
    if (!acc) return EBAD;
    for (int64_t x = 0; x < N; ++x) {
        int64_t j = 0;
        for (int i = 0; i < k; ++i) j = (j << 1) | ((x >> q[i]) & 1);
        acc[j] += (long double)(creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]));
    }
    for (int64_t j = 0; j < ((int64_t)1 << k); ++j) out[j] = (double)acc[j];
    free(acc);
    return OK;
}

/* Projective measurement of qubit q in the computational basis (Born rule).
 * p0 = sum_{bit q of x = 0} |psi[x]|^2 / sum_x |psi[x]|^2; the outcome is 0 if
 * u < p0, else 1 (forced = 0 or 1 imposes an outcome instead).  The amplitudes
 * of the other outcome are set to zero and the rest rescaled to unit norm.
 * Returns the outcome; *prob = its probability, *p0_out = p0. */
int orc_measure_qubit(int n, double* psi_ri, int q, double u, int forced, double* prob, double* p0_out) {
    const int64_t N = (int64_t)1 << n;
    cx* psi = (cx*)psi_ri;
    if (q < 0 || q >= n) return -1;
    long double s0 = 0, s1 = 0;
    for (int64_t x = 0; x < N; ++x) {
        const long double a = (long double)(creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]));
        if ((x >> q) & 1) s1 += a; else s0 += a;
    }
    const double p0 = (double)(s0 / (s0 + s1));
    const int out = forced >= 0 ? forced : (u < p0 ? 0 : 1);
    const double pk = out ? 1.0 - p0 : p0;
    const double scale = 1.0 / sqrt((double)(out ? s1 : s0));
    for (int64_t x = 0; x < N; ++x) {
        if ((int)((x >> q) & 1) == out) psi[x] *= scale;
        else psi[x] = 0;
    }
    *prob = pk;
    *p0_out = p0;
    return out;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
