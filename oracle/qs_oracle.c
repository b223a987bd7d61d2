/*
 * qs_oracle.c -- plain, slow, FP64 CPU oracle for the random-circuit
 * state-vector method of Boixo et al., "Characterizing Quantum Supremacy in
 * Near-Term Devices" (arXiv:1608.00263).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may link, load or
 * call this file; only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference arm use it.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * Every step is written the obvious way: no fusion, no blocking, no
 * reordering; sums run sequentially in index order in double precision.
 *
 * Conventions: bit j of a basis-state index is qubit j; a state of n qubits
 * is 2^n complex doubles stored as interleaved (re, im) pairs.
 *
 * Parity status per function:
 *   oracle_circuit_generate  -- rule checks pinned (Sec. "Convergence to
 *       Porter-Thomas" gate rules, Fig. two_dimers caption); the exact eight
 *       CZ layouts are a reading of a missing figure: layout parity unpinned
 *       (soft-pinned by Table I gates per level).
 *   oracle_circuit_generate_dense -- rule checks pinned (appendix "Depth to
 *       reach Porter-Thomas for denser 2D circuits": one CZ per qubit per CZ
 *       cycle, nearest neighbours on the torus, placement rules); the order
 *       of the four matchings is a reading: sequence parity unpinned.
 *   oracle_noisy_circuit     -- pinned by the error statistics of the model
 *       (rates and uniform Pauli choice) and by Eq. 6 against the measured
 *       cross entropy difference of noisy samples (Eqs. 5, aap).
 *   gate application         -- pinned (dense Kronecker unitary, Feynman path
 *       sum of Eqs. path1/phX/phT/phCZ, norm, time reversal).
 *   statistics, sampler, CE  -- pinned (closed forms Eqs. eu/eue, Porter-
 *       Thomas moments, brute-force CDF inversion, published SplitMix64
 *       outputs).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Gate record: same field meaning as the library's public gate struct, but
 * declared here on its own (the oracle includes no library header). */
typedef struct {
    uint8_t kind, q0, q1, pad;
    uint32_t cycle;
    double theta;
} oracle_gate;

enum { O_H = 0, O_X_HALF = 1, O_Y_HALF = 2, O_T = 3, O_CZ = 4,
       O_RX = 5, O_RY = 6, O_RZ = 7, O_CPHASE = 8 };

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): state advances by the     */
/* golden gamma, output is the Stafford "mix13" finaliser of the state.     */
/* ------------------------------------------------------------------------ */
static uint64_t splitmix_finalise(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static uint64_t splitmix_next(uint64_t *state)
{
    *state += 0x9E3779B97F4A7C15ULL;
    return splitmix_finalise(*state);
}

/* j-th output (0-based) of a SplitMix64 stream seeded with `seed`. */
uint64_t oracle_splitmix64_output(uint64_t seed, uint64_t j)
{
    uint64_t s = seed;
    uint64_t z = 0;
    for (uint64_t i = 0; i <= j; ++i) z = splitmix_next(&s);
    return z;
}

/* ------------------------------------------------------------------------ */
/* Circuit generator: Sec. "Convergence to Porter-Thomas" rules.             */
/*   cycle 0: H on every qubit;                                              */
/*   cycle t = 1..d: CZ layout number (t-1) mod 8, then a single-qubit gate  */
/*   on each qubit that was in a CZ at t-1 and is not in one at t: T if the  */
/*   qubit has had no single-qubit gate since the H layer, otherwise a       */
/*   uniform pick from {X^1/2, Y^1/2, T} minus the previous single-qubit gate */
/*   on that qubit.                                                          */
/* Reading of the missing layout figure (Fig. two_dimers): on an R x C grid  */
/*   H_a = horizontal edges (r,c)-(r,c+1) with (c + 2r) mod 4 == a,          */
/*   V_a = vertical edges (r,c)-(r+1,c) with (r + 2c) mod 4 == a,            */
/*   rotation H0 H2 V0 V2 H1 H3 V1 V3; edges touching dead sites dropped.    */
/* ------------------------------------------------------------------------ */

/* Fills `pair` with the CZ pairs of layout `layout` (0..7): qubit indices
 * (lower, higher), edges enumerated row by row then column by column.
 * Returns the number of pairs. */
static int layout_pairs(int rows, int cols, const uint8_t *dead,
                        const int *qubit_of_site, int layout, int *pair)
{
    static const int kind_of[8] = {0, 0, 1, 1, 0, 0, 1, 1};  /* 0=H, 1=V */
    static const int a_of[8] = {0, 2, 0, 2, 1, 3, 1, 3};
    int vertical = kind_of[layout], a = a_of[layout];
    int np = 0;
    for (int r = 0; r < rows; ++r) {
        for (int c = 0; c < cols; ++c) {
            int r2, c2;
            if (!vertical) {
                if (c + 1 >= cols || ((c + 2 * r) % 4) != a) continue;
                r2 = r; c2 = c + 1;
            } else {
                if (r + 1 >= rows || ((r + 2 * c) % 4) != a) continue;
                r2 = r + 1; c2 = c;
            }
            if (dead && (dead[r * cols + c] || dead[r2 * cols + c2])) continue;
            int qa = qubit_of_site[r * cols + c], qb = qubit_of_site[r2 * cols + c2];
            pair[2 * np] = qa < qb ? qa : qb;
            pair[2 * np + 1] = qa < qb ? qb : qa;
            ++np;
        }
    }
    return np;
}

/* Generates the circuit.  If out == NULL only the count is returned in
 * *ngates.  Returns 0 on success, -1 on bad arguments, -2 if cap is too
 * small. */
int oracle_circuit_generate(int rows, int cols, const uint8_t *dead, int depth,
                            uint64_t seed, oracle_gate *out, size_t cap,
                            size_t *ngates)
{
    if (rows < 1 || cols < 1 || depth < 0 || !ngates) return -1;
    int nsites = rows * cols;
    int *qubit_of_site = (int *)malloc(sizeof(int) * nsites);
    int n = 0;
    for (int s = 0; s < nsites; ++s)
        qubit_of_site[s] = (dead && dead[s]) ? -1 : n++;
    if (n < 1 || n > 64) { free(qubit_of_site); return -1; }

    int *pair = (int *)malloc(sizeof(int) * 4 * nsites);
    int *in_cz_prev = (int *)calloc(n, sizeof(int));
    int *in_cz_now = (int *)calloc(n, sizeof(int));
    int *last_1q = (int *)malloc(sizeof(int) * n);   /* -1: none since H */
    for (int q = 0; q < n; ++q) last_1q[q] = -1;
    uint64_t rng = seed;
    size_t count = 0;
    int rc = 0;

#define EMIT(K, A, B, CYC)                                                  \
    do {                                                                    \
        if (out) {                                                          \
            if (count >= cap) { rc = -2; goto done; }                       \
            out[count].kind = (uint8_t)(K); out[count].q0 = (uint8_t)(A);   \
            out[count].q1 = (uint8_t)(B); out[count].pad = 0;               \
            out[count].cycle = (uint32_t)(CYC); out[count].theta = 0.0;     \
        }                                                                   \
        ++count;                                                            \
    } while (0)

    for (int q = 0; q < n; ++q) EMIT(O_H, q, 0, 0);
    for (int t = 1; t <= depth; ++t) {
        int np = layout_pairs(rows, cols, dead, qubit_of_site, (t - 1) % 8, pair);
        memset(in_cz_now, 0, sizeof(int) * n);
        for (int i = 0; i < np; ++i) {
            EMIT(O_CZ, pair[2 * i], pair[2 * i + 1], t);
            in_cz_now[pair[2 * i]] = 1;
            in_cz_now[pair[2 * i + 1]] = 1;
        }
        for (int q = 0; q < n; ++q) {
            if (!in_cz_prev[q] || in_cz_now[q]) continue;
            int g;
            if (last_1q[q] < 0) {
                g = O_T;
            } else {
                int allowed[2], na = 0;
                const int menu[3] = {O_X_HALF, O_Y_HALF, O_T};
                for (int i = 0; i < 3; ++i)
                    if (menu[i] != last_1q[q]) allowed[na++] = menu[i];
                uint64_t z = splitmix_next(&rng);
                g = allowed[z >> 63];
            }
            EMIT(g, q, 0, t);
            last_1q[q] = g;
        }
        int *tmp = in_cz_prev; in_cz_prev = in_cz_now; in_cz_now = tmp;
    }
#undef EMIT
done:
    *ngates = count;
    free(qubit_of_site); free(pair); free(in_cz_prev); free(in_cz_now); free(last_1q);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Denser circuits of the appendix "Depth to reach Porter-Thomas for denser  */
/* 2D circuits": H on all qubits, then `layers` layers of (single-qubit      */
/* cycle, CZ cycle) on a rows x cols torus where each CZ cycle pairs every   */
/* qubit with one nearest neighbour.  Reading (the sequence is only said to  */
/* resemble Fig. two_dimers, with periodic boundaries): the four perfect     */
/* matchings, taken in the order of the sparse sequence H0 H2 V0 V2 H1 H3    */
/* V1 V3 with consecutive pairs merged, are                                  */
/*   0: horizontal bonds leaving an even column                              */
/*   1: vertical bonds leaving an even row                                   */
/*   2: horizontal bonds leaving an odd column (last column wraps to 0)      */
/*   3: vertical bonds leaving an odd row (last row wraps to 0)              */
/* Single-qubit placement follows Sec. "Convergence to Porter-Thomas": only  */
/* on qubits that were in a CZ in the previous cycle (so none in layer 1,    */
/* whose previous cycle is the H cycle), T first, then a pick from           */
/* {X^1/2, Y^1/2, T} without the previous gate (top bit of the next          */
/* SplitMix64 output).  Cycle numbers: 1q cycle of layer l = 2l-1, CZ cycle  */
/* = 2l.  Qubit of site (r, c) = r*cols + c.  Returns 0, -1 (bad arguments:  */
/* rows, cols even >= 2, at most 64 sites), -2 (cap too small).              */
/* ------------------------------------------------------------------------ */
int oracle_circuit_generate_dense(int rows, int cols, int layers, uint64_t seed,
                                  oracle_gate *out, size_t cap, size_t *ngates)
{
    if (!ngates || layers < 0 || rows < 2 || cols < 2 || rows % 2 || cols % 2 ||
        rows * cols > 64)
        return -1;
    const int n = rows * cols;
    int last_1q[64];
    for (int q = 0; q < n; ++q) last_1q[q] = -1;
    uint64_t rng = seed;
    size_t count = 0;
#define PUT(K, A, B, CYC)                                                   \
    do {                                                                    \
        if (out) {                                                          \
            if (count >= cap) { *ngates = count; return -2; }               \
            out[count].kind = (uint8_t)(K); out[count].q0 = (uint8_t)(A);   \
            out[count].q1 = (uint8_t)(B); out[count].pad = 0;               \
            out[count].cycle = (uint32_t)(CYC); out[count].theta = 0.0;     \
        }                                                                   \
        ++count;                                                            \
    } while (0)
    for (int q = 0; q < n; ++q) PUT(O_H, q, 0, 0);
    for (int layer = 1; layer <= layers; ++layer) {
        if (layer >= 2) {
            /* every qubit was in a CZ in the previous (CZ) cycle */
            for (int q = 0; q < n; ++q) {
                int g;
                if (last_1q[q] == -1) {
                    g = O_T;
                } else {
                    int allowed[2], na = 0;
                    if (last_1q[q] != O_X_HALF) allowed[na++] = O_X_HALF;
                    if (last_1q[q] != O_Y_HALF) allowed[na++] = O_Y_HALF;
                    if (last_1q[q] != O_T) allowed[na++] = O_T;
                    g = allowed[splitmix_next(&rng) >> 63];
                }
                PUT(g, q, 0, 2 * layer - 1);
                last_1q[q] = g;
            }
        }
        const int m = (layer - 1) % 4;
        for (int r = 0; r < rows; ++r) {
            for (int c = 0; c < cols; ++c) {
                int a = r * cols + c, b;
                if (m == 0 || m == 2) {            /* horizontal */
                    if (c % 2 != (m == 2)) continue;
                    b = r * cols + (c + 1) % cols;
                } else {                           /* vertical */
                    if (r % 2 != (m == 3)) continue;
                    b = ((r + 1) % rows) * cols + c;
                }
                PUT(O_CZ, a < b ? a : b, a < b ? b : a, 2 * layer);
            }
        }
    }
#undef PUT
    *ngates = count;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Digital error model (Sec. "Characterizing quantum supremacy", the         */
/* simulations with errors): a depolarising channel after every gate --      */
/* with probability r1 one of the 3 Paulis after a one-qubit gate, with      */
/* probability r2 one of the 15 non-identity two-qubit Paulis after a        */
/* two-qubit gate, all equally likely -- and an initialisation bit flip      */
/* with probability r_init per qubit.  One trajectory: draws are u = (z>>11) */
/* 2^-53 from one SplitMix64 stream seeded with `seed`, first one per qubit  */
/* (X before the circuit if u < r_init), then one per gate.  A one-qubit     */
/* error takes Pauli number floor(3u/r1) of (X, Y, Z); a two-qubit error     */
/* takes e = floor(15u/r2) + 1 in 1..15 and puts Pauli e/4 on the first      */
/* qubit and e%4 on the second (0 = none, 1..3 = X, Y, Z).  Paulis are       */
/* written as R_X(pi), R_Y(pi), R_Z(pi) (= -i times the Pauli; the global     */
/* phase leaves every probability unchanged).  Returns 0, -1 (bad           */
/* arguments), -2 (cap too small; *nout = needed count).                     */
/* ------------------------------------------------------------------------ */
int oracle_noisy_circuit(const oracle_gate *in, size_t ngates, int n, double r1, double r2,
                         double r_init, uint64_t seed, oracle_gate *out, size_t cap,
                         size_t *nout)
{
    if (!nout || n < 1 || n > 64 || r1 < 0 || r1 > 1 || r2 < 0 || r2 > 1 || r_init < 0 ||
        r_init > 1)
        return -1;
    uint64_t rng = seed;
    size_t count = 0;
    const int pauli_kind[4] = {-1, O_RX, O_RY, O_RZ};
#define APPEND(K, Q, CYC, TH)                                              \
    do {                                                                   \
        if (out && count < cap) {                                          \
            out[count].kind = (uint8_t)(K); out[count].q0 = (uint8_t)(Q);  \
            out[count].q1 = 0; out[count].pad = 0;                         \
            out[count].cycle = (uint32_t)(CYC); out[count].theta = (TH);   \
        }                                                                  \
        ++count;                                                           \
    } while (0)
    const uint32_t first_cycle = ngates ? in[0].cycle : 0;
    for (int q = 0; q < n; ++q) {
        double u = (double)(splitmix_next(&rng) >> 11) / 9007199254740992.0;
        if (u < r_init) APPEND(O_RX, q, first_cycle, M_PI);
    }
    for (size_t i = 0; i < ngates; ++i) {
        if (out && count < cap) out[count] = in[i];
        ++count;
        double u = (double)(splitmix_next(&rng) >> 11) / 9007199254740992.0;
        int two = in[i].kind == O_CZ || in[i].kind == O_CPHASE;
        if (two) {
            if (u < r2) {
                int e = (int)(15.0 * u / r2);
                if (e > 14) e = 14;
                e += 1;
                if (e / 4) APPEND(pauli_kind[e / 4], in[i].q0, in[i].cycle, M_PI);
                if (e % 4) APPEND(pauli_kind[e % 4], in[i].q1, in[i].cycle, M_PI);
            }
        } else if (u < r1) {
            int w = (int)(3.0 * u / r1);
            if (w > 2) w = 2;
            APPEND(pauli_kind[w + 1], in[i].q0, in[i].cycle, M_PI);
        }
    }
#undef APPEND
    *nout = count;
    return (out && count > cap) ? -2 : 0;
}

/* ------------------------------------------------------------------------ */
/* Gate matrices (Sec. "Convergence to Porter-Thomas"): X^1/2 and Y^1/2 are   */
/* pi/2 rotations about X and Y, T = diag(1, e^{i pi/4}), CZ = diag(1,1,1,-1).*/
/* Parameterised forms: R_P(theta) = exp(-i theta/2 P), CPHASE(phi) =        */
/* diag(1,1,1,e^{i phi}).  u is row-major [u11 u12; u21 u22].                */
/* For two-qubit kinds the 2x2 matrix is the one applied to the target when  */
/* the control bit is set.                                                   */
/* ------------------------------------------------------------------------ */
int oracle_gate_matrix(int kind, double theta, double complex u[4])
{
    const double s = 1.0 / sqrt(2.0);
    switch (kind) {
    case O_H:      u[0] = s; u[1] = s; u[2] = s; u[3] = -s; return 0;
    case O_X_HALF: u[0] = s; u[1] = -I * s; u[2] = -I * s; u[3] = s; return 0;
    case O_Y_HALF: u[0] = s; u[1] = -s; u[2] = s; u[3] = s; return 0;
    case O_T:      u[0] = 1; u[1] = 0; u[2] = 0; u[3] = cexp(I * M_PI / 4); return 0;
    case O_CZ:     u[0] = 1; u[1] = 0; u[2] = 0; u[3] = -1; return 0;
    case O_RX:
        u[0] = cos(theta / 2); u[1] = -I * sin(theta / 2);
        u[2] = -I * sin(theta / 2); u[3] = cos(theta / 2); return 0;
    case O_RY:
        u[0] = cos(theta / 2); u[1] = -sin(theta / 2);
        u[2] = sin(theta / 2); u[3] = cos(theta / 2); return 0;
    case O_RZ:
        u[0] = cexp(-I * theta / 2); u[1] = 0; u[2] = 0; u[3] = cexp(I * theta / 2);
        return 0;
    case O_CPHASE: u[0] = 1; u[1] = 0; u[2] = 0; u[3] = cexp(I * theta); return 0;
    default: return -1;
    }
}

/* Eq. sqgunitaryoperation: apply u to every pair of amplitudes whose indices
 * differ only in bit k. */
int oracle_apply_1q(double complex *psi, int n, int k, const double complex u[4])
{
    if (k < 0 || k >= n) return -1;
    uint64_t N = 1ULL << n, bit = 1ULL << k;
    /* every pair is updated independently: the loop may run on several
     * threads without changing any result */
#pragma omp parallel for schedule(static) if (n >= 16)
    for (uint64_t i = 0; i < N; ++i) {
        if (i & bit) continue;
        double complex a0 = psi[i], a1 = psi[i | bit];
        psi[i] = u[0] * a0 + u[1] * a1;
        psi[i | bit] = u[2] * a0 + u[3] * a1;
    }
    return 0;
}

/* Controlled-U (appendix "Quantum Simulation Details"): the same pair update
 * on target bit t, restricted to indices whose control bit c is set. */
int oracle_apply_controlled(double complex *psi, int n, int c, int t,
                            const double complex u[4])
{
    if (c < 0 || c >= n || t < 0 || t >= n || c == t) return -1;
    uint64_t N = 1ULL << n, cb = 1ULL << c, tb = 1ULL << t;
#pragma omp parallel for schedule(static) if (n >= 16)
    for (uint64_t i = 0; i < N; ++i) {
        if (!(i & cb) || (i & tb)) continue;
        double complex a0 = psi[i], a1 = psi[i | tb];
        psi[i] = u[0] * a0 + u[1] * a1;
        psi[i | tb] = u[2] * a0 + u[3] * a1;
    }
    return 0;
}

void oracle_state_zero(double complex *psi, int n)
{
    uint64_t N = 1ULL << n;
    for (uint64_t i = 0; i < N; ++i) psi[i] = 0;
    psi[0] = 1;
}

/* Applies the gate list in order.  Returns 0, or -1 on a malformed gate. */
int oracle_apply_circuit(double complex *psi, int n, const oracle_gate *g, size_t ng)
{
    double complex u[4];
    for (size_t i = 0; i < ng; ++i) {
        if (oracle_gate_matrix(g[i].kind, g[i].theta, u)) return -1;
        int rc;
        if (g[i].kind == O_CZ || g[i].kind == O_CPHASE)
            rc = oracle_apply_controlled(psi, n, g[i].q0, g[i].q1, u);
        else
            rc = oracle_apply_1q(psi, n, g[i].q0, u);
        if (rc) return -1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Output statistics                                                         */
/* ------------------------------------------------------------------------ */

/* p_U(x) = |<x|psi>|^2 */
void oracle_probabilities(const double complex *psi, int n, double *p)
{
    uint64_t N = 1ULL << n;
#pragma omp parallel for schedule(static) if (n >= 16)
    for (uint64_t i = 0; i < N; ++i) {
        double re = creal(psi[i]), im = cimag(psi[i]);
        p[i] = re * re + im * im;
    }
}

double oracle_norm(const double *p, int n)
{
    uint64_t N = 1ULL << n;
    double s = 0;
    for (uint64_t i = 0; i < N; ++i) s += p[i];
    return s;
}

/* Entropy H(p) = -sum p ln p (Eq. lps), with 0 ln 0 = 0. */
double oracle_entropy(const double *p, int n)
{
    uint64_t N = 1ULL << n;
    double s = 0;
    for (uint64_t i = 0; i < N; ++i)
        if (p[i] > 0) s -= p[i] * log(p[i]);
    return s;
}

/* Cross entropy of the uniform sampler with p (Eqs. 15 and eue with
 * p_cl = 1/N): -(1/N) sum ln p.  +inf if some p is exactly zero. */
double oracle_uniform_ce(const double *p, int n)
{
    uint64_t N = 1ULL << n;
    double s = 0;
    for (uint64_t i = 0; i < N; ++i) {
        if (p[i] <= 0) return INFINITY;
        s -= log(p[i]);
    }
    return s / (double)N;
}

/* Normalised inverse participation ratios (Sec. "Convergence to
 * Porter-Thomas"): out[k-1] = N^{k-1} sum_x p_x^k for k = 1..kmax, which the
 * Porter-Thomas distribution drives to k!. */
void oracle_moments(const double *p, int n, int kmax, double *out)
{
    uint64_t N = 1ULL << n;
    for (int k = 1; k <= kmax; ++k) {
        double s = 0;
        for (uint64_t i = 0; i < N; ++i) s += pow(p[i], k);
        out[k - 1] = s * pow((double)N, k - 1);
    }
}

/* Uniform deviate number j of a sampler stream: the top 53 bits of the j-th
 * SplitMix64 output, scaled to [0, 1). */
double oracle_sample_uniform(uint64_t seed, uint64_t j)
{
    uint64_t z = splitmix_finalise(seed + (j + 1) * 0x9E3779B97F4A7C15ULL);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

/* Inverse-CDF sampler: x_j = smallest i with C_i > u_j * C_{N-1}, where
 * C_i = sum_{t <= i} p_t accumulated in index order.  Returns 0, or -1 if the
 * total probability is not positive. */
int oracle_sample(const double *p, int n, uint64_t m, uint64_t seed, uint64_t *out)
{
    uint64_t N = 1ULL << n;
    double *C = (double *)malloc(sizeof(double) * N);
    if (!C) return -2;
    double acc = 0;
    for (uint64_t i = 0; i < N; ++i) { acc += p[i]; C[i] = acc; }
    if (!(acc > 0)) { free(C); return -1; }
    for (uint64_t j = 0; j < m; ++j) {
        double target = oracle_sample_uniform(seed, j) * acc;
        uint64_t lo = 0, hi = N - 1;      /* C[hi] = acc > target always */
        while (lo < hi) {
            uint64_t mid = lo + (hi - lo) / 2;
            if (C[mid] > target) hi = mid; else lo = mid + 1;
        }
        out[j] = lo;
    }
    free(C);
    return 0;
}

/* Sample estimate of the cross entropy (Eq. ae):
 *   CE = (1/m) sum_j ln(1/p(x_j)),   Delta H = H_0 - CE,  H_0 = ln N + gamma.
 * Returns CE; *delta_h receives Delta H. */
double oracle_cross_entropy(const double *p, int n, const uint64_t *x, uint64_t m,
                            double *delta_h)
{
    const double euler_gamma = 0.57721566490153286061;
    uint64_t N = 1ULL << n;
    double s = 0;
    for (uint64_t j = 0; j < m; ++j) {
        if (x[j] >= N) { if (delta_h) *delta_h = NAN; return NAN; }
        s -= log(p[x[j]]);
    }
    double ce = s / (double)m;
    if (delta_h) *delta_h = (double)n * log(2.0) + euler_gamma - ce;
    return ce;
}
