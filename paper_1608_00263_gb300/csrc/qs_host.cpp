// qs_host.cpp -- host-side parts of the library: error strings, gate
// definitions and validation, the random-circuit generator, and the fused
// pass planner.  No CUDA calls.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "qs_internal.h"

namespace qs {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

qs_status set_error(qs_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

void clear_error() { g_last_error.clear(); }

const char *last_error_cstr() { return g_last_error.c_str(); }

size_t dtype_bytes(qs_dtype dt) { return dt == QS_C128 ? 16 : 8; }

// ---------------------------------------------------------------------------
// gates (Sec. "Convergence to Porter-Thomas": H, X^1/2 and Y^1/2 as pi/2
// rotations, T = diag(1, e^{i pi/4}), CZ = diag(1,1,1,-1); parameterised
// R_P(theta) = exp(-i theta/2 P) and CPHASE(phi) = diag(1,1,1,e^{i phi}))
// ---------------------------------------------------------------------------
bool gate_is_two_qubit(int kind) { return kind == QS_CZ || kind == QS_CPHASE; }

bool gate_is_diagonal(int kind)
{
    return kind == QS_T || kind == QS_CZ || kind == QS_RZ || kind == QS_CPHASE;
}

void gate_matrix(int kind, double theta, Cplx u[4])
{
    const double h = std::sqrt(0.5);
    const double c = std::cos(theta / 2), s = std::sin(theta / 2);
    for (int i = 0; i < 4; ++i) u[i] = {0, 0};
    switch (kind) {
    case QS_H: u[0] = {h, 0}; u[1] = {h, 0}; u[2] = {h, 0}; u[3] = {-h, 0}; break;
    case QS_X_HALF: u[0] = {h, 0}; u[1] = {0, -h}; u[2] = {0, -h}; u[3] = {h, 0}; break;
    case QS_Y_HALF: u[0] = {h, 0}; u[1] = {-h, 0}; u[2] = {h, 0}; u[3] = {h, 0}; break;
    case QS_T: u[0] = {1, 0}; u[3] = {h, h}; break;
    case QS_CZ: u[0] = {1, 0}; u[3] = {-1, 0}; break;
    case QS_RX: u[0] = {c, 0}; u[1] = {0, -s}; u[2] = {0, -s}; u[3] = {c, 0}; break;
    case QS_RY: u[0] = {c, 0}; u[1] = {-s, 0}; u[2] = {s, 0}; u[3] = {c, 0}; break;
    case QS_RZ: u[0] = {c, -s}; u[3] = {c, s}; break;
    case QS_CPHASE: u[0] = {1, 0}; u[3] = {std::cos(theta), std::sin(theta)}; break;
    default: break;
    }
}

size_t leading_h_layer(const qs_gate *g, size_t ng, int n)
{
    if (ng < (size_t)n) return 0;
    uint64_t seen = 0;
    for (int i = 0; i < n; ++i) {
        if (g[i].kind != QS_H) return 0;
        const uint64_t b = 1ULL << g[i].q0;
        if (seen & b) return 0;
        seen |= b;
    }
    return (size_t)n;
}

size_t fold_diagonal_prefix(const qs_gate *g, size_t ng, std::vector<qs_gate> *rest, FoldArgs *f)
{
    std::memset(f, 0, sizeof(*f));
    rest->clear();
    rest->reserve(ng);
    uint64_t touched = 0;       // qubits that have met a non-diagonal gate
    uint8_t tcount[kMaxQubits] = {0};
    size_t nf = 0;
    for (size_t i = 0; i < ng; ++i) {
        const qs_gate &x = g[i];
        const uint64_t a = 1ULL << x.q0;
        const uint64_t b = gate_is_two_qubit(x.kind) ? 1ULL << x.q1 : 0;
        if (x.kind == QS_T && !(touched & a)) {
            tcount[x.q0] = (uint8_t)((tcount[x.q0] + 1) & 7);
            ++nf;
        } else if (x.kind == QS_CZ && !(touched & (a | b))) {
            f->nb[x.q0] ^= b;
            f->nb[x.q1] ^= a;
            ++nf;
        } else {
            // diagonal gates left in the list (T or CZ on a touched qubit,
            // RZ, CPHASE) commute with the folded ones and touch nothing
            if (x.kind != QS_T && x.kind != QS_CZ && x.kind != QS_RZ && x.kind != QS_CPHASE) touched |= a | b;
            rest->push_back(x);
        }
    }
    for (int q = 0; q < kMaxQubits; ++q) {
        if (tcount[q] & 1) f->m1 |= 1ULL << q;
        if (tcount[q] & 2) f->m2 |= 1ULL << q;
        if (tcount[q] & 4) f->m4 |= 1ULL << q;
    }
    f->nfold = (int)nf;
    return nf;
}

qs_status validate_gates(int n, const qs_gate *g, size_t ng)
{
    if (ng && !g) return set_error(QS_ERR_INVALID_ARG, "gates is NULL but ngates = %zu", ng);
    for (size_t i = 0; i < ng; ++i) {
        if (g[i].kind > QS_CPHASE)
            return set_error(QS_ERR_INVALID_ARG, "gate %zu: unknown kind %u", i, g[i].kind);
        if (g[i].q0 >= n)
            return set_error(QS_ERR_INVALID_ARG, "gate %zu: qubit %u >= n = %d", i, g[i].q0, n);
        if (gate_is_two_qubit(g[i].kind)) {
            if (g[i].q1 >= n)
                return set_error(QS_ERR_INVALID_ARG, "gate %zu: qubit %u >= n = %d", i, g[i].q1, n);
            if (g[i].q0 == g[i].q1)
                return set_error(QS_ERR_INVALID_ARG, "gate %zu: two-qubit gate on equal qubits %u",
                                 i, g[i].q0);
        }
        if (!std::isfinite(g[i].theta))
            return set_error(QS_ERR_INVALID_ARG, "gate %zu: non-finite angle", i);
    }
    return QS_OK;
}

// ---------------------------------------------------------------------------
// random circuits (Sec. "Convergence to Porter-Thomas")
// ---------------------------------------------------------------------------
namespace {

// SplitMix64 (Steele, Lea & Flood 2014): Weyl step by the golden gamma,
// then the 64-bit finaliser.
struct SplitMix64 {
    uint64_t x;
    explicit SplitMix64(uint64_t seed) : x(seed) {}
    uint64_t next()
    {
        x += 0x9E3779B97F4A7C15ULL;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
};

struct Grid {
    int rows, cols;
    std::vector<int> qubit;   // site -> qubit or -1
    int n = 0;
    Grid(int r, int c, const uint8_t *dead) : rows(r), cols(c), qubit(r * c, -1)
    {
        for (int s = 0; s < r * c; ++s)
            if (!(dead && dead[s])) qubit[s] = n++;
    }
    // CZ pairs of one of the eight layouts.  Layout order H0 H2 V0 V2 H1 H3
    // V1 V3; H_a: edges (r,c)-(r,c+1) with (c + 2r) % 4 == a; V_a: edges
    // (r,c)-(r+1,c) with (r + 2c) % 4 == a.
    std::vector<std::pair<int, int>> layout(int which) const
    {
        static const bool vertical[8] = {false, false, true, true, false, false, true, true};
        static const int offset[8] = {0, 2, 0, 2, 1, 3, 1, 3};
        std::vector<std::pair<int, int>> out;
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < cols; ++c) {
                int r2 = r, c2 = c;
                if (vertical[which]) {
                    if ((r + 2 * c) % 4 != offset[which]) continue;
                    r2 = r + 1;
                } else {
                    if ((c + 2 * r) % 4 != offset[which]) continue;
                    c2 = c + 1;
                }
                if (r2 >= rows || c2 >= cols) continue;
                int a = qubit[r * cols + c], b = qubit[r2 * cols + c2];
                if (a < 0 || b < 0) continue;
                out.emplace_back(std::min(a, b), std::max(a, b));
            }
        return out;
    }
};

}  // namespace

}  // namespace qs

using namespace qs;

extern "C" const char *qs_last_error(void) { return last_error_cstr(); }

extern "C" qs_status qs_circuit_generate(int rows, int cols, const uint8_t *dead,
                                         int depth, uint64_t seed, qs_gate *out,
                                         size_t *ngates)
{
    clear_error();
    if (rows < 1 || cols < 1 || rows * (int64_t)cols > 4096)
        return set_error(QS_ERR_INVALID_ARG, "bad grid %d x %d", rows, cols);
    if (depth < 0) return set_error(QS_ERR_INVALID_ARG, "negative depth");
    if (!ngates) return set_error(QS_ERR_INVALID_ARG, "ngates is NULL");
    Grid grid(rows, cols, dead);
    if (grid.n < 1 || grid.n > 64)
        return set_error(QS_ERR_INVALID_ARG, "grid has %d live sites (1..64 allowed)", grid.n);
    const size_t cap = out ? *ngates : 0;
    size_t count = 0;
    auto emit = [&](int kind, int a, int b, int cycle) {
        if (out && count < cap) {
            qs_gate &g = out[count];
            g.kind = (uint8_t)kind; g.q0 = (uint8_t)a; g.q1 = (uint8_t)b; g.pad = 0;
            g.cycle = (uint32_t)cycle; g.theta = 0.0;
        }
        ++count;
    };
    SplitMix64 rng(seed);
    const int n = grid.n;
    std::vector<char> busy_prev(n, 0), busy(n, 0);
    std::vector<int> previous(n, -1);   // last single-qubit gate since H
    for (int q = 0; q < n; ++q) emit(QS_H, q, 0, 0);
    for (int t = 1; t <= depth; ++t) {
        std::fill(busy.begin(), busy.end(), 0);
        for (auto &e : grid.layout((t - 1) % 8)) {
            emit(QS_CZ, e.first, e.second, t);
            busy[e.first] = busy[e.second] = 1;
        }
        for (int q = 0; q < n; ++q) {
            if (!busy_prev[q] || busy[q]) continue;
            int kind;
            if (previous[q] < 0) {
                kind = QS_T;
            } else {
                int choices[2], m = 0;
                for (int k : {QS_X_HALF, QS_Y_HALF, QS_T})
                    if (k != previous[q]) choices[m++] = k;
                kind = choices[rng.next() >> 63];
            }
            emit(kind, q, 0, t);
            previous[q] = kind;
        }
        busy_prev.swap(busy);
    }
    if (out && count > cap) {
        *ngates = count;
        return set_error(QS_ERR_INVALID_ARG, "output holds %zu gates, circuit has %zu", cap, count);
    }
    *ngates = count;
    return QS_OK;
}

// Dense layouts with periodic boundaries (appendix "Depth to reach
// Porter-Thomas for denser 2D circuits"): on an even rows x cols torus the
// CZ cycle of layer l uses pattern (l-1) mod 4 of
//   H_even: (r,c)-(r,c+1), c even      V_even: (r,c)-(r+1,c), r even
//   H_odd:  (r,c)-(r,c+1 mod cols), c odd
//   V_odd:  (r,c)-(r+1 mod rows,c), r odd
// so every qubit is in exactly one CZ per CZ cycle (the eight sparse
// layouts merged in consecutive pairs).  Layer l: cycle 2l-1 single-qubit
// gates under the rules of Sec. "Convergence to Porter-Thomas" (a gate only
// on a qubit in a CZ in the previous cycle, T first after H, then different
// from the previous one), cycle 2l the CZ cycle.
extern "C" qs_status qs_circuit_generate_dense(int rows, int cols, int layers, uint64_t seed,
                                               qs_gate *out, size_t *ngates)
{
    clear_error();
    if (rows < 2 || cols < 2 || (rows & 1) || (cols & 1) || rows * cols > 64)
        return set_error(QS_ERR_INVALID_ARG, "dense layouts need an even torus of <= 64 sites, got %d x %d",
                         rows, cols);
    if (layers < 0) return set_error(QS_ERR_INVALID_ARG, "negative layer count");
    if (!ngates) return set_error(QS_ERR_INVALID_ARG, "ngates is NULL");
    const int n = rows * cols;
    const size_t cap = out ? *ngates : 0;
    size_t count = 0;
    auto emit = [&](int kind, int a, int b, int cycle) {
        if (out && count < cap) {
            qs_gate &g = out[count];
            g.kind = (uint8_t)kind; g.q0 = (uint8_t)a; g.q1 = (uint8_t)b; g.pad = 0;
            g.cycle = (uint32_t)cycle; g.theta = 0.0;
        }
        ++count;
    };
    SplitMix64 rng(seed);
    std::vector<int> previous(n, -1);
    for (int q = 0; q < n; ++q) emit(QS_H, q, 0, 0);
    for (int l = 1; l <= layers; ++l) {
        // the previous cycle was a CZ cycle covering every qubit, except
        // before layer 1 (the H cycle)
        if (l > 1) {
            for (int q = 0; q < n; ++q) {
                int kind;
                if (previous[q] < 0) {
                    kind = QS_T;
                } else {
                    int choices[2], m = 0;
                    for (int k : {QS_X_HALF, QS_Y_HALF, QS_T})
                        if (k != previous[q]) choices[m++] = k;
                    kind = choices[rng.next() >> 63];
                }
                emit(kind, q, 0, 2 * l - 1);
                previous[q] = kind;
            }
        }
        const int pat = (l - 1) % 4;
        const bool vert = pat & 1, odd = pat >= 2;
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < cols; ++c) {
                if ((vert ? r : c) % 2 != (odd ? 1 : 0)) continue;
                const int r2 = vert ? (r + 1) % rows : r, c2 = vert ? c : (c + 1) % cols;
                const int a = r * cols + c, b = r2 * cols + c2;
                emit(QS_CZ, std::min(a, b), std::max(a, b), 2 * l);
            }
    }
    if (out && count > cap) {
        *ngates = count;
        return set_error(QS_ERR_INVALID_ARG, "output holds %zu gates, circuit has %zu", cap, count);
    }
    *ngates = count;
    return QS_OK;
}

// Digital error model of Sec. "Characterizing quantum supremacy" (the
// depolarising channel after each gate): one trajectory of the channel.
// Draws come from one SplitMix64 stream seeded with `seed`, u = (z >> 11)
// 2^-53 per draw, in this order: one draw per qubit for the initialisation
// bit flip (X if u < r_init), then one draw per gate of the list: after a
// one-qubit gate, if u < r1 the Pauli floor(3u / r1) of (X, Y, Z); after a
// two-qubit gate, if u < r2 the pair number e = floor(15u / r2) + 1 (base-4
// digits (e / 4, e % 4) = (P on q0, P on q1), 0 = I, 1..3 = X, Y, Z).
// Paulis are emitted as R_X(pi), R_Y(pi), R_Z(pi) (the Pauli up to the global
// phase -i), in the cycle of the gate they follow.
extern "C" qs_status qs_noisy_circuit(const qs_gate *gates, size_t ngates, int n, double r1, double r2,
                                      double r_init, uint64_t seed, qs_gate *out, size_t *nout)
{
    clear_error();
    if (!nout || n < 1 || n > 64) return set_error(QS_ERR_INVALID_ARG, "bad arguments");
    if (!(r1 >= 0 && r1 <= 1 && r2 >= 0 && r2 <= 1 && r_init >= 0 && r_init <= 1))
        return set_error(QS_ERR_INVALID_ARG, "error rates must lie in [0, 1]");
    if (qs_status st = validate_gates(n, gates, ngates)) return st;
    const size_t cap = out ? *nout : 0;
    size_t count = 0;
    auto put = [&](const qs_gate &g) {
        if (out && count < cap) out[count] = g;
        ++count;
    };
    auto pauli = [&](int which, int q, uint32_t cycle) {   // which: 1 X, 2 Y, 3 Z
        static const int kind[4] = {-1, QS_RX, QS_RY, QS_RZ};
        qs_gate g{};
        g.kind = (uint8_t)kind[which]; g.q0 = (uint8_t)q; g.cycle = cycle; g.theta = M_PI;
        put(g);
    };
    SplitMix64 rng(seed);
    auto uniform = [&]() { return (double)(rng.next() >> 11) * (1.0 / 9007199254740992.0); };
    const uint32_t c0 = ngates ? gates[0].cycle : 0;
    for (int q = 0; q < n; ++q)
        if (uniform() < r_init) pauli(1, q, c0);
    for (size_t i = 0; i < ngates; ++i) {
        const qs_gate &g = gates[i];
        put(g);
        const double u = uniform();
        if (gate_is_two_qubit(g.kind)) {
            if (u < r2) {
                const int e = std::min(14, (int)(15.0 * u / r2)) + 1;
                if (e / 4) pauli(e / 4, g.q0, g.cycle);
                if (e % 4) pauli(e % 4, g.q1, g.cycle);
            }
        } else if (u < r1) {
            pauli(std::min(2, (int)(3.0 * u / r1)) + 1, g.q0, g.cycle);
        }
    }
    if (out && count > cap) {
        *nout = count;
        return set_error(QS_ERR_INVALID_ARG, "output holds %zu gates, trajectory has %zu", cap, count);
    }
    *nout = count;
    return QS_OK;
}

// One discrete error (appendix "Residual correlations after discrete
// errors"): the gate list with Pauli `pauli` (1 X, 2 Y, 3 Z, written as
// R_P(pi)) on `qubit` inserted after the last gate whose cycle is <= `cycle`.
extern "C" qs_status qs_single_error_circuit(const qs_gate *gates, size_t ngates, int n, uint32_t cycle,
                                             int qubit, int pauli, qs_gate *out, size_t *nout)
{
    clear_error();
    if (!nout || qubit < 0 || qubit >= n || pauli < 1 || pauli > 3)
        return set_error(QS_ERR_INVALID_ARG, "bad arguments");
    if (qs_status st = validate_gates(n, gates, ngates)) return st;
    const size_t need = ngates + 1;
    if (out && *nout < need) {
        *nout = need;
        return set_error(QS_ERR_INVALID_ARG, "output holds %zu gates, need %zu", *nout, need);
    }
    *nout = need;
    if (!out) return QS_OK;
    size_t at = 0;
    while (at < ngates && gates[at].cycle <= cycle) ++at;
    static const int kind[4] = {-1, QS_RX, QS_RY, QS_RZ};
    for (size_t i = 0; i < at; ++i) out[i] = gates[i];
    qs_gate e{};
    e.kind = (uint8_t)kind[pauli]; e.q0 = (uint8_t)qubit; e.cycle = cycle; e.theta = M_PI;
    out[at] = e;
    for (size_t i = at; i < ngates; ++i) out[i + 1] = gates[i];
    return QS_OK;
}

// First index i of an entropy series such that every entry from i on lies
// within 4 sigma of the Porter-Thomas entropy ln N - 1 + gamma, sigma =
// 0.75 * 2^(-n/2) (Sec. "Convergence to Porter-Thomas", Fig. pt_depth).
extern "C" qs_status qs_pt_convergence(const double *entropy, size_t count, int n, size_t *first)
{
    clear_error();
    if ((count && !entropy) || !first || n < 1 || n > 64)
        return set_error(QS_ERR_INVALID_ARG, "bad arguments");
    const double h_pt = n * std::log(2.0) - 1.0 + 0.57721566490153286061;
    const double tol = 4.0 * 0.75 * std::pow(2.0, -0.5 * n);
    size_t i = count;
    while (i > 0 && std::fabs(entropy[i - 1] - h_pt) <= tol) --i;
    *first = i;
    return QS_OK;
}

namespace qs {

// ---------------------------------------------------------------------------
// planner
//
// A pass keeps t qubits ("tile qubits", always including the c lowest for
// coalesced runs) local: every CTA owns the 2^t amplitudes that share the
// values of the other n - t qubits.  Non-diagonal gates need their qubit in
// the tile; diagonal gates (T, CZ, RZ, CPHASE) never do, because the bits of
// out-of-tile qubits are constant per tile (the appendix's observation that
// diagonal gates need no communication).  A pass applies, in circuit order,
// every pending gate whose qubits are not blocked; a gate that cannot be
// applied blocks its qubits for the rest of the pass, so the applied set is
// closed under dependencies.  Inside a pass the same rule with r "register"
// qubits splits the gates into phases; each phase is one shared-memory round
// trip of the tile.
// ---------------------------------------------------------------------------
namespace {

struct PGate {
    int kind;
    int q0, q1;
    bool two, diag;
    double theta;
};

// Returns the indices (in order) of gates applicable with the local set
// `local` (bitmask over qubits), among gates not yet done.  A gate left
// pending blocks its qubits for the later gates that do not commute with it:
// a non-diagonal gate for every later gate on its qubit, a diagonal gate only
// for later non-diagonal gates (diagonal gates commute with each other).
// The scan stops once every qubit of `allq` is blocked for all gates: no
// later gate can then apply.
static void collect(const std::vector<PGate> &g, const std::vector<int> &cand,
                    const std::vector<char> &done, uint64_t local,
                    std::vector<int> *out, int *count, uint64_t allq = ~0ULL)
{
    uint64_t blocked = 0;      // a non-diagonal gate is pending on the qubit
    uint64_t blocked_nd = 0;   // a diagonal gate is pending on the qubit
    int cnt = 0;
    if (out) out->clear();
    for (int i : cand) {
        if (done[i]) continue;
        if (blocked == allq) break;
        const PGate &x = g[i];
        uint64_t qm = (1ULL << x.q0) | (x.two ? (1ULL << x.q1) : 0);
        bool ok = !(qm & blocked) && (x.diag || ((qm & ~local) == 0 && !(qm & blocked_nd)));
        if (ok) {
            ++cnt;
            if (out) out->push_back(i);
        } else if (x.diag) {
            blocked_nd |= qm;
        } else {
            blocked |= qm;
        }
    }
    *count = cnt;
}

// First pending non-diagonal gate index per qubit (large if none).
static void first_pending(const std::vector<PGate> &g, const std::vector<int> &cand,
                          const std::vector<char> &done, int n, std::vector<int> *first)
{
    first->assign(n, 1 << 30);
    for (int i : cand) {
        if (done[i] || g[i].diag) continue;
        int q = g[i].q0;
        if ((*first)[q] > i) (*first)[q] = i;
    }
}

// Pending diagonal gates per qubit.
static void diag_pending(const std::vector<PGate> &g, const std::vector<int> &cand,
                         const std::vector<char> &done, int n, std::vector<int> *cnt)
{
    cnt->assign(n, 0);
    for (int i : cand) {
        if (done[i] || !g[i].diag) continue;
        ++(*cnt)[g[i].q0];
        if (g[i].two) ++(*cnt)[g[i].q1];
    }
}

// Greedy choice of `want` qubits added to `base` from `pool`, maximising the
// number of applicable gates; ties go to the qubit whose next non-diagonal
// gate is earliest, then to the qubit with the fewest pending diagonal gates
// (a register phase applies those to whole threads when their qubits are
// not register bits).
static uint64_t choose_local(const std::vector<PGate> &g, const std::vector<int> &cand,
                             const std::vector<char> &done, int n, uint64_t base,
                             uint64_t pool, int want, uint64_t allq = ~0ULL)
{
    std::vector<int> first, ndiag;
    first_pending(g, cand, done, n, &first);
    diag_pending(g, cand, done, n, &ndiag);
    uint64_t local = base;
    for (int step = 0; step < want; ++step) {
        int best_q = -1, best_cnt = -1, best_first = 1 << 30, best_diag = 1 << 30;
        for (int q = 0; q < n; ++q) {
            if (!((pool >> q) & 1) || ((local >> q) & 1)) continue;
            int cnt;
            collect(g, cand, done, local | (1ULL << q), nullptr, &cnt, allq);
            if (cnt > best_cnt || (cnt == best_cnt && (first[q] < best_first ||
                                                       (first[q] == best_first && ndiag[q] < best_diag)))) {
                best_q = q; best_cnt = cnt; best_first = first[q]; best_diag = ndiag[q];
            }
        }
        if (best_q < 0) break;
        local |= 1ULL << best_q;
    }
    return local;
}

// Tile choice of a pass with a lookahead: for the first `look_steps`
// additions, the `look_top` candidates with the most applicable gates are
// each completed greedily to the full tile and scored by the gates the
// completed tile applies; the remaining additions are greedy.  Fewer passes
// than the plain greedy choice on the paper's circuits: 10 % at 30 qubits
// (8 steps, 8 candidates, ~40 ms of host time against ~80 ms of evolution),
// 14 % at 34 qubits (every step and candidate, ~0.2 s against ~1.4 s).
// Host planning of the next circuit overlaps the current evolution.
static uint64_t choose_tile(const std::vector<PGate> &g, const std::vector<int> &cand,
                            const std::vector<char> &done, int n, uint64_t base, uint64_t pool,
                            int want, uint64_t allq, int look_steps, int look_top)
{
    uint64_t local = base;
    for (int step = 0; step < want && step < look_steps; ++step) {
        std::vector<int> first;
        first_pending(g, cand, done, n, &first);
        struct C { int cnt, first, q; };
        std::vector<C> cs;
        for (int q = 0; q < n; ++q) {
            if (!((pool >> q) & 1) || ((local >> q) & 1)) continue;
            int cnt;
            collect(g, cand, done, local | (1ULL << q), nullptr, &cnt, allq);
            cs.push_back({cnt, first[q], q});
        }
        if (cs.empty()) return local;
        std::sort(cs.begin(), cs.end(), [](const C &a, const C &b) {
            return a.cnt != b.cnt ? a.cnt > b.cnt : (a.first != b.first ? a.first < b.first : a.q < b.q);
        });
        if ((int)cs.size() > look_top) cs.resize(look_top);
        int best_q = -1, best = -1;
        for (const C &c : cs) {
            const uint64_t full = choose_local(g, cand, done, n, local | (1ULL << c.q), pool, want - step - 1, allq);
            int cnt;
            collect(g, cand, done, full, nullptr, &cnt, allq);
            if (cnt > best) { best = cnt; best_q = c.q; }
        }
        local |= 1ULL << best_q;
    }
    const int added = __builtin_popcountll(local & ~base);
    return choose_local(g, cand, done, n, local, pool, want - added, allq);
}

// Shared-memory wavefronts of one phase's slot loads (the stores mirror
// them).  A warp's shared access is served per group of lanes -- 16 lanes
// for 8-byte accesses, 8 for 16-byte ones -- and a group costs the largest
// number of distinct 4-byte words that fall in one bank.  The group's lanes
// differ in the `g` tile bits `grp`; the other lane bits and every register
// slot only XOR a constant into the (linear) swizzled addresses, which
// permutes the banks, so one group of slot 0 gives the cost of all.
static int group_wavefronts(const int *grp, int g, int esz, bool paired)
{
    const uint32_t CE = 16 / esz;
    const int per = (paired ? 16 : esz) / 4;   // 4-byte words per lane access
    uint32_t w[16 * 4];
    int nw = 0;
    for (int l = 0; l < (1 << g); ++l) {
        uint32_t e = 0;
        for (int k = 0; k < g; ++k) e |= (uint32_t)((l >> k) & 1) << grp[k];
        const uint32_t w0 = tile_swizzle(e, CE) * (uint32_t)esz / 4;
        for (int i = 0; i < per; ++i) w[nw++] = w0 + (uint32_t)i;
    }
    std::sort(w, w + nw);
    nw = (int)(std::unique(w, w + nw) - w);
    int cnt[32] = {0}, worst = 0;
    for (int i = 0; i < nw; ++i) worst = std::max(worst, ++cnt[w[i] & 31]);
    return worst;
}

// Thread-bit order of a register phase: among the non-register tile bits,
// the lowest lane bits (4 for 8-byte slot accesses, 3 for 16-byte ones) are
// the set that minimises the lane group's shared-memory wavefronts (ties keep
// the lowest bits); the remaining non-register bits follow in ascending order.
static void choose_thread_bits(const uint8_t *R, int r, int t, int esz, uint8_t *T)
{
    int tb[kMaxTileBits], nt = 0;
    for (int b = 0; b < t; ++b) {
        bool reg = false;
        for (int j = 0; j < r; ++j) reg |= R[j] == b;
        if (!reg) tb[nt++] = b;
    }
    const bool paired = esz == 8 && R[0] == 0;
    const int g = std::min(paired || esz == 16 ? 3 : 4, nt);
    int best_mask = (1 << g) - 1, best = 1 << 30;
    for (int m = 0; m < (1 << nt); ++m) {
        if (__builtin_popcount(m) != g) continue;
        int grp[4], k = 0;
        for (int i = 0; i < nt; ++i)
            if ((m >> i) & 1) grp[k++] = tb[i];
        const int c = group_wavefronts(grp, g, esz, paired);
        if (c < best || (c == best && m < best_mask)) { best = c; best_mask = m; }
    }
    int k = 0;
    for (int i = 0; i < nt; ++i)
        if ((best_mask >> i) & 1) T[k++] = (uint8_t)tb[i];
    for (int i = 0; i < nt; ++i)
        if (!((best_mask >> i) & 1)) T[k++] = (uint8_t)tb[i];
}

static int popcount64(uint64_t x) { return __builtin_popcountll(x); }

// A tensor-core block phase is chosen when it absorbs at least this many
// gates and at least this fraction of what the best register phase would.
constexpr int kTcMinGates = 8;
constexpr double kTcRegRatio = 0.6;

// Gates absorbable into a tensor-core block on qubit set `block`: like
// collect(), but a diagonal gate also needs all its qubits in the block (a
// diagonal gate reaching outside would make the block operator differ
// between the columns of the tile).
static void collect_tc(const std::vector<PGate> &g, const std::vector<int> &cand,
                       const std::vector<char> &done, uint64_t block,
                       std::vector<int> *out, int *count)
{
    uint64_t blocked = 0;
    int cnt = 0;
    if (out) out->clear();
    for (int i : cand) {
        if (done[i]) continue;
        const PGate &x = g[i];
        uint64_t qm = (1ULL << x.q0) | (x.two ? (1ULL << x.q1) : 0);
        bool ok = !(qm & blocked) && (qm & ~block) == 0;
        if (ok) {
            ++cnt;
            if (out) out->push_back(i);
        } else {
            blocked |= qm;
        }
    }
    *count = cnt;
}

static uint64_t choose_tc_block(const std::vector<PGate> &g, const std::vector<int> &cand,
                                const std::vector<char> &done, int n, uint64_t pool, int want)
{
    std::vector<int> first;
    first_pending(g, cand, done, n, &first);
    uint64_t block = 0;
    for (int step = 0; step < want; ++step) {
        int best_q = -1, best_cnt = -1, best_first = 1 << 30;
        for (int q = 0; q < n; ++q) {
            if (!((pool >> q) & 1) || ((block >> q) & 1)) continue;
            int cnt;
            collect_tc(g, cand, done, block | (1ULL << q), nullptr, &cnt);
            if (cnt > best_cnt || (cnt == best_cnt && first[q] < best_first)) {
                best_q = q; best_cnt = cnt; best_first = first[q];
            }
        }
        if (best_q < 0) break;
        block |= 1ULL << best_q;
    }
    return block;
}

// Order of the block bits of a tensor-core phase.  The accumulator leaves
// tensor memory one row per lane: a warp holds block rows 16w'..16w'+15
// (index bits 0..3), real and imaginary parts on neighbouring lanes, and
// stores them as 4-byte words.  The four block bits put on index bits 0..3
// are the ones whose swizzled words fall in the fewest rounds per bank (zero
// conflicts when they spread over all banks); the other two follow.
static void order_tc_block(int *bq, uint8_t *R)
{
    int best = 1 << 30, best_m = 0x0f;
    for (int m = 0; m < (1 << kTcBits); ++m) {
        if (__builtin_popcount(m) != 4) continue;
        int sel[4], k = 0;
        for (int j = 0; j < kTcBits; ++j)
            if ((m >> j) & 1) sel[k++] = R[j];
        uint32_t w[32];
        for (int i = 0; i < 16; ++i) {
            uint32_t e = 0;
            for (int b = 0; b < 4; ++b) e |= (uint32_t)((i >> b) & 1) << sel[b];
            const uint32_t x = tile_swizzle(e, 2);
            w[2 * i] = 2 * x;
            w[2 * i + 1] = 2 * x + 1;
        }
        int cnt[32] = {0}, worst = 0;
        for (int i = 0; i < 32; ++i) worst = std::max(worst, ++cnt[w[i] & 31]);
        if (worst < best || (worst == best && m < best_m)) { best = worst; best_m = m; }
    }
    int nb[kTcBits];
    uint8_t nr[kTcBits];
    int k = 0;
    for (int pass = 0; pass < 2; ++pass)
        for (int j = 0; j < kTcBits; ++j)
            if ((((best_m >> j) & 1) != 0) == (pass == 0)) { nb[k] = bq[j]; nr[k] = R[j]; ++k; }
    for (int j = 0; j < kTcBits; ++j) { bq[j] = nb[j]; R[j] = nr[j]; }
}

// Block unitary (64 x 64, row-major, complex as re/im pairs) of `gates` on
// block qubits bq[0..5] (block bit j <-> qubit bq[j]), applied in order.
static void block_unitary(const std::vector<PGate> &g, const std::vector<int> &gates,
                          const int *bq, std::vector<Cplx> *U)
{
    const int D = 1 << kTcBits;
    U->assign((size_t)D * D, Cplx{0, 0});
    for (int i = 0; i < D; ++i) (*U)[(size_t)i * D + i] = {1, 0};
    auto bit_of = [&](int q) {
        for (int j = 0; j < kTcBits; ++j)
            if (bq[j] == q) return j;
        return -1;
    };
    auto mul = [](Cplx a, Cplx b) { return Cplx{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; };
    auto add = [](Cplx a, Cplx b) { return Cplx{a.re + b.re, a.im + b.im}; };
    for (int gi : gates) {
        const PGate &x = g[gi];
        Cplx u[4];
        gate_matrix(x.kind, x.theta, u);
        if (x.two) {
            const int ja = bit_of(x.q0), jb = bit_of(x.q1);
            for (int r = 0; r < D; ++r)
                if (((r >> ja) & 1) && ((r >> jb) & 1))
                    for (int c = 0; c < D; ++c) (*U)[(size_t)r * D + c] = mul(u[3], (*U)[(size_t)r * D + c]);
        } else {
            const int j = bit_of(x.q0);
            for (int r = 0; r < D; ++r) {
                if ((r >> j) & 1) continue;
                const int r1 = r | (1 << j);
                for (int c = 0; c < D; ++c) {
                    const Cplx a0 = (*U)[(size_t)r * D + c], a1 = (*U)[(size_t)r1 * D + c];
                    (*U)[(size_t)r * D + c] = add(mul(u[0], a0), mul(u[1], a1));
                    (*U)[(size_t)r1 * D + c] = add(mul(u[2], a0), mul(u[3], a1));
                }
            }
        }
    }
}

}  // namespace

// IEEE 754 binary16 from a double, round to nearest even (format: 1 sign,
// 5 exponent bits with bias 15, 10 fraction bits; subnormals below 2^-14).
uint16_t f64_to_f16_bits(double x)
{
    const uint16_t sign = std::signbit(x) ? 0x8000 : 0;
    const double a = std::fabs(x);
    if (std::isnan(a)) return sign | 0x7e00;
    if (a >= 65520.0) return sign | 0x7c00;                  // rounds past 65504
    if (a < std::ldexp(1.0, -14)) {                           // subnormal range
        const double r = std::nearbyint(a * std::ldexp(1.0, 24));   // units of 2^-24
        return sign | (uint16_t)r;                            // r = 1024 is the smallest normal
    }
    int e;
    std::frexp(a, &e);                                        // a = f 2^e, f in [0.5, 1)
    int E = e - 1;                                            // a = 1.m 2^E
    double r = std::nearbyint((std::ldexp(a, -E) - 1.0) * 1024.0);
    if (r == 1024.0) { r = 0; ++E; }
    if (E > 15) return sign | 0x7c00;
    return sign | (uint16_t)((E + 15) << 10) | (uint16_t)r;
}

double f16_bits_to_f64(uint16_t h)
{
    const int s = h >> 15, e = (h >> 10) & 31, f = h & 1023;
    double v;
    if (e == 0) v = std::ldexp((double)f, -24);
    else if (e == 31) v = f ? NAN : INFINITY;
    else v = std::ldexp(1.0 + f / 1024.0, e - 15);
    return s ? -v : v;
}

// Rounds x to `frac` fraction bits, round to nearest even (no range limit:
// the 8-bit exponent of BF16 and TF32 covers every value a block holds).
static double round_frac_bits(double x, int frac)
{
    if (x == 0 || !std::isfinite(x)) return x;
    int e;
    std::frexp(x, &e);                        // |x| = f 2^e, f in [0.5, 1)
    const double q = std::ldexp(1.0, e - 1 - frac);   // spacing at |x|
    return std::nearbyint(x / q) * q;         // nearbyint: ties to even
}

uint16_t f64_to_bf16_bits(double x)
{
    const float f = (float)round_frac_bits(x, 7);   // exact in FP32
    uint32_t w;
    std::memcpy(&w, &f, 4);
    return (uint16_t)(w >> 16);
}

double bf16_bits_to_f64(uint16_t h)
{
    const uint32_t w = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &w, 4);
    return f;
}

uint32_t f64_to_tf32_bits(double x)
{
    const float f = (float)round_frac_bits(x, 10);  // exact in FP32, low 13 bits zero
    uint32_t w;
    std::memcpy(&w, &f, 4);
    return w;
}

double tf32_bits_to_f64(uint32_t w)
{
    float f;
    std::memcpy(&f, &w, 4);
    return f;
}

namespace {

// Realified block A = [[Re U, -Im U], [Im U, Re U]] split into the terms of
// `precision` (term t = the operand type's rounding of what terms 0..t-1
// leave) and packed for tensor memory (see tc_words_per_block).
static void pack_block(const std::vector<Cplx> &U, int precision, std::vector<uint32_t> *words)
{
    const TcPrec tp = tc_prec(precision);
    const int D = 1 << kTcBits, MK = 2 * D;
    const int wpt = MK * tp.elem_bytes / 4;          // words per term per row
    const size_t base = words->size();
    words->resize(base + (size_t)tc_words_per_block(precision));
    for (int m = 0; m < MK; ++m) {
        uint32_t *row = words->data() + base + (size_t)m * tp.terms * wpt;
        for (int k = 0; k < MK; ++k) {
            // output rows interleave re / im of block row m / 2; input
            // columns are the re block then the im block
            const Cplx &u = U[(size_t)(m / 2) * D + (k % D)];
            double a;
            if (!(m & 1)) a = k < D ? u.re : -u.im;
            else a = k < D ? u.im : u.re;
            for (int t = 0; t < tp.terms; ++t) {
                uint32_t *w = row + t * wpt;
                double v;
                if (tp.fmt == 2) {
                    w[k] = f64_to_tf32_bits(a);
                    v = tf32_bits_to_f64(w[k]);
                } else {
                    const uint16_t h = tp.fmt == 1 ? f64_to_bf16_bits(a) : f64_to_f16_bits(a);
                    v = tp.fmt == 1 ? bf16_bits_to_f64(h) : f16_bits_to_f64(h);
                    if (k & 1) w[k / 2] |= (uint32_t)h << 16;
                    else w[k / 2] = h;
                }
                a -= v;
            }
        }
    }
}

}  // namespace

// Persistent ensemble work list (declared with its order and dependency
// rules in qs_internal.h).
static uint64_t tiles_per_item(int t)
{
    return t >= kPassItemBits ? 1 : (1ULL << (kPassItemBits - t));
}

void build_work(const std::vector<int> &n, const std::vector<uint64_t> &off, const std::vector<Plan> &plans,
                const std::vector<std::vector<char>> &full, const std::vector<int> &idx,
                const std::vector<size_t> &hl, bool stats, Work *W)
{
    *W = Work();
    const size_t C = n.size();
    std::vector<int> first_pass(C, 0);
    std::vector<uint32_t> ninit(C, 0), npass(C, 0), nstat(C, 0), before(C, 0);
    int max_passes = 0;
    for (int i : idx) {
        first_pass[i] = (int)W->passes.size();
        const int pb = (int)W->phases.size(), ob = (int)W->ops.size();
        for (DevPass p : plans[i].passes) {
            p.phase_begin += pb;
            W->passes.push_back(p);
        }
        for (DevPhase h : plans[i].phases) {
            h.op_begin += ob;
            h.op_end += ob;
            W->phases.push_back(h);
        }
        W->ops.insert(W->ops.end(), plans[i].ops.begin(), plans[i].ops.end());
        max_passes = std::max(max_passes, (int)plans[i].passes.size());
        W->bytes += (double)plans[i].passes.size() * 16.0 * std::ldexp(1.0, n[i]);
        const uint64_t N = 1ULL << n[i];
        ninit[i] = (uint32_t)((N + kWorkChunk - 1) / kWorkChunk);
        nstat[i] = stats ? ninit[i] : 0;
        for (const DevPass &p : plans[i].passes) {
            const uint64_t nt = 1ULL << (n[i] - p.t), per = tiles_per_item(p.t);
            npass[i] += (uint32_t)((nt + per - 1) / per);
        }
    }
    auto item = [&](uint32_t kind, int i) {
        PersistItem w;
        std::memset(&w, 0, sizeof w);
        w.kind = kind;
        w.inst = (uint32_t)i;
        w.total = ninit[i] + npass[i] + nstat[i];
        return w;
    };
    for (int i : idx) {
        const uint64_t N = 1ULL << n[i];
        const float v = hl[i] ? (float)std::pow(2.0, -0.5 * n[i]) : 0.f;
        for (uint64_t a = 0; a < N; a += kWorkChunk) {
            PersistItem w = item(kPersistInit, i);
            w.amp_off = off[i] + a;
            w.lo = (uint32_t)std::min<uint64_t>(kWorkChunk, N - a);
            w.f0 = v;
            w.f1 = hl[i] ? v : (a == 0 ? 1.f : 0.f);
            W->items.push_back(w);
        }
        before[i] = ninit[i];
    }
    std::vector<int> order(idx);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return n[x] > n[y]; });
    for (int r = 0; r < max_passes; ++r)
        for (int i : order) {
            if (r >= (int)plans[i].passes.size()) continue;
            const DevPass &p = plans[i].passes[r];
            const uint32_t kind = full[i][r] ? kPersistPassFull : kPersistPass;
            const uint64_t nt = 1ULL << (n[i] - p.t), per = tiles_per_item(p.t);
            uint32_t cnt = 0;
            for (uint64_t t0 = 0; t0 < nt; t0 += per, ++cnt) {
                PersistItem w = item(kind, i);
                w.amp_off = off[i];
                w.pass = (uint32_t)(first_pass[i] + r);
                w.lo = (uint32_t)t0;
                w.hi = (uint32_t)std::min<uint64_t>(nt, t0 + per);
                w.need = before[i];
                W->items.push_back(w);
            }
            before[i] += cnt;
        }
    if (stats)
        for (int i : idx) {
            const uint64_t N = 1ULL << n[i];
            const uint32_t first = (uint32_t)W->nslots;
            for (uint64_t a = 0; a < N; a += kWorkChunk) {
                PersistItem w = item(kPersistStats, i);
                w.amp_off = off[i] + a;
                w.lo = (uint32_t)std::min<uint64_t>(kWorkChunk, N - a);
                w.pass = (uint32_t)W->nslots++;
                w.hi = first;
                w.nslots = nstat[i];
                w.f0 = (float)std::ldexp(1.0, n[i]);
                w.need = ninit[i] + npass[i];
                W->items.push_back(w);
            }
        }
}

PlanParams default_plan_params(int n, qs_dtype dt, const qs_opts *o)
{
    PlanParams pp;
    pp.n = n;
    pp.mode = o ? o->mode : QS_MODE_FUSED;
    pp.r = dt == QS_C128 ? 4 : 5;
    int tile = dt == QS_C128 ? 12 : 13;
    if (o && o->tile_log2 > 0) tile = o->tile_log2;
    pp.t = std::min(tile, n);
    // the always-resident low qubits leave at least one tile bit free when
    // the tile is smaller than the state (else no pass could bring in
    // another qubit); a 16-byte load still takes consecutive amplitudes
    pp.c = std::min(dt == QS_C128 ? 4 : 5, pp.t < n ? pp.t - 1 : pp.t);
    pp.k = kTcBits;
    pp.tc_ok = pp.mode == QS_MODE_FUSED_TC && dt == QS_C64 && pp.t == 13 ? 1 : 0;
    pp.precision = (o && o->precision != QS_PREC_DEFAULT) ? o->precision : QS_PREC_FP16X3;
    pp.esz = dt == QS_C128 ? 16 : 8;
    // a deeper lookahead pays where a pass costs the most (host planning of
    // the next circuit overlaps the current evolution)
    if (n >= 32)
        pp.look_steps = pp.look_top = 64;
    else if (n >= 28)
        pp.look_steps = pp.look_top = 8;
    pp.r = std::min(pp.r, pp.t);
    return pp;
}

double plan_bytes(const Plan &p, qs_dtype dt)
{
    return (double)p.passes.size() * 2.0 * std::ldexp(1.0, p.n) * (double)dtype_bytes(dt);
}

// The last register phase of a pass always multiplies every slot by a
// thread-uniform factor (the pass-wide scale), so diagonal ops that reach it
// as thread-uniform ops cost no dispatch.  A diagonal op of an earlier
// phase moves to that phase's tail when none of its qubits is a register
// bit of the last phase and no non-diagonal op on one of its qubits follows
// it in the pass (diagonal ops commute with each other and with
// non-diagonal ops on other qubits, so the pass's product is unchanged).
static void hoist_diagonals_to_last_phase(Plan *P, const DevPass &dp)
{
    const int p0 = dp.phase_begin, np = dp.nphases;
    if (np < 2) return;
    for (int ph = 0; ph < np; ++ph)
        if (P->phases[p0 + ph].kind != 0) return;     // tensor-core passes keep their layout
    auto qubits = [&](int ph, const DevOp &d) {
        uint64_t q = d.qmask;
        for (int j = 0; j < dp.r; ++j)
            if ((d.rmask >> j) & 1) q |= 1ULL << dp.L[P->phases[p0 + ph].R[j]];
        return q;
    };
    auto nondiag_qubit = [&](int ph, const DevOp &d) -> uint64_t {
        if (d.type == OP_PHASE || d.type == OP_NEG) return 0;
        return 1ULL << dp.L[P->phases[p0 + ph].R[d.a]];
    };
    uint64_t last_reg = 0;
    for (int j = 0; j < dp.r; ++j) last_reg |= 1ULL << dp.L[P->phases[p0 + np - 1].R[j]];
    // qubits touched by non-diagonal ops from each position to the end of
    // the pass, scanned backwards
    std::vector<std::vector<DevOp>> keep(np);
    std::vector<DevOp> moved;
    uint64_t later_nd = 0;
    for (int o = P->phases[p0 + np - 1].op_begin; o < P->phases[p0 + np - 1].op_end; ++o)
        later_nd |= nondiag_qubit(np - 1, P->ops[o]);
    for (int ph = np - 2; ph >= 0; --ph) {
        const DevPhase &H = P->phases[p0 + ph];
        std::vector<DevOp> kept_rev;
        for (int o = H.op_end - 1; o >= H.op_begin; --o) {
            const DevOp &d = P->ops[o];
            const bool diag = d.type == OP_PHASE || d.type == OP_NEG;
            if (diag && d.rmask) {
                const uint64_t q = qubits(ph, d);
                if (!(q & last_reg) && !(q & later_nd)) {
                    DevOp m = d;
                    m.rmask = 0;
                    m.qmask = q;
                    moved.push_back(m);
                    continue;
                }
            }
            later_nd |= nondiag_qubit(ph, d);
            kept_rev.push_back(d);
        }
        keep[ph].assign(kept_rev.rbegin(), kept_rev.rend());
    }
    if (moved.empty()) return;
    for (int o = P->phases[p0 + np - 1].op_begin; o < P->phases[p0 + np - 1].op_end; ++o)
        keep[np - 1].push_back(P->ops[o]);
    // the moved ops join the last phase's thread-uniform tail (diagonal ops
    // commute, so their order there is free)
    for (const DevOp &m : moved) keep[np - 1].push_back(m);
    int o = P->phases[p0].op_begin;
    for (int ph = 0; ph < np; ++ph) {
        DevPhase &H = P->phases[p0 + ph];
        H.op_begin = o;
        for (const DevOp &d : keep[ph]) P->ops[o++] = d;
        H.op_end = o;
    }
}

qs_status build_plan(const PlanParams &pp, const qs_gate *gin, size_t ng, Plan *out)
{
    const int n = pp.n;
    if (pp.t < 1 || pp.t > kMaxTileBits || pp.t > n || pp.r < 1 || pp.r > kMaxRegBits ||
        pp.r > pp.t || pp.c < 0 || pp.c > pp.t)
        return set_error(QS_ERR_INVALID_ARG, "bad plan parameters t=%d r=%d c=%d n=%d",
                         pp.t, pp.r, pp.c, n);
    std::vector<PGate> g(ng);
    for (size_t i = 0; i < ng; ++i) {
        g[i].kind = gin[i].kind;
        g[i].q0 = gin[i].q0;
        g[i].q1 = gin[i].q1;
        g[i].two = gate_is_two_qubit(gin[i].kind);
        g[i].diag = gate_is_diagonal(gin[i].kind);
        g[i].theta = gin[i].theta;
    }
    Plan &P = *out;
    P = Plan();
    P.n = n; P.t = pp.t; P.r = pp.r; P.c = pp.c; P.mode = pp.mode;
    P.precision = pp.precision;
    P.gates = (int)ng;

    std::vector<char> done(ng, 0);
    std::vector<int> all(ng);
    for (size_t i = 0; i < ng; ++i) all[i] = (int)i;
    size_t remaining = ng;
    const uint64_t allq = (n == 64) ? ~0ULL : ((1ULL << n) - 1);
    const uint64_t low = (pp.c >= 64) ? ~0ULL : ((1ULL << pp.c) - 1);
    std::vector<int> pass_gates, phase_gates;
    while (remaining) {
        uint64_t local = choose_tile(g, all, done, n, low & allq, allq & ~low, pp.t - pp.c, allq, pp.look_steps,
                                     pp.look_top);
        int cnt;
        collect(g, all, done, local, &pass_gates, &cnt, allq);
        if (cnt == 0) return set_error(QS_ERR_INVALID_ARG, "planner made no progress");
        DevPass dp;
        std::memset(&dp, 0, sizeof dp);
        dp.t = popcount64(local);
        dp.n = n;
        dp.r = std::min(pp.r, dp.t);
        dp.phase_begin = (int)P.phases.size();
        dp.ngates = cnt;
        int tb = 0, gb = 0;
        int tile_bit_of[64];
        for (int q = 0; q < n; ++q) {
            if ((local >> q) & 1) { tile_bit_of[q] = tb; dp.L[tb++] = (uint8_t)q; }
            else { tile_bit_of[q] = -1; dp.G[gb++] = (uint8_t)q; }
        }
        double gre = 1.0, gim = 0.0;
        int deferred = 0;
        // phases inside the pass
        std::vector<char> pdone(ng, 1);
        for (int i : pass_gates) pdone[i] = 0;
        size_t prem = pass_gates.size();
        int pass_ops = 0;
        int tc_in_pass = 0;
        while (prem && dp.nphases < kMaxPhasesPerPass && pass_ops < kMaxOpsPerPass) {
            uint64_t reg = choose_local(g, pass_gates, pdone, n, 0, local, dp.r);
            collect(g, pass_gates, pdone, reg, &phase_gates, &cnt);
            if (cnt == 0) return set_error(QS_ERR_INVALID_ARG, "planner made no phase progress");
            if (pp.tc_ok && tc_in_pass < kMaxTcPerPass && dp.t == 13) {
                // tensor-core block candidate: worth it when it absorbs many
                // gates compared with the register phase
                const uint64_t blk = choose_tc_block(g, pass_gates, pdone, n, local, kTcBits);
                std::vector<int> tc_gates;
                int tcnt = 0;
                collect_tc(g, pass_gates, pdone, blk, &tc_gates, &tcnt);
                if (popcount64(blk) == kTcBits && tcnt >= kTcMinGates &&
                    (double)tcnt >= kTcRegRatio * (double)cnt) {
                    DevPhase ph;
                    std::memset(&ph, 0, sizeof ph);
                    int bq[kTcBits], j = 0;
                    for (int q = 0; q < n; ++q)
                        if ((blk >> q) & 1) { bq[j] = q; ph.R[j++] = (uint8_t)tile_bit_of[q]; }
                    order_tc_block(bq, ph.R);
                    ph.kind = 1;
                    ph.tc_block = (int)(P.tc_words.size() / tc_words_per_block(pp.precision));
                    ph.defer_before = deferred;
                    ph.op_begin = ph.op_end = (int)P.ops.size();
                    std::vector<Cplx> U;
                    block_unitary(g, tc_gates, bq, &U);
                    pack_block(U, pp.precision, &P.tc_words);
                    for (int gi : tc_gates) { pdone[gi] = 1; --prem; }
                    P.phases.push_back(ph);
                    ++dp.nphases;
                    ++tc_in_pass;
                    continue;
                }
            }
            // keep the pass within the kernel's op table; a prefix of the
            // phase's (ordered, dependency-closed) gate list stays closed
            {
                // ops of a gate: 5 for RX, 3 for RY, else 1
                size_t keep = 0;
                int ops_needed = 0;
                for (int gi : phase_gates) {
                    const int k = g[gi].kind == QS_RX ? 5 : g[gi].kind == QS_RY ? 3 : 1;
                    if (pass_ops + ops_needed + k > kMaxOpsPerPass) break;
                    ops_needed += k;
                    ++keep;
                }
                if (keep == 0 && dp.nphases == 0 && pass_ops == 0)
                    return set_error(QS_ERR_INVALID_ARG, "op table too small");
                phase_gates.resize(keep);
                pass_ops += ops_needed;
                if (keep == 0) break;
            }
            DevPhase ph;
            std::memset(&ph, 0, sizeof ph);
            int reg_bit_of[64];
            int j = 0;
            for (int q = 0; q < n; ++q) reg_bit_of[q] = -1;
            for (int q = 0; q < n; ++q)
                if ((reg >> q) & 1) { reg_bit_of[q] = j; ph.R[j++] = (uint8_t)tile_bit_of[q]; }
            // pad with unused tile bits so the phase always has dp.r register bits
            for (int b = 0; j < dp.r && b < dp.t; ++b) {
                bool used = false;
                for (int i2 = 0; i2 < j; ++i2) used |= ph.R[i2] == b;
                if (!used) ph.R[j++] = (uint8_t)b;
            }
            std::sort(ph.R, ph.R + dp.r);
            choose_thread_bits(ph.R, dp.r, dp.t, pp.esz, ph.T);
            for (int q = 0; q < n; ++q) reg_bit_of[q] = -1;
            for (int i2 = 0; i2 < dp.r; ++i2) reg_bit_of[dp.L[ph.R[i2]]] = i2;
            ph.op_begin = (int)P.ops.size();
            for (int gi : phase_gates) {
                const PGate &x = g[gi];
                DevOp op;
                std::memset(&op, 0, sizeof op);
                if (!x.diag) {
                    op.a = (uint8_t)reg_bit_of[x.q0];
                    switch (x.kind) {
                    case QS_H: op.type = OP_H; ++deferred; break;
                    case QS_X_HALF: op.type = OP_XH; ++deferred; break;
                    case QS_Y_HALF: op.type = OP_YH; ++deferred; break;
                    default: {
                        // RY(theta) is a rotation by phi = theta/2, written as
                        // three in-place shears (Paeth): x -= t y, y += s x,
                        // x -= t y with t = tan(phi/2), s = sin(phi).  phi is
                        // first reduced to [-pi/2, pi/2]; each pi removed is
                        // a factor -1 folded into the pass-wide scale.
                        // RX(theta) = S RY(-theta) S^dagger, S = diag(1, i).
                        const bool rx = x.kind == QS_RX;
                        double phi = (rx ? -x.theta : x.theta) / 2;
                        const double k = std::nearbyint(phi / M_PI);
                        phi -= k * M_PI;
                        if (std::fmod(std::fabs(k), 2.0) == 1.0) { gre = -gre; gim = -gim; }
                        const double t = std::tan(phi / 2), sn = std::sin(phi);
                        DevOp ph = op;
                        ph.type = OP_PHASE;
                        ph.rmask = (uint8_t)(1u << op.a);
                        ph.qmask = 0;
                        if (rx) { ph.m[0] = 0; ph.m[1] = -1; P.ops.push_back(ph); }
                        DevOp sh = op;
                        sh.type = OP_SHX; sh.m[0] = -t; P.ops.push_back(sh);
                        sh.type = OP_SHY; sh.m[0] = sn; P.ops.push_back(sh);
                        sh.type = OP_SHX; sh.m[0] = -t;
                        if (rx) { P.ops.push_back(sh); ph.m[1] = 1; op = ph; }
                        else op = sh;
                    }
                    }
                } else {
                    int qs2[2] = {x.q0, x.q1};
                    for (int e = 0; e < (x.two ? 2 : 1); ++e) {
                        int q = qs2[e];
                        if (reg_bit_of[q] >= 0) op.rmask |= (uint8_t)(1u << reg_bit_of[q]);
                        else op.qmask |= 1ULL << q;
                    }
                    if (x.kind == QS_CZ) {
                        op.type = OP_NEG;
                    } else {
                        op.type = OP_PHASE;
                        double ang;
                        if (x.kind == QS_T) {
                            ang = M_PI / 4;
                        } else if (x.kind == QS_RZ) {
                            // diag(e^{-i th/2}, e^{i th/2}) = e^{-i th/2} diag(1, e^{i th})
                            ang = x.theta;
                            double c = std::cos(-x.theta / 2), s = std::sin(-x.theta / 2);
                            double nr = gre * c - gim * s, ni = gre * s + gim * c;
                            gre = nr; gim = ni;
                        } else {
                            ang = x.theta;   // CPHASE
                        }
                        op.m[0] = std::cos(ang);
                        op.m[1] = std::sin(ang);
                        if (x.kind == QS_T) { op.m[0] = std::sqrt(0.5); op.m[1] = std::sqrt(0.5); }
                    }
                }
                P.ops.push_back(op);
                pdone[gi] = 1;
                --prem;
            }
            // diagonal ops whose selection lies wholly outside the register
            // set only scale a thread's slots by a constant: they commute
            // with every other op of the phase and go to its end
            std::stable_partition(P.ops.begin() + ph.op_begin, P.ops.end(), [](const DevOp &o) {
                return !((o.type == OP_PHASE || o.type == OP_NEG) && o.rmask == 0);
            });
            ph.op_end = (int)P.ops.size();
            P.phases.push_back(ph);
            ++dp.nphases;
        }
        if (pp.hoist_diagonals) hoist_diagonals_to_last_phase(&P, dp);
        int placed = 0;
        for (int i : pass_gates)
            if (pdone[i]) { done[i] = 1; --remaining; ++placed; }
        dp.ngates = placed;
        // later passes scan only the gates still pending
        all.erase(std::remove_if(all.begin(), all.end(), [&](int i) { return done[i] != 0; }), all.end());
        double sc = std::ldexp(1.0, -(deferred / 2));
        if (deferred & 1) sc *= std::sqrt(0.5);
        dp.deferred = deferred;
        dp.gscale_re = gre * sc;
        dp.gscale_im = gim * sc;
        P.passes.push_back(dp);
    }
    return QS_OK;
}

}  // namespace qs

extern "C" qs_status qs_plan_circuit(int n, qs_dtype dt, const qs_gate *gates,
                                     size_t ngates, const qs_opts *opts,
                                     qs_plan_stats *stats)
{
    clear_error();
    if (n < 1 || n > kMaxQubits) return set_error(QS_ERR_INVALID_ARG, "n = %d out of range 1..%d", n, kMaxQubits);
    if (dt != QS_C64 && dt != QS_C128) return set_error(QS_ERR_INVALID_ARG, "bad dtype");
    if (!stats) return set_error(QS_ERR_INVALID_ARG, "stats is NULL");
    qs_status st = validate_gates(n, gates, ngates);
    if (st) return st;
    int mode = opts ? opts->mode : QS_MODE_FUSED;
    std::memset(stats, 0, sizeof *stats);
    stats->gates = (int)ngates;
    if (mode == QS_MODE_PLAIN) {
        stats->passes = (int)ngates;
        double N = std::ldexp(1.0, n) * (double)dtype_bytes(dt);
        for (size_t i = 0; i < ngates; ++i) {
            int k = gates[i].kind;
            stats->bytes += k == QS_T ? N : (k == QS_CZ || k == QS_CPHASE) ? 0.5 * N : 2.0 * N;
        }
        return QS_OK;
    }
    if (mode != QS_MODE_FUSED && mode != QS_MODE_FUSED_TC)
        return set_error(QS_ERR_INVALID_ARG, "unknown mode %d", mode);
    if (mode == QS_MODE_FUSED_TC && opts && (opts->precision < QS_PREC_DEFAULT || opts->precision > QS_PREC_TF32))
        return set_error(QS_ERR_INVALID_ARG, "tensor-core precision %d is not a qs_precision", opts->precision);
    PlanParams pp = default_plan_params(n, dt, opts);
    Plan plan;
    st = build_plan(pp, gates, ngates, &plan);
    if (st) return st;
    stats->passes = (int)plan.passes.size();
    stats->phases = (int)plan.phases.size();
    stats->ops = (int)plan.ops.size();
    stats->tile_log2 = pp.t;
    stats->reg_log2 = pp.r;
    stats->bytes = plan_bytes(plan, dt);
    return QS_OK;
}
