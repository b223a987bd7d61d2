// CPU emulator of the library's fused-pass plan format (test support only).
//
// Builds a plan with the library's own host planner and executes it on a
// double-precision state with the semantics the fused kernels give each
// op: tiles gathered through the pass's qubit map, phases over register
// bits, diagonal ops selected by register and qubit masks, deferred 1/sqrt2
// factors applied at the end of each pass.  Comparing its result with the
// oracle checks the planner (dependency order, register mapping, masks,
// scales) without a GPU.
#include <complex>
#include <cstring>
#include <vector>

#include "../paper_1608_00263_gb300/csrc/qs_internal.h"

using cd = std::complex<double>;
using namespace qs;

extern "C" uint16_t emul_f16(double x) { return f64_to_f16_bits(x); }
extern "C" uint16_t emul_bf16(double x) { return f64_to_bf16_bits(x); }
extern "C" uint32_t emul_tf32(double x) { return f64_to_tf32_bits(x); }
extern "C" double emul_f16_back(uint16_t h) { return f16_bits_to_f64(h); }

// Tensor-core phase: apply the stored block matrix (hi + lo, decoded) to
// every column of the tile: the 64 amplitudes over the block bits, as
// realified vectors [re; im]; output rows interleave re and im.
static void apply_tc(const Plan &plan, const DevPass &P, const DevPhase &H, std::vector<cd> &tile)
{
    const TcPrec tp = tc_prec(plan.precision);
    const int wpt = 128 * tp.elem_bytes / 4;        // words per term per row
    const uint32_t *w = plan.tc_words.data() + (size_t)H.tc_block * tc_words_per_block(plan.precision);
    static double A[128][128];
    for (int m = 0; m < 128; ++m)
        for (int k = 0; k < 128; ++k) {
            double a = 0;
            for (int t = 0; t < tp.terms; ++t) {
                const uint32_t *row = w + (size_t)m * tp.terms * wpt + t * wpt;
                if (tp.fmt == 2) {
                    a += tf32_bits_to_f64(row[k]);
                } else {
                    const uint32_t word = row[k / 2];
                    const uint16_t b = (k & 1) ? (uint16_t)(word >> 16) : (uint16_t)(word & 0xffff);
                    a += tp.fmt == 1 ? bf16_bits_to_f64(b) : f16_bits_to_f64(b);
                }
            }
            A[m][k] = a;
        }
    uint64_t bmask = 0;
    for (int j = 0; j < kTcBits; ++j) bmask |= 1ULL << H.R[j];
    for (uint64_t col = 0; col < tile.size(); ++col) {
        if (col & bmask) continue;
        double v[128], o[128];
        for (int b = 0; b < 64; ++b) {
            uint64_t e = col;
            for (int j = 0; j < kTcBits; ++j) e |= (uint64_t)((b >> j) & 1) << H.R[j];
            v[b] = tile[e].real();
            v[64 + b] = tile[e].imag();
        }
        for (int m = 0; m < 128; ++m) {
            double s = 0;
            for (int k = 0; k < 128; ++k) s += A[m][k] * v[k];
            o[m] = s;
        }
        for (int b = 0; b < 64; ++b) {
            uint64_t e = col;
            for (int j = 0; j < kTcBits; ++j) e |= (uint64_t)((b >> j) & 1) << H.R[j];
            tile[e] = cd(o[2 * b], o[2 * b + 1]);
        }
    }
}

extern "C" int emulate_plan_mode(int n, const qs_gate *g, size_t ng, int t, int r, int c, int mode,
                                 double *psi_interleaved, int *passes_out, int *tc_phases_out);

extern "C" int emulate_plan(int n, const qs_gate *g, size_t ng, int t, int r, int c,
                            double *psi_interleaved, int *passes_out)
{
    return emulate_plan_mode(n, g, ng, t, r, c, QS_MODE_FUSED, psi_interleaved, passes_out, nullptr);
}

// Executes a built plan on a double-precision state (the semantics the
// fused kernels give each op).
static int emulate_built_plan(const Plan &plan, double *psi_interleaved, int *passes_out,
                              int *tc_phases_out = nullptr)
{
    cd *psi = reinterpret_cast<cd *>(psi_interleaved);
    for (const DevPass &P : plan.passes) {
        const int T = P.t, ngl = P.n - T;
        std::vector<cd> tile(size_t(1) << T);
        for (uint64_t tau = 0; tau < (1ULL << ngl); ++tau) {
            uint64_t base = 0;
            for (int i = 0; i < ngl; ++i) base |= ((tau >> i) & 1ULL) << P.G[i];
            auto addr = [&](uint64_t e) {
                uint64_t a = base;
                for (int b = 0; b < T; ++b) a |= ((e >> b) & 1ULL) << P.L[b];
                return a;
            };
            for (uint64_t e = 0; e < tile.size(); ++e) tile[e] = psi[addr(e)];
            for (int ph = 0; ph < P.nphases; ++ph) {
                const DevPhase &H = plan.phases[P.phase_begin + ph];
                if (H.kind == 1) {
                    apply_tc(plan, P, H, tile);
                    continue;
                }
                for (int o = H.op_begin; o < H.op_end; ++o) {
                    const DevOp &op = plan.ops[o];
                    if (op.type == OP_PHASE || op.type == OP_NEG) {
                        cd f = op.type == OP_NEG ? cd(-1, 0) : cd(op.m[0], op.m[1]);
                        for (uint64_t e = 0; e < tile.size(); ++e) {
                            bool sel = (addr(e) & op.qmask) == op.qmask;
                            for (int j = 0; j < P.r; ++j)
                                if ((op.rmask >> j) & 1) sel = sel && ((e >> H.R[j]) & 1);
                            if (sel) tile[e] *= f;
                        }
                    } else if (op.type == OP_SHX || op.type == OP_SHY) {
                        const uint64_t bit = 1ULL << H.R[op.a];
                        for (uint64_t e = 0; e < tile.size(); ++e) {
                            if (e & bit) continue;
                            if (op.type == OP_SHX) tile[e] += op.m[0] * tile[e | bit];
                            else tile[e | bit] += op.m[0] * tile[e];
                        }
                    } else {
                        const uint64_t bit = 1ULL << H.R[op.a];
                        cd u[4];
                        if (op.type == OP_H) { u[0] = 1; u[1] = 1; u[2] = 1; u[3] = -1; }
                        else if (op.type == OP_XH) { u[0] = 1; u[1] = cd(0, -1); u[2] = cd(0, -1); u[3] = 1; }
                        else if (op.type == OP_YH) { u[0] = 1; u[1] = -1; u[2] = 1; u[3] = 1; }
                        else for (int k = 0; k < 4; ++k) u[k] = cd(op.m[2 * k], op.m[2 * k + 1]);
                        for (uint64_t e = 0; e < tile.size(); ++e) {
                            if (e & bit) continue;
                            cd x = tile[e], y = tile[e | bit];
                            tile[e] = u[0] * x + u[1] * y;
                            tile[e | bit] = u[2] * x + u[3] * y;
                        }
                    }
                }
            }
            const cd gs(P.gscale_re, P.gscale_im);
            for (uint64_t e = 0; e < tile.size(); ++e) psi[addr(e)] = tile[e] * gs;
        }
    }
    if (passes_out) *passes_out = (int)plan.passes.size();
    if (tc_phases_out) {
        int k = 0;
        for (const DevPhase &H : plan.phases) k += H.kind == 1;
        *tc_phases_out = k;
    }
    return 0;
}

extern "C" int emulate_plan_prec(int n, const qs_gate *g, size_t ng, int t, int r, int c, int mode, int precision,
                                 double *psi_interleaved, int *passes_out, int *tc_phases_out)
{
    PlanParams pp{n, t, r, c, mode, kTcBits, mode == QS_MODE_FUSED_TC && t == 13 ? 1 : 0};
    pp.precision = precision;
    Plan plan;
    if (build_plan(pp, g, ng, &plan) != QS_OK) return -1;
    return emulate_built_plan(plan, psi_interleaved, passes_out, tc_phases_out);
}

extern "C" int emulate_plan_mode(int n, const qs_gate *g, size_t ng, int t, int r, int c, int mode,
                                 double *psi_interleaved, int *passes_out, int *tc_phases_out)
{
    PlanParams pp{n, t, r, c, mode, kTcBits, mode == QS_MODE_FUSED_TC && t == 13 ? 1 : 0};
    Plan plan;
    if (build_plan(pp, g, ng, &plan) != QS_OK) return -1;
    return emulate_built_plan(plan, psi_interleaved, passes_out, tc_phases_out);
}

// Symbolic check of a plan built with the library's own default parameters
// for (n, dtype, mode): every op is mapped back to the gate it applies
// (kind and qubits, through the phase's register map and the pass's tile
// map), and the sequence of ops must be a reordering of the gate list that
// keeps every pair of non-commuting gates (a shared qubit, at least one of
// them non-diagonal) in circuit order.  Also checks the tile and register
// maps and each pass's count of deferred 1/sqrt2 factors.  Needs no state,
// so it runs at any n.  Supports plans whose gates are one op each (H,
// X^1/2, Y^1/2, T, CZ, RZ, CPHASE) and no tensor-core phases.  Returns 0,
// or a negative code naming the first violated rule; *passes_out receives
// the number of passes.
// check_plan_against: the plan is built from `g_plan` and checked against
// the circuit order of `g` (the same list for check_plan_order; a different
// one lets a test show that the check rejects a wrong order).
extern "C" int check_plan_against(int n, int dtype, int mode, const qs_gate *g_plan, const qs_gate *g,
                                  size_t ng, int *passes_out)
{
    qs_opts o{};
    o.mode = mode;
    PlanParams pp = default_plan_params(n, (qs_dtype)dtype, &o);
    Plan plan;
    if (build_plan(pp, g_plan, ng, &plan) != QS_OK) return -1;
    if (passes_out) *passes_out = (int)plan.passes.size();
    std::vector<char> used(ng, 0);
    size_t applied = 0;
    auto qmask_of = [&](const qs_gate &x) {
        uint64_t m = 1ULL << x.q0;
        if (gate_is_two_qubit(x.kind)) m |= 1ULL << x.q1;
        return m;
    };
    for (const DevPass &P : plan.passes) {
        // tile map: P.t distinct qubits in ascending order, the rest in G
        uint64_t tile = 0, glob = 0;
        for (int b = 0; b < P.t; ++b) {
            if (P.L[b] >= n || (b && P.L[b] <= P.L[b - 1])) return -2;
            tile |= 1ULL << P.L[b];
        }
        for (int i = 0; i < n - P.t; ++i) {
            if (P.G[i] >= n || ((tile >> P.G[i]) & 1) || (i && P.G[i] <= P.G[i - 1])) return -3;
            glob |= 1ULL << P.G[i];
        }
        if ((tile | glob) != ((n == 64) ? ~0ULL : ((1ULL << n) - 1))) return -3;
        int nondiag = 0;
        for (int ph = 0; ph < P.nphases; ++ph) {
            const DevPhase &H = plan.phases[P.phase_begin + ph];
            if (H.kind != 0) return -4;
            uint32_t rbits = 0;
            for (int j = 0; j < P.r; ++j) {
                if (H.R[j] >= P.t || ((rbits >> H.R[j]) & 1)) return -5;
                rbits |= 1u << H.R[j];
            }
            for (int op_i = H.op_begin; op_i < H.op_end; ++op_i) {
                const DevOp &op = plan.ops[op_i];
                int kind = -1;
                uint64_t qm = 0;
                if (op.type == OP_H || op.type == OP_XH || op.type == OP_YH) {
                    if (op.a >= P.r) return -6;
                    kind = op.type == OP_H ? QS_H : op.type == OP_XH ? QS_X_HALF : QS_Y_HALF;
                    qm = 1ULL << P.L[H.R[op.a]];
                    ++nondiag;
                } else if (op.type == OP_NEG || op.type == OP_PHASE) {
                    uint64_t rq = 0;
                    for (int j = 0; j < P.r; ++j)
                        if ((op.rmask >> j) & 1) rq |= 1ULL << P.L[H.R[j]];
                    if (op.rmask >> P.r) return -7;
                    if (rq & op.qmask) return -7;
                    qm = rq | op.qmask;
                    const int nq = __builtin_popcountll(qm);
                    if (op.type == OP_NEG) kind = nq == 2 ? QS_CZ : -1;
                    else kind = nq == 2 ? QS_CPHASE : -2;   // T or RZ: resolved below
                } else {
                    return -8;
                }
                // earliest unused gate of this kind on these qubits
                size_t pick = ng;
                for (size_t i = 0; i < ng; ++i) {
                    if (used[i] || qmask_of(g[i]) != qm) continue;
                    const int k = g[i].kind;
                    const bool match = kind == -2 ? (k == QS_T || k == QS_RZ) : k == kind;
                    if (match) { pick = i; break; }
                }
                if (pick == ng) return -9;
                // no earlier pending gate may fail to commute with it
                const bool dg = gate_is_diagonal(g[pick].kind);
                for (size_t j = 0; j < pick; ++j) {
                    if (used[j] || !(qmask_of(g[j]) & qm)) continue;
                    if (!(dg && gate_is_diagonal(g[j].kind))) return -10;
                }
                used[pick] = 1;
                ++applied;
            }
        }
        if (P.deferred != nondiag) return -11;
    }
    return applied == ng ? 0 : -12;
}

extern "C" int check_plan_order(int n, int dtype, int mode, const qs_gate *g, size_t ng, int *passes_out)
{
    return check_plan_against(n, dtype, mode, g, g, ng, passes_out);
}

// Numerical emulation as emulate_plan, with the tile lookahead chosen by the
// caller (the library deepens it for large states: 8 additions among 8
// candidates at 28-31 qubits, every addition and candidate from 32 on).
extern "C" int emulate_plan_look(int n, const qs_gate *g, size_t ng, int t, int r, int c, int look_steps,
                                 int look_top, double *psi_interleaved, int *passes_out)
{
    PlanParams pp{n, t, r, c, QS_MODE_FUSED, kTcBits, 0};
    pp.look_steps = look_steps;
    pp.look_top = look_top;
    Plan plan;
    if (build_plan(pp, g, ng, &plan) != QS_OK) return -1;
    return emulate_built_plan(plan, psi_interleaved, passes_out);
}
