// CPU emulator of the library's fused-pass plan format (test support only).
//
// Builds a plan with the library's own host planner and executes it on a
// double-precision state with the semantics the fused kernels give each
// op: tiles gathered through the pass's qubit map, phases over register
// bits, diagonal ops selected by register and qubit masks, deferred 1/sqrt2
// factors applied at the end of each pass.  Comparing its result with the
// oracle checks the planner (dependency order, register mapping, masks,
// scales) without a GPU.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <utility>
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

// Tiles [lo, hi) of pass P of a plan (phase and op indexes into `plan`)
// on a double-precision state, with the semantics the fused kernels give
// each op.
static void emulate_tiles(const Plan &plan, const DevPass &P, uint64_t lo, uint64_t hi, cd *psi)
{
    {
        const int T = P.t, ngl = P.n - T;
        std::vector<cd> tile(size_t(1) << T);
        for (uint64_t tau = lo; tau < hi; ++tau) {
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
}

// Executes a built plan on a double-precision state.
static int emulate_built_plan(const Plan &plan, double *psi_interleaved, int *passes_out,
                              int *tc_phases_out = nullptr)
{
    cd *psi = reinterpret_cast<cd *>(psi_interleaved);
    for (const DevPass &P : plan.passes) emulate_tiles(plan, P, 0, 1ULL << (P.n - P.t), psi);
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

// ---------------------------------------------------------------------------
// Persistent ensemble engine: the library's work list (build_work) run on
// double-precision states under a randomized schedule of `workers`
// concurrent workers that follows the device protocol: a worker takes the
// next item from the queue, waits until done[inst] >= need, runs it and
// increments done[inst]; the last statistics item of an instance to finish
// sums the instance's partials in slot order.  The list is checked first.
// Returns 0, or the failed check: -1 planning, -2 item bounds, -3 coverage,
// -4 level structure, -5 deadlock, -6 totals.  corrupt = 1 / 2 lowers /
// raises the need of the list's last pass item by one before the checks (a
// planted mistake the level check must catch).
// ---------------------------------------------------------------------------
static void work_stats_chunk(const cd *a, uint64_t cnt, double N, double *c)
{
    for (int k = 0; k < 12; ++k) c[k] = 0;
    for (uint64_t i = 0; i < cnt; ++i) {
        const double y = std::norm(a[i]) * N;
        const double ly = std::log(y);
        c[0] += y;
        c[1] += y > 0 ? y * ly : 0.0;
        c[2] += ly;
        double yk = y;
        for (int k = 2; k <= 10; ++k) {
            yk *= y;
            c[k + 1] += yk;
        }
    }
}

static bool covers_once(std::vector<std::pair<uint64_t, uint64_t>> r, uint64_t end)
{
    std::sort(r.begin(), r.end());
    uint64_t at = 0;
    for (auto &x : r) {
        if (x.first != at || x.second <= x.first) return false;
        at = x.second;
    }
    return at == end;
}

extern "C" int emulate_work(int count, const int *nq, const qs_gate *gates, const uint64_t *offsets, int workers,
                            uint64_t seed, int corrupt, double *psi_out, double *sums_out, int *nitems_out)
{
    std::vector<int> n(nq, nq + count), idx(count);
    std::vector<uint64_t> off(count);
    std::vector<size_t> hl(count);
    std::vector<Plan> plans(count);
    std::vector<std::vector<char>> full(count);
    uint64_t total = 0;
    for (int i = 0; i < count; ++i) {
        idx[i] = i;
        off[i] = total;
        total += 1ULL << n[i];
        const size_t ng = (size_t)(offsets[i + 1] - offsets[i]);
        hl[i] = leading_h_layer(gates + offsets[i], ng, n[i]);
        if (ng > hl[i]) {
            qs_opts o{};
            o.mode = QS_MODE_FUSED;
            if (build_plan(default_plan_params(n[i], QS_C64, &o), gates + offsets[i] + hl[i], ng - hl[i], &plans[i]))
                return -1;
        }
        full[i].assign(plans[i].passes.size(), 0);
    }
    Work W;
    build_work(n, off, plans, full, idx, hl, true, &W);
    if (corrupt)
        for (size_t j = W.items.size(); j-- > 0;)
            if (W.items[j].kind == kPersistPass && W.items[j].need > 0) {
                W.items[j].need += corrupt == 1 ? -1 : 1;
                break;
            }
    const std::vector<PersistItem> &it = W.items;
    if (nitems_out) *nitems_out = (int)it.size();
    Plan view;
    view.passes = W.passes;
    view.phases = W.phases;
    view.ops = W.ops;
    // bounds
    std::vector<int> first_pass(count, 0);
    for (int i = 0, acc = 0; i < count; ++i) {
        first_pass[i] = acc;
        acc += (int)plans[i].passes.size();
    }
    std::vector<std::vector<std::pair<uint64_t, uint64_t>>> init_r(count), stat_r(count);
    std::vector<std::vector<std::vector<std::pair<uint64_t, uint64_t>>>> pass_r(count);
    for (int i = 0; i < count; ++i) pass_r[i].resize(plans[i].passes.size());
    std::vector<uint32_t> nitem(count, 0);
    for (const PersistItem &w : it) {
        if (w.inst >= (uint32_t)count || w.kind > kPersistStats) return -2;
        const int i = (int)w.inst;
        const uint64_t N = 1ULL << n[i];
        ++nitem[i];
        if (w.kind == kPersistInit || w.kind == kPersistStats) {
            if (w.amp_off < off[i] || w.lo == 0 || w.amp_off + w.lo > off[i] + N) return -2;
            (w.kind == kPersistInit ? init_r : stat_r)[i].push_back({w.amp_off - off[i], w.amp_off - off[i] + w.lo});
            if (w.kind == kPersistStats &&
                (w.pass >= (uint32_t)W.nslots || w.hi + w.nslots > (uint32_t)W.nslots || w.pass < w.hi ||
                 w.pass >= w.hi + w.nslots))
                return -2;
        } else {
            const int r = (int)w.pass - first_pass[i];
            if (w.amp_off != off[i] || r < 0 || r >= (int)plans[i].passes.size()) return -2;
            const DevPass &P = W.passes[w.pass];
            if (P.n != n[i] || w.lo >= w.hi || w.hi > (1ULL << (n[i] - P.t))) return -2;
            pass_r[i][r].push_back({w.lo, w.hi});
        }
    }
    for (int i = 0; i < count; ++i) {
        const uint64_t N = 1ULL << n[i];
        if (!covers_once(init_r[i], N) || !covers_once(stat_r[i], N)) return -3;
        for (size_t r = 0; r < plans[i].passes.size(); ++r)
            if (!covers_once(pass_r[i][r], 1ULL << (n[i] - plans[i].passes[r].t))) return -3;
    }
    // dependencies: an initial chunk waits for nothing, an item of pass r
    // for every initial chunk and every item of passes 0..r-1, a statistics
    // chunk for every pass item
    std::vector<std::vector<uint32_t>> level_start(count);
    for (int i = 0; i < count; ++i) {
        uint32_t acc = (uint32_t)init_r[i].size();
        level_start[i].push_back(acc);
        for (auto &pr : pass_r[i]) {
            acc += (uint32_t)pr.size();
            level_start[i].push_back(acc);
        }
    }
    for (const PersistItem &w : it) {
        const int i = (int)w.inst;
        const uint32_t want = w.kind == kPersistInit    ? 0u
                              : w.kind == kPersistStats ? level_start[i].back()
                                                        : level_start[i][w.pass - first_pass[i]];
        if (w.need != want) return -4;
    }
    // level structure: need = the number of the instance's items with a
    // smaller need, all of which come earlier in the list
    for (int i = 0; i < count; ++i) {
        std::vector<std::pair<uint32_t, size_t>> lv;      // (need, list position)
        for (size_t j = 0; j < it.size(); ++j)
            if (it[j].inst == (uint32_t)i) {
                if (it[j].total != nitem[i]) return -6;
                lv.push_back({it[j].need, j});
            }
        for (auto &x : lv) {
            uint32_t smaller = 0;
            size_t last = 0;
            bool any = false;
            for (auto &y : lv)
                if (y.first < x.first) {
                    ++smaller;
                    last = std::max(last, y.second);
                    any = true;
                }
            if (smaller != x.first || (any && last > x.second)) return -4;
        }
    }
    // randomized schedule
    cd *psi = reinterpret_cast<cd *>(psi_out);
    std::vector<double> part((size_t)std::max(1, W.nslots) * 12, 0.0);
    std::vector<uint32_t> done(count, 0);
    uint64_t z = seed;
    auto rnd = [&]() {
        z += 0x9E3779B97F4A7C15ULL;
        uint64_t x = z;
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
        return x ^ (x >> 31);
    };
    size_t head = 0;
    std::vector<size_t> inflight;
    while (head < it.size() || !inflight.empty()) {
        std::vector<size_t> ready;
        for (size_t k = 0; k < inflight.size(); ++k)
            if (done[it[inflight[k]].inst] >= it[inflight[k]].need) ready.push_back(k);
        const bool can_take = head < it.size() && (int)inflight.size() < workers;
        if (!can_take && ready.empty()) return -5;
        if (can_take && (ready.empty() || (rnd() & 1))) {
            inflight.push_back(head++);
            continue;
        }
        const size_t k = ready[rnd() % ready.size()];
        const PersistItem w = it[inflight[k]];
        inflight.erase(inflight.begin() + (long)k);
        if (w.kind == kPersistInit) {
            for (uint32_t e = 0; e < w.lo; ++e) psi[w.amp_off + e] = cd(w.f0, 0.0);
            psi[w.amp_off] = cd(w.f1, 0.0);
        } else if (w.kind == kPersistStats) {
            work_stats_chunk(psi + w.amp_off, w.lo, (double)w.f0, &part[(size_t)w.pass * 12]);
        } else {
            emulate_tiles(view, W.passes[w.pass], w.lo, w.hi, psi + w.amp_off);
        }
        if (++done[w.inst] == w.total && w.kind == kPersistStats)
            for (int c = 0; c < 12; ++c) {
                double s = 0;
                for (uint32_t j = 0; j < w.nslots; ++j) s += part[(size_t)(w.hi + j) * 12 + c];
                sums_out[(size_t)w.inst * 12 + c] = s;
            }
    }
    for (int i = 0; i < count; ++i)
        if (done[i] != nitem[i]) return -6;
    return 0;
}

// The library's diagonal-prefix fold (the gates after a leading Hadamard
// layer): the kept gates in order into `rest` (room for ng), their number
// into *nrest, the fold masks into nb[kMaxQubits] and m[3] (T-count bits
// 0, 1, 2); returns the number of gates folded.
extern "C" int emul_fold(const qs_gate *g, size_t ng, qs_gate *rest, int *nrest, uint64_t *nb, uint64_t *m)
{
    std::vector<qs_gate> r;
    FoldArgs f;
    const size_t nf = fold_diagonal_prefix(g, ng, &r, &f);
    for (size_t i = 0; i < r.size(); ++i) rest[i] = r[i];
    *nrest = (int)r.size();
    for (int q = 0; q < kMaxQubits; ++q) nb[q] = f.nb[q];
    m[0] = f.m1;
    m[1] = f.m2;
    m[2] = f.m4;
    return (int)nf;
}
