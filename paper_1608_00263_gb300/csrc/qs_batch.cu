// qs_batch.cu -- batched ensemble of independent random circuits.
//
// The paper averages statistics over ensembles of circuit instances (Sec.
// "Characterizing quantum supremacy": 10 instances per point; Sec.
// "Convergence to Porter-Thomas": means and spreads over instances).  Here
// every instance keeps its complex64 state resident in one device buffer.
// The default engine runs a whole batch as one persistent launch: a work
// list of initial-state chunks, every instance's fused passes (round-major:
// pass r of every instance before pass r + 1 of any) and statistics chunks,
// taken from a device queue, each item waiting only for its own instance's
// earlier items (per-instance completion counters, bounded waits).  The
// lockstep engine instead makes round r one launch of the batched
// fused-pass kernel over (instance, tile range) items of every instance's
// pass r (one launch per tile size), with the statistics in two more
// launches.  Either way the device work of a run is captured once into a
// CUDA graph and replayed while the gate lists stay the same.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <utility>
#include <vector>

#include "qs_device.cuh"

using namespace qs;

namespace {

constexpr int kItemTiles = 8;              // tiles per work item of a round
constexpr uint64_t kStatChunk = kWorkChunk;   // amplitudes per statistics item

// Initial states, one statistics item (<= 2^16 amplitudes of one instance,
// a multiple of 32 at a 32-amplitude boundary) per block iteration: every
// amplitude fill[j] (2^(-n/2) where the instance's circuit opens with a
// Hadamard layer: the uniform state; else 0), then the item's first
// amplitude first[j] (1 at the start of an instance in |0...0>).
__global__ void k_batch_init(float2 *amps, const uint64_t *item_off, const uint64_t *item_cnt,
                             const float *fill, const float *first, int nitems)
{
    for (int j = blockIdx.x; j < nitems; j += gridDim.x) {
        float4 *a = reinterpret_cast<float4 *>(amps + item_off[j]);
        const uint64_t units = item_cnt[j] / 2;
        const float v = fill[j];
        const float4 u = make_float4(v, 0.f, v, 0.f);
        for (uint64_t e = threadIdx.x; e < units; e += blockDim.x) a[e] = u;
        if (threadIdx.x == 0) a[0] = make_float4(first[j], 0.f, v, 0.f);
    }
}

uint64_t fnv1a(const void *data, size_t n, uint64_t h = 1469598103934665603ULL)
{
    const unsigned char *p = (const unsigned char *)data;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ULL;
    }
    return h;
}

}  // namespace

struct qs_batch {
    int count = 0;
    std::vector<int> n;
    std::vector<uint64_t> off;        // element offset of each state
    uint64_t total = 0;               // elements
    float2 *amps = nullptr;
    cudaStream_t user_stream = nullptr, cap_stream = nullptr;
    int device = 0, num_sms = 1;
    // current plan and graph
    uint64_t key = 0;
    bool ready = false;
    void *dev = nullptr;              // plan + items + statistics tables
    double *part = nullptr, *sums = nullptr;
    cudaGraphExec_t exec = nullptr;
    int kmax_last = 0;
    std::vector<double> host_sums;
    double round_bytes = 0;           // algorithmic bytes of the prepared rounds
    // options (qs_batch_set_options): a fixed tile size for every instance
    // (0 = the planner's default), or the autotuned size of each n
    int tile_log2 = 0;
    int autotune = 0;
    int engine = QS_BATCH_PERSISTENT;
    uint32_t *sync = nullptr;         // persistent engine: PersistCtl, then done[count]
    std::map<int, int> tile_for_n;    // tile bits chosen per instance size (autotune)
    std::map<int, double> tune_ms;     // the winner's time per size class
    std::vector<int> tile_used;        // tile bits of each instance's plan (0: no pass)
};

static void batch_release_plan(qs_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    if (b->dev) cudaFree(b->dev);
    if (b->part) cudaFree(b->part);
    if (b->sums) cudaFree(b->sums);
    if (b->sync) cudaFree(b->sync);
    b->dev = nullptr;
    b->sync = nullptr;
    b->part = b->sums = nullptr;
    b->ready = false;
}

// Tile sizes chosen by the autotuner, per (device, qubits, engine): a process-wide
// cache, so later batches with instances of the same size skip the timing.
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int>, int> g_tuned_tile;

// Plans for instances `idx` with tile size tbits[i] (0 = default), on host
// threads.  plans[i] is left empty for instances not listed or whose list
// is only the Hadamard layer.
static qs_status plan_instances(const qs_batch *b, const qs_gate *gates, const uint64_t *offsets,
                                const std::vector<size_t> &hl, const std::vector<int> &idx,
                                const std::vector<int> &tbits, std::vector<Plan> *plans)
{
    plans->assign(b->count, Plan());
    std::vector<qs_status> st(idx.size(), QS_OK);
    std::vector<std::string> msg(idx.size());
    const unsigned nth = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (unsigned w = 0; w < nth; ++w)
        pool.emplace_back([&, w]() {
            for (size_t k = w; k < idx.size(); k += nth) {
                const int i = idx[k];
                const size_t ng = (size_t)(offsets[i + 1] - offsets[i]) - hl[i];
                if (ng == 0) continue;
                qs_opts o{};
                o.mode = QS_MODE_FUSED;
                o.tile_log2 = tbits[i];
                PlanParams pp = default_plan_params(b->n[i], QS_C64, &o);
                st[k] = build_plan(pp, gates + offsets[i] + hl[i], ng, &(*plans)[i]);
                if (st[k]) msg[k] = last_error_cstr();
            }
        });
    for (auto &t : pool) t.join();
    for (size_t k = 0; k < idx.size(); ++k)
        if (st[k]) return set_error(st[k], "instance %d: %s", idx[k], msg[k].c_str());
    return QS_OK;
}

// Lockstep rounds of the listed instances: the concatenated plans and the
// work items (instance, pass, <= kItemTiles tiles) of every (round, tile
// size), laid out for one device buffer.
struct RoundLaunch {
    int round, tbits;
    size_t first, count;
    bool full;          // some item's pass needs the full interpreter
};
struct Rounds {
    std::vector<DevPass> passes;
    std::vector<DevPhase> phases;
    std::vector<DevOp> ops;
    std::vector<unsigned char> items;
    std::vector<RoundLaunch> launches;
    double bytes = 0;                // algorithmic bytes (16 per amplitude per pass)
};

static void build_rounds(const qs_batch *b, const std::vector<Plan> &plans, const std::vector<int> &idx,
                         Rounds *R)
{
    *R = Rounds();
    std::vector<int> first_pass(b->count, 0);
    int max_passes = 0;
    for (int i : idx) {
        first_pass[i] = (int)R->passes.size();
        const int pb = (int)R->phases.size(), ob = (int)R->ops.size();
        for (DevPass p : plans[i].passes) {
            p.phase_begin += pb;
            R->passes.push_back(p);
        }
        for (DevPhase h : plans[i].phases) {
            h.op_begin += ob;
            h.op_end += ob;
            R->phases.push_back(h);
        }
        R->ops.insert(R->ops.end(), plans[i].ops.begin(), plans[i].ops.end());
        max_passes = std::max(max_passes, (int)plans[i].passes.size());
        R->bytes += (double)plans[i].passes.size() * 16.0 * std::ldexp(1.0, b->n[i]);
    }
    const size_t isz = batch_item_bytes();
    for (int r = 0; r < max_passes; ++r)
        for (int tb = 5; tb <= 13; ++tb) {
            RoundLaunch L{r, tb, R->items.size() / isz, 0, false};
            for (int i : idx) {
                if (r >= (int)plans[i].passes.size()) continue;
                const DevPass &p = plans[i].passes[r];
                if (p.t != tb) continue;
                L.full = L.full || plan_pass_needs_full(plans[i], r);
                const uint64_t ntiles = 1ULL << (b->n[i] - p.t);
                for (uint64_t t0 = 0; t0 < ntiles; t0 += kItemTiles) {
                    const uint64_t t1 = std::min<uint64_t>(ntiles, t0 + kItemTiles);
                    R->items.resize(R->items.size() + isz);
                    batch_item_fill(R->items.data() + R->items.size() - isz, b->off[i],
                                    (uint32_t)(first_pass[i] + r), (uint32_t)t0, (uint32_t)t1);
                    ++L.count;
                }
            }
            if (L.count) R->launches.push_back(L);
        }
}

// Section offsets of a Rounds layout in a device buffer: passes | phases |
// ops | items, each 256-byte aligned.
struct RoundOffsets {
    size_t pass, phase, op, item, total;
};
static RoundOffsets round_offsets(const Rounds &R)
{
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    RoundOffsets o;
    o.pass = 0;
    o.phase = align(o.pass + R.passes.size() * sizeof(DevPass));
    o.op = align(o.phase + R.phases.size() * sizeof(DevPhase));
    o.item = align(o.op + R.ops.size() * sizeof(DevOp));
    o.total = align(o.item + R.items.size());
    return o;
}

static void round_pack(const Rounds &R, const RoundOffsets &o, unsigned char *host)
{
    std::memcpy(host + o.pass, R.passes.data(), R.passes.size() * sizeof(DevPass));
    std::memcpy(host + o.phase, R.phases.data(), R.phases.size() * sizeof(DevPhase));
    std::memcpy(host + o.op, R.ops.data(), R.ops.size() * sizeof(DevOp));
    if (!R.items.empty()) std::memcpy(host + o.item, R.items.data(), R.items.size());
}

static qs_status launch_rounds(const qs_batch *b, cudaStream_t st, const Rounds &R, const RoundOffsets &o,
                               const unsigned char *D)
{
    const size_t isz = batch_item_bytes();
    for (const RoundLaunch &L : R.launches)
        if (qs_status rs = launch_batch_round(st, b->num_sms, b->amps, D + o.item + L.first * isz, (int)L.count,
                                              L.tbits, (const DevPass *)(D + o.pass),
                                              (const DevPhase *)(D + o.phase), (const DevOp *)(D + o.op), L.full))
            return rs;
    return QS_OK;
}

// The per-pass interpreter choice of the listed instances' plans (the
// persistent work items carry it).
static std::vector<std::vector<char>> full_flags(const std::vector<Plan> &plans)
{
    std::vector<std::vector<char>> f(plans.size());
    for (size_t i = 0; i < plans.size(); ++i)
        for (size_t r = 0; r < plans[i].passes.size(); ++r) f[i].push_back(plan_pass_needs_full(plans[i], (int)r));
    return f;
}

// Work layout in one device buffer: passes | phases | ops | items, each
// 256-byte aligned.
static RoundOffsets work_offsets(const Work &W)
{
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    RoundOffsets o;
    o.pass = 0;
    o.phase = align(o.pass + W.passes.size() * sizeof(DevPass));
    o.op = align(o.phase + W.phases.size() * sizeof(DevPhase));
    o.item = align(o.op + W.ops.size() * sizeof(DevOp));
    o.total = align(o.item + W.items.size() * sizeof(PersistItem));
    return o;
}

static void work_pack(const Work &W, const RoundOffsets &o, unsigned char *host)
{
    std::memcpy(host + o.pass, W.passes.data(), W.passes.size() * sizeof(DevPass));
    std::memcpy(host + o.phase, W.phases.data(), W.phases.size() * sizeof(DevPhase));
    std::memcpy(host + o.op, W.ops.data(), W.ops.size() * sizeof(DevOp));
    if (!W.items.empty()) std::memcpy(host + o.item, W.items.data(), W.items.size() * sizeof(PersistItem));
}

// Zeroes the queue head, the abort / error words and the completion
// counters, then launches the persistent kernel over the packed work.
static qs_status launch_work(const qs_batch *b, cudaStream_t st, const Work &W, const RoundOffsets &o,
                             const unsigned char *D, uint32_t *sync, double *part, double *sums)
{
    const size_t words = sizeof(PersistCtl) / 4 + (size_t)b->count;
    QS_CUDA_TRY(cudaMemsetAsync(sync, 0, words * 4, st));
    bool any_full = false;
    for (const PersistItem &w : W.items) any_full = any_full || w.kind == kPersistPassFull;
    return launch_batch_persistent(st, b->num_sms, b->amps, (const PersistItem *)(D + o.item), (int)W.items.size(),
                                   (const DevPass *)(D + o.pass), (const DevPhase *)(D + o.phase),
                                   (const DevOp *)(D + o.op), sync + sizeof(PersistCtl) / 4, (PersistCtl *)sync,
                                   part, sums, any_full);
}

// Reads the persistent kernel's error word after its stream has finished.
static qs_status work_error(const uint32_t *sync)
{
    PersistCtl c;
    QS_CUDA_TRY(cudaMemcpy(&c, sync, sizeof c, cudaMemcpyDeviceToHost));
    if (c.err) return set_error(QS_ERR_TIMEOUT, "ensemble kernel: a dependency wait ran out");
    return QS_OK;
}

// One untimed and one timed run (CUDA events) of the listed instances'
// evolution with the given plans on the batch's engine; *ms = the timed
// run.  The runs overwrite those instances' states.
static qs_status time_plans(qs_batch *b, const std::vector<Plan> &plans, const std::vector<int> &idx,
                            const std::vector<size_t> &hl, cudaEvent_t e0, cudaEvent_t e1, float *ms, bool *empty)
{
    Rounds R;
    Work W;
    RoundOffsets o;
    std::vector<unsigned char> host;
    if (b->engine == QS_BATCH_ROUNDS) {
        build_rounds(b, plans, idx, &R);
        *empty = R.launches.empty();
        o = round_offsets(R);
        host.assign(o.total, 0);
        round_pack(R, o, host.data());
    } else {
        build_work(b->n, b->off, plans, full_flags(plans), idx, hl, false, &W);
        *empty = W.passes.empty();
        o = work_offsets(W);
        host.assign(o.total, 0);
        work_pack(W, o, host.data());
    }
    if (*empty) return QS_OK;
    void *dev = nullptr, *sync = nullptr;
    cudaError_t e = cudaMalloc(&dev, o.total);
    if (e == cudaSuccess) e = cudaMalloc(&sync, sizeof(PersistCtl) + 4 * (size_t)b->count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (dev) cudaFree(dev);
        return set_error(QS_ERR_OOM, "autotune plan buffer: %s", cudaGetErrorString(e));
    }
    qs_status rc = QS_OK;
    e = cudaMemcpy(dev, host.data(), o.total, cudaMemcpyHostToDevice);
    auto run = [&]() -> qs_status {
        if (b->engine == QS_BATCH_ROUNDS) return launch_rounds(b, b->cap_stream, R, o, (const unsigned char *)dev);
        return launch_work(b, b->cap_stream, W, o, (const unsigned char *)dev, (uint32_t *)sync, nullptr, nullptr);
    };
    if (e == cudaSuccess) rc = run();
    if (e == cudaSuccess && !rc) {
        cudaEventRecord(e0, b->cap_stream);
        rc = run();
        cudaEventRecord(e1, b->cap_stream);
        if (!rc) e = cudaEventSynchronize(e1);
        if (!rc && e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    }
    cudaError_t ef = cudaStreamSynchronize(b->cap_stream);
    if (e == cudaSuccess) e = ef;
    if (!rc && e != cudaSuccess) rc = set_error(QS_ERR_CUDA, "autotune run: %s", cudaGetErrorString(e));
    if (!rc && b->engine != QS_BATCH_ROUNDS) rc = work_error((const uint32_t *)sync);
    cudaFree(dev);
    cudaFree(sync);
    return rc;
}

// Autotuner: for every instance size n not yet in the cache, time the
// evolution of the batch's own instances of that size (their real circuits,
// on their own state memory, which the run resets afterwards) on the
// batch's engine with each candidate tile size -- 9..13 qubits, capped at
// n -- and keep the fastest.  One untimed and one timed run (CUDA events)
// per candidate.  The cache is per (device, n, engine).
static qs_status batch_autotune(qs_batch *b, const qs_gate *gates, const uint64_t *offsets,
                                const std::vector<size_t> &hl)
{
    std::map<int, std::vector<int>> by_n;
    for (int i = 0; i < b->count; ++i) by_n[b->n[i]].push_back(i);
    if (qs_status s0 = batch_kernel_setup()) return s0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    QS_CUDA_TRY(cudaEventCreate(&e0));
    QS_CUDA_TRY(cudaEventCreate(&e1));
    qs_status rc = QS_OK;
    for (auto &kv : by_n) {
        const int n = kv.first;
        {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            auto it = g_tuned_tile.find(std::make_tuple(b->device, n, b->engine));
            if (it != g_tuned_tile.end()) {
                b->tile_for_n[n] = it->second;
                continue;
            }
        }
        int best_t = 0;
        double best_ms = 1e300;
        for (int t = std::min(9, n); t <= std::min(13, n); ++t) {
            std::vector<int> tb(b->count, t);
            std::vector<Plan> plans;
            if ((rc = plan_instances(b, gates, offsets, hl, kv.second, tb, &plans))) break;
            float ms = 0;
            bool empty = false;
            if ((rc = time_plans(b, plans, kv.second, hl, e0, e1, &ms, &empty))) break;
            if (empty) break;                       // only Hadamard layers: nothing to time
            if (ms < best_ms) {
                best_ms = ms;
                best_t = t;
            }
        }
        if (rc) break;
        if (best_t) {
            b->tile_for_n[n] = best_t;
            b->tune_ms[n] = best_ms;
            std::lock_guard<std::mutex> lock(g_tune_mu);
            g_tuned_tile[std::make_tuple(b->device, n, b->engine)] = best_t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

extern "C" qs_status qs_batch_create(int count, const int *nqubits, void *cuda_stream, qs_batch **out)
{
    clear_error();
    if (count < 1 || !nqubits || !out) return set_error(QS_ERR_INVALID_ARG, "bad batch arguments");
    qs_batch *b = new qs_batch();
    b->count = count;
    b->user_stream = (cudaStream_t)cuda_stream;
    for (int i = 0; i < count; ++i) {
        if (nqubits[i] < 5 || nqubits[i] > 30) {
            delete b;
            return set_error(QS_ERR_INVALID_ARG, "instance %d: n = %d outside 5..30", i, nqubits[i]);
        }
        b->n.push_back(nqubits[i]);
        b->off.push_back(b->total);
        b->total += 1ULL << nqubits[i];
    }
    cudaGetDevice(&b->device);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    cudaError_t e = cudaMalloc((void **)&b->amps, b->total * sizeof(float2));
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return set_error(QS_ERR_OOM, "batch states (%llu amplitudes): %s", (unsigned long long)b->total,
                         cudaGetErrorString(e));
    }
    e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaFree(b->amps);
        delete b;
        return set_error(QS_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
    }
    *out = b;
    return QS_OK;
}

extern "C" qs_status qs_batch_set_options(qs_batch *b, const qs_opts *opts)
{
    clear_error();
    if (!b) return set_error(QS_ERR_INVALID_ARG, "batch is NULL");
    const int mode = opts ? opts->mode : QS_MODE_FUSED;
    if (mode == QS_MODE_FUSED_TC)
        return set_error(QS_ERR_UNSUPPORTED, "the batched pass has no tensor-core form");
    if (mode != QS_MODE_FUSED) return set_error(QS_ERR_INVALID_ARG, "batch mode must be QS_MODE_FUSED");
    const int t = opts ? opts->tile_log2 : 0, at = opts ? opts->autotune : 0;
    if (t != 0 && (t < 5 || t > 13)) return set_error(QS_ERR_INVALID_ARG, "tile_log2 %d outside 5..13", t);
    if (at != 0 && at != 1) return set_error(QS_ERR_INVALID_ARG, "autotune must be 0 or 1");
    if (at && t) return set_error(QS_ERR_INVALID_ARG, "autotune chooses the tile size: tile_log2 must be 0");
    b->tile_log2 = t;
    b->autotune = at;
    b->tile_for_n.clear();
    b->tune_ms.clear();
    b->ready = false;                 // the next run replans
    return QS_OK;
}

extern "C" qs_status qs_batch_set_engine(qs_batch *b, int engine)
{
    clear_error();
    if (!b) return set_error(QS_ERR_INVALID_ARG, "batch is NULL");
    if (engine != QS_BATCH_PERSISTENT && engine != QS_BATCH_ROUNDS)
        return set_error(QS_ERR_INVALID_ARG, "engine %d is neither QS_BATCH_PERSISTENT nor QS_BATCH_ROUNDS", engine);
    if (engine != b->engine) {
        b->engine = engine;
        b->tile_for_n.clear();
        b->tune_ms.clear();
        b->ready = false;             // the next run replans
    }
    return QS_OK;
}

extern "C" qs_status qs_batch_plan_info(const qs_batch *b, int *tile_log2, double *run_bytes)
{
    clear_error();
    if (!b) return set_error(QS_ERR_INVALID_ARG, "batch is NULL");
    if (!b->ready) return set_error(QS_ERR_INVALID_ARG, "no run has been prepared yet");
    if (tile_log2)
        for (int i = 0; i < b->count; ++i) tile_log2[i] = b->tile_used[i];
    if (run_bytes) {
        // rounds, the initial states (one write) and the statistics (one read)
        *run_bytes = b->round_bytes + 16.0 * (double)b->total;
    }
    return QS_OK;
}

extern "C" qs_status qs_batch_destroy(qs_batch *b)
{
    clear_error();
    if (!b) return QS_OK;
    cudaStreamSynchronize(b->user_stream);
    batch_release_plan(b);
    if (b->amps) cudaFree(b->amps);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
    return QS_OK;
}

extern "C" qs_status qs_batch_state(const qs_batch *b, int i, void **device_amps)
{
    clear_error();
    if (!b || !device_amps || i < 0 || i >= b->count) return set_error(QS_ERR_INVALID_ARG, "bad instance");
    *device_amps = b->amps + b->off[i];
    return QS_OK;
}

extern "C" qs_status qs_batch_sample(qs_batch *b, uint64_t k, uint64_t seed, double r_mes, uint64_t *out)
{
    clear_error();
    if (!b || (k && !out)) return set_error(QS_ERR_INVALID_ARG, "bad arguments");
    if (!(r_mes >= 0 && r_mes <= 1)) return set_error(QS_ERR_INVALID_ARG, "r_mes must lie in [0, 1]");
    if (k > (1ULL << 40) / (uint64_t)b->count) return set_error(QS_ERR_INVALID_ARG, "too many samples");
    return batch_sampler_run(b->user_stream, b->num_sms, b->amps, b->off.data(), b->n.data(), b->count, k, seed,
                             r_mes, out);
}

extern "C" qs_status qs_batch_correlation(qs_batch *b, const qs_state *ref, double *corr)
{
    clear_error();
    if (!b || !ref || !corr) return set_error(QS_ERR_INVALID_ARG, "bad arguments");
    if (ref->dt != QS_C64) return set_error(QS_ERR_INVALID_ARG, "reference state must be complex64");
    for (int i = 0; i < b->count; ++i)
        if (b->n[i] != ref->n)
            return set_error(QS_ERR_INVALID_ARG, "instance %d has %d qubits, reference %d", i, b->n[i], ref->n);
    // the reference is read on the batch's stream after its own pending work
    if (ref->stream != b->user_stream) {
        cudaError_t e = cudaStreamSynchronize(ref->stream);
        if (e != cudaSuccess) return set_error(QS_ERR_CUDA, "reference stream: %s", cudaGetErrorString(e));
    }
    std::vector<double> h((size_t)b->count * 5);
    if (qs_status st = batch_overlap_run(b->user_stream, b->num_sms, b->amps, ref->amps, b->off.data(), b->count,
                                         ref->n, h.data()))
        return st;
    const double N = std::ldexp(1.0, ref->n);
    for (int i = 0; i < b->count; ++i) {
        const double *v = &h[(size_t)i * 5];
        const double ma = v[2] / N, mb = v[4] / N;
        const double cov = v[0] / N - ma * mb;
        const double va = v[1] / N - ma * ma, vb = v[3] / N - mb * mb;
        corr[i] = (va > 0 && vb > 0) ? cov / std::sqrt(va * vb) : 0.0;
    }
    return QS_OK;
}

extern "C" qs_status qs_batch_mean_probabilities(qs_batch *b, double *out)
{
    clear_error();
    if (!b || !out) return set_error(QS_ERR_INVALID_ARG, "bad arguments");
    for (int i = 1; i < b->count; ++i)
        if (b->n[i] != b->n[0]) return set_error(QS_ERR_INVALID_ARG, "instances differ in size");
    const uint64_t N = 1ULL << b->n[0];
    double *d = nullptr;
    QS_CUDA_TRY(cudaMallocAsync((void **)&d, N * sizeof(double), b->user_stream));
    qs_status st = batch_mean_probs_run(b->user_stream, b->num_sms, b->amps, b->count, b->n[0], d);
    cudaError_t e = cudaSuccess;
    if (st == QS_OK) e = cudaMemcpyAsync(out, d, N * sizeof(double), cudaMemcpyDeviceToHost, b->user_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->user_stream);
    cudaFreeAsync(d, b->user_stream);
    if (st == QS_OK && e != cudaSuccess) st = set_error(QS_ERR_CUDA, "mean probabilities: %s", cudaGetErrorString(e));
    return st;
}

// Ends the capture of a run on the batch's private stream and instantiates
// its graph (rs: the status of the captured launches).
static qs_status batch_end_capture(qs_batch *b, qs_status rs)
{
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
    if (rs) {
        if (graph) cudaGraphDestroy(graph);
        return rs;
    }
    if (e != cudaSuccess) return set_error(QS_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return set_error(QS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    b->ready = true;
    return QS_OK;
}

// Plans every instance, lays out the concatenated plan, work items and
// statistics items in one device buffer, and records the run as a graph.
static qs_status batch_prepare(qs_batch *b, const qs_gate *gates, const uint64_t *offsets)
{
    const int C = b->count;
    // an instance whose circuit opens with a Hadamard layer starts from the
    // uniform state (written by k_batch_init) and plans the rest
    std::vector<size_t> hl(C);
    for (int i = 0; i < C; ++i)
        hl[i] = leading_h_layer(gates + offsets[i], (size_t)(offsets[i + 1] - offsets[i]), b->n[i]);
    if (b->autotune)
        if (qs_status s0 = batch_autotune(b, gates, offsets, hl)) return s0;
    std::vector<int> all(C), tbits(C, b->tile_log2);
    for (int i = 0; i < C; ++i) {
        all[i] = i;
        if (b->autotune && b->tile_for_n.count(b->n[i])) tbits[i] = b->tile_for_n[b->n[i]];
    }
    std::vector<Plan> plans;
    if (qs_status s0 = plan_instances(b, gates, offsets, hl, all, tbits, &plans)) return s0;
    b->tile_used.assign(C, 0);
    for (int i = 0; i < C; ++i)
        if (!plans[i].passes.empty()) b->tile_used[i] = plans[i].passes[0].t;
    if (b->engine == QS_BATCH_PERSISTENT) {
        // one persistent launch: initial states, passes, statistics
        Work W;
        build_work(b->n, b->off, plans, full_flags(plans), all, hl, true, &W);
        b->round_bytes = W.bytes;
        const RoundOffsets wo = work_offsets(W);
        std::vector<unsigned char> host(wo.total, 0);
        work_pack(W, wo, host.data());
        batch_release_plan(b);
        QS_CUDA_TRY(cudaMalloc(&b->dev, wo.total));
        QS_CUDA_TRY(cudaMalloc((void **)&b->part, (size_t)std::max(1, W.nslots) * kStatSums * sizeof(double)));
        QS_CUDA_TRY(cudaMalloc((void **)&b->sums, (size_t)C * kStatSums * sizeof(double)));
        QS_CUDA_TRY(cudaMalloc((void **)&b->sync, sizeof(PersistCtl) + 4 * (size_t)C));
        QS_CUDA_TRY(cudaMemcpy(b->dev, host.data(), wo.total, cudaMemcpyHostToDevice));
        if (qs_status s0 = batch_kernel_setup()) return s0;
        QS_CUDA_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        const qs_status rs =
            launch_work(b, b->cap_stream, W, wo, (const unsigned char *)b->dev, b->sync, b->part, b->sums);
        return batch_end_capture(b, rs);
    }
    Rounds R;
    build_rounds(b, plans, all, &R);
    b->round_bytes = R.bytes;
    // statistics items
    std::vector<uint64_t> s_off, s_cnt;
    std::vector<float> s_scale, s_fill, s_first;
    std::vector<int> first_item(C + 1);
    for (int i = 0; i < C; ++i) {
        first_item[i] = (int)s_off.size();
        const uint64_t N = 1ULL << b->n[i];
        const float v = hl[i] ? (float)std::pow(2.0, -0.5 * b->n[i]) : 0.f;
        for (uint64_t a = 0; a < N; a += kStatChunk) {
            s_off.push_back(b->off[i] + a);
            s_cnt.push_back(std::min<uint64_t>(kStatChunk, N - a));
            s_scale.push_back((float)std::ldexp(1.0, b->n[i]));
            s_fill.push_back(v);
            s_first.push_back(hl[i] ? v : (a == 0 ? 1.f : 0.f));
        }
    }
    first_item[C] = (int)s_off.size();
    const int nsi = (int)s_off.size();

    // one device buffer: rounds (passes | phases | ops | items) | s_off |
    // s_cnt | s_scale | first_item | inst_off | fill | first
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const RoundOffsets ro = round_offsets(R);
    size_t o_so = ro.total;
    size_t o_sc = align(o_so + s_off.size() * 8);
    size_t o_ss = align(o_sc + s_cnt.size() * 8);
    size_t o_fi = align(o_ss + s_scale.size() * 4);
    size_t o_io = align(o_fi + first_item.size() * 4);
    size_t o_vf = align(o_io + b->off.size() * 8);
    size_t o_v1 = align(o_vf + s_fill.size() * 4);
    size_t total = align(o_v1 + s_first.size() * 4);
    std::vector<unsigned char> host(total, 0);
    round_pack(R, ro, host.data());
    std::memcpy(host.data() + o_so, s_off.data(), s_off.size() * 8);
    std::memcpy(host.data() + o_sc, s_cnt.data(), s_cnt.size() * 8);
    std::memcpy(host.data() + o_ss, s_scale.data(), s_scale.size() * 4);
    std::memcpy(host.data() + o_fi, first_item.data(), first_item.size() * 4);
    std::memcpy(host.data() + o_io, b->off.data(), b->off.size() * 8);
    std::memcpy(host.data() + o_vf, s_fill.data(), s_fill.size() * 4);
    std::memcpy(host.data() + o_v1, s_first.data(), s_first.size() * 4);
    batch_release_plan(b);
    QS_CUDA_TRY(cudaMalloc(&b->dev, total));
    QS_CUDA_TRY(cudaMalloc((void **)&b->part, (size_t)nsi * kStatSums * sizeof(double)));
    QS_CUDA_TRY(cudaMalloc((void **)&b->sums, (size_t)C * kStatSums * sizeof(double)));
    QS_CUDA_TRY(cudaMemcpy(b->dev, host.data(), total, cudaMemcpyHostToDevice));
    unsigned char *D = (unsigned char *)b->dev;

    // record: reset all states, rounds, statistics
    if (qs_status s0 = batch_kernel_setup()) return s0;
    QS_CUDA_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    qs_status rs = QS_OK;
    k_batch_init<<<std::min(nsi, 16 * b->num_sms), 256, 0, b->cap_stream>>>(
        b->amps, (const uint64_t *)(D + o_so), (const uint64_t *)(D + o_sc), (const float *)(D + o_vf),
        (const float *)(D + o_v1), nsi);
    rs = launch_rounds(b, b->cap_stream, R, ro, D);
    if (!rs)
        rs = launch_batch_stats(b->cap_stream, b->num_sms, b->amps, (const uint64_t *)(D + o_so),
                                (const uint64_t *)(D + o_sc), (const float *)(D + o_ss), nsi,
                                (const int *)(D + o_fi), C, b->part, b->sums);
    return batch_end_capture(b, rs);
}

static qs_status batch_run_impl(qs_batch *b, const qs_gate *gates, const uint64_t *offsets, int kmax,
                                double *stats)
{
    clear_error();
    if (!b || !offsets || (kmax && !stats) || kmax < 0 || kmax > kMaxMoments)
        return set_error(QS_ERR_INVALID_ARG, "bad batch run arguments");
    if (offsets[0] != 0) return set_error(QS_ERR_INVALID_ARG, "offsets[0] must be 0");
    for (int i = 0; i < b->count; ++i) {
        if (offsets[i + 1] < offsets[i]) return set_error(QS_ERR_INVALID_ARG, "offsets decrease at %d", i);
        if (qs_status s2 = validate_gates(b->n[i], gates + offsets[i], (size_t)(offsets[i + 1] - offsets[i])))
            return set_error(s2, "instance %d: %s", i, last_error_cstr());
    }
    uint64_t key = fnv1a(offsets, (b->count + 1) * sizeof(uint64_t));
    key = fnv1a(gates, (size_t)offsets[b->count] * sizeof(qs_gate), key);
    if (!b->ready || key != b->key) {
        if (qs_status s2 = batch_prepare(b, gates, offsets)) return s2;
        b->key = key;
    }
    QS_CUDA_TRY(cudaGraphLaunch(b->exec, b->user_stream));
    b->host_sums.resize((size_t)b->count * kStatSums);
    QS_CUDA_TRY(cudaMemcpyAsync(b->host_sums.data(), b->sums, b->host_sums.size() * sizeof(double),
                                cudaMemcpyDeviceToHost, b->user_stream));
    PersistCtl ctl{};
    if (b->sync)
        QS_CUDA_TRY(cudaMemcpyAsync(&ctl, b->sync, sizeof ctl, cudaMemcpyDeviceToHost, b->user_stream));
    QS_CUDA_TRY(cudaStreamSynchronize(b->user_stream));
    if (ctl.err) return set_error(QS_ERR_TIMEOUT, "ensemble kernel: a dependency wait ran out");
    const int w = 3 + kmax;
    if (stats)
        for (int i = 0; i < b->count; ++i) {
            double *o = stats + (size_t)i * w;
            stats_from_sums(&b->host_sums[(size_t)i * kStatSums], b->n[i], kmax, &o[0], &o[1], &o[2], o + 3);
        }
    return QS_OK;
}

extern "C" qs_status qs_batch_run(qs_batch *b, const qs_gate *gates, const uint64_t *offsets, int kmax,
                                  double *stats)
{
    const qs_status st = batch_run_impl(b, gates, offsets, kmax, stats);
    return st ? st : check_poll_all();
}

namespace qs {
QS_CHECK_READER(check_poll_batch)
}

extern "C" qs_status qs_batch_apply(qs_batch *b, const qs_gate *gates, const uint64_t *offsets)
{
    return qs_batch_run(b, gates, offsets, 0, nullptr);
}
