// qs_api.cu -- the C ABI entry points of include/qs.h (host side): argument
// validation, memory classification, planning and dispatch to the kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "qs_device.cuh"

using namespace qs;

namespace {

constexpr size_t kWsDoubles = 1 << 16;

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device-side address of page-locked host memory (cudaHostAlloc /
// cudaHostRegister: mapped into the device's address space), else nullptr.
void *pinned_device_view(void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Writes a deferred reset before the state is read or changed.
qs_status materialize(const qs_state *s)
{
    if (!s->zero_pending) return QS_OK;
    s->zero_pending = false;
    ++s->version;
    return launch_init_zero(const_cast<qs_state *>(s));
}

qs_status check_state(const qs_state *s)
{
    if (!s) return set_error(QS_ERR_INVALID_ARG, "state is NULL");
    return QS_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

uint64_t fnv1a(const void *data, size_t n, uint64_t h = 1469598103934665603ULL)
{
    const unsigned char *p = (const unsigned char *)data;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ULL;
    }
    return h;
}

qs_status alloc_workspace(qs_state *s)
{
    QS_CUDA_TRY(cudaMalloc((void **)&s->ws_f64, kWsDoubles * sizeof(double)));
    s->ws_f64_count = kWsDoubles;
    QS_CUDA_TRY(cudaMalloc((void **)&s->ws_u64, 64 * sizeof(uint64_t)));
    QS_CUDA_TRY(cudaHostAlloc(&s->hbox, kHostBoxBytes, cudaHostAllocMapped));
    QS_CUDA_TRY(cudaHostGetDevicePointer(&s->hbox_dev, s->hbox, 0));
    return QS_OK;
}

qs_status new_state(int n, qs_dtype dt, void *stream, qs_state **out)
{
    if (n < 1 || n > kMaxQubits) return set_error(QS_ERR_INVALID_ARG, "n = %d out of range 1..%d", n, kMaxQubits);
    if (dt != QS_C64 && dt != QS_C128) return set_error(QS_ERR_INVALID_ARG, "bad dtype %d", (int)dt);
    if (!out) return set_error(QS_ERR_INVALID_ARG, "out is NULL");
    int dev = 0;
    QS_CUDA_TRY(cudaGetDevice(&dev));
    qs_state *s = new qs_state();
    s->n = n;
    s->dt = dt;
    s->amps = nullptr;
    s->owns = false;
    s->stream = (cudaStream_t)stream;
    s->device = dev;
    s->ws_f64 = nullptr;
    s->ws_u64 = nullptr;
    cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (s->num_sms <= 0) s->num_sms = 1;
    *out = s;
    return QS_OK;
}

void free_state(qs_state *s)
{
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    if (s->ro_stream) cudaStreamSynchronize(s->ro_stream);
    if (s->ro_buf) cudaFree(s->ro_buf);
    if (s->ro_ready) cudaEventDestroy(s->ro_ready);
    if (s->ro_done) cudaEventDestroy(s->ro_done);
    if (s->ro_stream) cudaStreamDestroy(s->ro_stream);
    if (s->owns && s->amps) cudaFree(s->amps);
    if (s->ws_f64) cudaFree(s->ws_f64);
    if (s->ws_u64) cudaFree(s->ws_u64);
    if (s->hbox) cudaFreeHost(s->hbox);
    if (s->rc_buf) cudaFree(s->rc_buf);
    if (s->stage) cudaFreeHost(s->stage);
    for (DevicePlanSlot &c : s->plan_cache.slot) {
        if (c.dev) cudaFree(c.dev);
        if (c.staging) cudaFreeHost(c.staging);
        if (c.done) cudaEventDestroy(c.done);
    }
    delete s;
}

}  // namespace

extern "C" const char *qs_version(void) { return "qs 1.0 sm_103a"; }

extern "C" qs_status qs_state_create(int n, qs_dtype dt, void *cuda_stream, qs_state **out)
{
    clear_error();
    qs_state *s = nullptr;
    qs_status st = new_state(n, dt, cuda_stream, &s);
    if (st) return st;
    const size_t bytes = (size_t(1) << n) * dtype_bytes(dt);
    cudaError_t e = cudaMalloc(&s->amps, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_state(s);
        return set_error(QS_ERR_OOM, "cannot allocate %zu bytes for %d qubits: %s", bytes, n,
                         cudaGetErrorString(e));
    }
    s->owns = true;
    if ((st = alloc_workspace(s)) || (st = launch_init_zero(s))) {
        free_state(s);
        return st;
    }
    s->is_zero = true;
    *out = s;
    return QS_OK;
}

extern "C" qs_status qs_state_attach(int n, qs_dtype dt, void *device_amps, void *cuda_stream,
                                     qs_state **out)
{
    clear_error();
    if (!device_amps) return set_error(QS_ERR_INVALID_ARG, "device_amps is NULL");
    if (((uintptr_t)device_amps & 15) != 0) return set_error(QS_ERR_INVALID_ARG, "device_amps not 16-byte aligned");
    if (!is_device_ptr(device_amps)) return set_error(QS_ERR_INVALID_ARG, "device_amps is not device memory");
    qs_state *s = nullptr;
    qs_status st = new_state(n, dt, cuda_stream, &s);
    if (st) return st;
    s->amps = device_amps;
    s->owns = false;
    s->escaped = true;
    if ((st = alloc_workspace(s))) {
        free_state(s);
        return st;
    }
    *out = s;
    return QS_OK;
}

extern "C" qs_status qs_state_destroy(qs_state *s)
{
    clear_error();
    free_state(s);
    return QS_OK;
}

extern "C" qs_status qs_state_amplitudes(const qs_state *s, void **device_amps)
{
    clear_error();
    if (qs_status st = check_state(s)) return st;
    if (!device_amps) return set_error(QS_ERR_INVALID_ARG, "device_amps is NULL");
    DeviceGuard g(s->device);
    if (qs_status st = materialize(s)) return st;
    s->escaped = true;
    *device_amps = s->amps;
    return QS_OK;
}

extern "C" qs_status qs_state_reset(qs_state *s)
{
    clear_error();
    if (qs_status st = check_state(s)) return st;
    DeviceGuard g(s->device);
    s->is_zero = true;
    ++s->version;
    if (s->escaped) {
        s->zero_pending = false;
        return launch_init_zero(s);
    }
    s->zero_pending = true;   // written by the next use (or skipped, see qs_apply_circuit)
    return QS_OK;
}

static qs_status get_plan(qs_state *s, const qs_gate *gates, size_t ng, const qs_opts *o,
                          const Plan **plan, const void **dev, DevicePlanSlot **slot_out = nullptr)
{
    PlanParams pp = default_plan_params(s->n, s->dt, o);
    uint64_t key = fnv1a(gates, ng * sizeof(qs_gate));
    key = fnv1a(&pp, sizeof pp, key);
    DevicePlanCache &pc = s->plan_cache;
    DevicePlanSlot *c = nullptr;
    for (DevicePlanSlot &x : pc.slot)
        if (x.valid && x.key == key && x.ngates == ng) c = &x;
    if (!c) {
        // least recently used slot; wait until the device is done with it
        c = pc.slot[0].last_use <= pc.slot[1].last_use ? &pc.slot[0] : &pc.slot[1];
        if (c->done) QS_CUDA_TRY(cudaEventSynchronize(c->done));
        c->valid = false;
        Plan p;
        if (qs_status st = build_plan(pp, gates, ng, &p)) return st;
        const size_t b_pass = p.passes.size() * sizeof(DevPass);
        const size_t b_phase = p.phases.size() * sizeof(DevPhase);
        const size_t b_ops = p.ops.size() * sizeof(DevOp);
        const size_t b_blk = p.tc_words.size() * sizeof(uint32_t);
        const size_t total = b_pass + b_phase + b_ops + b_blk + 16;
        if (c->bytes < total) {
            if (c->dev) cudaFree(c->dev);
            if (c->staging) cudaFreeHost(c->staging);
            c->dev = c->staging = nullptr;
            c->bytes = 0;
            const size_t cap = total + total / 2;
            cudaError_t e = cudaMalloc(&c->dev, cap);
            if (e == cudaSuccess) e = cudaMallocHost(&c->staging, cap);
            if (e != cudaSuccess) {
                cudaGetLastError();
                if (c->dev) cudaFree(c->dev);
                c->dev = nullptr;
                c->staging = nullptr;
                return set_error(QS_ERR_OOM, "plan upload: %s", cudaGetErrorString(e));
            }
            c->bytes = cap;
        }
        unsigned char *h = static_cast<unsigned char *>(c->staging);
        std::memset(h, 0, total);
        std::memcpy(h, p.passes.data(), b_pass);
        std::memcpy(h + b_pass, p.phases.data(), b_phase);
        std::memcpy(h + b_pass + b_phase, p.ops.data(), b_ops);
        if (b_blk) std::memcpy(h + b_pass + b_phase + b_ops, p.tc_words.data(), b_blk);
        QS_CUDA_TRY(cudaMemcpyAsync(c->dev, h, total, cudaMemcpyHostToDevice, s->stream));
        if (!c->done) QS_CUDA_TRY(cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming));
        QS_CUDA_TRY(cudaEventRecord(c->done, s->stream));
        c->key = key;
        c->ngates = ng;
        c->plan = std::move(p);
        c->valid = true;
    }
    c->last_use = ++pc.clock;
    *plan = &c->plan;
    *dev = c->dev;
    if (slot_out) *slot_out = c;
    return QS_OK;
}

// Marks the slot busy until the work just enqueued on the stream completes.
static qs_status slot_in_use(qs_state *s, DevicePlanSlot *c)
{
    QS_CUDA_TRY(cudaEventRecord(c->done, s->stream));
    return QS_OK;
}

// ---- autotune (qs_opts.autotune = 1) ----
// Fused forms chosen per (device, n, dtype, requested mode, precision) by
// timing candidate tile sizes -- and, for QS_MODE_FUSED_TC, the register
// form at the default tile -- on a scratch copy of the state; cached for the
// rest of the process.  States above kAutotuneMaxQubits keep the defaults
// (13-qubit tiles, the fastest measured from 20 qubits on).
constexpr int kAutotuneMaxQubits = 26;
static std::mutex g_autotune_mu;
static std::map<std::tuple<int, int, int, int, int>, std::pair<int, int>> g_autotune;   // -> (mode, tile)

static qs_status autotune_opts(qs_state *s, const qs_gate *gates, size_t ngates, const qs_opts *o, qs_opts *out)
{
    *out = *o;
    out->autotune = 0;
    out->tile_log2 = 0;
    if (o->mode == QS_MODE_PLAIN || s->n > kAutotuneMaxQubits) return QS_OK;
    const auto key = std::make_tuple(s->device, s->n, (int)s->dt, o->mode, o->precision);
    {
        std::lock_guard<std::mutex> lock(g_autotune_mu);
        auto it = g_autotune.find(key);
        if (it != g_autotune.end()) {
            out->mode = it->second.first;
            out->tile_log2 = it->second.second;
            return QS_OK;
        }
    }
    const int rb = s->dt == QS_C128 ? 4 : 5;
    std::vector<std::pair<int, int>> cand;            // (mode, tile)
    const int tmax = std::min(s->n, s->dt == QS_C128 ? 12 : 13);
    for (int t = std::max(rb, std::min(9, s->n)); t <= tmax; ++t) cand.push_back({QS_MODE_FUSED, t});
    if (o->mode == QS_MODE_FUSED_TC && s->dt == QS_C64 && s->n >= 13) cand.push_back({QS_MODE_FUSED_TC, 13});
    if (cand.size() <= 1) return QS_OK;
    // scratch copy of the state, evolved by every candidate in turn
    const size_t bytes = ((size_t)1 << s->n) * dtype_bytes(s->dt);
    void *scratch = nullptr;
    QS_CUDA_TRY(cudaMallocAsync(&scratch, bytes, s->stream));
    qs_state *t = nullptr;
    qs_status rc = materialize(s);
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(scratch, s->amps, bytes, cudaMemcpyDeviceToDevice, s->stream);
        if (e != cudaSuccess) rc = set_error(QS_ERR_CUDA, "autotune copy: %s", cudaGetErrorString(e));
    }
    if (!rc) rc = qs_state_attach(s->n, s->dt, scratch, s->stream, &t);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = set_error(QS_ERR_CUDA, "autotune events");
    std::pair<int, int> best{0, 0};
    float best_ms = 3.4e38f;
    for (size_t c = 0; !rc && c < cand.size(); ++c) {
        qs_opts co = *o;
        co.autotune = 0;
        co.mode = cand[c].first;
        co.tile_log2 = cand[c].first == QS_MODE_FUSED ? cand[c].second : 0;
        float ms = 0;
        if ((rc = qs_apply_circuit(t, gates, ngates, &co))) break;     // untimed: plans, uploads
        cudaEventRecord(e0, s->stream);
        if ((rc = qs_apply_circuit(t, gates, ngates, &co))) break;
        cudaEventRecord(e1, s->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = set_error(QS_ERR_CUDA, "autotune timing");
            break;
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = cand[c];
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (t) qs_state_destroy(t);
    cudaFreeAsync(scratch, s->stream);
    if (rc) return rc;
    clear_error();
    out->mode = best.first;
    out->tile_log2 = best.first == QS_MODE_FUSED ? best.second : 0;
    std::lock_guard<std::mutex> lock(g_autotune_mu);
    g_autotune[key] = best;
    return QS_OK;
}

static qs_status qs_apply_circuit_impl(qs_state *s, const qs_gate *gates, size_t ngates,
                                      const qs_opts *opts)
{
    clear_error();
    if (qs_status st = check_state(s)) return st;
    if (qs_status st = validate_gates(s->n, gates, ngates)) return st;
    if (opts && opts->autotune != 0 && opts->autotune != 1)
        return set_error(QS_ERR_INVALID_ARG, "autotune must be 0 or 1");
    qs_opts tuned;
    if (opts && opts->autotune == 1 && ngates) {
        if (opts->tile_log2) return set_error(QS_ERR_INVALID_ARG, "autotune chooses the tile size: tile_log2 must be 0");
        if (opts->mode == QS_MODE_FUSED_TC && (opts->precision < QS_PREC_DEFAULT || opts->precision > QS_PREC_TF32))
            return set_error(QS_ERR_INVALID_ARG, "tensor-core precision %d is not a qs_precision", opts->precision);
        if (opts->mode != QS_MODE_PLAIN && opts->mode != QS_MODE_FUSED && opts->mode != QS_MODE_FUSED_TC)
            return set_error(QS_ERR_INVALID_ARG, "unknown mode %d", opts->mode);
        DeviceGuard g(s->device);
        if (qs_status st = autotune_opts(s, gates, ngates, opts, &tuned)) return st;
        opts = &tuned;
    }
    const int mode = opts ? opts->mode : QS_MODE_FUSED;
    if (mode != QS_MODE_PLAIN && mode != QS_MODE_FUSED && mode != QS_MODE_FUSED_TC)
        return set_error(QS_ERR_INVALID_ARG, "unknown mode %d", mode);
    const int rb = s->dt == QS_C128 ? 4 : 5;
    if (mode == QS_MODE_FUSED && opts && opts->tile_log2 && (opts->tile_log2 < rb || opts->tile_log2 > rb + 8))
        return set_error(QS_ERR_INVALID_ARG, "tile_log2 %d outside %d..%d", opts->tile_log2, rb, rb + 8);
    if (mode == QS_MODE_FUSED_TC && opts && (opts->precision < QS_PREC_DEFAULT || opts->precision > QS_PREC_TF32))
        return set_error(QS_ERR_INVALID_ARG, "tensor-core precision %d is not a qs_precision", opts->precision);
    if (ngates == 0) return QS_OK;
    DeviceGuard g(s->device);
    ++s->version;
    // Sec. pt, cycle 0: on |0...0> a leading layer of Hadamards on every
    // qubit gives the uniform superposition: written in one pass, or, when
    // fused passes follow, generated by the first pass in shared memory (the
    // state is then neither written by a fill nor read by that pass)
    double uniform = 0.0;
    FoldArgs fold{};
    std::vector<qs_gate> rest;
    if (s->is_zero && !s->escaped) {
        if (size_t h = leading_h_layer(gates, ngates, s->n)) {
            s->zero_pending = false;
            if (ngates > h && mode != QS_MODE_PLAIN && s->n >= rb) {
                uniform = std::pow(2.0, -0.5 * s->n);
                ++s->version;
                // the T and CZ gates that reach the uniform state before any
                // non-diagonal gate on their qubits become its phases, formed
                // by the same first pass (register form, gates left to run)
                if (mode == QS_MODE_FUSED && fold_diagonal_prefix(gates + h, ngates - h, &rest, &fold) > 0 &&
                    !rest.empty()) {
                    gates = rest.data();
                    ngates = rest.size();
                    h = 0;
                } else {
                    fold.nfold = 0;
                }
            } else if (qs_status st = launch_init_uniform(s)) {
                return st;
            }
            gates += h;
            ngates -= h;
        }
    }
    if (qs_status st = materialize(s)) return st;
    s->is_zero = false;
    if (ngates == 0) return QS_OK;
    if (mode == QS_MODE_PLAIN || s->n < rb) {
        for (size_t i = 0; i < ngates; ++i)
            if (qs_status st = launch_plain_gate(s, gates[i])) return st;
        return QS_OK;
    }
    const Plan *plan;
    const void *dev;
    DevicePlanSlot *slot;
    if (qs_status st = get_plan(s, gates, ngates, opts, &plan, &dev, &slot)) {
        // the leading layer is still applied, as when it is written first
        if (uniform != 0.0) launch_init_uniform(s);
        return st;
    }
    if (qs_status st = run_fused_plan(s, *plan, dev, uniform, fold.nfold > 0 ? &fold : nullptr)) return st;
    return slot_in_use(s, slot);
}

extern "C" qs_status qs_prepare_circuit(qs_state *s, const qs_gate *gates, size_t ngates,
                                        const qs_opts *opts)
{
    clear_error();
    if (qs_status st = check_state(s)) return st;
    if (qs_status st = validate_gates(s->n, gates, ngates)) return st;
    const int mode = opts ? opts->mode : QS_MODE_FUSED;
    const int rb = s->dt == QS_C128 ? 4 : 5;
    if (ngates == 0 || mode == QS_MODE_PLAIN || s->n < rb) return QS_OK;
    if (mode != QS_MODE_FUSED && mode != QS_MODE_FUSED_TC)
        return set_error(QS_ERR_INVALID_ARG, "unknown mode %d", mode);
    if (mode == QS_MODE_FUSED_TC && opts && (opts->precision < QS_PREC_DEFAULT || opts->precision > QS_PREC_TF32))
        return set_error(QS_ERR_INVALID_ARG, "tensor-core precision %d is not a qs_precision", opts->precision);
    DeviceGuard g(s->device);
    // a leading Hadamard layer is written as the uniform state when the
    // circuit starts from |0...0> (the usual reset + apply): plan the rest
    std::vector<qs_gate> rest;
    if (!s->escaped) {
        const size_t h = leading_h_layer(gates, ngates, s->n);
        if (h && ngates > h && s->n >= rb && mode == QS_MODE_FUSED) {
            // as qs_apply_circuit: the folded diagonal prefix is no pass's work
            FoldArgs fold;
            if (fold_diagonal_prefix(gates + h, ngates - h, &rest, &fold) > 0 && !rest.empty()) {
                const Plan *plan;
                const void *dev;
                return get_plan(s, rest.data(), rest.size(), opts, &plan, &dev);
            }
        }
        gates += h;
        ngates -= h;
        if (ngates == 0) return QS_OK;
    }
    const Plan *plan;
    const void *dev;
    return get_plan(s, gates, ngates, opts, &plan, &dev);
}

static qs_status qs_probabilities_impl(const qs_state *s, void *out, int out_is_fp64)
{
    clear_error();
    if (qs_status st = check_state(s)) return st;
    if (!out) return set_error(QS_ERR_INVALID_ARG, "out is NULL");
    DeviceGuard g(s->device);
    if (qs_status st = materialize(s)) return st;
    const uint64_t N = 1ULL << s->n;
    const size_t esz = out_is_fp64 ? 8 : 4;
    if (is_device_ptr(out)) return launch_probabilities(s, out, out_is_fp64, 0, N);
    // an asynchronous read-out still copying may target the same host memory
    if (s->ro_done) QS_CUDA_TRY(cudaStreamWaitEvent(s->stream, s->ro_done, 0));
    if (void *view = pinned_device_view(out)) {
        // page-locked host output: the kernel writes it directly (one pass)
        if (qs_status st = launch_probabilities(s, view, out_is_fp64, 0, N)) return st;
        QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
        return QS_OK;
    }
    // pageable host output: convert in device chunks and copy back
    const uint64_t chunk = N < (1ULL << 24) ? N : (1ULL << 24);
    void *buf = nullptr;
    QS_CUDA_TRY(cudaMallocAsync(&buf, chunk * esz, s->stream));
    qs_status st = QS_OK;
    for (uint64_t f = 0; f < N && !st; f += chunk) {
        st = launch_probabilities(s, buf, out_is_fp64, f, chunk);
        if (st) break;
        cudaError_t e = cudaMemcpyAsync((char *)out + f * esz, buf, chunk * esz, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) st = set_error(QS_ERR_CUDA, "probabilities copy: %s", cudaGetErrorString(e));
    }
    cudaFreeAsync(buf, s->stream);
    cudaStreamSynchronize(s->stream);
    return st;
}

extern "C" qs_status qs_probabilities_async(const qs_state *s, void *out, int out_is_fp64)
{
    clear_error();
    if (qs_status st = check_state(s)) return st;
    if (!out) return set_error(QS_ERR_INVALID_ARG, "out is NULL");
    if (is_device_ptr(out) || !pinned_device_view(out)) return qs_probabilities(s, out, out_is_fp64);
    DeviceGuard g(s->device);
    if (qs_status st = materialize(s)) return st;
    const uint64_t N = 1ULL << s->n;
    const size_t esz = out_is_fp64 ? 8 : 4;
    const size_t bytes = N * esz;
    if (!s->ro_done) {
        cudaStream_t cs = nullptr;
        cudaEvent_t ready = nullptr, done = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            if (ready) cudaEventDestroy(ready);
            if (cs) cudaStreamDestroy(cs);
            return set_error(QS_ERR_CUDA, "read-out stream: %s", cudaGetErrorString(e));
        }
        s->ro_stream = cs;
        s->ro_ready = ready;
        s->ro_done = done;
    }
    if (s->ro_bytes < bytes) {
        // the buffer is replaced only after its last copy has finished
        QS_CUDA_TRY(cudaStreamSynchronize(s->ro_stream));
        if (s->ro_buf) cudaFree(s->ro_buf);
        s->ro_buf = nullptr;
        s->ro_bytes = 0;
        cudaError_t e = cudaMalloc(&s->ro_buf, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s->ro_buf = nullptr;
            return set_error(QS_ERR_OOM, "read-out buffer of %zu bytes: %s", bytes, cudaGetErrorString(e));
        }
        s->ro_bytes = bytes;
    }
    // complex64 states split the read-out at a chunk boundary: chunks
    // [0, csplit) straight into the host memory, the rest through ro_buf
    // (complex128 states and unaligned host memory take the copy engine only)
    void *view = pinned_device_view(out);
    const bool split = s->dt == QS_C64 && ((uintptr_t)view % 16) == 0;
    const uint64_t nchunks = readout_chunks(s);
    uint64_t csplit = 0;
    if (split) csplit = std::min<uint64_t>(nchunks, (uint64_t)std::llround(s->ro_frac * (double)nchunks));
    // a state of one partial chunk (n < 8) is written whole, never split
    if (split && N < 256 && csplit > 0) csplit = nchunks;
    const size_t direct = split ? std::min<size_t>(bytes, (size_t)csplit * 256 * esz) : 0;
    // the buffer is free once the previous copy has finished (an event never
    // recorded is complete)
    QS_CUDA_TRY(cudaStreamWaitEvent(s->stream, s->ro_done, 0));
    if (split && csplit > 0) {
        if (qs_status st = readout_c64(s, view, out_is_fp64 ? 2 : 1, s->ro_buf, csplit)) return st;
    } else {
        if (qs_status st = launch_probabilities(s, s->ro_buf, out_is_fp64, 0, N)) return st;
    }
    QS_CUDA_TRY(cudaEventRecord(s->ro_ready, s->stream));
    QS_CUDA_TRY(cudaStreamWaitEvent(s->ro_stream, s->ro_ready, 0));
    // 64 MB pieces: the small device-to-host copies of later calls (scalar
    // results, samples) share the copy engine and would otherwise wait for
    // the whole read-out, and with them the host's next launches
    constexpr size_t kPiece = size_t(64) << 20;
    for (size_t f = direct; f < bytes; f += kPiece)
        QS_CUDA_TRY(cudaMemcpyAsync((char *)out + f, (const char *)s->ro_buf + (f - direct),
                                    std::min(kPiece, bytes - f), cudaMemcpyDeviceToHost, s->ro_stream));
    QS_CUDA_TRY(cudaEventRecord(s->ro_done, s->ro_stream));
    return QS_OK;
}

extern "C" qs_status qs_readout_share(qs_state *s, double share, double *current)
{
    clear_error();
    if (qs_status st = check_state(s)) return st;
    if (share > 1.0) return set_error(QS_ERR_INVALID_ARG, "share %g above 1", share);
    if (share >= 0.0) s->ro_frac = share;
    else if (share < 0.0) s->ro_frac = 0.0;
    if (current) *current = s->ro_frac;
    return QS_OK;
}

extern "C" qs_status qs_state_sync(const qs_state *s)
{
    clear_error();
    if (qs_status st = check_state(s)) return st;
    DeviceGuard g(s->device);
    QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (s->ro_stream) QS_CUDA_TRY(cudaStreamSynchronize(s->ro_stream));
    return QS_OK;
}

static qs_status qs_sample_impl(const qs_state *s, uint64_t k, uint64_t seed, uint64_t *out)
{
    clear_error();
    if (qs_status st = check_state(s)) return st;
    if (k && !out) return set_error(QS_ERR_INVALID_ARG, "out is NULL");
    DeviceGuard g(s->device);
    if (qs_status st = materialize(s)) return st;
    if (k == 0) return sampler_run(s, 0, seed, nullptr);
    if (is_device_ptr(out)) return sampler_run(s, k, seed, out);
    // host output: the search kernel writes page-locked memory directly
    // (the caller's, or the state's mapped staging, then copied on the host)
    void *view = pinned_device_view(out), *stage = nullptr;
    if (!view)
        if (qs_status st = stage_view(s, k * sizeof(uint64_t), &stage, &view)) return st;
    if (qs_status st = sampler_run(s, k, seed, (uint64_t *)view)) return st;
    QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (stage) std::memcpy(out, stage, k * sizeof(uint64_t));
    return QS_OK;
}

static qs_status qs_cross_entropy_impl(const qs_state *s, const uint64_t *samples, uint64_t m,
                                      double *ce, double *delta_h)
{
    clear_error();
    if (qs_status st = check_state(s)) return st;
    if (m == 0) return set_error(QS_ERR_INVALID_ARG, "empty sample");
    if (!samples) return set_error(QS_ERR_INVALID_ARG, "samples is NULL");
    DeviceGuard g(s->device);
    if (qs_status st = materialize(s)) return st;
    double c = 0;
    qs_status st;
    if (is_device_ptr(samples)) {
        st = cross_entropy_run(s, samples, m, &c);
    } else if (void *view = pinned_device_view(const_cast<uint64_t *>(samples))) {
        // page-locked host samples are read by the kernel in place
        st = cross_entropy_run(s, (const uint64_t *)view, m, &c);
    } else {
        // pageable host samples: copied into the mapped staging on the host
        void *stage = nullptr, *dv = nullptr;
        if ((st = stage_view(s, m * sizeof(uint64_t), &stage, &dv))) return st;
        std::memcpy(stage, samples, m * sizeof(uint64_t));
        st = cross_entropy_run(s, (const uint64_t *)dv, m, &c);
    }
    if (st) return st;
    const double euler_gamma = 0.57721566490153286061;
    if (ce) *ce = c;
    if (delta_h) *delta_h = s->n * std::log(2.0) + euler_gamma - c;
    return QS_OK;
}

static qs_status qs_pt_moments_impl(const qs_state *s, int kmax, double *moments, double *entropy,
                                   double *uniform_ce, double *norm)
{
    clear_error();
    if (qs_status st = check_state(s)) return st;
    if (kmax < 0 || kmax > kMaxMoments) return set_error(QS_ERR_INVALID_ARG, "kmax %d outside 0..%d", kmax, kMaxMoments);
    if (kmax > 0 && !moments) return set_error(QS_ERR_INVALID_ARG, "moments is NULL");
    DeviceGuard g(s->device);
    if (qs_status st = materialize(s)) return st;
    return stats_moments(s, kmax, moments, entropy, uniform_ce, norm);
}

extern "C" qs_status qs_state_copy_out(const qs_state *s, void *host_amps)
{
    clear_error();
    if (qs_status st = check_state(s)) return st;
    if (!host_amps) return set_error(QS_ERR_INVALID_ARG, "host_amps is NULL");
    DeviceGuard g(s->device);
    if (qs_status st = materialize(s)) return st;
    const size_t bytes = (size_t(1) << s->n) * dtype_bytes(s->dt);
    QS_CUDA_TRY(cudaMemcpyAsync(host_amps, s->amps, bytes, cudaMemcpyDefault, s->stream));
    QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return QS_OK;
}

extern "C" qs_status qs_state_copy_in(qs_state *s, const void *host_amps)
{
    clear_error();
    if (qs_status st = check_state(s)) return st;
    if (!host_amps) return set_error(QS_ERR_INVALID_ARG, "host_amps is NULL");
    DeviceGuard g(s->device);
    const size_t bytes = (size_t(1) << s->n) * dtype_bytes(s->dt);
    s->zero_pending = false;
    s->is_zero = false;
    ++s->version;
    QS_CUDA_TRY(cudaMemcpyAsync(s->amps, host_amps, bytes, cudaMemcpyDefault, s->stream));
    QS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return QS_OK;
}

static qs_status qs_adjoint_gradient_impl(qs_state *s, const qs_gate *gates, size_t ngates,
                                         const uint64_t *samples, uint64_t m, const qs_opts *opts,
                                         double *loss, double *grad)
{
    clear_error();
    if (qs_status st = check_state(s)) return st;
    if (qs_status st = validate_gates(s->n, gates, ngates)) return st;
    if (m == 0 || !samples) return set_error(QS_ERR_INVALID_ARG, "empty sample");
    if (ngates && !grad) return set_error(QS_ERR_INVALID_ARG, "grad is NULL");
    DeviceGuard g(s->device);
    s->zero_pending = false;
    if (qs_status st = launch_init_zero(s)) return st;
    s->is_zero = true;
    if (qs_status st = qs_apply_circuit(s, gates, ngates, opts)) return st;
    uint64_t *buf = nullptr;
    const uint64_t *dx = samples;
    if (!is_device_ptr(samples)) {
        QS_CUDA_TRY(cudaMallocAsync((void **)&buf, m * sizeof(uint64_t), s->stream));
        cudaError_t e = cudaMemcpyAsync(buf, samples, m * sizeof(uint64_t), cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) {
            cudaFreeAsync(buf, s->stream);
            return set_error(QS_ERR_CUDA, "sample upload: %s", cudaGetErrorString(e));
        }
        dx = buf;
    }
    double ce = 0;
    qs_status st = cross_entropy_run(s, dx, m, &ce);   // also range-checks the samples
    if (!st) st = adjoint_run(s, gates, ngates, dx, m, grad);
    ++s->version;   // the reverse sweep leaves the state un-applied
    if (buf) cudaFreeAsync(buf, s->stream);
    cudaStreamSynchronize(s->stream);
    if (!st && loss) *loss = ce;
    return st;
}

extern "C" qs_status qs_cycle_statistics(qs_state *s, const qs_gate *gates, size_t ngates, const qs_opts *opts,
                                         int kmax, double *stats, size_t capacity, size_t *ncycles)
{
    clear_error();
    if (qs_status st = check_state(s)) return st;
    if (qs_status st = validate_gates(s->n, gates, ngates)) return st;
    if (!ncycles || kmax < 0 || kmax > kMaxMoments) return set_error(QS_ERR_INVALID_ARG, "bad arguments");
    for (size_t i = 1; i < ngates; ++i)
        if (gates[i].cycle < gates[i - 1].cycle)
            return set_error(QS_ERR_INVALID_ARG, "gate %zu: cycle numbers decrease", i);
    // cycle groups
    std::vector<size_t> starts;
    for (size_t i = 0; i < ngates; ++i)
        if (i == 0 || gates[i].cycle != gates[i - 1].cycle) starts.push_back(i);
    *ncycles = starts.size();
    if (!stats || capacity < starts.size()) return QS_OK;   // count query
    DeviceGuard g(s->device);
    s->zero_pending = false;
    if (qs_status st = launch_init_zero(s)) return st;
    s->is_zero = true;
    const int w = 4 + kmax;
    std::vector<double> mom(kMaxMoments);
    for (size_t c = 0; c < starts.size(); ++c) {
        const size_t b = starts[c], e = c + 1 < starts.size() ? starts[c + 1] : ngates;
        if (qs_status st = qs_apply_circuit(s, gates + b, e - b, opts)) return st;
        double *row = stats + c * w;
        row[0] = (double)gates[b].cycle;
        if (qs_status st = stats_moments(s, kmax, mom.data(), &row[2], &row[3], &row[1])) return st;
        for (int k = 0; k < kmax; ++k) row[4 + k] = mom[k];
    }
    return QS_OK;
}

// ---- public entry points that launch device work: in the checked build
// they end with a poll of the device check words ----
extern "C" qs_status qs_apply_circuit(qs_state *s, const qs_gate *gates, size_t ngates, const qs_opts *opts)
{
    const qs_status st = qs_apply_circuit_impl(s, gates, ngates, opts);
    return st ? st : check_poll_all();
}

extern "C" qs_status qs_probabilities(const qs_state *s, void *out, int out_is_fp64)
{
    const qs_status st = qs_probabilities_impl(s, out, out_is_fp64);
    return st ? st : check_poll_all();
}

extern "C" qs_status qs_sample(const qs_state *s, uint64_t k, uint64_t seed, uint64_t *out)
{
    const qs_status st = qs_sample_impl(s, k, seed, out);
    return st ? st : check_poll_all();
}

extern "C" qs_status qs_pt_moments(const qs_state *s, int kmax, double *moments, double *entropy, double *uniform_ce, double *norm)
{
    const qs_status st = qs_pt_moments_impl(s, kmax, moments, entropy, uniform_ce, norm);
    return st ? st : check_poll_all();
}

extern "C" qs_status qs_cross_entropy(const qs_state *s, const uint64_t *samples, uint64_t m, double *ce, double *delta_h)
{
    const qs_status st = qs_cross_entropy_impl(s, samples, m, ce, delta_h);
    return st ? st : check_poll_all();
}

extern "C" qs_status qs_adjoint_gradient(qs_state *s, const qs_gate *gates, size_t ngates, const uint64_t *samples, uint64_t m, const qs_opts *opts, double *loss, double *grad)
{
    const qs_status st = qs_adjoint_gradient_impl(s, gates, ngates, samples, m, opts, loss, grad);
    return st ? st : check_poll_all();
}

namespace qs {
QS_CHECK_READER(check_poll_api)

qs_status check_poll_all()
{
#ifdef QS_CHECKED
    QS_CUDA_TRY(cudaDeviceSynchronize());
    for (qs_status (*f)() : {check_poll_api, check_poll_plain, check_poll_fused, check_poll_stats,
                             check_poll_batch, check_poll_adjoint})
        if (qs_status st = f()) return st;
#endif
    return QS_OK;
}
}  // namespace qs

#ifdef QS_CHECKED
// A guarded access one element past a 4-element buffer: the check records
// site 901 and skips the access.
__global__ void k_check_probe(float *buf, uint64_t n, uint64_t i)
{
    if (QS_DCHECK(i < n, 901)) buf[i] = 1.f;
}
#endif

extern "C" qs_status qs_check_probe(void)
{
    clear_error();
#ifdef QS_CHECKED
    float *buf = nullptr;
    QS_CUDA_TRY(cudaMalloc((void **)&buf, 4 * sizeof(float)));
    k_check_probe<<<1, 1>>>(buf, 4, 4);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(buf);
    if (e != cudaSuccess) return set_error(QS_ERR_CUDA, "check probe: %s", cudaGetErrorString(e));
    return check_poll_all();
#else
    return set_error(QS_ERR_UNSUPPORTED, "not a checked build (QS_CHECKED)");
#endif
}

extern "C" int qs_build_flags(void)
{
#ifdef QS_CHECKED
    return QS_BUILD_CHECKED;
#else
    return 0;
#endif
}
