#!/usr/bin/env python3
"""Benchmark of the random-circuit state-vector hot path on GB300.

One step = one pass of the whole path over one synthetic circuit instance:
generate the circuit (grid rules of Sec. "Convergence to Porter-Thomas"),
reset the state, plan + evolve (fused tile passes), write the 2^n output
probabilities, Porter-Thomas statistics (moments 1..10, entropy, uniform
cross entropy, norm), draw m samples, sample cross entropy (Eq. ae).  Each
step uses a new circuit seed, so nothing is cached between steps.

Metric: cycles/s = circuit depth / step time.  Default workload: the 5x6
grid, 30 qubits, depth 40, complex64, 1e6 samples.

Prints one JSON line (rank 0).  With --impl reference the oracle (FP64 CPU)
is timed instead on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "grid5x6_n30_d40": dict(rows=5, cols=6, dead=(), depth=40, m=1_000_000, fp64_probs=True),
    "grid6x6m2_n34_d40": dict(rows=6, cols=6, dead=((0, 0), (5, 5)), depth=40, m=1_000_000,
                              fp64_probs=False),
    "grid4x5_n20_d25": dict(rows=4, cols=5, dead=(), depth=25, m=100_000, fp64_probs=True),
    # small case for profiler captures (2.1 GB state)
    "grid4x7_n28_d40": dict(rows=4, cols=7, dead=(), depth=40, m=1_000_000, fp64_probs=True),
}
DEFAULT_WORKLOAD = "grid5x6_n30_d40"
METRIC = "cycles/s (random circuit, state-vector evolution + statistics + sampling)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--mode", choices=["fused", "tc"], default="fused")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the one-off plain-mode comparison run")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="time only the 24-qubit adjoint gradient (a profiling case)")
    ap.add_argument("--ensemble-only", action="store_true",
                    help="time only the 4096-circuit ensemble (a profiling case)")
    ap.add_argument("--ensemble-runs", default="default,autotuned,lockstep_default",
                    help="ensemble runs to time: default, autotuned (persistent engine), "
                         "lockstep_default (lockstep engine)")
    ap.add_argument("--ensemble-count", type=int, default=4096,
                    help="instances of the ensemble recipe (the first K; a smaller profiling case)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_seed(rank):
    """Circuit-seed base of a replica: ranks run disjoint circuit streams."""
    return 1_000_003 * rank


def job_max_ms(local_ms, dist, device):
    """Max of a timing over all ranks (the job's wall time)."""
    if dist is None:
        return float(local_ms)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, max_ms):
    """Whole-job throughput: units processed by all ranks / max time."""
    return units_per_rank * world / (max_ms / 1000.0)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def kernel_launches_per_step(passes):
    # fused passes (the first one generates the leading Hadamard layer's
    # uniform state itself) + fused read-out (probabilities, statistics
    # partials and chunk sums: 1) + statistics (final sum, read-back = 2) +
    # sampler (3 scan kernels, read-back, search = 5) + cross entropy
    # (kernel, final sum, 2 read-backs = 4)
    return passes + 1 + 2 + 5 + 4


def leading_h_layer(qs, g, n):
    """Length of a leading layer of H on every qubit (n, else 0): applied to
    |0...0>, the library generates that layer's uniform state in the first
    fused pass (or writes it as one uniform fill)."""
    import numpy as np
    if len(g) < n or not np.all(g["kind"][:n] == qs.QS_H):
        return 0
    return n if len(set(g["q0"][:n].tolist())) == n else 0


def fold_diagonal_prefix(qs, g):
    """Gates left to run after the library folds the diagonal prefix that
    follows a leading Hadamard layer (register form): a T or CZ none of whose
    qubits has met a non-diagonal gate becomes a phase of the first pass's
    generated state.  Returns (number folded, remaining gates)."""
    import numpy as np
    touched, keep, nf = 0, [], 0
    diag = (qs.QS_T, qs.QS_CZ, qs.QS_RZ, qs.QS_CPHASE)
    for i in range(len(g)):
        k, a, b = int(g["kind"][i]), int(g["q0"][i]), int(g["q1"][i])
        two = k in (qs.QS_CZ, qs.QS_CPHASE)
        m = (1 << a) | ((1 << b) if two else 0)
        if (k == qs.QS_T or k == qs.QS_CZ) and not touched & m:
            nf += 1
            continue
        if k not in diag:
            touched |= m
        keep.append(i)
    return nf, g[np.array(keep, dtype=np.int64)]


def device_state_copy(qs, torch, h, n):
    """A device copy of a complex64 state (as 2^(n+1) floats)."""
    ptr = qs.qs_state_amplitudes(h)
    out = torch.empty(2 << n, dtype=torch.float32, device="cuda")
    src = torch.as_tensor(_CudaArray(ptr, 2 << n), device="cuda")
    out.copy_(src)
    return out


def device_rel_l2(qs, torch, h, n, ref):
    """||psi - ref|| / ||ref|| over device memory, in FP64 chunks."""
    src = torch.as_tensor(_CudaArray(qs.qs_state_amplitudes(h), 2 << n), device="cuda")
    num = den = 0.0
    step = 1 << 27
    for i in range(0, 2 << n, step):
        a, b = src[i:i + step].double(), ref[i:i + step].double()
        num += float(torch.sum((a - b) ** 2))
        den += float(torch.sum(b * b))
    return math.sqrt(num / den)


class _CudaArray:
    """A raw device pointer of `count` float32 values, for torch.as_tensor."""

    def __init__(self, ptr, count):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": "<f4", "data": (ptr, False),
                                         "version": 3}


def applied_plan(qs, n, g, md, prec=0):
    """Launches and algorithmic bytes of applying g (complex64) to the reset
    state.  A leading Hadamard layer followed by fused passes is generated by
    the first pass in shared memory (that pass writes 2^n amplitudes and
    reads none), in the register form with the diagonal prefix after it
    folded in as phases (those gates are no pass's work); alone, or before
    plain per-gate kernels, it is one uniform fill (2^n amplitudes written)."""
    k = leading_h_layer(qs, g, n)
    N8 = 8.0 * (1 << n)
    if len(g) == k:
        return {"passes": 0, "launches": 1 if k else 0, "bytes": N8 if k else 0.0, "fill": k}
    rest = g[k:]
    if k and md == qs.QS_MODE_FUSED:
        nf, folded_rest = fold_diagonal_prefix(qs, rest)
        if nf and len(folded_rest):
            rest = folded_rest
    st = qs.qs_plan_circuit(n, qs.QS_C64, rest, mode=md, precision=prec)
    if md == qs.QS_MODE_PLAIN:
        return {"passes": st["passes"], "launches": st["passes"] + (1 if k else 0),
                "bytes": st["bytes"] + (N8 if k else 0.0), "fill": k}
    return {"passes": st["passes"], "launches": st["passes"],
            "bytes": st["bytes"] - (N8 if k else 0.0), "fill": k}


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    import paper_1608_00263_gb300 as qs
    from paper_1608_00263_gb300 import build as qs_build

    qs_build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    W = WORKLOADS[args.workload]
    dead = None
    if W["dead"]:
        dead = np.zeros(W["rows"] * W["cols"], dtype=np.uint8)
        for r, c in W["dead"]:
            dead[r * W["cols"] + c] = 1
    n = W["rows"] * W["cols"] - len(W["dead"])
    depth, m = W["depth"], W["m"]
    mode = qs.QS_MODE_FUSED if args.mode == "fused" else qs.QS_MODE_FUSED_TC
    stream = torch.cuda.current_stream()
    h = qs.qs_state_create(n, qs.QS_C64, stream)
    probs = torch.empty(1 << n, dtype=torch.float64 if W["fp64_probs"] else torch.float32,
                        device="cuda")
    samples = torch.empty(m, dtype=torch.int64, device="cuda")
    base_seed = replica_seed(rank)

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    apply_ms = []
    timed_gates = []
    results = {}

    def prepare(i):
        gates = qs.qs_circuit_generate(W["rows"], W["cols"], depth, base_seed + i, dead)  # a1
        qs.qs_prepare_circuit(h, gates, mode=mode)                                      # a3 (host plan)
        return gates

    # Host planning is pipelined with the device: circuit i+1 is generated and
    # planned while the GPU evolves circuit i (the state keeps two plans), so
    # each timed step holds one generate + plan and one evolution + read-out.
    def step(i, timed, gates):
        seed = base_seed + i
        qs.qs_state_reset(h)                                                         # a2
        # one call: the leading Hadamard layer's uniform state is generated
        # by the first fused pass; the events bracket the passes
        e0, e1 = ev(), ev()
        e0.record(stream)
        qs.qs_apply_circuit(h, gates, mode=mode)                                     # a2, a4-a6
        e1.record(stream)
        nxt = prepare(i + 1)                                                         # overlaps a4-a6
        qs.qs_probabilities(h, probs, fp64=W["fp64_probs"])                          # a7
        st = qs.qs_pt_moments(h, 10)                                                 # a8
        qs.qs_sample(h, m, 1000 + seed, out=samples)                                 # a9
        ce, dh = qs.qs_cross_entropy(h, samples)                                     # a10
        if timed:
            apply_ms.append((e0, e1))
            timed_gates.append(gates)
        results["last"] = dict(entropy=st["entropy"], norm=st["norm"], delta_h=dh, ce=ce)
        return nxt

    gates_next = prepare(0)
    for i in range(args.warmup):
        gates_next = step(i, False, gates_next)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    t_start, t_end = ev(), ev()
    torch.cuda.synchronize()
    t_start.record(stream)
    for i in range(args.steps):
        gates_next = step(args.warmup + i, True, gates_next)
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    passes_ms = sum(a.elapsed_time(b) for a, b in apply_ms)
    total_ms = job_max_ms(total_ms, dist, "cuda")
    plans_seen = [applied_plan(qs, n, g, mode) for g in timed_gates]
    passes_seen = [pl["passes"] for pl in plans_seen]
    value = job_value(depth * args.steps, world, total_ms)
    passes_total = sum(passes_seen)
    # algorithmic bytes: 16 per amplitude per pass (read + write), 8 for the
    # first pass of a circuit, which generates its input (the uniform state)
    bytes_total = sum(pl["bytes"] for pl in plans_seen)
    pass_bytes = bytes_total / passes_total      # average per launch
    avg_pass_ms = passes_ms / passes_total
    peaks, peak_src = load_peaks()
    hbm_peak = float(peaks["hbm_gbs"])
    achieved = pass_bytes / (avg_pass_ms / 1000.0) / 1e9
    traffic, traffic_launch = load_traffic(args.mode, n) or (None, None)

    # ---- e2e: same steps through the public API with host buffers ----
    probs_host = [torch.empty(1 << n, dtype=probs.dtype, pin_memory=True) for _ in range(2)]
    samples_host = np.empty(m, dtype=np.uint64)

    def e2e_run(asynchronous, seed0):
        """W untimed + K timed steps through the public API with host buffers:
        the gate list in, the probabilities and the samples out each step.
        Synchronous: the read-out kernel writes the page-locked buffer
        directly.  Asynchronous: qs_probabilities_async, the copy engine moves
        step i's probabilities (two buffers, alternating) while step i+1's
        circuit evolves; the timed region ends when the last copy has landed."""
        h2d = d2h = 0
        torch.cuda.synchronize()
        gates = qs.qs_circuit_generate(W["rows"], W["cols"], depth, seed0, dead)
        qs.qs_prepare_circuit(h, gates, mode=mode)
        t0 = None
        for i in range(args.warmup + args.steps):
            if i == args.warmup:
                qs.qs_state_sync(h)
                torch.cuda.synchronize()
                h2d = d2h = 0
                t0 = time.perf_counter()
            seed = seed0 + i
            qs.qs_state_reset(h)
            qs.qs_apply_circuit(h, gates, mode=mode)
            # the next circuit is generated and planned while this one evolves
            nxt = qs.qs_circuit_generate(W["rows"], W["cols"], depth, seed + 1, dead)
            qs.qs_prepare_circuit(h, nxt, mode=mode)
            if asynchronous:
                qs.qs_probabilities_async(h, probs_host[i % 2], fp64=W["fp64_probs"])
            else:
                qs.qs_probabilities(h, probs_host[0], fp64=W["fp64_probs"])
            qs.qs_pt_moments(h, 10)
            qs.qs_sample(h, m, 1000 + seed, out=samples_host)
            qs.qs_cross_entropy(h, samples_host)
            h2d += gates.nbytes + samples_host.nbytes
            d2h += probs_host[0].numel() * probs_host[0].element_size() + samples_host.nbytes + 8 * 14
            gates = nxt
        qs.qs_state_sync(h)
        torch.cuda.synchronize()
        ms = job_max_ms((time.perf_counter() - t0) * 1000.0, dist, "cuda")
        return job_value(depth * args.steps, world, ms), h2d, d2h

    e2e_value, h2d, d2h = e2e_run(False, base_seed + 10_000)
    e2e_async_value, _, _ = e2e_run(True, base_seed + 20_000)
    # share of the probabilities the read-out kernel wrote into host memory
    # itself in the asynchronous steps (the copy engine moved the rest)
    async_share = qs.qs_readout_share(h)

    # ---- one-off comparison of the forms (apply only, untimed region) ----
    compare = {}
    if not args.no_compare and rank == 0:
        gates = qs.qs_circuit_generate(W["rows"], W["cols"], depth, base_seed, dead)
        ref_state = None
        for name, md, prec in (("plain", qs.QS_MODE_PLAIN, 0), ("fused", qs.QS_MODE_FUSED, 0),
                               ("tc", qs.QS_MODE_FUSED_TC, qs.QS_PREC_FP16X3),
                               ("tc_bf16x3", qs.QS_MODE_FUSED_TC, qs.QS_PREC_BF16X3),
                               ("tc_bf16x6", qs.QS_MODE_FUSED_TC, qs.QS_PREC_BF16X6),
                               ("tc_tf32x3", qs.QS_MODE_FUSED_TC, qs.QS_PREC_TF32X3),
                               ("tc_tf32", qs.QS_MODE_FUSED_TC, qs.QS_PREC_TF32)):
            qs.qs_state_reset(h)
            qs.qs_prepare_circuit(h, gates, mode=md, precision=prec)
            torch.cuda.synchronize()
            a, b = ev(), ev()
            a.record(stream)
            qs.qs_apply_circuit(h, gates, mode=md, precision=prec)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            pst = applied_plan(qs, n, gates, md, prec)
            nrm = qs.qs_pt_moments(h, 0)["norm"]
            compare[name] = {"apply_ms": round(ms, 3), "cycles_per_s": round(depth / (ms / 1e3), 2),
                             "launches": pst["launches"], "norm": round(nrm, 7),
                             "norm_drift_within_1e-5": abs(nrm - 1) <= 1e-5,
                             "hbm_frac_of_measured": round(pst["bytes"] / (ms / 1e3) / 1e9 / hbm_peak, 4)}
            # relative L2 distance to the register form's state (both FP32
            # evolutions; the lossy operand precisions show their error here)
            if name == "fused":
                ref_state = device_state_copy(qs, torch, h, n)
            elif name.startswith("tc") and ref_state is not None:
                compare[name]["rel_l2_vs_fused"] = float("%.3e" % device_rel_l2(qs, torch, h, n, ref_state))
        del ref_state

    # ---- 34 qubits (6x6 grid minus two corners, depth 40): the three forms,
    # apply only, one circuit each (outside the timed region) ----
    n34 = None
    if rank == 0 and not args.no_compare and args.workload == DEFAULT_WORKLOAD:
        qs.qs_state_destroy(h)
        h = None
        del probs, samples, probs_host
        torch.cuda.empty_cache()
        n34 = forms_34(qs, torch, hbm_peak)
        h = qs.qs_state_create(n, qs.QS_C64, stream)

    ens = noisy = single = small = grad = None
    if rank == 0 and not args.no_compare and args.workload == DEFAULT_WORKLOAD:
        if h is not None:
            qs.qs_state_destroy(h)
        h = None
        torch.cuda.empty_cache()
        ens = ensemble_4096(qs, torch, hbm_peak, args.ensemble_runs.split(","))
        noisy = noisy_trajectories(qs, torch)
        single = single_error_sweep(qs, torch)
        small = grid20_forms(qs, torch)
        grad = adjoint_24(qs, torch)
        h = qs.qs_state_create(n, qs.QS_C64, stream)

    # arithmetic rates of this GPU (FMA chains, CUDA events): the roofline
    # denominators of the ALU-bound passes
    alu = {}
    for kind, name in ((0, "fp32_fma"), (1, "fp32x2_fma"), (2, "fp64_fma")):
        alu[name + "_tflops"] = round(2.0 * qs.qs_alu_rate(kind, stream) / 1e12, 2)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(W, dead, n)

    qs.qs_state_destroy(h)
    out = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "cycles/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded random circuits of the paper's grid rules)",
        "config": workload_config(args, n, world),
        "apply_cycles_per_s": round(depth * args.steps / (passes_ms / 1000.0), 3),
        "passes_per_circuit": passes_total / args.steps,
        "roofline": {"kernel": ("k_fused_pass<float,5,0,0>" if args.mode == "fused"
                                else "k_fused_pass<float,5,1,1>"),
                     "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak,
                     "peak_source": peak_src + " hbm_gbs", "unit": "GB/s",
                     "frac": round(achieved / hbm_peak, 4),
                     "frac_of_nominal_7900": round(achieved / 7900.0, 4), "traffic": traffic,
                     "traffic_launch": traffic_launch,
                     "bytes_per_launch": pass_bytes, "avg_launch_ms": round(avg_pass_ms, 4)},
        # e2e: the synchronous read-out (the read-out kernel writes the
        # page-locked buffer directly); the asynchronous one (the copy engine
        # moves step i's probabilities while step i + 1 evolves, timed until
        # the last copy has landed) beside it.  The copy engine's rate into
        # host memory differed by almost 2x from one machine to the next.
        "e2e": {"value": round(e2e_value, 3), "unit": "cycles/s",
                "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps,
                "readout": "qs_probabilities",
                "async_readout_value": round(e2e_async_value, 3),
                "async_direct_share": round(async_share, 3)},
        "gpu_launches": sum(kernel_launches_per_step(p) for p in passes_seen),
        "clocks": clk,
        "last_step": {k: round(v, 6) for k, v in results["last"].items()},
        "forms": compare,
        "n34": n34,
        "ensemble": ens,
        "noisy": noisy,
        "single_error": single,
        "grid4x5_n20_d25": small,
        "adjoint": grad,
        "alu_peaks": alu,
    }
    if cpu:
        out["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def forms_34(qs, torch, hbm_peak):
    """Apply-only cycles/s and fraction of measured HBM bandwidth of the plain,
    fused and tensor-core forms on the 34-qubit depth-40 circuit."""
    import numpy as np
    free, _ = torch.cuda.mem_get_info()
    n = 34
    if free < (8 << n) + (8 << 30):
        return {"skipped": "needs %.0f GB free, %.0f GB available" % (((8 << n) + (8 << 30)) / 1e9, free / 1e9)}
    W = WORKLOADS["grid6x6m2_n34_d40"]
    dead = np.zeros(36, dtype=np.uint8)
    dead[0] = dead[35] = 1
    g = qs.qs_circuit_generate(6, 6, W["depth"], 0, dead)
    h = qs.qs_state_create(n, qs.QS_C64)
    out = {"workload": "grid6x6m2_n34_d40", "state_gb": round((8 << n) / 1e9, 1)}
    try:
        for name, md in (("fused", qs.QS_MODE_FUSED), ("tc", qs.QS_MODE_FUSED_TC),
                         ("plain", qs.QS_MODE_PLAIN)):
            qs.qs_state_reset(h)
            qs.qs_prepare_circuit(h, g, mode=md)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            qs.qs_apply_circuit(h, g, mode=md)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            st = applied_plan(qs, n, g, md)
            nrm = qs.qs_pt_moments(h, 0)["norm"]
            out[name] = {"apply_ms": round(ms, 1), "cycles_per_s": round(W["depth"] / (ms / 1e3), 2),
                         "launches": st["launches"], "norm": round(nrm, 7),
                         "norm_drift_within_1e-5": abs(nrm - 1) <= 1e-5,
                         "hbm_frac_of_measured": round(st["bytes"] / (ms / 1e3) / 1e9 / hbm_peak, 4)}
    finally:
        qs.qs_state_destroy(h)
    return out


def ensemble_instance(s):
    """Instance s of the 4096-circuit ensemble: n uniform in 12..24, depth
    uniform in 10..40 (SplitMix64 finaliser of s), 3 or 4 grid rows."""
    M = (1 << 64) - 1

    def mix64(z):
        z &= M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)
    n = 12 + mix64(s) % 13
    depth = 10 + mix64(s ^ 0xD1B54A32D192ED03) % 31
    rows = 3 if n <= 15 else 4
    cols = -(-n // rows)
    dead = [0] * (rows * cols)
    for k in range(rows * cols - n):
        dead[rows * cols - 1 - k] = 1
    return n, depth, rows, cols, dead


def ensemble_4096(qs, torch, hbm_peak, runs=("default", "autotuned", "lockstep_default"), count=4096):
    """Aggregate cycles/s and effective bandwidth of the batched ensemble
    (graph replay of 4096 circuits, statistics included).  Persistent
    engine (one launch per run): with the default 13-qubit tiles and with
    the tile size autotuned per instance size; lockstep engine (one launch
    per round and tile size) with the default tiles, for comparison.
    `count` < 4096 takes the recipe's first instances (a profiling case)."""
    import numpy as np
    inst = [ensemble_instance(s) for s in range(count)]
    gl = [qs.qs_circuit_generate(r, c, d, s, np.array(dd, dtype=np.uint8))
          for s, (n, d, r, c, dd) in enumerate(inst)]
    cycles = sum(x[1] for x in inst)
    bytes_state = sum(8 << x[0] for x in inst)
    out = {"instances": count, "state_gb": round(bytes_state / 1e9, 1)}
    known = {"default": (qs.QS_BATCH_PERSISTENT, 0), "autotuned": (qs.QS_BATCH_PERSISTENT, 1),
             "lockstep_default": (qs.QS_BATCH_ROUNDS, 0)}
    b = qs.qs_batch_create([x[0] for x in inst])
    try:
        for name in runs:
            engine, tune = known[name]
            qs.qs_batch_set_engine(b, engine)
            qs.qs_batch_set_options(b, autotune=tune)
            t0 = time.perf_counter()
            qs.qs_batch_run(b, gl, kmax=10)            # (tune,) plan, capture, first run
            first = time.perf_counter() - t0
            reps = 3
            t0 = time.perf_counter()
            for _ in range(reps):
                st = qs.qs_batch_run(b, gl, kmax=10)
            dt = (time.perf_counter() - t0) / reps
            tiles, run_bytes = qs.qs_batch_plan_info(b)
            gbs = run_bytes / dt / 1e9
            rec = {"engine": "persistent" if engine == qs.QS_BATCH_PERSISTENT else "lockstep",
                   "first_run_s": round(first, 3), "replay_s": round(dt, 4),
                   "cycles_per_s": round(cycles / dt, 1), "algorithmic_gb": round(run_bytes / 1e9, 2),
                   "gbs": round(gbs, 1), "frac": round(gbs / hbm_peak, 4),
                   "mean_norm": round(float(np.mean(st[:, 0])), 7)}
            if tune:
                rec["tile_per_n"] = {int(n): int(t) for n, t in sorted(set(zip([x[0] for x in inst], tiles)))}
            out[name] = rec
    finally:
        qs.qs_batch_destroy(b)
    cand = [k for k in ("default", "autotuned", "lockstep_default") if k in out]
    best = max(cand, key=lambda k: out[k]["cycles_per_s"])
    out.update({"replay_s": out[best]["replay_s"], "cycles_per_s": out[best]["cycles_per_s"],
                "gbs": out[best]["gbs"], "frac": out[best]["frac"], "best": best})
    return out


def noisy_trajectories(qs, torch, T=4096, r=0.005):
    """Digital error model on the batched engine (Fig. pal setting: 5 x 4
    qubits, depth 40, r2 = r_init = r_mes = r, r1 = r/10): T trajectories,
    one sample each, cross entropy difference under the ideal circuit
    against Eq. 6.  Timed: trajectories on the GPU + batched sampling."""
    import numpy as np
    rows, cols, depth = 4, 5, 40
    n = rows * cols
    g = qs.qs_circuit_generate(rows, cols, depth, 0)
    g1 = int(np.sum(g["kind"] != qs.QS_CZ))
    g2 = int(np.sum(g["kind"] == qs.QS_CZ))
    t0 = time.perf_counter()
    lists = [qs.qs_noisy_circuit(g, n, r / 10, r, r, 7000 + t) for t in range(T)]
    gen_s = time.perf_counter() - t0
    b = qs.qs_batch_create([n] * T)
    h = qs.qs_state_create(n, qs.QS_C64)
    try:
        t0 = time.perf_counter()
        qs.qs_batch_run(b, lists, kmax=0)
        x = qs.qs_batch_sample(b, 1, 321, r).reshape(-1)
        run_s = time.perf_counter() - t0
        qs.qs_apply_circuit(h, g)
        ce, dh = qs.qs_cross_entropy(h, x)
    finally:
        qs.qs_batch_destroy(b)
        qs.qs_state_destroy(h)
    alpha = math.exp(-(r / 10) * g1 - r * g2 - 2 * r * n)
    return {"trajectories": T, "qubits": n, "depth": depth, "r": r, "host_generate_s": round(gen_s, 3),
            "gpu_run_s": round(run_s, 3), "trajectories_per_s": round(T / run_s, 1),
            "delta_h": round(dh, 4), "eq6_alpha": round(alpha, 4)}


def grid20_forms(qs, torch):
    """4 x 5 grid, 20 qubits, depth 25, seeds 0..9 (the paper averages 10
    instances): apply-only cycles/s of the fused form for complex64 and
    complex128 (the 8.4 / 16.8 MB states are L2-resident), and the sample
    cross entropy of 1e5 samples (sampler seed 1000 + circuit seed)."""
    n, depth = 20, 25
    out = {}
    for name, dt in (("c64", qs.QS_C64), ("c128", qs.QS_C128)):
        h = qs.qs_state_create(n, dt)
        try:
            ms_tot, dh_tot, bytes_tot = 0.0, 0.0, 0.0
            for seed in range(10):
                g = qs.qs_circuit_generate(4, 5, depth, seed)
                plan = qs.qs_plan_circuit(n, dt, g[leading_h_layer(qs, g, n):])
                esz = 8 if dt == qs.QS_C64 else 16
                bytes_tot += plan["bytes"] - esz * (1 << n)              # the first pass only writes
                qs.qs_state_reset(h)
                qs.qs_prepare_circuit(h, g)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                qs.qs_apply_circuit(h, g)
                b.record()
                torch.cuda.synchronize()
                ms_tot += a.elapsed_time(b)
                x = qs.qs_sample(h, 100000, 1000 + seed)
                dh_tot += qs.qs_cross_entropy(h, x)[1]
            # the state stays in L2 between passes: bytes moved per second of
            # apply, against the HBM copy rate for scale
            out[name] = {"apply_ms_mean": round(ms_tot / 10, 4), "cycles_per_s": round(10 * depth / (ms_tot / 1e3), 1),
                         "delta_h_mean": round(dh_tot / 10, 4),
                         "pass_bytes_gbs": round(bytes_tot / (ms_tot / 1e3) / 1e9, 1)}
        finally:
            qs.qs_state_destroy(h)
    return out


def adjoint_24(qs, torch):
    """Gradient configuration: 4 x 6 grid, 24 qubits, depth 30, every
    single-qubit gate and CZ parameterised (R_X / R_Y / R_Z, CPHASE), loss
    over 1e5 samples of the nominal circuit: time of one adjoint gradient
    (forward evolution + reverse sweep over all gates)."""
    import numpy as np
    g = qs.qs_circuit_generate(4, 6, 30, 0)
    nom = g.copy()
    for x in nom:
        k = int(x["kind"])
        if k == qs.QS_X_HALF:
            x["kind"], x["theta"] = qs.QS_RX, math.pi / 2
        elif k == qs.QS_Y_HALF:
            x["kind"], x["theta"] = qs.QS_RY, math.pi / 2
        elif k == qs.QS_T:
            x["kind"], x["theta"] = qs.QS_RZ, math.pi / 4
        elif k == qs.QS_CZ:
            x["kind"], x["theta"] = qs.QS_CPHASE, math.pi
    nparam = int(np.sum(nom["kind"] != qs.QS_H))
    h = qs.qs_state_create(24, qs.QS_C64)
    try:
        qs.qs_apply_circuit(h, nom)
        x = qs.qs_sample(h, 100000, 8)
        qs.qs_adjoint_gradient(h, nom, x)            # warm-up (plans, workspace)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss, grad = qs.qs_adjoint_gradient(h, nom, x)
        dt = time.perf_counter() - t0
    finally:
        qs.qs_state_destroy(h)
    return {"qubits": 24, "depth": 30, "gates": int(nom.size), "parameters": nparam,
            "samples": 100000, "gradient_ms": round(dt * 1e3, 2), "loss": round(loss, 6)}


def single_error_sweep(qs, torch):
    """Fig. 1error setting (5 x 4 qubits, depth 40): one batch instance per
    error location (every cycle, qubit, X and Z: 1640 circuits), Pearson
    correlation of each with the ideal output and the error-averaged
    distribution.  Timed: GPU run + correlations + mean distribution."""
    import numpy as np
    rows, cols, depth = 4, 5, 40
    n = rows * cols
    g = qs.qs_circuit_generate(rows, cols, depth, 0)
    locs = [(c, q, pauli) for c in range(depth + 1) for q in range(n) for pauli in (1, 3)]
    lists = [qs.qs_single_error_circuit(g, n, c, q, pauli) for c, q, pauli in locs]
    b = qs.qs_batch_create([n] * len(lists))
    h = qs.qs_state_create(n, qs.QS_C64)
    try:
        t0 = time.perf_counter()
        qs.qs_batch_run(b, lists, kmax=0)
        qs.qs_apply_circuit(h, g)
        corr = qs.qs_batch_correlation(b, h)
        avg = qs.qs_batch_mean_probabilities(b, n)
        run_s = time.perf_counter() - t0
        p = torch.empty(1 << n, dtype=torch.float64, device="cuda")
        qs.qs_probabilities(h, p)
        p = p.cpu().numpy()
    finally:
        qs.qs_batch_destroy(b)
        qs.qs_state_destroy(h)
    cyc = np.array([c for c, _, _ in locs])
    zs = np.array([pauli == 3 for _, _, pauli in locs])
    N = float(1 << n)
    def mean_corr(mask):
        return round(float(np.mean(corr[mask])), 4)
    return {"locations": len(locs), "qubits": n, "depth": depth, "gpu_run_s": round(run_s, 3),
            "circuits_per_s": round(len(locs) / run_s, 1),
            "mean_corr_X": {"cycles_0_4": mean_corr(~zs & (cyc <= 4)), "cycles_10_30": mean_corr(~zs & (cyc >= 10) & (cyc <= 30)),
                            "cycles_36_40": mean_corr(~zs & (cyc >= 36))},
            "mean_corr_Z": {"cycles_0_4": mean_corr(zs & (cyc <= 4)), "cycles_10_30": mean_corr(zs & (cyc >= 10) & (cyc <= 30)),
                            "cycles_36_40": mean_corr(zs & (cyc >= 36))},
            "ideal_N_sum_p2": round(float(N * np.sum(p * p)), 4),
            "averaged_N_sum_p2": round(float(N * np.sum(avg * avg)), 4)}


def load_traffic(mode, n):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    import hashlib
    # both forms are compiled from qs_fused.cu; each has its own capture
    src = os.path.join(ROOT, "paper_1608_00263_gb300", "csrc", "qs_fused.cu")
    try:
        digest = hashlib.sha1(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    r = rec.get(mode)
    if not r or r.get("source_sha1") != digest:
        return None
    # scale the captured launch's traffic to this state size
    return round(r["bytes_per_launch"] * (2.0 ** n) / (2.0 ** r["qubits"]), 1), r.get("launch")


ORACLE_SHARES = 64      # one oracle step = 1/64 of the whole step


class OracleStep:
    """The FP64 oracle on a bounded sample of the whole step: step i does
    1/64 of every leg of one full step of the workload --
      * evolution: gates [i G/64, (i+1) G/64) of the circuit (G gates, H
        layer included), applied in order to one 2^n-amplitude state, so 64
        consecutive steps evolve the whole circuit once;
      * read-out: probabilities of the state's slice i (2^n/64 amplitudes),
        norm, entropy, uniform cross entropy and moments 1..10 of a
        Porter-Thomas distributed slice of the same size (the output
        distribution's shape, Sec. pt; seeded), m/64 samples from that slice
        (inverse CDF) and their cross entropy.
    Its unit is 40/64 cycles of the 40-cycle step."""

    def __init__(self, W, dead, n):
        import numpy as np

        import oracle as O
        self.O, self.np = O, np
        self.n, self.W = n, W
        self.gates = O.generate_circuit(W["rows"], W["cols"], W["depth"], 0, dead)
        self.psi = O.zero_state(n)
        self.slice = (1 << n) // ORACLE_SHARES
        rng = np.random.default_rng(12345)
        pt = rng.exponential(size=self.slice)
        self.pt = pt / pt.sum() / ORACLE_SHARES       # a 1/64 share of a normalised distribution
        self.m = W["m"] // ORACLE_SHARES
        self.cycles = W["depth"] / ORACLE_SHARES

    def step(self, i):
        O, G = self.O, self.gates.size
        k = i % ORACLE_SHARES
        t0 = time.perf_counter()
        if k == 0 and i:
            self.psi = O.zero_state(self.n)          # the next circuit starts from |0...0>
        O.apply_circuit(self.psi, self.gates[k * G // ORACLE_SHARES:(k + 1) * G // ORACLE_SHARES])
        O.probabilities(self.psi[k * self.slice:(k + 1) * self.slice])
        p = self.pt
        O.norm(p), O.entropy(p), O.uniform_ce(p), O.moments(p, 10)
        x = O.sample(p, self.m, 1000 + i)
        O.cross_entropy(p, x)
        return time.perf_counter() - t0

    def describe(self):
        return ("FP64 oracle (OpenMP over all host cores), 1/%d of the whole %s step per oracle "
                "step: about %d of the circuit's %d gates on the 2^%d state, then probabilities of a "
                "2^%d slice and norm, entropy, uniform CE, moments 1..10, %d samples and their CE "
                "on a Porter-Thomas slice of that size; value = (%g cycles per oracle step) / time"
                % (ORACLE_SHARES, "x".join(map(str, (self.W["rows"], self.W["cols"]))),
                   self.gates.size // ORACLE_SHARES, self.gates.size, self.n,
                   self.n - int(math.log2(ORACLE_SHARES)), self.m, self.cycles))


def cpu_baseline(W, dead, n, steps=4):
    """Oracle (FP64 CPU) on a bounded sample of the whole step: `steps`
    consecutive 1/64 shares (OracleStep); returns cycles/s."""
    o = OracleStep(W, dead, n)
    dt = sum(o.step(i) for i in range(steps))
    return {"value": round(o.cycles * steps / dt, 5), "unit": "cycles/s", "cores": os.cpu_count(),
            "kind": "oracle", "sample": "%d oracle steps; %s" % (steps, o.describe())}


def workload_config(args, n, world):
    """The `config` object of both arms' lines: the workload timed."""
    W = WORKLOADS[args.workload]
    state = (8 << n) / 1e9
    size = "%.1f GB" % state if state >= 1 else "%.1f MB" % (state * 1e3)
    l2 = ("inputs larger than L2 (state %s)" % size if state > 0.129
          else "state L2-resident (%s), not flushed between steps" % size)
    return {"workload": args.workload, "qubits": n, "depth": W["depth"], "samples": W["m"],
            "state": "complex64 " + size, "form": args.mode, "l2": l2,
            "parallelism": "replicas" if world > 1 else "single GPU"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import numpy as np

    W = WORKLOADS[args.workload]
    dead = None
    if W["dead"]:
        dead = np.zeros(W["rows"] * W["cols"], dtype=np.uint8)
        for r, c in W["dead"]:
            dead[r * W["cols"] + c] = 1
    n = W["rows"] * W["cols"] - len(W["dead"])
    o = OracleStep(W, dead, n)
    for i in range(args.warmup):
        o.step(i)
    dt = sum(o.step(args.warmup + i) for i in range(args.steps))
    value = o.cycles * args.steps / dt
    sample = o.describe()
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "cycles/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(dt * 1000 / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded random circuits of the paper's grid rules)",
           "config": workload_config(args, n, world),
           "cpu_baseline": {"value": round(value, 5), "unit": "cycles/s", "cores": os.cpu_count(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 5), "unit": "cycles/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.ensemble_only:
        import torch

        import paper_1608_00263_gb300 as qs
        from paper_1608_00263_gb300 import build as qs_build
        qs_build.build()
        peaks, _ = load_peaks()
        print(json.dumps({"ensemble": ensemble_4096(qs, torch, float(peaks["hbm_gbs"]),
                                                    args.ensemble_runs.split(","), args.ensemble_count)}),
              flush=True)
    elif args.adjoint_only:
        import torch

        import paper_1608_00263_gb300 as qs
        from paper_1608_00263_gb300 import build as qs_build
        qs_build.build()
        print(json.dumps({"adjoint": adjoint_24(qs, torch)}), flush=True)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
