#!/usr/bin/env python3
"""Benchmark of the VQE hot path on GB300: batched energy + adjoint-gradient evaluations.

Workload (one "step"): 4096 independent hardware-efficient-ansatz instances, n ~ U{4..12}
qubits, L ~ U{2..8} layers of RY/RZ on every qubit plus a CNOT ladder, Pauli sums of
T ~ U{50..500} Z-heavy terms; each step evaluates every instance's energy and full adjoint
gradient in complex128 in one persistent launch replayed from a CUDA graph.  Inputs are
seeded and synthetic.  With torchrun (N > 1) every rank runs its own 4096 instances (weak
scaling, no collective on the data path).

Prints one JSON line (rank 0).  ``--impl reference`` times the plain CPU oracle instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "VQE energy+grad evals/s (batched, 4096 HEA instances n=4..12, complex128)"
UNIT = "evals/s"
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.070e9 / 1e12  # 2 DFMA/clk/SM x 2 flop x 152 SMs x 2.07 GHz


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--instances", type=int, default=4096)
    ap.add_argument("--seed", type=int, default=1002)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="batch",
                    choices=["batch", "serve", "kernels", "single", "h2", "classes", "tfim",
                             "fp64"],
                    help="batch: the batched evaluation step (default); serve: the request "
                         "loop (latency percentiles), printed as its own JSON line")
    ap.add_argument("--requests", type=int, default=300)
    ap.add_argument("--qubits", type=int, default=28)
    ap.add_argument("--ansatz", default="hea", choices=["hea", "uccsd"])
    ap.add_argument("--checkpoint-gb", type=float, default=0.0,
                    help="single: device memory for psi checkpoints of commuting layers "
                         "(sv_set_checkpoint_bytes); the default 0 keeps at most three "
                         "state-sized buffers")
    ap.add_argument("--autotune", action="store_true",
                    help="single: autotune the fused tile size first (sv_set_autotune)")
    ap.add_argument("--per-circuit-sample", type=int, default=512,
                    help="batch: instances timed through the one-circuit-per-launch path")
    ap.add_argument("--no-batch-autotune", dest="batch_autotune", action="store_false",
                    help="batch: use the fixed layout rule instead of letting the layout tuner "
                         "pick each qubit count's team size and segment widths "
                         "(sv_batch_set_autotune) before the timed steps")
    ap.add_argument("--no-extras", action="store_true",
                    help="batch: skip the FP64 probe, the 26-qubit kernel table and the "
                         "serving sample that the default line carries")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_indices(rank, instances):
    """Instances one rank evaluates: rank r takes indices [r*I, (r+1)*I) of the seeded batch,
    so the ranks' sets are disjoint and together cover the first I*world instances."""
    return list(range(rank * instances, (rank + 1) * instances))


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings (the slowest rank sets the job's time)."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_rate(instances, world, steps, seconds):
    """Evaluations per second of the whole job: every rank's instances, every step."""
    return instances * world * steps / seconds


def config(args, world):
    return {"workload": f"hea_batch_{args.instances}_n4-12_L2-8_T50-500",
            "instances_per_gpu": args.instances, "qubits": "4-12", "layers": "2-8",
            "terms": "50-500 (70% I/Z-only, weight<=4)", "seed": args.seed,
            "ansatz": "RY+RZ on all qubits + CNOT ladder per layer",
            "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": f"replicas{world}"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(", ") for r in self.file.read().splitlines() if r.strip()]
        os.unlink(self.file.name)
        if self.uuid:
            mine = [r for r in rows if len(r) > 1 and r[1].strip() == self.uuid]
            rows = mine or rows
        sm = [float(r[2]) for r in rows if len(r) >= 10 and r[2].strip().replace(".", "").isdigit()]
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, name in enumerate(names):
                if len(r) > 6 + k and r[6 + k].strip() == "Active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][3]),
                "samples": len(sm), "reasons": sorted(reasons),
                "power_w_max": max(float(r[4]) for r in rows if r[4].strip()[0].isdigit())}


def cpu_baseline(args, seconds, first_index=0, one_core_seconds=5.0):
    """The oracle (parameter-shift gradient, OpenMP over shifted evaluations) on consecutive
    instances of the same seeded workload: on all host cores until `seconds` elapse, then on
    one core for `one_core_seconds`."""
    import oracle
    from paper_2601_09951_gb300 import workloads as W
    cores = os.cpu_count() or 1

    def timed(threads, budget, start):
        oracle.set_threads(threads)
        done, t0, i = 0, time.perf_counter(), start
        while time.perf_counter() - t0 < budget:
            inst = W.hea_batch(args.instances, seed=args.seed, indices=[i % args.instances])[0]
            oracle.energy_grad(inst)
            done += 1
            i += 1
        return done, time.perf_counter() - t0, i

    done, dt, i = timed(cores, seconds, first_index)
    used = oracle.get_threads()
    done1, dt1, i1 = timed(1, one_core_seconds, first_index)
    oracle.set_threads(cores)
    return {"value": done / dt, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"instances {first_index}..{i - 1} of the same seeded workload "
                      f"({done} energy+gradient evaluations, parameter-shift, {dt:.1f} s)",
            "one_core": {"value": done1 / dt1, "unit": UNIT, "cores": 1,
                         "sample": f"instances {first_index}..{i1 - 1}, {done1} evaluations, "
                                   f"{dt1:.1f} s"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2601_09951_gb300 import workloads as W
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    per_step = 4
    times = []
    for s in range(args.warmup + args.steps):
        idx = [(s * per_step + k) % args.instances for k in range(per_step)]
        insts = W.hea_batch(args.instances, seed=args.seed, indices=idx)
        t0 = time.perf_counter()
        for inst in insts:
            oracle.energy_grad(inst)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = per_step * len(times) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(args, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(),
                             "kind": "oracle",
                             "sample": f"{per_step} instances per step, consecutive seeded "
                                       f"indices, parameter-shift gradient on {cores} cores"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serve_run(svqe, reqs, rate, serial=False, budget=64 << 30):
    """One pass of a request stream through the server: arrivals scaled to `rate` requests/s
    (None: all at once), p50/p99 latency from submit to completion, evals/s over the wall
    time."""
    import threading
    srv = svqe.Server(hbm_budget_bytes=budget, steps_per_tick=2, serial=serial)
    ids = [None] * len(reqs)
    t0 = time.perf_counter()

    def submitter():
        for k, r in enumerate(reqs):
            if rate:
                # arrival_s in the stream is for 1 request/s; scale it to `rate`
                delay = r["arrival_s"] / rate - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
            ids[k] = srv.submit(r, r["steps"], r["lr"])

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    lat, busy = [], {}
    for r, rid in zip(reqs, ids):
        _, _, info = srv.wait(rid, -1)
        lat.append(info.done_s - info.submit_s)
        # running time by size class (in the serial server: each request's own GPU time)
        cls = "n<=12" if info.n_qubits <= 12 else "n13-19" if info.n_qubits < 20 else "n20-24"
        busy[cls] = busy.get(cls, 0.0) + (info.done_s - info.admit_s)
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    evals = sum(r["steps"] for r in reqs)
    tot = sum(busy.values()) or 1.0
    return {"evals_per_s": evals / wall, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)), "wall_s": wall,
            "launches": int(st.launches), "peak_bytes": int(st.peak_bytes_in_use),
            "running_time_share": {k: v / tot for k, v in sorted(busy.items())}}


def run_serve(args):
    """Serving stream: Poisson arrivals of VQE requests (n log-uniform in 4..24, 20 gradient
    steps each).  Saturated throughput first (all requests at once), then arrivals at 25, 50,
    75 and 90 % of it with p50/p99 latency, beside the same stream through the serial
    one-request-at-a-time server at the same rates."""
    import torch
    torch.cuda.set_device(0)
    from paper_2601_09951_gb300 import build as libbuild
    libbuild.build()
    from paper_2601_09951_gb300 import svqe
    from paper_2601_09951_gb300 import workloads as W
    reqs = W.serve_stream(args.requests, 1.0, seed=1005)
    sat = serve_run(svqe, reqs, None)
    req_rate = args.requests / sat["wall_s"]  # requests/s at saturation
    sweep, serial = {}, {}
    for frac in (0.25, 0.5, 0.75, 0.9):
        sweep[f"{int(frac * 100)}%"] = serve_run(svqe, reqs, frac * req_rate)
        serial[f"{int(frac * 100)}%"] = serve_run(svqe, reqs, frac * req_rate, serial=True)
    serial_sat = serve_run(svqe, reqs, None, serial=True)
    line = {"metric": "serving: VQE energy+grad evals/s and p50/p99 request latency",
            "workload": f"serve_stream_{args.requests}_n4-24_20steps", "unit": "evals/s",
            "value": sat["evals_per_s"], "saturated": sat, "poisson": sweep,
            "serial_saturated": serial_sat, "serial_poisson": serial,
            "batched_over_serial_saturated": sat["evals_per_s"] / serial_sat["evals_per_s"],
            "data": "synthetic (seeded Poisson stream)", "dtype": "f64"}
    print(json.dumps(line), flush=True)


def serve_sample(svqe, W, n_requests=60):
    """The serving loop on a short seeded stream, for the default line: saturated throughput,
    then Poisson arrivals at 50 % of it (p50/p99), and the serial server saturated."""
    reqs = W.serve_stream(n_requests, 1.0, seed=1005)
    sat = serve_run(svqe, reqs, None)
    half = serve_run(svqe, reqs, 0.5 * n_requests / sat["wall_s"])
    serial = serve_run(svqe, reqs, None, serial=True)
    return {"workload": f"serve_stream_{n_requests}_n4-24_20steps",
            "saturated_evals_per_s": sat["evals_per_s"],
            "at_50%": {"evals_per_s": half["evals_per_s"], "p50_ms": half["p50_ms"],
                       "p99_ms": half["p99_ms"]},
            "serial_saturated_evals_per_s": serial["evals_per_s"],
            "batched_over_serial": sat["evals_per_s"] / serial["evals_per_s"]}


HBM_PEAK_GBS = 6678.2  # measured copy bandwidth (read + write) of a GB300

# dram__bytes_read.sum + dram__bytes_write.sum of one k_batch launch of the default workload,
# from one ncu capture of that launch, keyed by a hash of the kernel's sources: once the
# kernel changes the key no longer matches and traffic is null.
KBATCH_TRAFFIC = {"fa0046678f00f781": 373.54e6 + 519.86e6,
                  "69036a9ca5c72f5d": 373.48e6 + 519.67e6}
KBATCH_SOURCES = ("k_batch.cu", "svqe_internal.cuh", "svqe_types.h", "launch.h")


def kbatch_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KBATCH_SOURCES:
        with open(os.path.join(ROOT, "paper_2601_09951_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_PEAK_GBS, "measured copy bandwidth of this GPU model, built in"


def expval_flops_per_amp(ham):
    """FP64 flops per amplitude of the energy-only kernel (FMA = 2), summed over X-mask groups:
    the terms at k and k ^ x are conjugate, so each pair is taken once.  A one-term group costs
    1 DFMA per amplitude; a real or imaginary table 1 DMUL + 2 DFMA per pair, a complex one
    twice that; the diagonal group 1 DMUL + 2 DFMA per amplitude."""
    groups = {}  # x -> Y-count parities of its terms (real, imaginary or both)
    for x, z in zip(np.asarray(ham["x"], np.uint64).tolist(),
                    np.asarray(ham["z"], np.uint64).tolist()):
        groups.setdefault(x, []).append(bin(x & z).count("1") & 1)
    total = 0.0
    for x, par in groups.items():
        total += 5 if x == 0 else 2 if len(par) == 1 else 2.5 * len(set(par))
    return total


def kernel_table(svqe, W, torch, n, subset=None):
    """Per-kernel timing on the single-state path at n qubits (state larger than L2): each
    kernel type through the public API, CUDA events on the context's stream, algorithmic bytes
    and FP64 flops per amplitude, as listed beside each kernel below.  `subset`: names to run
    (None: all)."""
    N = 1 << n
    stream = torch.cuda.Stream()
    ctx = svqe.Context(n, stream=stream.cuda_stream)
    peak, src = _peaks()

    def one(gtype, wires, param=True):
        cb = W.CircuitBuilder(n)
        cb.add(gtype, wires, param="new" if param else None)
        return svqe.Circuit(cb.build())

    rows = {}

    def timed(name, fn, bytes_per_amp, flops_per_amp, reps=5):
        if subset is not None and not any(name.startswith(k) for k in subset):
            return
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / reps
        gbs = bytes_per_amp * N / ms / 1e6
        tf = flops_per_amp * N / ms / 1e9
        rows[name] = {"ms": ms, "bytes_per_amp": bytes_per_amp, "GB/s": gbs,
                      "hbm_frac": gbs / peak, "fp64_flops_per_amp": flops_per_amp,
                      "fp64_TFLOP/s": tf, "fp64_frac": tf / FP64_PEAK_TFLOPS}

    th = np.array([0.37])
    low, mid, high = n - 1, n // 2, 0  # qubit n-1 is bit 0
    timed("init_basis (a1)", lambda: ctx.init_reference(0), 16, 0)
    for q, tag in ((low, "bit0"), (mid, "mid"), (high, "top")):
        c = one(W.RY, [q])
        timed(f"RY {tag} (a2)", lambda c=c: ctx.apply_circuit(c, th), 32, 6)
    c = one(W.RZ, [mid])
    timed("RZ mid (a2)", lambda: ctx.apply_circuit(c, th), 32, 6)
    c = one(W.CNOT, [mid, low], param=False)
    timed("CNOT (a3)", lambda: ctx.apply_circuit(c, np.zeros(0)), 16, 0)
    # Wires on bit 0 put one untouched amplitude in every touched 32-byte sector (the DRAM
    # moves twice the algorithmic bytes); wires above bit 1 do not.
    c = one(W.SINGLE_EXC, [mid, low])
    timed("SingleExcitation bit0 (a4)", lambda: ctx.apply_circuit(c, th), 16, 3)
    c2 = one(W.SINGLE_EXC, [mid, high])
    timed("SingleExcitation mid/top (a4)", lambda: ctx.apply_circuit(c2, th), 16, 3)
    c = one(W.DOUBLE_EXC, [high, mid, mid + 1, low])
    timed("DoubleExcitation bit0 (a5)", lambda: ctx.apply_circuit(c, th), 4, 0.75)
    c3 = one(W.DOUBLE_EXC, [high, 1, mid, mid + 1])
    timed("DoubleExcitation mid/top (a5)", lambda: ctx.apply_circuit(c3, th), 4, 0.75)
    layer = W.hea_circuit(n, 1, ring=True)
    lc = svqe.Circuit(layer)
    lth = np.random.default_rng(0).uniform(-3, 3, layer["n_params"])
    # one HEA layer, fused passes: FP64 per amplitude = 6 per RY + 12 for the RZ run
    n_pass, _ = svqe.circuit_plan(lc)
    timed(f"fused HEA layer, {n_pass} passes (a6, forward)",
          lambda: ctx.apply_circuit(lc, lth), 32 * n_pass, 6 * n + 12)
    inst = W.hea_single(n, layers=1, n_terms=100)
    H = svqe.Ham(ctx, inst["ham"])
    G = H.info()[0]
    timed(f"expval {G} groups (a7)", lambda: ctx.expval(H), 16 * G,
          expval_flops_per_amp(inst["ham"]))
    c1 = svqe.Circuit(inst["circuit"])
    th1 = np.asarray(inst["theta"])
    e_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    g_d = torch.zeros(c1.n_params, dtype=torch.float64, device="cuda")
    th_d = torch.tensor(th1, device="cuda")
    timed("adjoint energy+gradient, 1 HEA layer (a8+a9)",
          lambda: ctx.adjoint_grad_dev(c1, th_d.data_ptr(), H, e_d.data_ptr(), g_d.data_ptr()),
          0, 0, reps=3)
    H.close()
    ctx.close()
    return rows, peak, src


def run_kernels(args):
    import torch
    torch.cuda.set_device(0)
    from paper_2601_09951_gb300 import build as libbuild
    libbuild.build()
    from paper_2601_09951_gb300 import svqe
    from paper_2601_09951_gb300 import workloads as W
    n = args.qubits
    rows, peak, src = kernel_table(svqe, W, torch, n)
    print(json.dumps({"metric": "single-state kernel throughput", "n_qubits": n,
                      "state_bytes": 16 * (1 << n), "hbm_peak_GBps": peak,
                      "hbm_peak_source": src, "fp64_peak_TFLOPs": FP64_PEAK_TFLOPS,
                      "kernels": rows}), flush=True)


PROBE_SHAPES = [(bps, thr, ch) for bps in (1, 2, 4, 8) for thr in (128, 256)
                for ch in (4, 8, 16)]


def fp64_rate(svqe, torch, seconds=1.0, shapes=None):
    """Measured FP64 FMA rate of the whole GPU (sv_fp64_probe).  Each shape (blocks per SM,
    threads per block, independent FMA chains per thread) is timed over short launches with
    CUDA events on the probe's stream; the fastest shape is then timed for about `seconds`
    with SM clocks sampled meanwhile.  Returns the rate in FMA/s and FP64 TFLOP/s (FMA = 2
    flops), per SM per clock at the median sampled clock, and every shape's rate."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    stream = torch.cuda.Stream()
    out = torch.empty(8 * sms * 256, dtype=torch.float64, device="cuda")

    def launch(shape, iters):
        bps, thr, ch = shape
        return svqe.fp64_probe(bps * sms, thr, ch, iters, out.data_ptr(), stream.cuda_stream)

    def rate_of(shape, iters, reps):
        ev = []
        n_fma = 0.0
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            n_fma = launch(shape, iters)
            b.record(stream)
            ev.append((a, b))
        torch.cuda.synchronize()
        ms = sorted(a.elapsed_time(b) for a, b in ev)
        return n_fma / (ms[len(ms) // 2] / 1e3), ms[len(ms) // 2]

    with torch.cuda.stream(stream):
        launch((1, 128, 4), 100)
        torch.cuda.synchronize()
        sweep = {}
        for shape in (shapes or PROBE_SHAPES):
            # about 20 ms per launch at 1e12 flop/s
            iters = max(100, int(1e10 / (shape[0] * sms * shape[1] * shape[2])))
            sweep[shape] = rate_of(shape, iters, 3)[0]
        best = max(sweep, key=sweep.get)
        iters = max(100, int(5e10 / (best[0] * sms * best[1] * best[2])))
        with ClockSampler() as clk:
            reps = max(3, int(seconds / 0.1))
            rate, med = rate_of(best, iters, reps)
        ck = clk.summary()
    mhz = ck.get("sm_mhz") or 0.0
    return {"fma_per_s": rate, "tflops": 2 * rate / 1e12,
            "fma_per_clk_per_sm": rate / (mhz * 1e6) / sms if mhz else None,
            "ms_per_launch_median": med, "sms": sms,
            "shape": f"{best[0]} blocks/SM x {best[1]} threads x {best[2]} chains x {iters} FMA",
            "sweep_tflops": {f"{b}x{t}x{c}": 2 * r / 1e12 for (b, t, c), r in sweep.items()},
            "clocks": ck}


def run_fp64(args):
    import torch
    torch.cuda.set_device(0)
    from paper_2601_09951_gb300 import build as libbuild
    libbuild.build()
    from paper_2601_09951_gb300 import svqe
    r = fp64_rate(svqe, torch, seconds=2.0)
    r.update({"metric": "FP64 FMA issue rate (sv_fp64_probe)", "unit": "TFLOP/s",
              "value": r["tflops"], "derived_peak_tflops": FP64_PEAK_TFLOPS,
              "derived_peak_what": "2 FMA/clk/SM x 2 flop x 152 SMs x 2.07 GHz"})
    print(json.dumps(r), flush=True)


def run_single(args):
    """Energy + adjoint gradient evaluations of one state: the UCCSD-shaped 20-qubit circuit
    (400 Givens gates, 2000 terms) or the hardware-efficient sweep at n qubits (10 layers,
    100 random strings), evals/s with CUDA events on the context's stream."""
    import torch
    torch.cuda.set_device(0)
    from paper_2601_09951_gb300 import build as libbuild
    libbuild.build()
    from paper_2601_09951_gb300 import svqe
    from paper_2601_09951_gb300 import workloads as W
    inst = W.uccsd_instance() if args.ansatz == "uccsd" else W.hea_single(args.qubits)
    n = inst["circuit"]["n"]
    stream = torch.cuda.Stream()
    ctx = svqe.Context(n, stream=stream.cuda_stream)
    ctx.set_checkpoint_bytes(int(args.checkpoint_gb * 2**30))
    if args.autotune:
        ctx.set_autotune(True)
    ctx.init_reference(inst["ref"])
    H = svqe.Ham(ctx, inst["ham"])
    C = svqe.Circuit(inst["circuit"])
    th_d = torch.tensor(np.asarray(inst["theta"]), device="cuda")
    e_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    g_d = torch.zeros(max(C.n_params, 1), dtype=torch.float64, device="cuda")
    call = lambda: ctx.adjoint_grad_dev(C, th_d.data_ptr(), H, e_d.data_ptr(), g_d.data_ptr())
    for _ in range(max(1, args.warmup)):
        call()
    torch.cuda.synchronize()
    reps = max(1, args.steps)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(reps):
        call()
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / reps
    print(json.dumps({"metric": "single-state energy+adjoint-gradient evals/s",
                      "workload": inst["name"], "n_qubits": n, "gates": len(C.gates),
                      "terms": len(inst["ham"]["coeff"]), "groups": H.info()[0],
                      "checkpoint_bytes": int(args.checkpoint_gb * 2**30),
                      "tile_bits": ctx.tile_bits(), "autotuned": bool(args.autotune),
                      "ms_per_eval": ms, "value": 1e3 / ms, "unit": "evals/s",
                      "dtype": "f64"}), flush=True)


def per_circuit(insts, sample):
    """The plain one-circuit-per-launch path on the same instances: each instance's energy and
    adjoint gradient through a single-state context (sv_adjoint_grad_dev: fused passes),
    one after another on one stream, for the first `sample` instances.  evals/s from CUDA
    events; launches per evaluation counted from the op lists."""
    import torch
    from paper_2601_09951_gb300 import svqe
    stream = torch.cuda.Stream()
    ctxs, prepared, launches = {}, [], 0
    for inst in insts[:sample]:
        n = inst["circuit"]["n"]
        if n not in ctxs:
            ctxs[n] = svqe.Context(n, stream=stream.cuda_stream)
            ctxs[n].init_reference(inst["ref"])
        C = svqe.Circuit(inst["circuit"])
        H = svqe.Ham(ctxs[n], inst["ham"])
        th = torch.tensor(np.asarray(inst["theta"], dtype=np.float64), device="cuda")
        g = torch.zeros(max(C.n_params, 1), dtype=torch.float64, device="cuda")
        prepared.append((ctxs[n], C, th, H, g))
        # init, coefficients, one forward and one backward kernel per fused pass, H psi + sum,
        # the partials' reset, per-op contributions + per-parameter sums
        launches += 2 * svqe.circuit_plan(inst["circuit"])[0] + 7
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    for ctx, C, th, H, g in prepared:
        ctx.adjoint_grad_dev(C, th.data_ptr(), H, e.data_ptr(), g.data_ptr())
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for ctx, C, th, H, g in prepared:
        ctx.adjoint_grad_dev(C, th.data_ptr(), H, e.data_ptr(), g.data_ptr())
    t1.record(stream)
    torch.cuda.synchronize()
    s = t0.elapsed_time(t1) / 1e3
    return {"value": len(prepared) / s, "unit": "evals/s",
            "sample": f"instances 0..{len(prepared) - 1} of the same workload, one "
                      "sv_adjoint_grad_dev per instance in sequence on one stream",
            "launches_per_eval": launches / len(prepared)}


def run_tfim(args):
    """The paper's CPU vs GPU scaling study shape (Sec. 5.2, Table 3): a transverse-field Ising
    chain at 4..26 qubits under a 2-layer hardware-efficient ansatz.  Per n, one line: the
    single-state energy + adjoint gradient (CUDA events), 100 gradient-descent steps through
    vqe_step (host wall time, energies copied back), and for n <= 14 the oracle's
    parameter-shift evaluation on one host core.  The paper's times (PennyLane, EPYC core vs
    H100, unstated iteration count) are context only."""
    import torch
    torch.cuda.set_device(0)
    from paper_2601_09951_gb300 import build as libbuild
    libbuild.build()
    from paper_2601_09951_gb300 import svqe
    from paper_2601_09951_gb300 import workloads as W
    import oracle
    paper = {4: (8.33, 0.79), 8: (6.54, 1.07), 12: (4.24, 1.20), 14: (9.10, 0.90),
             16: (5.67, 0.85), 18: (12.03, 0.84), 20: (46.77, 1.08), 22: (161.07, 2.21),
             24: (478.73, 5.87), 26: (1425.06, 17.71)}
    oracle.set_threads(1)
    for n in sorted(paper):
        inst = W.tfim_instance(n)
        stream = torch.cuda.Stream()
        ctx = svqe.Context(n, stream=stream.cuda_stream)
        ctx.init_reference(0)
        H = svqe.Ham(ctx, inst["ham"])
        C = svqe.Circuit(inst["circuit"])
        th = torch.tensor(np.asarray(inst["theta"]), device="cuda")
        e = torch.zeros(1, dtype=torch.float64, device="cuda")
        g = torch.zeros(C.n_params, dtype=torch.float64, device="cuda")
        call = lambda: ctx.adjoint_grad_dev(C, th.data_ptr(), H, e.data_ptr(), g.data_ptr())
        call()
        torch.cuda.synchronize()
        reps = 20 if n <= 22 else 5
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            call()
        t1.record(stream)
        torch.cuda.synchronize()
        eval_ms = t0.elapsed_time(t1) / reps
        w0 = time.perf_counter()
        _, es = ctx.vqe_step(C, H, np.asarray(inst["theta"]), 0.05, 100)
        gd_s = time.perf_counter() - w0
        line = {"metric": "TFIM scaling: energy+gradient ms and 100 GD steps",
                "n_qubits": n, "state_bytes": 16 << n, "gates": len(C.gates),
                "eval_ms": eval_ms, "gd100_s": gd_s, "e_first": float(es[0]),
                "e_last": float(es[-1]),
                "paper_context_s": {"cpu": paper[n][0], "gpu_h100": paper[n][1]}}
        if n <= 14:
            w0 = time.perf_counter()
            oracle.energy_grad(inst)
            line["oracle_1core_s_per_eval"] = time.perf_counter() - w0
        print(json.dumps(line), flush=True)
        del ctx, H


def run_classes(args):
    """Batched-kernel throughput by register size: for each n, a batch of instances of that n
    alone (hardware-efficient ansatz, 5 layers, 275 terms), enough to give every CTA several
    items of the n's team class.  One JSON line per n with its share of the FP64 peak."""
    import torch
    torch.cuda.set_device(0)
    from paper_2601_09951_gb300 import build as libbuild
    libbuild.build()
    from paper_2601_09951_gb300 import svqe
    from paper_2601_09951_gb300 import workloads as W
    per_item = {12: 1, 11: 2, 10: 4}
    for n in range(4, 13):
        ninst = 152 * 4 * per_item.get(n, 8)
        insts = [W.hea_instance(n, 5, 275, 77, stream=i + 1) for i in range(ninst)]
        stream = torch.cuda.Stream()
        b = svqe.Batch(insts, stream=stream.cuda_stream)
        th = torch.tensor(b.theta_of(insts), dtype=torch.float64, device="cuda")
        e = torch.empty(ninst, dtype=torch.float64, device="cuda")
        g = torch.empty(b.n_params, dtype=torch.float64, device="cuda")
        flops, _ = b.cost()
        with torch.cuda.stream(stream):
            for _ in range(max(3, args.warmup)):
                b.run_dev(th.data_ptr(), e.data_ptr(), g.data_ptr())
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            reps = max(1, min(args.steps, 20))
            t0.record(stream)
            for _ in range(reps):
                b.run_dev(th.data_ptr(), e.data_ptr(), g.data_ptr())
            t1.record(stream)
            torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / reps
        tf = flops / (ms * 1e-3) / 1e12
        print(json.dumps({"workload": f"hea_n{n}_L5_T275 x {ninst}", "n_qubits": n,
                          "ms_per_step": ms, "evals_per_s": ninst / ms * 1e3,
                          "fp64_tflops": tf, "frac_of_fp64_peak": tf / FP64_PEAK_TFLOPS}),
              flush=True)
        del b


def run_h2(args):
    """The paper's H2 potential-energy-surface procedure (Sec. 2.2, 3.4; Algorithm 1): 100 bond
    lengths, Adam with alpha = 0.01 from theta = 0, 300 iterations (the HPC runs of Sec. 5.2),
    then the stored energy E(theta*) -- the whole surface in one persistent launch plus one
    evaluation launch.  Coefficients are the seeded synthetic ones with the H2 Jordan-Wigner
    structure.  Beside it: the single-core oracle on a sample of bonds."""
    import torch
    torch.cuda.set_device(0)
    from paper_2601_09951_gb300 import build as libbuild
    libbuild.build()
    from paper_2601_09951_gb300 import svqe
    from paper_2601_09951_gb300 import workloads as W
    import oracle
    insts = W.h2_sweep(100)
    stream = torch.cuda.Stream()
    b = svqe.Batch(insts, stream=stream.cuda_stream)
    T = 300
    th = torch.zeros(100, dtype=torch.float64, device="cuda")
    e = torch.empty(100, dtype=torch.float64, device="cuda")
    g = torch.empty(100, dtype=torch.float64, device="cuda")
    times = []
    with torch.cuda.stream(stream):
        for rep in range(max(3, args.warmup) + max(1, args.steps)):
            th.zero_()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            b.adam_dev(th.data_ptr(), 0.01, T, None, reset=True)
            b.run_dev(th.data_ptr(), e.data_ptr(), g.data_ptr())
            t1.record(stream)
            torch.cuda.synchronize()
            if rep >= max(3, args.warmup):
                times.append(t0.elapsed_time(t1) / 1e3)
    gpu_s = float(np.median(times))
    # configuration 1 of the batched workloads: 100 bond lengths x 50 gradient-descent steps
    # at eta = 0.4 from theta = 0 (5000 evaluations): one persistent launch, against the
    # one-circuit path (vqe_step per bond length on one context)
    gd = []
    with torch.cuda.stream(stream):
        for rep in range(max(3, args.warmup) + max(1, args.steps)):
            th.zero_()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            b.vqe_dev(th.data_ptr(), 0.4, 50, None)
            t1.record(stream)
            torch.cuda.synchronize()
            if rep >= max(3, args.warmup):
                gd.append(t0.elapsed_time(t1) / 1e3)
    gd_s = float(np.median(gd))
    ctx = svqe.Context(4, stream=stream.cuda_stream)
    prepared = [(svqe.Circuit(i["circuit"]), svqe.Ham(ctx, i["ham"]), i["ref"]) for i in insts]
    for C, H, ref in prepared[:5]:
        ctx.init_reference(ref)
        ctx.vqe_step(C, H, np.zeros(C.n_params), 0.4, 50)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for C, H, ref in prepared:
        ctx.init_reference(ref)
        ctx.vqe_step(C, H, np.zeros(C.n_params), 0.4, 50)
    torch.cuda.synchronize()
    serial_gd_s = time.perf_counter() - t0
    oracle.set_threads(1)
    t0 = time.perf_counter()
    sample = [0, 50, 99]
    for i in sample:
        oracle.adam_trajectory(insts[i], 0.01, T)
    cpu_per_bond = (time.perf_counter() - t0) / len(sample)
    print(json.dumps({
        "metric": "H2 potential energy surface, 100 bond lengths x 300 Adam iterations",
        "unit": "s", "value": gpu_s, "higher_is_better": False,
        "evals_per_s": 100 * (T + 1) / gpu_s, "dtype": "f64",
        "oracle_1core_s_extrapolated": cpu_per_bond * 100,
        "oracle_sample": f"bonds {sample}, 300 Adam steps each, 1 thread",
        "paper_context_s": {"serial PennyLane Adam, 1 CPU core": 593.95,
                            "lightning.gpu, 1 H100": 164.91, "MPI-32 Optax+JIT": 5.04},
        "gd50": {"what": "100 bond lengths x 50 gradient-descent steps, eta = 0.4, theta0 = 0",
                 "batched_s": gd_s, "batched_evals_per_s": 5000 / gd_s,
                 "per_circuit_s": serial_gd_s, "per_circuit_evals_per_s": 5000 / serial_gd_s,
                 "per_circuit_path": "vqe_step per bond length on one 4-qubit context "
                                     "(host wall time, energies copied back per call)"},
        "data": "synthetic coefficients with the H2 Jordan-Wigner structure"}), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload != "batch":
        if rank == 0:
            {"serve": run_serve, "kernels": run_kernels, "single": run_single,
             "h2": run_h2, "classes": run_classes, "tfim": run_tfim,
             "fp64": run_fp64}[args.workload](args)
        return
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2601_09951_gb300 import build as libbuild
    libbuild.build()
    from paper_2601_09951_gb300 import svqe
    from paper_2601_09951_gb300 import workloads as W

    idx = replica_indices(rank, args.instances)
    insts = W.hea_batch(args.instances * world, seed=args.seed, indices=idx)
    stream = torch.cuda.Stream()
    tune_s = None
    if args.batch_autotune:
        svqe.batch_set_autotune(True)
        t0 = time.perf_counter()
    batch = svqe.Batch(insts, stream=stream.cuda_stream)
    if args.batch_autotune:
        tune_s = time.perf_counter() - t0
        svqe.batch_set_autotune(False)
    layout = {n: batch.layout(n) for n in range(4, 13) if batch.layout(n)[0]}
    theta_h = batch.theta_of(insts)
    P = batch.n_params
    theta = torch.tensor(theta_h, dtype=torch.float64, device="cuda")
    energy = torch.empty(len(insts), dtype=torch.float64, device="cuda")
    grad = torch.empty(P, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        if dist is not None:
            dist.barrier()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            batch.run_dev(theta.data_ptr(), energy.data_ptr(), grad.data_ptr())
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        uuid = None
        try:
            uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
        except Exception:
            pass
        with ClockSampler(uuid) as clk:
            barrier()
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            for s in range(args.steps):
                flush.zero_()
                starts[s].record(stream)
                batch.run_dev(theta.data_ptr(), energy.data_ptr(), grad.data_ptr())
                ends[s].record(stream)
            torch.cuda.synchronize()
            barrier()
            wall = time.perf_counter() - w0
        step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
        dev_s = sum(step_ms) / 1e3
        clocks = clk.summary()

        # End to end through the public API with pinned host buffers: H2D theta, the launch,
        # D2H energies and gradients, every step.
        th_h = torch.tensor(theta_h, dtype=torch.float64).pin_memory()
        e_h = torch.empty(len(insts), dtype=torch.float64).pin_memory()
        g_h = torch.empty(max(P, 1), dtype=torch.float64).pin_memory()
        for _ in range(2):
            batch.run_ptr(th_h.data_ptr(), e_h.data_ptr(), g_h.data_ptr())
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(args.steps):
            batch.run_ptr(th_h.data_ptr(), e_h.data_ptr(), g_h.data_ptr())
        torch.cuda.synchronize()
        barrier()
        e2e_s = time.perf_counter() - t0

    dev_s, e2e_s, wall = max_over_ranks([dev_s, e2e_s, wall], dist, "cuda")
    value = whole_job_rate(args.instances, world, args.steps, dev_s)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    flops, hbm_bytes = batch.cost()
    kernel_s = dev_s / args.steps
    achieved = flops / kernel_s / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dev_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded generator, shapes of the batched workload)",
        "config": config(args, world),
        "e2e": {"value": whole_job_rate(args.instances, world, args.steps, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": int(8 * P), "d2h_bytes_per_step": int(8 * (P + len(insts)))},
        "gpu_launches": args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                     "traffic": KBATCH_TRAFFIC.get(kbatch_hash()) if args.instances == 4096
                     and world >= 1 else None,
                     "kernel_source_hash": kbatch_hash(),
                     "kernel": "k_batch", "what": "FP64 pipe (2 DFMA/clk/SM x 152 SMs x "
                     "2.07 GHz); algorithmic FP64 flops per launch / mean launch time",
                     "flops_per_launch": flops, "hbm_bytes_per_launch": hbm_bytes},
        "clocks": clocks,
        "wall_s_incl_l2_flush": wall,
        "layout": {"tuned": bool(args.batch_autotune), "tuning_s": tune_s,
                   "per_qubits": {str(n): {"team_warps": w, "min_layer": ml,
                                           "min_diag_rz": md}
                                  for n, (w, ml, md) in layout.items()}},
    }
    if world == 1 and args.per_circuit_sample > 0:
        pc = per_circuit(insts, args.per_circuit_sample)
        pc["batched_over_per_circuit"] = value / pc["value"]
        line["per_circuit"] = pc
    if world == 1 and not args.no_extras:
        # the measured FP64 rate beside the derived peak
        probe = fp64_rate(svqe, torch, seconds=1.0)
        line["roofline"]["peak_probe"] = probe["tflops"]
        line["roofline"]["frac_of_probe"] = achieved / probe["tflops"]
        line["fp64_probe"] = {k: probe[k] for k in ("tflops", "fma_per_clk_per_sm", "shape",
                                                    "ms_per_launch_median")}
        line["fp64_probe"]["sm_mhz"] = probe["clocks"].get("sm_mhz")
        # the other two parts of the metric: HBM GB/s per kernel and serving latency
        batch.close()
        torch.cuda.empty_cache()
        rows, peak, src = kernel_table(svqe, W, torch, 26,
                                       subset=("RY mid", "CNOT", "expval"))
        line["kernels_26q"] = {k: {"ms": v["ms"], "GB/s": v["GB/s"], "hbm_frac": v["hbm_frac"]}
                               for k, v in rows.items()}
        line["kernels_26q"]["hbm_peak_GBps"] = peak
        torch.cuda.empty_cache()
        line["serve"] = serve_sample(svqe, W)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
