#!/usr/bin/env python3
"""Open-GRAPE gradient-evaluation benchmark on GB300.

One step = one full gradient evaluation of the d=120 transmon-resonator
reset problem (3-level transmon x N=40 resonator, N_t = 2000 slices, n_RK = 4
RK4 substeps, 3 initial states, 3 controls, 3 jump operators): forward RK4
propagation, cost, adjoint propagation and per-slice gradient traces, all in
libgrape.so kernels.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0).  Under torchrun every rank runs its own copy of
the problem (replicas, weak scaling) and the time is the max over ranks.

Other workloads (measurement cases of the batched, long-pulse and serving
forms; not the headline line):
  --workload batch256  the 256-problem batch in one graph-captured launch,
                       against one-at-a-time gradients of a sample
  --workload d600      one checkpointed gradient of the d=600 problem
                       (N_t = 40000, a checkpoint every 200 slices)
  --workload serve     a Poisson trace of pulse optimisations (50 projected
                       L-BFGS iterations each) through the serving loop, with
                       continuous batching and one job at a time
  --workload peaks     the measured FMA throughput of the FP32 and FP64 pipes
                       (the ALU roofs of the double-float and native kernels)
  --scale s            multiplies every problem's number of slices
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GRAPE grad evals/s (fwd+adjoint), % HBM roofline; served p50/p99 latency"
UNIT = "grad_evals/s"
FP64_NOMINAL_TFLOPS = 1.25       # GB300 FP64, nominal (context only)
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # FP32 FMA lanes x max clock (context only)
DF_FP32_OPS_PER_FLOP = 6.0       # pair-arithmetic cost of one FP64-equivalent flop
CPU_SAMPLE_SLICES = 200          # oracle sample: 200 of the 2000 slices
FP64_SAMPLE_SLICES = 200         # native-FP64 arm: the first 200 of the 2000 slices


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="df64", choices=["df64", "fp64"],
                    help="kernel arithmetic: double-float on FP32 pipes or native FP64")
    ap.add_argument("--workload", default="d120",
                    choices=["d120", "d20", "d120f", "d120p", "sweep", "batch256", "d600", "serve", "peaks"])
    ap.add_argument("--scale", type=float, default=None,
                    help="slice-count multiplier of the batch256/serve/d600 workloads")
    ap.add_argument("--jobs", type=int, default=32, help="serve: jobs in the trace")
    ap.add_argument("--sample", type=int, default=256,
                    help="batch256: problems timed one at a time (256 = all, no scaling)")
    ap.add_argument("--lanes", type=int, default=0, help="batch256: concurrent lanes (0 = automatic)")
    return ap.parse_args()


def dist_init(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world <= 1:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    dist.init_process_group(backend=backend)
    return rank, world, dist


def max_over_ranks(dist, values):
    """Element-wise maximum over all ranks: the job takes as long as its
    slowest rank."""
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(values, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def workload():
    import workloads
    return workloads.transmon_resonator_d120()


def algorithmic_counts(w, nb, nt, ndo):
    """Algorithmic FP64 flops and HBM bytes of one gradient evaluation.

    Lindblad action per entry and RK stage: 16 flops per Hamiltonian band
    (two complex multiply-adds), 4 per jump term (real coefficient times a
    complex entry, added) and 8 for the stage combinations.  Trace per
    stage pair: one complex multiply-add per entry and distinct control-band
    offset.  Bytes: every stage input is written once by the forward and the
    adjoint sweep and read once by the trace kernel, as a packed upper
    triangle (16 B per upper entry: the stage values are Hermitian)."""
    d2 = w.d * w.d
    entries = 4 * w.n_slices * w.n_rk * w.n_states * d2
    upper = 4 * w.n_slices * w.n_rk * w.n_states * (w.d * (w.d + 1) // 2)
    f_prop = (16 * nb + 4 * nt + 8) * entries
    f_trace = 8 * ndo * entries
    bytes_prop = 16 * upper
    return {"flops_forward": f_prop, "flops_adjoint": f_prop, "flops_trace": f_trace,
            "bytes_forward": bytes_prop, "bytes_adjoint": bytes_prop,
            "bytes_trace": 2 * bytes_prop, "entries": entries}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_sha(csrc=None):
    """sha256 over the kernel sources with comments, trailing blanks and
    empty lines removed (the profile summaries record it): any change of the
    code invalidates a recorded traffic figure, an edit of a comment does not."""
    csrc = csrc or os.path.join(ROOT, "paper_1609_03170_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("grape_kernels.cuh", "grape_num.cuh", "grape_internal.h"):
        text = open(os.path.join(csrc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        lines = (re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines())
        h.update("\n".join(ln for ln in lines if ln).encode())
        h.update(b"\0")
    return h.hexdigest()


def profiled_traffic(kernel_src_sha):
    """DRAM bytes per launch of the forward propagation kernel from the
    committed ncu summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "prop_h_kernel_transmon_resonator_d120.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_sha = re.search(r"kernel source sha256:\s*([0-9a-f]{12,64})", text)
    m_tr = re.search(r"traffic_bytes_per_full_launch:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_tr or not kernel_src_sha.startswith(m_sha.group(1)):
        return None
    return float(m_tr.group(1))


def cpu_baseline(threads=None):
    """The plain-C FP64 oracle on a bounded sample of the workload."""
    import workloads
    from oracle import sparse
    w = workloads.transmon_resonator_d120(n_slices=CPU_SAMPLE_SLICES)
    nthreads = threads or w.n_states
    _, _, _, secs = sparse.run_workload(w, mode=sparse.MODE_EXACT, threads=nthreads)
    frac = CPU_SAMPLE_SLICES / 2000.0
    return {"value": frac / secs, "unit": UNIT, "cores": min(nthreads, w.n_states),
            "kind": "oracle",
            "sample": f"d=120 problem with {CPU_SAMPLE_SLICES} of 2000 slices (same d, states, "
                      f"controls, RK substeps), {secs:.2f} s, scaled by {frac:g} grad evals; "
                      f"OpenMP over the {w.n_states} initial states"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import workloads
    from oracle import sparse
    sparse.build()
    w = workloads.transmon_resonator_d120(n_slices=40)
    frac = 40 / 2000.0
    for _ in range(args.warmup):
        sparse.run_workload(w, threads=w.n_states)
    times = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        times.append(sparse.run_workload(w, threads=w.n_states)[3])
    total = time.perf_counter() - t_all
    value = frac * args.steps / total
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "transmon_resonator_d120", "d": 120, "n_slices": 2000,
                   "n_rk": 4, "n_states": 3, "n_controls": 3, "n_jumps": 3,
                   "grad_mode": "exact"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": w.n_states, "kind": "oracle",
                         "sample": "each step: the d=120 problem with 40 of 2000 slices, "
                                   "scaled by 0.02 grad evals"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def _dtype(args):
    return "df64" if args.precision == "df64" else "f64"


def _base_line(args, workload, value, unit, ms, extra):
    line = {"metric": METRIC, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": _dtype(args), "data": "synthetic",
            "config": {"workload": workload}}
    line.update(extra)
    return line


def _prec(args):
    from paper_1609_03170_gb300 import _lib
    return _lib.GRAPE_PREC_FP64 if args.precision == "fp64" else _lib.GRAPE_PREC_DF64


def fma_peaks(dev):
    """FMA throughput of the FP32 and FP64 pipes (grape_fma_peak), with the
    SM clock sampled while the probes run."""
    from paper_1609_03170_gb300 import _lib
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    fp32, fp32_ms = _lib.grape_fma_peak(_lib.GRAPE_PREC_DF64)
    fp64, fp64_ms = _lib.grape_fma_peak(_lib.GRAPE_PREC_FP64)
    time.sleep(0.3)
    clk = clocks.stop()
    return {"fp32_tflops": fp32, "fp64_tflops": fp64, "fp32_run_ms": fp32_ms,
            "fp64_run_ms": fp64_ms, "clocks": clk,
            "how": "grape_fma_peak: independent FMA chains (8 per thread) on every SM, "
                   "best of 3 timed runs after a warm-up, CUDA events, 2 flops per FMA",
            "nominal": {"fp32_tflops": FP32_NOMINAL_TFLOPS, "fp64_tflops": FP64_NOMINAL_TFLOPS}}


def run_peaks(args):
    p = fma_peaks(0)
    if p["clocks"]:
        ghz = p["clocks"]["sm_mhz"] / 1000.0
        p["fp32_tflops_per_ghz"] = p["fp32_tflops"] / ghz
        p["fp64_tflops_per_ghz"] = p["fp64_tflops"] / ghz
    p["double_float_roof_tflops"] = p["fp32_tflops"] / DF_FP32_OPS_PER_FLOP
    print(json.dumps({"workload": "peaks", **p}), flush=True)


def run_batch256(args):
    import torch
    import workloads
    from paper_1609_03170_gb300 import GrapeBatch, GrapeProblem, _lib
    scale = 1.0 if args.scale is None else args.scale
    ws = []
    for i in range(256):
        nt = workloads.batch_problem(i).n_slices
        ws.append(workloads.batch_problem(i, n_slices=max(4, int(round(nt * scale)))))
    probs = [GrapeProblem.from_workload(w, precision=_prec(args)) for w in ws]
    us = [torch.from_numpy(w.u).cuda() for w in ws]
    stream = torch.cuda.Stream()
    # one problem at a time on one stream, on a sample (every 256/sample-th
    # problem), before the batch takes its lane storage; each sampled problem
    # gets its own short-lived handle so that its gradient storage is freed
    # before the next one
    idx = list(range(0, 256, max(1, 256 // args.sample)))[:args.sample]
    Fd = torch.empty(1, dtype=torch.float64, device="cuda")
    Gs = [torch.empty((w.n_slices, w.n_controls), dtype=torch.float64, device="cuda") for w in ws]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    seq_sample_ms = 0.0
    for i in idx:
        Pi = GrapeProblem.from_workload(ws[i], precision=_prec(args))
        _lib.grape_gradient(Pi.handle, us[i].data_ptr(), Fd.data_ptr(), Gs[i].data_ptr(),
                            stream.cuda_stream)
        torch.cuda.synchronize()
        ev0.record(stream)
        _lib.grape_gradient(Pi.handle, us[i].data_ptr(), Fd.data_ptr(), Gs[i].data_ptr(),
                            stream.cuda_stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        seq_sample_ms += ev0.elapsed_time(ev1)
        Pi.close()
    own = [p.geometry()[:2] for p in probs]
    t0 = time.perf_counter()
    B = GrapeBatch(probs, n_lanes=args.lanes)    # tunes the tile per d bucket
    tune_s = time.perf_counter() - t0
    tiles = {}
    for w, p, o in zip(ws, probs, own):
        b = f"d{32 * ((w.d - 1) // 32) + 1}-{32 * ((w.d - 1) // 32 + 1)}"
        tiles.setdefault(b, set()).add(p.geometry()[:2])
    tiles = {b: sorted(f"{c}x{t}" for c, t in v) for b, v in sorted(tiles.items())}
    F = torch.empty(256, dtype=torch.float64, device="cuda")
    Gs = [torch.empty((w.n_slices, w.n_controls), dtype=torch.float64, device="cuda") for w in ws]
    for _ in range(max(1, args.warmup)):
        B.gradient(us, F=F, grads=Gs, stream=stream)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        B.gradient(us, F=F, grads=Gs, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    work_all = sum(w.n_slices * w.n_states * w.d ** 2 for w in ws)
    work_sample = sum(ws[i].n_slices * ws[i].n_states * ws[i].d ** 2 for i in idx)
    seq_ms = seq_sample_ms * work_all / work_sample      # = seq_sample_ms when all are timed
    lanes, scratch, launches = B.info()
    print(json.dumps(_base_line(args, "batch256", 256 * 1000.0 / ms, UNIT, ms, {
        "config": {"workload": "batch256", "problems": 256, "slice_scale": scale,
                   "d_range": [min(w.d for w in ws), max(w.d for w in ws)],
                   "slices_range": [min(w.n_slices for w in ws), max(w.n_slices for w in ws)],
                   "lanes": lanes, "scratch_bytes": scratch,
                   "tiles_cluster_x_threads": tiles, "batch_create_s": tune_s},
        "one_at_a_time": {"problems_timed": len(idx), "timed_ms": seq_sample_ms,
                          "ms_all": seq_ms,
                          "value": 256 * 1000.0 / seq_ms, "unit": UNIT,
                          "how": ("every problem timed alone (CUDA events around its second gradient)"
                                  if len(idx) == 256 else
                                  "sample time scaled by (slices x states x d^2) of all / sample")},
        "speedup_vs_one_at_a_time": seq_ms / ms,
        "gpu_launches": launches * args.steps})), flush=True)


def run_d600(args):
    import torch
    import workloads
    from paper_1609_03170_gb300 import GrapeProblem
    scale = 1.0 if args.scale is None else args.scale
    n = max(2, int(round(40000 * scale)))
    w = workloads.transmon_resonator_d600(n_slices=n)
    P = GrapeProblem.from_workload(w, ckpt_stride=200, precision=_prec(args))
    u = torch.from_numpy(w.u).cuda()
    P.set_profiling(True)
    for _ in range(args.warmup):
        P.gradient(u)
    torch.cuda.synchronize()
    P.phase_times()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        F, G = P.gradient(u)
    torch.cuda.synchronize()
    s = (time.perf_counter() - t0) / args.steps
    ph = P.phase_times()
    P.status()
    print(json.dumps(_base_line(args, "transmon_resonator_d600", 1.0 / s, UNIT, 1000 * s, {
        "config": {"workload": "transmon_resonator_d600", "d": 600, "n_slices": n, "n_rk": 4,
                   "n_states": 1, "ckpt_stride": 200, "kernel": P.kernel(),
                   "device_bytes": P.memory_bytes()},
        "phases_ms_per_step": {k: v[0] / args.steps for k, v in ph.items()},
        "gpu_launches": P.gradient_launches() * args.steps})), flush=True)


def run_d20(args):
    """The small qubit-resonator problem (d=20, N_t=200): gradient evaluations
    per second on the device and of the plain-C oracle on the host."""
    import torch
    import workloads
    from oracle import sparse
    from paper_1609_03170_gb300 import GrapeProblem, _lib
    w = workloads.qubit_resonator_d20()
    P = GrapeProblem.from_workload(w, precision=_prec(args))
    stream = torch.cuda.Stream()
    u = torch.from_numpy(w.u).cuda()
    F = torch.empty(1, dtype=torch.float64, device="cuda")
    G = torch.empty((w.n_slices, w.n_controls), dtype=torch.float64, device="cuda")

    def step():
        _lib.grape_gradient(P.handle, u.data_ptr(), F.data_ptr(), G.data_ptr(), stream.cuda_stream)

    for _ in range(max(3, args.warmup)):
        step()
    stream.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    sparse.build()
    sparse.run_workload(w, threads=w.n_states)
    t0 = time.perf_counter()
    reps = 5
    for _ in range(reps):
        sparse.run_workload(w, threads=w.n_states)
    cpu = reps / (time.perf_counter() - t0)
    print(json.dumps(_base_line(args, "qubit_resonator_d20", 1000.0 / ms, UNIT, ms, {
        "config": {"workload": "qubit_resonator_d20", "d": 20, "n_slices": 200, "n_rk": 4,
                   "n_states": 2, "cluster": P.geometry()[0], "l2": "inputs fit in L2 (small case)"},
        "cpu_baseline": {"value": cpu, "unit": UNIT, "cores": w.n_states, "kind": "oracle",
                         "sample": "the whole d=20 problem, 5 gradient evaluations"},
        "gpu_launches": P.gradient_launches() * args.steps})), flush=True)


def run_d120f(args):
    """The d=120 problem with Gaussian-filtered controls (App. A): 200
    controls of Delta t = 10 delta t on the 2000 subpixels of the headline
    problem, bandwidth wB = 2 pi x 100 MHz with kappa = 2 pi x 1.1 MHz
    (the paper's reset parameters), i.e. w0 = (100 / 1.1) / 0.5887 kappa."""
    import torch
    import workloads
    from paper_1609_03170_gb300 import GaussianFilter, GrapeProblem
    w = workloads.transmon_resonator_d120()
    n_steps = w.n_slices // 10
    w0 = GaussianFilter.omega0_from_bandwidth(100.0 / 1.1)
    rng = np.random.default_rng(1609)
    u = torch.from_numpy(rng.uniform(-1, 1, size=(n_steps, w.n_controls))).cuda()
    P = GrapeProblem.from_workload(w, precision=_prec(args))
    stream = torch.cuda.Stream()
    for _ in range(max(3, args.warmup)):
        P.gradient_filtered(u, [w0] * w.n_controls, stream=stream)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        P.gradient_filtered(u, [w0] * w.n_controls, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    # the two filter launches alone, on the same stream
    f = GaussianFilter(n_steps, w.n_slices, w.T, w0, w.n_controls)
    gs = torch.ones((w.n_slices, w.n_controls), dtype=torch.float64, device="cuda")
    reps = 50
    ev0.record(stream)
    for _ in range(reps):
        f.apply(u, stream=stream)
        f.adjoint(gs, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    fms = ev0.elapsed_time(ev1) / reps
    print(json.dumps(_base_line(args, "transmon_resonator_d120_filtered", 1000.0 / ms, UNIT, ms, {
        "config": {"workload": "transmon_resonator_d120_filtered", "d": 120, "n_controls_steps": n_steps,
                   "n_subpixels": w.n_slices, "omega0_kappa": w0, "n_rk": 4, "n_states": 3},
        "filter_ms_per_step": fms, "filter_share": fms / ms,
        "gpu_launches": (P.gradient_launches() + 2) * args.steps})), flush=True)


def run_d120p(args):
    """The d=120 problem with the paper's photon-number penalty,
    Phi = Phi_0 - beta Phi_p with beta = 0.2 / T (Sec. 5, App. B)."""
    import torch
    import workloads
    from paper_1609_03170_gb300 import GrapeProblem
    w = workloads.transmon_resonator_d120()
    P = GrapeProblem.from_workload(w, precision=_prec(args))
    P.set_photon_penalty(w.phys.Q, w.phys.N, 0.2 / w.T)
    u = torch.from_numpy(w.u).cuda()
    stream = torch.cuda.Stream()
    for _ in range(max(3, args.warmup)):
        P.gradient(u, stream=stream)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        P.gradient(u, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    print(json.dumps(_base_line(args, "transmon_resonator_d120_penalty", 1000.0 / ms, UNIT, ms, {
        "config": {"workload": "transmon_resonator_d120_penalty", "d": 120, "n_slices": w.n_slices,
                   "n_rk": 4, "n_states": 3, "beta": 0.2 / w.T},
        "gpu_launches": P.gradient_launches() * args.steps})), flush=True)


def _fit_exponent(ds, ts):
    """Least-squares slope of log T against log d."""
    x, y = np.log(np.asarray(ds, float)), np.log(np.asarray(ts, float))
    return float(np.polyfit(x, y, 1)[0])


def _expm_first_order_seconds(w):
    """The paper's "standard" method on the host: the d^2 x d^2 Liouvillian
    of every slice exponentiated (scipy expm), rho propagated as a vector,
    lambda propagated back with the transposed propagators, and the
    first-order gradient of Eq. (dphidu).  Oracle code, timed only."""
    import scipy.linalg
    from oracle import liouville, operators
    t0 = time.perf_counter()
    m = operators.build(w.phys)
    dt = w.T / w.n_slices
    props = [scipy.linalg.expm(dt * liouville.superop(operators.hamiltonian(m, w.u[j]), m.jumps))
             for j in range(w.n_slices)]
    ders = [liouville.control_superop(Hk) for Hk in m.Hc]
    r = [liouville.vec(w.rho0[0])]
    for Mj in props:
        r.append(Mj @ r[-1])
    lam = liouville.vec(w.sigma.T)
    G = np.zeros(w.u.shape)
    for j in reversed(range(w.n_slices)):
        for k, Dk in enumerate(ders):
            G[j, k] = float(np.real(lam @ (Dk @ r[j + 1]))) * dt
        lam = lam @ props[j]
    return time.perf_counter() - t0


def run_sweep(args):
    """Fig. 2 of the paper on GB300: time per evaluation of Phi and its
    first-order gradient against d for the Jaynes-Cummings reset problem
    (200 slices, one state), with the plain-C RK oracle and the expm
    "standard" method on the host, and the power-law exponents."""
    import torch
    import workloads
    from oracle import sparse
    from paper_1609_03170_gb300 import GrapeProblem, _lib
    gpu_d = [6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512]
    cpu_d = [6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256]
    expm_d = [6, 8, 10, 12, 16, 20]
    stream = torch.cuda.Stream()
    gpu = {}
    for d in gpu_d:
        w = workloads.jaynes_cummings(d)
        P = GrapeProblem.from_workload(w, grad_mode=_lib.GRAPE_GRAD_FIRST_ORDER)
        u = torch.from_numpy(w.u).cuda()
        F = torch.empty(1, dtype=torch.float64, device="cuda")
        G = torch.empty_like(u)
        for _ in range(3):
            _lib.grape_gradient(P.handle, u.data_ptr(), F.data_ptr(), G.data_ptr(), stream.cuda_stream)
        reps = 10
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(reps):
            _lib.grape_gradient(P.handle, u.data_ptr(), F.data_ptr(), G.data_ptr(), stream.cuda_stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        gpu[d] = {"ms": ev0.elapsed_time(ev1) / reps, "kernel": P.kernel(), "cluster": P.geometry()[0]}
        P.close()
    sparse.build()
    cpu = {}
    for d in cpu_d:
        w = workloads.jaynes_cummings(d)
        sparse.run_workload(w, mode=sparse.MODE_FIRST_ORDER, threads=1)
        cpu[d] = 1000.0 * sparse.run_workload(w, mode=sparse.MODE_FIRST_ORDER, threads=1)[3]
    expm = {d: 1000.0 * _expm_first_order_seconds(workloads.jaynes_cummings(d)) for d in expm_d}
    big = [d for d in gpu_d if d >= 128]
    line = _base_line(args, "jaynes_cummings_sweep", _fit_exponent(big, [gpu[d]["ms"] for d in big]),
                      "exponent", gpu[gpu_d[-1]]["ms"], {
        "metric": "T_grad scaling exponent xi (T_grad ~ d^xi), Fig. 2 workload",
        "higher_is_better": False,
        "config": {"workload": "jaynes_cummings_sweep", "n_slices": 200, "n_rk": 1, "n_states": 1,
                   "grad_mode": "first_order", "g_kappa": 100.0, "delta_kappa": 10.0,
                   "T": "pi/g", "alpha": "sqrt(d/8)"},
        "gpu_ms": {str(d): round(v["ms"], 4) for d, v in gpu.items()},
        "gpu_kernel": {str(d): f'{v["kernel"]}/{v["cluster"]}' for d, v in gpu.items()},
        "cpu_rk_oracle_ms": {str(d): round(v, 3) for d, v in cpu.items()},
        "cpu_expm_ms": {str(d): round(v, 2) for d, v in expm.items()},
        "exponents": {
            "gpu_d>=128": _fit_exponent(big, [gpu[d]["ms"] for d in big]),
            "gpu_all": _fit_exponent(gpu_d, [gpu[d]["ms"] for d in gpu_d]),
            "cpu_rk_oracle": _fit_exponent(cpu_d, [cpu[d] for d in cpu_d]),
            "cpu_expm": _fit_exponent(expm_d, [expm[d] for d in expm_d]),
            "paper": {"rk": 1.9, "expm": 5.8}},
        "cpu_baseline": {"value": cpu[cpu_d[-1]], "unit": "ms", "cores": 1, "kind": "oracle",
                         "sample": f"first-order gradient at d={cpu_d[-1]}, 200 slices"},
        "gpu_launches": None})
    print(json.dumps(line), flush=True)


def serve_trace(n_jobs, scale, rate, seed=1609):
    """Seeded trace: (arrival time, workload); 88% batch-distribution problems,
    10% d=120 / N_t=2000 problems, 2% d=300 / N_t=10000 problems (slice
    counts times `scale`).  The job mix comes from one seeded stream and the
    Poisson arrival times (mean rate `rate`) from another, so a trace at a
    different rate has the same jobs in the same order."""
    import workloads
    rng = np.random.default_rng(seed)
    t = np.cumsum(np.random.default_rng(seed + 1).exponential(1.0 / rate, size=n_jobs))
    out = []
    for k in range(n_jobs):
        r = rng.uniform()
        if r < 0.88:
            i = int(rng.integers(0, 256))
            nt = workloads.batch_problem(i).n_slices
            w = workloads.batch_problem(i, n_slices=max(4, int(round(nt * scale))))
        elif r < 0.98:
            w = workloads.transmon_resonator_d120(n_slices=max(4, int(round(2000 * scale))))
        else:
            phys = workloads.Physics(Q=3, N=100, chi=(0.0, 1.0, 2.6), kerr=-0.01, kappa=1.0,
                                     controls=("res_x", "res_y"))
            nt = max(4, int(round(10000 * scale)))
            w = workloads.make("d300", phys, T=0.003 * nt, n_slices=nt, n_rk=4,
                               states=[(0, 2.0), (1, 2.0 + 1.0j), (2, 1.5j)], u_bound=1.0)
        out.append((float(t[k]), w))
    return out


def run_serve_once(trace, max_slots):
    from paper_1609_03170_gb300 import GrapeProblem, GrapeServer
    probs = [GrapeProblem.from_workload(w) for _, w in trace]
    srv = GrapeServer(max_slots=max_slots)
    t0 = time.perf_counter()
    tickets = []
    pending = {}
    results = {}
    k = 0
    last_report = 0.0
    while len(results) < len(trace):
        now = time.perf_counter() - t0
        if now - last_report > 10.0:
            sys.stderr.write(f"serve slots={max_slots}: {now:.0f} s, submitted {k}, done {len(results)}\n")
            last_report = now
        while k < len(trace) and trace[k][0] <= now:
            tk = srv.submit(probs[k], trace[k][1].u, max_iters=50, lbfgs_m=10,
                            u_min=-5.0, u_max=5.0)
            pending[tk] = k
            k += 1
        for tk in list(pending):
            r = srv.poll(tk, timeout_s=0.0)
            if r is not None:
                results[pending.pop(tk)] = r
        time.sleep(0.0005)
    makespan = time.perf_counter() - t0
    srv.close()
    lat = np.array([results[i][4] for i in range(len(trace))])
    return {"jobs_per_s": len(trace) / makespan, "makespan_s": makespan,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "max_slots": max_slots,
            "evaluations": int(sum(results[i][2] for i in range(len(trace))))}


def run_serve(args):
    scale = 1.0 if args.scale is None else args.scale
    trace = serve_trace(args.jobs, scale, 50.0)
    batched = run_serve_once(trace, 24)
    serial = run_serve_once(trace, 1)
    # the same jobs arriving at 0.8x the measured capacity
    trace08 = serve_trace(args.jobs, scale, 0.8 * batched["jobs_per_s"])
    at08 = run_serve_once(trace08, 24)
    print(json.dumps(_base_line(args, "serve", batched["jobs_per_s"], "jobs/s",
                                1000 * batched["makespan_s"], {
        "config": {"workload": "serve", "jobs": args.jobs, "arrivals": "Poisson 50 jobs/s",
                   "mix_by_job": [f"{w.name}:d{w.d}:Nt{w.n_slices}" for _, w in trace],
                   "slice_scale": scale, "iterations": 50, "box": 5.0,
                   "mix": "88% batch-distribution, 10% d=120/N_t=2000, 2% d=300/N_t=10000 "
                          "(slice counts x scale)"},
        "continuous_batching": batched, "serial_same_gpu": serial,
        "at_0.8x_capacity": at08,
        "throughput_vs_serial": batched["jobs_per_s"] / serial["jobs_per_s"]})), flush=True)


def native_fp64_arm(args, dev):
    """The same gradient in native FP64 (GRAPE_PREC_FP64) on a bounded sample:
    the first FP64_SAMPLE_SLICES slices of the d=120 problem (the same d,
    states, controls and RK substeps), scaled to the whole problem, with the
    adjoint launches' FP64-equivalent flops against the measured FP64 roof."""
    import torch
    import workloads
    from paper_1609_03170_gb300 import GrapeProblem, _lib
    from paper_1609_03170_gb300 import problem as _problem
    w = workloads.transmon_resonator_d120(n_slices=FP64_SAMPLE_SLICES)
    P = GrapeProblem.from_workload(w, precision=_lib.GRAPE_PREC_FP64)
    stream = torch.cuda.Stream()
    u = torch.from_numpy(w.u).cuda()
    F = torch.empty(1, dtype=torch.float64, device="cuda")
    G = torch.empty((w.n_slices, w.n_controls), dtype=torch.float64, device="cuda")

    def step():
        _lib.grape_gradient(P.handle, u.data_ptr(), F.data_ptr(), G.data_ptr(), stream.cuda_stream)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    reps = 3
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(reps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / reps
    P.set_profiling(True)
    P.phase_times()
    for _ in range(reps):
        step()
    torch.cuda.synchronize()
    ph = P.phase_times()
    bm = _problem.band_model(w.phys)
    nb, nt, ndo = band_counts(bm)
    counts = algorithmic_counts(w, nb, nt, ndo)
    adj_ms, adj_n = ph["adjoint"]
    achieved = counts["flops_adjoint"] * reps / (adj_ms * 1e-3) / 1e12
    scale = 2000.0 / FP64_SAMPLE_SLICES
    P.close()
    return {"value": 1000.0 / (ms * scale), "unit": UNIT, "ms_per_step": ms * scale,
            "dtype": "f64",
            "sample": f"first {FP64_SAMPLE_SLICES} of the 2000 slices (same d, states, controls, "
                      f"substeps), {ms:.2f} ms per gradient, scaled x{scale:g}",
            "adjoint_tflops": achieved, "roof": "measured FP64 FMA throughput (alu_peaks.fp64_tflops)"}


def band_counts(bm):
    """Bands of A = H_eff (union of H0, control and c^+c offsets), jump
    terms and distinct control-band offsets of a band model."""
    offs = set(int(o) for o in bm.H0.offsets)
    for h in bm.Hc:
        offs |= set(int(o) for o in h.offsets)
    for c in bm.jumps:
        for o1 in c.offsets:
            for o2 in c.offsets:
                offs.add(int(o2) - int(o1))
    nt = sum(len(c.offsets) ** 2 for c in bm.jumps)
    ndo = len(set(int(o) for h in bm.Hc for o in h.offsets))
    return len(offs), nt, ndo


def main():
    args = parse()
    if args.workload != "d120":
        import torch
        torch.cuda.set_device(0)
        {"batch256": run_batch256, "d600": run_d600, "serve": run_serve,
         "d20": run_d20, "d120f": run_d120f, "d120p": run_d120p,
         "sweep": run_sweep, "peaks": run_peaks}[args.workload](args)
        return
    rank, world, dist = dist_init(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
        if dist:
            dist.destroy_process_group()
        return

    import numpy as np
    import torch
    from paper_1609_03170_gb300 import GrapeProblem, _lib

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    w = workload()
    prec = _lib.GRAPE_PREC_FP64 if args.precision == "fp64" else _lib.GRAPE_PREC_DF64
    P = GrapeProblem.from_workload(w, precision=prec)
    stream = torch.cuda.Stream()
    u_dev = torch.from_numpy(w.u).cuda()
    F_dev = torch.empty(1, dtype=torch.float64, device="cuda")
    G_dev = torch.empty((w.n_slices, w.n_controls), dtype=torch.float64, device="cuda")

    def step_device():
        _lib.grape_gradient(P.handle, u_dev.data_ptr(), F_dev.data_ptr(), G_dev.data_ptr(),
                            stream.cuda_stream)

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            step_device()
    stream.synchronize()
    launches_per_step = P.gradient_launches()

    # ---- device-resident timing (value), no per-launch events -------------
    clocks = ClockSampler(dev)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall = time.perf_counter()
    ev0.record(stream)
    for _ in range(args.steps):
        step_device()
    ev1.record(stream)
    torch.cuda.synchronize()
    wall_ms = 1000.0 * (time.perf_counter() - t_wall) / args.steps
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1) / args.steps

    # ---- per-launch durations of each kernel (CUDA events on the launching
    # streams), a second pass of the same steps -------------------------------
    P.set_profiling(True)
    P.phase_times()
    for _ in range(args.steps):
        step_device()
    torch.cuda.synchronize()
    phases = P.phase_times()
    P.set_profiling(False)

    # ---- end to end through the public API with pinned host buffers ------
    u_host = torch.empty((w.n_slices, w.n_controls), dtype=torch.float64, pin_memory=True)
    u_host.copy_(torch.from_numpy(w.u))
    F_host = torch.empty(1, dtype=torch.float64, pin_memory=True)
    G_host = torch.empty((w.n_slices, w.n_controls), dtype=torch.float64, pin_memory=True)
    _lib.grape_gradient(P.handle, u_host.data_ptr(), F_host.data_ptr(), G_host.data_ptr(),
                        stream.cuda_stream)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _lib.grape_gradient(P.handle, u_host.data_ptr(), F_host.data_ptr(), G_host.data_ptr(),
                            stream.cuda_stream)
    e2e_s = (time.perf_counter() - t0) / args.steps
    clk = clocks.stop()

    # ---- measured FMA throughput (the ALU roofs) and the native-FP64 arm ---
    peaks_alu = fma_peaks(dev)
    fp64_arm = None
    if args.precision == "df64":
        fp64_arm = native_fp64_arm(args, dev)

    if dist:
        ms, e2e_s = max_over_ranks(dist, [ms, e2e_s])
    if rank != 0:
        dist.destroy_process_group()
        return

    from paper_1609_03170_gb300 import problem as _problem
    bm = _problem.band_model(w.phys)
    nb, nt, ndo = band_counts(bm)
    counts = algorithmic_counts(w, nb, nt, ndo)

    fwd_ms, fwd_n = phases["forward"]
    adj_ms, adj_n = phases["adjoint"]
    tr_ms, tr_n = phases["trace"]
    dom = "forward" if fwd_ms >= adj_ms else "adjoint"
    dom_total_ms, dom_n = phases[dom]
    dom_ms = dom_total_ms / max(dom_n, 1)                      # average launch duration
    flops_per_launch = counts["flops_" + dom] * args.steps / max(dom_n, 1)
    achieved = flops_per_launch / (dom_ms * 1e-3) / 1e12
    sha = kernel_source_sha()
    traffic = profiled_traffic(sha)
    if traffic is not None:
        traffic *= flops_per_launch / counts["flops_" + dom]   # profile is per full sweep
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    if args.precision == "fp64":
        peak_tflops = peaks_alu["fp64_tflops"]
        peak_source = "of measured: FP64 FMA throughput (grape_fma_peak) in this run"
    else:
        # double-float: FP64-equivalent flops on the FP32 pipes; the roof is the
        # FP32 FMA rate measured in this run divided by the FP32 instructions
        # one FP64-equivalent flop costs in the pair arithmetic (12 per real
        # multiply-add: TwoProduct 2, cross terms 2, TwoSum 6, error
        # gathering 2 -> 6 per flop)
        peak_tflops = peaks_alu["fp32_tflops"] / DF_FP32_OPS_PER_FLOP
        peak_source = ("of measured: FP32 FMA throughput (grape_fma_peak) in this run / 6 FP32 "
                       "instructions per FP64-equivalent flop")
    step_bytes = counts["bytes_forward"] + counts["bytes_adjoint"] + counts["bytes_trace"]
    value = world * 1000.0 / ms
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "df64" if args.precision == "df64" else "f64", "data": "synthetic",
        "config": {"workload": "transmon_resonator_d120", "d": w.d, "n_slices": w.n_slices,
                   "n_rk": w.n_rk, "n_states": w.n_states, "n_controls": w.n_controls,
                   "n_jumps": len(bm.jumps), "grad_mode": "exact",
                   "cluster": P.geometry()[0], "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2: %.1f GB of stage storage written and read per step"
                         % (step_bytes / 1e9)},
        "roofline": {"bound": "alu", "kernel": f"prop_kernel ({dom})", "achieved": achieved,
                     "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops,
                     "traffic": traffic,
                     "flops_per_launch": flops_per_launch,
                     "launches_per_step": dom_n / args.steps,
                     "ms_per_launch": dom_ms,
                     "peak_source": peak_source},
        "hbm": {"bytes_per_step": step_bytes, "achieved_gbs": step_bytes / (ms * 1e-3) / 1e9,
                "peak_gbs": hbm_peak, "frac": step_bytes / (ms * 1e-3) / 1e9 / hbm_peak,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"},
        "phases_ms_per_step": {k: v[0] / args.steps for k, v in phases.items()},
        "wall_ms_per_step": wall_ms,
        "e2e": {"value": world / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(u_host.numel() * 8),
                "d2h_bytes_per_step": int(F_host.numel() * 8 + G_host.numel() * 8)},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "alu_peaks": peaks_alu,
    }
    if fp64_arm is not None:
        fp64_arm["frac"] = fp64_arm["adjoint_tflops"] / peaks_alu["fp64_tflops"]
        fp64_arm["df64_speedup"] = value / fp64_arm["value"]
        line["fp64"] = fp64_arm
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
