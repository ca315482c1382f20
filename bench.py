#!/usr/bin/env python
"""Benchmark of the batched FP64 PDF interpolation on one or more GB300s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Headline workload (one step): x*f for 13 flavours at 1e7 points of the
NNPDF-shaped grid (196 x knots, 50 Q rows in 4 subgrids) plus alpha_s at 1e7
further points: `xfxQ2` + `alphasQ2` through the C ABI on device-resident
inputs.  `value` = x*f evaluations per second over all ranks; "alphas" times
the alpha_s launch alone; "e2e" times the same step from pinned host memory
(copies in and out inside the timed region).  The other forms
of the hot path are timed in the same run and reported under "forms": the
small 50 x 20 grid (1e5 points x 11 flavours + alpha_s, L2 flushed before each
step), forward+backward (pointwise, 1e7 points, autograd adjoint), the batched
graph-captured launch (400 uneven requests over 3 grids), the fused
luminosity (1e8 events, forward and forward+backward), VEGAS on the fused
luminosity, and VEGAS around a single-top-like integrand written as user
code.  "sweep" holds the x*f throughput against the number of points (1e3 to
1e8, the paper's Fig. 2 axis), with the oracle's under cpu_baseline.

Timing: W warm-up steps, then K steps between a barrier + synchronize and
CUDA events on the launching stream; the max over ranks is reported.  Inputs
and outputs of every timed step exceed the 129 MB L2.  SM clocks and throttle
reasons are sampled with nvidia-smi during the timed region.  N > 1 runs one
independent replica of the workload per rank (the points are independent; no
collective is needed): "scaling": "weak".

`--impl reference` times the FP64 CPU oracle (the plain C implementation of
the same definition) on the host cores, on bounded samples of the same
workload, and prints the same JSON line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP64 xf(x,Q²) evals/sec on 1 GB300, fwd and fwd+bwd, % of roofline"
WORKLOAD = ("NNPDF-shaped grid: 196 x knots in [1e-9,1], Q subgrids 8/12/20/10 knots split at "
            "1.51/4.92/172.5 GeV, 13 flavours; 1e7 points x 13 flavours + 1e7 alpha_s points")
N_POINTS = 10_000_000


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ------------------------------------------------------------------- clocks

class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons (200 ms)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# -------------------------------------------------------------- reference arm

def cpu_oracle_rate(points, cores, budget_s=10.0, chunk=200_000, max_points=None):
    """Oracle x*f evals/s on the host cores over chunks of the headline
    workload until ``budget_s`` seconds of wall time have elapsed."""
    from oracle.oracle import OracleGrid, set_threads
    from paper_2012_08221_gb300 import synth
    set_threads(cores)
    g = synth.grid_nnpdf()
    o = OracleGrid.from_synth(g)
    x, q2 = points
    done, t0 = 0, time.perf_counter()
    limit = max_points or x.size
    while done < limit:
        m = min(chunk, limit - done)
        o.xfxq2_batch(g.pids, x[done:done + m], q2[done:done + m])
        done += m
        if budget_s is not None and time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return done * g.n_flav / dt, done, dt


def host_cpu_model():
    """The host CPU's name from /proc/cpuinfo ("model name" on x86; the
    implementer and part numbers on Arm), else the platform's machine name."""
    import platform
    try:
        txt = open("/proc/cpuinfo").read()
    except OSError:
        return platform.machine()
    fields = {}
    for line in txt.splitlines():
        k, _, v = line.partition(":")
        k, v = k.strip(), v.strip()
        if k and v and k not in fields:
            fields[k] = v
    if "model name" in fields:
        return fields["model name"]
    if "CPU part" in fields:
        return (f"{platform.machine()} CPU implementer {fields.get('CPU implementer', '?')} "
                f"part {fields['CPU part']}")
    return platform.machine()


def _timed_rate(fn, units):
    t0 = time.perf_counter()
    fn()
    return units / (time.perf_counter() - t0)


def forms_cpu_baselines(cores):
    """The oracle on bounded samples of each additional form (a few seconds
    each): rates in the unit of the form's GPU value."""
    import numpy as np

    from oracle.oracle import OracleGrid, set_threads
    from paper_2012_08221_gb300 import synth
    set_threads(cores)
    out = {}
    g1 = synth.grid_small()
    o1 = OracleGrid.from_synth(g1)
    x1, q1 = synth.queries_small()

    def small():
        o1.xfxq2_batch(g1.pids, x1, q1)
        o1.alphas_batch(q1)
    small()
    out["small"] = {"value": _timed_rate(small, x1.size * g1.n_flav), "unit": "evals/s", "cores": cores,
                    "kind": "oracle", "sample": f"the whole workload ({x1.size} points and alpha_s)"}
    gs = synth.grid_small(seed=1003, pids=synth.PIDS_13)
    o3 = OracleGrid.from_synth(gs)
    pid, x, q2, w = synth.queries_pointwise(20_000)

    def fb():
        o3.xfxq2_pw(pid, x, q2)
        o3.grad_pw(pid, x, q2)
        o3.dgrid_pw(pid, x, q2, w)
    out["fwd_bwd"] = {"value": _timed_rate(fb, x.size), "unit": "evals/s (fwd+bwd)", "cores": cores,
                      "kind": "oracle", "sample": "20000 points of the pointwise workload "
                      "(grid gradient summed serially)"}
    grids = [synth.grid_set_a(), synth.grid_set_b(), synth.grid_set_c()]
    ogs = [OracleGrid.from_synth(gg) for gg in grids]
    reqs = synth.batches_uneven(grids, n_batches=400)
    done, evals, t0 = 0, 0, time.perf_counter()
    for b in reqs:
        m = min(b.x.size, 20_000)
        ogs[b.set_index].xfxq2_batch(b.pids, b.x[:m], b.q2[:m], member=b.member)
        evals += m * b.pids.size
        done += 1
        if time.perf_counter() - t0 > 5.0:
            break
    out["batched"] = {"value": evals / (time.perf_counter() - t0), "unit": "evals/s", "cores": cores,
                      "kind": "oracle", "sample": f"first <= 20000 points of the first {done} requests"}
    g5 = synth.grid_nnpdf(seeds=(1005, 1006, 1007))
    o5 = OracleGrid.from_synth(g5)
    ev = synth.events_lhc(40_000)
    r_f = _timed_rate(lambda: o5.lumi(ev), ev.ln_tau.size * 2 * g5.n_flav)
    sub = synth.Events(ev.ln_tau[:2000], ev.y[:2000], ev.flags[:2000], ev.ln_mu2[:2000], ev.ln_x1[:2000],
                       ev.ln_s)
    r_b = _timed_rate(lambda: (o5.lumi(sub), o5.lumi_dgrid(sub)), 2000 * 2 * g5.n_flav)
    out["lumi"] = {"fwd": {"value": r_f, "unit": "evals/s", "cores": cores, "kind": "oracle",
                           "sample": "40000 events"},
                   "fwd_bwd": {"value": r_b, "unit": "evals/s (fwd+bwd)", "cores": cores, "kind": "oracle",
                               "sample": "2000 events (grid gradient summed serially)"}}
    return out


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    from paper_2012_08221_gb300 import synth
    cores = len(os.sched_getaffinity(0))
    x, q2, _ = synth.queries_nnpdf()
    per_step = 500_000
    for w in range(args.warmup):
        s = (w * per_step) % (x.size - per_step)
        cpu_oracle_rate((x[s:s + per_step], q2[s:s + per_step]), cores, budget_s=None)
    t0 = time.perf_counter()
    for k in range(args.steps):
        s = ((args.warmup + k) * per_step) % (x.size - per_step)
        cpu_oracle_rate((x[s:s + per_step], q2[s:s + per_step]), cores, budget_s=None)
    dt = time.perf_counter() - t0
    value = args.steps * per_step * 13 / dt
    line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "sample_per_step": f"{per_step} points x 13 flavours"},
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": "evals/s", "cores": cores,
                             "sample": f"{per_step} consecutive points of the 1e7-point workload per step"},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm

def kernel_source(path, name):
    """The text of the function `name` defined in `path` (a kernel or its
    launcher): from the template line above its signature to its closing
    brace."""
    text = open(os.path.join(ROOT, path)).read()
    m = re.search(r"^(template <[^\n]*>\n)?[A-Za-z_][^\n;]*\b" + re.escape(name) + r"\(", text, re.M)
    if m is None:
        raise KeyError(f"{name} not in {path}")
    i = text.index("{", m.end())
    depth = 0
    for j in range(i, len(text)):
        depth += {"{": 1, "}": -1}.get(text[j], 0)
        if depth == 0:
            return text[m.start():j + 1]
    raise ValueError(f"unbalanced braces after {name} in {path}")


def source_hash(files):
    """Hash of a kernel's sources: whole files, or "path::kernel" for the one
    function (so that host code beside it does not invalidate a capture)."""
    h = hashlib.sha256()
    for f in files:
        if "::" in f:
            path, name = f.split("::")
            h.update(kernel_source(path, name).encode())
        else:
            h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def _capture(kernel):
    """The committed ncu figures of `kernel` (profiles/traffic.json) if they
    were taken on the kernel's current sources, else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    e = d.get(kernel)
    if not e or e.get("source_hash") != source_hash(e.get("files", [])):
        return None
    return e


def measured_traffic(kernel, units):
    """DRAM bytes (read + write) per launch of `kernel` over `units` points,
    scaled from the committed ncu capture's bytes per point, if that capture
    was taken on the current sources of the kernel (else None)."""
    e = _capture(kernel)
    return None if e is None else e["dram_bytes_per_unit"] * units


def measured_pipe(kernel):
    """FP64-pipe occupancy (% of active cycles) of the same capture, or None."""
    e = _capture(kernel)
    return None if e is None else e.get("fp64_pipe_active_pct")


def reduce_max(v, world, device):
    """Max of a float over all ranks (identity for one rank)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms_max):
    """Replicas: every rank processes `units_per_rank`; the job's rate is all
    ranks' units over the slowest rank's time."""
    return world * units_per_rank / (ms_max * 1e-3)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# FP64 FMA issue rate per SM per clock on GB300: ncu reports a peak of 304
# DFMA thread-instructions per cycle for 152 SMs.
DFMA_PER_SM_CLK = 2


def fp64_derived_peak(sm_count):
    """FP64 FLOP/s from the unit counts and the maximum SM clock: SMs x 2
    DFMA per clock x 2 flops x max MHz (the roofline's denominator)."""
    mhz = float(peaks().get("sm_max_mhz", 2070.0))
    return sm_count * DFMA_PER_SM_CLK * 2 * mhz * 1e6, mhz


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--forms", default="all",
                    help="comma list of small,fwdbwd,batched,lumi,vegas,vegas_user or all/none")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the throughput-against-length sweep")
    ap.add_argument("--points", type=int, default=N_POINTS,
                    help="points of the headline workload (smaller only for profiling captures)")
    ap.add_argument("--lumi-events", type=int, default=100_000_000,
                    help="events of the luminosity form (smaller only for profiling captures)")
    ap.add_argument("--vegas-points", type=int, default=10_000_000,
                    help="points per VEGAS iteration")
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="size factor of the batched form's requests (smaller only for profiling)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2012_08221_gb300 import build, synth, work
    build.build()
    from paper_2012_08221_gb300.pdf import PDF, fp64_mixed, fp64_mma_peak, fp64_peak

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def max_ranks(v):
        return reduce_max(v, world, dev)

    probe = fp64_peak()                             # FLOP/s, FMA chains (burst)
    mma_probe = {"m8n8k4_tflops": fp64_mma_peak("m8n8k4") / 1e12,
                 **{k + "_tflops": v / 1e12 for k, v in fp64_mixed().items()}}
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak, peak_mhz = fp64_derived_peak(sms)
    stream = torch.cuda.current_stream(dev)

    def timed(step, K, W, kernel_step=None):
        """Returns (ms per step max over ranks, mean kernel ms or None)."""
        for _ in range(W):
            step()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        kev = [] if kernel_step else None
        e0.record(stream)
        for _ in range(K):
            if kernel_step:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                kernel_step(a, b)
                kev.append((a, b))
            else:
                step()
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1) / K
        kms = statistics.mean(a.elapsed_time(b) for a, b in kev) if kev else None
        return max_ranks(ms), kms

    # ---------------------------------------------------- headline workload
    g = synth.grid_nnpdf()
    pdf = PDF.from_grid(g, device=dev)
    npts = args.points
    x, q2, q2a = synth.queries_nnpdf(npts, seed=2002)
    X = torch.as_tensor(x, device=dev)
    Q = torch.as_tensor(q2, device=dev)
    QA = torch.as_tensor(q2a, device=dev)
    OUT = torch.empty((npts, g.n_flav), dtype=torch.float64, device=dev)
    AS = torch.empty(npts, dtype=torch.float64, device=dev)
    pids = g.pids

    def step():
        pdf.xfxQ2(pids, X, Q, out=OUT)
        pdf.alphasQ2(QA, out=AS)

    def kstep(a, b):
        a.record(stream)
        pdf.xfxQ2(pids, X, Q, out=OUT)
        b.record(stream)
        pdf.alphasQ2(QA, out=AS)

    clocks = Clocks(local)
    clocks.start()
    ms, k_ms = timed(step, args.steps, args.warmup, kstep)
    evals = npts * g.n_flav
    value = whole_job_rate(evals, world, ms)
    flops_launch = npts * work.xfxq2_point_flops(g.n_flav)
    flops_matrix = npts * work.xfxq2_point_flops_matrix_form(g.n_flav)
    bytes_launch = npts * work.xfxq2_point_bytes(g.n_flav)
    achieved = flops_launch / (k_ms * 1e-3)
    traffic = measured_traffic("k_xfxq2", npts)
    roofline = {"bound": "alu", "pipe": "fp64", "kernel": "k_xfxq2",
                "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "flops_per_point": work.xfxq2_point_flops(g.n_flav),
                "frac_matrix_form": flops_matrix / (k_ms * 1e-3) / peak,
                "flops_per_point_matrix_form": work.xfxq2_point_flops_matrix_form(g.n_flav),
                "frac_note": "frac counts the flops of the patch form the kernel runs (15 FMA per flavour, "
                             "table log); frac_matrix_form counts 40 F + 50 flops per point, the separable-"
                             "weight form (20 FMA per flavour + weights), which does more arithmetic than the "
                             "kernel and so can exceed 1; the headroom left is 100 - ncu_fp64_pipe_active_pct",
                "peak_source": f"derived: {sms} SMs x {DFMA_PER_SM_CLK} DFMA/clk x 2 flop x {peak_mhz:.0f} MHz "
                               f"(max SM clock)",
                "probe": {"value": probe / 1e12, "unit": "TFLOP/s",
                          "what": "FP64 FMA chains measured in this run (pdf_probe_fp64_peak)"},
                "fp64_tensor_probe": {**mma_probe,
                                      "what": "mma.sync f64 chains alone (pdf_probe_fp64_mma_peak), and equal "
                                              "FP64 work as DFMA alone, DMMA alone and both interleaved in each "
                                              "warp (pdf_probe_fp64_mixed): a mixed rate near the slower one, not "
                                              "their sum, means one shared FP64 pipe"},
                "traffic": traffic,
                "ncu_fp64_pipe_active_pct": measured_pipe("k_xfxq2"),
                "algorithmic_bytes": bytes_launch,
                "achieved_gbs": bytes_launch / (k_ms * 1e-3) / 1e9,
                "hbm_peak_gbs": peaks().get("hbm_gbs", 6790.7),
                "hbm_frac": (bytes_launch / (k_ms * 1e-3)) / (peaks().get("hbm_gbs", 6790.7) * 1e9),
                "kernel_ms": k_ms}

    # alpha_s alone (reported separately: one evaluation per Q^2)
    ms_as, _ = timed(lambda: pdf.alphasQ2(QA, out=AS), args.steps, args.warmup)
    alphas = {"value": whole_job_rate(npts, world, ms_as), "unit": "evals/s", "ms_per_step": ms_as,
              "kernel": "k_alphas", "points": npts,
              "fp64_frac": npts * work.alphas_point_flops() / (ms_as * 1e-3) / peak,
              "hbm_frac": (16 * npts / (ms_as * 1e-3)) / (peaks().get("hbm_gbs", 6790.7) * 1e9)}

    # --------------------------- throughput against the query length (Fig. 2)
    sweep = None
    if not args.no_sweep:
        gen = torch.Generator(device=dev)
        gen.manual_seed(2010)
        sweep = {"what": "xfxQ2 over 13 flavours on the NNPDF-shaped grid against the number of points "
                         "(ln x ~ U[ln 1e-8, 0), ln Q^2 ~ U[0, ln 1e10]); below ~1e6 points the inputs and "
                         "outputs stay in L2 and the launch is latency-bound",
                 "n": [], "ms": [], "evals_per_s": [], "fp64_frac": [],
                 "ms_graph": [], "note_graph": "the same call captured once in a CUDA graph and replayed: "
                                               "the host-side cost of the Python call left out"}
        for n_s in (10 ** 3, 10 ** 4, 10 ** 5, 10 ** 6, 10 ** 7, 10 ** 8):
            Xs = torch.exp(torch.rand(n_s, generator=gen, dtype=torch.float64, device=dev) * math.log(1e-8))
            Qs = torch.exp(torch.rand(n_s, generator=gen, dtype=torch.float64, device=dev) * math.log(1e10))
            Os = torch.empty((n_s, g.n_flav), dtype=torch.float64, device=dev)
            ms_s, _ = timed(lambda: pdf.xfxQ2(pids, Xs, Qs, out=Os), 5 if n_s >= 10 ** 8 else 20, args.warmup)
            sweep["n"].append(n_s)
            sweep["ms"].append(ms_s)
            sweep["evals_per_s"].append(world * n_s * g.n_flav / (ms_s * 1e-3))
            sweep["fp64_frac"].append(n_s * work.xfxq2_point_flops(g.n_flav) / (ms_s * 1e-3) / peak)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                pdf.xfxQ2(pids, Xs, Qs, out=Os)
            ms_g, _ = timed(graph.replay, 5 if n_s >= 10 ** 8 else 20, args.warmup)
            sweep["ms_graph"].append(ms_g)
            del Xs, Qs, Os, graph

    forms = {}
    want = set(["small", "combined", "fwdbwd", "batched", "lumi", "vegas", "vegas_user"] if args.forms == "all" else
               ([] if args.forms == "none" else args.forms.split(",")))

    # ------------- x*f and alpha_s at the same Q^2: one launch against two
    if "combined" in want:
        OUTc = torch.empty_like(OUT)
        ASc = torch.empty_like(AS)

        def two_calls():
            pdf.xfxQ2(pids, X, Q, out=OUTc)
            pdf.alphasQ2(Q, out=ASc)

        ms_two, _ = timed(two_calls, args.steps, args.warmup)
        ms_one, _ = timed(lambda: pdf.xfxQ2_alphasQ2(pids, X, Q, out=OUTc, alphas=ASc), args.steps, args.warmup)
        forms["combined"] = {
            "workload": "NNPDF-shaped grid, 1e7 points x 13 flavours and alpha_s at the same Q^2 (as an "
                        "integrand needs them at each point's factorisation scale)",
            "value": whole_job_rate(evals + npts, world, ms_one), "unit": "evals/s (x*f and alpha_s)",
            "ms_per_step": ms_one, "kernel": "k_xfxq2 with alpha_s (xfxQ2_alphasQ2)",
            "two_calls": {"ms_per_step": ms_two, "what": "xfxQ2 then alphasQ2 on the same arrays"},
            "fp64_frac": npts * (work.xfxq2_point_flops(g.n_flav) + 6) / (ms_one * 1e-3) / peak}
        del OUTc, ASc

    # ------------------------- the small grid: 50 x 20 knots, 11 flavours
    if "small" in want:
        g1 = synth.grid_small()
        p1 = PDF.from_grid(g1, device=dev)
        x1h, q1h = synth.queries_small()
        n1 = x1h.size
        X1, Q1 = torch.as_tensor(x1h, device=dev), torch.as_tensor(q1h, device=dev)
        O1 = torch.empty((n1, g1.n_flav), dtype=torch.float64, device=dev)
        A1 = torch.empty(n1, dtype=torch.float64, device=dev)
        flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device=dev)     # 256 MB > L2

        def step1():                     # alpha_s at the same Q^2: one launch
            p1.xfxQ2_alphasQ2(g1.pids, X1, Q1, out=O1, alphas=A1)

        def step1_two():
            p1.xfxQ2(g1.pids, X1, Q1, out=O1)
            p1.alphasQ2(Q1, out=A1)

        def flushed(fn, K):
            """Mean device time of fn, L2 flushed before each call (outside
            the events)."""
            for _ in range(args.warmup):
                fn()
            barrier()
            evs = []
            for _ in range(K):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                evs.append((a, b))
            barrier()
            return max_ranks(statistics.mean(a.elapsed_time(b) for a, b in evs))

        ms1 = flushed(step1, 20)
        ms1_two = flushed(step1_two, 20)
        graph1 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph1):
            step1()
        ms1g = flushed(graph1.replay, 20)
        forms["small"] = {
            "workload": f"50 x 20 grid (x in [1e-7, 1], one Q subgrid [1.65, 1e4] GeV), {g1.n_flav} flavours; "
                        f"{n1} points x {g1.n_flav} flavours + alpha_s at the same {n1} Q^2",
            "value": whole_job_rate(n1 * g1.n_flav, world, ms1), "unit": "evals/s", "ms_per_step": ms1,
            "ms_graph": ms1g, "value_graph": whole_job_rate(n1 * g1.n_flav, world, ms1g),
            "entry_point": "xfxQ2_alphasQ2 (x*f and alpha_s at the same Q^2 in one launch)",
            "two_calls": {"ms_per_step": ms1_two, "what": "xfxQ2 then alphasQ2 on the same arrays"},
            "fp64_frac": n1 * (work.xfxq2_point_flops(g1.n_flav) + 6) / (ms1 * 1e-3) / peak,
            "l2": "flushed (256 MB write) before every timed step; the step's data fit in L2",
            "note": "1e5 points occupy about half of one wave of resident threads (152 SMs x 1280): "
                    "the time is mostly one thread's latency (11 patches after coefficient loads that "
                    "miss the flushed L2)"}
        del flush, graph1

    # --------------------------------------------------- forward + backward
    if "fwdbwd" in want:
        gs = synth.grid_small(seed=1003, pids=synth.PIDS_13)
        p3 = PDF.from_grid(gs, device=dev)
        pid, x3, q3, w3 = synth.queries_pointwise()
        P3, X3, Q3, W3 = (torch.as_tensor(a, device=dev) for a in (pid, x3, q3, w3))
        V3 = torch.as_tensor(gs.values, device=dev)
        O3 = torch.empty(x3.size, dtype=torch.float64, device=dev)
        GV = torch.zeros(gs.values.shape[1:], dtype=torch.float64, device=dev)

        T3 = p3.new_tape(x3.size)            # the forward's adjoint tape (32 B per point)
        D3 = p3.new_dtape(x3.size)           # its patch derivatives and bins (20 B per point)

        def step3():
            p3.bind_values(V3)
            p3.xfxQ2_pw(P3, X3, Q3, out=O3, tape=T3, dtape=D3)
            GV.zero_()
            p3.xfxQ2_backward(P3, X3, Q3, W3, pointwise=True, grad_values=GV, tape=T3, dtape=D3)

        def kstep3(a, b):
            p3.bind_values(V3)
            p3.xfxQ2_pw(P3, X3, Q3, out=O3, tape=T3, dtape=D3)
            GV.zero_()
            a.record(stream)
            p3.xfxQ2_backward(P3, X3, Q3, W3, pointwise=True, grad_values=GV, tape=T3, dtape=D3)
            b.record(stream)

        def step3n():                        # the same without the tape
            p3.bind_values(V3)
            p3.xfxQ2_pw(P3, X3, Q3, out=O3)
            GV.zero_()
            p3.xfxQ2_backward(P3, X3, Q3, W3, pointwise=True, grad_values=GV)

        # the step as a user writes it: L = sum_i w_i xf_{a_i}(x_i, Q^2_i)
        # through torch.autograd (the Function's forward keeps the tape)
        from paper_2012_08221_gb300.autograd import xfxQ2_pw as ad_xfxQ2_pw
        VA = V3.clone().requires_grad_(True)
        XA, QA3 = X3.clone().requires_grad_(True), Q3.clone().requires_grad_(True)

        def step3a():
            VA.grad = XA.grad = QA3.grad = None
            L3 = (ad_xfxQ2_pw(p3, VA, P3, XA, QA3) * W3).sum()
            L3.backward()

        # the matrix form through autograd: every flavour at each point
        from paper_2012_08221_gb300.autograd import xfxQ2 as ad_xfxQ2
        nm = 1_000_000
        VM = V3.clone().requires_grad_(True)
        XM, QM = X3[:nm].clone().requires_grad_(True), Q3[:nm].clone().requires_grad_(True)
        WM = torch.as_tensor(np.random.default_rng(7).standard_normal((nm, gs.n_flav)), device=dev)

        def step3m():
            VM.grad = XM.grad = QM.grad = None
            (ad_xfxQ2(p3, VM, gs.pids, XM, QM) * WM).sum().backward()

        ms3a, _ = timed(step3a, args.steps, args.warmup)
        ms3, kb = timed(step3, args.steps, args.warmup, kstep3)
        ms3n, _ = timed(step3n, max(3, args.steps // 2), args.warmup)
        ms3m, _ = timed(step3m, args.steps, args.warmup)
        n3 = x3.size
        fl = n3 * (work.pw_fwd_point_flops(dtape=True) + work.pw_bwd_sorted_point_flops(dtape=True))
        forms["fwd_bwd"] = {
            "workload": "pointwise x*f and its adjoint (dL/dx, dL/dQ^2, dL/dgrid) at 1e7 points, "
                        "50x20 grid, 13 flavours, L = sum w_i xf_{a_i}, through torch.autograd",
            "value": world * n3 / (ms3a * 1e-3), "unit": "evals/s (fwd+bwd)", "ms_per_step": ms3a,
            "fp64_frac": (fl / (ms3a * 1e-3)) / peak,
            "fp64_frac_separable_count": n3 * work.pw_fwd_bwd_point_flops_separable() / (ms3a * 1e-3) / peak,
            "flops_per_point": {"fwd": work.pw_fwd_point_flops(dtape=True),
                                "bwd": work.pw_bwd_sorted_point_flops(dtape=True),
                                "separable_fwd_bwd": work.pw_fwd_bwd_point_flops_separable()},
            "bwd_kernel": {"kernels": "k_bwd_count, k_scan, k_bwd_rec, k_bwd_accum (from the tape; grid "
                                      "gradient sorted by cell and flavour)", "ms": kb,
                           "frac": n3 * work.pw_bwd_sorted_point_flops(dtape=True) / (kb * 1e-3) / peak,
                           "frac_separable_count": n3 * work.pw_bwd_point_flops_separable() / (kb * 1e-3) / peak},
            "tape": "the forward pass writes 32 bytes per point (cells, local coordinates, flags) that the "
                    "adjoint reads instead of searching the knots and taking logarithms again, and 20 bytes "
                    "of patch derivatives (computed with the value) and the point's bin, which spare the "
                    "adjoint the coefficients and let it count its bins from 4 bytes per point",
            "direct_calls": {"ms_per_step": ms3, "value": world * n3 / (ms3 * 1e-3),
                             "what": "the same two library calls without autograd (no torch "
                                     "multiply, sum or gradient accumulation)"},
            "without_tape": {"ms_per_step": ms3n, "value": world * n3 / (ms3n * 1e-3),
                             "what": "direct calls, the adjoint recomputing the coordinates"},
            "matrix_form": {"workload": "1e6 points x all 13 flavours, L = sum w_ia xf_a(x_i, Q^2_i), "
                                        "through torch.autograd (xfxQ2 with the pid list)",
                            "value": world * nm * gs.n_flav / (ms3m * 1e-3), "unit": "evals/s (fwd+bwd)",
                            "ms_per_step": ms3m}}
        del P3, X3, Q3, W3, O3, T3, D3, VA, XA, QA3, VM, XM, QM, WM

    # ------------------------------------------------------------- batched
    if "batched" in want:
        from paper_2012_08221_gb300.batch import Batch
        grids = [synth.grid_set_a(), synth.grid_set_b(), synth.grid_set_c()]
        pdfs = [PDF.from_grid(gg, device=dev) for gg in grids]
        reqs = []
        ev4 = 0
        fl4 = 0
        for b in synth.batches_uneven(grids, scale=args.batch_scale):
            xb, qb = torch.as_tensor(b.x, device=dev), torch.as_tensor(b.q2, device=dev)
            ob = torch.empty((b.x.size, b.pids.size), dtype=torch.float64, device=dev)
            reqs.append((pdfs[b.set_index], b.member, b.pids, xb, qb, ob))
            ev4 += b.x.size * b.pids.size
            fl4 += b.x.size * work.xfxq2_point_flops(b.pids.size)
        B = Batch(reqs, autotune=True)
        ms4, _ = timed(B.run, args.steps, args.warmup)
        forms["batched"] = {
            "workload": "400 requests, sizes log-uniform in [1e3,1e6] (%d points), 1-3 pids each, "
                        "sets A (101 replicas 50x20), B (100x30, 3 subgrids), C (50 replicas 150x45, "
                        "4 subgrids); one graph-captured persistent launch" % sum(r[3].numel() for r in reqs),
            "value": world * ev4 / (ms4 * 1e-3), "unit": "evals/s", "ms_per_step": ms4,
            "fp64_frac": (fl4 / (ms4 * 1e-3)) / peak, "tuned": B.info()}
        del reqs, B

    # ---------------------------------------------------------- luminosity
    if "lumi" in want:
        from paper_2012_08221_gb300.lumi import DeviceEvents, luminosity, luminosity_backward
        g5 = synth.grid_nnpdf(seeds=(1005, 1006, 1007))
        p5 = PDF.from_grid(g5, device=dev)
        n5 = args.lumi_events
        ev = DeviceEvents.from_host(synth.events_lhc(n5), device=dev)
        LUM = torch.empty(n5, dtype=torch.float64, device=dev)
        L5 = torch.empty((), dtype=torch.float64, device=dev)
        GV5 = torch.zeros(g5.values.shape[1:], dtype=torch.float64, device=dev)
        SAVE = torch.empty((n5, 2, g5.n_flav), dtype=torch.float64, device=dev)

        def step5():
            luminosity(p5, ev, want_lum=True, want_alphas=True, out=L5)

        def step5b():                       # forward keeps the partner factors
            luminosity(p5, ev, want_lum=False, want_alphas=False, out=L5, save_p=SAVE)
            GV5.zero_()
            luminosity_backward(p5, ev, 1.0, GV5, saved_p=SAVE)

        def step5r():                       # backward recomputes them
            luminosity(p5, ev, want_lum=False, want_alphas=False, out=L5)
            GV5.zero_()
            luminosity_backward(p5, ev, 1.0, GV5)

        K5 = max(3, args.steps // 2)
        ms5, _ = timed(step5, K5, args.warmup)
        ms5b, _ = timed(step5b, max(2, K5 // 2), args.warmup)
        ms5r, _ = timed(step5r, 2, args.warmup)
        ev5 = n5 * 2 * g5.n_flav
        forms["lumi"] = {
            "workload": f"{n5:.0e} events at sqrt(s) = 13 TeV (5% low tail), x1 and x2 over 13 flavours, "
                        "luminosity sum_a f_a(x1) f_-a(x2) and alpha_s per event, L = mean",
            "fwd": {"value": world * ev5 / (ms5 * 1e-3), "unit": "evals/s", "ms_per_step": ms5,
                    "fp64_frac": n5 * work.lumi_event_flops(g5.n_flav) / (ms5 * 1e-3) / peak},
            "fwd_bwd": {"value": world * ev5 / (ms5b * 1e-3), "unit": "evals/s (fwd+bwd)",
                        "ms_per_step": ms5b, "partner_factors": "saved by the forward pass",
                        "fp64_frac": n5 * (work.lumi_event_flops(g5.n_flav) +
                                           work.lumi_bwd_event_flops(g5.n_flav, saved=True))
                        / (ms5b * 1e-3) / peak},
            "fwd_bwd_recompute": {"value": world * ev5 / (ms5r * 1e-3), "unit": "evals/s (fwd+bwd)",
                                  "ms_per_step": ms5r, "partner_factors": "recomputed by the backward pass",
                                  "fp64_frac": n5 * (work.lumi_event_flops(g5.n_flav) +
                                                     work.lumi_bwd_event_flops(g5.n_flav))
                                  / (ms5r * 1e-3) / peak}}
        del ev, LUM, SAVE
    # ------------------------------------------------------- VEGAS integration
    if "vegas" in want:
        from paper_2012_08221_gb300.vegas import VegasLumi
        gv = synth.grid_nnpdf()
        pv = PDF.from_grid(gv, device=dev)
        n_it, n_pts = 5, args.vegas_points
        gen = torch.Generator(device=dev)
        gen.manual_seed(2006)
        U = [torch.rand((n_pts, 2), generator=gen, dtype=torch.float64, device=dev) for _ in range(n_it)]
        ln_tau_min, ln_s = math.log(1e-6), 2 * math.log(13000.0)
        res = {}

        def step6():
            res["r"] = VegasLumi(pv, ln_tau_min, ln_s, n_bins=50).integrate(n_iter=n_it, n_per_iter=n_pts,
                                                                              uniforms=U)

        ms6, _ = timed(step6, 2, args.warmup)
        r = res["r"]
        pts = n_it * n_pts
        forms["vegas"] = {
            "workload": f"VEGAS integral of the parton luminosity over (ln tau, y), tau > 1e-6, sqrt(s) = 13 TeV; "
                        f"{n_it} adapting iterations x {n_pts} points, 50 bins per dimension",
            "value": world * pts * 2 * gv.n_flav / (ms6 * 1e-3), "unit": "evals/s",
            "points_per_s": world * pts / (ms6 * 1e-3), "ms_per_step": ms6,
            "fp64_frac": pts * work.vegas_point_flops(gv.n_flav) / (ms6 * 1e-3) / peak,
            "integral": r.integral, "error": r.error, "chi2_dof": r.chi2_dof}
        del U

    # ------------------------------------- VEGAS around a user integrand
    if "vegas_user" in want:
        from paper_2012_08221_gb300.vegas import Vegas
        gs = synth.grid_nnpdf()
        ps = PDF.from_grid(gs, device=dev)
        n_it, n_pts = 5, args.vegas_points
        gen = torch.Generator(device=dev)
        gen.manual_seed(2007)
        U = [torch.rand((n_pts, 3), generator=gen, dtype=torch.float64, device=dev) for _ in range(n_it)]
        b_pid = np.array([5], dtype=np.int32)
        q_pids = np.array([2, 4, -1, -3], dtype=np.int32)
        mt, mw, s_had = 173.0, 80.4, 13000.0 ** 2
        ln_tau_min = math.log(mt * mt / s_had)

        def single_top_like(r):
            # phase space (tau, y, cos theta), a t-channel W propagator and
            # b x (u, c, d-bar, s-bar) luminosity: the shape of a single-top
            # LO integrand, with a toy matrix element
            ln_tau = (1.0 - r[:, 0]) * ln_tau_min
            tau = torch.exp(ln_tau)
            y = (2.0 * r[:, 1] - 1.0) * (-0.5 * ln_tau)
            x1, x2 = torch.exp(0.5 * ln_tau + y), torch.exp(0.5 * ln_tau - y)
            shat = tau * s_had
            that = -(shat - mt * mt) * (1.0 - (2.0 * r[:, 2] - 1.0)) / 2.0
            me2 = shat * (shat - mt * mt) / (that - mw * mw) ** 2
            q2 = torch.full_like(x1, mt * mt)
            lum = ps.xfxQ2(b_pid, x1, q2)[:, 0] * ps.xfxQ2(q_pids, x2, q2).sum(1) / (x1 * x2)
            return (-ln_tau_min) * tau * (-ln_tau) * 2.0 * me2 * lum / (2.0 * shat)

        res = {}

        def step7():
            res["r"] = Vegas(3, n_bins=50, device=dev).integrate(single_top_like, n_iter=n_it,
                                                                 n_per_iter=n_pts, uniforms=U)

        ms7, _ = timed(step7, 2, args.warmup)
        r = res["r"]
        pts = n_it * n_pts
        forms["vegas_user"] = {
            "workload": f"VEGAS over 3 dimensions around a single-top-like LO integrand written as user code "
                        f"(torch operations; xfxQ2 for b at x1 and u, c, d-bar, s-bar at x2, Q = 173 GeV); "
                        f"{n_it} adapting iterations x {n_pts} points, 50 bins per dimension",
            "value": world * pts * 5 / (ms7 * 1e-3), "unit": "evals/s",
            "points_per_s": world * pts / (ms7 * 1e-3), "ms_per_step": ms7,
            "integral": r.integral, "error": r.error, "chi2_dof": r.chi2_dof}
        del U

    clk = clocks.stop()

    # ----------------------------------------------------------- end to end
    # the whole step from pinned host memory: x*f through xfxQ2_host (its own
    # copy/compute pipeline) and, on a side stream at the same time, the alpha_s
    # points copied in, evaluated and copied back in four pieces (which share
    # the host link with the x*f copies better than one large copy each way:
    # 6.44 vs 6.77 ms per 1e7-point step; x*f alone 5.80 ms)
    xh = torch.as_tensor(x).pin_memory()
    qh = torch.as_tensor(q2).pin_memory()
    qah = torch.as_tensor(q2a).pin_memory()
    oh = torch.empty((npts, g.n_flav), dtype=torch.float64).pin_memory()
    ash = torch.empty(npts, dtype=torch.float64).pin_memory()
    side = torch.cuda.Stream(dev)

    def e2e_step():
        with torch.cuda.stream(side):
            m = (npts + 3) // 4
            for s0 in range(0, npts, m):
                s1 = min(npts, s0 + m)
                QA[s0:s1].copy_(qah[s0:s1], non_blocking=True)
                pdf.alphasQ2(QA[s0:s1], out=AS[s0:s1])
                ash[s0:s1].copy_(AS[s0:s1], non_blocking=True)
        pdf.xfxQ2_host(pids, xh, qh, out=oh)
        side.synchronize()

    e2e_step()
    KE = max(2, min(args.steps, 5))
    barrier()
    t0 = time.perf_counter()
    for _ in range(KE):
        e2e_step()
    barrier()
    e2e_s = max_ranks((time.perf_counter() - t0) / KE)
    e2e = {"value": world * evals / e2e_s, "unit": "evals/s", "h2d_bytes_per_step": 24 * npts,
           "d2h_bytes_per_step": 8 * (g.n_flav + 1) * npts, "ms_per_step": 1e3 * e2e_s,
           "entry_point": "xfxQ2_host (pinned host buffers, chunked copy/compute overlap) and alphasQ2 "
                          "with its copies on a second stream"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = len(os.sched_getaffinity(0))
        rate, done, dt = cpu_oracle_rate((x, q2), cores, budget_s=10.0)
        rate1, done1, dt1 = cpu_oracle_rate((x, q2), 1, budget_s=3.0, chunk=20_000)
        cpu = {"value": rate, "unit": "evals/s", "cores": cores, "kind": "oracle",
               "sample": f"first {done} points of the 1e7-point workload x 13 flavours ({dt:.1f} s)",
               "cpu_model": host_cpu_model(),
               "single_core": {"value": rate1, "unit": "evals/s",
                               "sample": f"first {done1} points, one thread ({dt1:.1f} s)"}}
        if sweep is not None:
            # the oracle against the query length, as the GPU sweep (small N only)
            cs = {"n": [], "evals_per_s": []}
            for n_s in (10 ** 3, 10 ** 4, 10 ** 5, 10 ** 6):
                r_s, _, _ = cpu_oracle_rate((x, q2), cores, budget_s=None, max_points=n_s)
                cs["n"].append(n_s)
                cs["evals_per_s"].append(r_s)
            cpu["sweep"] = cs
        if forms:
            fcpu = forms_cpu_baselines(cores)
            for k in forms:
                if k in fcpu and k != "lumi":
                    forms[k]["cpu_baseline"] = fcpu[k]
            if "lumi" in forms:
                forms["lumi"]["fwd"]["cpu_baseline"] = fcpu["lumi"]["fwd"]
                forms["lumi"]["fwd_bwd"]["cpu_baseline"] = fcpu["lumi"]["fwd_bwd"]

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded NNPDF-shaped grid and log-uniform queries)",
                "config": {"workload": WORKLOAD if npts == N_POINTS else WORKLOAD + f" (reduced to {npts} points)",
                           "n_points": npts, "n_flav": int(g.n_flav), "alphas_points": npts, "parallelism": f"replicas x{world}",
                           "l2": "inputs + outputs of a step (1.36 GB) exceed the 129 MB L2"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": 2 * args.steps, "clocks": clk, "alphas": alphas, "forms": forms,
                "sweep": sweep}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
