"""Benchmark of the QUAPI tensor propagator on one GB300 (or N replicas under torchrun).

One bench step = one complete propagation of the large memory-bound spin-boson
workload (M=2, Delta k_max=14: 4^14 = 268,435,456 tensor entries; Ohmic alpha=0.5,
wc=2.5, beta=0.5, dt=0.15, 1000 steps, rho read out at the final step only):
growth phase, 987 fused steady-state steps, the final readout.

Metric: tensor element-updates/s = (M^2)^L logical entries x (N - L + 1)
full-tensor passes / time.  value: FP32 form in the Hermitian half layout,
tables and rho0 resident on the device (quapi_propagate_device); e2e: the
public host API per step (quapi_setup from host arrays + quapi_propagate to
host rho + quapi_destroy).  forms: the full layout, the plain FP64 form (the
baseline the other forms' speedups refer to) and the DF64 form.  roofline:
the dominant kernel (the fused steady-state step) timed alone with CUDA
events on its stream; algorithmic bytes = one read and one write of every
stored entry; traffic = the ncu DRAM bytes per launch recorded in profiles/.
t_terms_per_s = value x M^2 (each output entry sums M^2 terms).  Also in forms:
rho at every step (allPoints) and the 256-instance batched workload.

--impl reference: the FP64 CPU oracle on the host cores, a bounded sample of
the same workload per step (a few steady-state steps on a full-size tensor).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QUAPI tensor element-updates/s (M=2, dkmax=14; FP32 form; FP64 / DF64 forms and full layout in forms)"
UNIT = "element-updates/s"
WORKLOAD = "spin_boson_L14"


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


KERNEL_SOURCES = ("propagate.cu", "half_layout.cuh", "quapi_internal.h")


def kernel_source_sha():
    """sha256[:16] over the step kernels' source files (propagate.cu, half_layout.cuh, quapi_internal.h)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1205_6872_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


DATASHEET_HBM_GBPS = 7900.0  # GB300 HBM3e nominal


def recorded_traffic(kernel_key):
    """Per-launch DRAM bytes from the committed ncu summary, if the kernel sources are unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic_per_launch.txt")
    try:
        sha = kernel_source_sha()
        with open(path) as fh:
            for line in fh:
                parts = line.split()
                if len(parts) >= 3 and not line.startswith("#") and parts[0] == kernel_key:
                    if parts[2] == sha:
                        return float(parts[1])
    except OSError:
        pass
    return None


GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")


def golden_rho(name):
    """rho of the FP64 oracle stored for a workload (tests/golden/<name>.json, written by
    tests/golden/make_golden.py from the oracle alone): {step: M x M complex}, or None if absent."""
    try:
        with open(os.path.join(GOLDEN_DIR, f"{name}.json")) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    out = {}
    for k, v in d["rho"].items():
        a = np.array(v, dtype=np.float64)
        z = a[:, 0] + 1j * a[:, 1]
        m = int(round(len(z) ** 0.5))
        out[int(k)] = z.reshape(m, m)
    return out


def golden_instances(name):
    """Per-instance final rho of a stored batched oracle run (list of M x M complex), or None."""
    try:
        with open(os.path.join(GOLDEN_DIR, f"{name}.json")) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    out = []
    for inst in d["instances"]:
        a = np.array(inst["rho"], dtype=np.float64)
        z = a[:, 0] + 1j * a[:, 1]
        m = int(round(len(z) ** 0.5))
        out.append(z.reshape(m, m))
    return out


def vs_oracle(rho, gold, step):
    """max |rho - rho_oracle| over the entries of rho at one step (None without a stored value)."""
    if gold is None or step not in gold:
        return None
    return float(np.abs(np.asarray(rho).reshape(gold[step].shape) - gold[step]).max())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
            os.unlink(self.path)
        except OSError:
            pass
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons),
                       samples=len(sm))
        return out


def dist_setup():
    from paper_1205_6872_gb300 import replicas
    return replicas.env_ranks()


def barrier(world):
    from paper_1205_6872_gb300 import replicas
    replicas.barrier()


def max_over_ranks(value, world):
    from paper_1205_6872_gb300 import replicas
    return replicas.reduce_max(value)


def element_updates(p):
    return float((p.M * p.M) ** p.L) * float(p.N - p.L + 1)


def tensor_entries(p, half):
    from paper_1205_6872_gb300 import layout
    return layout.count(p.L, p.M) if half else (p.M * p.M) ** p.L


def entry_bytes(q, precision):
    return 8 if precision == q.QUAPI_FP32 else 16


def time_form(q, torch, p, precision, steps, warmup, stream, world, sampler=None, half=False):
    opts = q.quapi_opts_init(precision=precision, cuda_stream=stream, hermitian=int(half))
    ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L, opts)
    try:
        rho0 = torch.tensor(np.asarray(p.rho0).reshape(-1), dtype=torch.complex128, device="cuda")
        rho = torch.empty(p.M * p.M, dtype=torch.complex128, device="cuda")
        with torch.cuda.stream(stream):
            # at least two: the second call with the same arguments captures the propagation graph, so
            # that the timed calls replay it as every later call does
            for _ in range(max(warmup, 2)):
                q.quapi_propagate_device(ctx, rho0, [p.N], rho)
        stream.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        l0 = q.quapi_kernel_launches()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            q.quapi_propagate_device(ctx, rho0, [p.N], rho)
        e1.record(stream)
        e1.synchronize()
        launches = q.quapi_kernel_launches() - l0
        clocks = sampler.stop() if sampler else None
        barrier(world)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        ms = max_over_ranks(ms, world)
        rho_final = rho.cpu().numpy().reshape(p.M, p.M)
        # dominant kernel alone: the fused steady-state step on a full tensor
        n_el = tensor_entries(p, half)
        dt_ = torch.complex64 if precision == 32 else torch.complex128
        gen = torch.Generator(device="cuda").manual_seed(1)
        A = torch.randn(n_el, dtype=dt_, device="cuda", generator=gen)
        B = torch.empty_like(A)
        torch.cuda.synchronize()  # A was filled on torch's current stream
        reps = 20
        with torch.cuda.stream(stream):
            for _ in range(3):
                q.quapi_step_device(ctx, p.L + 1, A, B, None)
        k0 = torch.cuda.Event(enable_timing=True)
        k1 = torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        for r in range(reps):
            src, dst = (A, B) if r % 2 == 0 else (B, A)
            q.quapi_step_device(ctx, p.L + 1, src, dst, None)
        k1.record(stream)
        k1.synchronize()
        kern_ms_direct = k0.elapsed_time(k1) / reps
        # the same launches replayed from a CUDA graph: the kernel's own time without the host's launch
        # sequence between launches (which bounds the small, L2-resident tensors' direct launches)
        kern_ms = kern_ms_direct
        try:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream, capture_error_mode="thread_local"):
                for r in range(reps):
                    src, dst = (A, B) if r % 2 == 0 else (B, A)
                    q.quapi_step_device(ctx, p.L + 1, src, dst, None)
            with torch.cuda.stream(stream):  # replay() launches into the current stream
                for _ in range(2):
                    graph.replay()
                k0.record(stream)
                graph.replay()
                k1.record(stream)
            k1.synchronize()
            kern_ms = k0.elapsed_time(k1) / reps
            del graph
        except Exception as exc:  # capture refused: keep the direct launches' time
            print(f"kernel-alone graph capture failed ({exc}); direct launches timed", file=sys.stderr)
        del A, B
        torch.cuda.empty_cache()
    finally:
        q.quapi_destroy(ctx)
    algo = 2.0 * tensor_entries(p, half) * entry_bytes(q, precision)  # one read and one write per stored entry
    return dict(ms=ms, launches=launches, clocks=clocks, rho=rho_final, kernel_ms=kern_ms, bytes=algo,
                kernel_GBps=algo / (kern_ms / 1e3) / 1e9, kernel_ms_direct=kern_ms_direct)


def time_all_points(q, torch, p, precision, steps, warmup, stream, world, half=True):
    """rho at every step 0..N (the paper's allPoints): the readout is fused into each of the N steps."""
    opts = q.quapi_opts_init(precision=precision, cuda_stream=stream, hermitian=int(half))
    ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L, opts)
    try:
        grid = list(range(p.N + 1))
        rho0 = torch.tensor(np.asarray(p.rho0).reshape(-1), dtype=torch.complex128, device="cuda")
        rho = torch.empty(len(grid) * p.M * p.M, dtype=torch.complex128, device="cuda")
        with torch.cuda.stream(stream):
            for _ in range(max(warmup, 2)):  # the second call captures the propagation graph
                q.quapi_propagate_device(ctx, rho0, grid, rho)
        stream.synchronize()
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            q.quapi_propagate_device(ctx, rho0, grid, rho)
        e1.record(stream)
        e1.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1) / steps, world)
        rhos = rho.cpu().numpy().reshape(len(grid), p.M, p.M)
    finally:
        q.quapi_destroy(ctx)
    return dict(ms=ms, rhos=rhos)


def time_e2e(q, torch, p, precision, steps, warmup, half=False):
    """Public host API per step: setup from host arrays, propagate to host rho, destroy."""
    def one():
        ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L,
                            q.quapi_opts_init(precision=precision, hermitian=int(half)))
        try:
            return q.quapi_propagate(ctx, p.rho0, [p.N], p.M)
        finally:
            q.quapi_destroy(ctx)
    for _ in range(max(1, warmup)):
        one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / steps


def batch_updates(probs):
    return float(sum((p.M * p.M) ** p.L * max(p.N - p.L + 1, 0) for p in probs))


def batch_hbm_bytes(probs, half, entry_bytes=8, resident_bytes=32 * 1024):
    """Algorithmic HBM bytes of one batched run: one read and one write of every stored entry at every
    step (growth and the final readout included) of each instance too large to stay in shared memory."""
    from paper_1205_6872_gb300 import layout as ly
    total = 0
    for p in probs:
        M2 = p.M * p.M
        if 2 * M2 ** p.L * entry_bytes <= resident_bytes:
            continue
        stored = (lambda n: ly.count(n, p.M)) if half else (lambda n: M2 ** n)
        for n in range(1, p.N + 1):
            if n < p.L and n < p.N:
                total += (stored(n) + stored(n + 1)) * entry_bytes
            elif n < p.N:
                total += 2 * stored(p.L) * entry_bytes
            else:
                total += stored(min(n, p.L)) * entry_bytes
    return float(total)


def time_batched(q, torch, steps, warmup, world, rank):
    """256 spin-boson instances: one batched FP32 launch (autotuned, graph replay), with the tiled
    instances in the Hermitian half layout and in the full layout, and one DF64 (FP64-equivalent)
    launch in the half layout, vs the same instances solved one after another with the plain FP64
    propagator.  Under N ranks each rank takes a contiguous shard
    of the instances."""
    from paper_1205_6872_gb300 import replicas
    from paper_1205_6872_gb300 import workloads as wl
    allp = wl.batched_256()
    a, b = replicas.shard(len(allp), rank, world)
    probs = allp[a:b]
    ups = batch_updates(probs)
    rho0s = [p.rho0 for p in probs]
    Ns = [p.N for p in probs]
    batched_s, r32 = {}, {}
    # keys: 1 = FP32 half layout, 0 = FP32 full layout, 2 = DF64 (FP64-equivalent) half layout
    for half in (1, 0, 2):
        prec = q.QUAPI_DF64 if half == 2 else q.QUAPI_FP32
        c32 = [q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L,
                             q.quapi_opts_init(precision=prec, tune=1, hermitian=int(half != 0))) for p in probs]
        try:
            for _ in range(max(warmup, 1)):
                q.quapi_propagate_batch(c32, rho0s, Ns)  # first call tunes and captures the graph
            torch.cuda.synchronize()
            replicas.barrier()
            t0 = time.perf_counter()
            for _ in range(steps):
                r32[half] = q.quapi_propagate_batch(c32, rho0s, Ns)
            batched_s[half] = replicas.reduce_max((time.perf_counter() - t0) / steps)
        finally:
            for c in c32:
                q.quapi_destroy(c)
    c64 = [q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L,
                         q.quapi_opts_init(precision=q.QUAPI_FP64)) for p in probs]
    try:
        rho0 = torch.tensor(np.asarray(probs[0].rho0).reshape(-1), dtype=torch.complex128, device="cuda")
        outs = torch.empty((len(probs), 4), dtype=torch.complex128, device="cuda")
        for _ in range(2):  # a direct call, then the one that captures each instance's propagation graph
            for c, p, i in zip(c64, probs, range(len(probs))):
                q.quapi_propagate_device(c, rho0, [p.N], outs[i])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c, p, i in zip(c64, probs, range(len(probs))):
            q.quapi_propagate_device(c, rho0, [p.N], outs[i])
        torch.cuda.synchronize()
        seq_s = replicas.reduce_max(time.perf_counter() - t0)
        r64 = outs.cpu().numpy().reshape(-1, 2, 2)
    finally:
        for c in c64:
            q.quapi_destroy(c)
    diff = {h: replicas.reduce_max(max(float(np.abs(x - y).max()) for x, y in zip(r32[h], r64))) for h in (0, 1, 2)}
    gold = golden_instances("batched_256")
    if gold is not None:
        gold = gold[a:b]
        vs_or = {h: replicas.reduce_max(max(float(np.abs(x - y).max()) for x, y in zip(r, gold)))
                 for h, r in list(r32.items()) + [("fp64", list(r64))]}
    else:
        vs_or = {h: None for h in (0, 1, 2, "fp64")}
    total = replicas.reduce_sum(ups)
    peak, _ = measured_peaks()
    gbps = {h: replicas.reduce_sum(batch_hbm_bytes(probs, h == 1)) / batched_s[h] / 1e9 for h in (0, 1)}
    return dict(workload="batched_256", instances=len(allp), layout="half (tiled instances)",
                value=total / batched_s[1], unit=UNIT, ms_per_batch=1000.0 * batched_s[1],
                full_layout_value=total / batched_s[0], full_layout_ms_per_batch=1000.0 * batched_s[0],
                sequential_fp64_ms=1000.0 * seq_s, sequential_fp64_value=total / seq_s,
                speedup_vs_sequential_fp64=seq_s / batched_s[1], fp32_vs_fp64_max_abs=diff[1],
                fp32_full_vs_fp64_max_abs=diff[0],
                algorithmic_GBps=gbps[1], frac_of_hbm=gbps[1] / peak,
                full_layout_algorithmic_GBps=gbps[0], full_layout_frac_of_hbm=gbps[0] / peak,
                df64_half_value=total / batched_s[2], df64_half_ms_per_batch=1000.0 * batched_s[2],
                df64_half_speedup_vs_sequential_fp64=seq_s / batched_s[2], df64_half_vs_fp64_max_abs=diff[2],
                max_abs_vs_oracle=dict(fp32_half=vs_or[1], fp32_full=vs_or[0], df64_half=vs_or[2],
                                       sequential_fp64=vs_or["fp64"],
                                       reference="tests/golden/batched_256.json (FP64 oracle, rho at N = 200)"))


def cpu_oracle_sample(p, nsteps):
    """The FP64 oracle's steady-state step on a full-size tensor, nsteps times (host cores)."""
    import oracle
    import oracle.recurrence as rec
    from oracle.eta import Spectral
    from paper_1205_6872_gb300 import workloads as wl
    run = oracle.OracleRun(p.s, p.H, Spectral(p.jkind, p.ja, p.wc), p.beta, p.dt, p.L)
    G, g, n_in, summed = rec.step_tables(run.eta, p.s, run.K, p.L, p.L + 1)
    A = wl.random_tensor((p.M * p.M) ** p.L, seed=11)
    t0 = time.perf_counter()
    for _ in range(nsteps):
        A = rec.apply_step(A, G, g, n_in, summed)
    dt = time.perf_counter() - t0
    return dt


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    from paper_1205_6872_gb300 import workloads as wl
    p = wl.spin_boson_L14()
    per_step = 2  # steady-state steps of the full-size tensor per bench step
    for _ in range(args.warmup):
        cpu_oracle_sample(p, 1)
    t = [cpu_oracle_sample(p, per_step) for _ in range(args.steps)]
    ms = 1000.0 * sum(t) / len(t)
    ups = per_step * float((p.M * p.M) ** p.L) / (ms / 1000.0)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = f"{per_step} steady-state steps of the 4^14-entry tensor per bench step (FP64 oracle, OpenMP)"
    line = dict(metric=METRIC, value=ups, unit=UNIT, n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD, M=p.M, dkmax=p.L, N=p.N, form="fp64 oracle (CPU)", layout="full",
                            readout="justFinalPoint", parallelism="replicas1", sample=sample),
                cpu_baseline=dict(value=ups, unit=UNIT, cores=cores, kind="oracle", sample=sample),
                e2e=dict(value=ups, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))
    return 0


def run_kernel_only(args):
    """The fused steady-state step alone on a workload (--workload) at memory length --dkmax
    (with --with-readout: fused with the rho readout, plus the final rho reduction).

    One device buffer (the context's workspace) holds both tensors; 3 warm-up
    launches, then --reps timed launches.  Used for ncu captures on a small case.
    """
    import torch
    from paper_1205_6872_gb300 import quapi as q
    from paper_1205_6872_gb300 import workloads as wl
    torch.cuda.set_device(0)
    p = wl.CONFIGS[args.workload]()
    L = args.dkmax if args.dkmax else p.L
    prec = {"fp32": q.QUAPI_FP32, "fp64": q.QUAPI_FP64, "df64": q.QUAPI_DF64}[args.form]
    tbytes, _ = q.quapi_query_memory(p.M, L, prec)
    if args.hermitian:
        from paper_1205_6872_gb300 import layout
        tbytes = 2 * layout.count(L, p.M) * (8 if prec == q.QUAPI_FP32 else 16)
    algo_bytes = tbytes  # one read and one write of every stored entry
    tbytes = 2 * (((tbytes // 2) + 255) // 256 * 256)  # the second tensor 256-byte aligned
    ws = torch.empty(tbytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    ctx = q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, L,
                        q.quapi_opts_init(precision=prec, cuda_stream=stream, workspace=ws,
                                          workspace_bytes=tbytes, hermitian=int(args.hermitian)))
    try:
        half = tbytes // 2
        A, B = ws.data_ptr(), ws.data_ptr() + half
        rho = (torch.empty(p.M * p.M, dtype=torch.complex128, device="cuda")
               if (args.with_readout or args.readout_only) else None)
        if args.readout_only:
            B = None
        with torch.cuda.stream(stream):
            ws.view(torch.float32).normal_()
        for _ in range(3):
            q.quapi_step_device(ctx, L + 1, A, B, rho)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for r in range(args.reps):
            src, dst = (A, B) if (r % 2 == 0 or B is None) else (B, A)
            q.quapi_step_device(ctx, L + 1, src, dst, rho)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / args.reps
    finally:
        q.quapi_destroy(ctx)
    gbs = algo_bytes / (ms / 1000.0) / 1e9
    print(json.dumps(dict(mode="kernel-only", workload=args.workload, M=p.M, form=args.form, dkmax=L,
                          hermitian=bool(args.hermitian),
                          with_readout=bool(args.with_readout), readout_only=bool(args.readout_only), kernel_ms=ms,
                          GBps=gbs, logical_updates_per_s=float((p.M * p.M) ** L) / (ms / 1000.0))))
    return 0


def run_batched_only(args):
    """One batched launch (form --form) over --batch-n seeded spin-boson instances (3 warm-up runs,
    then --reps timed runs), optionally in the half layout and autotuned.  Used for ncu captures of the
    batched kernel on a small case."""
    import torch
    from paper_1205_6872_gb300 import quapi as q
    from paper_1205_6872_gb300 import workloads as wl
    torch.cuda.set_device(0)
    probs = wl.batched_256(n=args.batch_n, N=args.batch_steps)
    prec = {"fp32": q.QUAPI_FP32, "fp64": q.QUAPI_FP64, "df64": q.QUAPI_DF64}[args.form]
    opts = q.quapi_opts_init(precision=prec, tune=int(args.tune), hermitian=int(args.hermitian))
    ctxs = [q.quapi_setup(p.s, p.H, p.jkind, p.ja, p.wc, p.beta, p.dt, p.L, opts) for p in probs]
    try:
        rho0s, Ns = [p.rho0 for p in probs], [p.N for p in probs]
        for _ in range(3):
            q.quapi_propagate_batch(ctxs, rho0s, Ns)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.reps):
            q.quapi_propagate_batch(ctxs, rho0s, Ns)
        ms = 1000.0 * (time.perf_counter() - t0) / args.reps
    finally:
        for c in ctxs:
            q.quapi_destroy(c)
    print(json.dumps(dict(mode="batched-only", form=args.form, instances=len(probs), N=args.batch_steps,
                          hermitian=bool(args.hermitian),
                          tune=bool(args.tune), ms_per_batch=ms,
                          value=batch_updates(probs) / (ms / 1e3), unit=UNIT)))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 and DF64 form measurements")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-instance batched measurement")
    ap.add_argument("--kernel-only", action="store_true",
                    help="time only the fused steady-state step kernel (profiling case)")
    ap.add_argument("--dkmax", type=int, default=0, help="memory length for --kernel-only (0: the workload's)")
    ap.add_argument("--workload", default=WORKLOAD, help="workload of --kernel-only (spin_boson_L14, three_level_L8, ...)")
    ap.add_argument("--form", default="fp32", choices=["fp32", "fp64", "df64"],
                    help="form for --kernel-only / --batched-only")
    ap.add_argument("--reps", type=int, default=3, help="timed launches for --kernel-only")
    ap.add_argument("--hermitian", action="store_true", help="--kernel-only / --batched-only: Hermitian half layout")
    ap.add_argument("--readout-only", action="store_true",
                    help="--kernel-only: the rho readout alone (no tensor written; justFinalPoint's last launch)")
    ap.add_argument("--with-readout", action="store_true",
                    help="--kernel-only: the step fused with the rho readout (what allPoints runs at every step)")
    ap.add_argument("--tune", action="store_true", help="--batched-only: autotune the launch shape")
    ap.add_argument("--batched-only", action="store_true",
                    help="time only the batched launch on a seeded batch (profiling case)")
    ap.add_argument("--batch-n", type=int, default=256, help="instances for --batched-only")
    ap.add_argument("--batch-steps", type=int, default=200, help="final step per instance for --batched-only")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel_only:
        return run_kernel_only(args)
    if args.batched_only:
        return run_batched_only(args)

    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1205_6872_gb300 import quapi as q
    from paper_1205_6872_gb300 import workloads as wl
    q.load()
    p = wl.spin_boson_L14()
    stream = torch.cuda.Stream()
    sampler = ClockSampler(local)
    ups = element_updates(p)
    peak, peak_kind = measured_peaks()

    gold = golden_rho(WORKLOAD)

    def form_entry(r, layout_name, ref=None):
        d = dict(value=world * ups / (r["ms"] / 1000.0), unit=UNIT, ms_per_step=r["ms"], layout=layout_name,
                 kernel_ms=r["kernel_ms"], kernel_GBps=r["kernel_GBps"], kernel_frac_of_hbm=r["kernel_GBps"] / peak,
                 kernel_ms_direct_launches=r["kernel_ms_direct"],
                 max_abs_vs_oracle=vs_oracle(r["rho"], gold, p.N),
                 rho_final=[[float(z.real), float(z.imag)] for z in r["rho"].reshape(-1)])
        if ref is not None:
            d["max_abs_vs_fp64_full"] = float(np.abs(r["rho"] - ref["rho"]).max())
        return d

    # headline: FP32 form, Hermitian half layout (the fastest configuration for a Hermitian rho0)
    r32h = time_form(q, torch, p, q.QUAPI_FP32, args.steps, args.warmup, stream, world, sampler, half=True)
    value = world * ups / (r32h["ms"] / 1000.0)
    forms = {"fp32_half": form_entry(r32h, "half")}
    r32f = time_form(q, torch, p, q.QUAPI_FP32, args.steps, args.warmup, stream, world, half=False)
    forms["fp32_full"] = form_entry(r32f, "full")
    if not args.no_fp64:
        r64f = time_form(q, torch, p, q.QUAPI_FP64, args.steps, args.warmup, stream, world, half=False)
        forms["fp64_full"] = form_entry(r64f, "full")
        forms["fp64_full"]["bound"] = "alu (FP64 pipe saturated; DFMA 1.2 TFLOP/s on this part)"
        r64h = time_form(q, torch, p, q.QUAPI_FP64, args.steps, args.warmup, stream, world, half=True)
        forms["fp64_half"] = form_entry(r64h, "half", r64f)
        rdff = time_form(q, torch, p, q.QUAPI_DF64, args.steps, args.warmup, stream, world, half=False)
        forms["df64_full"] = form_entry(rdff, "full", r64f)
        rdfh = time_form(q, torch, p, q.QUAPI_DF64, args.steps, args.warmup, stream, world, half=True)
        forms["df64_half"] = form_entry(rdfh, "half", r64f)
        forms["fp32_full"]["max_abs_vs_fp64_full"] = float(np.abs(r32f["rho"] - r64f["rho"]).max())
        forms["speedups_over_plain_fp64"] = dict(
            fp32_half=r64f["ms"] / r32h["ms"], fp32_full=r64f["ms"] / r32f["ms"],
            df64_half=r64f["ms"] / rdfh["ms"], df64_full=r64f["ms"] / rdff["ms"], fp64_half=r64f["ms"] / r64h["ms"])
        headline_vs_fp64 = float(np.abs(r32h["rho"] - r64f["rho"]).max())
    else:
        headline_vs_fp64 = None
    # the other workloads: one propagation each, the plain FP64 form and the FP32 form (half layout where
    # M = 2), with the FP32 form's speedup over plain FP64 and its max abs difference on the final rho
    if not args.no_fp64:
        others = (("spin_boson_L6", wl.spin_boson_L6()), ("biased_L12", wl.biased_L12()),
                  ("three_level_L8", wl.three_level_L8()), ("quantum_dot_L11", wl.quantum_dot()))
        for name, po in others:
            half = True  # every workload's rho0 is Hermitian (M = 2 and M = 3)
            r64o = time_form(q, torch, po, q.QUAPI_FP64, 1, 1, stream, world, half=False)
            r32o = time_form(q, torch, po, q.QUAPI_FP32, 1, 1, stream, world, half=half)
            for tag, r in (("fp64_full", r64o), ("fp32_half" if half else "fp32_full", r32o)):
                forms[f"{name}_{tag}"] = dict(
                    value=world * element_updates(po) / (r["ms"] / 1000.0), unit=UNIT, ms_per_step=r["ms"],
                    layout="half" if (half and tag.startswith("fp32")) else "full", M=po.M, dkmax=po.L, N=po.N,
                    kernel_ms=r["kernel_ms"], kernel_GBps=r["kernel_GBps"], kernel_frac_of_hbm=r["kernel_GBps"] / peak,
                    kernel_ms_direct_launches=r["kernel_ms_direct"])
            forms[f"{name}_fp32_speedup_over_fp64"] = r64o["ms"] / r32o["ms"]
            forms[f"{name}_fp32_vs_fp64_max_abs"] = float(np.abs(r32o["rho"] - r64o["rho"]).max())
            go = golden_rho(name)
            forms[f"{name}_fp64_full"]["max_abs_vs_oracle"] = vs_oracle(r64o["rho"], go, po.N)
            forms[f"{name}_{'fp32_half' if half else 'fp32_full'}"]["max_abs_vs_oracle"] = vs_oracle(r32o["rho"], go, po.N)
    rap = time_all_points(q, torch, p, q.QUAPI_FP32, args.steps, args.warmup, stream, world, half=True)
    forms["fp32_half_all_points"] = dict(
        value=world * ups / (rap["ms"] / 1000.0), unit=UNIT, ms_per_step=rap["ms"], layout="half",
        readout=f"allPoints: rho at all {p.N + 1} steps (readout fused into every step)",
        rho_final_vs_just_final_point=float(np.abs(rap["rhos"][-1] - r32h["rho"]).max()),
        max_abs_vs_oracle=(max(vs_oracle(rap["rhos"][k], gold, k) for k in gold) if gold else None),
        oracle_steps_compared=(len(gold) if gold else 0),
        max_trace_deviation=float(np.abs(np.trace(rap["rhos"], axis1=1, axis2=2) - 1.0).max()))
    if not args.no_batched:
        forms["batched_256_fp32"] = time_batched(q, torch, args.steps, args.warmup, world, rank)
    e2e_s = time_e2e(q, torch, p, q.QUAPI_FP32, args.steps, min(args.warmup, 1), half=True)
    e2e_s = max_over_ranks(e2e_s, world)
    achieved = r32h["kernel_GBps"]
    traffic = recorded_traffic("herm_step_kernel_fp32_m2")
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=r32h["ms"], higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
        data="synthetic",
        config=dict(workload=WORKLOAD, M=p.M, dkmax=p.L, N=p.N, form="fp32", layout="hermitian half",
                    readout="justFinalPoint", parallelism=f"replicas{world}",
                    l2="inputs larger than L2: each step streams two 1.07 GB tensors"),
        roofline=dict(bound="hbm", achieved=achieved, peak=peak, unit="GB/s", frac=achieved / peak,
                      traffic=traffic, peak_source=peak_kind, kernel="herm_step_kernel<FP32> (half layout)",
                      kernel_ms=r32h["kernel_ms"], algorithmic_bytes_per_launch=r32h["bytes"],
                      traffic_GBps=(traffic / (r32h["kernel_ms"] / 1e3) / 1e9) if traffic else None,
                      frac_of_datasheet=achieved / DATASHEET_HBM_GBPS),
        t_terms_per_s=value * p.M * p.M,
        e2e=dict(value=world * ups / e2e_s, unit=UNIT, seconds_per_step=e2e_s,
                 h2d_bytes_per_step=8 * p.M + 16 * p.M * p.M * 2, d2h_bytes_per_step=16 * p.M * p.M),
        gpu_launches=int(r32h["launches"]),
        clocks=r32h["clocks"],
        max_abs_vs_fp64_full=headline_vs_fp64,
        max_abs_vs_oracle=vs_oracle(r32h["rho"], gold, p.N),
        oracle_reference=f"tests/golden/{WORKLOAD}.json: FP64 oracle rho at N = {p.N} (written by make_golden.py)",
        forms=forms,
        paper_context=dict(
            note="the paper's own MATLAB timings on other hardware: context, not a baseline for this workload",
            hardware="Intel Xeon Nehalem 2.8 GHz CPU / Nvidia C2020 (Fermi) GPU, MATLAB, FP64",
            table1_dkmax11_gpu_s=21.130031, table1_dkmax11_cpu_s=1198.620937,
            derived_gpu_element_updates_per_s=0.196e9,
            derivation="4^11 entries x 989 steady steps / 21.13 s, assuming Table 1 used the profiled 989-step run"),
        rho_final=[[float(z.real), float(z.imag)] for z in r32h["rho"].reshape(-1)],
    )
    if not args.no_fp64:
        # the same roofline for the FP64-accuracy form (DF64, half layout): the paper's precision
        ach = rdfh["kernel_GBps"]
        tr = recorded_traffic("herm_step_kernel_df64_m2")
        line["roofline_fp64_equiv"] = dict(
            bound="hbm", achieved=ach, peak=peak, unit="GB/s", frac=ach / peak, traffic=tr, peak_source=peak_kind,
            kernel="herm_step_kernel<DF64> (half layout)", kernel_ms=rdfh["kernel_ms"],
            algorithmic_bytes_per_launch=rdfh["bytes"], form="df64", dtype="f32x2 (double-float, FP64-equivalent)",
            value=world * ups / (rdfh["ms"] / 1000.0), ms_per_step=rdfh["ms"],
            max_abs_vs_oracle=vs_oracle(rdfh["rho"], gold, p.N))
    if rank == 0 and world == 1 and not args.no_cpu:
        from oracle import clib
        nst = 2
        t = cpu_oracle_sample(p, nst)
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        line["cpu_baseline"] = dict(value=nst * float((p.M * p.M) ** p.L) / t, unit=UNIT, cores=cores,
                                    kind="oracle",
                                    sample=f"{nst} steady-state steps of the 4^14-entry tensor (FP64 oracle)")
        # the same oracle on one core (one steady-state step)
        clib.set_threads(1)
        try:
            t1 = cpu_oracle_sample(p, 1)
        finally:
            clib.set_threads(cores)
        line["cpu_baseline"]["single_core"] = dict(
            value=float((p.M * p.M) ** p.L) / t1, unit=UNIT, cores=1,
            sample="1 steady-state step of the 4^14-entry tensor (FP64 oracle)")
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
