"""Benchmark: FDTD Gcell-updates/s of the single large lossy line (768x384x256 cells of
20 nm, FP32 fields, 12-cell PML, two ports with 128-frequency running DFTs).

One bench step = `--chunk` FDTD time steps of the whole hot path (H update, E update with
materials and CPML, soft source, port V/I integrals, running DFTs), replayed from captured
CUDA graphs.  Inputs (1.8 GB of fields) are far larger than the 126 MB L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank advances its own replica of the line (the single grid is not
decomposed across GPUs): value = all ranks' cell updates / max rank time, scaling "weak".
The reference arm times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FDTD Gcell-updates/s & %HBM roofline; batched S-param solves/s vs surrogate"
UNIT = "Gcell-updates/s"
BYTES_PER_CELL_FP32 = 51.0   # 6 components read + written once (48 B) + 3 edge-class bytes


def workload(nz: int = 256):
    """The lossy line; a smaller nz (same stack, fewer planes of air) is only for profiling
    captures that must stay small."""
    from paper_2208_04371_b300 import workloads as W
    return W.config_lossy_line(nz=nz, nsteps=0)


def stencil_traffic(kernel: str):
    """DRAM bytes per launch of the dominant stencil kernel from the committed ncu capture
    (k_yee_tb2: one two-step launch; k_yee_tma_batch: all work kinds of one step), or None
    when the kernel's source has changed since the counters were taken."""
    import hashlib
    name = {"k_yee_tb2": "k_yee_tb2_traffic_lossy_line_768x384x256.json",
            "k_yee_tma_batch": "k_yee_tma_batch_traffic_lossy_line_768x384x256.json"}.get(kernel)
    path = os.path.join(ROOT, "profiles", name) if name else ""
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    for rel, digest in d["source_sha256"].items():
        f = os.path.join(ROOT, rel)
        if not os.path.exists(f) or hashlib.sha256(open(f, "rb").read()).hexdigest() != digest:
            return None
    return d["dram_bytes_per_launch"] if "dram_bytes_per_launch" in d else d["dram_bytes_per_step"]


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d["hbm_gbs"], "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int, directory: str = ""):
        self.dev = device_index
        self.proc = None
        # the raw samples (the JSON line carries their summary); --clocks-dir keeps them
        self.path = os.path.join(directory or tempfile.gettempdir(), f"yf_bench_clocks_rank{device_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


ORACLE_BYTES_PER_POINT = 27 * 8 + 3   # the oracle's full-size arrays: fields, coefficients, psi


def oracle_workload(force_slice: bool = False):
    """The lossy line itself when the host can hold the oracle's full-size arrays (about
    16.4 GB at 768x384x256), else (or when asked) a named 256x128x256 slice with the same
    cell stack."""
    p = workload()
    need = (p.nx + 1) * (p.ny + 1) * (p.nz + 1) * ORACLE_BYTES_PER_POINT
    if force_slice:
        need = float("inf")
    try:
        import psutil
        avail = psutil.virtual_memory().available
    except Exception:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    if avail > 1.3 * need:
        return p, False
    from paper_2208_04371_b300 import workloads as W
    return W.config_lossy_line(nx=256, ny=128, nz=256, nsteps=0), True


class OracleSampler:
    """The FP64 oracle held open on the lossy line (set-up done once, outside every timer);
    each `sample()` times the next few oracle steps alone, about `target_s` seconds."""

    def __init__(self, target_s: float, force_slice: bool = False):
        from oracle import yee
        self.p, self.sliced = oracle_workload(force_slice)
        self.threads = os.cpu_count() or 1
        self.st = yee.Stepper(self.p, threads=self.threads)
        per = self.st.advance(1)                    # first step: page faults, caches
        per = self.st.advance(1)
        self.nsteps = int(max(2, min(200, round(target_s / max(per, 1e-4)))))

    def sample(self):
        """(Gcell/s, seconds) of the next nsteps steps on all host cores."""
        sec = self.st.advance(self.nsteps, threads=self.threads)
        return self.p.cells * self.nsteps / sec / 1e9, sec

    def single_thread(self):
        sec = self.st.advance(1, threads=1)
        self.st.lib.oracle_set_threads(self.threads)
        return self.p.cells / sec / 1e9

    def desc(self):
        where = (f"a {self.p.nx}x{self.p.ny}x{self.p.nz} slice of the lossy-line stack"
                 ) if self.sliced else f"the {self.p.name}"
        return (f"FP64 oracle on {where}, {self.nsteps} steps per sample, stepping alone timed "
                f"(allocation and coefficient / CPML set-up outside the timer), OpenMP over "
                f"k-planes on {self.threads} threads")

    def close(self):
        self.st.close()


def cpu_oracle_sample(target_s: float = 5.0, samples: int = 3):
    """The cpu_baseline leg: the median of `samples` samples of about target_s seconds each
    (the host's cores may be shared, so single samples scatter), plus one single-thread step.
    Returns (Gcell/s, threads, description, single-thread Gcell/s)."""
    s = OracleSampler(target_s)
    try:
        rates = [s.sample()[0] for _ in range(samples)]
        rate1 = s.single_thread()
        rate = float(np.median(rates))
        return rate, s.threads, (s.desc() + f"; median of {samples} samples (spread "
                                 f"{min(rates):.3f}-{max(rates):.3f}); single thread "
                                 f"{rate1:.4f} Gcell/s (1 step)"), rate1
    finally:
        s.close()


def oracle_mlp_rate() -> float:
    """Queries/s of the FP64 MLP oracle's forward (numpy) for the 4-member ensemble on 1024
    queries of the surrogate's input distribution, best of two (the first warms the BLAS)."""
    import time as _t
    from oracle import mlp as omlp
    from paper_2208_04371_b300 import workloads as W
    from paper_2208_04371_b300 import yf
    params = [yf.mlp_unflatten(W.mlp_init(0x5EED + 7919 * e)) for e in range(4)]
    xs = W.surrogate_inputs(W.SplitMix64(0x51), 1024)
    lo, hi = np.array(W.SURROGATE_LO), np.array(W.SURROGATE_HI)
    xm = (xs - lo) * (2.0 / (hi - lo)) - 1.0
    best = 0.0
    for _ in range(2):
        t0 = _t.perf_counter()
        for prm in params:
            omlp.forward(prm, xm)
        best = max(best, 1024 / (_t.perf_counter() - t0))
    return best


def cpu_baseline_table() -> dict:
    """The cpu_baseline leg for every workload (the bench line carries the lossy line's): the
    FP64 oracle on the host's cores and on one thread, each beside the GPU figure it sets off.
    C1 the 64x32x24 FP64 microstrip in full (2000 steps); C3 every 32nd instance of the
    batched sweep (8 of 256), stepping alone timed and extrapolated to solves/s per cell update;
    C4 the 256x128x128 long-run line on a bounded subrun; C5 the FP64 MLP forward of the
    4-member ensemble on 1024 queries (numpy, its BLAS on all threads, then one).  GPU figures:
    C1 and C4 timed here through the library; C3 and C5 are the bench line's batched and
    surrogate legs."""
    import subprocess
    import sys
    import torch
    from oracle import yee
    from paper_2208_04371_b300 import workloads as W
    from paper_2208_04371_b300 import yf
    threads = os.cpu_count() or 1

    def oracle_rate(probs, nsteps, nsteps1):
        cells = sec = cells1 = sec1 = 0.0
        for p in probs:
            with yee.Stepper(p, threads=threads) as st:
                st.advance(1)                       # first touch of the arrays
                sec += st.advance(nsteps, threads=threads)
                sec1 += st.advance(nsteps1, threads=1)
            cells += p.cells * nsteps
            cells1 += p.cells * nsteps1
        return cells / sec / 1e9, cells1 / sec1 / 1e9, sec + sec1

    def gpu_rate(p, prec, nsteps):
        s = torch.cuda.Stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with yf.Grid(p, prec=prec, stream=s.cuda_stream) as g:
            g.step(64)
            g.sync()
            e0.record(s)
            g.step(nsteps)
            e1.record(s)
            e1.synchronize()
            g.sync()
        return p.cells * nsteps / (e0.elapsed_time(e1) / 1e3) / 1e9

    out = {"threads": threads, "kind": "oracle"}
    p1 = W.config_small_fp64()
    a, one, sec = oracle_rate([p1], p1.nsteps, p1.nsteps)
    out["C1 FP64 microstrip 64x32x24, 2000 steps"] = {
        "oracle_gcell_s": a, "oracle_single_thread_gcell_s": one, "oracle_seconds": sec,
        "gpu_gcell_s": gpu_rate(p1, yf.FP64, p1.nsteps)}
    probs = W.config_batched()
    sub = probs[::32]
    a, one, sec = oracle_rate(sub, 40, 4)
    mean_cells = float(np.mean([p.cells for p in probs]))
    out["C3 batched sweep, 8 of 256 instances sampled"] = {
        "oracle_gcell_s": a, "oracle_single_thread_gcell_s": one, "oracle_seconds": sec,
        "oracle_solves_per_s": a * 1e9 / (mean_cells * probs[0].nsteps),
        "steps_sampled": 40, "gpu": "the bench line's batched leg"}
    p4 = W.config_long_run(nsteps=0)
    a, one, sec = oracle_rate([p4], 200, 20)
    out["C4 long-run line 256x128x128, 200-step subrun"] = {
        "oracle_gcell_s": a, "oracle_single_thread_gcell_s": one, "oracle_seconds": sec,
        "gpu_gcell_s": gpu_rate(p4, yf.FP32, 2000)}
    qa = oracle_mlp_rate()
    # one BLAS thread: the same forward in a child process started with one thread
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-mlp-rate"], env=env,
                       capture_output=True, text=True, check=True)
    q1 = float(r.stdout.strip().splitlines()[-1])
    out["C5 surrogate ensemble, 1024 queries"] = {
        "oracle_queries_per_s": qa, "oracle_single_thread_queries_per_s": q1,
        "gpu": "the bench line's surrogate leg"}
    return out


def run_reference(args, rank, world):
    """The oracle arm: rank 0 times the FP64 CPU oracle; other ranks exit without work.
    One bench step is one bounded sample of oracle steps on the same line, so that the whole
    --steps K --warmup W run stays within a few minutes."""
    if rank != 0:
        return
    per_sample = max(2.0, min(args.ref_seconds, 150.0 / max(args.steps + args.warmup, 1)))
    s = OracleSampler(per_sample, force_slice=args.oracle_slice)
    try:
        for _ in range(args.warmup):
            s.sample()
        rates, secs = [], []
        for _ in range(args.steps):
            r, sec = s.sample()
            rates.append(r)
            secs.append(sec)
        desc = s.desc()
        p, nsteps, threads = s.p, s.nsteps, s.threads
    finally:
        s.close()
    # the median sample: the host's cores may be shared with other work, which scatters
    # single samples; the cpu_baseline leg of the GPU arm takes the same median
    value = float(np.median(rates))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": p.cells * nsteps / (value * 1e9) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": p.name, "cells": p.cells,
                                        "steps_per_bench_step": nsteps,
                                        "l2": "inputs larger than L2 (host memory)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": desc + f"; median of {len(rates)} samples (spread "
                                          f"{min(rates):.3f}-{max(rates):.3f})"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batched_leg(stream, steps: int = 64, accuracy: bool = True) -> dict:
    """256 uneven microstrip instances (64-192 cells per axis, 8-cell PML, 20000 steps,
    64 frequencies) advanced together by the batched solver (variant 4: two steps per pass
    over each instance's inner box, the frames one), against the same instances solved one at
    a time by the single-grid solver.  Both FP32 fields with FP64 spectra; each batched
    instance equals its single-grid variant-4 run bit for bit.  Solves/s extrapolates the timed
    steps to the 20000 steps of one solve."""
    import torch
    from paper_2208_04371_b300 import workloads as W
    from paper_2208_04371_b300 import yf
    probs = W.config_batched()
    nsolve = probs[0].nsteps
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with yf.Batch(probs, prec=yf.FP32, stream=stream.cuda_stream, variant=4) as b:
        tile = b.autotune(None, reps=2)
        b.step(32)
        b.sync()
        e0.record(stream)
        b.step(steps)
        e1.record(stream)
        e1.synchronize()
        ms_b = e0.elapsed_time(e1) / steps
        cells = b.cells
    ms_single = 0.0
    for p in probs:
        with yf.Grid(p, prec=yf.FP32, stream=stream.cuda_stream) as g:
            g.step(32)
            g.sync()
            e0.record(stream)
            g.step(steps)
            e1.record(stream)
            e1.synchronize()
            ms_single += e0.elapsed_time(e1) / steps
    return {"workload": f"{len(probs)} uneven microstrip instances, {nsolve} steps each",
            "cells": cells, "variant": 4, "tile_y_kseg": list(tile),
            "ms_per_step": ms_b, "gcell_s": cells / (ms_b / 1e3) / 1e9,
            "solves_per_s": len(probs) / (ms_b * nsolve / 1e3),
            "single_instance_solves_per_s": len(probs) / (ms_single * nsolve / 1e3),
            "single_instance_gcell_s": cells / (ms_single / 1e3) / 1e9,
            "accuracy": batched_accuracy(stream, probs) if accuracy else None}


def batched_steps(stream, variant: int, steps: int) -> dict:
    """The batched sweep's stepping alone (for launch lists): the 256 instances at tiling 8 x 32,
    two untimed steps, then `steps` timed steps."""
    import torch
    from paper_2208_04371_b300 import workloads as W
    from paper_2208_04371_b300 import yf
    probs = W.config_batched()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with yf.Batch(probs, prec=yf.FP32, stream=stream.cuda_stream, tile_y=8, kseg=32, variant=variant) as b:
        b.step(2)
        b.sync()
        e0.record(stream)
        b.step(steps)
        e1.record(stream)
        e1.synchronize()
        b.sync()
        ms = e0.elapsed_time(e1) / max(1, steps)
        return {"variant": variant, "steps": steps, "ms_per_step": ms, "gcell_s": b.cells / (ms / 1e3) / 1e9}


def batched_accuracy(stream, probs, stride: int = 32) -> dict:
    """Measured accuracy of the batched FP32 solves: every `stride`-th instance of the sweep
    (8 of 256, seeded sizes) solved for its full step count twice by the batched solver,
    with FP32 fields on the timed path (variant 4) and with FP64 fields (one step per pass;
    FP64 spectra both times), and the 50-ohm S and the power-mode S* compared:
    max |S_ij(FP32) - S_ij(FP64)| over ports and frequencies."""
    import time as _t
    from paper_2208_04371_b300 import yf
    idx = list(range(0, len(probs), stride))
    sub = [probs[i] for i in idx]
    nsolve = sub[0].nsteps
    res = {}
    t0 = _t.perf_counter()
    for prec in (yf.FP32, yf.FP64):
        with yf.Batch(sub, prec=prec, stream=stream.cuda_stream, variant=4 if prec == yf.FP32 else 2) as b:
            b.step(nsolve)
            b.sync()
            res[prec] = [b.sparams(q) for q in range(len(sub))]
    dS = [float(np.max(np.abs(a["S"] - c["S"]))) for a, c in zip(res[yf.FP32], res[yf.FP64])]
    dSs = [float(np.max(np.abs(a["S_star"] - c["S_star"])))
           for a, c in zip(res[yf.FP32], res[yf.FP64])]
    return {"instances": idx, "cells": [p.cells for p in sub], "steps": nsolve,
            "reference": "the same instances, batched solver with FP64 fields",
            "max_abs_dS": max(dS), "max_abs_dS_star": max(dSs), "per_instance_dS": dS,
            "budget": 1e-3, "seconds": _t.perf_counter() - t0}


def surrogate_leg(stream, n: int = 65536, members: int = 4, reps: int = 20) -> dict:
    """Surrogate ensemble inference: `members` networks (6 -> 4 x 512 GELU -> 512, BF16
    tcgen05 GEMMs, FP32 accumulation) on a batch of n seeded line descriptors, ensemble mean,
    disagreement and gate.  Timed with CUDA events on the library's stream; inputs resident."""
    import torch
    from paper_2208_04371_b300 import workloads as W
    from paper_2208_04371_b300 import yf
    m = yf.Mlp(members, 512, n, W.SURROGATE_LO, W.SURROGATE_HI, stream=stream.cuda_stream)
    try:
        for e in range(members):
            m.set_params(e, W.mlp_init(0x5EED + 7919 * e))
        xh = np.stack([W.uniform_array(0x51 + k, n, lo, hi) for k, (lo, hi) in
                       enumerate(zip(W.SURROGATE_LO, W.SURROGATE_HI))], axis=1).astype(np.float32)
        x = torch.from_numpy(xh).cuda()
        y = torch.empty((n, yf.MLP_OUT), dtype=torch.float32, device="cuda")
        est = torch.empty(n, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        for _ in range(3):
            m.query(x, y, est)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            m.query(x, y, est)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        launches, flops_per_query = m.query_stats()
        # training throughput: graph-replayed Adam steps of member 0 at the handle's batch (512)
        nt, steps = 16384, 200
        g = torch.Generator(device="cpu").manual_seed(11)
        xt = torch.from_numpy(xh[:nt]).cuda()
        tt = (torch.rand((nt, yf.MLP_OUT), generator=g) * 2 - 1).cuda()
        idx = torch.randint(0, nt, (steps * m.batch,), generator=g, dtype=torch.int32).cuda()
        lr = torch.full((steps,), 1e-4, dtype=torch.float32).cuda()
        m.fit(0, xt, tt, idx, lr, 10)
        m.sync()
        e0.record(stream)
        m.fit(0, xt, tt, idx, lr, steps)
        e1.record(stream)
        e1.synchronize()
        m.sync()
        train_samples_s = steps * m.batch / (e0.elapsed_time(e1) / 1e3)
    finally:
        m.close()
    tflops = flops_per_query * n / (ms / 1e3) / 1e12
    pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops": 1800.0}
    # comparison only: torch.matmul BF16 on one hidden layer's shape, same box and stream
    with torch.cuda.stream(stream):
        a = torch.randn((n, 512), device="cuda").to(torch.bfloat16)
        w = torch.randn((512, 512), device="cuda").to(torch.bfloat16)
        for _ in range(3):
            torch.matmul(a, w.t())
        e0.record(stream)
        for _ in range(50):
            torch.matmul(a, w.t())
        e1.record(stream)
        e1.synchronize()
    mm_tflops = 2.0 * n * 512 * 512 * 50 / (e0.elapsed_time(e1) / 1e3) / 1e12
    return {"workload": f"{members}-member ensemble, {n} queries per batch",
            "queries_per_s": n / (ms / 1e3), "ms_per_batch": ms, "launches_per_batch": launches,
            "gemm_tflops": tflops, "bf16_peak_tflops": pk["bf16_tflops"],
            "frac_of_bf16_peak": tflops / pk["bf16_tflops"],
            "training_samples_per_s": train_samples_s,
            "torch_matmul_bf16_tflops_same_layer_shape": mm_tflops}


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2208_04371_b300 import yf
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod

    def barrier():
        if dist is not None:
            dist.barrier()

    p = workload(args.nz)
    stream = torch.cuda.Stream()
    kseg = args.kseg or (32 if args.variant == 4 else 16)
    g = yf.Grid(p, prec=yf.FP32, stream=stream.cuda_stream, variant=args.variant, kseg=kseg,
                box_seg=args.box_seg if args.variant == 4 else 0,
                box_ty=args.box_ty if args.variant == 4 else 0)
    chunk = args.chunk
    launches_per_bench_step = yf.launches(g.h, chunk)
    box = yf.tb_box(g.h) if args.variant == 4 else None
    for _ in range(args.warmup):
        g.step(chunk)
    g.sync()

    sampler = ClockSampler(local_rank, args.clocks_dir)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        g.step(chunk)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    g.sync()
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    cell_updates = p.cells * chunk * args.steps * world
    value = cell_updates / (ms / 1e3) / 1e9
    per_gpu_value = value / world

    # per-kernel durations (CUDA events around every launch, same stream, right after the
    # timed region) for the roofline of the stencil
    prof = yf.profile_steps(g.h, chunk)
    peak, peak_kind = peaks()

    def kname_for(variant, prof):
        return "k_yee_tb2" if variant == 4 else "k_yee_tma_batch"
    traffic = stencil_traffic(kname_for(args.variant, prof)) if args.nz == 256 else None
    if args.variant == 4:
        # the two-step box kernel: each launch advances every box node two time steps, so on
        # the per-cell-update basis (51 B per cell update) it does 2 x 51 B of algorithmic work
        # per node; a one-pass kernel's figure (51 B per node per launch) is kept beside it
        kname = "k_yee_tb2"
        nodes = (box[1] - box[0] + 1) * (box[3] - box[2] + 1) * (box[5] - box[4] + 1) if box else 0
        updates = 2 * nodes
        unit_note = "bytes per launch (two time steps of the inner box)"
    else:
        fused = [k for k in prof if k.startswith("k_yee_")]
        kname = fused[0] if fused else "k_update_h + k_update_e"
        nodes = p.cells
        updates = p.cells
        unit_note = "bytes per step (all work kinds)"
    stencil_ms = prof[kname] if kname in prof else prof["k_update_h"] + prof["k_update_e"]
    algo = BYTES_PER_CELL_FP32 * updates
    achieved = algo / (stencil_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": kname,
            "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
            "frac": achieved / peak,
            "basis": "51 B per cell update x cell updates per launch "
                     f"({updates} = {updates // max(nodes, 1)} x {nodes} nodes)",
            "traffic": traffic,
            "traffic_unit": unit_note,
            "algorithmic_bytes": algo,
            "bytes_per_cell_update": BYTES_PER_CELL_FP32,
            "kernel_ms_per_launch": stencil_ms,
            "kernel_ms": prof}
    if args.variant == 4:
        # the same launch counted as one pass over the box (51 B per node): what a kernel
        # that does not block in time could reach at most
        roof["one_pass"] = {"achieved": BYTES_PER_CELL_FP32 * nodes / (stencil_ms / 1e3) / 1e9,
                            "frac": BYTES_PER_CELL_FP32 * nodes / (stencil_ms / 1e3) / 1e9 / peak}
    if traffic:
        # the DRAM bytes the launch actually moved (committed ncu capture) per its live time
        roof["dram"] = {"achieved": traffic / (stencil_ms / 1e3) / 1e9,
                        "frac": traffic / (stencil_ms / 1e3) / 1e9 / peak}
    # whole-step rate on the 51 B basis: two time steps per HBM pass on the inner box, one on
    # the frame, so this effective fraction may exceed what a one-pass kernel can reach
    roof["effective"] = {"T": "2 on the inner box, 1 on the frame" if args.variant == 4 else "1",
                         "box_fraction_of_nodes": (nodes / ((p.nx + 1) * (p.ny + 1) * (p.nz + 1)))
                         if args.variant == 4 else 0.0,
                         "achieved": BYTES_PER_CELL_FP32 * per_gpu_value,
                         "frac": BYTES_PER_CELL_FP32 * per_gpu_value / peak}

    # end to end through the public API: new geometry from pinned host memory every step
    # (yf_reset + yf_set_materials), the chunk of steps, and the port spectra read back
    e2e = None
    if not args.no_e2e:
        ids_host = torch.from_numpy(p.ids).pin_memory()
        e2e_ms = []
        nf = len(p.freqs)
        for it in range(max(3, args.steps // 4) + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            yf.reset(g.h)
            yf.set_materials(g.h, ids_host, p.eps_r, p.sigma, p.mu_r, p.is_pec)
            g.step(chunk)
            V, I = yf.read_port_dft(g.h, 0, nf)
            V2, I2 = yf.read_port_dft(g.h, 1, nf)
            if it > 0:
                e2e_ms.append((time.perf_counter() - t0) * 1e3)
        e2e = {"value": p.cells * chunk * world / (np.median(e2e_ms) / 1e3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(p.ids.nbytes), "d2h_bytes_per_step": int(2 * 4 * nf * 8)}
    g.close()

    batched = None if args.no_batched else batched_leg(stream, accuracy=not args.no_accuracy)
    sur = None if args.no_surrogate else surrogate_leg(stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, threads, desc, r1 = cpu_oracle_sample()
        cpu = {"value": r, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc,
               "single_thread_value": r1}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": p.name, "cells": p.cells, "steps_per_bench_step": chunk,
                       "variant": args.variant, "tile_y": 8, "kseg": kseg,
                       "box_seg": (args.box_seg or 2 * kseg) if args.variant == 4 else None,
                       "box_tile_y": args.box_ty if args.variant == 4 else None,
                       "inner_box": box,
                       "l2": "inputs larger than L2 (1.8 GB of fields)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches_per_bench_step * args.steps,
            "clocks": clocks,
            "batched": batched,
            "surrogate": sur,
        }
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--chunk", type=int, default=64)
    ap.add_argument("--variant", type=int, default=4, choices=[2, 4],
                    help="stencil variant: 4 two-step inner box (default), 2 one step per pass")
    ap.add_argument("--kseg", type=int, default=0,
                    help="z-planes per one-step block (0: 32 for variant 4, 16 for variant 2)")
    ap.add_argument("--box-seg", type=int, default=-1,
                    help="variant 4: z-planes per two-step block (0: twice kseg; default nz: the box in one segment per tile column)")
    ap.add_argument("--box-ty", type=int, default=8, choices=[8, 16],
                    help="variant 4: y rows per two-step block (16: one block per SM)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the batched leg's FP32-vs-FP64 accuracy solves")
    ap.add_argument("--surrogate-only", action="store_true",
                    help="only the surrogate inference leg (profiling captures)")
    ap.add_argument("--oracle-mlp-rate", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-table", action="store_true",
                    help="only the cpu_baseline leg for every workload (FP64 oracle beside the GPU figures)")
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched sweep's stepping, tiling 8 x 32, --steps steps after 2 (profiling captures)")
    ap.add_argument("--batch-variant", type=int, default=4, choices=[2, 4],
                    help="with --batched-only: 4 two steps per pass over each instance's box, 2 one step")
    ap.add_argument("--nz", type=int, default=256,
                    help="planes of the lossy line (profiling captures only; the bench line is nz=256)")
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--oracle-slice", action="store_true",
                    help="time the oracle on a 256x128x256 slice of the line (quick checks)")
    ap.add_argument("--clocks-dir", default="",
                    help="directory for the raw nvidia-smi clock samples (default: the system temp directory)")
    args = ap.parse_args()
    if args.box_seg < 0:
        args.box_seg = args.nz   # at least the box's depth: one segment per tile column
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.surrogate_only:
        import torch
        torch.cuda.set_device(local_rank)
        print(json.dumps({"surrogate": surrogate_leg(torch.cuda.Stream())}), flush=True)
        return
    if args.oracle_mlp_rate:
        print(oracle_mlp_rate(), flush=True)
        return
    if args.cpu_table:
        import torch
        torch.cuda.set_device(local_rank)
        print(json.dumps({"cpu_baseline_table": cpu_baseline_table()}), flush=True)
        return
    if args.batched_only:
        import torch
        torch.cuda.set_device(local_rank)
        print(json.dumps({"batched_steps": batched_steps(torch.cuda.Stream(), args.batch_variant, args.steps)}),
              flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
