"""Long-run precision study: FP32 fields with three DFT accumulators against FP64.

Workload: the 256x128x128 lossless eps_r 3.9 microstrip (5 um cells, 256 DFT frequencies over
100-500 GHz) run for up to a million steps.  The ringing variant closes both x ends with PEC,
so the line keeps resonating and the running transforms (Sec. II-A: the transforms of Eq. 1-2, taken on the fly)
keep growing for the whole run.

One FP32-field grid accumulates its port spectra three ways at once (FP64, Kahan-compensated
FP32 pairs, plain FP32).  An FP64-field grid with FP64 accumulators is the reference.  For
each accumulator set the study reports:
  * spectrum_rel_err: max over ports and frequencies of |X - X_ref|, relative to max |X_ref|
    (V and I separately, the larger is kept);
  * s_abs_err: max over frequencies and entries of | |S_ij| - |S_ij,ref| | of the 50-ohm
    S-matrix from the uniform-line extraction (Eq. 1-2, 5-6), which is FP64 in every case.

    python -m paper_2208_04371_b300.precision_study --steps 1000000 --out study.json

With --lossy-line it instead runs the 768x384x256 lossy line on the benchmark's FP32 path
(two steps per pass over the inner box) beside an FP64-field run of the same line and
reports the field and S-parameter errors at the step counts of --marks.
"""
from __future__ import annotations

import argparse
import json
import time
from typing import Optional

import numpy as np

from . import workloads as W
from . import yf

ACCUMULATORS = (("fp64", yf.DFT_FP64), ("kahan32", yf.DFT_KAHAN32), ("fp32", yf.DFT_FP32))


def spectrum_rel_err(ref, got) -> float:
    (Vr, Ir), (Vg, Ig) = ref, got
    return float(max(np.max(np.abs(Vg - Vr)) / np.max(np.abs(Vr)),
                     np.max(np.abs(Ig - Ir)) / np.max(np.abs(Ir))))


def s_abs_err(ref, got) -> float:
    return float(np.max(np.abs(np.abs(got["S"]) - np.abs(ref["S"]))))


def accumulator_only(g32: "yf.Grid") -> dict:
    """Accumulation error alone: the FP32-field grid's Kahan and plain FP32 sets against its
    own FP64 set, all three fed the same samples."""
    own = g32.port_dfts(yf.DFT_FP64)
    return {name: spectrum_rel_err(own, g32.port_dfts(kind))
            for name, kind in ACCUMULATORS if kind != yf.DFT_FP64}


def compare(g32: "yf.Grid", g64: Optional["yf.Grid"]) -> dict:
    """Errors of each accumulator set of the FP32-field grid against the FP64 grid (when
    given), and against the FP32 grid's own FP64 accumulators."""
    out = {"acc_rel_err": accumulator_only(g32)}
    if g64 is None:
        return out
    ref_spec = g64.port_dfts(yf.DFT_FP64)
    ref_s = g64.sparams(yf.DFT_FP64)
    out["spectrum_rel_err"], out["s_abs_err"] = {}, {}
    for name, kind in ACCUMULATORS:
        out["spectrum_rel_err"][name] = spectrum_rel_err(ref_spec, g32.port_dfts(kind))
        out["s_abs_err"][name] = s_abs_err(ref_s, g32.sparams(kind))
    return out


def run(nsteps: int, ringing: bool, chunk: int = 50_000, checkpoints=(), log=print,
        with_fp64: bool = True) -> dict:
    """Advance the FP32 and (with_fp64) FP64 grids side by side; compare at each checkpoint
    step count (and at the end)."""
    prob = W.config_long_run(nsteps=nsteps, ringing=ringing)
    res = {"workload": prob.name, "cells": prob.cells, "steps": nsteps, "at": []}
    marks = sorted(set([c for c in checkpoints if 0 < c < nsteps] + [nsteps]))
    mask = yf.DFT_FP64 | yf.DFT_KAHAN32 | yf.DFT_FP32
    g64 = yf.Grid(prob, prec=yf.FP64, dft_mask=yf.DFT_FP64) if with_fp64 else None
    with yf.Grid(prob, prec=yf.FP32, dft_mask=mask) as g32:
        if g64 is not None and g32.dt != g64.dt:
            raise RuntimeError("the two grids must share one time step")
        t32 = t64 = 0.0
        done = 0
        for m in marks:
            while done < m:
                n = min(chunk, m - done)
                t = time.perf_counter()
                g32.step(n)
                g32.sync()
                t32 += time.perf_counter() - t
                if g64 is not None:
                    t = time.perf_counter()
                    g64.step(n)
                    g64.sync()
                    t64 += time.perf_counter() - t
                done += n
            row = {"steps": m, **compare(g32, g64)}
            res["at"].append(row)
            log(json.dumps({"workload": prob.name, **row}))
        res["fp32_fields_gcell_s"] = prob.cells * nsteps / t32 / 1e9
        if g64 is not None:
            res["fp64_fields_gcell_s"] = prob.cells * nsteps / t64 / 1e9
            res["peak_abs_s21"] = float(np.max(np.abs(g64.sparams()["S"][:, 1, 0])))
            g64.close()
    return res


def field_errors(g32: "yf.Grid", g64: "yf.Grid") -> dict:
    """Relative L2 over all six components of the FP32 grid's fields against the FP64
    grid's, ||F32 - F64|| / ||F64||, and the largest pointwise error relative to the largest
    FP64 value; both grids' components are read into device buffers one at a time."""
    import torch
    p = g32.prob
    shape = (p.nz + 1, p.ny + 1, p.nx + 1)
    b32 = torch.empty(shape, dtype=torch.float32, device="cuda")
    b64 = torch.empty(shape, dtype=torch.float64, device="cuda")
    err2 = ref2 = 0.0
    emax = rmax = 0.0
    for c in range(6):
        yf.read_fields(g32.h, c, b32)
        yf.read_fields(g64.h, c, b64)
        d = b32.double() - b64
        err2 += float(torch.sum(d * d))
        ref2 += float(torch.sum(b64 * b64))
        emax = max(emax, float(torch.max(torch.abs(d))))
        rmax = max(rmax, float(torch.max(torch.abs(b64))))
    return {"field_rel_l2": (err2 / ref2) ** 0.5 if ref2 > 0 else None,
            "field_max_rel": emax / rmax if rmax > 0 else None}


def lossy_line(marks=(2000, 20000), box_seg: int = 128, log=print) -> dict:
    """The single large lossy line (768 x 384 x 256 cells of 20 nm) on the benchmark's path,
    FP32 fields two steps per pass over the inner box, against the same line with FP64 fields
    (FP64 accumulators both), advanced side by side.  At each step count: relative field L2
    and pointwise error, and the S-parameter errors of the uniform-line extraction (S* and the
    50-ohm S, complex difference and difference of magnitudes)."""
    prob = W.config_lossy_line(nsteps=max(marks))
    res = {"workload": prob.name, "cells": prob.cells, "fp32_path": "two steps per pass over "
           f"the inner box (variant 4, kseg 32, box segments of {box_seg} planes)",
           "fp64_path": "FP64 fields, one step per pass", "at": []}
    t32 = t64 = 0.0
    with yf.Grid(prob, prec=yf.FP32, variant=4, kseg=32, box_seg=box_seg) as g32, \
            yf.Grid(prob, prec=yf.FP64) as g64:
        if g32.dt != g64.dt:
            raise RuntimeError("the two grids must share one time step")
        done = 0
        for m in sorted(marks):
            n = m - done
            t = time.perf_counter()
            g32.step(n)
            g32.sync()
            t32 += time.perf_counter() - t
            t = time.perf_counter()
            g64.step(n)
            g64.sync()
            t64 += time.perf_counter() - t
            done = m
            s32, s64 = g32.sparams(), g64.sparams()
            row = {"steps": m, **field_errors(g32, g64)}
            for key in ("S_star", "S"):
                row[f"{key}_abs_err"] = float(np.max(np.abs(s32[key] - s64[key])))
                row[f"{key}_mag_err"] = float(np.max(np.abs(np.abs(s32[key]) - np.abs(s64[key]))))
            row["max_abs_S21_fp64"] = float(np.max(np.abs(s64["S"][:, 1, 0])))
            res["at"].append(row)
            log(json.dumps({"workload": prob.name, **row}))
    res["fp32_fields_gcell_s"] = prob.cells * done / t32 / 1e9
    res["fp64_fields_gcell_s"] = prob.cells * done / t64 / 1e9
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=1_000_000)
    ap.add_argument("--out", default="precision_study.json")
    ap.add_argument("--accumulators-only", action="store_true",
                    help="skip the FP64-field reference grid (accumulator comparisons only)")
    ap.add_argument("--ringing-only", action="store_true")
    ap.add_argument("--lossy-line", action="store_true",
                    help="the 768x384x256 lossy line: FP32 fields on the benchmark's path against "
                         "FP64 fields, at the step counts of --marks")
    ap.add_argument("--marks", default="2000,20000")
    args = ap.parse_args()
    if args.lossy_line:
        result = lossy_line(tuple(int(x) for x in args.marks.split(",")))
        with open(args.out, "w") as f:
            json.dump(result, f, indent=1)
        print(json.dumps(result))
        return
    cps = [args.steps // 1000, args.steps // 100, args.steps // 10]
    variants = (True,) if args.ringing_only else (False, True)
    result = [run(args.steps, ringing, checkpoints=cps, with_fp64=not args.accumulators_only)
              for ringing in variants]
    with open(args.out, "w") as f:
        json.dump(result, f, indent=1)
    print(json.dumps(result))


if __name__ == "__main__":
    main()
