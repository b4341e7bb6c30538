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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=1_000_000)
    ap.add_argument("--out", default="precision_study.json")
    ap.add_argument("--accumulators-only", action="store_true",
                    help="skip the FP64-field reference grid (accumulator comparisons only)")
    ap.add_argument("--ringing-only", action="store_true")
    args = ap.parse_args()
    cps = [args.steps // 1000, args.steps // 100, args.steps // 10]
    variants = (True,) if args.ringing_only else (False, True)
    result = [run(args.steps, ringing, checkpoints=cps, with_fp64=not args.accumulators_only)
              for ringing in variants]
    with open(args.out, "w") as f:
        json.dump(result, f, indent=1)
    print(json.dumps(result))


if __name__ == "__main__":
    main()
