"""The Appendix's convergence test on the on-chip line of Sec. III.

The paper checks its grid by comparing |S*_11| of the line three ways: the wide pulse of
Sec. III (Eq. 3, sigma = 10.146 fs) on the original grid, a narrow pulse (sigma = 1.45 fs,
peak near 155 THz) on the same grid for a much shorter run, and the narrow pulse on a grid
twice as fine in every direction.  The pulses must agree wherever both carry energy, and the
two grids must agree with each other.

Here the line is `workloads.config_cmos_line` with its anisotropic cells (50 x 20 x 5 nm in
this build's frame) at any base size, refined r = 1, 2, 4 ... times (every cell size divided
by r, every cell count multiplied by r, the time step halving with the cells at CFL 0.9 and
the step count doubling, so each level covers the same physical time).  S*_11 comes from the
two runs of Sec. II-A (the incident run on the line made uniform with port 1's cross-section,
and the total run), advanced together by the batched solver in FP32 fields, and Eq. 1 through
the library's FP64 extraction kernel.

    python -m paper_2208_04371_b300.convergence --nx 96 --ny 40 --nz 64 --pml 6 \\
        --steps 6000 --levels 1,2,4 --out convergence.json
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import workloads as W
from . import yf

SIGMA_WIDE = 10.146e-15      # Sec. III
SIGMA_NARROW = 1.45e-15      # Appendix


def line(base, r: int, sigma: float, nsteps: int, freqs, uniform: bool) -> "W.Problem":
    nx, ny, nz, pml = base
    p = W.config_cmos_line(nx=nx, ny=ny, nz=nz, pml=pml, nsteps=nsteps * r, driven=0,
                           uniform=uniform, nfreq=len(freqs), refine=r, sigma=sigma)
    p.freqs = np.asarray(freqs, dtype=np.float64)
    return p


def s11_star(base, r: int, sigma: float, nsteps: int, freqs, stream=None) -> dict:
    """S*_11 of the line refined r times, driven at port 1 by the Eq. 3 pulse of width sigma,
    after nsteps * r steps (the same physical time at every level)."""
    inc = line(base, r, sigma, nsteps, freqs, uniform=True)
    tot = line(base, r, sigma, nsteps, freqs, uniform=False)
    t = time.perf_counter()
    with yf.Batch([inc, tot], prec=yf.FP32, stream=stream) as b:
        b.step(inc.nsteps)
        b.sync()
        Vi, Ii = b.port_dfts(0)
        Vt, _ = b.port_dfts(1)
        dt = b.dt
    el = time.perf_counter() - t
    sp = yf.sparams(freqs, Vi[:1], Ii[:1], Vt[:1][None, :, :])
    return {"r": r, "sigma": sigma, "steps": inc.nsteps, "dt": dt, "cells": inc.cells,
            "S11": sp["S_star"][:, 0, 0], "seconds": el}


def orders(levels) -> dict:
    """Successive differences max_f |S*_11(2r) - S*_11(r)| and the observed orders
    log2(d_k / d_{k+1}) of a sequence of doubling levels."""
    d = [float(np.max(np.abs(levels[k + 1]["S11"] - levels[k]["S11"])))
         for k in range(len(levels) - 1)]
    p = [math.log2(d[k] / d[k + 1]) for k in range(len(d) - 1) if d[k + 1] > 0]
    return {"differences": d, "orders": p}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=96)
    ap.add_argument("--ny", type=int, default=40)
    ap.add_argument("--nz", type=int, default=64)
    ap.add_argument("--pml", type=int, default=6)
    ap.add_argument("--steps", type=int, default=6000,
                    help="steps of the narrow-pulse run at the coarsest level")
    ap.add_argument("--wide-steps", type=int, default=20000,
                    help="steps of the wide-pulse run (coarsest level only)")
    ap.add_argument("--levels", default="1,2,4")
    ap.add_argument("--f-lo", type=float, default=2e12)
    ap.add_argument("--f-hi", type=float, default=60e12)
    ap.add_argument("--nfreq", type=int, default=30)
    ap.add_argument("--out", default="convergence.json")
    args = ap.parse_args()
    base = (args.nx, args.ny, args.nz, args.pml)
    freqs = W.linear_freqs(args.f_lo, args.f_hi, args.nfreq)
    narrow = [s11_star(base, int(r), SIGMA_NARROW, args.steps, freqs)
              for r in args.levels.split(",")]
    wide = s11_star(base, 1, SIGMA_WIDE, args.wide_steps, freqs)
    out = {"line": f"on-chip line {args.nx}x{args.ny}x{args.nz} cells of 50x20x5 nm, PML {args.pml}",
           "freqs_hz": list(freqs),
           "narrow": [{k: (v if k != "S11" else [[c.real, c.imag] for c in v]) for k, v in L.items()}
                      for L in narrow],
           "wide": {k: (v if k != "S11" else [[c.real, c.imag] for c in v]) for k, v in wide.items()},
           "wide_vs_narrow_max_abs": float(np.max(np.abs(wide["S11"] - narrow[0]["S11"]))),
           **orders(narrow)}
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: v for k, v in out.items() if k not in ("narrow", "wide", "freqs_hz")}))


if __name__ == "__main__":
    main()
