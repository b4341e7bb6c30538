"""The paper's on-chip line (Sec. III) through the four-run S-parameter protocol of Sec. II-A.

For each driven port, an incident run on the uniformised line (the driven port's
cross-section along the whole length) and a total run on the real line; the spectra of the
four runs go through the library's FP64 extraction (Eq. 1, 2, 5-6), and the Telegrapher
RLCG (end of Sec. II-A) of the first half's line comes from its own uniform run.  Geometry,
cells, pulse and the conductivity assumptions are those of workloads.config_cmos_line.

    python -m paper_2208_04371_b300.cmos_line --steps 200000 --out cmos.json

Every run is an FP32 grid on the two-step path (variant 4), one after another on one GPU.
"""
import argparse
import json
import time

import numpy as np

from . import workloads as W


def run_protocol(yf, nsteps: int, nx=120, ny=200, nz=800, pml=10, nfreq=64, variant=4, kseg=32,
                 log=print):
    """The four runs; returns (result dict, cell updates, seconds)."""
    import torch
    dfts, dt, cells, secs, line1 = {}, None, 0, 0.0, None
    for d in (0, 1):
        runs = []
        for u in (True, False):
            p = W.config_cmos_line(nx=nx, ny=ny, nz=nz, nsteps=nsteps, driven=d, uniform=u,
                                   nfreq=nfreq, pml=pml)
            prec = yf.FP32
            with yf.Grid(p, prec=prec, variant=variant, kseg=kseg) as g:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                g.step(nsteps)
                g.sync()
                el = time.perf_counter() - t0
                runs.append(g.port_dfts())
                dt = g.dt
                if d == 0 and u:
                    # the first half's line alone: uniform-line extraction of this run
                    line1 = g.sparams()
            cells += p.cells * nsteps
            secs += el
            log(f"{p.name}: {nsteps} steps in {el:.1f} s ({p.cells * nsteps / el / 1e9:.1f} Gcell/s)")
        dfts[d] = tuple(runs)
    f = W.config_cmos_line(nx=nx, ny=ny, nz=nz, nsteps=nsteps, nfreq=nfreq, pml=pml).freqs
    Vinc = np.array([dfts[0][0][0][0], dfts[1][0][0][1]])
    Iinc = np.array([dfts[0][0][1][0], dfts[1][0][1][1]])
    Vtot = np.array([dfts[0][1][0], dfts[1][1][0]])
    sp = yf.sparams(f, Vinc, Iinc, Vtot)
    # RLCG per unit length of the first half's line between the two port planes
    q = W.config_cmos_line(nx=nx, ny=ny, nz=nz, nfreq=nfreq, pml=pml)
    length = (q.ports[1].plane - q.ports[0].plane) * q.dx
    rl = yf.rlcg(f, line1["S_star"], line1["Zr"], length)
    res = {"freqs_hz": f.tolist(), "dt": dt, "steps": nsteps,
           "S11": sp["S"][:, 0, 0].tolist(), "S21": sp["S"][:, 1, 0].tolist(),
           "S12": sp["S"][:, 0, 1].tolist(), "S22": sp["S"][:, 1, 1].tolist(),
           "Sstar11": sp["S_star"][:, 0, 0].tolist(), "Sstar22": sp["S_star"][:, 1, 1].tolist(),
           "Sstar21": sp["S_star"][:, 1, 0].tolist(), "Sstar12": sp["S_star"][:, 0, 1].tolist(),
           "Zr": sp["Zr"].tolist(), "tau21": sp["tau"][:, 1, 0].tolist(),
           "line1_Zc": line1["Zc"].tolist(),
           "line1_R": rl["R"].tolist(), "line1_L": rl["L"].tolist(), "line1_G": rl["G"].tolist(),
           "line1_C": rl["C"].tolist()}
    return res, cells, secs


def _jsonable(x):
    if isinstance(x, list):
        return [_jsonable(v) for v in x]
    if isinstance(x, complex):
        return [x.real, x.imag]
    return x


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=1_400_000)
    ap.add_argument("--out", default="")
    args = ap.parse_args()
    from . import yf
    res, cells, secs = run_protocol(yf, args.steps)
    res["gcell_per_s"] = cells / secs / 1e9
    S = np.array(res["S21"]); R = np.array(res["S12"])
    res["reciprocity_max_rel"] = float(np.max(np.abs(S - R)) / np.max(np.abs(S)))
    print(f"4 runs, {cells:.3e} cell updates, {secs:.1f} s, {res['gcell_per_s']:.1f} Gcell/s; "
          f"max |S21 - S12| / max |S21| = {res['reciprocity_max_rel']:.2e}")
    if args.out:
        with open(args.out, "w") as fh:
            json.dump({k: _jsonable(v) for k, v in res.items()}, fh)


if __name__ == "__main__":
    main()
