"""The paper's on-chip line (Sec. III) through the four-run S-parameter protocol of Sec. II-A.

For each driven port, an incident run on the uniformised line (the driven port's
cross-section along the whole length) and a total run on the real line; the spectra of the
four runs go through the library's FP64 extraction (Eq. 1, 2, 5-6), and the Telegrapher
RLCG (end of Sec. II-A) of the first half's line comes from its own uniform run.  Geometry,
cells, pulse and the conductivity assumptions are those of workloads.config_cmos_line.

    python -m paper_2208_04371_b300.cmos_line --steps 1400000 --marks 40000,80000,200000 --out cmos.json

Every run is an FP32 grid on the two-step path (variant 4); the four advance together, each on
its own stream, and the extraction is repeated at each step count of --marks.
"""
import argparse
import json
import time

import numpy as np

from . import workloads as W


def _extract(yf, f, dfts, line1, length):
    """Eq. 1, 2, 5-6 of the four runs' spectra, and the first half's Telegrapher RLCG."""
    Vinc = np.array([dfts[0][0][0][0], dfts[1][0][0][1]])
    Iinc = np.array([dfts[0][0][1][0], dfts[1][0][1][1]])
    Vtot = np.array([dfts[0][1][0], dfts[1][1][0]])
    sp = yf.sparams(f, Vinc, Iinc, Vtot)
    rl = yf.rlcg(f, line1["S_star"], line1["Zr"], length)
    return {"S11": sp["S"][:, 0, 0].tolist(), "S21": sp["S"][:, 1, 0].tolist(),
            "S12": sp["S"][:, 0, 1].tolist(), "S22": sp["S"][:, 1, 1].tolist(),
            "Sstar11": sp["S_star"][:, 0, 0].tolist(), "Sstar22": sp["S_star"][:, 1, 1].tolist(),
            "Sstar21": sp["S_star"][:, 1, 0].tolist(), "Sstar12": sp["S_star"][:, 0, 1].tolist(),
            "Zr": sp["Zr"].tolist(), "tau21": sp["tau"][:, 1, 0].tolist(),
            "line1_Zc": line1["Zc"].tolist(),
            "line1_R": rl["R"].tolist(), "line1_L": rl["L"].tolist(), "line1_G": rl["G"].tolist(),
            "line1_C": rl["C"].tolist()}


def run_protocol(yf, nsteps: int, nx=120, ny=200, nz=800, pml=10, nfreq=64, variant=4, kseg=32,
                 log=print, marks=(), chunk=20000):
    """The four runs, advanced together (each grid on its own stream), with the extraction
    at every step count of `marks` and at the end; returns (result dict of the last, list of
    results at the marks, cell updates, seconds)."""
    import torch
    probs, grids, streams = [], [], []
    for d in (0, 1):
        for u in (True, False):
            p = W.config_cmos_line(nx=nx, ny=ny, nz=nz, nsteps=nsteps, driven=d, uniform=u,
                                   nfreq=nfreq, pml=pml)
            st = torch.cuda.Stream()
            probs.append(p)
            streams.append(st)
            grids.append(yf.Grid(p, prec=yf.FP32, stream=st.cuda_stream, variant=variant, kseg=kseg))
    try:
        f = probs[0].freqs
        q = W.config_cmos_line(nx=nx, ny=ny, nz=nz, nfreq=nfreq, pml=pml)
        length = (q.ports[1].plane - q.ports[0].plane) * q.dx
        stops = sorted(set([m for m in marks if 0 < m < nsteps] + [nsteps]))
        at, done, secs = [], 0, 0.0
        for m in stops:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            while done < m:
                n = min(chunk, m - done)
                for g in grids:
                    g.step(n)
                done += n
            for g in grids:
                g.sync()
            secs += time.perf_counter() - t0
            dfts = {0: (grids[0].port_dfts(), grids[1].port_dfts()),
                    1: (grids[2].port_dfts(), grids[3].port_dfts())}
            res = _extract(yf, f, dfts, grids[0].sparams(), length)
            res["steps"] = m
            at.append(res)
            cells = sum(p.cells for p in probs) * m
            log(f"{m} steps: {cells:.3e} cell updates in {secs:.1f} s ({cells / secs / 1e9:.1f} Gcell/s)")
        final = dict(at[-1])
        final.update({"freqs_hz": f.tolist(), "dt": grids[0].dt})
    finally:
        for g in grids:
            g.close()
    return final, at, sum(p.cells for p in probs) * nsteps, secs


def _jsonable(x):
    if isinstance(x, list):
        return [_jsonable(v) for v in x]
    if isinstance(x, complex):
        return [x.real, x.imag]
    return x


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=1_400_000)
    ap.add_argument("--marks", default="", help="step counts at which to extract as well, e.g. 40000,80000")
    ap.add_argument("--out", default="")
    args = ap.parse_args()
    from . import yf
    marks = [int(x) for x in args.marks.split(",") if x]
    res, at, cells, secs = run_protocol(yf, args.steps, marks=marks)
    res["gcell_per_s"] = cells / secs / 1e9
    S = np.array(res["S21"]); R = np.array(res["S12"])
    res["reciprocity_max_rel"] = float(np.max(np.abs(S - R)) / np.max(np.abs(S)))
    # how the results move with the run length: max |X(m) - X(final)| for each earlier mark
    res["change_to_final"] = [
        {"steps": a["steps"],
         **{k: float(np.max(np.abs(np.array(a[k]) - np.array(res[k]))))
            for k in ("S11", "S21", "Sstar11", "Sstar21", "line1_Zc")}}
        for a in at[:-1]]
    print(f"4 runs, {cells:.3e} cell updates, {secs:.1f} s, {res['gcell_per_s']:.1f} Gcell/s; "
          f"max |S21 - S12| / max |S21| = {res['reciprocity_max_rel']:.2e}")
    print(json.dumps(res["change_to_final"]))
    if args.out:
        with open(args.out, "w") as fh:
            json.dump({k: _jsonable(v) for k, v in res.items()}, fh)


if __name__ == "__main__":
    main()
