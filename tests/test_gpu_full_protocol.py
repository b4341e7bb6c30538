"""The full S-parameter protocol of Sec. II-A on the GPU: for each driven port an incident run
on the uniformised line and a total run on the real circuit (4 runs for a two-port), here as
four instances of one batched solve (FP32 fields, FP64 spectra), extracted by the library's
FP64 kernel (Eq. 1, 2, 5-6).  The circuit is a microstrip with a wider section placed
asymmetrically along it (a step discontinuity).

Checks: reciprocity |S*_12 - S*_21| / |S*_21| <= 1e-3 (the paper notes the two transmission
delays coincide, Sec. III); the discontinuity reflects (|S*_11| > 0.2 somewhere in band);
and every entry of S* and S within 1e-3 of the FP64 oracle's four runs (the FP32 budget)."""
import numpy as np
import pytest

from oracle import post, yee
from paper_2208_04371_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _widened_line(driven, uniform, nsteps=2500):
    nx = 128
    p = W.microstrip(nx, 32, 24, 5e-6, sub_cells=8, strip_j0=13, strip_j1=19, eps_r=3.8,
                     sigma=0.0, pml=8, bc=(1, 1, 0, 0, 0, 1), courant=0.99, nsteps=nsteps,
                     freqs=W.linear_freqs(100e9, 400e9, 31), f0=250e9, bw=250e9, src_plane=10,
                     port_planes=(24, 104))
    if not uniform:
        p.sheets.append((2, 8, 55, 70, 10, 22))
    p.source.plane = 10 if driven == 0 else nx - 10
    return p


def _assemble(dfts):
    """(V_inc, I_inc, V_tot) of the protocol from {driven: ((V, I) incident, (V, I) total)}."""
    Vinc = np.array([dfts[0][0][0][0], dfts[1][0][0][1]])
    Iinc = np.array([dfts[0][0][1][0], dfts[1][0][1][1]])
    Vtot = np.array([dfts[0][1][0], dfts[1][1][0]])
    return Vinc, Iinc, Vtot


def test_four_run_protocol_on_the_gpu_is_reciprocal_and_matches_the_oracle(gpu):
    probs = [_widened_line(d, u) for d in (0, 1) for u in (True, False)]
    with gpu.Batch(probs, prec=gpu.FP32) as b:
        b.step(probs[0].nsteps)
        b.sync()
        got = {d: (b.port_dfts(2 * d), b.port_dfts(2 * d + 1)) for d in (0, 1)}
        dt = b.dt
    Vinc, Iinc, Vtot = _assemble(got)
    sp = gpu.sparams(probs[0].freqs, Vinc, Iinc, Vtot)
    Ss = sp["S_star"]
    assert np.max(np.abs(Ss[:, 0, 1] - Ss[:, 1, 0]) / np.abs(Ss[:, 1, 0])) <= 1e-3
    assert np.abs(Ss[:, 0, 0]).max() > 0.2

    ref = {}
    for d in (0, 1):
        runs = []
        for u in (True, False):
            p = _widened_line(d, u)
            r = yee.run(p, dt=dt)
            runs.append(post.port_dfts(r["V"], r["I"], p.freqs, r["dt"]))
        ref[d] = tuple(runs)
    So, Zo = post.sstar(*_assemble(ref))
    Sno = post.renormalize(So, Zo)
    assert np.max(np.abs(Ss - So)) <= 1e-3
    assert np.max(np.abs(sp["S"] - Sno)) <= 1e-3
