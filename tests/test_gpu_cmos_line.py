"""The paper's on-chip line (Sec. III; the last of the ranked follow-on workloads) on the GPU.

1. Parity: the same stack on a reduced grid (96 x 40 x 64 cells of the paper's 50 x 20 x 5 nm,
   same strip, step, oxide gap, Al block and conductivities), 2500 steps (past the pulse
   peak at 3 sigma = 2100 steps), each driven side, against the FP64 oracle: FP64 fields
   relative L2 <= 1e-12 and port spectra <= 1e-10; FP32 fields <= 1e-5, on the one-step path
   and on the two-step path (this grid has an inner box).
2. Physics at full size (120 x 200 x 800 cells, dt = 0.0145 fs as printed): the uniform run of
   the first half's line, 40000 steps.  Strip and ground are separated by homogeneous SiO2, so
   the line is TEM with eps_eff = 3.9 and, for w/h = 1 (2 um strip 2 um above the ground),
   Hammerstad's closed form gives Z0 = 60/sqrt(3.9) ln(8 h/w + w/(4 h)) = 64.1 ohm; at the
   lowest frequency (2 THz, strip thinner than a skin depth, R/(omega L) about 0.2) the
   extracted Z_c must lie within 10 % of it (measured 64.8 - 3.5j ohm)."""
import math

import numpy as np
import pytest

from oracle import post, yee
from paper_2208_04371_b300 import workloads as W

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


@pytest.mark.parametrize("driven", [0, 1])
def test_reduced_cmos_line_matches_oracle(gpu, driven):
    p = W.config_cmos_line(nx=96, ny=40, nz=64, pml=6, nsteps=2500, nfreq=16, driven=driven)
    ref = yee.run(p, want_fields=True)
    Vo, Io = post.port_dfts(ref["V"], ref["I"], p.freqs, ref["dt"])
    with gpu.Grid(p, prec=gpu.FP64, variant=2) as g:
        g.step(p.nsteps)
        g.sync()
        f = g.fields()
        V, I = g.port_dfts()
    assert rel_l2(f, ref["fields"]) <= 1e-12
    assert np.max(np.abs(V - Vo)) <= 1e-10 * np.max(np.abs(Vo))
    assert np.max(np.abs(I - Io)) <= 1e-10 * np.max(np.abs(Io))
    for v in (2, 4):
        with gpu.Grid(p, prec=gpu.FP32, variant=v) as g:
            if v == 4:
                assert gpu.tb_box(g.h) is not None
            g.step(p.nsteps)
            g.sync()
            f = g.fields()
        assert rel_l2(f, ref["fields"]) <= 1e-5, v


def test_full_size_first_half_line_impedance(gpu):
    p = W.config_cmos_line(nsteps=40000, driven=0, uniform=True)
    with gpu.Grid(p, prec=gpu.FP32, variant=4, kseg=32) as g:
        assert g.dt == pytest.approx(0.0145e-15, rel=2e-3)
        g.step(p.nsteps)
        g.sync()
        sp = g.sparams()
    zc = sp["Zc"][0]
    z0 = 60.0 / math.sqrt(3.9) * math.log(8.0 + 0.25)
    assert np.isfinite(sp["S"]).all()
    assert abs(zc - z0) <= 0.10 * z0, zc
