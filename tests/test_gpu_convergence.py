"""Self-convergence of the whole path under grid refinement (the paper's appendix studies the
same question by doubling its resolution; its own experiment, on the on-chip line with
anisotropic cells, is reproduced at the end of this file).  The 64 x 32 x 24 microstrip of 5 um cells is
rebuilt in fixed physical units at 2.5 um, 1.25 um and 0.625 um cells: every cell count,
the CPML thickness, the strip, source and port positions scale with the refinement, the
pulse and frequencies stay in hertz, and the step count doubles with each level (Courant 0.99).

Yee's scheme is second order in the bulk; the staircased strip edges and the one-cell I-loop
margin (whose physical size shrinks with the cell) bring first-order terms, and the coarsest
grid (a 6-cell strip on an 8-cell substrate) is not yet in the asymptotic range.  So the test
asks for convergence at least of first order on average, not a per-level order: the S*
differences between successive levels must decrease monotonically, fall by at least 4 over
the last two doublings, and the finest pair must agree within 0.05.  (Measured: 0.018,
0.013, 0.0018.)"""
import math

import numpy as np
import pytest

from oracle import post, yee
from paper_2208_04371_b300 import convergence as C
from paper_2208_04371_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _line(r):
    """The microstrip refined r times (r = 1, 2, 4, 8)."""
    p = W.microstrip(64 * r, 32 * r, 24 * r, 5e-6 / r, sub_cells=8 * r, strip_j0=13 * r,
                     strip_j1=19 * r, eps_r=3.8, sigma=0.0, pml=8 * r,
                     bc=(1, 1, 0, 0, 0, 1), courant=0.99, nsteps=2000 * r,
                     freqs=W.linear_freqs(100e9, 400e9, 48), f0=250e9, bw=200e9,
                     src_plane=10 * r, port_planes=(14 * r, 50 * r))
    return p


def test_sparams_converge_under_refinement(gpu):
    S = []
    for r in (1, 2, 4, 8):
        p = _line(r)
        with gpu.Grid(p, prec=gpu.FP32) as g:
            g.step(p.nsteps)
            g.sync()
            S.append(g.sparams()["S_star"])
    d = [np.max(np.abs(S[k + 1] - S[k])) for k in range(3)]
    print("successive S* differences:", d)
    assert d[2] < d[1] < d[0]
    assert d[2] * 4 <= d[0]
    assert d[2] <= 0.05


# The Appendix's convergence test on the on-chip line of Sec. III, with its anisotropic cells
# (50 x 20 x 5 nm here: dz is a tenth of dx), on a reduced grid of 96 x 40 x 64 cells (the same
# strip, step, oxide gap, Al block and conductivities as the full line).  The lossy Pd strip
# leaves a slow low-frequency tail, so the narrow pulse runs 24000 steps (348 fs) at the
# coarsest level, and the same physical time at each finer level.
BASE = (96, 40, 64, 6)
FREQS = W.linear_freqs(2e12, 60e12, 30)


@pytest.fixture(scope="module")
def appendix(gpu):
    narrow = [C.s11_star(BASE, r, C.SIGMA_NARROW, 24000, FREQS) for r in (1, 2, 4)]
    wide = C.s11_star(BASE, 1, C.SIGMA_WIDE, 48000, FREQS)
    return narrow, wide


def test_appendix_wide_and_narrow_pulses_agree(appendix):
    """The paper: |S*_11| from the wide pulse (sigma = 10.146 fs) and the narrow one (1.45 fs)
    are indistinguishable where both pulses carry energy.  Here: within 3e-3 from 6 THz up
    (measured at most 1.4e-3), and within 1e-2 at the lowest frequencies, where the wide
    pulse's tail is still settling after 48000 steps (7.5e-3 at 2 THz)."""
    narrow, wide = appendix
    d = np.abs(wide["S11"] - narrow[0]["S11"])
    assert np.max(d[FREQS >= 6e12]) <= 3e-3
    assert np.max(d) <= 1e-2


def test_appendix_refinement_converges(appendix):
    """The narrow pulse on grids 1, 2 and 4 times finer in every direction (non-cubic cells
    throughout): the S*_11 differences between successive levels shrink, the 2x and 4x grids
    agree within 1e-2, and the observed order log2(d_1 / d_2) is at least 1 (measured 0.025,
    0.0083: 1.56).  Staircased strip edges and a skin depth (21 nm at 60 THz) resolved by a
    few cells keep the rate below the bulk scheme's second order."""
    narrow, _ = appendix
    o = C.orders(narrow)
    d = o["differences"]
    print("S*_11 differences between levels:", d, "observed order:", o["orders"])
    assert d[1] < d[0]
    assert d[1] <= 1e-2
    assert o["orders"][0] >= 1.0


def test_appendix_coarsest_level_matches_oracle(appendix):
    """The coarsest narrow-pulse level against the FP64 oracle's two runs (incident and
    total) and Eq. 1: within the FP32 budget of 1e-3 (measured 1.3e-5)."""
    narrow, _ = appendix
    inc = C.line(BASE, 1, C.SIGMA_NARROW, 24000, FREQS, uniform=True)
    tot = C.line(BASE, 1, C.SIGMA_NARROW, 24000, FREQS, uniform=False)
    ri, rt = yee.run(inc), yee.run(tot)
    assert ri["dt"] == narrow[0]["dt"]
    Vi, Ii = post.port_dfts(ri["V"], ri["I"], FREQS, ri["dt"])
    Vt, _ = post.port_dfts(rt["V"], rt["I"], FREQS, rt["dt"])
    S, _ = post.sstar(Vi[:1], Ii[:1], Vt[:1][None])
    assert np.max(np.abs(S[:, 0, 0] - narrow[0]["S11"])) <= 1e-3
