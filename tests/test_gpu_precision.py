"""Precision variants on the long-run workload (256x128x128 lossless eps_r 3.9 microstrip,
256 frequencies): FP32 fields with FP64, Kahan-compensated FP32 and plain FP32 running-DFT
accumulators (the transforms of Sec. II-A, Eq. 1-2), the FP64-field GPU run as the long-run reference, and a 2000-step
subrun against the FP64 oracle.

Tolerances:
  FP64 fields vs oracle            relative L2 <= 1e-12; spectra <= 1e-10 of their max
  FP32 fields vs oracle            relative L2 <= 1e-5 (ringing variant: the fields stay at
                                   their peak scale, so the ratio measures FP32 rounding)
  FP32-field spectra vs oracle     <= 1e-4 of their max (a port integral is a sum in FP64
                                   of FP32 field values, so it inherits the ~1e-5 field error)
  FP32 |S_ij| vs oracle / FP64 run <= 1e-3 absolute
  Kahan vs FP64 accumulators fed the same samples: <= 1e-6 of the spectrum max.  The bound
  is the per-term rounding of each product to FP32 (eps/2 |t|) plus Kahan's 2 eps sum|t|;
  with sum|t| within a few times max|X| for a resonating line this is ~1e-6 at most.
"""
import numpy as np
import pytest

from oracle import post, yee
from paper_2208_04371_b300 import precision_study as PS
from paper_2208_04371_b300 import workloads as W

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def rel_max(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.fixture(scope="module")
def ringing_2k():
    p = W.config_long_run(nsteps=2000, ringing=True)
    return p, yee.run(p, want_fields=True)


@pytest.fixture(scope="module")
def line_2k():
    p = W.config_long_run(nsteps=2000, ringing=False)
    return p, yee.run(p)


def _all(gpu):
    return gpu.DFT_FP64 | gpu.DFT_KAHAN32 | gpu.DFT_FP32


def test_subrun_fp64_fields_match_oracle(gpu, ringing_2k):
    p, ref = ringing_2k
    with gpu.Grid(p, prec=gpu.FP64) as g:
        g.step(p.nsteps)
        g.sync()
        f = g.fields()
        V, I = g.port_dfts()
    assert rel_l2(f, ref["fields"]) <= 1e-12
    Vo, Io = post.port_dfts(ref["V"], ref["I"], p.freqs, ref["dt"])
    assert rel_max(V, Vo) <= 1e-10 and rel_max(I, Io) <= 1e-10


def test_subrun_fp32_fields_and_accumulators_match_oracle(gpu, ringing_2k):
    p, ref = ringing_2k
    with gpu.Grid(p, prec=gpu.FP32, dft_mask=_all(gpu)) as g:
        g.step(p.nsteps)
        g.sync()
        f = g.fields()
        spectra = {k: g.port_dfts(k) for k in (gpu.DFT_FP64, gpu.DFT_KAHAN32, gpu.DFT_FP32)}
    assert rel_l2(f, ref["fields"]) <= 1e-5
    Vo, Io = post.port_dfts(ref["V"], ref["I"], p.freqs, ref["dt"])
    for kind, (V, I) in spectra.items():
        assert rel_max(V, Vo) <= 1e-4, kind
        assert rel_max(I, Io) <= 1e-4, kind


def test_subrun_fp32_sparams_match_oracle(gpu, line_2k):
    p, ref = line_2k
    Vo, Io = post.port_dfts(ref["V"], ref["I"], p.freqs, ref["dt"])
    So, Zo = post.sstar_uniform(Vo, Io, [1, -1])
    Sno = post.renormalize(So, Zo)
    with gpu.Grid(p, prec=gpu.FP32, dft_mask=_all(gpu)) as g:
        g.step(p.nsteps)
        g.sync()
        for kind in (gpu.DFT_FP64, gpu.DFT_KAHAN32, gpu.DFT_FP32):
            sp = g.sparams(kind)
            assert np.max(np.abs(np.abs(sp["S_star"]) - np.abs(So))) <= 1e-3, kind
            assert np.max(np.abs(np.abs(sp["S"]) - np.abs(Sno))) <= 1e-3, kind


def test_kahan_tracks_fp64_accumulators_over_a_long_ringing_run(gpu):
    """The three accumulator sets of one FP32-field grid see identical samples, so their
    differences are accumulation error alone.  After 1e5 steps on the resonating line Kahan
    stays at the FP32 product-rounding level while plain FP32 drifts."""
    n = 100_000
    p = W.config_long_run(nsteps=n, ringing=True)
    with gpu.Grid(p, prec=gpu.FP32, dft_mask=_all(gpu)) as g:
        g.step(n)
        g.sync()
        V64, I64 = g.port_dfts(gpu.DFT_FP64)
        Vk, Ik = g.port_dfts(gpu.DFT_KAHAN32)
        V32, I32 = g.port_dfts(gpu.DFT_FP32)
    ek = max(rel_max(Vk, V64), rel_max(Ik, I64))
    e32 = max(rel_max(V32, V64), rel_max(I32, I64))
    assert ek <= 1e-6
    assert e32 > 10 * ek
    # worst case of plain recursive summation: n eps/2 relative to the largest partial sum
    assert e32 <= n * 2.0 ** -24


def test_fp32_fields_match_fp64_run_in_sparams(gpu):
    """The study's own comparison on a 20000-step run of the terminated line: FP32 fields with
    FP64 or Kahan accumulators stay within 1e-3 in |S_ij| of the FP64-field run."""
    res = PS.run(20_000, ringing=False, chunk=10_000, checkpoints=(10_000,), log=lambda s: None)
    assert [r["steps"] for r in res["at"]] == [10_000, 20_000]
    last = res["at"][-1]
    assert last["s_abs_err"]["fp64"] <= 1e-3
    assert last["s_abs_err"]["kahan32"] <= 1e-3
    assert last["spectrum_rel_err"]["kahan32"] <= 1e-4
