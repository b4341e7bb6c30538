"""Batched multi-instance solve: every instance equals the single-grid path (bitwise, same
kernels and tiling) and the FP64 oracle (1e-12 relative field L2)."""
import numpy as np
import pytest

from oracle import post, yee
from paper_2208_04371_b300 import workloads as W

pytestmark = pytest.mark.gpu

DIMS = [(48, 40, 36), (61, 45, 40), (70, 52, 33), (56, 64, 47), (40, 40, 40)]


def _instances(nsteps=300):
    rng = W.SplitMix64(0x5EED)
    probs = [W.batch_instance(rng, nsteps=nsteps, nfreq=24, dims=d) for d in DIMS]
    # vary the boundaries too: one instance with PEC side walls, one fully closed
    probs[3].bc = (1, 1, 0, 0, 0, 1)
    probs[4].bc = (0, 0, 0, 0, 0, 0)
    return probs


def rel_l2(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


@pytest.mark.parametrize("tile_y,kseg", [(8, 16), (4, 7), (16, 5)])
def test_batch_equals_single_grids_bitwise(gpu, tile_y, kseg):
    probs = _instances()
    n = 150
    with gpu.Batch(probs, prec=gpu.FP32, tile_y=tile_y, kseg=kseg) as b:
        b.step(n)
        b.sync()
        got = [b.fields(q) for q in range(len(probs))]
        dft = [b.port_dfts(q) for q in range(len(probs))]
        dt = b.dt
    for q, p in enumerate(probs):
        with gpu.Grid(p, prec=gpu.FP32, dt=dt, variant=2, tile_y=tile_y, kseg=kseg) as g:
            g.step(n)
            g.sync()
            assert np.array_equal(got[q], g.fields()), q
            V, I = g.port_dfts()
            assert np.array_equal(dft[q][0], V) and np.array_equal(dft[q][1], I), q


def test_batch_fp64_matches_oracle(gpu):
    probs = _instances(nsteps=200)[:3]
    with gpu.Batch(probs, prec=gpu.FP64) as b:
        b.step(200)
        b.sync()
        fields = [b.fields(q, prec=gpu.FP64) for q in range(3)]
        dfts = [b.port_dfts(q) for q in range(3)]
        sps = [b.sparams(q) for q in range(3)]
        dt = b.dt
    for q, p in enumerate(probs):
        ref = yee.run(p, nsteps=200, dt=dt, want_fields=True)
        assert rel_l2(fields[q], ref["fields"]) <= 1e-12, q
        Vo, Io = post.port_dfts(ref["V"], ref["I"], p.freqs, ref["dt"])
        assert np.max(np.abs(dfts[q][0] - Vo)) <= 1e-10 * np.max(np.abs(Vo))
        So, Zo = post.sstar_uniform(Vo, Io, [1, -1])
        assert np.max(np.abs(sps[q]["S_star"] - So)) <= 1e-8


def test_batch_shares_the_smallest_courant_step(gpu):
    probs = _instances()[:2]
    probs[1] = probs[1].replace(dx=2.5e-6)
    with gpu.Batch(probs, prec=gpu.FP32) as b:
        lim = min(yee.courant_dt(p.dx, p.dy, p.dz, 1.0) for p in probs)
        assert b.dt == pytest.approx(0.99 * lim, rel=1e-14)


def test_autotune_resets_state_and_caches(gpu, tmp_path):
    import json
    cache = str(tmp_path / "tiles.json")
    probs = _instances()[:3]
    with gpu.Batch(probs, prec=gpu.FP32) as b:
        ty, ks = b.autotune(cache, reps=2)
        assert ty in (4, 8, 16) and ks in (8, 16, 32)
        for q in range(3):
            assert not np.any(b.fields(q)), "tuning must leave the fields at zero"
        b.step(40)
        tuned = [b.fields(q) for q in range(3)]
    entries = json.load(open(cache))
    assert len(entries) == 1 and list(entries.values())[0][:2] == [ty, ks]
    with gpu.Batch(probs, prec=gpu.FP32, tile_y=ty, kseg=ks) as b:
        assert b.autotune(cache, reps=2) == (ty, ks)      # served from the cache
        b.step(40)
        for q in range(3):
            assert np.array_equal(b.fields(q), tuned[q])
    p = probs[0]
    with gpu.Grid(p, prec=gpu.FP32) as g:
        gt, gk = gpu.autotune(g.h, cache, reps=2)
        assert gt in (4, 8, 16) and gk in (8, 16, 32)
        assert gpu.steps_done(g.h) == 0 and not np.any(g.fields())
    assert len(json.load(open(cache))) == 2


def test_batch_takes_the_instances_courant_number(gpu):
    """A batch of lines built for CFL 0.9 (the on-chip line of Sec. III) steps with their own
    time step, not with the library's default of 0.99 of the Courant limit: the batch's dt and
    spectra equal the single-grid solver's bit for bit."""
    p = W.config_cmos_line(nx=96, ny=40, nz=64, pml=6, nsteps=300, nfreq=8)
    with gpu.Batch([p], prec=gpu.FP32) as b, gpu.Grid(p, prec=gpu.FP32) as g:
        assert b.dt == g.dt
        b.step(300)
        g.step(300)
        b.sync()
        g.sync()
        Vb, Ib = b.port_dfts(0)
        Vg, Ig = g.port_dfts()
    assert np.array_equal(Vb, Vg) and np.array_equal(Ib, Ig)


BOX_DIMS = [(120, 60, 40), (96, 48, 36), (150, 70, 44), (56, 40, 36), (100, 50, 30)]


@pytest.mark.parametrize("tile_y,kseg", [(8, 16), (4, 7)])
def test_two_step_batch_equals_single_grids_bitwise(gpu, tile_y, kseg):
    """Variant 4 for a batch: instances with inner boxes of one to three tile columns, one too
    small for a box and one closed by PEC walls; 151 steps (graph chunks of pairs, direct
    pairs and one single step).  Every instance equals its single-grid variant-4 run bit for bit,
    fields and port spectra."""
    rng = W.SplitMix64(0xB0C5)
    probs = [W.batch_instance(rng, nsteps=151, nfreq=16, dims=d) for d in BOX_DIMS]
    probs[4].bc = (0, 0, 0, 0, 0, 0)
    n = 151
    boxes = []
    with gpu.Batch(probs, prec=gpu.FP32, tile_y=tile_y, kseg=kseg, variant=4) as b:
        b.step(n)
        b.sync()
        got = [b.fields(q) for q in range(len(probs))]
        dft = [b.port_dfts(q) for q in range(len(probs))]
        dt = b.dt
    for q, p in enumerate(probs):
        with gpu.Grid(p, prec=gpu.FP32, dt=dt, variant=4, tile_y=tile_y, kseg=kseg) as g:
            boxes.append(gpu.tb_box(g.h))
            g.step(n)
            g.sync()
            assert np.array_equal(got[q], g.fields()), q
            V, I = g.port_dfts()
            assert np.array_equal(dft[q][0], V) and np.array_equal(dft[q][1], I), q
    assert sum(bx is not None for bx in boxes) >= 3 and boxes[3] is None, boxes


def test_two_step_batch_is_refused_for_fp64_and_after_a_step(gpu):
    rng = W.SplitMix64(0xB0C6)
    probs = [W.batch_instance(rng, nsteps=10, nfreq=8, dims=(96, 48, 36))]
    with gpu.Batch(probs, prec=gpu.FP64) as b:
        with pytest.raises(gpu.YFError):
            b.set_variant(4)
    with gpu.Batch(probs, prec=gpu.FP32) as b:
        b.step(2)
        with pytest.raises(gpu.YFError):
            b.set_variant(4)
        with pytest.raises(gpu.YFError):
            b.set_variant(3)


def test_two_step_batch_after_autotune_equals_single_grids(gpu, tmp_path):
    """The benchmark's order: a variant-4 batch autotuned (its tables rebuilt per tiling, every
    instance reset afterwards), then stepped; each instance still equals its single-grid
    variant-4 run bit for bit at the tiling the tuner chose."""
    rng = W.SplitMix64(0xB0C7)
    probs = [W.batch_instance(rng, nsteps=64, nfreq=8, dims=d) for d in BOX_DIMS[:3]]
    n = 64
    with gpu.Batch(probs, prec=gpu.FP32, variant=4) as b:
        ty, ks = b.autotune(str(tmp_path / "tiles.json"), reps=1)
        for q in range(len(probs)):
            assert not np.any(b.fields(q)), "tuning must leave the fields at zero"
        b.step(n)
        b.sync()
        got = [b.fields(q) for q in range(len(probs))]
        dt = b.dt
    for q, p in enumerate(probs):
        with gpu.Grid(p, prec=gpu.FP32, dt=dt, variant=4, tile_y=ty, kseg=ks) as g:
            g.step(n)
            g.sync()
            assert np.array_equal(got[q], g.fields()), q
