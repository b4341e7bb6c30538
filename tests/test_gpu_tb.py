"""Variant 4 (two time steps per pass over the inner box, FP32) through the C ABI.

The grid is 170 x 70 x 50 nodes with random lossy materials, a PEC block and PEC sheets that
cross the box boundary, CPML on five faces (the ground at z = 0 is PEC), a source plane and
two port planes near the x ends.  Its box is x 32..127, y 16..55, z 0..39: three tile columns,
five tile rows and two z segments of the two-step kernel (32 planes from the ground, then a
ragged 8), surrounded by every kind of single-step frame work.  A second geometry moves a port plane to the middle, which splits the
admissible tile columns (the box takes the longest run of them).

Bars (the FP32 budget used for every variant): fields relative L2 <= 1e-5 against the FP64
oracle at step 61 (odd: a graph chunk, pairs and one single step); port spectra within 1e-4
of their maximum.  Against variant 2 on the GPU, over 600 steps (the pulse crosses the box,
reaches both ports and the absorbing slabs), the same bars.  Graph replay against direct
pairs and checkpoint resume are bitwise."""
import os
import tempfile

import numpy as np
import pytest

from oracle import post, yee
from paper_2208_04371_b300 import workloads as W

pytestmark = pytest.mark.gpu

BOX = (32, 127, 16, 55, 0, 39)


def rel_l2(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def _tb_problem(port_mid=False, ny=70):
    nx, nz = 170, 50
    rng = W.SplitMix64(0x7B2)
    ids = np.array([rng.randint(0, 4) for _ in range(nx * ny * nz)], np.uint8).reshape(nz, ny, nx)
    ids[20:26, 30:38, 60:75] = 5
    p = W.Problem(nx=nx, ny=ny, nz=nz, dx=4e-6, dy=5e-6, dz=3e-6, courant=0.95, ids=ids,
                  eps_r=np.array([1.0, 2.2, 4.0, 9.8, 3.0, 1.0]),
                  sigma=np.array([0.0, 0.5, 0.0, 20.0, 1e4, 0.0]),
                  mu_r=np.ones(6), is_pec=np.array([0, 0, 0, 0, 0, 1], np.uint8),
                  sheets=[(2, 12, 5, 160, 30, 40), (1, 50, 20, 140, 2, 30), (0, 100, 10, 60, 3, 45)],
                  bc=(1, 1, 1, 1, 0, 1), pml_cells=8, pml_order=3, pml_kappa_max=3.0,
                  pml_alpha_max=2e8)
    p.source = W.Source(kind=W.WAVE_DIFF_GAUSS, plane=10, j0=30, j1=40, k0=0, k1=12,
                        amplitude=2.5, param0=3e-14)
    second = 90 if port_mid else 150
    p.ports = [W.Port(plane=16, direction=1, j0=30, j1=40, k0=0, k1=12, kb=12, kt=12, margin=1),
               W.Port(plane=second, direction=-1, j0=30, j1=40, k0=0, k1=12, kb=12, kt=12,
                      margin=2)]
    p.freqs = np.linspace(50e9, 2e12, 37)
    p.nsteps = 600
    return p


@pytest.fixture(scope="module")
def tb_ref():
    p = _tb_problem()
    return p, yee.run(p, nsteps=61, want_fields=True)


def test_box_is_the_documented_one(gpu):
    p = _tb_problem()
    with gpu.Grid(p, prec=gpu.FP32, variant=4) as g:
        assert gpu.tb_box(g.h) == BOX
    with gpu.Grid(_tb_problem(port_mid=True), prec=gpu.FP32, variant=4) as g:
        # admissible tile columns: 1 (x 32..63), then 3 and 4 past the port at x = 90
        assert gpu.tb_box(g.h) == (96, 159, 16, 55, 0, 39)


@pytest.mark.parametrize("tile_y,kseg", [(8, 16), (4, 5), (16, 7), (8, 1), (8, 32)])
def test_variant4_matches_oracle(gpu, tb_ref, tile_y, kseg):
    """Frame tile heights 4, 8, 16 (the box rows align to max(8, tile_y)) and box segments of
    2, 10, 14, 32 and 64 planes (2 kseg, at most 64)."""
    p, ref = tb_ref
    with gpu.Grid(p, prec=gpu.FP32, variant=4, tile_y=tile_y, kseg=kseg) as g:
        box = gpu.tb_box(g.h)
        assert box is not None and (box[2] % max(8, tile_y)) == 0 and (box[3] + 1) % max(8, tile_y) == 0
        g.step(61)
        g.sync()
        f = g.fields()
        V, I = g.port_dfts()
    assert rel_l2(f, ref["fields"]) <= 1e-5
    Vo, Io = post.port_dfts(ref["V"], ref["I"], p.freqs, ref["dt"])
    assert np.max(np.abs(V - Vo)) <= 1e-4 * np.max(np.abs(Vo))
    assert np.max(np.abs(I - Io)) <= 1e-4 * np.max(np.abs(Io))


@pytest.mark.parametrize("port_mid", [False, True])
def test_variant4_matches_variant2_over_a_long_run(gpu, port_mid):
    p = _tb_problem(port_mid)
    out = {}
    for v in (2, 4):
        with gpu.Grid(p, prec=gpu.FP32, variant=v) as g:
            g.step(p.nsteps)
            g.sync()
            out[v] = (g.fields(), *g.port_dfts())
    f2, V2, I2 = out[2]
    f4, V4, I4 = out[4]
    assert rel_l2(f4, f2) <= 1e-5
    assert np.max(np.abs(V4 - V2)) <= 1e-4 * np.max(np.abs(V2))
    assert np.max(np.abs(I4 - I2)) <= 1e-4 * np.max(np.abs(I2))


def test_variant_switches_mid_run(gpu):
    """2 -> 4 -> 2 -> 4 -> 2 with step counts that leave the third buffer current and the
    auxiliary copy out of step with the buffer index; equals variant 2 throughout."""
    p = _tb_problem()
    with gpu.Grid(p, prec=gpu.FP32, variant=2) as a, gpu.Grid(p, prec=gpu.FP32, variant=2) as b:
        a.step(19)
        for v, n in ((2, 5), (4, 4), (2, 3), (4, 5), (2, 2)):
            gpu.set_variant(b.h, v)
            b.step(n)
        a.sync()
        b.sync()
        assert rel_l2(b.fields(), a.fields()) <= 1e-5
        Va, _ = a.port_dfts()
        Vb, _ = b.port_dfts()
    assert np.max(np.abs(Vb - Va)) <= 1e-4 * np.max(np.abs(Va))


def test_graph_chunks_equal_direct_pairs(gpu):
    p = _tb_problem()
    with gpu.Grid(p, prec=gpu.FP32, variant=4) as a, gpu.Grid(p, prec=gpu.FP32, variant=4) as b:
        a.step(77)
        for _ in range(38):
            b.step(2)
        b.step(1)
        assert np.array_equal(a.fields(), b.fields())
        assert np.array_equal(a.port_dfts()[0], b.port_dfts()[0])


@pytest.mark.parametrize("box_ty,box_seg", [(8, 3), (8, 14), (8, 37), (16, 0), (16, 9)])
def test_box_shape_does_not_change_the_fields(gpu, box_ty, box_seg):
    """The box's 40 planes cut into segments of 3 (fourteen segments, the last of one plane),
    14 (a ragged last segment of 12) or 37 (then 3), and blocks 16 rows high (one block per
    SM), against the default (8 rows, 32 planes then 8), on the test grid made
    78 nodes wide so that its box (y 16..63) holds whole tiles of either height: each block
    recomputes its halo from step-n data, so the fields and spectra agree bit for bit, also
    after the shape changes mid-run."""
    p = _tb_problem(ny=78)
    with gpu.Grid(p, prec=gpu.FP32, variant=4) as a, \
            gpu.Grid(p, prec=gpu.FP32, variant=4, box_seg=box_seg, box_ty=box_ty) as b:
        assert gpu.tb_box(a.h) == gpu.tb_box(b.h) == (32, 127, 16, 63, 0, 39)
        a.step(40)
        b.step(40)
        assert np.array_equal(a.fields(), b.fields())
        gpu.set_box_shape(b.h, 0, 0)
        a.step(21)
        b.step(21)
        assert np.array_equal(a.fields(), b.fields())
        assert np.array_equal(a.port_dfts()[0], b.port_dfts()[0])
        assert np.array_equal(a.port_dfts()[1], b.port_dfts()[1])


def test_box_shape_rejects_bad_arguments(gpu):
    p = _tb_problem()
    with gpu.Grid(p, prec=gpu.FP32, variant=4) as g:
        for ty, seg in ((12, 0), (8, -1)):
            with pytest.raises(gpu.YFError) as e:
                gpu.set_box_shape(g.h, ty, seg)
            assert e.value.code == gpu.E_INVALID


def test_launch_count(gpu):
    p = _tb_problem()
    with gpu.Grid(p, prec=gpu.FP32, variant=4) as g:
        pair = gpu.launches(g.h, 2)
        single = gpu.launches(g.h, 1)
        assert gpu.launches(g.h, 77) == 38 * pair + single
        # frame kinds twice, the box kernel, per step the source and the side-stream epilogue
        assert 7 <= pair <= 15 and 2 <= single <= 6


def test_checkpoint_resume_is_bitwise(gpu):
    p = _tb_problem()
    with gpu.Grid(p, prec=gpu.FP32, variant=4) as a:
        a.step(100)
        full = a.fields()
        Va, _ = a.port_dfts()
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "ck.bin")
        with gpu.Grid(p, prec=gpu.FP32, variant=4) as b:
            b.step(50)
            gpu.checkpoint_save(b.h, path)
        with gpu.Grid(p, prec=gpu.FP32, variant=4) as c:
            gpu.checkpoint_load(c.h, path)
            c.step(50)
            assert np.array_equal(c.fields(), full)
            Vc, _ = c.port_dfts()
    assert np.array_equal(Va, Vc)


def test_variant4_rejects_fp64(gpu):
    p = _tb_problem()
    with gpu.Grid(p, prec=gpu.FP64) as g:
        with pytest.raises(gpu.YFError):
            gpu.set_variant(g.h, 4)


def test_lossy_line_variant4_matches_variant2_at_full_size(gpu):
    """The 768 x 384 x 256 lossy line (the timed workload) over 64 steps: the two-step path
    against the one-step path, fields and port spectra within the FP32 budget."""
    p = W.config_lossy_line(nsteps=64)
    out = {}
    for v in (2, 4):
        with gpu.Grid(p, prec=gpu.FP32, variant=v) as g:
            if v == 4:
                assert gpu.tb_box(g.h) == (32, 735, 16, 367, 0, 241)
            g.step(64)
            g.sync()
            out[v] = (g.fields(), *g.port_dfts())
    f2, V2, I2 = out[2]
    f4, V4, I4 = out[4]
    assert rel_l2(f4, f2) <= 1e-5
    assert np.max(np.abs(V4 - V2)) <= 1e-4 * np.max(np.abs(V2))


def test_grid_without_a_box_steps_exactly_like_variant2(gpu):
    """A grid too small for a box: every pair is two whole-grid one-step passes, the same
    launches as variant 2, so the fields agree bit for bit."""
    p = _tb_problem()
    p.nx = 60
    p.ids = p.ids[:, :, :60].copy()
    p.sheets = [(2, 12, 5, 50, 30, 40)]
    p.ports = [W.Port(plane=16, direction=1, j0=30, j1=40, k0=0, k1=12, kb=12, kt=12, margin=1),
               W.Port(plane=44, direction=-1, j0=30, j1=40, k0=0, k1=12, kb=12, kt=12, margin=1)]
    out = {}
    for v in (2, 4):
        with gpu.Grid(p, prec=gpu.FP32, variant=v) as g:
            if v == 4:
                assert gpu.tb_box(g.h) is None
            g.step(37)
            g.sync()
            out[v] = g.fields()
    assert np.array_equal(out[2], out[4])



def test_pec_cavity_variant4_matches_variant2(gpu):
    """A closed lossless PEC cavity (no CPML, source or ports) from seeded random fields: the
    box then reaches three nodes from every wall but the one at z = 0, where it starts.  200
    steps, two-step path against one-step."""
    nx, ny, nz = 100, 60, 40
    p = W.Problem(nx=nx, ny=ny, nz=nz, dx=1e-3, dy=0.8e-3, dz=1.1e-3, courant=0.95,
                  ids=np.zeros((nz, ny, nx), np.uint8), eps_r=np.array([1.0]),
                  sigma=np.array([0.0]), mu_r=np.array([1.0]), is_pec=np.array([0], np.uint8),
                  bc=(0,) * 6, pml_cells=0)
    f0 = W.uniform_array(0xCAB, 6 * (nz + 1) * (ny + 1) * (nx + 1), -1.0, 1.0).reshape(
        6, nz + 1, ny + 1, nx + 1)
    out = {}
    for v in (2, 4):
        with gpu.Grid(p, prec=gpu.FP32, variant=v) as g:
            if v == 4:
                assert gpu.tb_box(g.h) == (32, 95, 8, 55, 0, 37)
            g.set_fields(f0)
            g.step(200)
            g.sync()
            out[v] = g.fields()
    assert rel_l2(out[4], out[2]) <= 1e-5


@pytest.mark.parametrize("variant", [2, 4])
def test_reset_and_new_materials_resolve_bitwise(gpu, variant):
    """yf_reset, yf_set_materials from host memory (pageable, then pinned) and the PEC sheets
    again: a solve with other materials between two solves of the same problem leaves the
    third solve equal to the first bit for bit (fields and spectra), the path a re-solving
    caller takes.  The second solve differs from both."""
    import torch
    p = _tb_problem()
    ids_b = p.ids.copy()
    ids_b[10:30, 20:40, 50:90] = 3
    runs = []
    with gpu.Grid(p, prec=gpu.FP32, variant=variant) as g:
        for q, ids in enumerate((p.ids, ids_b, torch.from_numpy(p.ids).pin_memory())):
            if q > 0:
                gpu.reset(g.h)
                gpu.set_materials(g.h, ids, p.eps_r, p.sigma, p.mu_r, p.is_pec)
                for sh in p.sheets:
                    gpu.add_pec_sheet(g.h, *sh)
            g.step(61)
            g.sync()
            runs.append((g.fields(), *g.port_dfts()))
    assert np.array_equal(runs[2][0], runs[0][0])
    assert np.array_equal(runs[2][1], runs[0][1]) and np.array_equal(runs[2][2], runs[0][2])
    assert not np.array_equal(runs[1][0], runs[0][0])


def test_single_tile_box_matches_variant2(gpu):
    """A 67 x 19 x 20 closed PEC cavity from seeded random fields: its box is one 32 x 8 tile
    (x 32..63, y 8..15, z 0..17), so a single block writes the outer node layer on all four
    sides and both z faces.  301 steps (150 pairs and one single step), two-step path against
    one-step within the FP32 budget."""
    nx, ny, nz = 67, 19, 20
    p = W.Problem(nx=nx, ny=ny, nz=nz, dx=1e-3, dy=0.9e-3, dz=1.2e-3, courant=0.95,
                  ids=np.zeros((nz, ny, nx), np.uint8), eps_r=np.array([1.0]),
                  sigma=np.array([0.0]), mu_r=np.array([1.0]), is_pec=np.array([0], np.uint8),
                  bc=(0,) * 6, pml_cells=0)
    f0 = W.uniform_array(0x1713, 6 * (nz + 1) * (ny + 1) * (nx + 1), -1.0, 1.0).reshape(
        6, nz + 1, ny + 1, nx + 1)
    out = {}
    for v in (2, 4):
        with gpu.Grid(p, prec=gpu.FP32, variant=v) as g:
            if v == 4:
                assert gpu.tb_box(g.h) == (32, 63, 8, 15, 0, 17)
            g.set_fields(f0)
            g.step(301)
            g.sync()
            out[v] = g.fields()
    assert rel_l2(out[4], out[2]) <= 1e-5


def test_variant4_refuses_grids_beyond_its_32_bit_offsets(gpu):
    """The two-step kernel addresses a buffer's six components with 32-bit offsets, so a grid
    of more than (2^31 - 1) / 6 padded points is refused with YF_E_INVALID at its first step,
    before any launch, and the context stays usable.  1023 x 511 x 682 cells are 1024 x 512 x
    683 padded points: 6 x 358.1 M = 2.1485e9, just above 2^31 - 1 (the fields take 26 GB)."""
    h = gpu.grid_create(1023, 511, 682, 1e-6, 1e-6, 1e-6, prec=gpu.FP32)
    try:
        gpu.set_variant(h, 4, 8, 32)
        with pytest.raises(gpu.YFError) as e:
            gpu.step(h, 2)
        assert e.value.code == gpu.E_INVALID
    finally:
        gpu.grid_destroy(h)
    with gpu.Grid(_tb_problem(), prec=gpu.FP32, variant=4) as g:
        g.step(3)
        g.sync()
        assert np.isfinite(g.fields()).all()
