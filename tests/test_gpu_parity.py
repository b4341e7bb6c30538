"""GPU parity: the CUDA library (through the C ABI) against the FP64 CPU oracle.

Tolerances:
  FP64 fields      relative L2 over all six components <= 1e-12 after 2000 steps (the
                   two sides differ only in the rounding order of the same FP64 operations)
  FP64 port DFTs   relative (to the spectrum's max)    <= 1e-10
  FP32 fields      relative L2                         <= 1e-5 (unit roundoff 6e-8 times the
                   steps the error has grown over, with a margin)
  FP32 |S_ij|      absolute                            <= 1e-3
"""
import math
import os
import tempfile

import numpy as np
import pytest

from oracle import post, yee
from paper_2208_04371_b300 import workloads as W

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


@pytest.fixture(scope="module")
def small_fp64_ref():
    p = W.config_small_fp64()
    return p, yee.run(p, want_fields=True)


def test_small_microstrip_fp64_fields_and_dfts(gpu, small_fp64_ref):
    p, ref = small_fp64_ref
    with gpu.Grid(p, prec=gpu.FP64) as g:
        assert g.dt == pytest.approx(ref["dt"], rel=1e-15)
        g.step(p.nsteps)
        g.sync()
        f = g.fields()
        V, I = g.port_dfts()
    assert rel_l2(f, ref["fields"]) <= 1e-12
    Vo, Io = post.port_dfts(ref["V"], ref["I"], p.freqs, ref["dt"])
    for q in range(2):
        assert np.max(np.abs(V[q] - Vo[q])) <= 1e-10 * np.max(np.abs(Vo[q]))
        assert np.max(np.abs(I[q] - Io[q])) <= 1e-10 * np.max(np.abs(Io[q]))


def test_small_microstrip_fp32_within_budget(gpu, small_fp64_ref):
    """FP32 fields: relative L2 <= 1e-5 at the pulse peak (step 1000, t = t0), and at step
    2000 the error norm stays below 1e-5 of the run's field scale (the peak-time norm).
    By step 2000 the pulse has left through the PML and the remaining tail is ~140x smaller
    than the peak, so a ratio to the tail alone would measure the tail, not FP32."""
    p, ref = small_fp64_ref
    ref_mid = yee.run(p, nsteps=1000, want_fields=True)["fields"]
    with gpu.Grid(p, prec=gpu.FP32) as g:
        g.step(1000)
        f_mid = g.fields()
        g.step(p.nsteps - 1000)
        g.sync()
        f = g.fields()
        sp = gpu.read_sparams(g.h, len(p.freqs))
    assert rel_l2(f_mid, ref_mid) <= 1e-5
    scale = np.linalg.norm(ref_mid.ravel())
    assert np.linalg.norm((f - ref["fields"]).ravel()) / scale <= 1e-5
    Vo, Io = post.port_dfts(ref["V"], ref["I"], p.freqs, ref["dt"])
    So, Zo = post.sstar_uniform(Vo, Io, [1, -1])
    Sno = post.renormalize(So, Zo)
    assert np.max(np.abs(np.abs(sp["S_star"]) - np.abs(So))) <= 1e-3
    assert np.max(np.abs(np.abs(sp["S"]) - np.abs(Sno))) <= 1e-3


def test_sparams_kernel_matches_oracle_postprocessing(gpu, small_fp64_ref):
    """Uniform-line extraction on the GPU (FP64) vs the oracle's numpy route, same inputs."""
    p, ref = small_fp64_ref
    Vo, Io = post.port_dfts(ref["V"], ref["I"], p.freqs, ref["dt"])
    So, Zo = post.sstar_uniform(Vo, Io, [1, -1])
    Sn = post.renormalize(So, Zo)
    zc = post.zc_from_sstar(So, Zo)
    tau = post.phase_delay(So[:, 1, 0], p.freqs)
    r = gpu.sparams(p.freqs, np.array([Vo[0], Vo[1]]), np.array([Io[0], -Io[1]]),
                    np.zeros((2, 2, len(p.freqs)), complex))
    # the full-protocol call with V_tot = 0 gives S*_jj = -1; check Z_r there, then the
    # uniform-line call through a grid for the rest
    assert np.max(np.abs(r["Zr"] - Zo) / np.abs(Zo)) < 1e-13
    with gpu.Grid(p, prec=gpu.FP64) as g:
        g.step(p.nsteps)
        u = gpu.read_sparams(g.h, len(p.freqs))
    assert np.max(np.abs(u["S_star"] - So)) < 1e-10
    assert np.max(np.abs(u["S"] - Sn)) < 1e-10
    assert np.max(np.abs(u["Zc"] - zc) / np.abs(zc)) < 1e-9
    assert np.max(np.abs(u["tau"][:, 1, 0] - tau) / np.abs(tau)) < 1e-9


def test_full_protocol_sparams_kernel_vs_oracle(gpu):
    """Eq. 1, 2, 5-6, 8 on synthetic three-port spectra: GPU FP64 kernel vs numpy oracle."""
    rng = np.random.default_rng(5)
    N, F = 3, 40
    freqs = np.linspace(1e9, 40e9, F)
    Vi = rng.normal(size=(N, F)) + 1j * rng.normal(size=(N, F))
    Ii = Vi / (np.array([[30.0], [55.0], [80.0]]) + 1j * rng.normal(size=(N, F)))
    Vt = Vi[:, None, :] * (0.3 * (rng.normal(size=(N, N, F)) + 1j * rng.normal(size=(N, N, F))))
    So, Zo = post.sstar(Vi, Ii, Vt)
    Sn = post.renormalize(So, Zo)
    r = gpu.sparams(freqs, Vi, Ii, Vt)
    assert np.max(np.abs(r["S_star"] - So)) < 1e-12 * np.max(np.abs(So))
    assert np.max(np.abs(r["Zr"] - Zo)) < 1e-12 * np.max(np.abs(Zo))
    assert np.max(np.abs(r["S"] - Sn)) < 1e-11 * np.max(np.abs(Sn))


def _ragged_problem():
    """Ragged grid (no axis a multiple of 32), PML on five faces, random lossy materials,
    a PEC block, sheets on all three normals, a differential-Gaussian source."""
    nx, ny, nz = 45, 37, 29
    rng = W.SplitMix64(99)
    ids = np.array([rng.randint(0, 4) for _ in range(nx * ny * nz)], np.uint8).reshape(nz, ny, nx)
    ids[10:14, 15:20, 20:25] = 5
    p = W.Problem(nx=nx, ny=ny, nz=nz, dx=4e-6, dy=5e-6, dz=3e-6, courant=0.95, ids=ids,
                  eps_r=np.array([1.0, 2.2, 4.0, 9.8, 3.0, 1.0]),
                  sigma=np.array([0.0, 0.5, 0.0, 20.0, 1e4, 0.0]),
                  mu_r=np.ones(6), is_pec=np.array([0, 0, 0, 0, 0, 1], np.uint8),
                  sheets=[(2, 9, 5, 40, 15, 22), (1, 30, 3, 20, 4, 12), (0, 35, 10, 20, 3, 9)],
                  bc=(1, 1, 1, 1, 0, 1), pml_cells=6, pml_order=3, pml_kappa_max=3.0,
                  pml_alpha_max=2e8)
    p.source = W.Source(kind=W.WAVE_DIFF_GAUSS, plane=9, j0=15, j1=22, k0=0, k1=9,
                        amplitude=2.5, param0=3e-14)
    p.ports = [W.Port(plane=14, direction=1, j0=15, j1=22, k0=0, k1=9, kb=9, kt=9, margin=1),
               W.Port(plane=30, direction=-1, j0=15, j1=22, k0=0, k1=9, kb=9, kt=9, margin=2)]
    p.freqs = np.linspace(50e9, 2e12, 37)
    p.nsteps = 600
    return p


@pytest.fixture(scope="module")
def ragged_ref():
    p = _ragged_problem()
    return p, yee.run(p, want_fields=True)


@pytest.mark.parametrize("variant,tile_y,kseg", [(0, 8, 64), (1, 8, 64), (1, 4, 5), (1, 16, 7),
                                                 (2, 8, 64), (2, 4, 5), (2, 16, 7), (2, 8, 1),
                                                 (3, 8, 64), (3, 4, 5), (3, 16, 7), (3, 8, 1),
                                                 (3, 4, 2)])
def test_ragged_lossy_grid_fp64_parity(gpu, ragged_ref, variant, tile_y, kseg):
    """Reference and fused kernels, several tiles and z-segment lengths (segment starts
    recompute the plane below), against the oracle on a ragged lossy grid."""
    p, ref = ragged_ref
    with gpu.Grid(p, prec=gpu.FP64, variant=variant, tile_y=tile_y, kseg=kseg) as g:
        g.step(p.nsteps)
        g.sync()
        f = g.fields()
        V, I = g.port_dfts()
    assert rel_l2(f, ref["fields"]) <= 1e-12
    Vo, Io = post.port_dfts(ref["V"], ref["I"], p.freqs, ref["dt"])
    assert np.max(np.abs(V - Vo)) <= 1e-10 * np.max(np.abs(Vo))
    assert np.max(np.abs(I - Io)) <= 1e-10 * np.max(np.abs(Io))


def test_cavity_mode_on_gpu_follows_dispersion(gpu):
    """Exact discrete eigenmode written in through the ABI; FP64 GPU evolution matches the
    Yee dispersion closed form to roundoff."""
    nx, ny, nz, d = 20, 16, 12, 1e-3
    p = W.Problem(nx=nx, ny=ny, nz=nz, dx=d, dy=d, dz=d, courant=0.9,
                  ids=np.zeros((nz, ny, nx), np.uint8), eps_r=np.array([1.0]),
                  sigma=np.array([0.0]), mu_r=np.array([1.0]), is_pec=np.array([0], np.uint8),
                  bc=(0,) * 6, pml_cells=0)
    K, J, I = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    m, n = 3, 2
    shape = np.sin(m * math.pi * I / nx) * np.sin(n * math.pi * J / ny) * (K < nz)
    f0 = np.zeros((6, nz + 1, ny + 1, nx + 1))
    f0[2] = shape
    lam = sum((2 / d * math.sin(q * math.pi / (2 * N))) ** 2 for q, N in ((m, nx), (n, ny)))
    N = 500
    with gpu.Grid(p, prec=gpu.FP64) as g:
        g.set_fields(f0)
        g.step(N)
        out = g.fields()
        dt = g.dt
    c2 = 1.0 / (yee.MU0 * yee.EPS0)
    gg = dt * dt * c2 * lam
    th = math.acos(1 - gg / 2)
    aN = math.cos(N * th) + (1 - gg - math.cos(th)) / math.sin(th) * math.sin(N * th)
    assert np.max(np.abs(out[2] - aN * shape)) < 2e-12


def test_dft_accumulator_variants_agree(gpu):
    p = W.config_small_fp64()
    with gpu.Grid(p, prec=gpu.FP32, dft_mask=gpu.DFT_FP64 | gpu.DFT_KAHAN32 | gpu.DFT_FP32) as g:
        g.step(p.nsteps)
        V64, I64 = g.port_dfts(gpu.DFT_FP64)
        Vk, Ik = g.port_dfts(gpu.DFT_KAHAN32)
        V32, I32 = g.port_dfts(gpu.DFT_FP32)
    scale = np.max(np.abs(V64))
    assert np.max(np.abs(Vk - V64)) < 1e-6 * scale
    assert np.max(np.abs(V32 - V64)) < 1e-4 * scale


@pytest.mark.parametrize("variant,tile_y", [(0, 8), (1, 8), (2, 4), (2, 8), (2, 16), (3, 4),
                                            (3, 8), (3, 16)])
def test_fp32_variants_match_oracle_while_pulse_is_inside(gpu, ragged_ref, variant, tile_y):
    """Every FP32 kernel variant against the FP64 oracle at step 40 (the Eq. 3 pulse peaks at
    step 13 here, so the fields are still large): relative L2 <= 1e-5."""
    p, _ = ragged_ref
    ref = yee.run(p, nsteps=40, want_fields=True)["fields"]
    with gpu.Grid(p, prec=gpu.FP32, variant=variant, tile_y=tile_y, kseg=9) as g:
        g.step(40)
        g.sync()
        f = g.fields()
    assert rel_l2(f, ref) <= 1e-5


def test_graph_chunks_equal_single_steps(gpu):
    p = W.config_small_fp64()
    with gpu.Grid(p, prec=gpu.FP32) as a, gpu.Grid(p, prec=gpu.FP32) as b:
        a.step(77)
        for _ in range(77):
            b.step(1)
        assert np.array_equal(a.fields(), b.fields())
        assert gpu.steps_done(a.h) == 77


def test_checkpoint_resume_is_bitwise(gpu):
    p = _ragged_problem()
    with gpu.Grid(p, prec=gpu.FP32) as a:
        a.step(400)
        full = a.fields()
        Va, Ia = a.port_dfts()
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "ck.bin")
        with gpu.Grid(p, prec=gpu.FP32) as b:
            b.step(200)
            gpu.checkpoint_save(b.h, path)
        with gpu.Grid(p, prec=gpu.FP32) as c:
            gpu.checkpoint_load(c.h, path)
            c.step(200)
            assert np.array_equal(c.fields(), full)
            Vc, Ic = c.port_dfts()
    assert np.array_equal(Va, Vc) and np.array_equal(Ia, Ic)


def test_energy_monitor_matches_definition(gpu):
    """yf_energy on written fields equals sum eps E^2 + mu0 H^2 over live entries."""
    p = _ragged_problem()
    p.bc = (0,) * 6
    f = W.random_fields((p.nz + 1, p.ny + 1, p.nx + 1), seed=4)
    with gpu.Grid(p, prec=gpu.FP64, with_source=False, with_ports=False) as g:
        g.set_fields(f)
        got = gpu.energy(g.h)
        live = g.fields()
    # eps per E edge from the oracle's averaging rule, via an oracle run of 0 steps is not
    # available; use the live (sanitised) fields and the edge-average rule directly
    ids, er = p.ids, p.eps_r
    nz, ny, nx = ids.shape
    e = np.zeros(3)
    w = 0.0
    def cell(i, j, k):
        return er[ids[k, j, i]]
    for comp in range(3):
        arr = live[comp]
        ks, js, is_ = np.nonzero(arr)
        for k, j, i in zip(ks, js, is_):
            if comp == 0:
                cs = [(i, j - 1, k - 1), (i, j, k - 1), (i, j - 1, k), (i, j, k)]
            elif comp == 1:
                cs = [(i - 1, j, k - 1), (i, j, k - 1), (i - 1, j, k), (i, j, k)]
            else:
                cs = [(i - 1, j - 1, k), (i, j - 1, k), (i - 1, j, k), (i, j, k)]
            eps = sum(cell(*c) for c in cs) / 4.0 * yee.EPS0
            w += eps * arr[k, j, i] ** 2
    w += yee.MU0 * np.sum(live[3:] ** 2)
    w *= p.dx * p.dy * p.dz
    assert got == pytest.approx(w, rel=1e-12)


def test_nonfinite_port_sample_reports_unstable(gpu):
    p = W.config_small_fp64()
    with gpu.Grid(p, prec=gpu.FP32) as g:
        f = np.zeros((6, p.nz + 1, p.ny + 1, p.nx + 1))
        f[2, 3, 16, 14] = np.inf            # on port 1's V surface
        g.set_fields(f)
        g.step(1)
        with pytest.raises(gpu.YFError) as e:
            g.sync()
        assert e.value.code == gpu.E_UNSTABLE


def test_state_and_argument_errors(gpu):
    p = W.config_small_fp64()
    with gpu.Grid(p, prec=gpu.FP32) as g:
        with pytest.raises(gpu.YFError) as e:
            gpu.add_port(g.h, 0, 1, 13, 19, 0, 8, 8, 8, 1, p.freqs)
        assert e.value.code == gpu.E_INVALID
        g.step(1)
        with pytest.raises(gpu.YFError) as e:
            gpu.add_port(g.h, 20, 1, 13, 19, 0, 8, 8, 8, 1, p.freqs)
        assert e.value.code == gpu.E_STATE
    with pytest.raises(gpu.YFError) as e:
        bad = W.config_small_fp64()
        bad.mu_r = np.array([1.0, 2.0])
        gpu.Grid(bad)
    assert e.value.code == gpu.E_UNSUPPORTED


def _subbox_check(f0, f1, prob, box, nsteps, dt, tol):
    """Oracle on a sub-box seeded with the GPU's state at step n0 (f0, the box's nodes) for
    nsteps; compare the points farther than nsteps + 1 cells from every sub-box face (outside
    the dependency cone of the box boundary) with the GPU state f1 after those steps."""
    (x0, x1), (y0, y1), (z0, z1) = box
    sub = W.Problem(nx=x1 - x0, ny=y1 - y0, nz=z1 - z0, dx=prob.dx, dy=prob.dy, dz=prob.dz,
                    courant=prob.courant, ids=np.ascontiguousarray(prob.ids[z0:z1, y0:y1, x0:x1]),
                    eps_r=prob.eps_r, sigma=prob.sigma, mu_r=prob.mu_r, is_pec=prob.is_pec,
                    sheets=[], bc=(0,) * 6, pml_cells=0)
    r = yee.run(sub, nsteps=nsteps, dt=dt, fields_in=np.ascontiguousarray(f0), want_fields=True)
    m = nsteps + 2
    got = f1[:, m:-m, m:-m, m:-m]
    want = r["fields"][:, m:-m, m:-m, m:-m]
    scale = np.max(np.abs(want))
    assert scale > 0
    err = np.max(np.abs(got - want)) / scale
    assert err <= tol, err


@pytest.mark.parametrize("variant,kseg,box_seg", [(4, 32, 256), (2, 16, 0)])
def test_full_size_lossy_line_sampled_parity(gpu, variant, kseg, box_seg):
    """The 768x384x256 lossy line (FP32, the benchmark workload), in the benchmark's launch
    configuration (two steps per pass over the inner box, one box segment per tile column) and
    on the one-step path: after 120 steps, 8 more GPU steps agree element-wise with the oracle
    run on a sub-box seeded with the GPU state.  The sub-box (x 22..70) straddles the CPML frame
    and the inner box (from x = 32), around the strip, the oxide layers and the Si."""
    p = W.config_lossy_line(nsteps=0)
    j0, j1 = p.ports[0].j0, p.ports[0].j1
    box = ((22, 70), ((j0 + j1) // 2 - 30, (j0 + j1) // 2 + 30), (170, 226))
    with gpu.Grid(p, prec=gpu.FP32, variant=variant, kseg=kseg, box_seg=box_seg) as g:
        if variant == 4:
            assert gpu.tb_box(g.h) == (32, 735, 16, 367, 0, 241)
        g.step(120)
        f0 = g.fields(box)
        g.step(8)
        f1 = g.fields(box)
        dt = g.dt
    _subbox_check(f0, f1, p, box, 8, dt, 2e-5)


def test_rlcg_kernel_matches_oracle_on_synthetic_lines(gpu):
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    from test_oracle_post import _line_sstar
    cases = [(np.linspace(0.1e9, 20e9, 64), (5.0, 3.0e-7, 1.0e-3, 1.2e-10), 0.05, (40.0, 60.0)),
             (np.linspace(0.2e9, 30e9, 80), (0.0, 2.5e-7, 0.0, 1.0e-10), 0.083, (50.0, 50.0))]
    for freqs, (R, L, G, C), length, zr in cases:
        S = _line_sstar(R, L, G, C, length, freqs, np.array(zr))
        Zr = np.repeat(np.array(zr, dtype=complex)[:, None], len(freqs), axis=1)
        got = gpu.rlcg(freqs, S, Zr, length)
        ref = post.rlcg(S, Zr, freqs, length)
        w = 2 * np.pi * freqs
        ok = np.isfinite(ref["L"])                 # both give NaN where S* -> Z is singular
        assert np.array_equal(ok, np.isfinite(got["L"])) and ok.sum() >= len(freqs) - 2
        # R and G are small real parts of gamma Z_c and gamma / Z_c (cancellation against
        # w L, w C), and the S* -> Z -> ABCD route loses digits in proportion to
        # 1 / |sinh(gamma l)| (singular at beta l = m pi).  With CUDA's FP64 log/atan2/hypot
        # and fused multiply-adds the two implementations agree to about 1e-8 of the natural
        # scales (measured: gamma 4e-10 relative, R 1e-8 of w L): bound 1e-7 x condition
        tol = 1e-7 / np.maximum(np.abs(np.sinh(ref["gamma"][ok] * length)), 1e-3)
        assert np.all(np.abs(got["L"][ok] - ref["L"][ok]) <= tol * L)
        assert np.all(np.abs(got["C"][ok] - ref["C"][ok]) <= tol * C)
        assert np.all(np.abs(got["R"][ok] - ref["R"][ok]) <= tol * w[ok] * L)
        assert np.all(np.abs(got["G"][ok] - ref["G"][ok]) <= tol * w[ok] * C)
        assert np.all(np.abs(got["gamma"][ok] - ref["gamma"][ok]) <= tol * np.abs(ref["gamma"][ok]))


def test_full_size_lossy_line_whole_grid_parity_in_the_benchmark_configuration(gpu):
    """The benchmark itself, checked everywhere: the 768x384x256 lossy line for 128 steps (two
    graph chunks of the benchmark's 64) on its path (two steps per pass over the inner box,
    kseg 32, one box segment per tile column, the port epilogue on a side stream) against the
    FP64 oracle over the whole grid (16 GB of host memory, about half a minute on the host's
    cores): all six fields within the FP32 budget of 1e-5 relative L2, and the port spectra
    within 1e-4 of their maximum."""
    p = W.config_lossy_line(nsteps=128)
    ref = yee.run(p, want_fields=True)
    with gpu.Grid(p, prec=gpu.FP32, variant=4, kseg=32, box_seg=256) as g:
        assert gpu.tb_box(g.h) == (32, 735, 16, 367, 0, 241)
        g.step(64)
        g.step(64)
        g.sync()
        f = g.fields()
        V, I = g.port_dfts()
    assert rel_l2(f, ref["fields"]) <= 1e-5
    Vo, Io = post.port_dfts(ref["V"], ref["I"], p.freqs, ref["dt"])
    assert np.max(np.abs(V - Vo)) <= 1e-4 * np.max(np.abs(Vo))
    assert np.max(np.abs(I - Io)) <= 1e-4 * np.max(np.abs(Io))
