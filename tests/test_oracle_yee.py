"""Pins of the FP64 Yee oracle against closed forms, invariants and the paper's numbers.

None of these compare the oracle with itself: each checks it against something
the mathematics or the paper fixes (discrete eigenmodes, the energy invariant,
the Courant limit, printed worked numbers, brute-force long-domain references).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import post, yee
from paper_2208_04371_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_worked_numbers.json")


def _cavity(nx, ny, nz, dx, dy, dz, eps_r=1.0, courant=0.9):
    return W.Problem(nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz, courant=courant,
                     ids=np.zeros((nz, ny, nx), np.uint8), eps_r=np.array([eps_r]),
                     sigma=np.array([0.0]), mu_r=np.array([1.0]),
                     is_pec=np.array([0], np.uint8), bc=(0,) * 6, pml_cells=0)


# ---------------------------------------------------------------- paper's printed numbers

def test_cfl_timestep_matches_paper():
    g = json.load(open(GOLDEN))
    for case in g["cfl_dt"]:
        dt = yee.courant_dt(case["dx"], case["dy"], case["dz"], case["courant"])
        # the paper prints 3 significant digits
        assert dt == pytest.approx(case["dt"], rel=0.5 * 10 ** (1 - case["printed_digits"]) * 1.01)


def test_diff_gauss_spectrum_peaks_at_printed_frequency():
    """Eq. 3 pulse sampled by the oracle: its DFT magnitude peaks at the f_p the paper
    prints for each sigma (Sec. II-B, Sec. III, Appendix)."""
    g = json.load(open(GOLDEN))
    for case in g["pulse_peak"]:
        sg = case["sigma"]
        prob = _cavity(4, 4, 4, 1e-3, 1e-3, 1e-3)
        prob.source = W.Source(kind=W.WAVE_DIFF_GAUSS, param0=sg)
        dt = sg / 64.0
        n = 12 * 64
        s = yee.waveform_samples(prob, n, dt=dt)
        fp = case["f_peak"]
        freqs = np.linspace(0.5 * fp, 1.5 * fp, 4001)
        spec = np.abs(post.dft(s, freqs, (np.arange(n) + 1.0) * dt, dt))
        f_est = freqs[np.argmax(spec)]
        tol = 0.5 * 10 ** (math.floor(math.log10(fp)) - case["printed_digits"] + 1)
        assert abs(f_est - fp) <= tol + (freqs[1] - freqs[0]), (f_est, fp)


def test_diff_gauss_matches_closed_form_transform():
    """DFT of the sampled Eq. 3 pulse vs its continuous transform
    sigma (j 2 pi f) sqrt(pi) sigma exp(-(pi sigma f)^2) exp(-j 2 pi f t0)."""
    sg = 2e-12
    prob = _cavity(4, 4, 4, 1e-3, 1e-3, 1e-3)
    prob.source = W.Source(kind=W.WAVE_DIFF_GAUSS, param0=sg, t0=6 * sg)
    dt = sg / 40.0
    n = 12 * 40
    s = yee.waveform_samples(prob, n, dt=dt)
    freqs = np.linspace(5e9, 3.0 / (math.sqrt(2) * math.pi * sg), 50)
    got = post.dft(s, freqs, (np.arange(n) + 1.0) * dt, dt)
    t0 = 6 * sg
    want = sg * (2j * math.pi * freqs) * math.sqrt(math.pi) * sg * \
        np.exp(-(math.pi * sg * freqs) ** 2) * np.exp(-2j * math.pi * freqs * t0)
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 1e-9


def test_gauss_sine_band_edges_one_over_e():
    """Gaussian-modulated sine reading: tau = 2/(pi bw) puts the amplitude spectrum at
    1/e of its centre value at f0 +- bw/2 (closed-form transform of the sampled pulse)."""
    f0, bw = 300e9, 200e9
    prob = _cavity(4, 4, 4, 1e-3, 1e-3, 1e-3)
    prob.source = W.Source(kind=W.WAVE_GAUSS_SINE, param0=f0, param1=bw)
    tau = 2.0 / (math.pi * bw)
    dt = tau / 200.0
    n = int(8 * tau / dt)
    s = yee.waveform_samples(prob, n, dt=dt)
    freqs = np.array([f0 - bw / 2, f0, f0 + bw / 2])
    spec = np.abs(post.dft(s, freqs, (np.arange(n) + 1.0) * dt, dt))
    exact = tau * math.sqrt(math.pi) / 2 * (np.exp(-(math.pi * tau * (freqs - f0)) ** 2)
                                            - np.exp(-(math.pi * tau * (freqs + f0)) ** 2))
    assert np.allclose(spec, np.abs(exact), rtol=2e-3)
    assert spec[0] / spec[1] == pytest.approx(math.exp(-1), rel=1e-2)


def test_dft_of_bin_sinusoid_is_geometric_sum():
    """Direct-summation DFT of cos(2 pi f0 t_n) at f0 equals the closed geometric sum."""
    dt, n, f0 = 1e-12, 997, 37.0 / (997 * 1e-12)
    t = (np.arange(n) + 1.0) * dt
    x = np.cos(2 * math.pi * f0 * t)
    got = post.dft(x, np.array([f0]), t, dt)[0]
    # sum cos(a n') e^{-j a n'} = n/2 + 1/2 sum e^{-2 j a n'},  n' = 1..n
    a = 2 * math.pi * f0 * dt
    r = np.exp(-2j * a)
    geo = r * (1 - r ** n) / (1 - r)
    want = (n / 2.0 + 0.5 * geo) * dt
    assert abs(got - want) < 1e-12 * abs(want)


# ---------------------------------------------------------------- discrete cavity eigenmodes

def _mode_amplitude(lam, dt, eps, nsteps):
    """E^N / E^0 for an eigenmode with H^{-1/2} = 0:  a_0 = 1, a_1 = 1 - dt^2 c^2 lam,
    a_{n+1} = 2 cos(theta) a_n - a_{n-1},  cos(theta) = 1 - dt^2 c^2 lam / 2."""
    c2 = 1.0 / (yee.MU0 * yee.EPS0 * eps)
    g = dt * dt * c2 * lam
    th = math.acos(1.0 - g / 2.0)
    a1 = 1.0 - g
    A, B = 1.0, (a1 - math.cos(th)) / math.sin(th)
    return A * math.cos(nsteps * th) + B * math.sin(nsteps * th), th


@pytest.mark.parametrize("comp", ["ez", "ex", "ey"])
def test_cavity_eigenmode_follows_yee_dispersion(comp):
    """A single discrete PEC-cavity mode evolves with sin(w dt/2)/(c dt) =
    sqrt(sum_a (sin(k_a d_a / 2)/d_a)^2): the Yee dispersion relation, to roundoff."""
    nx, ny, nz = 10, 8, 6
    dx, dy, dz = 1.0e-3, 1.3e-3, 0.8e-3
    eps = 2.0
    prob = _cavity(nx, ny, nz, dx, dy, dz, eps_r=eps, courant=0.95)
    dt = yee.courant_dt(dx, dy, dz, 0.95)
    f = np.zeros((6, nz + 1, ny + 1, nx + 1))
    K, J, I = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    if comp == "ez":          # E_z(i, j, k+1/2) = sin(m pi i/nx) sin(n pi j/ny), all k < nz
        m, n = 2, 3
        shape = np.sin(m * math.pi * I / nx) * np.sin(n * math.pi * J / ny) * (K < nz)
        lam = (2 / dx * math.sin(m * math.pi / (2 * nx))) ** 2 + (2 / dy * math.sin(n * math.pi / (2 * ny))) ** 2
        kc2 = (m * math.pi / (nx * dx)) ** 2 + (n * math.pi / (ny * dy)) ** 2
        c = 2
    elif comp == "ex":        # E_x(i+1/2, j, k) = sin(n pi j/ny) sin(p pi k/nz), all i < nx
        n, p = 1, 2
        shape = np.sin(n * math.pi * J / ny) * np.sin(p * math.pi * K / nz) * (I < nx)
        lam = (2 / dy * math.sin(n * math.pi / (2 * ny))) ** 2 + (2 / dz * math.sin(p * math.pi / (2 * nz))) ** 2
        kc2 = (n * math.pi / (ny * dy)) ** 2 + (p * math.pi / (nz * dz)) ** 2
        c = 0
    else:                     # E_y(i, j+1/2, k) = sin(m pi i/nx) sin(p pi k/nz), all j < ny
        m, p = 3, 1
        shape = np.sin(m * math.pi * I / nx) * np.sin(p * math.pi * K / nz) * (J < ny)
        lam = (2 / dx * math.sin(m * math.pi / (2 * nx))) ** 2 + (2 / dz * math.sin(p * math.pi / (2 * nz))) ** 2
        kc2 = (m * math.pi / (nx * dx)) ** 2 + (p * math.pi / (nz * dz)) ** 2
        c = 1
    f[c] = shape
    N = 700
    r = yee.run(prob, nsteps=N, fields_in=f, want_fields=True)
    a_N, th = _mode_amplitude(lam, dt, eps, N)
    out = r["fields"]
    assert np.max(np.abs(out[c] - a_N * shape)) < 2e-12
    others = [q for q in range(3) if q != c]
    assert np.max(np.abs(out[others])) == 0.0
    # continuous limit: within O((k d)^2) of the cavity resonance (c/2) sqrt(sum (m/a)^2)
    w_d = th / dt
    w_c = math.sqrt(kc2) / math.sqrt(yee.MU0 * yee.EPS0 * eps)
    assert abs(w_d - w_c) / w_c < 0.08


def test_discrete_energy_is_invariant_in_lossless_cavity():
    """W^n = sum eps E^n.E^n + sum mu H^{n-1/2}.H^{n+1/2} is conserved by the Yee leapfrog
    in a closed PEC cavity, for any per-cell eps and mu and with PEC inclusions."""
    nx, ny, nz = 12, 10, 8
    rng = W.SplitMix64(7)
    ids = np.array([rng.randint(0, 3) for _ in range(nx * ny * nz)], np.uint8).reshape(nz, ny, nx)
    ids[4:6, 3:5, 5:7] = 4                     # a PEC block
    prob = W.Problem(nx=nx, ny=ny, nz=nz, dx=1e-3, dy=0.7e-3, dz=1.2e-3, courant=0.99, ids=ids,
                     eps_r=np.array([1.0, 2.5, 4.0, 9.0, 1.0]), sigma=np.zeros(5),
                     mu_r=np.array([1.0, 1.5, 1.0, 2.0, 1.0]),
                     is_pec=np.array([0, 0, 0, 0, 1], np.uint8),
                     sheets=[(2, 3, 2, 9, 2, 6), (0, 8, 1, 7, 2, 5)], bc=(0,) * 6, pml_cells=0)
    f = W.random_fields((nz + 1, ny + 1, nx + 1), seed=11)
    r = yee.run(prob, nsteps=10_000, fields_in=f, want_energy=True)
    e = r["energy"]
    assert e[0] > 0
    assert np.max(np.abs(e - e[0])) / e[0] < 1e-12


def test_courant_limit():
    """Above the 3-D Courant limit the leapfrog diverges; just below it stays bounded."""
    n = 16
    prob = _cavity(n, n, n, 1e-3, 1e-3, 1e-3)
    f = W.random_fields((n + 1, n + 1, n + 1), seed=3)
    f[3:] = 0.0
    dt_hi = yee.courant_dt(1e-3, 1e-3, 1e-3, 1.01)
    r = yee.run(prob, nsteps=400, dt=dt_hi, fields_in=f, want_fields=True)
    assert not np.all(np.isfinite(r["fields"])) or np.max(np.abs(r["fields"])) > 1e6
    small = _cavity(6, 5, 4, 1e-3, 1e-3, 1e-3)
    f2 = W.random_fields((5, 6, 7), seed=5)
    f2[3:] = 0.0
    dt_lo = yee.courant_dt(1e-3, 1e-3, 1e-3, 0.99)
    r2 = yee.run(small, nsteps=100_000, dt=dt_lo, fields_in=f2, want_fields=True, threads=1)
    assert np.max(np.abs(r2["fields"][:3])) < 10.0


# ---------------------------------------------------------------- absorbing layer, ports

def test_pml_reflection_below_minus_40db():
    """Brute force: the short line's port-1 voltage vs a line long enough that nothing
    comes back from its far end within the window.  The difference is what the far
    PML reflects."""
    short = W.config_small_fp64()
    long_ = W.microstrip(448, 32, 24, 5e-6, sub_cells=8, strip_j0=13, strip_j1=19, eps_r=3.8,
                         sigma=0.0, pml=8, bc=short.bc, courant=0.99, nsteps=2000,
                         freqs=short.freqs, f0=300e9, bw=200e9, src_plane=10,
                         port_planes=(14, 50))
    a = yee.run(short)
    b = yee.run(long_)
    v_s, v_l = a["V"][0], b["V"][0]
    refl = np.sum((v_s - v_l) ** 2) / np.sum(v_l ** 2)
    assert 10 * math.log10(refl) < -40.0


def _far_ports(p):
    """Ports 30 and 40 cells downstream of the source: in this small PEC-walled box the
    source's evanescent near field is still visible a few cells from the source plane
    (Z_r there carries a 10-30% imaginary part), so the physics checks sample the line
    further along."""
    p.ports = [W.Port(plane=40, direction=1, j0=13, j1=19, k0=0, k1=8, kb=8, kt=8),
               W.Port(plane=50, direction=-1, j0=13, j1=19, k0=0, k1=8, kb=8, kt=8)]
    return p


def test_uniform_line_impedance_is_real_and_near_quasistatic():
    """Lossless uniform microstrip (w/h = 0.75, eps_r 3.8): Z_r nearly real in band and
    within a loose 15% of the Hammerstad-Jensen quasi-static value (PEC side walls and a
    short air gap under the top PML make this a physics check, not a pin)."""
    p = _far_ports(W.config_small_fp64())
    r = yee.run(p)
    Vf, If = post.port_dfts(r["V"], r["I"], p.freqs, r["dt"])
    band = (p.freqs >= 200e9) & (p.freqs <= 400e9)
    for q in range(2):
        zr = Vf[q] / (If[q] * p.ports[q].direction)
        assert np.max(np.abs(zr[band].imag / zr[band].real)) < 0.02
        z_hj, _ = post.microstrip_z0_hammerstad(6 / 8, 3.8)
        assert abs(np.median(zr[band].real) - z_hj) / z_hj < 0.15
    # matched uniform line: nearly lossless transmission between the ports
    S, Zr = post.sstar_uniform(Vf, If, [1, -1])
    assert np.all(np.abs(np.abs(S[band, 1, 0]) - 1.0) < 1e-2)


def test_lossy_substrate_is_passive():
    """With a conducting substrate, |S11|^2 + |S21|^2 < 1 (Sec. III: losses)."""
    p = _far_ports(W.config_small_fp64())
    p.sigma = np.array([0.0, 5.0])
    r = yee.run(p)
    Vf, If = post.port_dfts(r["V"], r["I"], p.freqs, r["dt"])
    S, Zr = post.sstar_uniform(Vf, If, [1, -1])
    band = (p.freqs >= 200e9) & (p.freqs <= 400e9)
    Sn = post.renormalize(S, Zr)
    pw = np.abs(Sn[band, 0, 0]) ** 2 + np.abs(Sn[band, 1, 0]) ** 2
    assert np.all(pw < 1.0)
    assert np.all(np.abs(S[band, 1, 0]) < 0.99)


def _widened_line(driven, uniform, nsteps=2500):
    """128-cell microstrip with a wider strip section x in [55, 70] (asymmetric along the
    line); identical cross-sections at both ports; source 10 cells inside the driven end."""
    nx = 128
    p = W.microstrip(nx, 32, 24, 5e-6, sub_cells=8, strip_j0=13, strip_j1=19, eps_r=3.8,
                     sigma=0.0, pml=8, bc=(1, 1, 0, 0, 0, 1), courant=0.99, nsteps=nsteps,
                     freqs=W.linear_freqs(100e9, 400e9, 31), f0=250e9, bw=250e9, src_plane=10,
                     port_planes=(24, 104))
    if not uniform:
        p.sheets.append((2, 8, 55, 70, 10, 22))
    p.source.plane = 10 if driven == 0 else nx - 10
    return p


def test_two_run_protocol_is_reciprocal():
    """Full protocol of Sec. II-A (incident run on the uniformised line + total run per
    driven port, 4 runs) on an asymmetric discontinuity: S*_12 = S*_21 (Sec. III notes
    the S*_12 and S*_21 delays coincide), and the discontinuity reflects."""
    dfts = {}
    for d in (0, 1):
        inc, tot = _widened_line(d, True), _widened_line(d, False)
        ri, rt = yee.run(inc), yee.run(tot)
        dfts[d] = (post.port_dfts(ri["V"], ri["I"], inc.freqs, ri["dt"]),
                   post.port_dfts(rt["V"], rt["I"], tot.freqs, rt["dt"]))
    Vinc = np.array([dfts[0][0][0][0], dfts[1][0][0][1]])
    Iinc = np.array([dfts[0][0][1][0], dfts[1][0][1][1]])
    Vtot = np.array([dfts[0][1][0], dfts[1][1][0]])
    S, Zr = post.sstar(Vinc, Iinc, Vtot)
    rel = np.abs(S[:, 0, 1] - S[:, 1, 0]) / np.abs(S[:, 1, 0])
    assert rel.max() < 1e-3
    assert np.abs(S[:, 0, 0]).max() > 0.2
    # lossless: loose power balance only.  V (strip-averaged E_z, Eq. 4) and the loop
    # current do not carry the modal power exactly (Z_r keeps a few % imaginary part in
    # this boxed line), so |S11|^2 + |S21|^2 scatters by up to ~15% about 1.
    pw = np.abs(S[:, 0, 0]) ** 2 + np.abs(S[:, 1, 0]) ** 2
    assert np.max(np.abs(pw - 1.0)) < 0.25


# ---------------------------------------------------------------- lossy media, port integrals

@pytest.mark.parametrize("loss", [0.02, 30.0])
def test_lossy_cavity_mode_follows_time_centred_conductor_recurrence(loss):
    """Lossy dielectrics and metals (Sec. II-B, III; conductor reading: the conduction term
    taken at the mean of the two time levels).  In a PEC cavity uniformly filled with eps and
    sigma, one discrete mode (curl-curl eigenvalue lam) stays a mode.  With e_n its E^n
    amplitude and g_n that of curl H^{n-1/2}, the leapfrog is exactly
        g_{n+1} = g_n - (dt/mu0) lam e_n
        eps (e_{n+1} - e_n)/dt + sigma (e_{n+1} + e_n)/2 = g_{n+1},
    solved here for e_{n+1} from that discrete equation.  loss = sigma dt / (2 eps): 0.02 is
    a lossy dielectric, 30 a metal whose E factor per step is negative (the Cu of the lossy
    line sits near 125).  Any other conductor form (sigma dt/eps in place of sigma dt/2eps,
    the exponential update) drifts from this recurrence by far more than roundoff."""
    nx, ny, nz = 10, 8, 6
    dx, dy, dz = 1.0e-3, 1.3e-3, 0.8e-3
    eps_r = 2.0
    courant = 0.95
    dt = yee.courant_dt(dx, dy, dz, courant)
    eps = yee.EPS0 * eps_r
    sigma = 2.0 * loss * eps / dt
    prob = _cavity(nx, ny, nz, dx, dy, dz, eps_r=eps_r, courant=courant)
    prob.sigma = np.array([sigma])
    m, n = 2, 3
    K, J, I = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    shape = np.sin(m * math.pi * I / nx) * np.sin(n * math.pi * J / ny) * (K < nz)
    lam = (2 / dx * math.sin(m * math.pi / (2 * nx))) ** 2 + \
          (2 / dy * math.sin(n * math.pi / (2 * ny))) ** 2
    f = np.zeros((6, nz + 1, ny + 1, nx + 1))
    f[2] = shape
    N = 200 if loss < 1 else 40
    r = yee.run(prob, nsteps=N, fields_in=f, want_fields=True)
    e, g = 1.0, 0.0
    for _ in range(N):
        g = g - dt / yee.MU0 * lam * e
        e = ((eps / dt - sigma / 2.0) * e + g) / (eps / dt + sigma / 2.0)
    out = r["fields"]
    assert abs(e) > 1e-3                      # the mode has not simply died out
    assert np.max(np.abs(out[2] - e * shape)) < 2e-12
    assert np.max(np.abs(out[:2])) == 0.0
    # per step the mode's two amplitudes shrink by the determinant of the recurrence,
    # (eps/dt - sigma/2)/(eps/dt + sigma/2); for small loss that is exp(-sigma dt/eps), the
    # continuous medium's energy decay
    if loss < 1:
        det = (eps / dt - sigma / 2.0) / (eps / dt + sigma / 2.0)
        assert abs(math.log(det) + sigma * dt / eps) < (sigma * dt / eps) ** 3


def _port_box(nx, ny, nz, dx, dy, dz, port):
    prob = _cavity(nx, ny, nz, dx, dy, dz, eps_r=2.5, courant=0.9)
    prob.ports = [port]
    return prob


def test_port_voltage_integrates_a_linear_ez_profile_exactly():
    """Eq. 4, first line (reading: V = -(1/w) * surface sum of E_z dy dz with trapezoid
    weights across the strip).  An E_z that is linear in y across the strip and varies along
    z integrates exactly under the trapezoid rule:  with w = (j1 - j0) dy,
        V = -dz * sum_{k0 <= k < k1} (E0 + r k),
    whatever the slope s in y.  In a PEC cavity such a field is still in place after one
    step at every edge two or more cells from the walls, where the port sits.  Dropping the
    half weights, shifting the j range or the sign breaks the identity."""
    nx, ny, nz = 12, 14, 10
    dx, dy, dz = 1.0e-3, 0.7e-3, 1.2e-3
    j0, j1, k0, k1 = 4, 9, 3, 7
    port = W.Port(plane=6, direction=1, j0=j0, j1=j1, k0=k0, k1=k1, kb=k1, kt=k1, margin=1)
    prob = _port_box(nx, ny, nz, dx, dy, dz, port)
    E0, s, rz = 3.0, 0.75, -0.4
    K, J, I = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    f = np.zeros((6, nz + 1, ny + 1, nx + 1))
    f[2] = E0 + s * (J - 0.5 * (j0 + j1)) + rz * K
    r = yee.run(prob, nsteps=1, fields_in=f, want_fields=True)
    # the field on the V surface is unchanged by the step (it is linear there)
    surf = np.s_[k0:k1, j0:j1 + 1, port.plane]
    assert np.array_equal(r["fields"][2][surf], f[2][surf])
    want = -dz * sum(E0 + rz * k for k in range(k0, k1))
    assert abs(r["V"][0, 0] - want) < 1e-13 * abs(want)
    # a uniform E_z gives V = -E_z h exactly, h = (k1 - k0) dz
    f[2] = E0
    r = yee.run(prob, nsteps=1, fields_in=f)
    assert abs(r["V"][0, 0] + E0 * (k1 - k0) * dz) < 1e-13 * E0 * (k1 - k0) * dz


@pytest.mark.parametrize("margin,direction", [(1, 1), (2, -1)])
def test_loop_current_obeys_discrete_ampere_law(margin, direction):
    """Eq. 4, second line (the closed H loop around the conductor).  By the discrete Stokes
    theorem on the Yee grid, the loop sum of H.dl on the dual-grid rectangle in the plane
    x = i + 1/2 equals the flux of curl H through it, and in a lossless medium the E update
    turns that flux into  sum eps (E_x^{n+1} - E_x^n)/dt dy dz  over the E_x edges the loop
    encloses.  With random fields and no conductor inside the loop, the port current after
    one step (direction x the mean of the loops at plane -/+ 1/2) must equal that sum: any
    wrong corner index, segment sign, orientation or dy/dz weight breaks it."""
    nx, ny, nz = 12, 14, 12
    dx, dy, dz = 1.0e-3, 0.7e-3, 1.2e-3
    j0, j1, kb, kt = 5, 8, 5, 6
    port = W.Port(plane=6, direction=direction, j0=j0, j1=j1, k0=0, k1=kb, kb=kb, kt=kt,
                  margin=margin)
    prob = _port_box(nx, ny, nz, dx, dy, dz, port)
    dt = yee.courant_dt(dx, dy, dz, prob.courant)
    f = W.random_fields((nz + 1, ny + 1, nx + 1), seed=23)
    r = yee.run(prob, nsteps=1, fields_in=f, want_fields=True)
    dEx = r["fields"][0] - f[0]
    eps = yee.EPS0 * 2.5
    enc = np.s_[kb - margin + 1:kt + margin, j0 - margin + 1:j1 + margin]   # enclosed (k, j)

    def flux(i):
        return np.sum(eps * dEx[enc + (i,)] / dt) * dy * dz

    want = direction * 0.5 * (flux(port.plane - 1) + flux(port.plane))
    assert abs(want) > 1e-3 * np.max(np.abs(f[3:])) * dy          # a sizeable current
    assert abs(r["I"][0, 0] - want) < 1e-12 * np.max(np.abs(f[3:])) * (ny * dy + nz * dz)


def test_stepper_continues_the_run_exactly():
    """The held-open oracle (used to time the stepping alone) advances the same run: 120 +
    180 steps give the port histories of one 300-step run bit for bit (the source clock
    continues across calls)."""
    p = W.config_small_fp64()
    ref = yee.run(p, nsteps=300)
    with yee.Stepper(p, threads=2) as st:
        st.advance(120)
        V0, I0 = st.V.copy(), st.I.copy()
        sec = st.advance(180)
        V1, I1 = st.V, st.I
    assert sec > 0.0
    assert np.array_equal(np.concatenate([V0, V1], axis=1), ref["V"])
    assert np.array_equal(np.concatenate([I0, I1], axis=1), ref["I"])
