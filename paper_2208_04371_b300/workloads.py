"""Seeded synthetic workloads: geometry, materials, ports and frequency lists.

This module only *describes* problems (shapes, material tables, plane indices,
seeded parameter draws).  It holds none of the solver's arithmetic and imports
nothing from the CUDA library or from the oracle, so both sides and the tests
can build identical inputs from it.

The microstrip workloads stand in for the paper's transmission lines (Sec. II-B
microstrip: PEC ground, dielectric substrate, strip conductor; Sec. III: layered
oxide stack with a lossy metal line).  Propagation is along x, the strip width
along y and the height along z; the paper's own frame propagates along y, which
is a pure relabelling.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

# boundary kinds per face (-x, +x, -y, +y, -z, +z)
BC_PEC = 0
BC_PML = 1

# waveform kinds
WAVE_NONE = 0
WAVE_DIFF_GAUSS = 1      # differential Gaussian, Eq. 3 (param0 = sigma [s])
WAVE_GAUSS_SINE = 2      # Gaussian-modulated sine (param0 = f0 [Hz], param1 = bandwidth [Hz])
WAVE_TABLE = 3           # user table, one value per step


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014): a counter-based 64-bit generator."""

    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.state = seed & self.MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self.MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform on [lo, hi] inclusive."""
        return lo + self.next_u64() % (hi - lo + 1)


@dataclass
class Port:
    plane: int            # x index of the V surface (E_z edges at x = plane)
    direction: int        # +1: incident wave travels +x, -1: travels -x
    j0: int               # strip edges in y (node indices), V surface j in [j0, j1]
    j1: int
    k0: int               # V surface z range k in [k0, k1) (E_z edges)
    k1: int
    kb: int               # conductor bottom / top node in z (kb == kt for a sheet)
    kt: int
    margin: int = 1       # I loop lies `margin` cells outside the conductor
    width: float = 0.0    # strip width [m]; 0 -> (j1 - j0) * dy


@dataclass
class Source:
    kind: int = WAVE_NONE
    plane: int = 0
    j0: int = 0
    j1: int = 0
    k0: int = 0
    k1: int = 0
    amplitude: float = 1.0
    param0: float = 0.0
    param1: float = 0.0
    t0: float = -1.0                       # < 0: three envelope widths
    table: Optional[np.ndarray] = None     # WAVE_TABLE samples s((n+1) dt)


@dataclass
class Problem:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    courant: float
    ids: np.ndarray                        # uint8 (nz, ny, nx)
    eps_r: np.ndarray                      # per material
    sigma: np.ndarray
    mu_r: np.ndarray
    is_pec: np.ndarray                     # uint8 per material
    sheets: List[tuple] = field(default_factory=list)   # (axis, index, lo0, hi0, lo1, hi1)
    bc: tuple = (BC_PML, BC_PML, BC_PML, BC_PML, BC_PEC, BC_PML)
    pml_cells: int = 8
    pml_order: int = 3
    pml_sigma_scale: float = 1.0
    pml_kappa_max: float = 1.0
    pml_alpha_max: float = 0.0
    source: Source = field(default_factory=Source)
    ports: List[Port] = field(default_factory=list)
    freqs: np.ndarray = field(default_factory=lambda: np.zeros(0))
    nsteps: int = 0
    name: str = ""

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def linear_freqs(f_lo: float, f_hi: float, n: int) -> np.ndarray:
    return np.array([f_lo + k * (f_hi - f_lo) / (n - 1) for k in range(n)], dtype=np.float64)


def microstrip(nx: int, ny: int, nz: int, delta: float, *, sub_cells: int, strip_j0: int,
               strip_j1: int, eps_r: float, sigma: float, pml: int, bc: Sequence[int],
               courant: float, nsteps: int, freqs: np.ndarray, f0: float, bw: float,
               src_plane: int, port_planes: Sequence[int], uniform_cap: bool = False,
               name: str = "") -> Problem:
    """PEC ground at z = 0, substrate k in [0, sub_cells), zero-thickness PEC strip at
    k = sub_cells spanning the whole length in x, air above."""
    ids = np.zeros((nz, ny, nx), dtype=np.uint8)
    ids[:sub_cells] = 1
    eps = np.array([1.0, eps_r])
    sig = np.array([0.0, sigma])
    mu = np.array([1.0, 1.0])
    pec = np.array([0, 0], dtype=np.uint8)
    sheets = [(2, sub_cells, 0, nx, strip_j0, strip_j1)]
    src = Source(kind=WAVE_GAUSS_SINE, plane=src_plane, j0=strip_j0, j1=strip_j1, k0=0,
                 k1=sub_cells, amplitude=1.0, param0=f0, param1=bw)
    ports = []
    for idx, pl in enumerate(port_planes):
        ports.append(Port(plane=pl, direction=1 if idx == 0 else -1, j0=strip_j0, j1=strip_j1,
                          k0=0, k1=sub_cells, kb=sub_cells, kt=sub_cells, margin=1))
    return Problem(nx=nx, ny=ny, nz=nz, dx=delta, dy=delta, dz=delta, courant=courant,
                   ids=ids, eps_r=eps, sigma=sig, mu_r=mu, is_pec=pec, sheets=sheets,
                   bc=tuple(bc), pml_cells=pml, source=src, ports=ports, freqs=freqs,
                   nsteps=nsteps, name=name)


def config_small_fp64() -> Problem:
    """Plain FP64 microstrip: 64x32x24 cells of 5 um, eps_r 3.8 substrate of 8 cells,
    6-cell-wide PEC sheet strip, 8-cell PML on the x ends and the top (y walls PEC),
    Courant 0.99, 2000 steps, Gaussian-modulated sine at 300 GHz / 200 GHz bandwidth,
    64 DFT frequencies 100-500 GHz."""
    return microstrip(64, 32, 24, 5e-6, sub_cells=8, strip_j0=13, strip_j1=19, eps_r=3.8,
                      sigma=0.0, pml=8, bc=(BC_PML, BC_PML, BC_PEC, BC_PEC, BC_PEC, BC_PML),
                      courant=0.99, nsteps=2000, freqs=linear_freqs(100e9, 500e9, 64),
                      f0=300e9, bw=200e9, src_plane=10, port_planes=(14, 50),
                      name="microstrip 64x32x24 fp64")


def config_lossy_line(nx: int = 768, ny: int = 384, nz: int = 256, nsteps: int = 200_000,
                      scale_z: Optional[float] = None) -> Problem:
    """Single large lossy line: cells of 20 nm; Si (eps_r 11.7, 10 S/m) for k < 96,
    three SiO2 layers (eps_r 3.9) up to k = 192, a Cu strip (5.8e7 S/m) 50 cells wide and
    10 thick, air above; 12-cell PML on +-x, +-y and +z; PEC ground; pulse 50-300 GHz;
    128 DFT frequencies.  Smaller grids keep the same stack scaled by nz/256."""
    s = nz / 256.0 if scale_z is None else scale_z
    k_si, k_ox, k_cu = int(round(96 * s)), int(round(192 * s)), int(round(202 * s))
    k_cu = max(k_cu, k_ox + 1)
    wy = max(2, int(round(50 * ny / 384)))
    j0 = (ny - wy) // 2
    j1 = j0 + wy
    ids = np.zeros((nz, ny, nx), dtype=np.uint8)
    ids[:k_si] = 1
    third = (k_ox - k_si) // 3
    ids[k_si:k_si + third] = 2
    ids[k_si + third:k_si + 2 * third] = 3
    ids[k_si + 2 * third:k_ox] = 4
    ids[k_ox:k_cu, j0:j1, :] = 5
    eps = np.array([1.0, 11.7, 3.9, 3.9, 3.9, 1.0])
    sig = np.array([0.0, 10.0, 0.0, 0.0, 0.0, 5.8e7])
    mu = np.ones(6)
    pec = np.zeros(6, dtype=np.uint8)
    pml = 12
    src_plane = pml + 2
    src = Source(kind=WAVE_GAUSS_SINE, plane=src_plane, j0=j0, j1=j1, k0=0, k1=k_ox,
                 amplitude=1.0, param0=175e9, param1=250e9)
    ports = [Port(plane=src_plane + 4, direction=1, j0=j0, j1=j1, k0=0, k1=k_ox, kb=k_ox,
                  kt=k_cu, margin=1),
             Port(plane=nx - pml - 6, direction=-1, j0=j0, j1=j1, k0=0, k1=k_ox, kb=k_ox,
                  kt=k_cu, margin=1)]
    return Problem(nx=nx, ny=ny, nz=nz, dx=20e-9, dy=20e-9, dz=20e-9, courant=0.99, ids=ids,
                   eps_r=eps, sigma=sig, mu_r=mu, is_pec=pec, sheets=[],
                   bc=(BC_PML, BC_PML, BC_PML, BC_PML, BC_PEC, BC_PML), pml_cells=pml,
                   source=src, ports=ports, freqs=linear_freqs(50e9, 300e9, 128), nsteps=nsteps,
                   name=f"lossy line {nx}x{ny}x{nz} 20nm")


def batch_instance(rng: SplitMix64, nsteps: int = 20_000, nfreq: int = 64,
                   dims: Optional[tuple] = None) -> Problem:
    """One batched-sweep microstrip: dims 64-192 per axis, strip width 4-40 cells,
    substrate 6-30 cells, eps_r 2-12, substrate sigma 0-50 S/m, 8-cell PML, 5 um cells."""
    if dims is None:
        nx, ny, nz = rng.randint(64, 192), rng.randint(64, 192), rng.randint(64, 192)
    else:
        nx, ny, nz = dims
    w = rng.randint(4, 40)
    sub = rng.randint(6, 30)
    er = rng.uniform(2.0, 12.0)
    sg = rng.uniform(0.0, 50.0)
    pml = 8
    w = min(w, ny - 2 * pml - 8)
    sub = min(sub, nz - pml - 8)
    j0 = (ny - w) // 2
    return microstrip(nx, ny, nz, 5e-6, sub_cells=sub, strip_j0=j0, strip_j1=j0 + w, eps_r=er,
                      sigma=sg, pml=pml, bc=(BC_PML, BC_PML, BC_PML, BC_PML, BC_PEC, BC_PML),
                      courant=0.99, nsteps=nsteps, freqs=linear_freqs(100e9, 500e9, nfreq),
                      f0=300e9, bw=200e9, src_plane=pml + 2,
                      port_planes=(pml + 6, nx - pml - 6),
                      name=f"batch {nx}x{ny}x{nz} w{w} h{sub}")


def config_batched(n: int = 256, seed: int = 0x220804371, nsteps: int = 20_000) -> List[Problem]:
    rng = SplitMix64(seed)
    return [batch_instance(rng, nsteps=nsteps) for _ in range(n)]


def config_long_run(nsteps: int = 1_000_000, ringing: bool = False, nfreq: int = 256) -> Problem:
    """Long-run precision study: 256x128x128 lossless eps_r 3.9 microstrip (5 um cells),
    256 DFT frequencies.  The ringing variant closes both x ends with PEC so the line
    keeps resonating and the DFT accumulators keep growing."""
    bc = (BC_PEC, BC_PEC, BC_PML, BC_PML, BC_PEC, BC_PML) if ringing else \
         (BC_PML, BC_PML, BC_PML, BC_PML, BC_PEC, BC_PML)
    return microstrip(256, 128, 128, 5e-6, sub_cells=16, strip_j0=52, strip_j1=76, eps_r=3.9,
                      sigma=0.0, pml=8, bc=bc, courant=0.99, nsteps=nsteps,
                      freqs=linear_freqs(100e9, 500e9, nfreq), f0=300e9, bw=200e9,
                      src_plane=10, port_planes=(14, 256 - 14),
                      name="long-run 256x128x128" + (" ringing" if ringing else ""))


def config_microstrip_theory(nsteps: int = 60_000, nfreq: int = 128) -> Problem:
    """The paper's verification microstrip (Sec. II-B) in this build's frame (propagation
    along x): 1000 x 200 x 50 cells of 0.1 mm; SiO2 substrate (eps_r 3.8) 1 mm = 10 cells
    thick; zero-thickness PEC strip 57 cells wide (w/h = 5.7, designed for 25 ohm); CFL 0.9;
    Eq. 3 differential Gaussian, sigma = 11.254 ps, t0 = 3 sigma; 60000 steps.  8-cell PML on
    the x ends, y sides and top, PEC ground; source plane 10, ports at 30 and 970 (94 mm
    apart); 128 DFT frequencies over 0.2-40 GHz (the lowest keeps beta l under pi, so the
    phase of S*_21 unwraps from the first frequency; 60000 steps resolve about 0.1 GHz)."""
    nx, ny, nz, sub, w = 1000, 200, 50, 10, 57
    j0 = (ny - w) // 2
    prob = microstrip(nx, ny, nz, 1e-4, sub_cells=sub, strip_j0=j0, strip_j1=j0 + w, eps_r=3.8,
                      sigma=0.0, pml=8, bc=(BC_PML, BC_PML, BC_PML, BC_PML, BC_PEC, BC_PML),
                      courant=0.9, nsteps=nsteps, freqs=linear_freqs(0.2e9, 40e9, nfreq),
                      f0=20e9, bw=20e9, src_plane=10, port_planes=(30, nx - 30),
                      name="paper microstrip 1000x200x50 0.1mm")
    prob.source = Source(kind=WAVE_DIFF_GAUSS, plane=10, j0=j0, j1=j0 + w, k0=0, k1=sub,
                         amplitude=1.0, param0=11.254e-12)
    return prob


# assumed bulk conductivities (the paper does not give them) [S/m]
SIGMA_PD, SIGMA_AL = 9.5e6, 3.77e7


def config_cmos_line(nx: int = 120, ny: int = 200, nz: int = 800, nsteps: int = 1_400_000,
                     driven: int = 0, uniform: bool = False, nfreq: int = 64, pml: int = 10,
                     f_lo: float = 2e12, f_hi: float = 90e12, refine: int = 1,
                     sigma: float = 10.146e-15) -> Problem:
    """The paper's third example (Sec. III), an on-chip line, in this build's frame
    (propagation along x): cells of 50 x 20 x 5 nm (the paper's 20 x 50 x 5 nm with x and y
    exchanged), 120 x 200 x 800 cells = 6 x 4 x 4 um; SiO2 (eps_r 3.9) everywhere else; CFL 0.9
    (dt = 0.0145 fs, as printed); Eq. 3 differential Gaussian, sigma = 10.146 fs, t0 = 3 sigma;
    1.4 M steps in the paper.
      - Pd strip (assumed 9.5e6 S/m), half the width (2 um), 6 cells (30 nm) thick, centred in
        y and z, along the whole line; halfway along it steps up by 4 cells (20 nm);
      - Al block (assumed 3.77e7 S/m) under the second half (x from 3 um, centred 4.5 um down
        the line), the full width, from the ground up to 4 cells (20 nm of oxide) below the
        stepped strip;
      - PEC ground at z = 0; PML on the other faces.
    Cell counts other than the paper's keep the cell sizes and the z structure (strip, step,
    oxide gap) and scale the rest, for reduced parity cases.
    Ports: 1 at x = pml + 6 (V from the ground to the strip), 2 at x = nx - pml - 6 (V across
    the oxide gap from the Al to the strip); the source sits on the driven side, 4 cells
    outside its port.  uniform=True gives the incident-run line of Sec. II-A: the driven
    port's cross-section along the whole length.
    refine = r divides every cell size by r and multiplies every cell count (grid, PML,
    strip, step, port and source offsets) by r: the same line on a grid r times finer in
    each direction (the Appendix's convergence test doubles it).  sigma is the width of the
    Eq. 3 pulse (the Appendix's narrow pulse has 1.45 fs)."""
    r = refine
    dx, dy, dz = 50e-9 / r, 20e-9 / r, 5e-9 / r
    nx, ny, nz, pml = nx * r, ny * r, nz * r, pml * r
    w = ny // 2
    j0 = (ny - w) // 2
    j1 = j0 + w
    ks = nz // 2 - 3 * r        # strip bottom, first half
    kstep = 4 * r               # step height = oxide gap
    thick = 6 * r               # strip thickness
    half = nx // 2
    ids = np.zeros((nz, ny, nx), dtype=np.uint8)   # 0 SiO2, 1 Pd, 2 Al
    for x0, x1, low in ((0, half, False), (half, nx, True)):
        lowered = low if not uniform else (driven == 1)
        kb = ks + (kstep if lowered else 0)
        ids[kb:kb + thick, j0:j1, x0:x1] = 1
        if lowered:
            ids[:ks, :, x0:x1] = 2
    eps = np.array([3.9, 1.0, 1.0])
    sig = np.array([0.0, SIGMA_PD, SIGMA_AL])
    p1, p2 = pml + 6 * r, nx - pml - 6 * r
    ports = [Port(plane=p1, direction=1, j0=j0, j1=j1, k0=0, k1=ks, kb=ks, kt=ks + thick, margin=1),
             Port(plane=p2, direction=-1, j0=j0, j1=j1, k0=ks, k1=ks + kstep, kb=ks + kstep,
                  kt=ks + kstep + thick, margin=1)]
    if uniform and driven == 0:   # the first half's cross-section at both ports
        ports[1] = Port(plane=p2, direction=-1, j0=j0, j1=j1, k0=0, k1=ks, kb=ks, kt=ks + thick,
                        margin=1)
    if uniform and driven == 1:   # the second half's cross-section at both ports
        ports[0] = Port(plane=p1, direction=1, j0=j0, j1=j1, k0=ks, k1=ks + kstep, kb=ks + kstep,
                        kt=ks + kstep + thick, margin=1)
    if driven == 0:
        src = Source(kind=WAVE_DIFF_GAUSS, plane=p1 - 4 * r, j0=j0, j1=j1, k0=0, k1=ks,
                     amplitude=1.0, param0=sigma)
    else:
        src = Source(kind=WAVE_DIFF_GAUSS, plane=p2 + 4 * r, j0=j0, j1=j1, k0=ks, k1=ks + kstep,
                     amplitude=1.0, param0=sigma)
    return Problem(nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz, courant=0.9, ids=ids, eps_r=eps,
                   sigma=sig, mu_r=np.ones(3), is_pec=np.zeros(3, np.uint8),
                   bc=(BC_PML, BC_PML, BC_PML, BC_PML, BC_PEC, BC_PML), pml_cells=pml,
                   source=src, ports=ports, freqs=linear_freqs(f_lo, f_hi, nfreq), nsteps=nsteps,
                   name=f"cmos line {nx}x{ny}x{nz} driven {driven + 1}{' uniform' if uniform else ''}"
                        + (f" refined x{r}" if r > 1 else ""))


SURROGATE_LO = (4.0, 0.0, 6.0, 2.0, 0.0, 32.0)
SURROGATE_HI = (40.0, 10.0, 30.0, 12.0, 50.0, 160.0)


def surrogate_line(desc, nsteps: int = 8000, nfreq: int = 128, pml: int = 8) -> Problem:
    """The uniform microstrip a surrogate descriptor (width, thickness, substrate height in
    cells, eps_r, substrate sigma [S/m], length in cells) stands for: 5 um cells, PEC ground,
    strip of `thickness` PEC cells on the substrate (a zero-thickness sheet when 0), `length`
    cells between the two ports, port 1 ten cells past the source, 8-cell PML elsewhere,
    128 frequencies over 100-500 GHz."""
    w, tk, h = int(round(desc[0])), int(round(desc[1])), int(round(desc[2]))
    er, sg, L = float(desc[3]), float(desc[4]), int(round(desc[5]))
    gap_y, air = max(6, h), max(8, h)
    ny = w + 2 * gap_y + 2 * pml
    nz = h + tk + air + pml
    src = pml + 2
    p1 = src + 10
    p2 = p1 + L
    nx = p2 + 6 + pml
    j0 = pml + gap_y
    prob = microstrip(nx, ny, nz, 5e-6, sub_cells=h, strip_j0=j0, strip_j1=j0 + w, eps_r=er,
                      sigma=sg, pml=pml, bc=(BC_PML, BC_PML, BC_PML, BC_PML, BC_PEC, BC_PML),
                      courant=0.99, nsteps=nsteps, freqs=linear_freqs(100e9, 500e9, nfreq),
                      f0=300e9, bw=200e9, src_plane=src, port_planes=(p1, p2),
                      name=f"line w{w} t{tk} h{h} er{er:.2f} s{sg:.1f} L{L}")
    if tk > 0:
        ids = prob.ids.copy()
        ids[h:h + tk, j0:j0 + w, :] = 2
        prob = prob.replace(ids=ids, eps_r=np.append(prob.eps_r, 1.0),
                            sigma=np.append(prob.sigma, 0.0), mu_r=np.append(prob.mu_r, 1.0),
                            is_pec=np.append(prob.is_pec, 1).astype(np.uint8))
        for pt in prob.ports:
            pt.kt = h + tk
    return prob


def surrogate_inputs(rng: SplitMix64, n: int) -> np.ndarray:
    """Line descriptors for the surrogate: (width cells 4-40, thickness cells 0-10,
    substrate cells 6-30, eps_r 2-12, sigma S/m 0-50, length cells 32-160)."""
    out = np.zeros((n, 6), dtype=np.float64)
    for r in range(n):
        out[r] = (rng.randint(4, 40), rng.randint(0, 10), rng.randint(6, 30),
                  rng.uniform(2.0, 12.0), rng.uniform(0.0, 50.0), rng.randint(32, 160))
    return out


def splitmix64_array(seed: int, n: int) -> np.ndarray:
    """The first n outputs of SplitMix64(seed), vectorised: output i mixes seed + (i+1) gamma."""
    with np.errstate(over="ignore"):
        st = np.uint64(seed & SplitMix64.MASK) + (np.arange(1, n + 1, dtype=np.uint64)
                                                  * np.uint64(0x9E3779B97F4A7C15))
        z = (st ^ (st >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform_array(seed: int, n: int, lo: float, hi: float) -> np.ndarray:
    return lo + (hi - lo) * ((splitmix64_array(seed, n) >> np.uint64(11)).astype(np.float64)
                             * (1.0 / (1 << 53)))


MLP_SIZES = (6, 512, 512, 512, 512, 512)


def mlp_init(seed: int, bias_scale: float = 0.0, sizes=MLP_SIZES) -> np.ndarray:
    """Seeded initial surrogate weights, flat in the yfmlp.h layout (W_l [out][in], b_l):
    uniform with variance 2 / fan_in for the GELU layers, 1 / fan_in for the linear output
    layer; biases uniform in [-bias_scale, bias_scale]."""
    parts = []
    for l, (fin, fout) in enumerate(zip(sizes[:-1], sizes[1:])):
        last = l == len(sizes) - 2
        a = np.sqrt((3.0 if last else 6.0) / fin)
        parts.append(uniform_array(seed * 1000003 + 2 * l, fin * fout, -a, a))
        parts.append(uniform_array(seed * 1000003 + 2 * l + 1, fout, -bias_scale, bias_scale)
                     if bias_scale > 0 else np.zeros(fout))
    return np.concatenate(parts)


def random_fields(shape_zyx: tuple, seed: int) -> np.ndarray:
    """Six seeded random component arrays of shape (nz+1, ny+1, nx+1), values in [-1, 1)."""
    rng = SplitMix64(seed)
    n = int(np.prod(shape_zyx))
    vals = np.array([rng.uniform(-1.0, 1.0) for _ in range(6 * n)], dtype=np.float64)
    return vals.reshape((6,) + tuple(shape_zyx))
