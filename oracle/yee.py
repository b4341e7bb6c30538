"""ctypes wrapper around the FP64 CPU Yee oracle (yee_oracle.c).

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may use this module.  It shares no code with the
CUDA library.

`run(problem)` takes a workload description (any object with the attributes of
paper_2208_04371_b300.workloads.Problem) and returns the port time histories
V(t_{n+1}) and I(t_{n+1/2}) and, optionally, the final fields.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "yee_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

C0 = 299792458.0
MU0 = 1.25663706212e-6
EPS0 = 8.8541878128e-12


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, OpenMP over k-planes)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fno-fast-math",
               "-fopenmp", "-fPIC", "-shared", SRC, "-o", LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(LIB + ".tmp", LIB)
    return LIB


class _Problem(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("dt", C.c_double),
        ("ids", C.POINTER(C.c_uint8)),
        ("nmat", C.c_int),
        ("eps_r", C.POINTER(C.c_double)), ("sigma", C.POINTER(C.c_double)),
        ("mu_r", C.POINTER(C.c_double)),
        ("is_pec", C.POINTER(C.c_uint8)),
        ("nsheets", C.c_int),
        ("sheets", C.POINTER(C.c_int)),
        ("bc", C.c_int * 6),
        ("pml_n", C.c_int), ("pml_order", C.c_int),
        ("pml_sigma_scale", C.c_double), ("pml_kappa_max", C.c_double),
        ("pml_alpha_max", C.c_double),
        ("src_kind", C.c_int),
        ("src_plane", C.c_int), ("src_j0", C.c_int), ("src_j1", C.c_int),
        ("src_k0", C.c_int), ("src_k1", C.c_int),
        ("src_amp", C.c_double), ("src_p0", C.c_double), ("src_p1", C.c_double),
        ("src_t0", C.c_double),
        ("src_table", C.POINTER(C.c_double)), ("src_table_len", C.c_long),
        ("nports", C.c_int),
        ("ports", C.POINTER(C.c_int)),
        ("port_width", C.POINTER(C.c_double)),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.oracle_run.restype = C.c_int
        _lib.oracle_run.argtypes = [C.POINTER(_Problem), C.c_long, C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), C.POINTER(C.c_double)]
        _lib.oracle_open.restype = C.c_void_p
        _lib.oracle_open.argtypes = [C.POINTER(_Problem)]
        _lib.oracle_advance.restype = C.c_int
        _lib.oracle_advance.argtypes = [C.c_void_p, C.POINTER(_Problem), C.c_long,
                                        C.POINTER(C.c_double), C.POINTER(C.c_double),
                                        C.POINTER(C.c_double)]
        _lib.oracle_close.restype = None
        _lib.oracle_close.argtypes = [C.c_void_p]
        _lib.oracle_set_threads.restype = None
        _lib.oracle_set_threads.argtypes = [C.c_int]
        _lib.oracle_waveform.restype = C.c_double
        _lib.oracle_waveform.argtypes = [C.POINTER(_Problem), C.c_long]
    return _lib


def courant_dt(dx: float, dy: float, dz: float, courant: float) -> float:
    """CFL step: dt = C / (c0 sqrt(dx^-2 + dy^-2 + dz^-2))  (Sec. II-B and III)."""
    return courant / (C0 * math.sqrt(1.0 / dx ** 2 + 1.0 / dy ** 2 + 1.0 / dz ** 2))


def envelope_t0(kind: int, p0: float, p1: float, t0: float) -> float:
    """Peak time: t0 = 3 sigma for Eq. 3; t0 = 3 tau (tau = 2/(pi bw)) for the
    Gaussian-modulated sine; an explicit t0 >= 0 is used as given."""
    if t0 >= 0.0:
        return t0
    if kind == 1:
        return 3.0 * p0
    if kind == 2:
        return 3.0 * (2.0 / (math.pi * p1))
    return 0.0


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _make(prob, dt: float):
    keep = []
    s = _Problem()
    s.nx, s.ny, s.nz = prob.nx, prob.ny, prob.nz
    s.dx, s.dy, s.dz, s.dt = prob.dx, prob.dy, prob.dz, dt
    ids = np.ascontiguousarray(prob.ids, dtype=np.uint8)
    assert ids.shape == (prob.nz, prob.ny, prob.nx)
    eps = np.ascontiguousarray(prob.eps_r, dtype=np.float64)
    sig = np.ascontiguousarray(prob.sigma, dtype=np.float64)
    mu = np.ascontiguousarray(prob.mu_r, dtype=np.float64)
    pec = np.ascontiguousarray(prob.is_pec, dtype=np.uint8)
    keep += [ids, eps, sig, mu, pec]
    s.ids, s.nmat = _ptr(ids, C.c_uint8), len(eps)
    s.eps_r, s.sigma, s.mu_r, s.is_pec = (_ptr(eps, C.c_double), _ptr(sig, C.c_double),
                                          _ptr(mu, C.c_double), _ptr(pec, C.c_uint8))
    sh = np.ascontiguousarray(np.array(prob.sheets, dtype=np.int32).reshape(-1, 6))
    keep.append(sh)
    s.nsheets, s.sheets = sh.shape[0], _ptr(sh, C.c_int)
    for f in range(6):
        s.bc[f] = int(prob.bc[f])
    s.pml_n, s.pml_order = prob.pml_cells, prob.pml_order
    s.pml_sigma_scale, s.pml_kappa_max, s.pml_alpha_max = (prob.pml_sigma_scale,
                                                           prob.pml_kappa_max, prob.pml_alpha_max)
    src = prob.source
    s.src_kind = src.kind
    s.src_plane, s.src_j0, s.src_j1, s.src_k0, s.src_k1 = src.plane, src.j0, src.j1, src.k0, src.k1
    s.src_amp, s.src_p0, s.src_p1 = src.amplitude, src.param0, src.param1
    s.src_t0 = envelope_t0(src.kind, src.param0, src.param1, src.t0)
    if src.table is not None:
        tab = np.ascontiguousarray(src.table, dtype=np.float64)
        keep.append(tab)
        s.src_table, s.src_table_len = _ptr(tab, C.c_double), len(tab)
    ports = np.array([[p.plane, p.direction, p.j0, p.j1, p.k0, p.k1, p.kb, p.kt, p.margin]
                      for p in prob.ports], dtype=np.int32).reshape(-1, 9)
    widths = np.array([p.width if p.width > 0 else (p.j1 - p.j0) * prob.dy for p in prob.ports],
                      dtype=np.float64)
    ports = np.ascontiguousarray(ports)
    keep += [ports, widths]
    s.nports, s.ports, s.port_width = len(prob.ports), _ptr(ports, C.c_int), _ptr(widths, C.c_double)
    return s, keep


def run(prob, nsteps: Optional[int] = None, dt: Optional[float] = None, fields_in=None,
        want_fields: bool = False, want_energy: bool = False, threads: Optional[int] = None):
    """Run the oracle.  Returns dict(V, I, dt, fields (6,nz+1,ny+1,nx+1) or None, energy)."""
    lib = _load()
    lib.oracle_set_threads(int(threads) if threads is not None else (os.cpu_count() or 1))
    n = prob.nsteps if nsteps is None else nsteps
    if dt is None:
        dt = courant_dt(prob.dx, prob.dy, prob.dz, prob.courant)
    s, keep = _make(prob, dt)
    npts = (prob.nx + 1) * (prob.ny + 1) * (prob.nz + 1)
    np_ = max(len(prob.ports), 1)
    V = np.zeros((np_, max(n, 1)))
    I = np.zeros((np_, max(n, 1)))
    fin = None
    if fields_in is not None:
        fin = np.ascontiguousarray(fields_in, dtype=np.float64).reshape(6 * npts)
        keep.append(fin)
    fout = np.zeros(6 * npts) if want_fields else None
    en = np.zeros(max(n, 1)) if want_energy else None
    rc = lib.oracle_run(C.byref(s), n, _ptr(V, C.c_double), _ptr(I, C.c_double),
                        _ptr(fin, C.c_double) if fin is not None else None,
                        _ptr(fout, C.c_double) if fout is not None else None,
                        _ptr(en, C.c_double) if en is not None else None)
    if rc != 0:
        raise MemoryError("oracle_run failed to allocate")
    shp = (6, prob.nz + 1, prob.ny + 1, prob.nx + 1)
    return dict(V=V[:len(prob.ports), :n], I=I[:len(prob.ports), :n], dt=dt,
                fields=fout.reshape(shp) if fout is not None else None,
                energy=en[:n] if en is not None else None)


class Stepper:
    """The oracle held open between calls: set-up once (zero fields), then `advance(n)`
    runs the next n steps and returns the seconds those steps alone took (allocation and
    the coefficient / CPML set-up are outside every timer); their port samples are left in
    `V` and `I`.  For timing the oracle's stepping rate; `close()` frees its memory."""

    def __init__(self, prob, threads: Optional[int] = None):
        self.lib = _load()
        self.lib.oracle_set_threads(int(threads) if threads is not None else (os.cpu_count() or 1))
        self.prob = prob
        self.dt = courant_dt(prob.dx, prob.dy, prob.dz, prob.courant)
        self.s, self.keep = _make(prob, self.dt)
        self.h = self.lib.oracle_open(C.byref(self.s))
        if not self.h:
            raise MemoryError("oracle_open failed to allocate")

    def advance(self, nsteps: int, threads: Optional[int] = None) -> float:
        if threads is not None:
            self.lib.oracle_set_threads(int(threads))
        np_ = max(len(self.prob.ports), 1)
        V = np.zeros((np_, max(nsteps, 1)))
        I = np.zeros((np_, max(nsteps, 1)))
        sec = C.c_double(0.0)
        rc = self.lib.oracle_advance(self.h, C.byref(self.s), nsteps, _ptr(V, C.c_double),
                                     _ptr(I, C.c_double), C.byref(sec))
        if rc != 0:
            raise MemoryError("oracle_advance failed to allocate")
        self.V, self.I = V[:len(self.prob.ports), :nsteps], I[:len(self.prob.ports), :nsteps]
        return sec.value

    def close(self):
        if self.h:
            self.lib.oracle_close(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def waveform_samples(prob, nsteps: int, dt: Optional[float] = None) -> np.ndarray:
    """The source waveform s((n+1) dt), n = 0..nsteps-1, as the oracle evaluates it."""
    lib = _load()
    if dt is None:
        dt = courant_dt(prob.dx, prob.dy, prob.dz, prob.courant)
    s, keep = _make(prob, dt)
    return np.array([lib.oracle_waveform(C.byref(s), n + 1) for n in range(nsteps)])
