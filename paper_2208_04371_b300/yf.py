"""ctypes binding of libyeefdtd.so (include/yeefdtd.h): argument marshalling only.

Every computation happens inside the CUDA library; this module converts Python
values to the C ABI and raises YFError on a non-zero status.  Importing it fails
loudly when the compiled library is missing: there is no fallback.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); a CUDA tensor
is passed by its device pointer.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libyeefdtd.so")

if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is missing: run `python -m paper_2208_04371_b300.build` "
                      "(or __graft_entry__.build()) first")
_lib = C.CDLL(_LIB_PATH)

OK, E_INVALID, E_OOM, E_CUDA, E_STATE, E_TIMEOUT, E_UNSTABLE, E_UNSUPPORTED = range(8)
FP32, FP64 = 0, 1
HOST, DEVICE = 0, 1
BC_PEC, BC_PML = 0, 1
EX, EY, EZ, HX, HY, HZ = range(6)
WAVE_NONE, WAVE_DIFF_GAUSS, WAVE_GAUSS_SINE, WAVE_TABLE = range(4)
DFT_FP64, DFT_KAHAN32, DFT_FP32 = 1, 2, 4

_NAMES = {0: "YF_OK", 1: "YF_E_INVALID", 2: "YF_E_OOM", 3: "YF_E_CUDA", 4: "YF_E_STATE",
          5: "YF_E_TIMEOUT", 6: "YF_E_UNSTABLE", 7: "YF_E_UNSUPPORTED"}


class YFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class Waveform(C.Structure):
    _fields_ = [("kind", C.c_int), ("amplitude", C.c_double), ("p0", C.c_double),
                ("p1", C.c_double), ("t0", C.c_double), ("table", C.POINTER(C.c_double)),
                ("table_len", C.c_long)]


class PortDesc(C.Structure):
    _fields_ = [("axis", C.c_int), ("plane", C.c_int), ("direction", C.c_int), ("j0", C.c_int),
                ("j1", C.c_int), ("k0", C.c_int), ("k1", C.c_int), ("kb", C.c_int),
                ("kt", C.c_int), ("margin", C.c_int), ("width", C.c_double)]


class PortDfts(C.Structure):
    _fields_ = [("V_re", C.POINTER(C.c_double)), ("V_im", C.POINTER(C.c_double)),
                ("I_re", C.POINTER(C.c_double)), ("I_im", C.POINTER(C.c_double))]


class InstanceDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double),
                ("dy", C.c_double), ("dz", C.c_double), ("ids", C.c_void_p), ("nmat", C.c_int),
                ("eps_r", C.POINTER(C.c_double)), ("sigma", C.POINTER(C.c_double)),
                ("mu_r", C.POINTER(C.c_double)), ("is_pec", C.c_void_p), ("nsheets", C.c_int),
                ("sheets", C.POINTER(C.c_int)), ("bc", C.c_int * 6), ("pml_cells", C.c_int),
                ("pml_order", C.c_int), ("pml_sigma_scale", C.c_double),
                ("pml_kappa_max", C.c_double), ("pml_alpha_max", C.c_double),
                ("src_plane", C.c_int), ("src_j0", C.c_int), ("src_j1", C.c_int),
                ("src_k0", C.c_int), ("src_k1", C.c_int), ("src", Waveform), ("nports", C.c_int),
                ("ports", C.POINTER(PortDesc)), ("nfreq", C.c_int),
                ("freqs", C.POINTER(C.c_double))]


_vp = C.c_void_p
_dp = C.POINTER(C.c_double)
_i = C.c_int
_d = C.c_double
_SIGS = {
    "yf_last_error": (C.c_char_p, []),
    "yf_courant_dt": (_i, [_d, _d, _d, _d, _dp]),
    "yf_grid_create": (_i, [_i, _i, _i, _d, _d, _d, _d, _i, _vp, C.POINTER(_vp)]),
    "yf_grid_destroy": (_i, [_vp]),
    "yf_grid_dt": (_i, [_vp, _dp]),
    "yf_set_materials": (_i, [_vp, _vp, _i, _i, _dp, _dp, _dp, _vp]),
    "yf_add_pec_sheet": (_i, [_vp, _i, _i, _i, _i, _i, _i]),
    "yf_set_boundaries": (_i, [_vp, C.POINTER(_i)]),
    "yf_set_pml": (_i, [_vp, _i, _i, _d, _d, _d]),
    "yf_set_source": (_i, [_vp, _i, _i, _i, _i, _i, _i, C.POINTER(Waveform)]),
    "yf_add_port": (_i, [_vp, C.POINTER(PortDesc), _i, _dp, C.POINTER(_i)]),
    "yf_set_dft_mode": (_i, [_vp, _i]),
    "yf_step": (_i, [_vp, C.c_long]),
    "yf_sync": (_i, [_vp]),
    "yf_steps_done": (_i, [_vp, C.POINTER(C.c_long)]),
    "yf_read_fields": (_i, [_vp, _i, _vp, _i]),
    "yf_write_fields": (_i, [_vp, _i, _vp, _i]),
    "yf_energy": (_i, [_vp, _dp]),
    "yf_read_port_dft": (_i, [_vp, _i, _i, _dp, _dp, _dp, _dp]),
    "yf_sparams": (_i, [_i, _i, _dp, C.POINTER(PortDfts), C.POINTER(PortDfts), _d, _dp, _dp,
                        _dp, _dp, _dp]),
    "yf_read_sparams": (_i, [_vp, _d, _dp, _dp, _dp, _dp, _dp]),
    "yf_read_sparams_acc": (_i, [_vp, _i, _d, _dp, _dp, _dp, _dp, _dp]),
    "yf_launches_per_step": (_i, [_vp, C.POINTER(_i)]),
    "yf_launches": (_i, [_vp, C.c_long, C.POINTER(C.c_long)]),
    "yf_tb_box": (_i, [_vp, C.POINTER(_i)]),
    "yf_bounded_wait_check": (_i, [_i, _d]),
    "yf_rlcg": (_i, [_i, _dp, _dp, _dp, _d, _dp, _dp, _dp, _dp, _dp]),
    "yf_sparams_noalloc": (_i, [_i, _i, _vp, _vp, _vp, _vp, _d, _vp, _vp, _vp, _vp, _vp, _vp]),
    "yf_reset": (_i, [_vp]),
    "yf_set_variant": (_i, [_vp, _i, _i, _i]),
    "yf_set_box_shape": (_i, [_vp, _i, _i]),
    "yf_profile_steps": (_i, [_vp, C.c_long, _dp, C.POINTER(_i)]),
    "yf_kernel_name": (C.c_char_p, [_vp, _i]),
    "yf_autotune": (_i, [_vp, C.c_char_p, _i, C.POINTER(_i), C.POINTER(_i)]),
    "yf_batch_autotune": (_i, [_vp, C.c_char_p, _i, C.POINTER(_i), C.POINTER(_i)]),
    "yf_batch_create": (_i, [_i, C.POINTER(InstanceDesc), _d, _i, _vp, C.POINTER(_vp)]),
    "yf_batch_destroy": (_i, [_vp]),
    "yf_batch_set_tiling": (_i, [_vp, _i, _i]),
    "yf_batch_set_variant": (_i, [_vp, _i]),
    "yf_batch_step": (_i, [_vp, C.c_long]),
    "yf_batch_sync": (_i, [_vp]),
    "yf_batch_info": (_i, [_vp, C.POINTER(_i), C.POINTER(C.c_long), _dp, C.POINTER(C.c_long)]),
    "yf_batch_grid": (_i, [_vp, _i, C.POINTER(_vp)]),
    "yf_batch_read_port_dft": (_i, [_vp, _i, _i, _i, _dp, _dp, _dp, _dp]),
    "yf_mlp_create": (_i, [_i, _i, _i, _dp, _dp, _vp, C.POINTER(_vp)]),
    "yf_mlp_destroy": (_i, [_vp]),
    "yf_mlp_set_params": (_i, [_vp, _i, _dp]),
    "yf_mlp_get_params": (_i, [_vp, _i, _dp]),
    "yf_mlp_set_adam": (_i, [_vp, _d, _d, _d, _d]),
    "yf_mlp_grads": (_i, [_vp, _i, _vp, _vp, _i, _dp, _dp]),
    "yf_mlp_train_step": (_i, [_vp, _i, _vp, _vp, _i, _dp]),
    "yf_mlp_query": (_i, [_vp, _vp, _i, _i, _vp, _vp, _i]),
    "yf_mlp_gate": (_i, [_vp, _vp, _i, _d, _d, _i, _vp, C.POINTER(_i)]),
    "yf_mlp_query_stats": (_i, [_vp, C.POINTER(_i), _dp]),
    "yf_mlp_fit": (_i, [_vp, _i, _vp, _vp, _i, _vp, _vp, C.c_long]),
    "yf_mlp_sync": (_i, [_vp, _dp]),
    "yf_checkpoint_save": (_i, [_vp, C.c_char_p]),
    "yf_checkpoint_load": (_i, [_vp, C.c_char_p]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

DECLARED = tuple(_SIGS)


def library_path() -> str:
    return _LIB_PATH


def last_error() -> str:
    return (_lib.yf_last_error() or b"").decode()


def _check(st: int):
    if st != OK:
        raise YFError(st, last_error())


def _ptr(a, ctype=None):
    """(pointer, where, keep-alive) for a numpy array or torch tensor."""
    if a is None:
        return None, HOST, None
    if hasattr(a, "data_ptr"):      # torch tensor
        where = DEVICE if a.is_cuda else HOST
        a = a.contiguous()
        p = C.c_void_p(a.data_ptr())
        return (C.cast(p, C.POINTER(ctype)) if ctype else p), where, a
    arr = np.ascontiguousarray(a)
    p = arr.ctypes.data_as(C.POINTER(ctype)) if ctype else C.c_void_p(arr.ctypes.data)
    return p, HOST, arr


def _f64(a):
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return arr.ctypes.data_as(_dp), arr


# ----------------------------------------------------------------- thin wrappers (same names)

def courant_dt(dx, dy, dz, courant) -> float:
    out = C.c_double()
    _check(_lib.yf_courant_dt(dx, dy, dz, courant, C.byref(out)))
    return out.value


def grid_create(nx, ny, nz, dx, dy, dz, dt=0.0, prec=FP32, stream=None) -> int:
    h = C.c_void_p()
    s = C.c_void_p(int(stream)) if stream else None
    _check(_lib.yf_grid_create(nx, ny, nz, dx, dy, dz, dt, prec, s, C.byref(h)))
    return h.value


def grid_destroy(g):
    _check(_lib.yf_grid_destroy(C.c_void_p(g)))


def grid_dt(g) -> float:
    out = C.c_double()
    _check(_lib.yf_grid_dt(C.c_void_p(g), C.byref(out)))
    return out.value


def set_materials(g, ids, eps_r, sigma, mu_r=None, is_pec=None):
    p, where, keep = _ptr(ids)
    e, ke = _f64(eps_r)
    s, ks = _f64(sigma)
    m, km = (_f64(mu_r) if mu_r is not None else (None, None))
    pe = None
    if is_pec is not None:
        kp = np.ascontiguousarray(np.asarray(is_pec, dtype=np.uint8))
        pe = C.c_void_p(kp.ctypes.data)
    _check(_lib.yf_set_materials(C.c_void_p(g), p, where, len(ke), e, s, m, pe))


def add_pec_sheet(g, normal_axis, index, lo0, hi0, lo1, hi1):
    _check(_lib.yf_add_pec_sheet(C.c_void_p(g), normal_axis, index, lo0, hi0, lo1, hi1))


def set_boundaries(g, bc: Sequence[int]):
    arr = (C.c_int * 6)(*[int(b) for b in bc])
    _check(_lib.yf_set_boundaries(C.c_void_p(g), arr))


def set_pml(g, ncells=8, order=3, sigma_scale=1.0, kappa_max=1.0, alpha_max=0.0):
    _check(_lib.yf_set_pml(C.c_void_p(g), ncells, order, sigma_scale, kappa_max, alpha_max))


def set_source(g, plane, j0, j1, k0, k1, kind, amplitude=1.0, p0=0.0, p1=0.0, t0=-1.0,
               table=None, axis=0):
    w = Waveform(kind=kind, amplitude=amplitude, p0=p0, p1=p1, t0=t0, table=None, table_len=0)
    keep = None
    if table is not None:
        tp, keep = _f64(table)
        w.table, w.table_len = tp, len(keep)
    _check(_lib.yf_set_source(C.c_void_p(g), axis, plane, j0, j1, k0, k1, C.byref(w)))


def add_port(g, plane, direction, j0, j1, k0, k1, kb, kt, margin, freqs, width=0.0, axis=0) -> int:
    d = PortDesc(axis=axis, plane=plane, direction=direction, j0=j0, j1=j1, k0=k0, k1=k1, kb=kb,
                 kt=kt, margin=margin, width=width)
    fp, keep = _f64(freqs)
    pid = C.c_int()
    _check(_lib.yf_add_port(C.c_void_p(g), C.byref(d), len(keep), fp, C.byref(pid)))
    return pid.value


def set_dft_mode(g, mask):
    _check(_lib.yf_set_dft_mode(C.c_void_p(g), mask))


def step(g, n):
    _check(_lib.yf_step(C.c_void_p(g), int(n)))


def sync(g):
    _check(_lib.yf_sync(C.c_void_p(g)))


def steps_done(g) -> int:
    n = C.c_long()
    _check(_lib.yf_steps_done(C.c_void_p(g), C.byref(n)))
    return n.value


def read_fields(g, comp, out):
    """Fill `out` (numpy or torch, shape (nz+1, ny+1, nx+1), grid precision)."""
    p, where, keep = _ptr(out)
    _check(_lib.yf_read_fields(C.c_void_p(g), comp, p, where))
    return out


def write_fields(g, comp, src):
    p, where, keep = _ptr(src)
    _check(_lib.yf_write_fields(C.c_void_p(g), comp, p, where))


def energy(g) -> float:
    out = C.c_double()
    _check(_lib.yf_energy(C.c_void_p(g), C.byref(out)))
    return out.value


def read_port_dft(g, port, nfreq, kind=DFT_FP64):
    """Returns (V, I) complex arrays of length nfreq."""
    a = np.zeros((4, nfreq))
    ptrs = [a[q].ctypes.data_as(_dp) for q in range(4)]
    _check(_lib.yf_read_port_dft(C.c_void_p(g), port, kind, *ptrs))
    return a[0] + 1j * a[1], a[2] + 1j * a[3]


def _cplx_out(shape):
    buf = np.zeros(shape + (2,))
    return buf, buf.ctypes.data_as(_dp)


def _as_complex(buf):
    return buf[..., 0] + 1j * buf[..., 1]


def sparams(freqs, V_inc, I_inc, V_tot, z_ref=50.0):
    """Full protocol: V_inc, I_inc (N, F) complex; V_tot (N driven, N port, F) complex.
    Returns dict(S_star (F,N,N), S (F,N,N), Zr (N,F), Zc (F,) or None, tau (F,N,N))."""
    V_inc = np.asarray(V_inc); I_inc = np.asarray(I_inc); V_tot = np.asarray(V_tot)
    N, F = V_inc.shape
    keep = []

    def spec(v, i=None):
        arrs = [np.ascontiguousarray(v.real), np.ascontiguousarray(v.imag)]
        if i is not None:
            arrs += [np.ascontiguousarray(i.real), np.ascontiguousarray(i.imag)]
        else:
            arrs += [np.zeros(F), np.zeros(F)]
        keep.extend(arrs)
        return PortDfts(*[x.ctypes.data_as(_dp) for x in arrs])

    inc = (PortDfts * N)(*[spec(V_inc[j], I_inc[j]) for j in range(N)])
    tot = (PortDfts * (N * N))(*[spec(V_tot[j, i]) for j in range(N) for i in range(N)])
    fr, kf = _f64(freqs)
    ss, ssp = _cplx_out((F, N, N))
    s, sp = _cplx_out((F, N, N))
    zr, zrp = _cplx_out((N, F))
    zc, zcp = _cplx_out((F,))
    tau = np.zeros((F, N, N))
    _check(_lib.yf_sparams(N, F, fr, inc, tot, z_ref, ssp, sp, zrp, zcp if N == 2 else None,
                           tau.ctypes.data_as(_dp)))
    return dict(S_star=_as_complex(ss), S=_as_complex(s), Zr=_as_complex(zr),
                Zc=_as_complex(zc) if N == 2 else None, tau=tau)


def sparams_noalloc(nports, nfreq, freqs, V_inc, I_inc, V_tot, S, Zr, S_star=None, Zc=None,
                    tau=None, z_ref=50.0, stream=None):
    """Allocation-free extraction: every argument is a CUDA tensor owned by the caller
    (float64; complex values interleaved as a trailing dimension of 2).  Asynchronous on
    `stream` (a cudaStream_t handle, or None for the legacy default stream)."""
    def ptr(t):
        return None if t is None else C.c_void_p(t.data_ptr())
    _check(_lib.yf_sparams_noalloc(nports, nfreq, ptr(freqs), ptr(V_inc), ptr(I_inc), ptr(V_tot),
                                   z_ref, ptr(S_star), ptr(S), ptr(Zr), ptr(Zc), ptr(tau),
                                   C.c_void_p(int(stream)) if stream else None))


def read_sparams(g, nfreq, z_ref=50.0, kind=DFT_FP64):
    ss, ssp = _cplx_out((nfreq, 2, 2))
    s, sp = _cplx_out((nfreq, 2, 2))
    zr, zrp = _cplx_out((2, nfreq))
    zc, zcp = _cplx_out((nfreq,))
    tau = np.zeros((nfreq, 2, 2))
    if kind == DFT_FP64:
        _check(_lib.yf_read_sparams(C.c_void_p(g), z_ref, ssp, sp, zrp, zcp, tau.ctypes.data_as(_dp)))
    else:
        _check(_lib.yf_read_sparams_acc(C.c_void_p(g), kind, z_ref, ssp, sp, zrp, zcp,
                                        tau.ctypes.data_as(_dp)))
    return dict(S_star=_as_complex(ss), S=_as_complex(s), Zr=_as_complex(zr), Zc=_as_complex(zc),
                tau=tau)


def rlcg(freqs, S_star, Zr, length):
    """Telegrapher's model: dict(gamma [F] complex, R, L, G, C [F]) from S* [F,2,2] and
    Z_r [2,F] (complex arrays, as sparams returns them) of a line of `length` metres."""
    fr, kf = _f64(freqs)
    F = len(kf)
    ss = np.ascontiguousarray(np.stack([np.asarray(S_star).real, np.asarray(S_star).imag], axis=-1))
    zr = np.ascontiguousarray(np.stack([np.asarray(Zr).real, np.asarray(Zr).imag], axis=-1))
    g = np.zeros((F, 2))
    out = [np.zeros(F) for _ in range(4)]
    _check(_lib.yf_rlcg(F, fr, ss.ctypes.data_as(_dp), zr.ctypes.data_as(_dp), float(length),
                        g.ctypes.data_as(_dp), *[o.ctypes.data_as(_dp) for o in out]))
    return dict(gamma=g[:, 0] + 1j * g[:, 1], R=out[0], L=out[1], G=out[2], C=out[3])


def set_variant(g, variant, tile_y=8, kseg=16):
    _check(_lib.yf_set_variant(C.c_void_p(g), variant, tile_y, kseg))


def set_box_shape(g, tile_y=0, planes=0):
    """Variant 4: tile height (8 or 16; 0: 8) and z-planes (0: twice kseg) of the two-step
    blocks; the fields do not depend on either."""
    _check(_lib.yf_set_box_shape(C.c_void_p(g), int(tile_y), int(planes)))


def autotune(g, cache_path=None, reps=4):
    """(tile_y, kseg) chosen for grid g (before its first step); state is reset to zero."""
    ty, ks = C.c_int(), C.c_int()
    _check(_lib.yf_autotune(C.c_void_p(g), cache_path.encode() if cache_path else None, reps,
                            C.byref(ty), C.byref(ks)))
    return ty.value, ks.value


def reset(g):
    _check(_lib.yf_reset(C.c_void_p(g)))


def profile_steps(g, n):
    """{kernel name: mean ms per launch} over n un-graphed steps (CUDA events)."""
    ms = (C.c_double * 8)()
    nk = C.c_int()
    _check(_lib.yf_profile_steps(C.c_void_p(g), int(n), ms, C.byref(nk)))
    return {_lib.yf_kernel_name(C.c_void_p(g), q).decode(): ms[q] for q in range(nk.value)}


def bounded_wait_check(preset_flag: bool, limit_seconds: float):
    _check(_lib.yf_bounded_wait_check(1 if preset_flag else 0, limit_seconds))


def launches_per_step(g) -> int:
    n = C.c_int()
    _check(_lib.yf_launches_per_step(C.c_void_p(g), C.byref(n)))
    return n.value


def tb_box(g):
    """Variant 4's inner box (x0, x1, y0, y1, z0, z1), or None when the grid has none."""
    b = (_i * 6)()
    _check(_lib.yf_tb_box(C.c_void_p(g), b))
    return None if b[0] < 0 else tuple(b)


def launches(g, nsteps: int) -> int:
    """Kernel launches that step(g, nsteps) issues from the current state."""
    n = C.c_long()
    _check(_lib.yf_launches(C.c_void_p(g), int(nsteps), C.byref(n)))
    return n.value


def checkpoint_save(g, path):
    _check(_lib.yf_checkpoint_save(C.c_void_p(g), path.encode()))


def checkpoint_load(g, path):
    _check(_lib.yf_checkpoint_load(C.c_void_p(g), path.encode()))


# ----------------------------------------------------------------- problem set-up helper

class Grid:
    """Owns one yf_grid handle configured from a workloads.Problem."""

    def __init__(self, prob, prec=FP32, stream=None, dt: Optional[float] = None,
                 dft_mask: int = DFT_FP64, with_source: bool = True, with_ports: bool = True,
                 variant: Optional[int] = None, tile_y: int = 8, kseg: int = 16,
                 box_seg: int = 0, box_ty: int = 0):
        self.prob = prob
        self.prec = prec
        if dt is None:
            dt = courant_dt(prob.dx, prob.dy, prob.dz, prob.courant)
        self.h = grid_create(prob.nx, prob.ny, prob.nz, prob.dx, prob.dy, prob.dz, dt, prec, stream)
        self.dt = grid_dt(self.h)
        try:
            set_materials(self.h, prob.ids, prob.eps_r, prob.sigma, prob.mu_r, prob.is_pec)
            for sh in prob.sheets:
                add_pec_sheet(self.h, *sh)
            set_boundaries(self.h, prob.bc)
            set_pml(self.h, prob.pml_cells, prob.pml_order, prob.pml_sigma_scale,
                    prob.pml_kappa_max, prob.pml_alpha_max)
            s = prob.source
            if with_source and s.kind != WAVE_NONE:
                set_source(self.h, s.plane, s.j0, s.j1, s.k0, s.k1, s.kind, s.amplitude, s.param0,
                           s.param1, s.t0, s.table)
            self.nports = 0
            if with_ports:
                for p in prob.ports:
                    add_port(self.h, p.plane, p.direction, p.j0, p.j1, p.k0, p.k1, p.kb, p.kt,
                             p.margin, prob.freqs, p.width)
                    self.nports += 1
            set_dft_mode(self.h, dft_mask)
            if variant is not None:
                set_variant(self.h, variant, tile_y, kseg)
            if box_seg or box_ty:
                set_box_shape(self.h, box_ty, box_seg)
        except Exception:
            grid_destroy(self.h)
            self.h = None
            raise

    def step(self, n):
        step(self.h, n)

    def sync(self):
        sync(self.h)

    def fields(self, box=None) -> np.ndarray:
        """All six components as float64 (6, nz+1, ny+1, nx+1), or only the node box
        ((x0, x1), (y0, y1), (z0, z1)) inclusive of x1, y1, z1 when given."""
        p = self.prob
        dt = np.float32 if self.prec == FP32 else np.float64
        buf = np.zeros((p.nz + 1, p.ny + 1, p.nx + 1), dtype=dt)
        if box is None:
            sl = (slice(None),) * 3
        else:
            (x0, x1), (y0, y1), (z0, z1) = box
            sl = (slice(z0, z1 + 1), slice(y0, y1 + 1), slice(x0, x1 + 1))
        out = None
        for c in range(6):
            read_fields(self.h, c, buf)
            part = buf[sl]
            if out is None:
                out = np.zeros((6,) + part.shape)
            out[c] = part
        return out

    def set_fields(self, f: np.ndarray):
        dt = np.float32 if self.prec == FP32 else np.float64
        for c in range(6):
            write_fields(self.h, c, np.ascontiguousarray(f[c], dtype=dt))

    def port_dfts(self, kind=DFT_FP64):
        nf = len(self.prob.freqs)
        V = np.zeros((self.nports, nf), complex)
        I = np.zeros((self.nports, nf), complex)
        for q in range(self.nports):
            V[q], I[q] = read_port_dft(self.h, q, nf, kind)
        return V, I

    def sparams(self, kind=DFT_FP64, z_ref=50.0):
        """Uniform-line extraction (two ports, driven at port 0) from accumulator set `kind`."""
        return read_sparams(self.h, len(self.prob.freqs), z_ref, kind)

    def close(self):
        if self.h is not None:
            grid_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- batched instances

class Batch:
    """Owns a yf_batch of workloads.Problem instances (one shared time step)."""

    def __init__(self, probs, prec=FP32, stream=None, dt: float = 0.0, tile_y: int = 8,
                 kseg: int = 16, variant: int = 2):
        self.probs = list(probs)
        if dt <= 0.0:
            # the instances' own Courant numbers: the smallest of their time steps
            dt = min(courant_dt(p.dx, p.dy, p.dz, p.courant) for p in self.probs)
        n = len(self.probs)
        descs = (InstanceDesc * n)()
        self._keep = []
        for q, p in enumerate(self.probs):
            d = descs[q]
            d.nx, d.ny, d.nz, d.dx, d.dy, d.dz = p.nx, p.ny, p.nz, p.dx, p.dy, p.dz
            ids = np.ascontiguousarray(p.ids, dtype=np.uint8)
            eps, ke = _f64(p.eps_r)
            sig, ks = _f64(p.sigma)
            mu, km = _f64(p.mu_r)
            pec = np.ascontiguousarray(np.asarray(p.is_pec, dtype=np.uint8))
            sh = np.ascontiguousarray(np.array(p.sheets, dtype=np.int32).reshape(-1, 6))
            fr, kf = _f64(p.freqs)
            ports = (PortDesc * max(1, len(p.ports)))()
            for k, pt in enumerate(p.ports):
                ports[k] = PortDesc(axis=0, plane=pt.plane, direction=pt.direction, j0=pt.j0,
                                    j1=pt.j1, k0=pt.k0, k1=pt.k1, kb=pt.kb, kt=pt.kt,
                                    margin=pt.margin, width=pt.width)
            self._keep += [ids, ke, ks, km, pec, sh, kf, ports]
            d.ids = C.c_void_p(ids.ctypes.data)
            d.nmat = len(ke)
            d.eps_r, d.sigma, d.mu_r = eps, sig, mu
            d.is_pec = C.c_void_p(pec.ctypes.data)
            d.nsheets = sh.shape[0]
            d.sheets = sh.ctypes.data_as(C.POINTER(C.c_int))
            for f in range(6):
                d.bc[f] = int(p.bc[f])
            d.pml_cells, d.pml_order = p.pml_cells, p.pml_order
            d.pml_sigma_scale, d.pml_kappa_max, d.pml_alpha_max = (p.pml_sigma_scale,
                                                                   p.pml_kappa_max,
                                                                   p.pml_alpha_max)
            s = p.source
            d.src_plane, d.src_j0, d.src_j1, d.src_k0, d.src_k1 = s.plane, s.j0, s.j1, s.k0, s.k1
            d.src = Waveform(kind=s.kind, amplitude=s.amplitude, p0=s.param0, p1=s.param1,
                             t0=s.t0, table=None, table_len=0)
            d.nports = len(p.ports)
            d.ports = ports
            d.nfreq = len(kf)
            d.freqs = fr
        h = C.c_void_p()
        st = C.c_void_p(int(stream)) if stream else None
        _check(_lib.yf_batch_create(n, descs, dt, prec, st, C.byref(h)))
        self.h = h.value
        if (tile_y, kseg) != (8, 16):
            _check(_lib.yf_batch_set_tiling(C.c_void_p(self.h), tile_y, kseg))
        if variant != 2:
            _check(_lib.yf_batch_set_variant(C.c_void_p(self.h), variant))
        self._keep.append(descs)
        cells = C.c_long()
        dtv = C.c_double()
        _check(_lib.yf_batch_info(C.c_void_p(self.h), None, C.byref(cells), C.byref(dtv), None))
        self.cells, self.dt = cells.value, dtv.value

    def set_tiling(self, tile_y, kseg):
        _check(_lib.yf_batch_set_tiling(C.c_void_p(self.h), tile_y, kseg))

    def set_variant(self, variant):
        _check(_lib.yf_batch_set_variant(C.c_void_p(self.h), variant))

    def autotune(self, cache_path=None, reps=3):
        ty, ks = C.c_int(), C.c_int()
        _check(_lib.yf_batch_autotune(C.c_void_p(self.h),
                                      cache_path.encode() if cache_path else None, reps,
                                      C.byref(ty), C.byref(ks)))
        return ty.value, ks.value

    def step(self, n):
        _check(_lib.yf_batch_step(C.c_void_p(self.h), int(n)))

    def sync(self):
        _check(_lib.yf_batch_sync(C.c_void_p(self.h)))

    def grid(self, inst) -> int:
        g = C.c_void_p()
        _check(_lib.yf_batch_grid(C.c_void_p(self.h), inst, C.byref(g)))
        return g.value

    def port_dfts(self, inst, kind=DFT_FP64):
        p = self.probs[inst]
        nf = len(p.freqs)
        V = np.zeros((len(p.ports), nf), complex)
        I = np.zeros((len(p.ports), nf), complex)
        for q in range(len(p.ports)):
            a = np.zeros((4, nf))
            _check(_lib.yf_batch_read_port_dft(C.c_void_p(self.h), inst, q, kind,
                                               *[a[r].ctypes.data_as(_dp) for r in range(4)]))
            V[q], I[q] = a[0] + 1j * a[1], a[2] + 1j * a[3]
        return V, I

    def sparams(self, inst, z_ref=50.0):
        return read_sparams(self.grid(inst), len(self.probs[inst].freqs), z_ref)

    def fields(self, inst, prec=None) -> np.ndarray:
        p = self.probs[inst]
        dt_ = np.float32 if (prec or FP32) == FP32 else np.float64
        out = np.zeros((6, p.nz + 1, p.ny + 1, p.nx + 1))
        buf = np.zeros((p.nz + 1, p.ny + 1, p.nx + 1), dtype=dt_)
        g = self.grid(inst)
        for c in range(6):
            read_fields(g, c, buf)
            out[c] = buf
        return out

    def close(self):
        if getattr(self, "h", None):
            _lib.yf_batch_destroy(C.c_void_p(self.h))
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- surrogate MLP (yfmlp.h)

MLP_IN, MLP_WIDTH, MLP_OUT, MLP_LAYERS, MLP_PARAMS = 6, 512, 512, 5, 1054208


def mlp_unflatten(flat: np.ndarray):
    """Flat parameter vector -> [(W_l (out, in), b_l (out,))] in the yfmlp.h layout."""
    out, off = [], 0
    for l in range(MLP_LAYERS):
        fin = MLP_IN if l == 0 else MLP_WIDTH
        W = flat[off:off + MLP_WIDTH * fin].reshape(MLP_WIDTH, fin)
        off += MLP_WIDTH * fin
        b = flat[off:off + MLP_WIDTH]
        off += MLP_WIDTH
        out.append((W, b))
    assert off == MLP_PARAMS
    return out


def mlp_flatten(params) -> np.ndarray:
    return np.concatenate([np.concatenate([np.asarray(W).ravel(), np.asarray(b).ravel()])
                           for W, b in params])


class Mlp:
    """Owns one yf_mlp handle (an ensemble of `members` surrogate networks)."""

    def __init__(self, members: int, train_batch: int, max_query: int, in_lo, in_hi, stream=None):
        h = C.c_void_p()
        lo, klo = _f64(in_lo)
        hi, khi = _f64(in_hi)
        s = C.c_void_p(int(stream)) if stream else None
        _check(_lib.yf_mlp_create(members, train_batch, max_query, lo, hi, s, C.byref(h)))
        self.h = h.value
        self.members, self.batch, self.max_query = members, train_batch, max_query

    def set_params(self, member: int, flat: np.ndarray):
        p, k = _f64(flat)
        assert k.size == MLP_PARAMS
        _check(_lib.yf_mlp_set_params(C.c_void_p(self.h), member, p))

    def get_params(self, member: int) -> np.ndarray:
        out = np.zeros(MLP_PARAMS)
        _check(_lib.yf_mlp_get_params(C.c_void_p(self.h), member, out.ctypes.data_as(_dp)))
        return out

    def set_adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(_lib.yf_mlp_set_adam(C.c_void_p(self.h), lr, beta1, beta2, eps))

    @staticmethod
    def _f32(a):
        if hasattr(a, "data_ptr"):
            assert str(a.dtype) == "torch.float32"
            a = a.contiguous()
            return C.c_void_p(a.data_ptr()), (DEVICE if a.is_cuda else HOST), a
        arr = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
        return C.c_void_p(arr.ctypes.data), HOST, arr

    def grads(self, member: int, x, t):
        """(loss, flat gradient) of one batch, no update."""
        px, wx, kx = self._f32(x)
        pt, wt, kt = self._f32(t)
        assert wx == wt
        loss = C.c_double()
        g = np.zeros(MLP_PARAMS)
        _check(_lib.yf_mlp_grads(C.c_void_p(self.h), member, px, pt, wx, C.byref(loss),
                                 g.ctypes.data_as(_dp)))
        return loss.value, g

    def train_step(self, member: int, x, t, want_loss: bool = False):
        px, wx, kx = self._f32(x)
        pt, wt, kt = self._f32(t)
        assert wx == wt
        loss = C.c_double()
        _check(_lib.yf_mlp_train_step(C.c_void_p(self.h), member, px, pt, wx,
                                      C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def fit(self, member: int, x, t, idx, lr, steps: int):
        """Graph-replayed Adam steps on device tensors: x [n, 6], t [n, 512] float32,
        idx [steps * batch] int32 rows, lr [steps] float32.  Asynchronous (see sync)."""
        for a in (x, t, idx, lr):
            assert hasattr(a, "data_ptr") and a.is_cuda and a.is_contiguous()
        assert idx.numel() >= steps * self.batch and lr.numel() >= steps
        _check(_lib.yf_mlp_fit(C.c_void_p(self.h), member, C.c_void_p(x.data_ptr()),
                               C.c_void_p(t.data_ptr()), int(x.shape[0]),
                               C.c_void_p(idx.data_ptr()), C.c_void_p(lr.data_ptr()), int(steps)))

    def sync(self) -> float:
        loss = C.c_double()
        _check(_lib.yf_mlp_sync(C.c_void_p(self.h), C.byref(loss)))
        return loss.value

    def query(self, x, y=None, est=None):
        """Ensemble mean [n, 512] and disagreement [n].  With torch CUDA tensors y and est given,
        everything stays on the device (asynchronous)."""
        px, wx, kx = self._f32(x)
        n = int(kx.shape[0])
        if y is None:
            yo = np.zeros((n, MLP_OUT), dtype=np.float32)
            eo = np.zeros(n, dtype=np.float32)
            _check(_lib.yf_mlp_query(C.c_void_p(self.h), px, n, wx, C.c_void_p(yo.ctypes.data),
                                     C.c_void_p(eo.ctypes.data), HOST))
            return yo, eo
        _check(_lib.yf_mlp_query(C.c_void_p(self.h), px, n, wx, C.c_void_p(y.data_ptr()),
                                 C.c_void_p(est.data_ptr()) if est is not None else None, DEVICE))
        return y, est

    def gate(self, est, scale: float, threshold: float):
        """(flags int32 [n], number flagged) for host est."""
        e = np.ascontiguousarray(np.asarray(est, dtype=np.float32))
        flags = np.zeros(e.size, dtype=np.int32)
        cnt = C.c_int()
        _check(_lib.yf_mlp_gate(C.c_void_p(self.h), C.c_void_p(e.ctypes.data), e.size, scale,
                                threshold, HOST, C.c_void_p(flags.ctypes.data), C.byref(cnt)))
        return flags, cnt.value

    def query_stats(self):
        n = C.c_int()
        fl = C.c_double()
        _check(_lib.yf_mlp_query_stats(C.c_void_p(self.h), C.byref(n), C.byref(fl)))
        return n.value, fl.value

    def close(self):
        if getattr(self, "h", None):
            _lib.yf_mlp_destroy(C.c_void_p(self.h))
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
