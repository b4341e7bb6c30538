"""FP64 post-processing oracle: DFT of port histories and network-parameter extraction.

TEST INFRASTRUCTURE ONLY (tests/, __graft_entry__.smoke(), bench.py's CPU legs).
Shares no code with the CUDA library.

Follows Sec. II-A of arXiv 2208.04371:
  - DFT of the port voltage / current histories (Sec. II-A, F[.] in Eq. 1-2),
    here by direct summation with cos/sin of 2 pi frac(f t) at each sample's
    own time (V at t_{n+1}, I at t_{n+1/2}), convention X(f) = sum x e^{-j2pi f t} dt;
  - port reference impedance Z_r = F[V_inc] / F[I_inc]         (Eq. 2);
  - power-mode matrix S*                                       (Eq. 1);
  - renormalisation of S* to 50 ohm references                 (Eq. 5-6);
  - S* -> Z -> ABCD -> overall characteristic impedance Z_c    (end of Sec. II-A);
  - phase delay tau = theta / (360 f), theta unwrapped, degrees (Eq. 8).

Readings of the paper taken here (the printed text is garbled or silent):
  * Eq. 5: B = (Z* - Z_r)(Z* + Z_r)^{-1}; the "*" on G*, Z_r*, B* and A* marks
    the new 50 ohm reference, not complex conjugation, so B* = B and A* = A;
    A = G*^{-1} G (I - B).
  * theta = -unwrap(arg S*_21), so tau > 0 under the e^{-j omega t} DFT sign.
  * Uniform-line mode: port 1's reference is the forward wave's V/I with I taken
    along +x (against port 1's own direction); a synthetic forward wave with
    unequal references pins it (tests/test_oracle_post.py).
  * Eq. 7 (lossless line between 50 ohm ports): the printed S21 numerator
    (1 - kappa^2) kappa breaks |S11|^2 + |S21|^2 = 1; the textbook numerator
    (1 - Gamma^2) kappa is used, with kappa = e^{-j beta l} under this DFT sign.
"""
from __future__ import annotations

import math

import numpy as np


def dft(x: np.ndarray, freqs: np.ndarray, times: np.ndarray, dt: float) -> np.ndarray:
    """X(f_k) = sum_n x_n exp(-j 2 pi f_k t_n) dt, direct summation in FP64."""
    out = np.zeros(len(freqs), dtype=np.complex128)
    for k, f in enumerate(freqs):
        ft = f * times
        ph = 2.0 * math.pi * (ft - np.floor(ft))
        out[k] = np.sum(x * np.cos(ph)) * dt - 1j * np.sum(x * np.sin(ph)) * dt
    return out


def port_dfts(V: np.ndarray, I: np.ndarray, freqs: np.ndarray, dt: float):
    """DFT of each port's V (sampled at (n+1) dt) and I (sampled at (n+1/2) dt)."""
    n = V.shape[1]
    tv = (np.arange(n) + 1.0) * dt
    ti = (np.arange(n) + 0.5) * dt
    Vf = np.array([dft(V[p], freqs, tv, dt) for p in range(V.shape[0])])
    If = np.array([dft(I[p], freqs, ti, dt) for p in range(I.shape[0])])
    return Vf, If


def zref(V_inc: np.ndarray, I_inc: np.ndarray) -> np.ndarray:
    """Eq. 2: Z_r(f) = F[V_inc] / F[I_inc]."""
    return V_inc / I_inc


def sstar(V_inc: np.ndarray, I_inc: np.ndarray, V_tot: np.ndarray) -> tuple:
    """Eq. 1 for an N-port network measured with the two-run protocol.

    V_inc[j], I_inc[j] : (N, F) incident-run DFTs at the driven port j
    V_tot[j, i]        : (N, N, F) total-run DFT at port i when port j is driven
    Returns (S* as (F, N, N), Z_r as (N, F)).
    """
    N, F = V_inc.shape
    Zr = zref(V_inc, I_inc)
    S = np.zeros((F, N, N), dtype=np.complex128)
    for j in range(N):
        for i in range(N):
            if i == j:
                S[:, j, j] = (V_tot[j, j] - V_inc[j]) / V_inc[j]
            else:
                S[:, i, j] = V_tot[j, i] / V_inc[j] * np.sqrt(Zr[j] / Zr[i])
    return S, Zr


def sstar_uniform(Vf: np.ndarray, If: np.ndarray, directions) -> tuple:
    """Uniform two-port line driven at port 0 only: the incident and total runs
    coincide, S*_11 = S*_22 = 0 and S*_12 = S*_21 by symmetry.  Z_r at port 1 is
    taken from the same forward wave, whose current flows against port 1's own
    incident direction."""
    Zr0 = Vf[0] / If[0]
    Zr1 = Vf[1] / (If[1] * (-1.0))
    s21 = Vf[1] / Vf[0] * np.sqrt(Zr0 / Zr1)
    F = Vf.shape[1]
    S = np.zeros((F, 2, 2), dtype=np.complex128)
    S[:, 1, 0] = s21
    S[:, 0, 1] = s21
    return S, np.array([Zr0, Zr1])


def renormalize(S_star: np.ndarray, Zr: np.ndarray, z_new: float = 50.0) -> np.ndarray:
    """Eq. 5-6: S = A^{-1} (S* - B)(I - B S*)^{-1} A with
    B = diag((z_new - Z_r)/(z_new + Z_r)), G = diag(1/sqrt|Re Z_r|),
    G* = diag(1/sqrt(z_new)), A = G*^{-1} G (I - B)."""
    F, N, _ = S_star.shape
    out = np.zeros_like(S_star)
    Id = np.eye(N, dtype=np.complex128)
    for f in range(F):
        z = Zr[:, f]
        B = np.diag((z_new - z) / (z_new + z))
        G = np.diag(1.0 / np.sqrt(np.abs(z.real)))
        Gs_inv = np.diag(np.full(N, math.sqrt(z_new), dtype=np.complex128))
        A = Gs_inv @ G @ (Id - B)
        M = (S_star[f] - B) @ np.linalg.inv(Id - B @ S_star[f])
        out[f] = np.linalg.inv(A) @ M @ A
    return out


def renormalize_pseudowave(S_star: np.ndarray, Zr: np.ndarray, z_new: float = 50.0) -> np.ndarray:
    """Cross-check route: Z = sqrt(Z_r)(I + S*)(I - S*)^{-1} sqrt(Z_r), then
    S = (Z - z_new)(Z + z_new)^{-1}."""
    F, N, _ = S_star.shape
    out = np.zeros_like(S_star)
    Id = np.eye(N, dtype=np.complex128)
    for f in range(F):
        Z = zmatrix(S_star[f], Zr[:, f])
        out[f] = (Z - z_new * Id) @ np.linalg.inv(Z + z_new * Id)
    return out


def zmatrix(S: np.ndarray, zr: np.ndarray) -> np.ndarray:
    """Impedance matrix of one frequency from S and per-port references (pseudo-waves)."""
    N = S.shape[0]
    Id = np.eye(N, dtype=np.complex128)
    R = np.diag(np.sqrt(zr.astype(np.complex128)))
    return R @ (Id + S) @ np.linalg.inv(Id - S) @ R


def zc_from_sstar(S_star: np.ndarray, Zr: np.ndarray) -> np.ndarray:
    """Two-port S* -> Z -> ABCD (A = Z11/Z21, B = det Z / Z21, C = 1/Z21) and the
    overall characteristic impedance Z_c = sqrt(B/C) on the Re >= 0 branch."""
    F = S_star.shape[0]
    out = np.zeros(F, dtype=np.complex128)
    for f in range(F):
        Z = zmatrix(S_star[f], Zr[:, f])
        det = Z[0, 0] * Z[1, 1] - Z[0, 1] * Z[1, 0]
        Bm = det / Z[1, 0]
        Cm = 1.0 / Z[1, 0]
        zc = np.sqrt(Bm / Cm)
        if zc.real < 0:
            zc = -zc
        out[f] = zc
    return out


def rlcg(S_star: np.ndarray, Zr: np.ndarray, freqs: np.ndarray, length: float) -> dict:
    """Telegrapher's model of a two-port (end of Sec. II-A): S* -> Z -> ABCD, then
    gamma l = +-acosh((A + D) / 2) + 2 pi j k (cosh is even and periodic).  The lowest
    frequency takes beta l in [0, pi] (it must lie below pi, as for Eq. 8); every further
    frequency takes the candidate nearest the line's trend, beta l grown in proportion to f
    from the last frequency with a finite result (acosh folds beta l into [0, pi]).  The sign
    of alpha follows from beta > 0.  Z_c = sqrt(B / C) with Re >= 0; per unit length
    R + j w L = gamma Z_c, G + j w C = gamma / Z_c.  Where the conversion is singular (I - S*
    not invertible: a matched lossless line at beta l = m pi) the results are NaN."""
    F = S_star.shape[0]
    gl = np.full(F, np.nan + 0j)
    zc = np.full(F, np.nan + 0j)
    prev, fprev = None, None
    for f in range(F):
        with np.errstate(all="ignore"):
            try:
                Z = zmatrix(S_star[f], Zr[:, f])
            except np.linalg.LinAlgError:
                continue
            A, Bm, Cm, D = (Z[0, 0] / Z[1, 0], (Z[0, 0] * Z[1, 1] - Z[0, 1] * Z[1, 0]) / Z[1, 0],
                            1.0 / Z[1, 0], Z[1, 1] / Z[1, 0])
            z = np.sqrt(Bm / Cm)
            g = np.arccosh(0.5 * (A + D))
        if not (np.isfinite(g) and np.isfinite(z)):
            continue
        zc[f] = z if z.real >= 0 else -z
        if prev is None:
            g = g if (g.imag > 0 or (g.imag == 0 and g.real >= 0)) else -g
        else:
            pred = prev.imag * freqs[f] / fprev
            best = None
            for c in (g, -g):
                c = c + 2j * np.pi * np.round((pred - c.imag) / (2 * np.pi))
                if best is None or abs(c.imag - pred) < abs(best.imag - pred):
                    best = c
            g = best
        prev, fprev = g, freqs[f]
        gl[f] = g
    gamma = gl / length
    w = 2 * np.pi * freqs
    zs, yp = gamma * zc, gamma / zc
    return dict(gamma=gamma, Zc=zc, R=zs.real, L=zs.imag / w, G=yp.real, C=yp.imag / w)


def unwrap_deg(phase_deg: np.ndarray) -> np.ndarray:
    """Unwrap with period 360 degrees, in increasing-frequency order, starting at
    the first (lowest) frequency: each jump beyond 180 degrees is corrected."""
    out = np.array(phase_deg, dtype=np.float64)
    offset = 0.0
    for k in range(1, len(out)):
        d = phase_deg[k] - phase_deg[k - 1]
        if d > 180.0:
            offset -= 360.0
        elif d < -180.0:
            offset += 360.0
        out[k] = phase_deg[k] + offset
    return out


def phase_delay(s_ij: np.ndarray, freqs: np.ndarray) -> np.ndarray:
    """Eq. 8: tau = theta / (360 f), theta = -unwrap(arg S*_ij) in degrees."""
    theta = -unwrap_deg(np.degrees(np.angle(s_ij)))
    return theta / (360.0 * freqs)


# ---- closed forms used as pins -------------------------------------------------------------

def lossless_line_s(kappa: np.ndarray, gamma: float) -> tuple:
    """Eq. 7 (with the textbook S21 numerator): a lossless line of impedance Z0 between
    references z_ref, Gamma = (Z0 - z_ref)/(Z0 + z_ref), kappa = e^{-j beta l}."""
    den = 1.0 - kappa ** 2 * gamma ** 2
    s11 = (1.0 - kappa ** 2) * gamma / den
    s21 = (1.0 - gamma ** 2) * kappa / den
    return s11, s21


def microstrip_z0_hammerstad(w_over_h: float, eps_r: float) -> tuple:
    """Quasi-static microstrip impedance (Hammerstad-Jensen simplified forms), used only
    as a loose physical check of the simulated Z_r."""
    u = w_over_h
    eeff = (eps_r + 1) / 2 + (eps_r - 1) / 2 / math.sqrt(1 + 12 / u)
    if u <= 1:
        z0 = 60 / math.sqrt(eeff) * math.log(8 / u + u / 4)
    else:
        z0 = 120 * math.pi / (math.sqrt(eeff) * (u + 1.393 + 0.667 * math.log(u + 1.444)))
    return z0, eeff
