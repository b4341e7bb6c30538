"""Pins of the FP64 post-processing oracle (Eq. 1, 2, 5-6, 7, 8) against closed forms."""
import json
import math
import os

import numpy as np
import pytest

from oracle import post

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_worked_numbers.json")


def _matched_line(z0, beta_l):
    """S* of a uniform line between matched (Z_r = Z0) ports: [[0, k], [k, 0]], k = e^{-j beta l}."""
    kap = np.exp(-1j * beta_l)
    S = np.zeros((len(kap), 2, 2), dtype=np.complex128)
    S[:, 0, 1] = S[:, 1, 0] = kap
    Zr = np.full((2, len(kap)), z0, dtype=np.complex128)
    return S, Zr, kap


def test_gamma_printed_in_paper():
    g = json.load(open(GOLDEN))["lossless_line"]
    gam = (g["z0"] - g["z_ref"]) / (g["z0"] + g["z_ref"])
    assert round(gam, g["printed_digits"]) == g["gamma"]


def test_renormalisation_reproduces_eq7_closed_form():
    """Eq. 5-6 applied to the matched 25-ohm line returns Eq. 7 (textbook S21 numerator)."""
    bl = np.linspace(0.05, 7.0, 97)
    S, Zr, kap = _matched_line(25.0, bl)
    Sn = post.renormalize(S, Zr, 50.0)
    s11, s21 = post.lossless_line_s(kap, -1.0 / 3.0)
    assert np.max(np.abs(Sn[:, 0, 0] - s11)) < 1e-14
    assert np.max(np.abs(Sn[:, 1, 0] - s21)) < 1e-14
    assert np.max(np.abs(Sn[:, 1, 1] - s11)) < 1e-14
    assert np.max(np.abs(Sn[:, 0, 1] - s21)) < 1e-14
    # lossless: power balance to roundoff
    assert np.max(np.abs(np.abs(Sn[:, 0, 0]) ** 2 + np.abs(Sn[:, 1, 0]) ** 2 - 1.0)) < 1e-14


def test_printed_eq7_s21_numerator_breaks_power_balance():
    """Why the textbook numerator is taken: the printed (1 - kappa^2) kappa is not lossless."""
    kap = np.exp(-1j * np.linspace(0.3, 3.0, 10))
    gam = -1.0 / 3.0
    s11 = (1 - kap ** 2) * gam / (1 - kap ** 2 * gam ** 2)
    s21_printed = (1 - kap ** 2) * kap / (1 - kap ** 2 * gam ** 2)
    assert np.max(np.abs(np.abs(s11) ** 2 + np.abs(s21_printed) ** 2 - 1.0)) > 0.1


def test_renormalisation_routes_agree_for_real_unequal_references():
    """Eq. 5-6 (reading: * marks the new reference) equals the pseudo-wave route
    Z = sqrt(Zr)(I+S*)(I-S*)^{-1}sqrt(Zr), S = (Z-50)(Z+50)^{-1} for real references."""
    rng = np.random.default_rng(1)
    F = 16
    S = (rng.normal(size=(F, 3, 3)) + 1j * rng.normal(size=(F, 3, 3))) * 0.2
    Zr = np.stack([np.full(F, 25.0), np.full(F, 40.0), np.full(F, 90.0)]).astype(np.complex128)
    a = post.renormalize(S, Zr)
    b = post.renormalize_pseudowave(S, Zr)
    assert np.max(np.abs(a - b)) < 1e-12


def test_identity_renormalisation():
    """References already at 50 ohm: S = S*."""
    rng = np.random.default_rng(2)
    S = (rng.normal(size=(5, 2, 2)) + 1j * rng.normal(size=(5, 2, 2))) * 0.3
    Zr = np.full((2, 5), 50.0 + 0j)
    assert np.max(np.abs(post.renormalize(S, Zr) - S)) < 1e-14


def test_characteristic_impedance_and_delay_of_matched_line():
    """A uniform line with known Z0 and beta: Z_c = Z0 (ABCD route) and tau = l/v (Eq. 8)."""
    z0, v, l = 37.5, 1.7e8, 2.0e-3
    freqs = np.linspace(1e9, 300e9, 200)
    bl = 2 * math.pi * freqs / v * l
    S, Zr, kap = _matched_line(z0, bl)
    zc = post.zc_from_sstar(S, Zr)
    # I - S* is singular at beta l = m pi, so the bound allows its conditioning there
    assert np.max(np.abs(zc - z0)) / z0 < 1e-10
    tau = post.phase_delay(S[:, 1, 0], freqs)
    assert np.max(np.abs(tau - l / v)) / (l / v) < 1e-12


def test_sstar_two_run_protocol_on_synthetic_waves():
    """Eq. 1-2 on synthetic incident / total spectra of a known 2-port with distinct port
    impedances recovers the power-mode matrix that generated them."""
    F = 8
    f = np.linspace(1, 2, F)
    Z = np.array([20.0 + 1j * f, 70.0 - 2j * f])                 # port references
    # a reciprocal power-normalised S* to recover
    s11, s22, s21 = 0.3 * np.exp(1j * f), -0.2 * np.exp(-0.5j * f), 0.7 * np.exp(-2j * f)
    Vinc = np.array([1.0 + 0.5j * f, 0.8 - 0.1j * f])
    Iinc = Vinc / Z
    Vtot = np.zeros((2, 2, F), dtype=np.complex128)
    Vtot[0, 0] = Vinc[0] * (1 + s11)
    Vtot[0, 1] = s21 * Vinc[0] / np.sqrt(Z[0] / Z[1])
    Vtot[1, 1] = Vinc[1] * (1 + s22)
    Vtot[1, 0] = s21 * Vinc[1] / np.sqrt(Z[1] / Z[0])
    S, Zr = post.sstar(Vinc, Iinc, Vtot)
    assert np.allclose(Zr, Z, rtol=1e-14)
    assert np.allclose(S[:, 0, 0], s11, atol=1e-14)
    assert np.allclose(S[:, 1, 1], s22, atol=1e-14)
    assert np.allclose(S[:, 1, 0], s21, atol=1e-14)
    assert np.allclose(S[:, 0, 1], s21, atol=1e-14)


def test_unwrap_handles_multiple_turns():
    ph = np.linspace(0, -1500.0, 400)
    wrapped = (ph + 180.0) % 360.0 - 180.0
    assert np.allclose(post.unwrap_deg(wrapped), ph, atol=1e-9)


def _line_sstar(R, L, G, C, length, freqs, zr):
    """S* of a uniform line of known per-unit-length R, L, G, C between real references zr,
    built from its ABCD matrix (cosh, sinh of gamma l) through the impedance matrix and the
    pseudo-wave relation S = (Zn - I)(Zn + I)^{-1}, Zn = R^{-1} Z R^{-1} (written here, not
    taken from the module under test)."""
    w = 2 * np.pi * freqs
    zs, yp = R + 1j * w * L, G + 1j * w * C
    gam, zc = np.sqrt(zs * yp), np.sqrt(zs / yp)
    out = np.zeros((len(freqs), 2, 2), complex)
    for f in range(len(freqs)):
        ch, sh = np.cosh(gam[f] * length), np.sinh(gam[f] * length)
        A, B, Cm, D = ch, zc[f] * sh, sh / zc[f], ch
        Z = np.array([[A / Cm, (A * D - B * Cm) / Cm], [1 / Cm, D / Cm]])
        Rn = np.diag(1 / np.sqrt(zr))
        Zn = Rn @ Z @ Rn
        out[f] = (Zn - np.eye(2)) @ np.linalg.inv(Zn + np.eye(2))
    return out


def test_rlcg_recovers_a_lossy_line():
    freqs = np.linspace(0.1e9, 20e9, 64)
    R, L, G, C, length = 5.0, 3.0e-7, 1.0e-3, 1.2e-10, 0.05
    zr = np.array([40.0, 60.0])
    S = _line_sstar(R, L, G, C, length, freqs, zr)
    out = post.rlcg(S, np.repeat(zr[:, None], len(freqs), axis=1), freqs, length)
    assert np.allclose(out["R"], R, rtol=1e-8)
    assert np.allclose(out["L"], L, rtol=1e-10)
    assert np.allclose(out["G"], G, rtol=1e-7)
    assert np.allclose(out["C"], C, rtol=1e-10)
    assert np.allclose(out["Zc"], np.sqrt((R + 2j * np.pi * freqs * L) / (G + 2j * np.pi * freqs * C)),
                       rtol=1e-10)


def test_rlcg_of_a_lossless_line_has_no_loss_terms():
    freqs = np.linspace(0.2e9, 30e9, 80)
    # beta l reaches 78 rad (unwrapping needed) and stays off multiples of pi, where
    # sinh(gamma l) = 0 and the ABCD matrix carries no Z_c
    L, C, length = 2.5e-7, 1.0e-10, 0.083
    S = _line_sstar(0.0, L, 0.0, C, length, freqs, np.array([50.0, 50.0]))
    out = post.rlcg(S, np.full((2, len(freqs)), 50.0), freqs, length)
    w = 2 * np.pi * freqs
    assert np.all(np.abs(out["R"]) <= 1e-8 * w * L) and np.all(np.abs(out["G"]) <= 1e-8 * w * C)
    assert np.allclose(out["L"], L, rtol=1e-10) and np.allclose(out["C"], C, rtol=1e-10)


@pytest.mark.parametrize("z0a,z0b", [(30.0, 80.0), (55.0 - 10j, 20.0 + 4j)])
def test_sstar_uniform_recovers_kappa_and_both_references(z0a, z0b):
    """Uniform-line mode (one run, S*_11 = 0): a forward wave that leaves port 0 with
    V0 = a, I0 = a / Z0a (current along port 0's +x) and reaches port 1 as
    V1 = kappa a sqrt(Z0b / Z0a), I1 = V1 / Z0b flowing along +x, i.e. recorded as -I1 in
    port 1's own -x direction.  Power-mode transmission b_1 / a_0 = (V1/sqrt Z0b)/(V0/sqrt
    Z0a) = kappa, and each port's reference is its own wave impedance.  The unequal
    references make a wrong sign of port 1's current, which only rotates sqrt(Z_r0/Z_r1) by
    90 degrees, visible."""
    F = 12
    f = np.linspace(0.5, 2.0, F)
    kap = 0.9 * np.exp(-1.7j * f)
    a = (1.0 + 0.3j * f) * 1e-3
    V0, I0 = a, a / z0a
    V1 = kap * a * np.sqrt(z0b / z0a)
    I1_fwd = V1 / z0b
    Vf = np.array([V0, V1])
    If = np.array([I0, -I1_fwd])
    S, Zr = post.sstar_uniform(Vf, If, [1, -1])
    assert np.allclose(Zr[0], z0a, rtol=1e-14) and np.allclose(Zr[1], z0b, rtol=1e-14)
    assert np.max(np.abs(S[:, 1, 0] - kap)) < 1e-14
    assert np.max(np.abs(S[:, 0, 1] - kap)) < 1e-14
    assert np.max(np.abs(S[:, 0, 0])) == 0.0 and np.max(np.abs(S[:, 1, 1])) == 0.0
