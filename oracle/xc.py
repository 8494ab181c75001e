"""Adiabatic LDA exchange-correlation kernel f_xc[n0](r) (Sec. II A, the second functional
derivative of E_xc in the coupling matrix K).

Spin-unpolarised total-density kernel f_xc(n) = d^2 (n eps_xc(n)) / dn^2 with
  * Slater exchange, eps_x = -(3/4) (3/pi)^(1/3) n^(1/3);
  * Perdew-Wang 1992 correlation (Phys. Rev. B 45, 13244, Eq. 10 with p = 1 and the zeta = 0
    parameters of its Table I), eps_c(rs) = -2A (1 + a1 rs) ln(1 + 1 / (2A (b1 rs^1/2 + b2 rs
    + b3 rs^3/2 + b4 rs^2))), rs = (3 / (4 pi n))^(1/3).
The paper uses PBE (Sec. IV); the synthetic workloads use LDA. Where n0 < 1e-10 bohr^-3 the
kernel is set to zero (density floor; truncated Gaussians give n0 = 0 outside their spheres).
"""
import numpy as np

PW92_A = 0.031091
PW92_ALPHA1 = 0.21370
PW92_BETA = (7.5957, 3.5876, 1.6382, 0.49294)
DENSITY_FLOOR = 1e-10
CX = 0.75 * (3.0 / np.pi) ** (1.0 / 3.0)


def rs_of_n(n):
    return (3.0 / (4.0 * np.pi * n)) ** (1.0 / 3.0)


def eps_x(n):
    """Slater exchange energy per electron (Ha)."""
    return -CX * np.cbrt(n)


def _q1(rs):
    b1, b2, b3, b4 = PW92_BETA
    s = np.sqrt(rs)
    q1 = 2.0 * PW92_A * (b1 * s + b2 * rs + b3 * rs * s + b4 * rs * rs)
    dq1 = 2.0 * PW92_A * (0.5 * b1 / s + b2 + 1.5 * b3 * s + 2.0 * b4 * rs)
    d2q1 = 2.0 * PW92_A * (-0.25 * b1 / (rs * s) + 0.75 * b3 / s + 2.0 * b4)
    return q1, dq1, d2q1


def eps_c(rs):
    """PW92 correlation energy per electron (Ha), unpolarised."""
    q1, _, _ = _q1(rs)
    return -2.0 * PW92_A * (1.0 + PW92_ALPHA1 * rs) * np.log1p(1.0 / q1)


def eps_c_derivs(rs):
    """eps_c and its first two derivatives with respect to rs."""
    q1, dq1, d2q1 = _q1(rs)
    q0 = -2.0 * PW92_A * (1.0 + PW92_ALPHA1 * rs)
    dq0 = -2.0 * PW92_A * PW92_ALPHA1
    lg = np.log1p(1.0 / q1)
    den = q1 * q1 + q1
    dlg = -dq1 / den
    d2lg = -d2q1 / den + dq1 * dq1 * (2.0 * q1 + 1.0) / (den * den)
    e = q0 * lg
    de = dq0 * lg + q0 * dlg
    d2e = 2.0 * dq0 * dlg + q0 * d2lg
    return e, de, d2e


def exc_density(n):
    """n * eps_xc(n): the LDA energy per unit volume."""
    return n * (eps_x(n) + eps_c(rs_of_n(n)))


def fxc_lda(n0):
    """f_xc = d^2(n eps_xc)/dn^2 at the ground-state density, with the density floor."""
    n0 = np.asarray(n0, dtype=np.float64)
    out = np.zeros_like(n0)
    ok = n0 >= DENSITY_FLOOR
    n = n0[ok]
    fx = -(1.0 / 3.0) * (3.0 / np.pi) ** (1.0 / 3.0) / np.cbrt(n * n)
    rs = rs_of_n(n)
    _, de, d2e = eps_c_derivs(rs)
    fc = -(rs / (3.0 * n)) * ((2.0 / 3.0) * de - (rs / 3.0) * d2e)
    out[ok] = fx + fc
    return out
