"""Pins of the oracle's LDA kernel and Hartree solve against facts outside the oracle."""
import os

import numpy as np
import pytest

from oracle import hartree, xc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ueg_xc.txt")


def _golden():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            kind, rs, val, tol = line.split()
            rows.append((kind, float(rs), float(val), float(tol)))
    return rows


@pytest.mark.parametrize("row", _golden())
def test_uniform_gas_energies(row):
    kind, rs, val, tol = row
    if kind == "exchange_times_rs":
        n = 3.0 / (4.0 * np.pi * rs ** 3)
        got = xc.eps_x(n) * rs
    else:
        got = xc.eps_c(np.array(rs))
    assert abs(got - val) <= tol


def test_correlation_high_density_limit():
    # Gell-Mann--Brueckner: d eps_c / d ln rs -> (1 - ln 2) / pi^2 as rs -> 0
    rs = np.array([1e-9, 1e-8])
    e = xc.eps_c(rs)
    slope = (e[1] - e[0]) / np.log(10.0)
    assert abs(slope - (1.0 - np.log(2.0)) / np.pi ** 2) < 2e-5


@pytest.mark.parametrize("n", [1e-6, 1e-4, 1e-2, 0.3, 5.0])
def test_fxc_is_second_derivative_of_energy_density(n):
    # central second difference of n*eps_xc(n), relative step 1e-3 -> truncation error ~1e-7
    d = 1e-3 * n
    e = xc.exc_density(np.array([n - d, n, n + d]))
    fd = (e[0] - 2.0 * e[1] + e[2]) / (d * d)
    got = xc.fxc_lda(np.array([n]))[0]
    assert abs(got - fd) <= 1e-5 * abs(fd)


def test_fxc_floor_and_sign():
    f = xc.fxc_lda(np.array([0.0, 1e-11, 1e-9, 1e-3, 1.0]))
    assert f[0] == 0.0 and f[1] == 0.0
    assert np.all(f[2:] < 0.0)   # LDA kernel is negative


def _gaussian_on_grid(n, cell, r0, sigma, q):
    """Periodic sum of q (pi sigma^2)^{-3/2} exp(-|r - r0|^2 / sigma^2) sampled on the grid."""
    x = np.arange(n) * cell / n
    out = np.zeros((n, n, n))
    for sx in (-1, 0, 1):
        for sy in (-1, 0, 1):
            for sz in (-1, 0, 1):
                dx = x[:, None, None] - r0[0] + sx * cell
                dy = x[None, :, None] - r0[1] + sy * cell
                dz = x[None, None, :] - r0[2] + sz * cell
                out += np.exp(-(dx * dx + dy * dy + dz * dz) / sigma ** 2)
    return q * out / (np.pi * sigma ** 2) ** 1.5


def test_hartree_matches_analytic_fourier_series():
    # v(r) = (1/V) sum_{G != 0} 4 pi / G^2 * q exp(-G^2 sigma^2 / 4) exp(i G (r - r0)),
    # summed explicitly over the same G set; aliasing (exp(-Gmax^2 sigma^2 / 4)) and image
    # truncation are < 1e-15 here.
    n, cell, sigma, q = 24, 10.0, 1.6, 1.3
    r0 = np.array([3.1, 5.7, 8.2])
    rho = _gaussian_on_grid(n, cell, r0, sigma, q)
    v = hartree.hartree(rho[None], cell)[0]
    m = np.fft.fftfreq(n, d=1.0 / n)
    x = np.arange(n) * cell / n
    ref = np.zeros((n, n, n))
    for mx in m:
        for my in m:
            for mz in m:
                if mx == 0 and my == 0 and mz == 0:
                    continue
                g = 2.0 * np.pi * np.array([mx, my, mz]) / cell
                g2 = g @ g
                amp = 4.0 * np.pi / g2 * q * np.exp(-g2 * sigma ** 2 / 4.0) / cell ** 3
                ph = (np.exp(1j * g[0] * (x - r0[0]))[:, None, None]
                      * np.exp(1j * g[1] * (x - r0[1]))[None, :, None]
                      * np.exp(1j * g[2] * (x - r0[2]))[None, None, :])
                ref += np.real(amp * ph)
    assert np.max(np.abs(v - ref)) < 1e-11 * np.max(np.abs(ref))


def test_hartree_energy_positive_and_neutral_mean():
    rng = np.random.default_rng(3)
    rho = rng.standard_normal((2, 12, 12, 12))
    v = hartree.hartree(rho, 9.0)
    assert np.all(np.einsum("sxyz,sxyz->s", rho, v) > 0.0)
    assert np.max(np.abs(v.mean(axis=(1, 2, 3)))) < 1e-12
