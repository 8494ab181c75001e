"""Pins of the oscillator-strength oracle (oracle/spectrum.py) against facts that do not come
from the module itself:

* the uncoupled problem (K = 0) has omega_cv = eps_c - eps_v and f_cv = (2/3) (eps_c - eps_v)
  |d_cv|^2 in closed form;
* the finite-basis Thomas-Reiche-Kuhn sum rule: with A - B = D diagonal, sum_i f_i over every
  excitation of the full problem equals (2/3) sum_a d_a^T D d_a whatever the coupling K (a
  dropped omega factor, a p used for q or a wrong normalisation breaks it);
* in the Tamm-Dancoff approximation the same sum is (2/3) sum_a d_a^T A d_a instead: it moves
  with K, the sum-rule violation of Sec. II A;
* the grid dipole of one Gaussian of known centre against its centre (closed form);
* the PCG's converged Ritz pairs (O2) reproduce the dense strengths of the lowest states;
* the Lorentzian's area is sum f and its peak height f / (pi gamma).
"""
import numpy as np
import pytest

from oracle import spectrum
from paper_1507_08157_gb300 import synthetic as sy


def test_uncoupled_strengths_closed_form(tiny_casida):
    om, f, mu = spectrum.dense_strengths(tiny_casida, "d_only")
    d = spectrum.ks_dipoles(tiny_casida)
    eps = tiny_casida.ks_differences()
    order = np.argsort(eps)
    assert np.allclose(om, eps[order], rtol=0, atol=1e-13)
    ref = (2.0 / 3.0) * eps * np.sum(d ** 2, axis=0)
    assert np.allclose(f, ref[order], rtol=1e-11, atol=1e-15)


def test_sum_rule_holds_for_the_full_problem(tiny_casida):
    d = spectrum.ks_dipoles(tiny_casida)
    eps = tiny_casida.ks_differences()
    trk = (2.0 / 3.0) * np.sum(eps[None, :] * d ** 2)
    _, f_full, _ = spectrum.dense_strengths(tiny_casida, "full")
    assert abs(np.sum(f_full) - trk) <= 1e-11 * trk
    # not trivially: the coupling moves the individual strengths
    _, f0, _ = spectrum.dense_strengths(tiny_casida, "d_only")
    assert np.max(np.abs(np.sort(f_full) - np.sort(f0))) > 1e-6 * np.max(f0)


def test_tda_sum_follows_a_not_d(tiny_casida):
    d = spectrum.ks_dipoles(tiny_casida)
    A, _, _, K = tiny_casida.matrices("full")
    _, f_tda, _ = spectrum.dense_strengths(tiny_casida, "tda")
    ref = (2.0 / 3.0) * np.einsum("ai,ij,aj->", d, A, d)
    assert abs(np.sum(f_tda) - ref) <= 1e-11 * abs(ref)
    shift = (2.0 / 3.0) * np.einsum("ai,ij,aj->", d, K, d)
    assert abs(shift) > 1e-8 * abs(ref)         # the TDA sum differs from the full one


def test_grid_dipole_of_a_gaussian():
    n, cell = 40, 20.0
    x = spectrum.positions(n, cell)
    c = np.array([1.3, -2.1, 0.7])
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    g = np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / 1.5)
    dV = (cell / n) ** 3
    g /= dV * g.sum()                            # unit charge
    mu = spectrum.grid_dipoles(g[None], cell, dV)[0]
    assert np.allclose(mu, c, atol=1e-10)        # a well-sampled Gaussian's discrete centroid


@pytest.mark.slow
def test_pcg_ritz_strengths_match_dense(tiny_system, tiny_operator, tiny_casida):
    from oracle import solver
    k = 3
    pcg = solver.PCG(tiny_operator, sy.initial_guess(tiny_system, k, 1))
    pcg.solve(tol=1e-9, max_iter=600)
    om, f, _ = spectrum.ritz_strengths(pcg)
    om_d, f_d, _ = spectrum.dense_strengths(tiny_casida, "full")
    assert np.max(np.abs(om - om_d[:k])) < 1e-9
    assert np.max(np.abs(f - f_d[:k])) <= 1e-6 * max(np.max(f_d[:k]), 1e-12) + 1e-12


def test_lorentzian_area_and_height():
    om = np.array([0.1, 0.13])
    f = np.array([0.4, 0.25])
    gamma = spectrum.LORENTZ_HWHM_EV / 27.211386246
    E = np.linspace(-40.0, 40.0, 2_000_001)
    S = spectrum.lorentzian_spectrum(E, om, f, gamma)
    area = np.sum(S) * (E[1] - E[0])
    assert abs(area - f.sum()) < 1e-4 * f.sum()  # tails beyond +-40 Ha hold ~2 gamma / (pi 40)
    single = spectrum.lorentzian_spectrum([0.1], om[:1], f[:1], gamma)[0]
    assert np.isclose(single, f[0] / (np.pi * gamma), rtol=1e-14)
