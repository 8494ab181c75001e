"""Pins of the oracle's box arithmetic against brute force on the whole grid."""
import numpy as np

from oracle import grid
from paper_1507_08157_gb300 import synthetic as sy


def _wrapped_system():
    # 2 atoms, one near a cell corner so its box wraps on all three axes; 20^3 grid (ragged vs 8)
    return sy.generate(sy.Recipe(natoms=2, cell_ang=7.0, ngrid=20, radius_ang=2.8, seed=5))


def test_boxes_wrap_and_normalise(tiny_system):
    s = tiny_system
    for fs in (s.phi, s.chi):
        full = grid.full_grid(fs, s.n)
        norms = s.dV * np.einsum("fxyz,fxyz->f", full, full)
        assert np.allclose(norms, 1.0, atol=1e-12)


def test_overlaps_match_full_grid(tiny_system):
    # the generator's S must be the Gram matrix of the tabulated functions
    s = tiny_system
    for fs, S in ((s.phi, s.S_phi), (s.chi, s.S_chi)):
        F = grid.full_grid(fs, s.n).reshape(fs.nfun, -1)
        assert np.allclose(s.dV * F @ F.T, S, atol=1e-12)


def test_response_density_matches_full_grid():
    s = _wrapped_system()
    chi = grid.BoxedSet(s.chi, s.n)
    phi = grid.BoxedSet(s.phi, s.n)
    rng = np.random.default_rng(0)
    P = rng.standard_normal((3, s.chi.nfun, s.phi.nfun))
    got = grid.response_density(chi, phi, P)
    X = grid.full_grid(s.chi, s.n).reshape(s.chi.nfun, -1)
    F = grid.full_grid(s.phi, s.n).reshape(s.phi.nfun, -1)
    ref = np.einsum("ar,sab,br->sr", X, P, F).reshape(got.shape)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_potential_integrals_match_full_grid():
    s = _wrapped_system()
    chi = grid.BoxedSet(s.chi, s.n)
    phi = grid.BoxedSet(s.phi, s.n)
    rng = np.random.default_rng(1)
    V = rng.standard_normal((2, s.n, s.n, s.n))
    got = grid.potential_integrals(chi, phi, V, s.dV)
    X = grid.full_grid(s.chi, s.n).reshape(s.chi.nfun, -1)
    F = grid.full_grid(s.phi, s.n).reshape(s.phi.nfun, -1)
    ref = s.dV * np.einsum("ar,sr,br->sab", X, V.reshape(2, -1), F)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_ground_state_density_integrates_to_electron_count(tiny_system):
    s = tiny_system
    assert abs(s.dV * s.n0.sum() - 2 * s.n_occ) < 1e-10
    F = grid.full_grid(s.phi, s.n).reshape(s.phi.nfun, -1)
    ref = 2.0 * np.einsum("ar,ab,br->r", F, s.P_v, F).reshape(s.n0.shape)
    assert np.max(np.abs(ref - s.n0)) < 1e-12 * np.max(s.n0)
