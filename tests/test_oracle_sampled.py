"""Pins of the oracle's point-by-point and pair-by-pair forms (oracle/grid.py: density_at,
integrals_at), used to check the full-size workload on sampled outputs: on small systems they
must equal the full-grid routines (themselves pinned against brute force on the whole grid) at
every sampled point and pair, including points outside every support and boxes that wrap the
periodic cell."""
import numpy as np

from oracle import grid
from paper_1507_08157_gb300 import synthetic as sy


def _case(recipe):
    s = sy.generate(recipe)
    return s, grid.BoxedSet(s.chi, s.n), grid.BoxedSet(s.phi, s.n)


def test_density_at_equals_full_grid(tiny_system):
    s = tiny_system
    chi, phi = grid.BoxedSet(s.chi, s.n), grid.BoxedSet(s.phi, s.n)
    Pp, Pq = sy.random_kernels(s, 2, 3)
    full = grid.response_density(chi, phi, Pq)
    rng = np.random.default_rng(4)
    pts = [tuple(int(v) for v in rng.integers(0, s.n, size=3)) for _ in range(60)] + [(0, 0, 0), (s.n - 1,) * 3]
    got = grid.density_at(chi, phi, Pq, pts)
    ref = np.array([[full[q][p] for p in pts] for q in range(2)])
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(full))


def test_integrals_at_equals_full_sums():
    s, chi, phi = _case(sy.Recipe(natoms=2, cell_ang=7.0, ngrid=20, radius_ang=2.8, seed=5))   # wrapping boxes
    rng = np.random.default_rng(6)
    V = rng.normal(size=(2, s.n, s.n, s.n))
    full = grid.potential_integrals(chi, phi, V, s.dV)
    pairs = [(int(a), int(b)) for a, b in zip(rng.integers(0, s.chi.nfun, 25), rng.integers(0, s.phi.nfun, 25))]
    got = grid.integrals_at(chi, phi, V, s.dV, pairs)
    ref = np.array([[full[q][a, b] for (a, b) in pairs] for q in range(2)])
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(full))


def test_density_at_wrapping_boxes_against_brute_force():
    s, chi, phi = _case(sy.Recipe(natoms=2, cell_ang=7.0, ngrid=20, radius_ang=2.8, nchi=9, seed=5))
    _, Pq = sy.random_kernels(s, 2, 8)
    X = grid.full_grid(s.chi, s.n).reshape(s.chi.nfun, -1)
    F = grid.full_grid(s.phi, s.n).reshape(s.phi.nfun, -1)
    rng = np.random.default_rng(9)
    pts = [tuple(int(v) for v in rng.integers(0, s.n, size=3)) for _ in range(40)]
    idx = [(p[0] * s.n + p[1]) * s.n + p[2] for p in pts]
    ref = np.einsum("ar,sab,br->sr", X[:, idx], Pq, F[:, idx])
    got = grid.density_at(chi, phi, Pq, pts)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_points_outside_every_support_are_zero():
    # two atoms in a 4 A cube at the centre of a 16 A cell, 3 A radius: the corners are empty
    s, chi, phi = _case(sy.Recipe(natoms=2, cell_ang=16.0, ngrid=48, radius_ang=3.0, cluster_ang=4.0, seed=7))
    _, Pq = sy.random_kernels(s, 1, 10)
    pts = [(0, 0, 0), (s.n - 1, 0, s.n - 1), (2, s.n - 3, 1)]
    assert np.all(grid.density_at(chi, phi, Pq, pts) == 0.0)
    assert np.any(grid.density_at(chi, phi, Pq, [(s.n // 2,) * 3]) != 0.0)
