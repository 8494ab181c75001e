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
