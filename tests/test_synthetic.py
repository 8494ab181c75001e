"""Host-side checks of the input generator (paper_1507_08157_gb300/synthetic.py):

* the linear-scaling series recipe: cell and grid sizes of the 500/1000/2000-atom members, and a
  small core + shell geometry that keeps the minimum separation, the core atoms inside the core
  sphere, the shell atoms between the two spheres, and the requested atom density;
* the spawned process pool that large systems use for the table sums gives the same overlaps,
  projectors and ground-state density as the threaded path, bit for bit.
"""
import math

import numpy as np

from paper_1507_08157_gb300 import synthetic as sy


def test_scaling_series_sizes():
    got = [(sy.scaling_recipe(N).cell_ang, sy.scaling_recipe(N).ngrid) for N in (500, 1000, 2000)]
    assert got == [(48.0, 192), (54.0, 216), (60.0, 240)]
    r = sy.scaling_recipe(500)
    assert (r.nphi, r.nchi, r.radius_ang, r.kernel_cutoff_ang, r.core_atoms) == (4, 9, 8.0, 15.0, 140)


def test_core_shell_geometry():
    natoms, core, density, sep = 60, 20, 0.1, 1.4
    cell = 40.0 * sy.BOHR_PER_ANG
    rho = density / sy.BOHR_PER_ANG ** 3
    pos = sy._rsa_sphere_positions(np.random.default_rng(3), natoms, cell, sep * sy.BOHR_PER_ANG, rho, core)
    r = np.linalg.norm(pos - 0.5 * cell, axis=1) / sy.BOHR_PER_ANG
    r_in = (3.0 * core / (4.0 * math.pi * density)) ** (1.0 / 3.0)
    r_out = (3.0 * natoms / (4.0 * math.pi * density)) ** (1.0 / 3.0)
    assert np.all(r[:core] <= r_in + 1e-9)
    assert np.all((r[core:] >= r_in - 1e-9) & (r[core:] <= r_out + 1e-9))
    d = pos[:, None, :] - pos[None, :, :]
    dist = np.sqrt(np.sum(d * d, axis=-1)) / sy.BOHR_PER_ANG
    assert np.min(dist + 1e9 * np.eye(natoms)) >= sep


def test_process_pool_matches_threads(monkeypatch):
    rec = sy.Recipe(natoms=5, cell_ang=10.0, ngrid=30, nchi=9, radius_ang=4.0, seed=21)
    a = sy.generate(rec)
    monkeypatch.setattr(sy, "_POOL_MIN_JOBS", 0)
    b = sy.generate(rec)
    for name in ("S_phi", "S_chi", "P_v", "P_c", "n0"):
        assert np.array_equal(getattr(a, name), getattr(b, name)), name
