"""Host-side checks of the input generator (paper_1507_08157_gb300/synthetic.py):

* the linear-scaling series recipe: cell and grid sizes of the 500/1000/2000-atom members, and a
  small core + shell geometry that keeps the minimum separation, the core atoms inside the core
  sphere, the shell atoms between the two spheres, and the requested atom density;
* the spawned process pool that large systems use for the table sums gives the same overlaps,
  projectors and ground-state density as the threaded path, bit for bit.
"""
import dataclasses
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


def test_separable_overlaps_equal_grid_sums():
    # 8 A functions (the series' radius): beyond it the Gaussians are below exp(-44) of their
    # peak, so the factored axis sums equal the grid sums of the hard-cut tables to rounding
    B = sy.BOHR_PER_ANG
    cell, n = 40.0 * B, 120
    R, h = 8.0 * B, cell / n
    pos = sy._rsa_positions(np.random.default_rng(1), 30, cell, 1.4 * B)
    for nper in (4, 9):
        par = {}
        fs = sy._tabulate(np.random.default_rng(2), pos, nper, cell, n, R, (0.6 * B, 1.2 * B), np.float64, par)
        grid = sy._overlap_matrix(fs, nper, pos, cell, n, h ** 3, 2.0 * R)
        sep = sy._separable_overlaps(fs, nper, pos, cell, n, h ** 3, 2.0 * R, par)
        assert np.max(np.abs(grid - sep)) < 1e-13


def test_fast_recipe_matches_plain_and_atomic_density():
    # the fast path (float32 tables, separable sums, one eigendecomposition) against the plain
    # path on the same recipe; its n0 is the superposition of on-site valence densities
    rec = sy.Recipe(natoms=12, cell_ang=40.0, ngrid=120, nchi=9, radius_ang=8.0, seed=6)
    a = sy.generate(rec)
    b = sy.generate(dataclasses.replace(rec, fast=True))
    assert b.phi.val.dtype == np.float32 and b.chi.val.dtype == np.float32
    assert np.max(np.abs(a.phi.val - b.phi.val)) <= 1e-7 * np.max(np.abs(a.phi.val))
    for name in ("S_phi", "S_chi"):
        assert np.max(np.abs(getattr(a, name) - getattr(b, name))) < 1e-13, name
    for name in ("P_v", "P_c", "H_chi"):
        assert np.max(np.abs(getattr(a, name) - getattr(b, name))) < 1e-9, name
    assert np.min(b.n0) >= -1e-12
    nper = rec.nphi
    onsite = sum(np.sum(b.P_v[i * nper:(i + 1) * nper, i * nper:(i + 1) * nper] *
                        b.S_phi[i * nper:(i + 1) * nper, i * nper:(i + 1) * nper]) for i in range(rec.natoms))
    assert abs(np.sum(b.n0) * (b.cell / b.n) ** 3 - 2.0 * onsite) <= 1e-5 * 2.0 * onsite
