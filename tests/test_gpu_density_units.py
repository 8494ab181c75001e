"""The tensor-core response density on dense tiles (density_units_kernel): tiles whose chi or phi
lists exceed the per-tile kernels are cut into units of at most 320 chi and 128 phi, each unit's
part of rho added with float32 reductions. Checked against the FP64 oracle (oracle/grid.py)
element by element:

* dense90: 90 atoms (4 phi + 9 chi, 4.5 A functions) in a 12 A cell on a 36^3 grid: up to ~800 chi
  and ~360 phi on a tile, so every tile is several units (both lists cut) and the per-tile
  kernels cannot take the system;
* dense24 with the units forced (TDDFT_DENSITY_UNITS=1) on tiles that fit one unit, against the
  oracle and against the per-tile persistent kernel.

float16 operands with float32 accumulation: 2e-3 of the largest entry, as in the other
tensor-core density tests.
"""
import numpy as np
import pytest

from oracle import operator as oop
from paper_1507_08157_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

TOL = 2e-3


@pytest.fixture(scope="module")
def tddft():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_08157_gb300 import build, tddft as td
    build.build()
    td.load()
    return td


@pytest.fixture(scope="module")
def dense90():
    return sy.generate(sy.Recipe(natoms=90, cell_ang=12.0, ngrid=36, nchi=9, radius_ang=4.5, seed=77))


@pytest.fixture(scope="module")
def dense24():
    return sy.generate(sy.Recipe(natoms=24, cell_ang=12.0, ngrid=36, nchi=9, radius_ang=4.5, seed=31))


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_units_density_and_apply_match_oracle(tddft, dense90):
    s = dense90
    ctx = tddft.Context(s, precision="mixed", precond="none")
    op = oop.Operator(s)
    Pp, Pq = sy.random_kernels(s, 3, 4)
    rho = ctx.response_density(Pq)
    ref = op.response_density(Pq)
    for q in range(3):
        assert _rel(rho[q], ref[q]) <= TOL, q
    fp, fq = ctx.apply(Pp, Pq)
    rp, rq = op.apply(Pp, Pq)
    for q in range(3):
        assert _rel(fq[q], rq[q]) <= TOL, q
        assert _rel(fp[q], rp[q]) <= 3e-5, q


def test_forced_units_on_small_tiles(tddft, dense24, monkeypatch):
    s = dense24
    _, Pq = sy.random_kernels(s, 2, 5)
    per_tile = tddft.Context(s, precision="mixed", precond="none").response_density(Pq)
    monkeypatch.setenv("TDDFT_DENSITY_UNITS", "1")
    units = tddft.Context(s, precision="mixed", precond="none").response_density(Pq)
    ref = oop.Operator(s).response_density(Pq)
    for q in range(2):
        assert _rel(units[q], ref[q]) <= TOL, q
        assert _rel(units[q], per_tile[q]) <= TOL, q


def test_autotuner_picks_and_keeps_a_candidate(tddft, dense24):
    # every candidate is timed, one per stage is chosen and installed, and the context's results
    # after tuning still match the oracle
    s = dense24
    ctx = tddft.Context(s, precision="mixed", precond="none")
    rows = ctx.autotune(4)
    stages = {r["stage"] for r in rows}
    assert stages == {"response_density", "potential_integrals"}
    for st in stages:
        cand = [r for r in rows if r["stage"] == st]
        assert len(cand) >= 2 and sum(r["chosen"] for r in cand) == 1
        best = min(cand, key=lambda r: r["ms"])
        assert best["chosen"] and all(r["ms"] > 0 for r in cand)
    assert any(r["kind"] == "per-tile" for r in rows if r["stage"] == "response_density")
    Pp, Pq = sy.random_kernels(s, 2, 6)
    fp, fq = ctx.apply(Pp, Pq)
    rp, rq = oop.Operator(s).apply(Pp, Pq)
    for q in range(2):
        assert _rel(fq[q], rq[q]) <= TOL, q
