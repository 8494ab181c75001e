"""Parity of the CUDA operator path with the FP64 oracle, element by element, through the C ABI.

Cases: a 3-atom system on a 30^3 grid (tiles of 8 leave a ragged tail of 6), a 2-atom system whose
boxes wrap the periodic cell on every axis (20^3), a 9-chi (s, p, d) system, the 8-atom /
48^3 workload, and a dense 24-atom system whose tiles are cut into several tensor-core
integrals units. Tolerances, relative to the largest reference entry:
  * FP64 mode: 1e-10;
  * mixed mode, float32 stages (FFT Poisson + f_xc, potential integrals, matrix products on
    three-term-split TF32 tensor cores): 3e-5 (float32 roundoff 6e-8 times ~500-term tile sums and
    ~1000-term products, with margin);
  * mixed mode, response density and potential integrals on the tensor cores: float16 operands
    (unit roundoff 2^-11 = 4.9e-4) with float32 accumulation; the rounding errors of the
    products are independent, so the error is ~4.9e-4 times the rms term times sqrt(#terms),
    i.e. ~4.9e-4 of the result's own scale: 2e-3 of the largest entry. The same bound covers f in
    the full and TDA modes, whose coupling term is built from them.
"""
import numpy as np
import pytest

from oracle import grid as ogrid
from oracle import hartree as ohartree
from oracle import operator as oop
from oracle import xc as oxc
from paper_1507_08157_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 3e-5}
TOL_DENSITY = {"fp64": 1e-10, "mixed": 2e-3}


@pytest.fixture(scope="module")
def tddft():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_08157_gb300 import build, tddft as td
    build.build()
    td.load()
    return td


def _systems():
    return {
        "tiny30": sy.Recipe(natoms=3, cell_ang=10.0, ngrid=30, radius_ang=4.0, seed=11),
        "wrap20": sy.Recipe(natoms=2, cell_ang=7.0, ngrid=20, radius_ang=2.8, seed=5),
        "d9": sy.Recipe(natoms=3, cell_ang=10.0, ngrid=30, nchi=9, radius_ang=4.0, seed=12),
        # dense: up to 162 chi and 72 phi per tile, 36^3 grid (ragged tail of 4)
        "dense24": sy.Recipe(natoms=24, cell_ang=12.0, ngrid=36, nchi=9, radius_ang=4.5, seed=31),
    }


_CACHE = {}


def system(name):
    if name not in _CACHE:
        rec = sy.CONFIG_SMALL if name == "small48" else _systems()[name]
        _CACHE[name] = sy.generate(rec)
    return _CACHE[name]


def _err(got, ref):
    return float(np.max(np.abs(np.asarray(got) - ref)) / max(np.max(np.abs(ref)), 1e-300))


@pytest.mark.parametrize("name", ["tiny30", "wrap20", "small48"])
def test_fxc_matches_oracle(tddft, name):
    s = system(name)
    ctx = tddft.Context(s, precision="fp64")
    got = ctx.fxc()
    ref = oxc.fxc_lda(s.n0)
    assert _err(got, ref) < 1e-13


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["tiny30", "wrap20", "d9", "small48"])
def test_response_density(tddft, name, prec):
    s = system(name)
    ctx = tddft.Context(s, precision=prec)
    P = sy.random_kernels(s, 3, 1)[0]
    got = ctx.response_density(P)
    ref = ogrid.response_density(ogrid.BoxedSet(s.chi, s.n), ogrid.BoxedSet(s.phi, s.n), P)
    assert _err(got, ref) < TOL_DENSITY[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name,k", [("tiny30", 3), ("wrap20", 1), ("small48", 2)])
def test_response_potential_fft(tddft, name, k, prec):
    # k odd exercises the unpaired last state of the two-states-per-complex-FFT packing
    s = system(name)
    ctx = tddft.Context(s, precision=prec)
    rng = np.random.default_rng(2)
    rho = rng.standard_normal((k, s.n, s.n, s.n))
    got = ctx.response_potential(rho)
    ref = ohartree.hartree(rho, s.cell) + oxc.fxc_lda(s.n0)[None] * rho
    assert _err(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["tiny30", "wrap20", "d9"])
def test_potential_integrals(tddft, name, prec):
    s = system(name)
    ctx = tddft.Context(s, precision=prec)
    V = np.random.default_rng(3).standard_normal((2, s.n, s.n, s.n))
    got = ctx.potential_integrals(V)
    ref = ogrid.potential_integrals(ogrid.BoxedSet(s.chi, s.n), ogrid.BoxedSet(s.phi, s.n), V, s.dV)
    assert _err(got, ref) < TOL_DENSITY[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("mode", ["full", "tda", "d_only"])
@pytest.mark.parametrize("name", ["tiny30", "d9", "small48"])
def test_apply_matches_oracle(tddft, name, mode, prec):
    s = system(name)
    ctx = tddft.Context(s, precision=prec, mode=mode)
    Pp, Pq = sy.random_kernels(s, 3, 4)
    fp, fq = ctx.apply(Pp, Pq)
    rp, rq = oop.Operator(s).apply(Pp, Pq, mode=mode)
    tol = TOL[prec] if mode == "d_only" else TOL_DENSITY[prec]
    assert _err(fp, rp) < (TOL[prec] if mode != "tda" else tol)
    assert _err(fq, rq) < tol


def test_apply_device_pointers(tddft):
    import torch
    s = system("tiny30")
    ctx = tddft.Context(s, precision="fp64")
    Pp, Pq = sy.random_kernels(s, 2, 5)
    hp, hq = ctx.apply(Pp, Pq)
    dp, dq = ctx.apply(torch.from_numpy(Pp).cuda(), torch.from_numpy(Pq).cuda())
    # the integrals accumulate tiles with atomics: equal up to the summation order
    assert _err(dp.cpu().numpy(), hp) < 1e-14 and _err(dq.cpu().numpy(), hq) < 1e-14


def test_apply_is_linear_and_deterministic(tddft):
    s = system("tiny30")
    ctx = tddft.Context(s, precision="fp64")
    Pp, Pq = sy.random_kernels(s, 2, 6)
    a = ctx.apply(Pp, Pq)
    b = ctx.apply(Pp, Pq)
    c2 = ctx.apply(2.0 * Pp, 2.0 * Pq)
    assert _err(b[1], a[1]) < 1e-14          # atomics in the integrals: equal to roundoff
    assert _err(c2[1], 2.0 * a[1]) < 1e-12


def test_invalid_sizes_are_rejected(tddft):
    import dataclasses
    s = system("tiny30")
    bad = dataclasses.replace(s, n=28)       # 28 = 4 * 7 is not 2/3/5-smooth
    with pytest.raises(tddft.TddftError) as e:
        tddft.Context(bad, precision="fp64")
    assert e.value.status == tddft.E_INVALID


@pytest.mark.parametrize("chunk", ["128,16", "384,128"])
def test_integrals_units_of_dense_tiles(tddft, monkeypatch, chunk):
    # "128,16" cuts every tile of the dense system into units of at most 128 chi and 16 phi
    # (up to 2 x 5 units per tile, each adding its part into the output); "384,128" is the
    # default, under which these tiles are whole units
    s = system("dense24")
    monkeypatch.setenv("TDDFT_INTEGRALS_CHUNK", chunk)
    ctx = tddft.Context(s, precision="mixed")
    V = np.random.default_rng(9).standard_normal((3, s.n, s.n, s.n))
    got = ctx.potential_integrals(V)
    ref = ogrid.potential_integrals(ogrid.BoxedSet(s.chi, s.n), ogrid.BoxedSet(s.phi, s.n), V, s.dV)
    assert _err(got, ref) < TOL_DENSITY["mixed"]
    Pp, Pq = sy.random_kernels(s, 2, 8)
    fp, fq = ctx.apply(Pp, Pq)
    rp, rq = oop.Operator(s).apply(Pp, Pq)
    assert _err(fp, rp) < TOL["mixed"] and _err(fq, rq) < TOL_DENSITY["mixed"]
    ctx.close()
