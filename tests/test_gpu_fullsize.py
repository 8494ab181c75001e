"""The chromophore-140 workload at full size (140 atoms, 120^3 grid, 4 phi + 9 chi per atom, 8 A
radius, 12 A kernel cutoff, k = 10 states), in the launch configuration the benchmark times
(mixed precision: tensor-core response density and integrals, TF32 products), checked against
the FP64 oracle:

* response density at 400 sampled grid points (40 per state), the oracle evaluating the
  definition point by point (oracle/grid.py: density_at);
* potential integrals at 300 (chi, phi) pairs drawn uniformly, over a smooth potential, the
  oracle summing each pair over the two functions' common box (integrals_at);
* the Hartree + f_xc potential of the GPU's own density on the whole grid (numpy FFT);
* the Kohn-Sham difference part of the operator (mode d_only: P^c H^chi P - P H^phi P^v) on
  every entry.

Tolerances as in the small-system operator tests, relative to the largest entry of the state:
2e-3 for the float16 grid contractions, 3e-5 for the float32 FFT and the split-TF32 products.
"""
import numpy as np
import pytest

from oracle import grid as ogrid
from oracle import operator as ooperator
from oracle import hartree as ohartree
from oracle import xc as oxc
from paper_1507_08157_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

K = 10


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
def chromo():
    s = sy.generate(sy.CONFIG_CHROMOPHORE)
    return s, ogrid.BoxedSet(s.chi, s.n), ogrid.BoxedSet(s.phi, s.n)


@pytest.fixture(scope="module")
def ctx(tddft, chromo):
    return tddft.Context(chromo[0], precision="mixed", precond="exact")


def _kernels(s):
    _, Pq = sy.random_kernels(s, K, 41)
    return Pq


def test_density_sampled(ctx, chromo):
    s, chi, phi = chromo
    P = _kernels(s)
    rho = ctx.response_density(P)
    rng = np.random.default_rng(42)
    for q in range(K):
        pts = [tuple(int(v) for v in rng.integers(0, s.n, size=3)) for _ in range(40)]
        ref = ogrid.density_at(chi, phi, P[q:q + 1], pts)[0]
        got = np.array([rho[q][p] for p in pts])
        scale = np.max(np.abs(rho[q]))
        assert np.max(np.abs(got - ref)) <= 2e-3 * scale, q


def _smooth_potential(s, q):
    x = np.arange(s.n) * (2.0 * np.pi / s.n)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    return (np.cos(X + 0.3 * q) + 0.5 * np.sin(2.0 * Y - 0.1 * q) + 0.25 * np.cos(3.0 * Z + X)
            + 0.1 * q)


def test_integrals_sampled(ctx, chromo):
    s, chi, phi = chromo
    V = np.stack([_smooth_potential(s, q) for q in range(K)])
    out = ctx.potential_integrals(V)
    rng = np.random.default_rng(43)
    for q in range(K):
        # uniform over all pairs: an entry the kernel wrongly leaves at zero is caught as well
        pairs = [(int(rng.integers(s.chi.nfun)), int(rng.integers(s.phi.nfun))) for _ in range(30)]
        ref = ogrid.integrals_at(chi, phi, V[q:q + 1], s.dV, pairs)[0]
        got = np.array([out[q][a, b] for a, b in pairs])
        assert np.max(np.abs(got - ref)) <= 2e-3 * np.max(np.abs(out[q])), q


def test_potential_full_grid(ctx, chromo):
    s = chromo[0]
    rho = ctx.response_density(_kernels(s)[:4])
    got = ctx.response_potential(rho)
    ref = ohartree.hartree(rho, s.cell) + oxc.fxc_lda(s.n0)[None] * rho
    for q in range(4):
        assert np.max(np.abs(got[q] - ref[q])) <= 3e-5 * np.max(np.abs(ref[q])), q


def test_ks_difference_every_entry(tddft, chromo):
    s = chromo[0]
    ctx_d = tddft.Context(s, precision="mixed", mode="d_only")
    Pp, Pq = sy.random_kernels(s, 4, 44)
    fp, fq = ctx_d.apply(Pp, Pq)
    rp, rq = ooperator.Operator(s).apply(Pp, Pq, mode=ooperator.D_ONLY)
    for f, ref in ((fp, rp), (fq, rq)):
        for q in range(f.shape[0]):
            assert np.max(np.abs(f[q] - ref[q])) <= 3e-5 * np.max(np.abs(ref[q])), q
