"""The first member of the linear-scaling series in the launch configuration `bench.py --scaling`
times: 500 atoms (a 140-atom core and a shell at 0.1 atoms per A^3, 48 A cell, 192^3 grid, 4 phi +
9 chi per atom, 8 A radius, every density matrix truncated at 15 A), k = 4 states, mixed precision,
the truncated form of Sec. IV (tddft_create_sparse: cluster-blocked matrices, block-sparse
products on the tensor cores). At this atom density a grid tile holds more functions than the
per-tile tensor-core density kernels take (256 phi), so both the density and the integrals cut
such tiles into tensor-core units (float16 operands). Checked against the FP64
oracle (oracle/sparse.py for the truncated products, oracle/grid.py point by point):

* the Kohn-Sham difference part (mode d_only: T(M_c P) - T(P M_v)) on every entry of the
  kernel pattern;
* the response density at 160 sampled grid points (density_at), on the tensor-core units of
  dense tiles (float16 operands);
* the potential integrals at 160 (chi, phi) pairs of the pattern over a smooth potential
  (integrals_at), cut to the pattern.

Tolerances, relative to the largest entry of each state: 1e-4 for the split-TF32 block products
with K up to N_chi = 4500; 2e-3 for the density and the integrals on float16 tensor-core operands
(as in the small-system tests).
"""
import numpy as np
import pytest

from oracle import grid as ogrid
from oracle import operator as ooperator
from oracle import sparse as osp
from paper_1507_08157_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

K = 4
TOL = 1e-4
TOL_F16 = 2e-3


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
def shell500():
    s = sy.generate(sy.scaling_recipe(500))
    return s, ogrid.BoxedSet(s.chi, s.n), ogrid.BoxedSet(s.phi, s.n)


@pytest.fixture(scope="module")
def ctx(tddft, shell500):
    return tddft.Context(shell500[0], precision="mixed", precond="none", sparse=True)


def _kernels(ctx, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((K, ctx.nnz))


def test_density_sampled(ctx, shell500):
    s, chi, phi = shell500
    x = _kernels(ctx, 51)
    rho = ctx.response_density(x)
    P = ctx.from_pattern(x)
    rng = np.random.default_rng(52)
    centre = s.n // 2
    for q in range(K):
        # half the points inside the cluster, half anywhere
        pts = [tuple(int(v) for v in centre + rng.integers(-s.n // 5, s.n // 5, size=3)) for _ in range(20)]
        pts += [tuple(int(v) for v in rng.integers(0, s.n, size=3)) for _ in range(20)]
        ref = ogrid.density_at(chi, phi, P[q:q + 1], pts)[0]
        got = np.array([rho[q][p] for p in pts])
        assert np.max(np.abs(got - ref)) <= TOL_F16 * np.max(np.abs(rho[q])), q


def test_integrals_sampled(ctx, shell500):
    s, chi, phi = shell500
    x = np.arange(s.n) * (2.0 * np.pi / s.n)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    V = np.stack([np.cos(X + 0.3 * q) + 0.5 * np.sin(2.0 * Y - 0.1 * q) + 0.25 * np.cos(3.0 * Z + X)
                  for q in range(K)])
    out = ctx.from_pattern(ctx.potential_integrals(V))
    rng = np.random.default_rng(53)
    rows, cols = ctx.kp_rows, ctx.kp_cols
    for q in range(K):
        pick = rng.integers(0, rows.size, size=40)
        pairs = [(int(rows[i]), int(cols[i])) for i in pick]
        ref = ogrid.integrals_at(chi, phi, V[q:q + 1], s.dV, pairs)[0]
        got = np.array([out[q][a, b] for a, b in pairs])
        assert np.max(np.abs(got - ref)) <= TOL_F16 * np.max(np.abs(out[q])), q


def test_ks_difference_every_entry(tddft, shell500):
    s = shell500[0]
    ctx_d = tddft.Context(s, precision="mixed", mode="d_only", precond="none", sparse=True)
    op = osp.TruncatedOperator(s)
    xp, xq = _kernels(ctx_d, 54)[:2], _kernels(ctx_d, 55)[:2]
    fp, fq = ctx_d.apply(xp, xq)
    rp, rq = op.apply(ctx_d.from_pattern(xp), ctx_d.from_pattern(xq), mode=ooperator.D_ONLY)
    for f, ref in ((fp, rp), (fq, rq)):
        for q in range(f.shape[0]):
            got = ctx_d.from_pattern(f[q:q + 1])[0]
            assert np.max(np.abs(got - ref[q])) <= TOL * np.max(np.abs(ref[q])), q
    ctx_d.close()
