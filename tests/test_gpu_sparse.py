"""The truncated (linear-scaling) form on the GPU (tddft_create_sparse: cluster-blocked matrices,
block-sparse products on the CUDA cores in FP64 and on the tensor cores in mixed precision)
against the truncated FP64 oracle (oracle/sparse.py), element by element, through the C ABI.

Systems:
* sparse48: 48 atoms (4 phi + 9 chi per atom, so clusters of at most 14 atoms and 128-row
  blocks) in a 22 A cell on a 64^3 grid, 3.5 A functions, kernel and density-kernel cutoffs of 6 A
  (about a tenth of the atom pairs kept): several clusters, block pairs that are skipped, output
  blocks without any pair, atom pairs cut inside present blocks;
* tiny: 3 atoms with cutoffs covering the cell, where the truncated form is the plain one and
  the sparse context must equal the dense context.

Tolerances as in the dense operator tests: FP64 1e-10 of the largest entry; mixed 3e-5 for
products on the split-TF32 tensor cores, 2e-3 once the float16 grid contractions enter.
"""
import dataclasses

import numpy as np
import pytest

from oracle import operator as oop
from oracle import sparse as osp
from paper_1507_08157_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

B = sy.BOHR_PER_ANG
TOL = {"fp64": 1e-10, "mixed": 3e-5}
TOL_GRID = {"fp64": 1e-10, "mixed": 2e-3}


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
def sparse48():
    rec = sy.Recipe(natoms=48, cell_ang=22.0, ngrid=64, nchi=9, radius_ang=3.5, kernel_cutoff_ang=6.0,
                    density_kernel_cutoff_ang=6.0, seed=41)
    s = sy.generate(rec)
    return s, osp.TruncatedOperator(s)


@pytest.fixture(scope="module")
def tiny():
    s = sy.generate(sy.Recipe(natoms=3, cell_ang=10.0, ngrid=30, radius_ang=4.0, seed=11))
    big = s.cell * np.sqrt(3.0)
    return dataclasses.replace(s, kernel_cutoff=big, density_kernel_cutoff=big)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_pattern_is_the_oracle_mask(tddft, sparse48):
    s, op = sparse48
    ctx = tddft.Context(s, sparse=True, precision="fp64", precond="none")
    dense = ctx.from_pattern(np.ones((1, ctx.nnz)))[0]
    assert np.array_equal(dense, op.mask)
    assert ctx.nnz == int(op.mask.sum())
    mask = ctx.pattern()
    d = osp.min_image_distances(s.pos, s.pos, s.cell)
    assert np.array_equal(mask.astype(bool), d <= s.kernel_cutoff)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("mode", ["full", "tda", "d_only"])
def test_apply_matches_truncated_oracle(tddft, sparse48, prec, mode):
    s, op = sparse48
    ctx = tddft.Context(s, sparse=True, precision=prec, mode=mode, precond="none")
    Pp, Pq = sy.random_kernels(s, 3, 7)
    Pp, Pq = op.mask * Pp, op.mask * Pq
    fp, fq = ctx.apply(ctx.to_pattern(Pp), ctx.to_pattern(Pq))
    rp, rq = op.apply(Pp, Pq, mode)
    tol = TOL[prec] if mode == "d_only" else TOL_GRID[prec]
    for got, ref in ((fp, rp), (fq, rq)):
        for q in range(3):
            assert _rel(ctx.from_pattern(got[q:q + 1])[0], ref[q]) <= tol, (mode, q)


def test_entries_off_the_pattern_are_ignored(tddft, sparse48):
    # the boundary carries only the pattern's values: a dense input's other entries never enter
    s, op = sparse48
    ctx = tddft.Context(s, sparse=True, precision="fp64", mode="d_only", precond="none")
    Pp, Pq = sy.random_kernels(s, 1, 8)
    fp, _ = ctx.apply(ctx.to_pattern(Pp), ctx.to_pattern(Pq))
    rp, _ = op.apply(op.mask * Pp, op.mask * Pq, oop.D_ONLY)
    assert _rel(ctx.from_pattern(fp)[0], rp[0]) <= TOL["fp64"]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_components_match_oracle(tddft, sparse48, prec):
    s, op = sparse48
    ctx = tddft.Context(s, sparse=True, precision=prec, precond="none")
    _, Pq = sy.random_kernels(s, 2, 9)
    Pq = op.mask * Pq
    rho = ctx.response_density(ctx.to_pattern(Pq))
    rref = op.response_density(Pq)
    for q in range(2):
        assert _rel(rho[q], rref[q]) <= TOL_GRID[prec]
    V = op.response_potential(rref)
    out = ctx.potential_integrals(V)
    vref = op.T(oop.grid.potential_integrals(op.chi, op.phi, V, s.dV))
    for q in range(2):
        assert _rel(ctx.from_pattern(out[q:q + 1])[0], vref[q]) <= TOL_GRID[prec]


def test_covering_cutoffs_equal_dense_context(tddft, tiny):
    sp = tddft.Context(tiny, sparse=True, precision="fp64", precond="none")
    de = tddft.Context(tiny, precision="fp64", precond="none")
    Pp, Pq = sy.random_kernels(tiny, 2, 5)
    fp, fq = sp.apply(sp.to_pattern(Pp), sp.to_pattern(Pq))
    gp, gq = de.apply(Pp, Pq)
    assert sp.nnz == tiny.chi.nfun * tiny.phi.nfun
    assert _rel(sp.from_pattern(fp), gp) <= 1e-12
    assert _rel(sp.from_pattern(fq), gq) <= 1e-12


@pytest.mark.parametrize("precond", ["iter", "none"])
def test_pcg_steps_match_truncated_oracle_fp64(tddft, sparse48, precond):
    s, op = sparse48
    k = 2
    Y0 = sy.initial_guess(s, k, 11)
    ctx = tddft.Context(s, sparse=True, precision="fp64", precond=precond)
    st = ctx.state(ctx.to_pattern(Y0))
    ref = osp.TruncatedPCG(op, Y0, precond=precond)
    g = st.get()
    assert _rel(ctx.from_pattern(g["Pp"]), ref.Pp) <= 1e-8
    for _ in range(3):
        om, res = st.step()
        om_r, res_r = ref.step()
        assert np.max(np.abs(om - om_r)) <= 1e-9
        assert np.max(np.abs(res - res_r)) <= 1e-7 * max(1.0, float(np.max(res_r)))
    g = st.get()
    assert _rel(ctx.from_pattern(g["Pq"]), ref.Pq) <= 1e-7
    assert _rel(ctx.from_pattern(g["fq"]), ref.fq) <= 1e-7


def test_pcg_steps_mixed_follow_oracle(tddft, sparse48):
    s, op = sparse48
    k = 2
    Y0 = sy.initial_guess(s, k, 12)
    ctx = tddft.Context(s, sparse=True, precision="mixed", precond="iter")
    st = ctx.state(ctx.to_pattern(Y0))
    ref = osp.TruncatedPCG(op, Y0, precond="iter")
    for _ in range(3):
        om, _ = st.step()
        om_r, _ = ref.step()
        assert np.max(np.abs(om - om_r)) <= 1e-4 * max(1.0, float(np.max(np.abs(om_r))))


def test_sparse_context_refuses_other_preconditioners(tddft, sparse48):
    s, _ = sparse48
    for pre in ("exact", "learned"):
        with pytest.raises(tddft.TddftError) as e:
            tddft.Context(s, sparse=True, precision="fp64", precond=pre)
        assert e.value.status == tddft.E_INVALID
    with pytest.raises(tddft.TddftError) as e:
        tddft.Context(dataclasses.replace(s, kernel_cutoff=0.0), sparse=True, precision="fp64", precond="none")
    assert e.value.status == tddft.E_INVALID


def _atom_pattern(M, row_atom, col_atom, natoms):
    """Atom pairs whose block of M holds a nonzero entry."""
    pat = np.zeros((natoms, natoms), dtype=np.int64)
    I, J = np.nonzero(M)
    pat[row_atom[I], col_atom[J]] = 1
    return pat


def test_profiled_product_work_is_the_atom_triple_count(tddft, sparse48):
    # The library's profiler counts the block products' work as 2 n_I n_K n_J over the atom
    # triples (I, K, J) that contribute to an output pair (I, J) of the kernel pattern: written out
    # here by brute force from the atom patterns of the inputs and of M_c = P^c H^chi,
    # M_v = H^phi P^v (Sec. IV truncation of P at the density-kernel cutoff).
    s, op = sparse48
    na = s.natoms
    ca, pa = s.chi.atom, s.phi.atom
    nchi = np.bincount(ca, minlength=na)
    nphi = np.bincount(pa, minlength=na)
    pk = (_atom_pattern(op.mask, ca, pa, na) > 0).astype(np.int64)
    Pc = _atom_pattern(op.Pc, ca, ca, na)
    Hc = _atom_pattern(s.H_chi, ca, ca, na)
    Pv = _atom_pattern(op.Pv, pa, pa, na)
    Hv = _atom_pattern(s.H_phi, pa, pa, na)
    Mc = ((Pc @ Hc) > 0).astype(np.int64)
    Mv = ((Hv @ Pv) > 0).astype(np.int64)
    left = 2 * np.sum(pk * np.outer(nchi, nphi) * (Mc @ (nchi[:, None] * pk)))
    right = 2 * np.sum(pk * np.outer(nchi, nphi) * ((pk * nphi[None, :]) @ Mv))
    k = 2
    ctx = tddft.Context(s, sparse=True, precision="fp64", mode="d_only", precond="none")
    Pp, Pq = sy.random_kernels(s, k, 4)
    dp, dq = ctx.to_pattern(op.mask * Pp), ctx.to_pattern(op.mask * Pq)
    ctx.profile(True)
    ctx.apply(dp, dq)
    prof = ctx.profile_read()
    ctx.profile(False)
    launches, _, flops, _ = prof["gemm"]
    assert launches == 2
    assert flops == pytest.approx(2 * k * float(left + right), rel=1e-12)


def test_pcg_eight_steps_follow_oracle_with_4a_cutoffs(tddft):
    # 12 atoms with 4 A cutoffs (about half of the atom pairs cut): eight FP64 steps of the
    # inner-CG PCG on the GPU equal the truncated oracle's, with the exact L-gradient of the
    # truncated map, and the two agree on every fallback decision (none on this system)
    s = sy.generate(sy.Recipe(natoms=12, cell_ang=14.0, ngrid=40, nchi=9, radius_ang=3.5, kernel_cutoff_ang=4.0,
                              density_kernel_cutoff_ang=4.0, seed=41))
    k = 2
    Y0 = sy.initial_guess(s, k, 1)
    ctx = tddft.Context(s, sparse=True, precision="fp64", precond="iter")
    st = ctx.state(ctx.to_pattern(Y0))
    ref = osp.TruncatedPCG(osp.TruncatedOperator(s), Y0, precond="iter")
    for _ in range(8):
        om, res = st.step()
        om_r, res_r = ref.step()
        assert np.max(np.abs(om - om_r)) <= 1e-8
        assert np.max(np.abs(res - res_r)) <= 1e-6 * max(1.0, float(np.max(res_r)))
    assert st.stats()[1] == ref.fallbacks
