"""Pins of the truncated (linear-scaling) oracle, oracle/sparse.py, against things other than itself.

* Cutoffs that cover the cell: every mask is all ones and the truncated operator, metric, maps
  and PCG iterates are those of the plain O2 oracle (itself pinned to the dense Casida matrix).
* The patterns: the minimum-image distance against a brute-force minimum over the 27 periodic
  images, and the truncated ground-state kernels against entry-by-entry selection.
* The product semantics: each truncated product equals, entry by entry, the plain sum over the
  inner index kept only where the result's pattern allows it (not the product of truncated
  factors), by explicit loops on a small system.
* The truncation converges: the operator's error against the untruncated one shrinks as the
  cutoffs grow and vanishes once they cover the cell.
"""
import dataclasses
import itertools

import numpy as np
import pytest

from oracle import operator as oop
from oracle import solver as osol
from oracle import sparse as osp
from paper_1507_08157_gb300 import synthetic as sy

B = sy.BOHR_PER_ANG


@pytest.fixture(scope="module")
def four():
    """4 atoms in a 12 A cell (4 phi + 9 chi per atom), some pairs beyond a few A."""
    return sy.generate(sy.Recipe(natoms=4, cell_ang=12.0, ngrid=36, nchi=9, radius_ang=4.0, seed=23))


def _cut(s, r_cut_ang, r_k_ang):
    return dataclasses.replace(s, kernel_cutoff=r_cut_ang * B, density_kernel_cutoff=r_k_ang * B)


def test_distance_against_periodic_images(four):
    d = osp.min_image_distances(four.pos, four.pos, four.cell)
    for i, j in itertools.product(range(four.natoms), repeat=2):
        best = min(np.linalg.norm(four.pos[i] - four.pos[j] + four.cell * np.array(sh))
                   for sh in itertools.product((-1, 0, 1), repeat=3))
        assert abs(d[i, j] - best) < 1e-12


def test_covering_cutoffs_reduce_to_plain_oracle(four):
    big = 0.9 * four.cell * np.sqrt(3.0) / B   # beyond every minimum-image distance
    s = _cut(four, big, big)
    op = osp.TruncatedOperator(s)
    ref = oop.Operator(s)
    assert np.all(op.mask == 1.0)
    Pp, Pq = sy.random_kernels(s, 2, 3)
    for mode in (oop.FULL, oop.TDA, oop.D_ONLY):
        a, b = op.apply(Pp, Pq, mode), ref.apply(Pp, Pq, mode)
        for x, y in zip(a, b):
            assert np.max(np.abs(x - y)) <= 1e-12 * np.max(np.abs(y))
    assert abs(op.inner(Pp[0], Pq[1]) - ref.inner(Pp[0], Pq[1])) <= 1e-12 * abs(ref.inner(Pp[0], Pq[1]))
    for f in ("project", "l_gradient", "ks_difference", "pc_x_pv"):
        x, y = getattr(op, f)(Pp[1]), getattr(ref, f)(Pp[1])
        assert np.max(np.abs(x - y)) <= 1e-12 * np.max(np.abs(y)), f


def test_covering_cutoffs_pcg_steps_equal_plain(four):
    big = 0.9 * four.cell * np.sqrt(3.0) / B
    s = _cut(four, big, big)
    Y0 = sy.initial_guess(s, 2, 4)
    a = osp.TruncatedPCG(osp.TruncatedOperator(s), Y0)
    b = osol.PCG(oop.Operator(s), Y0)
    for _ in range(4):
        (oa, ra), (ob, rb) = a.step(), b.step()
        assert np.max(np.abs(oa - ob)) < 1e-10
        assert np.max(np.abs(ra - rb)) < 1e-8 * max(1.0, np.max(rb))


def test_ground_state_kernels_truncated_by_atom_pairs(four):
    s = _cut(four, 5.0, 4.0)
    op = osp.TruncatedOperator(s)
    nc, nv = s.chi.nfun, s.phi.nfun
    for (P, Pt, fs) in ((s.P_c, op.Pc, s.chi), (s.P_v, op.Pv, s.phi)):
        n = fs.nfun
        for a in range(n):
            for b in range(n):
                i, j = fs.atom[a], fs.atom[b]
                dist = min(np.linalg.norm(s.pos[i] - s.pos[j] + s.cell * np.array(sh))
                           for sh in itertools.product((-1, 0, 1), repeat=3))
                want = P[a, b] if dist <= 4.0 * B else 0.0
                assert Pt[a, b] == want
    assert 0 < op.mask.sum() < nc * nv


def test_truncated_products_entry_by_entry(four):
    # tiny cutoffs so that many entries are truncated; plain triple loops
    s = _cut(four, 5.0, 4.0)
    op = osp.TruncatedOperator(s)
    nc, nv = s.chi.nfun, s.phi.nfun
    rng = np.random.default_rng(8)
    X = op.mask * rng.standard_normal((nc, nv))
    keep = np.zeros((nc, nv), dtype=bool)
    for a in range(nc):
        for b in range(nv):
            i, j = s.chi.atom[a], s.phi.atom[b]
            dist = min(np.linalg.norm(s.pos[i] - s.pos[j] + s.cell * np.array(sh))
                       for sh in itertools.product((-1, 0, 1), repeat=3))
            keep[a, b] = dist <= 5.0 * B

    def tprod(A, Bm):
        out = np.zeros((A.shape[0], Bm.shape[1]))
        for a in range(A.shape[0]):
            for b in range(Bm.shape[1]):
                if keep[a, b]:
                    out[a, b] = sum(A[a, c] * Bm[c, b] for c in range(A.shape[1]))
        return out

    Mc = op.Pc @ s.H_chi
    Mv = s.H_phi @ op.Pv
    want = tprod(Mc, X) - tprod(X, Mv)
    assert np.max(np.abs(op.ks_difference(X) - want)) <= 1e-12 * np.max(np.abs(want))
    cov = tprod(tprod(s.S_chi, X), s.S_phi)
    Y = op.mask * rng.standard_normal((nc, nv))
    assert abs(op.inner(X, Y) - float(np.sum(cov * Y))) <= 1e-12 * abs(float(np.sum(cov * Y)))
    # Eq. auxiliary as two truncated products of the exact constants R_c, R_v
    proj = tprod(tprod(op.Pc @ s.S_chi, X), s.S_phi @ op.Pv)
    assert np.max(np.abs(op.project(X) - proj)) <= 1e-12 * np.max(np.abs(proj))
    # the inner product's result is truncated too: one truncation of the whole chain differs
    once = op.mask * (op.Pc @ s.S_chi @ X @ s.S_phi @ op.Pv)
    assert np.max(np.abs(once - proj)) > 1e-6 * np.max(np.abs(proj))


def test_truncation_error_shrinks_with_cutoff(four):
    Pp, Pq = sy.random_kernels(four, 1, 6)
    big = 0.9 * four.cell * np.sqrt(3.0) / B
    ref = oop.Operator(_cut(four, big, big))
    mask_small = osp.TruncatedOperator(_cut(four, 3.0, 3.0)).mask
    Pp, Pq = mask_small * Pp, mask_small * Pq      # inputs inside every pattern below
    _, fq_ref = ref.apply(Pp, Pq)
    errs = []
    for r in (3.0, 4.0, 6.0, big):    # every atom pair is within 6 A in this cell
        op = osp.TruncatedOperator(_cut(four, r, r))
        _, fq = op.apply(Pp, Pq)
        errs.append(np.max(np.abs(fq - fq_ref)))
    assert max(errs[2:]) <= 1e-12 * np.max(np.abs(fq_ref))
    assert errs[0] > errs[1] > 1e3 * errs[2]


def test_non_descent_preconditioner_falls_back_to_the_gradient(four, monkeypatch):
    # plant a preconditioner that points uphill (G = -g): every step must detect <G_L, z> <= 0
    # and take the search gradient itself, i.e. follow the unpreconditioned PCG step for step
    s = _cut(four, 6.0, 6.0)
    Y0 = sy.initial_guess(s, 2, 6)
    planted = osp.TruncatedPCG(osp.TruncatedOperator(s), Y0, precond="iter")
    monkeypatch.setattr(planted, "apply_preconditioner", lambda g: -g)
    plain = osp.TruncatedPCG(osp.TruncatedOperator(s), Y0, precond="none")
    for _ in range(4):
        (oa, ra), (ob, rb) = planted.step(), plain.step()
        assert np.max(np.abs(oa - ob)) < 1e-12
        assert np.max(np.abs(ra - rb)) < 1e-10 * max(1.0, np.max(rb))
    assert planted.fallbacks == 4 and plain.fallbacks == 0


def test_descending_preconditioner_is_kept(four):
    # the inner CG of a well-posed truncated system descends: no fallback
    s = _cut(four, 6.0, 6.0)
    pcg = osp.TruncatedPCG(osp.TruncatedOperator(s), sy.initial_guess(s, 2, 6), precond="iter")
    for _ in range(4):
        pcg.step()
    assert pcg.fallbacks == 0


def test_l_gradient_is_the_adjoint_of_the_truncated_map(four):
    # <G_L(g), z>_F must equal the slope <g, P(z)> = sum cov(g) * P(z) for every g and every z on
    # the pattern, with P(z) = T(T(R_c z) R_v): the L-gradient is exact for the truncated map
    s = _cut(four, 5.0, 5.0)
    op = osp.TruncatedOperator(s)
    assert 0.0 < op.mask.mean() < 1.0 and op.Pc.astype(bool).sum() < s.P_c.astype(bool).sum()
    rng = np.random.default_rng(3)
    for _ in range(3):
        g = rng.standard_normal(op.mask.shape)
        z = op.mask * rng.standard_normal(op.mask.shape)
        lhs = float(np.sum(op.l_gradient(g) * z))
        rhs = op.inner(g, op.project(z))
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(rhs))
    # the untruncated-style expression T(T(A_c g) A_v) is not that gradient once products are cut
    g = rng.standard_normal(op.mask.shape)
    z = op.mask * rng.standard_normal(op.mask.shape)
    naive = float(np.sum(op.T(op.T(op.Ac @ g) @ op.Av) * z))
    assert abs(naive - op.inner(g, op.project(z))) > 1e-6 * abs(op.inner(g, op.project(z)))
