"""Pins of the chi/phi-space operator (O2) against the dense Kohn-Sham-space definition (O1) and
the structural facts of Secs. II and III."""
import numpy as np
import pytest

from oracle import casida, operator
from paper_1507_08157_gb300 import synthetic as sy


def _ks_vectors(cas, k, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((k, cas.nc, cas.nv))


def test_operator_equals_casida_action(tiny_system, tiny_casida, tiny_operator):
    # For P = D_c X C_v^T: f_p = D_c (D X) C_v^T and f_q = D_c ((D + 2K) X) C_v^T (Eqs. 2-3 with
    # A - B = D, A + B = D + 2K; Eq. operator_RPA)
    cas, op = tiny_casida, tiny_operator
    A, B, d, K = cas.matrices()
    X = _ks_vectors(cas, 2, 0)
    Y = _ks_vectors(cas, 2, 1)
    Pp = np.array([cas.to_ngwf(x) for x in X])
    Pq = np.array([cas.to_ngwf(y) for y in Y])
    fp, fq = op.apply(Pp, Pq)
    for s in range(2):
        refp = cas.to_ngwf((d * X[s].ravel()).reshape(X[s].shape))
        refq = cas.to_ngwf(((A + B) @ Y[s].ravel()).reshape(Y[s].shape))
        assert np.max(np.abs(fp[s] - refp)) < 1e-10 * np.max(np.abs(refp))
        assert np.max(np.abs(fq[s] - refq)) < 1e-10 * np.max(np.abs(refq))


def test_tda_mode_is_a_on_both_blocks(tiny_casida, tiny_operator):
    cas, op = tiny_casida, tiny_operator
    A, _, _, _ = cas.matrices()
    X = _ks_vectors(cas, 1, 2)
    P = np.array([cas.to_ngwf(X[0])])
    fp, fq = op.apply(P, P, mode=operator.TDA)
    ref = cas.to_ngwf((A @ X[0].ravel()).reshape(X[0].shape))
    assert np.allclose(fp[0], ref, atol=1e-10 * np.max(np.abs(ref)))
    assert np.allclose(fq[0], ref, atol=1e-10 * np.max(np.abs(ref)))


def test_ks_maps_are_inverse_and_isometric(tiny_casida, tiny_operator):
    # <X, Y> = Tr[X^T S^chi Y S^phi] is the Euclidean product of the KS-space vectors
    cas, op = tiny_casida, tiny_operator
    X, Y = _ks_vectors(cas, 2, 3)
    Px, Py = cas.to_ngwf(X), cas.to_ngwf(Y)
    assert np.allclose(cas.to_ks(Px), X, atol=1e-10)
    assert abs(op.inner(Px, Py) - np.sum(X * Y)) < 1e-10 * np.sqrt(np.sum(X * X) * np.sum(Y * Y))


def test_adjointness_and_invariance(tiny_system, tiny_operator):
    # A - B and A + B are symmetric (Sec. II B), and f keeps the invariance constraint
    # P^c S^chi f S^phi P^v = f (Eq. invariance) for invariant inputs.
    op = tiny_operator
    rng = np.random.default_rng(4)
    X = np.array([op.project(rng.standard_normal(op.mask.shape)) for _ in range(2)])
    Y = np.array([op.project(rng.standard_normal(op.mask.shape)) for _ in range(2)])
    fX = op.apply(X, X)
    fY = op.apply(Y, Y)
    for blk in (0, 1):
        lhs = op.inner(X[0], fY[blk][0])
        rhs = op.inner(fX[blk][0], Y[0])
        assert abs(lhs - rhs) < 1e-10 * abs(lhs)
        f = fX[blk][1]
        assert np.allclose(op.project(f), f, atol=1e-10 * np.max(np.abs(f)))


def test_hartree_only_coupling_is_positive(tiny_system):
    cas = casida.Casida(tiny_system, fxc_kind="none")
    _, _, _, K = cas.matrices()
    assert np.min(np.linalg.eigvalsh(K)) > -1e-12


def test_cutoff_covering_cell_changes_nothing(tiny_system):
    import dataclasses
    s = tiny_system
    wide = dataclasses.replace(s, kernel_cutoff=np.sqrt(3.0) / 2.0 * s.cell + 1e-9)
    op_w = operator.Operator(wide)
    op_n = operator.Operator(s)
    rng = np.random.default_rng(6)
    L = rng.standard_normal(op_n.mask.shape)
    assert np.all(op_w.mask == 1.0)
    assert np.array_equal(op_w.project(L), op_n.project(L))


def test_mask_is_atom_pair_distance(tiny_system):
    import dataclasses
    s = dataclasses.replace(tiny_system, kernel_cutoff=4.0 / 0.529177210903)
    m = operator.kernel_mask(s)
    for a in range(s.chi.nfun):
        for b in range(s.phi.nfun):
            d = s.pos[s.chi.atom[a]] - s.pos[s.phi.atom[b]]
            d -= s.cell * np.round(d / s.cell)
            assert m[a, b] == (1.0 if np.linalg.norm(d) <= s.kernel_cutoff else 0.0)
