"""Pins of the oracle PCG solver (O2) against dense diagonalisation (O1) and closed forms."""
import dataclasses

import numpy as np
import pytest

from oracle import casida, operator, solver
from paper_1507_08157_gb300 import synthetic as sy


def test_full_spectrum_comes_in_pm_pairs(tiny_casida):
    # Eq. (1): solutions at +omega and -omega; the positive ones equal the symmetric-form roots
    ev = tiny_casida.full_spectrum()
    assert np.max(np.abs(ev.imag)) < 1e-10
    re = np.sort(ev.real)
    m = re.size // 2
    assert np.allclose(-re[:m][::-1], re[m:], atol=1e-10)
    assert np.allclose(re[m:], tiny_casida.omega_symmetric(), atol=1e-10)


def test_d_only_gives_ks_differences(tiny_system, tiny_casida, tiny_operator):
    k = 3
    Y0 = sy.initial_guess(tiny_system, k, 0)
    pcg = solver.PCG(tiny_operator, Y0, mode=operator.D_ONLY)
    om, res, it = pcg.solve(tol=1e-8, max_iter=200)
    ref = np.sort(tiny_casida.ks_differences())[:k]
    assert np.max(np.abs(om - ref)) < 1e-10
    assert np.max(res) <= 1e-8


def test_full_tddft_matches_dense(tiny_system, tiny_casida, tiny_operator):
    k = 3
    Y0 = sy.initial_guess(tiny_system, k, 1)
    pcg = solver.PCG(tiny_operator, Y0)
    om, res, it = pcg.solve(tol=1e-7, max_iter=300)
    ref = tiny_casida.omega_symmetric()[:k]
    assert np.max(np.abs(om - ref)) < 1e-9
    assert np.max(pcg.pairing_errors()) < 1e-6


def test_tda_mode_matches_eig_a(tiny_system, tiny_casida, tiny_operator):
    k = 2
    Y0 = sy.initial_guess(tiny_system, k, 2)
    pcg = solver.PCG(tiny_operator, Y0, mode=operator.TDA)
    om, res, it = pcg.solve(tol=1e-7, max_iter=300)
    assert np.max(np.abs(om - tiny_casida.omega_tda()[:k])) < 1e-9


def test_full_lowest_below_tda(tiny_casida):
    # the Thouless functional at Y = 0 is the TDA Rayleigh quotient (Sec. II B), so omega_1 <= omega_1^TDA
    assert tiny_casida.omega_symmetric()[0] <= tiny_casida.omega_tda()[0] + 1e-14


def test_unpreconditioned_reaches_same_energies(tiny_system, tiny_casida, tiny_operator):
    Y0 = sy.initial_guess(tiny_system, 1, 3)
    pcg = solver.PCG(tiny_operator, Y0, precond="none")
    om, res, it = pcg.solve(tol=1e-7, max_iter=800)
    assert abs(om[0] - tiny_casida.omega_symmetric()[0]) < 1e-9


def test_truncation_is_variational_and_descending(tiny_system, tiny_casida):
    # restricting L to a pattern restricts the trial space (Eq. auxiliary): every iterate's Ritz
    # values stay above the exact ones, and each step lowers the sum functional (Eq. min_multiple)
    s = dataclasses.replace(tiny_system, kernel_cutoff=3.0 / 0.529177210903)
    op = operator.Operator(s)
    assert 0.0 < op.mask.mean() < 1.0
    pcg = solver.PCG(op, sy.initial_guess(s, 2, 4))
    ref = tiny_casida.omega_symmetric()[:2]
    last = np.inf
    for _ in range(40):
        Q, om, gp, gq, res = pcg.evaluate()
        assert np.all(om >= ref - 1e-10)
        total = float(np.sum(om))
        assert total <= last + 1e-12
        last = total
        pcg.update(Q, om, gp, gq)


def test_cutoff_covering_cell_follows_untruncated_path(tiny_system):
    # with r_cut >= sqrt(3) L / 2 the L-gradient route gives the plain preconditioned gradient
    wide = dataclasses.replace(tiny_system, kernel_cutoff=np.sqrt(3.0) / 2.0 * tiny_system.cell + 1e-9)
    Y0 = sy.initial_guess(tiny_system, 2, 6)
    a = solver.PCG(operator.Operator(tiny_system), Y0)
    b = solver.PCG(operator.Operator(wide), Y0)
    for _ in range(6):
        oa, _ = a.step()
        ob, _ = b.step()
        assert np.max(np.abs(oa - ob)) < 1e-10


def test_gradient_is_orthogonal_to_subspace(tiny_system, tiny_operator):
    # Sec. III C: <g_i, x_j>_E = 0 for all j
    Y0 = sy.initial_guess(tiny_system, 3, 5)
    pcg = solver.PCG(tiny_operator, Y0)
    Q, om, gp, gq, res = pcg.evaluate()
    for i in range(3):
        for j in range(3):
            e = pcg.inner(gp[i], pcg.Pp[j]) + pcg.inner(gq[i], pcg.Pq[j])
            assert abs(e) < 1e-10 * (res[i] + 1.0)


def test_line_step_minimises_sum_functional_on_scan():
    # Omega(lambda) = Tr[M(lambda)^-1 N(lambda)] / 2 for x + lambda d; compare with a dense scan
    rng = np.random.default_rng(7)
    m, k = 12, 3
    for trial in range(8):
        B = rng.standard_normal((m, m))
        A = B @ B.T + 0.5 * np.eye(m)
        Vx = np.linalg.qr(rng.standard_normal((m, k)))[0]
        Vd = 0.3 * rng.standard_normal((m, k))
        N0, N2 = Vx.T @ A @ Vx, Vd.T @ A @ Vd
        N1 = Vx.T @ A @ Vd + Vd.T @ A @ Vx
        M0, M1, M2 = Vx.T @ Vx, Vx.T @ Vd + Vd.T @ Vx, Vd.T @ Vd
        lam = solver.line_step(N0, N1, N2, M0, M1, M2)
        f0, d0 = solver.sum_functional(0.0, N0, N1, N2, M0, M1, M2)
        if d0 >= 0:
            assert lam == 0.0
            continue
        # a local minimum: stationary, and no lower value in a neighbourhood of 10% of lambda
        fl, dl = solver.sum_functional(lam, N0, N1, N2, M0, M1, M2)
        assert abs(dl) < 1e-10 * abs(f0)
        assert fl < f0
        near = np.linspace(0.9 * lam, 1.1 * lam, 2001)
        vals = np.array([solver.sum_functional(t, N0, N1, N2, M0, M1, M2)[0] for t in near])
        assert fl <= np.min(vals) + 1e-12 * abs(fl)


def test_sum_functional_derivative_matches_difference():
    rng = np.random.default_rng(9)
    m, k = 10, 2
    B = rng.standard_normal((m, m))
    A = B @ B.T + np.eye(m)
    Vx, Vd = rng.standard_normal((m, k)), rng.standard_normal((m, k))
    args = (Vx.T @ A @ Vx, Vx.T @ A @ Vd + Vd.T @ A @ Vx, Vd.T @ A @ Vd,
            Vx.T @ Vx, Vx.T @ Vd + Vd.T @ Vx, Vd.T @ Vd)
    for t in (0.0, 0.1, 0.7):
        h = 1e-6
        fp = solver.sum_functional(t + h, *args)[0]
        fm = solver.sum_functional(t - h, *args)[0]
        d = solver.sum_functional(t, *args)[1]
        assert abs((fp - fm) / (2 * h) - d) < 1e-6 * max(1.0, abs(d))


def test_gram_schmidt_gives_identity():
    rng = np.random.default_rng(8)
    B = rng.standard_normal((4, 4))
    Mg = B @ B.T + 0.5 * np.eye(4)
    C = solver.gram_schmidt_coefficients(Mg, [2, 0, 3, 1])
    assert np.allclose(C @ Mg @ C.T, np.eye(4), atol=1e-12)
    # lower triangular in the processing order
    order = [2, 0, 3, 1]
    for a, i in enumerate(order):
        for j in order[a + 1:]:
            assert C[i, j] == 0.0


def test_adaptive_inner_tolerance_reaches_dense_eigenvalues(tiny_system, tiny_operator, tiny_casida):
    """Loose-then-tight inner tolerance (suggested in Sec. IV A) changes the path, not the fixed
    point, and spends fewer inner CG iterations than the fixed 1e-4 tolerance."""
    from oracle import solver as osolver
    from paper_1507_08157_gb300 import synthetic as sy
    Y0 = sy.initial_guess(tiny_system, 2, 1)
    fixed = osolver.PCG(tiny_operator, Y0)
    om_f, _, _ = fixed.solve(tol=1e-7, max_iter=400)
    adapt = osolver.PCG(tiny_operator, Y0, precond_adaptive=True)
    om_a, _, _ = adapt.solve(tol=1e-7, max_iter=400)
    ref = tiny_casida.omega_symmetric()[:2]
    assert np.max(np.abs(np.sort(om_a) - ref)) < 1e-6
    assert np.max(np.abs(np.sort(om_f) - ref)) < 1e-6
    assert adapt.inner_iters < fixed.inner_iters


def test_exact_preconditioner_solves_eq_precond(tiny_system, tiny_operator):
    """The exact preconditioner (Kohn-Sham closed form) solves P^c H^chi G - G H^phi P^v = g for
    g in the conduction x valence subspace, and the inner CG converges to it."""
    op = tiny_operator
    rng = np.random.default_rng(21)
    g = op.Pc @ rng.normal(size=(op.Pc.shape[0], op.Pv.shape[0])) @ op.Pv
    ex = solver.PCG(op, sy.initial_guess(tiny_system, 1, 1), precond="exact")
    G = ex.exact_preconditioner(g)
    L = op.Pc @ op.Hc @ G - G @ op.Hv @ op.Pv
    assert np.max(np.abs(L - g)) <= 1e-10 * np.max(np.abs(g))
    it = solver.PCG(op, sy.initial_guess(tiny_system, 1, 1), precond_tol=1e-13, precond_maxit=2000)
    Gi = it.apply_preconditioner(g)
    assert np.max(np.abs(Gi - G)) <= 1e-8 * np.max(np.abs(G))


def test_exact_preconditioner_reaches_dense_eigenvalues(tiny_system, tiny_operator, tiny_casida):
    pcg = solver.PCG(tiny_operator, sy.initial_guess(tiny_system, 2, 1), precond="exact")
    omega, res, it = pcg.solve(tol=1e-8, max_iter=300)
    assert np.max(np.abs(np.sort(omega) - tiny_casida.omega_symmetric()[:2])) < 1e-9
