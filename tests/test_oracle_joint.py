"""Pins of the joint-representation oracle (oracle/joint.py, Eq. proj) and of the dense
reference in that representation (oracle/casida.py, conduction="projector"):

* orthonormal special case: with S = 1 and the phi the first block of the joint set, Eq. proj
  reduces to P^c = 1 - diag(P^v, 0);
* on a generated joint system: P^c S P^c = P^c, P^c S^{varphi phi} P^v = 0 and tr(P^c S) =
  N_joint - N_occ (the whole unoccupied space of the joint functions);
* the projector route of the dense reference equals the spectral route when P^c is the spectral
  projector of H^chi (the existing systems);
* the joint system has real excitation energies, and the paper's PCG (O2) run in the joint
  representation reaches its dense eigenvalues.
"""
import numpy as np
import pytest

from oracle import casida, joint
from paper_1507_08157_gb300 import synthetic as sy


def test_orthonormal_special_case():
    rng = np.random.default_rng(1)
    nv, nj = 5, 12
    C = np.linalg.qr(rng.normal(size=(nv, nv)))[0][:, :2]
    Pv = C @ C.T                                         # projector, S^phi = 1
    S = np.eye(nj)
    Sjp = np.zeros((nj, nv))
    Sjp[:nv, :nv] = np.eye(nv)
    Pc = joint.conduction_projector(S, Sjp, Pv)
    ref = np.eye(nj)
    ref[:nv, :nv] -= Pv
    assert np.allclose(Pc, ref, atol=1e-14)


@pytest.fixture(scope="module")
def tiny_joint(tiny_system):
    ji = sy.joint_inputs(tiny_system, seed=5)
    Pc = joint.conduction_projector(ji.S_joint, ji.S_joint_phi, tiny_system.P_v)
    return ji, Pc, sy.with_joint(tiny_system, ji, Pc)


def test_joint_projector_properties(tiny_system, tiny_joint):
    ji, Pc, s = tiny_joint
    S = ji.S_joint
    assert np.max(np.abs(Pc @ S @ Pc - Pc)) <= 1e-9 * np.max(np.abs(Pc))
    assert np.max(np.abs(Pc @ ji.S_joint_phi @ tiny_system.P_v)) <= 1e-9 * np.max(np.abs(Pc))
    nj = S.shape[0]
    assert abs(np.trace(Pc @ S) - (nj - tiny_system.n_occ)) < 1e-8
    assert s.n_cond == nj - tiny_system.n_occ


def test_projector_route_equals_spectral_route(tiny_system):
    a = casida.Casida(tiny_system)
    b = casida.Casida(tiny_system, conduction="projector")
    assert np.allclose(a.eps_c, b.eps_c, atol=1e-12)
    assert np.allclose(a.omega_symmetric(), b.omega_symmetric(), atol=1e-12)


def test_joint_energies_real(tiny_joint):
    _, _, s = tiny_joint
    cj = casida.Casida(s, conduction="projector")
    assert np.min(cj.ks_differences()) > 0.0
    om = cj.omega_symmetric()                           # raises if A+B or A-B is indefinite
    assert np.all(np.isfinite(om)) and om[0] > 0.0


@pytest.mark.slow
def test_pcg_in_joint_representation_reaches_dense(tiny_joint):
    """The paper's algorithm (operator and PCG, O2) run with chi := the joint functions and the
    P^c of Eq. proj reaches the dense eigenvalues of that representation."""
    from oracle import operator, solver
    _, _, s = tiny_joint
    ref = casida.Casida(s, conduction="projector").omega_symmetric()[:2]
    pcg = solver.PCG(operator.Operator(s), sy.initial_guess(s, 2, 3))
    om, res, it = pcg.solve(tol=1e-8, max_iter=400)
    assert np.max(np.abs(np.sort(om) - ref)) < 1e-8
