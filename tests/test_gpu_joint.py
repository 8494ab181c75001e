"""The joint unoccupied representation {varphi} = {phi} (+) {chi} on the GPU (Sec. II C, Eq. proj):

* tddft_joint_projector against the oracle's Eq. proj, element by element (float64, 1e-10 of
  the largest entry);
* a context with chi := the joint functions and the device-made P^c solves to the dense
  eigenvalues of that representation (the oracle's P^c and projector-route Casida): 1e-6 Ha in
  FP64, 1e-5 Ha in mixed precision.
"""
import numpy as np
import pytest

from oracle import casida, joint
from paper_1507_08157_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu


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
def tiny():
    return sy.generate(sy.Recipe(natoms=3, cell_ang=10.0, ngrid=30, radius_ang=4.0, seed=11))


@pytest.fixture(scope="module")
def joint_case(tiny):
    ji = sy.joint_inputs(tiny, seed=5)
    Pc_ref = joint.conduction_projector(ji.S_joint, ji.S_joint_phi, tiny.P_v)
    dense = casida.Casida(sy.with_joint(tiny, ji, Pc_ref), conduction="projector").omega_symmetric()
    return ji, Pc_ref, dense


def test_joint_projector_matches_oracle(tddft, tiny, joint_case):
    ji, Pc_ref, _ = joint_case
    Pc = tddft.joint_projector(ji.S_joint, ji.S_joint_phi, tiny.P_v)
    assert np.max(np.abs(Pc - Pc_ref)) <= 1e-10 * np.max(np.abs(Pc_ref))


@pytest.mark.parametrize("prec,tol,acc", [("fp64", 1e-8, 1e-6), ("mixed", 1e-5, 1e-5)])
def test_joint_representation_solve(tddft, tiny, joint_case, prec, tol, acc):
    ji, _, dense = joint_case
    Pc = tddft.joint_projector(ji.S_joint, ji.S_joint_phi, tiny.P_v)
    s = sy.with_joint(tiny, ji, Pc)
    k = 3
    ctx = tddft.Context(s, precision=prec, tol=tol, max_iter=400)
    om, res, it, rc = ctx.state(sy.initial_guess(s, k, 2)).solve()
    assert rc == tddft.OK, (rc, it, res)
    assert np.max(np.abs(om - dense[:k])) <= acc
