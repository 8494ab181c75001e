"""The joint unoccupied representation {varphi} = {phi} (+) {chi} (Sec. II C, Eq. proj): test
infrastructure, the plain CPU oracle (only tests, the smoke check and the benchmark's CPU
baseline use it).

Eq. proj defines the conduction projector on the joint functions as the inverse overlap minus
the part of it the occupied space spans:

    P^c = S^-1 - S^-1 S^{varphi phi} P^v S^{phi varphi} S^-1

with S the joint overlap and S^{varphi phi} the overlaps of the joint functions with the phi.
Written out with a dense inverse; pinned in tests/test_oracle_joint.py by the orthonormal
special case (where it reduces to 1 - P^v on the phi block), by idempotency in the S metric, by
orthogonality to the occupied space and by its trace.
"""
import numpy as np
import scipy.linalg


def conduction_projector(S_joint, S_joint_phi, P_v):
    """Eq. proj."""
    X = scipy.linalg.inv(S_joint)
    T = S_joint_phi @ P_v @ S_joint_phi.T
    return X - X @ T @ X
