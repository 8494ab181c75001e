import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built library")
    config.addinivalue_line("markers", "slow: larger CPU oracle cases")


@pytest.fixture(scope="session")
def tiny_system():
    """3 atoms, 10 A cell, 30^3 grid (tiles of 8 leave a ragged tail), 4 phi + 4 chi per atom."""
    from paper_1507_08157_gb300 import synthetic as sy
    return sy.generate(sy.Recipe(natoms=3, cell_ang=10.0, ngrid=30, radius_ang=4.0, seed=11))


@pytest.fixture(scope="session")
def tiny_system_d():
    """3 atoms with 9 chi (s, p, d) per atom on a 30^3 grid."""
    from paper_1507_08157_gb300 import synthetic as sy
    return sy.generate(sy.Recipe(natoms=3, cell_ang=10.0, ngrid=30, nchi=9, radius_ang=4.0, seed=12))


@pytest.fixture(scope="session")
def tiny_casida(tiny_system):
    from oracle import casida
    return casida.Casida(tiny_system)


@pytest.fixture(scope="session")
def tiny_operator(tiny_system):
    from oracle import operator
    return operator.Operator(tiny_system)
