"""Config 2's accuracy statement: the lowest 10 excitations of chromophore-140 (140 atoms, 30 A
cell, 120^3 grid, 4 phi + 9 chi per atom, 8 A radius) converged on the GPU to a 1e-5 Ha residual
in mixed precision (float32 / float16 grid work on the tensor cores, float64 traces and small
algebra) and in FP64 mode agree to 1e-5 Ha. The response kernels are not truncated here (the
benchmark's 12 A cutoff changes the eigenproblem; its own convergence is reported by the bench).

How the oracle pins this size: the FP64 oracle cannot iterate a 140-atom system (minutes per
operator application), so the pins are (1) the operator in the launch configuration of the
benchmark against the oracle, element by element and at sampled points (test_gpu_fullsize.py),
(2) the converged energies of the same code against the dense oracle on the parity systems
(test_gpu_solver.py), and (3) here, the FP64 GPU mode as the reference of the mixed mode and the
pairing check of the converged Ritz pairs (each half of the Tsiper numerator equals omega).

The FP64 solve starts from the mixed solution's q vectors, which shortens it.
"""
import dataclasses

import numpy as np
import pytest

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
    return dataclasses.replace(s, kernel_cutoff=0.0)


def test_lowest_ten_mixed_against_fp64(tddft, chromo):
    s = chromo
    Y0 = sy.initial_guess(s, K, 0)
    cm = tddft.Context(s, precision="mixed", precond="exact", tol=1e-5, max_iter=400)
    sm = cm.state(Y0)
    om_m, res_m, it_m, rc_m = sm.solve()
    assert rc_m == tddft.OK, (rc_m, it_m, res_m)
    assert np.max(res_m) <= 1e-5
    q = sm.get()["Pq"]
    sm.close()
    cm.close()
    cf = tddft.Context(s, precision="fp64", precond="exact", tol=1e-5, max_iter=400)
    sf = cf.state(q)
    om_f, res_f, it_f, rc_f = sf.solve()
    assert rc_f == tddft.OK, (rc_f, it_f, res_f)
    assert np.max(res_f) <= 1e-5
    assert np.max(np.abs(om_m - om_f)) <= 1e-5, (om_m, om_f)
    # the lowest excitation lies at the synthetic gap (2 eV = 0.0735 Ha) or above it
    assert om_f[0] > 0.07 and np.all(np.diff(om_f) >= -1e-12)
    print("mixed %d iterations, fp64 %d; omega (Ha) %s" % (it_m, it_f, np.array2string(om_f, precision=8)))
