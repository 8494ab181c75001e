"""A batch of uneven systems through the C ABI (tddft_create_batch / tddft_solve_batch).

Several seeded systems of different atom counts, cells, grids and state counts are set up in one
call (each context on a stream of its own) and solved concurrently by host threads. Each
system's converged omega must equal the dense eigenvalues (the plain definition) to 1e-6 Ha in
FP64 and 1e-5 Ha in mixed precision, and agree with the same system solved alone to 1e-9 Ha
(FP64); bad arguments are refused before any work.
"""
import numpy as np
import pytest

from oracle import casida
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


RECIPES = [sy.Recipe(natoms=2, cell_ang=10.0, ngrid=30, radius_ang=4.0, seed=31),
           sy.Recipe(natoms=3, cell_ang=10.0, ngrid=30, radius_ang=4.0, seed=32),
           sy.Recipe(natoms=4, cell_ang=11.0, ngrid=32, radius_ang=4.0, seed=33),
           sy.Recipe(natoms=3, cell_ang=11.0, ngrid=36, radius_ang=4.5, seed=34)]
KS = [1, 2, 3, 2]


@pytest.fixture(scope="module")
def systems():
    return [sy.generate(r) for r in RECIPES]


@pytest.fixture(scope="module")
def dense(systems):
    return [casida.Casida(s).omega_symmetric() for s in systems]


# mixed precision converges to the method's 1e-5 Ha residual and stays within 1e-5 Ha of the
# dense eigenvalues
@pytest.mark.parametrize("prec,tol,acc", [("fp64", 1e-8, 1e-6), ("mixed", 1e-5, 1e-5)])
def test_batch_reaches_the_dense_eigenvalues(tddft, systems, dense, prec, tol, acc):
    ctxs = tddft.create_batch(systems, precision=prec, tol=tol, max_iter=400)
    states = [c.state(sy.initial_guess(s, k, 5 + i)) for i, (c, s, k) in enumerate(zip(ctxs, systems, KS))]
    res, iters, status = tddft.solve_batch(states, nthreads=4)
    assert list(status) == [tddft.OK] * len(systems), (status, iters)
    for (om, r), ref, k in zip(res, dense, KS):
        assert om.shape == (k,)
        assert np.max(np.abs(om - ref[:k])) <= acc
    if prec == "fp64":
        for i in (0, 2):                    # the same system alone, on the caller's stream
            c = tddft.Context(systems[i], precision=prec, tol=tol, max_iter=400)
            om, _, it, rc = c.state(sy.initial_guess(systems[i], KS[i], 5 + i)).solve()
            assert rc == tddft.OK
            assert np.max(np.abs(om - res[i][0])) <= 1e-9


def test_batch_refuses_bad_arguments(tddft, systems):
    ctxs = tddft.create_batch(systems[:2], precision="fp64")
    st = ctxs[0].state(sy.initial_guess(systems[0], 1, 1))
    st2 = ctxs[0].state(sy.initial_guess(systems[0], 1, 2))
    with pytest.raises(tddft.TddftError):
        tddft.solve_batch([st, st2])         # one context twice
    res, _, status = tddft.solve_batch([st])
    assert status[0] in (tddft.OK, tddft.E_NOT_CONVERGED)


RECIPES_K = [sy.Recipe(natoms=4, cell_ang=11.0, ngrid=32, radius_ang=4.0, seed=41),
             sy.Recipe(natoms=5, cell_ang=11.0, ngrid=32, radius_ang=4.0, seed=42),
             sy.Recipe(natoms=4, cell_ang=12.0, ngrid=36, radius_ang=4.0, seed=43),
             sy.Recipe(natoms=6, cell_ang=12.0, ngrid=36, radius_ang=4.0, seed=44),
             sy.Recipe(natoms=5, cell_ang=12.0, ngrid=36, radius_ang=4.0, seed=45),
             sy.Recipe(natoms=4, cell_ang=11.0, ngrid=32, radius_ang=4.0, seed=46)]
KS_K = [6, 5, 8, 7, 5, 6]   # each k ends at a gap of the spectrum (>= 6 % to the next state)


def test_batch_of_many_states_runs_concurrently(tddft):
    # 5 to 8 states per system: the trace kernels then take more than 48 KB of shared memory, a
    # launch attribute that must not race between the host threads of the batch (FP64, so that
    # the eigenvalues are checked at the FP64 accuracy)
    systems = [sy.generate(r) for r in RECIPES_K]
    ctxs = tddft.create_batch(systems, precision="fp64", tol=1e-8, max_iter=400)
    states = [c.state(sy.initial_guess(s, k, 20 + i)) for i, (c, s, k) in enumerate(zip(ctxs, systems, KS_K))]
    res, iters, status = tddft.solve_batch(states, nthreads=6)
    assert list(status) == [tddft.OK] * len(systems), [(st, c.last_error()) for st, c in zip(status, ctxs)]
    for (om, r), s, k in zip(res, systems, KS_K):
        ref = casida.Casida(s).omega_symmetric()
        assert np.max(np.abs(om - ref[:k])) <= 1e-6
