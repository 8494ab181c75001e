"""Edge cases of the C ABI on the GPU:

* state counts: k = 0 (apply and state creation) and k = 17 (one past the 16-pair maximum of a
  state) are refused with INVALID; k = 16 steps with the FP64 oracle;
* all-zero response kernels give exactly zero in every mode and precision (every stage is
  linear, and the tensor-core paths' per-state scale of an all-zero input is 1);
* a one-atom system (4 phi, 4 chi; two occupied and two unoccupied functions) against the
  oracle, FP64 and mixed.
"""
import numpy as np
import pytest

from oracle import operator as oop, solver as osolver
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
def one_atom():
    return sy.generate(sy.Recipe(natoms=1, cell_ang=8.0, ngrid=24, radius_ang=3.0, seed=17))


def _err(got, ref):
    return float(np.max(np.abs(np.asarray(got) - ref)) / max(np.max(np.abs(ref)), 1e-300))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_zero_states_are_refused(tddft, tiny, prec):
    ctx = tddft.Context(tiny, precision=prec)
    empty = np.zeros((0, ctx.nc, ctx.nv))
    with pytest.raises(tddft.TddftError) as e:
        ctx.apply(empty, empty)
    assert e.value.status == tddft.E_INVALID
    with pytest.raises(tddft.TddftError) as e:
        ctx.state(empty)
    assert e.value.status == tddft.E_INVALID
    ctx.apply(*sy.random_kernels(tiny, 1, 2))          # the context stays usable


def test_more_than_sixteen_pairs_are_refused(tddft, tiny):
    ctx = tddft.Context(tiny, precision="fp64")
    with pytest.raises(tddft.TddftError) as e:
        ctx.state(sy.initial_guess(tiny, 17, 5))
    assert e.value.status == tddft.E_INVALID


def test_sixteen_pairs_step_with_the_oracle(tddft, tiny):
    k = 16
    Y0 = sy.initial_guess(tiny, k, 6)
    ref = osolver.PCG(oop.Operator(tiny), Y0)
    st = tddft.Context(tiny, precision="fp64").state(Y0)
    for _ in range(2):
        om_r, _ = ref.step()
        om_g, _ = st.step()
        assert np.max(np.abs(om_g - om_r)) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("mode", ["full", "tda", "d_only"])
def test_zero_kernels_give_zero(tddft, tiny, prec, mode):
    ctx = tddft.Context(tiny, precision=prec, mode=mode)
    z = np.zeros((2, ctx.nc, ctx.nv))
    fp, fq = ctx.apply(z, z)
    assert np.all(fp == 0.0) and np.all(fq == 0.0)


@pytest.mark.parametrize("prec,tol,tol_grid", [("fp64", 1e-10, 1e-10), ("mixed", 3e-5, 2e-3)])
def test_one_atom_system(tddft, one_atom, prec, tol, tol_grid):
    s = one_atom
    assert (s.chi.nfun, s.phi.nfun, s.n_occ, s.n_cond) == (4, 4, 2, 2)
    ctx = tddft.Context(s, precision=prec)
    Pp, Pq = sy.random_kernels(s, 2, 7)
    fp, fq = ctx.apply(Pp, Pq)
    rp, rq = oop.Operator(s).apply(Pp, Pq)
    assert _err(fp, rp) < tol and _err(fq, rq) < tol_grid
