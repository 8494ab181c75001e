"""Checkpoint and resume of a PCG state through the C ABI (tddft_state_export / tddft_state_import).

* a state exported after some steps and imported on the same context, or on a fresh context of
  the same system, continues as the uninterrupted state does: the first evaluation after the
  import is bit for bit the same (the checkpoint holds everything a step reads from earlier
  steps), later steps agree to the run-to-run rounding of the grid integrals (their atomic
  accumulation order varies), and both still follow the FP64 oracle's PCG (omega to 1e-10 Ha);
* the same in mixed precision and with a truncated kernel pattern (Eq. auxiliary);
* a checkpoint of another precision or size, or a damaged one, is refused with INVALID.
"""
import dataclasses

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


@pytest.mark.parametrize("prec,trunc,fresh", [("fp64", False, False), ("fp64", False, True),
                                              ("fp64", True, True), ("mixed", False, True)])
def test_resume_reproduces_the_uninterrupted_run(tddft, tiny, prec, trunc, fresh):
    s = dataclasses.replace(tiny, kernel_cutoff=3.0 / 0.529177210903) if trunc else tiny
    k = 2
    Y0 = sy.initial_guess(s, k, 3)
    ctx = tddft.Context(s, precision=prec)
    st = ctx.state(Y0)
    ref = osolver.PCG(oop.Operator(s), Y0) if prec == "fp64" else None
    for _ in range(3):
        st.step()
        if ref is not None:
            ref.step()
    blob = st.export()
    assert len(blob) == 48 + 8 * (k + 5) + 8 * 2 * k * ctx.nc * ctx.nv * (8 if prec == "fp64" else 4)
    ctx2 = tddft.Context(s, precision=prec) if fresh else ctx
    st2 = ctx2.import_state(blob)
    assert st2.k == k and st2.stats()[0] == st.stats()[0] == 3
    tol = 1e-12 if prec == "fp64" else 1e-6
    for it in range(4):
        om_a, res_a = st.step()
        om_b, res_b = st2.step()
        if it == 0:
            assert np.array_equal(om_a, om_b) and np.array_equal(res_a, res_b)
        assert np.max(np.abs(om_a - om_b)) <= tol
        assert np.max(np.abs(res_a - res_b) / res_a) <= 1e3 * tol
        if ref is not None:
            om_r, _ = ref.step()
            assert np.max(np.abs(om_b - om_r)) < 1e-10
    a, b = st.get(), st2.get()
    for name in a:
        assert np.max(np.abs(a[name] - b[name])) <= 1e3 * tol * np.max(np.abs(a[name]))
    assert st.stats()[:2] == st2.stats()[:2]


def test_bad_checkpoints_are_refused(tddft, tiny):
    k = 2
    ctx = tddft.Context(tiny, precision="fp64")
    st = ctx.state(sy.initial_guess(tiny, k, 4))
    st.step()
    blob = st.export()
    other = tddft.Context(tiny, precision="mixed")
    with pytest.raises(tddft.TddftError) as e:
        other.import_state(blob)                       # precision differs
    assert e.value.status == tddft.E_INVALID
    small = sy.generate(sy.Recipe(natoms=2, cell_ang=10.0, ngrid=30, radius_ang=4.0, seed=12))
    with pytest.raises(tddft.TddftError):
        tddft.Context(small, precision="fp64").import_state(blob)   # sizes differ
    with pytest.raises(tddft.TddftError):
        ctx.import_state(blob[:-8])                    # truncated
    bad = bytearray(blob)
    bad[0:8] = b"NOTACKPT"
    with pytest.raises(tddft.TddftError):
        ctx.import_state(bytes(bad))
    st.step()                                          # the context stays usable
