"""Failure detection of the tensor-core kernels' bounded waits, without faulting or hanging the GPU.

tddft_wait_check launches a kernel that waits, with the context's spin_limit_cycles, on a barrier
nothing completes. The wait must expire, the kernel must return, and the call must report
TDDFT_E_TIMEOUT through the same error word every tensor-core kernel uses. The context must stay
usable: an operator application on it afterwards matches the oracle, and a second check expires
again (the error word was cleared in between).
"""
import time

import numpy as np
import pytest

from oracle import operator as oop
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


def test_short_limit_expires_and_context_stays_usable(tddft, tiny):
    # 2e7 cycles: about 10 ms at the GB300's clocks, far above any wait of a healthy kernel on
    # this system, far below the 2 s default
    ctx = tddft.Context(tiny, precision="mixed", precond="none", spin_limit_cycles=20_000_000)
    t0 = time.perf_counter()
    assert ctx.wait_check() == tddft.E_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert "expired" in tddft.load().tddft_last_error(ctx._ctx).decode()
    Pp, Pq = sy.random_kernels(tiny, 2, 5)
    fp, fq = ctx.apply(Pp, Pq)
    rp, rq = oop.Operator(tiny).apply(Pp, Pq)
    for got, ref in ((fp, rp), (fq, rq)):
        assert np.max(np.abs(got - ref)) <= 1e-3 * np.max(np.abs(ref))
    assert ctx.wait_check() == tddft.E_TIMEOUT
    ctx.close()


def test_default_limit_also_reports_timeout(tddft, tiny):
    # the default limit (4e9 cycles, about 2 s) expires as well, only later
    ctx = tddft.Context(tiny, precision="fp64", precond="none")
    t0 = time.perf_counter()
    assert ctx.wait_check() == tddft.E_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    ctx.close()
