"""The allocation-free response density (tddft_response_density_noalloc) against the regular
entry point, through the C ABI.

The two calls run the same tensor-core kernel on the same float32 values of P (the regular entry
rounds the float64 input to float32 on the device, torch rounds it the same way here), so their
densities agree to float32 roundoff of the epilogue; the bound is 1e-6 of max|rho|. Two calls in
a row on different inputs check that the call clears its fixed scratch (the per-state maxima)
before use. This file is collected last so that it also runs after the other GPU tests.
"""
import numpy as np
import pytest

from paper_1507_08157_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

TOL = 1e-6


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
def small():
    return sy.generate(sy.CONFIG_SMALL)


def _err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_noalloc_density_matches_regular_entry(tddft, small):
    import torch
    ctx = tddft.Context(small, precision="mixed")
    n = small.n
    rho = torch.empty((5, n, n, n), dtype=torch.float32, device="cuda")
    # two calls in a row; the second has larger values, so stale maxima would show
    for seed, scale in ((21, 1.0), (22, 37.0)):
        _, Pq = sy.random_kernels(small, 5, seed)
        Pq = Pq * scale
        ref = ctx.response_density(Pq)
        P32 = torch.from_numpy(Pq).to(torch.float32).cuda()
        got = ctx.response_density_noalloc(P32, rho)
        torch.cuda.synchronize()
        assert _err(got.cpu().numpy().astype(np.float64), ref) < TOL


def test_noalloc_density_rejects_bad_sizes(tddft, small):
    import torch
    ctx = tddft.Context(small, precision="mixed")
    n = small.n
    big = tddft.NOALLOC_MAX_STATES + 1
    P = torch.zeros((big, ctx.nc, ctx.nv), dtype=torch.float32, device="cuda")
    rho = torch.empty((big, n, n, n), dtype=torch.float32, device="cuda")
    with pytest.raises(tddft.TddftError) as e:
        ctx.response_density_noalloc(P, rho)
    assert e.value.status == tddft.E_INVALID
    # float64 contexts have no allocation-free path
    ctx64 = tddft.Context(small, precision="fp64")
    with pytest.raises(tddft.TddftError) as e:
        ctx64.response_density_noalloc(P[:1].contiguous(), rho[:1].contiguous())
    assert e.value.status == tddft.E_INVALID
