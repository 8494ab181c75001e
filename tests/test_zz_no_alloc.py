"""The allocation-free response density (tddft_response_density_noalloc) against the regular
entry point, through the C ABI.

Some callers cannot allocate device memory when they need a density (a pool allocator that
already holds the device memory, or a loop where cudaMalloc / cudaFree would synchronise the
device); the allocation-free entry serves them from a fixed static scratch array.

The two entries run two different tensor-core kernels on the same float32 values of P (the
regular entry rounds the float64 input to float32 on the device, torch rounds it the same way
here): on this workload the regular entry takes the persistent kernel over (tile, state) items
with the vector P gather (density_tc_persistent_kernel), the allocation-free entry the per-tile
kernel with the element-wise gather (density_tc_kernel). Both round the scaled P block to float16
the same way and accumulate in float32 on the tensor cores; they differ only in the order of the
float32 epilogue sums, so the densities agree to 1e-6 of max|rho|. Two calls in a row on
different inputs check that the call clears its fixed scratch (the per-state maxima) before use.
This file is collected last so that it also runs after the other GPU tests.
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
