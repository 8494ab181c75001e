"""Oscillator strengths and spectra on the GPU through the C ABI, against the FP64 oracle
(oracle/spectrum.py):

* step parity: after PCG steps from the same start, the Ritz energies, strengths and dipoles of
  the GPU state equal the oracle's (FP64: omega to 1e-10 Ha, f and |mu| to 1e-8 of their scale);
* converged states reproduce the dense strengths of the lowest excitations (FP64 to 1e-6 of the
  largest strength; mixed precision to 4e-3: the tensor-core response density has float16
  operands, 2e-3 of its scale per point as in the operator tests, and f is quadratic in it);
* the device Lorentzian spectrum equals the oracle's to 1e-12.
"""
import numpy as np
import pytest

from oracle import operator as oop, solver as osolver, spectrum
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
def dense(tiny):
    from oracle import casida
    return spectrum.dense_strengths(casida.Casida(tiny), "full")


def _aligned(mu, ref):
    s = np.sign(np.sum(mu * ref, axis=1))
    s[s == 0] = 1.0
    return mu * s[:, None]


def test_ritz_strengths_step_parity(tddft, tiny):
    k = 3
    Y0 = sy.initial_guess(tiny, k, 7)
    ref = osolver.PCG(oop.Operator(tiny), Y0)
    ctx = tddft.Context(tiny, precision="fp64")
    st = ctx.state(Y0)
    for _ in range(4):
        ref.step()
        st.step()
    om, f, mu = st.oscillator_strengths()
    om_r, f_r, mu_r = spectrum.ritz_strengths(ref)
    assert np.max(np.abs(om - om_r)) < 1e-10
    assert np.max(np.abs(f - f_r)) <= 1e-8 * np.max(f_r)
    assert np.max(np.abs(_aligned(mu, mu_r) - mu_r)) <= 1e-8 * np.max(np.abs(mu_r))


@pytest.mark.parametrize("prec,tol,acc", [("fp64", 1e-9, 1e-6), ("mixed", 1e-6, 4e-3)])
def test_converged_strengths_match_dense(tddft, tiny, dense, prec, tol, acc):
    k = 3
    ctx = tddft.Context(tiny, precision=prec, tol=tol, max_iter=600)
    st = ctx.state(sy.initial_guess(tiny, k, 1))
    _, _, it, rc = st.solve()
    assert rc == tddft.OK, (rc, it)
    om, f, _ = st.oscillator_strengths()
    om_d, f_d, _ = dense
    assert np.max(np.abs(om - om_d[:k])) <= (1e-6 if prec == "fp64" else 1e-5)
    assert np.max(np.abs(f - f_d[:k])) <= acc * np.max(f_d[:k])


def test_spectrum_matches_oracle(tddft, tiny):
    ctx = tddft.Context(tiny, precision="mixed")
    rng = np.random.default_rng(3)
    om = np.sort(rng.uniform(0.05, 0.3, size=7))
    f = rng.uniform(0.0, 0.5, size=7)
    E = np.linspace(0.0, 0.4, 1001)
    gamma = spectrum.LORENTZ_HWHM_EV / 27.211386246
    S = ctx.spectrum(om, f, E, gamma)
    ref = spectrum.lorentzian_spectrum(E, om, f, gamma)
    assert np.max(np.abs(S - ref)) <= 1e-12 * np.max(ref)
    with pytest.raises(tddft.TddftError):
        ctx.spectrum(om, f, E, -1.0)
