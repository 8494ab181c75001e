"""Oscillator strengths and broadened absorption spectra (test infrastructure: the plain CPU
oracle; only tests, the smoke check and the benchmark's CPU baseline use this module).

The paper reports every result as excitation energies with oscillator strengths and as spectra
broadened by Lorentzians of 0.025 eV (Sec. IV: the azobenzene table and the bacteriochlorophyll
spectra). It does not print the formulas; the standard linear-response ones are used:

* transition dipole of excitation i: mu_i = integral of r rho^q_i(r) d^3r, rho^q_i the response
  density of q_i = X_i + Y_i (Sec. II C builds rho from the q kernel), with the pair normalised
  as in Eq. Tsiper_multiple (<p_i, q_i> = 1);
* oscillator strength f_i = (2/3) omega_i |mu_i|^2 (spin dropped as everywhere in the paper's
  equations);
* spectrum S(E) = sum_i f_i (gamma / pi) / ((E - omega_i)^2 + gamma^2), gamma the half width at
  half maximum.

Readings (the paper is silent on them): the position operator of the periodic cell is the grid
coordinate measured from the cell centre, x_a(i) = i h - L/2 for grid index i along axis a; the
Ritz pairs of a converged PCG subspace are the current pairs rotated by the eigenvectors of the
symmetrised Q of the subspace diagonalisation (Sec. III C), which keeps <p_i, q_j> = delta_ij.

Two routes: O1 (dense, KS product space: dipoles d_cv = <psi_c| r |psi_v> on the grid and the
eigenvectors of the symmetric form) and O2 (the PCG iterate: the grid response density of each
Ritz q). Pins: the finite-basis Thomas-Reiche-Kuhn sum rule of the full problem (sum_i f_i over
all excitations does not depend on the coupling K), the closed form of the uncoupled case, the
TDA sum (which does depend on K, the sum-rule violation the paper mentions in Sec. II A), and
the Lorentzian's area and peak height.
"""
import numpy as np
import scipy.linalg

LORENTZ_HWHM_EV = 0.025


def positions(n, cell):
    """x_a(i) = i h - L/2 on an n-point axis of a cell of side L (bohr)."""
    return np.arange(n) * (cell / n) - 0.5 * cell


def grid_dipoles(rho, cell, dV):
    """mu[s, a] = dV sum_r x_a(r) rho_s(r) for rho[s, n, n, n] (axis order x, y, z)."""
    n = rho.shape[1]
    x = positions(n, cell)
    mx = np.einsum("sijk,i->s", rho, x)
    my = np.einsum("sijk,j->s", rho, x)
    mz = np.einsum("sijk,k->s", rho, x)
    return dV * np.stack([mx, my, mz], axis=1)


def strengths(omega, mu):
    """f_i = (2/3) omega_i |mu_i|^2."""
    return (2.0 / 3.0) * np.asarray(omega) * np.sum(np.asarray(mu) ** 2, axis=1)


def lorentzian_spectrum(E, omega, f, gamma):
    """S(E) = sum_i f_i (gamma / pi) / ((E - omega_i)^2 + gamma^2)."""
    E = np.asarray(E, dtype=np.float64)[:, None]
    return np.sum(np.asarray(f)[None, :] * (gamma / np.pi) / ((E - np.asarray(omega)[None, :]) ** 2 + gamma ** 2),
                  axis=1)


# ---- O1: dense KS product space --------------------------------------------------------------------
def ks_dipoles(cas):
    """d[a, cv] = dV sum_r x_a(r) psi_c(r) psi_v(r), cv flattened c-major like the Casida matrices."""
    s = cas.sys
    psi_c, psi_v = cas.ks_orbitals()
    n = s.n
    rho = (psi_c[:, None, :] * psi_v[None, :, :]).reshape(cas.nc * cas.nv, n, n, n)
    return grid_dipoles(rho, s.cell, s.dV).T


def dense_pairs(cas, mode="full"):
    """All excitations of the dense problem: omega ascending and q = X + Y per column, normalised
    so that p^T q = 1 (for TDA and the uncoupled case p = q = X with X^T X = 1)."""
    A, B, _, _ = cas.matrices(mode)
    if mode == "tda":
        om, X = scipy.linalg.eigh(A)
        return om, X
    w, U = scipy.linalg.eigh(A - B)
    H = U @ np.diag(np.sqrt(w)) @ U.T                       # (A - B)^{1/2}
    om2, F = scipy.linalg.eigh(H @ (A + B) @ H)
    om = np.sqrt(om2)
    return om, (H @ F) / np.sqrt(om)[None, :]               # q = (A - B)^{1/2} F / sqrt(omega)


def dense_strengths(cas, mode="full"):
    """(omega, f, mu) of every excitation of the dense problem (mode full, tda or d_only)."""
    om, q = dense_pairs(cas, mode)
    d = ks_dipoles(cas)
    mu = (d @ q).T
    return om, strengths(om, mu), mu


# ---- O2: the PCG iterate ------------------------------------------------------------------------------
def ritz_strengths(pcg):
    """(omega, f, mu) of the Ritz pairs of a PCG state (oracle.solver.PCG): rotate q by the
    eigenvectors of the symmetrised Q, dipoles of the rotated response densities."""
    k = pcg.k
    Q = 0.5 * np.array([[pcg.inner(pcg.Pp[j], pcg.fp[i]) + pcg.inner(pcg.Pq[j], pcg.fq[i])
                         for j in range(k)] for i in range(k)])
    om, U = np.linalg.eigh(0.5 * (Q + Q.T))
    rho = pcg.op.response_density(pcg.Pq)
    mu_j = grid_dipoles(rho, pcg.op.cell, pcg.op.dV)         # dipoles of the current q_j
    mu = U.T @ mu_j                                        # the dipole is linear in q
    return om, strengths(om, mu), mu
