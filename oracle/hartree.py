"""Hartree response potential (Sec. II A, the 1/|r - r'| term of K) on the periodic grid.

v_H(G) = 4 pi rho(G) / |G|^2 with G = 2 pi m / L for the integer frequencies m of the discrete
Fourier transform; the G = 0 term is dropped (neutralising background). The paper uses open
boundary conditions for an isolated molecule (Sec. IV A); the synthetic cells are periodic with
the G = 0 term removed, which keeps the Hartree kernel positive semidefinite.
"""
import numpy as np


def g2_grid(n, cell):
    m = np.fft.fftfreq(n, d=1.0 / n)
    g = 2.0 * np.pi * m / cell
    return g[:, None, None] ** 2 + g[None, :, None] ** 2 + g[None, None, :] ** 2


def hartree(rho, cell):
    """v_H on the grid for one or more real densities rho[..., n, n, n]."""
    n = rho.shape[-1]
    g2 = g2_grid(n, cell)
    kern = np.zeros_like(g2)
    nz = g2 > 0
    kern[nz] = 4.0 * np.pi / g2[nz]
    rg = np.fft.fftn(rho, axes=(-3, -2, -1))
    return np.real(np.fft.ifftn(rg * kern, axes=(-3, -2, -1)))
