"""Dense Casida reference (O1): the plain definition of Sec. II A, for tiny systems.

Steps:
 1. Kohn-Sham states of the synthetic ground state: H^phi c = eps S^phi c (lowest n_occ are the
    valence states), H^chi d = eps S^chi d (lowest n_cond are the conduction states).
 2. psi_v, psi_c on the full grid, products rho_cv = psi_c psi_v, and the coupling matrix
    K_{cv,c'v'} = dV sum_r rho_cv(r) [v_H[rho_c'v'](r) + f_xc(r) rho_c'v'(r)].
 3. A = D + K, B = K with D_{cv,c'v'} = delta (eps_c - eps_v) (Eq. 2, 3).
 4. Eigenvalues of the full matrix [[A, B], [-B, -A]] of Eq. (1); of the symmetric form
    (A-B)^{1/2} (A+B) (A-B)^{1/2} (whose eigenvalues are omega^2, A - B = D diagonal here); and of
    A alone (Tamm-Dancoff, Eq. TDA).

Index order of X: cv flattened with c major, so that P = D_c X C_v^T maps a KS-space vector to the
mixed chi/phi representation (Sec. II C).
"""
import numpy as np
import scipy.linalg

from . import grid, hartree, xc


class Casida:
    def __init__(self, sys, fxc_kind="lda", conduction="spectral"):
        """conduction: "spectral" takes the lowest n_cond states of H^chi d = eps S^chi d;
        "projector" diagonalises H^chi on the range of the given P^c (the joint representation of
        Eq. proj, where the unoccupied space is the range of P^c, not a set of lowest states)."""
        self.sys = sys
        eps_v, C = scipy.linalg.eigh(sys.H_phi, sys.S_phi)
        self.eps_v = eps_v[:sys.n_occ]
        self.Cv = C[:, :sys.n_occ]
        if conduction == "spectral":
            eps_c, Dm = scipy.linalg.eigh(sys.H_chi, sys.S_chi)
            self.eps_c = eps_c[:sys.n_cond]
            self.Dc = Dm[:, :sys.n_cond]
        else:
            # S-orthonormal basis of range(P^c): eigenvectors of S^1/2 P^c S^1/2 with eigenvalue 1
            w, U = scipy.linalg.eigh(sys.S_chi)
            Sh = U @ np.diag(np.sqrt(w)) @ U.T
            Smh = U @ np.diag(1.0 / np.sqrt(w)) @ U.T
            pw, PU = scipy.linalg.eigh(Sh @ sys.P_c @ Sh)
            B = PU[:, pw > 0.5]
            eps_c, Y = scipy.linalg.eigh(B.T @ Smh @ sys.H_chi @ Smh @ B)
            self.eps_c = eps_c
            self.Dc = Smh @ B @ Y
        self.fxc = xc.fxc_lda(sys.n0) if fxc_kind == "lda" else np.zeros_like(sys.n0)
        self.nc, self.nv = self.Dc.shape[1], sys.n_occ

    def ks_orbitals(self):
        n = self.sys.n
        phi = grid.full_grid(self.sys.phi, n).reshape(self.sys.phi.nfun, -1)
        chi = grid.full_grid(self.sys.chi, n).reshape(self.sys.chi.nfun, -1)
        return self.Dc.T @ chi, self.Cv.T @ phi   # psi_c [nc, n^3], psi_v [nv, n^3]

    def coupling(self):
        """K_{cv,c'v'} (Hartree + f_xc), [nc*nv, nc*nv]."""
        n = self.sys.n
        psi_c, psi_v = self.ks_orbitals()
        rho = (psi_c[:, None, :] * psi_v[None, :, :]).reshape(self.nc * self.nv, n, n, n)
        w = hartree.hartree(rho, self.sys.cell) + self.fxc[None] * rho
        K = self.sys.dV * rho.reshape(rho.shape[0], -1) @ w.reshape(w.shape[0], -1).T
        return 0.5 * (K + K.T)

    def ks_differences(self):
        return (self.eps_c[:, None] - self.eps_v[None, :]).ravel()

    def matrices(self, mode="full"):
        d = self.ks_differences()
        K = self.coupling() if mode != "d_only" else np.zeros((d.size, d.size))
        A = np.diag(d) + K
        B = K if mode == "full" else np.zeros_like(K)
        return A, B, d, K

    def full_spectrum(self, mode="full"):
        """All eigenvalues of [[A, B], [-B, -A]], sorted by real part."""
        A, B, _, _ = self.matrices(mode)
        M = np.block([[A, B], [-B, -A]])
        ev = scipy.linalg.eigvals(M)
        return ev[np.argsort(ev.real)]

    def omega_symmetric(self, mode="full"):
        """Positive excitation energies from (A-B)^{1/2}(A+B)(A-B)^{1/2}, ascending."""
        A, B, _, _ = self.matrices(mode)
        w, U = scipy.linalg.eigh(A - B)
        if np.min(w) <= 0:
            raise ValueError("A - B is not positive definite")
        half = U @ np.diag(np.sqrt(w)) @ U.T
        om2 = scipy.linalg.eigvalsh(half @ (A + B) @ half)
        if np.min(om2) <= 0:
            raise ValueError("A + B is not positive definite: complex excitation energies")
        return np.sqrt(om2)

    def omega_tda(self):
        A, _, _, _ = self.matrices("full")
        return scipy.linalg.eigvalsh(A)

    # -- maps between the KS product space and the chi/phi representation ----------------------
    def to_ngwf(self, X):
        """P = D_c X C_v^T for X[nc, nv]."""
        return self.Dc @ X @ self.Cv.T

    def to_ks(self, P):
        """X = D_c^T S^chi P S^phi C_v."""
        return self.Dc.T @ self.sys.S_chi @ P @ self.sys.S_phi @ self.Cv
