"""The full-TDDFT operator in the mixed chi/phi representation (O2), float64.

Eq. operator_RPA (Sec. III A):
    f_p = P^c H^chi P^p - P^p H^phi P^v
    f_q = P^c H^chi P^q - P^q H^phi P^v + 2 P^c V_SCF[P^q] P^v
with V_SCF[P] the matrix <chi_a| v_H[rho] + f_xc rho |phi_b> of the response density
rho(r) = sum chi_a P_ab phi_b (Secs. II A, II C). Only one V_SCF is built per state.

Modes used by the fixed-point checks: "full" (as above), "tda" (B = 0: both blocks become A,
f_p = D p + K p and f_q = D q + K q), "d_only" (K = 0).

Also here: the trace inner product <X, Y> = Tr[X^T S^chi Y S^phi] of Eqs. functional_TDA /
functional_RPA, the kernel-cutoff mask, and the auxiliary-matrix map of Eq. auxiliary,
P = P^c S^chi L S^phi P^v.
"""
import numpy as np

from . import grid, hartree, xc

FULL, TDA, D_ONLY = "full", "tda", "d_only"


class Operator:
    def __init__(self, sys, fxc_kind="lda"):
        self.sys = sys
        self.n = sys.n
        self.cell = sys.cell
        self.dV = sys.dV
        self.chi = grid.BoxedSet(sys.chi, sys.n)
        self.phi = grid.BoxedSet(sys.phi, sys.n)
        self.fxc = xc.fxc_lda(sys.n0) if fxc_kind == "lda" else np.zeros_like(sys.n0)
        self.Sc, self.Sv = sys.S_chi, sys.S_phi
        self.Hc, self.Hv = sys.H_chi, sys.H_phi
        self.Pc, self.Pv = sys.P_c, sys.P_v
        self.mask = kernel_mask(sys)
        self.Mc = self.Pc @ self.Hc
        self.Mv = self.Hv @ self.Pv

    # -- V_SCF (Secs. II A, II C) --------------------------------------------------------------
    def response_density(self, P):
        return grid.response_density(self.chi, self.phi, P)

    def response_potential(self, rho):
        return hartree.hartree(rho, self.cell) + self.fxc[None] * rho

    def v_scf(self, P):
        """<chi_a| v_H[rho] + f_xc rho |phi_b> for a batch P[s]."""
        rho = self.response_density(P)
        V = self.response_potential(rho)
        return grid.potential_integrals(self.chi, self.phi, V, self.dV)

    # -- Eq. operator_RPA -----------------------------------------------------------------------
    def apply(self, Pp, Pq, mode=FULL):
        Pp = np.asarray(Pp, dtype=np.float64)
        Pq = np.asarray(Pq, dtype=np.float64)
        Pc, Hc, Hv, Pv = self.Pc, self.Hc, self.Hv, self.Pv
        fp = np.stack([Pc @ Hc @ X - X @ Hv @ Pv for X in Pp])
        fq = np.stack([Pc @ Hc @ X - X @ Hv @ Pv for X in Pq])
        if mode == FULL:
            Vq = self.v_scf(Pq)
            fq += np.stack([2.0 * Pc @ Vs @ Pv for Vs in Vq])
        elif mode == TDA:
            Vp = self.v_scf(Pp)
            Vq = self.v_scf(Pq)
            fp += np.stack([Pc @ Vs @ Pv for Vs in Vp])
            fq += np.stack([Pc @ Vs @ Pv for Vs in Vq])
        elif mode != D_ONLY:
            raise ValueError(mode)
        return fp, fq

    # -- traces and maps ------------------------------------------------------------------------
    def inner(self, X, Y):
        """Tr[X^T S^chi Y S^phi]."""
        return float(np.trace(X.T @ self.Sc @ Y @ self.Sv))

    def project(self, L):
        """Eq. auxiliary: P = P^c S^chi L S^phi P^v (L masked to the kernel pattern)."""
        return self.Pc @ self.Sc @ (self.mask * L) @ self.Sv @ self.Pv

    def ks_difference(self, X):
        """The left-hand side of Eq. precond for one matrix: P^c H^chi X - X H^phi P^v."""
        return self.Mc @ X - X @ self.Mv

    def pc_x_pv(self, G):
        """P^c G P^v (the projection of an L-space gradient back to a response kernel)."""
        return self.Pc @ G @ self.Pv

    def l_gradient(self, g):
        """Gradient with respect to L of a functional whose contravariant P-gradient is g:
        mask * ((P^c S^chi)^T S^chi g S^phi (S^phi P^v)^T)."""
        Rc = self.Pc @ self.Sc
        Rv = self.Sv @ self.Pv
        return self.mask * (Rc.T @ self.Sc @ g @ self.Sv @ Rv.T)


def kernel_mask(sys):
    """Atom-pair pattern of the response kernels: entry (a, b) is kept when the minimum-image
    distance between the atoms of chi_a and phi_b is within the kernel cutoff. All ones when the
    cutoff is <= 0 (no truncation)."""
    nc, nv = sys.chi.nfun, sys.phi.nfun
    if sys.kernel_cutoff <= 0.0:
        return np.ones((nc, nv))
    pa = sys.pos[sys.chi.atom]
    pb = sys.pos[sys.phi.atom]
    d = pa[:, None, :] - pb[None, :, :]
    d -= sys.cell * np.round(d / sys.cell)
    dist = np.sqrt(np.sum(d * d, axis=-1))
    return (dist <= sys.kernel_cutoff).astype(np.float64)
