"""The truncated (linear-scaling) form of the operator and the solver (O2 with truncation), float64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. IV of the paper ("Linear-scaling capabilities") gets O(N) cost by truncating every density
matrix involved -- the ground-state kernels P^v, P^c and the response kernels P^p, P^q -- so that
every matrix-matrix product scales linearly; Sec. III A adds the auxiliary matrices L of
Eq. auxiliary, P = P^c S^chi L S^phi P^v, which may be truncated arbitrarily. The paper does not
spell out the product semantics; this module fixes them (the readings are listed in the design
notes) and writes them out with dense numpy matrices and 0/1 masks:

* patterns by the minimum-image distance of the owning atoms:
    Pi   -- (chi on atom I, phi on atom J) kept when d(I, J) <= r_cut (the kernel cutoff);
    K_cc -- (chi on I, chi on J) kept when d(I, J) <= r_K (the density-kernel cutoff), K_vv
            likewise for phi; r_K <= 0 keeps every pair;
* the ground-state kernels are truncated: P^c_t = K_cc * P^c, P^v_t = K_vv * P^v;
* products of ground-state matrices are exact (computed once): M_c = P^c_t H^chi,
  M_v = H^phi P^v_t, R_c = P^c_t S^chi, R_v = S^phi P^v_t, A_c = S^chi P^c_t S^chi,
  A_v = S^phi P^v_t S^phi;
* every product whose result is a chi x phi matrix is truncated to Pi, T(X) = Pi * X, the way a
  sparse-matrix library stores each product in the fixed pattern of its result; a chain of two
  products is truncated after each one.

Then (Eq. operator_RPA)
    f_p = T(M_c P^p) - T(P^p M_v)
    f_q = T(M_c P^q) - T(P^q M_v) + 2 T(T(P^c_t V) P^v_t),   V = T(V_SCF[P^q]),
the metric of the traces (Eqs. functional_RPA, ortho) is <X, Y> = sum_ab cov(X)_ab Y_ab with
cov(X) = T(T(S^chi X) S^phi) (for untruncated matrices: Tr[X^T S^chi Y S^phi]),
Eq. auxiliary is P = T(T(R_c L) R_v) with L on Pi, the L-gradient is that map's adjoint applied
to cov(g), G_L = T(R_c^T T(cov(g) R_v^T)), the preconditioner's operator (Eq. precond)
T(M_c G) - T(G M_v), and the search gradient T(T(P^c_t G_L) P^v_t). The slope of the sum
functional along a direction is taken in L space, <G_L, z>_F, which equals <g, Z> with
Z = T(T(R_c z) R_v) exactly. When the inner CG's result does not descend (<G_L, z> <= 0: the
truncated operator need not be positive definite) the step takes the search gradient itself.

With both cutoffs covering the cell every mask is all ones and this is the plain O2 oracle.
"""
import numpy as np

from .operator import D_ONLY, FULL, TDA, Operator
from .solver import PCG


def min_image_distances(pos_a, pos_b, cell):
    """[len(pos_a), len(pos_b)] minimum-image distances in a cubic periodic cell."""
    d = pos_a[:, None, :] - pos_b[None, :, :]
    d -= cell * np.round(d / cell)
    return np.sqrt(np.sum(d * d, axis=-1))


def pair_mask(sys, fa, fb, cutoff):
    """0/1 mask over (function of set fa, function of set fb): 1 when the owning atoms are within
    the cutoff (all ones for cutoff <= 0)."""
    if cutoff <= 0.0:
        return np.ones((fa.nfun, fb.nfun))
    dist = min_image_distances(sys.pos[fa.atom], sys.pos[fb.atom], sys.cell)
    return (dist <= cutoff).astype(np.float64)


class TruncatedOperator(Operator):
    """The operator, metric and maps of the truncated (linear-scaling) form."""

    def __init__(self, sys, fxc_kind="lda"):
        if sys.kernel_cutoff <= 0.0:
            raise ValueError("the truncated form needs a kernel cutoff")
        super().__init__(sys, fxc_kind)
        rK = getattr(sys, "density_kernel_cutoff", 0.0)
        self.Pc = sys.P_c * pair_mask(sys, sys.chi, sys.chi, rK)
        self.Pv = sys.P_v * pair_mask(sys, sys.phi, sys.phi, rK)
        self.Mc = self.Pc @ self.Hc
        self.Mv = self.Hv @ self.Pv
        self.Rc = self.Pc @ self.Sc
        self.Rv = self.Sv @ self.Pv
        self.Ac = self.Sc @ self.Pc @ self.Sc
        self.Av = self.Sv @ self.Pv @ self.Sv
        self.RcT = self.Sc @ self.Pc        # R_c^T = (P^c S^chi)^T
        self.RvT = self.Pv @ self.Sv        # R_v^T = (S^phi P^v)^T

    def T(self, X):
        return self.mask * X

    def apply(self, Pp, Pq, mode=FULL):
        Pp = np.asarray(Pp, dtype=np.float64)
        Pq = np.asarray(Pq, dtype=np.float64)
        fp = np.stack([self.ks_difference(X) for X in Pp])
        fq = np.stack([self.ks_difference(X) for X in Pq])
        if mode == FULL:
            Vq = self.T(self.v_scf(Pq))
            fq += np.stack([2.0 * self.pc_x_pv(Vs) for Vs in Vq])
        elif mode == TDA:
            Vp = self.T(self.v_scf(Pp))
            Vq = self.T(self.v_scf(Pq))
            fp += np.stack([self.pc_x_pv(Vs) for Vs in Vp])
            fq += np.stack([self.pc_x_pv(Vs) for Vs in Vq])
        elif mode != D_ONLY:
            raise ValueError(mode)
        return fp, fq

    def ks_difference(self, X):
        return self.T(self.Mc @ X) - self.T(X @ self.Mv)

    def pc_x_pv(self, G):
        return self.T(self.T(self.Pc @ G) @ self.Pv)

    def cov(self, X):
        return self.T(self.T(self.Sc @ X) @ self.Sv)

    def inner(self, X, Y):
        return float(np.sum(self.cov(X) * Y))

    def project(self, L):
        return self.T(self.T(self.Rc @ (self.mask * L)) @ self.Rv)

    def l_gradient(self, g):
        """The gradient of the sum functional with respect to L through the truncated map
        P = T(T(R_c L) R_v): with the slope along D in P taken as <g, D> = sum cov(g) * D, it is
        the map's adjoint applied to cov(g), T(R_c^T T(cov(g) R_v^T)) (the truncations of the map
        in reverse order; without truncation this is S P^c S g S P^v S)."""
        return self.T(self.RcT @ self.T(self.cov(g) @ self.RvT))


class TruncatedPCG(PCG):
    """The PCG of Sec. III C on the truncated operator (preconditioner "iter" or "none")."""

    def __init__(self, op, Y0, **kw):
        if not isinstance(op, TruncatedOperator):
            raise TypeError("TruncatedPCG needs a TruncatedOperator")
        if kw.get("precond", "iter") not in ("iter", "none"):
            raise ValueError("the truncated form has the inner-CG preconditioner or none")
        super().__init__(op, Y0, **kw)

    def gradient_when_not_descent(self):
        """With every product cut to the pattern and P^c, P^v truncated, the inner CG's operator
        T(M_c G) - T(G M_v) need not be positive definite on the pattern (the truncated P^c is no
        longer a projector, and H^chi's large eigenvalues magnify the difference), so the CG can
        stop on non-positive curvature with a result that does not descend. The paper's
        preconditioner is only meant to speed up the descent (Sec. III B), so such a step takes
        the search gradient itself (counted in fallbacks)."""
        return self.precond == "iter"

    def gdot(self, gp, gq, zp, zq, Zp, Zq):
        """sum_i <G_L,i, z_i>_F, the slope in L space."""
        return float(sum(np.sum(self.GLp[i] * zp[i]) + np.sum(self.GLq[i] * zq[i]) for i in range(self.k)))
