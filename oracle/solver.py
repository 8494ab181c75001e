"""Preconditioned conjugate-gradient solver for the lowest N_omega full-TDDFT states (O2), float64.

Follows Sec. III of the paper:
  * trial pairs x_i = (P^p_i, P^q_i) = P^c S^chi L_i S^phi P^v (Eq. auxiliary; L_i = the search
    variables, masked to the kernel pattern; with no truncation the mask is all ones);
  * operator f_i = f(x_i) of Eq. operator_RPA;
  * Q_ij = (<p_j, f_p,i> + <q_j, f_q,i>) / 2 (Sec. III C);
  * multi-state gradient g_i = f_i - sum_j Q_ij (P^q_j ; P^p_j) (Sec. III C, with the M-normalised
    pairs of Eq. ortho, so each denominator 2 Tr[p_j S q_j S] is 2);
  * preconditioner: the linear system of Eq. precond, L(G) = P^c H^chi G - G H^phi P^v = g,
    solved by CG in the trace inner product to a relative residual eps_tol (or 50 iterations);
  * update P_i -> P_i + lambda d_i with one line step for all states, chosen to minimise the sum
    functional of Eq. Tsiper_multiple (Eq. min_multiple) along the line;
  * the sign flip of Sec. III C and Gram-Schmidt in the metric of Eq. ortho after every step;
  * final energies from the eigenvalues of Q (Sec. III C).

Readings where the paper is silent (Algorithms 1 and 2 of its supplement are not available):
  * random start: X random and Y = 0, i.e. p = q (the metric of Eq. ortho is then positive);
  * gradient coefficient: Eq. tsip_grad's bracket is the sum of both traces (= 2 omega); the
    derivative of Eq. functional_RPA under the normalisation constraint, the j = i term of the
    multi-state gradient and the orthogonality of g to the subspace all give omega, so Q_ij is used;
  * line step: along x_i(lambda) = x_i + lambda Delta_i the sum of the Tsiper energies of the
    re-orthonormalised set is Omega(lambda) = Tr[M(lambda)^-1 N(lambda)] / 2 with the k x k
    matrices N_ij = <x_i, f(x_j)>_E and M_ij = (<p_i,q_j> + <p_j,q_i>)/2, each quadratic in
    lambda. A minimum on the descent side is found to machine precision: a sign change of
    dOmega/dlambda is bracketed by doubling a Newton estimate (a non-positive-definite M counts as
    past the minimum), then located by Illinois regula falsi;
  * conjugation: Polak-Ribiere on the whole set, beta = max(0, sum_i <g_i, z_i - z_prev,i> /
    sum_i <g_prev,i, z_prev,i>), z the projected preconditioned gradient; reset every 10
    iterations, after a sign flip, and whenever the conjugate direction is not a descent direction;
  * truncation (Eq. auxiliary): the search runs in L. The L-gradient is
    G_L = mask * ((P^c S^chi)^T S^chi g S^phi (S^phi P^v)^T) and the preconditioned direction is
    z = mask * Pinv(P^c G_L P^v), Pinv the inner-CG solve of Eq. precond. C -> Pinv(P^c C P^v) is
    positive semidefinite in the Frobenius product, so z is always a descent direction; without
    truncation P^c G_L P^v = g and this is the plain preconditioned gradient;
  * residual: sqrt(<g_p, g_p> + <g_q, g_q>) without truncation; with truncation the Frobenius
    norm of G_L (the P-space gradient does not vanish at the constrained minimum);
  * convergence: max residual <= tol and max change of the eigenvalues of Q <= tol / 10;
  * Gram-Schmidt: states in ascending order of Q_ii, classical Gram-Schmidt run twice on the
    coefficient vectors of the M Gram matrix (which the line search already holds); a
    non-positive norm after projection is a breakdown;
  * f is carried along by the same linear combinations and recomputed from scratch every
    ``reapply_every`` iterations, after P is recomputed from L by Eq. auxiliary (the two agree
    in exact arithmetic; in float32 this keeps P on the invariant subspace).
"""
import numpy as np

from .operator import FULL


class Breakdown(RuntimeError):
    pass


def _chol_solve(M, B):
    """Solve M X = B for symmetric positive definite M; None if M is not positive definite."""
    try:
        c = np.linalg.cholesky(M)
    except np.linalg.LinAlgError:
        return None
    y = np.linalg.solve(c, B)
    return np.linalg.solve(c.T, y)


def sum_functional(lam, N0, N1, N2, M0, M1, M2):
    """Omega(lambda) = Tr[M^-1 N] / 2 and dOmega/dlambda; (inf, inf) if M is not positive definite."""
    M = M0 + lam * M1 + lam * lam * M2
    N = N0 + lam * N1 + lam * lam * N2
    dM = M1 + 2.0 * lam * M2
    dN = N1 + 2.0 * lam * N2
    W = _chol_solve(M, N)
    if W is None:
        return np.inf, np.inf
    X = _chol_solve(M, dN)
    Z = _chol_solve(M, dM @ W)
    return 0.5 * np.trace(W), 0.5 * (np.trace(X) - np.trace(Z))


def line_step(N0, N1, N2, M0, M1, M2):
    """A minimiser lambda > 0 of the sum functional along the line (0 if not a descent line):
    bracket a sign change of dOmega/dlambda from below by doubling a Newton estimate, then
    Illinois regula falsi inside the bracket to machine precision."""
    _, d0 = sum_functional(0.0, N0, N1, N2, M0, M1, M2)
    if not np.isfinite(d0) or d0 >= 0.0:
        return 0.0
    # Newton estimate of the step from the model with M0 = I
    h0 = np.trace(2.0 * N2 - 2.0 * M1 @ N1 + 2.0 * M1 @ M1 @ N0 - 2.0 * M2 @ N0) * 0.5
    hi = -d0 / h0 if h0 > 0.0 and np.isfinite(h0) else 1.0
    lo, dlo, d = 0.0, d0, d0
    for _ in range(60):
        _, d = sum_functional(hi, N0, N1, N2, M0, M1, M2)
        if d >= 0.0:
            break
        lo, dlo, hi = hi, d, 2.0 * hi
    dhi = d
    for _ in range(200):          # past the positive-definite region: bisect to a finite end
        if np.isfinite(dhi):
            break
        mid = 0.5 * (lo + hi)
        _, d = sum_functional(mid, N0, N1, N2, M0, M1, M2)
        if d < 0.0:
            lo, dlo = mid, d
        else:
            hi, dhi = mid, d
    side = 0
    for _ in range(100):
        if not hi - lo > 4e-16 * hi:
            break
        x = hi - dhi * (hi - lo) / (dhi - dlo) if (np.isfinite(dhi) and dhi != dlo) else 0.5 * (lo + hi)
        if not lo < x < hi:
            x = 0.5 * (lo + hi)
        _, d = sum_functional(x, N0, N1, N2, M0, M1, M2)
        if d == 0.0:
            return x
        if d < 0.0:
            lo, dlo = x, d
            if side == -1:
                dhi *= 0.5
            side = -1
        else:
            hi, dhi = x, d
            if side == 1:
                dlo *= 0.5
            side = 1
    return 0.5 * (lo + hi)


def gram_schmidt_coefficients(Mg, order):
    """Coefficient matrix C (rows = new vectors in terms of old) making the M Gram matrix the
    identity, processing states in ``order``; classical Gram-Schmidt applied twice."""
    k = Mg.shape[0]
    C = np.zeros((k, k))
    done = []
    for i in order:
        v = np.zeros(k)
        v[i] = 1.0
        for _ in range(2):
            coef = [float(v @ Mg @ C[j]) for j in done]
            for cj, j in zip(coef, done):
                v = v - cj * C[j]
        nrm = float(v @ Mg @ v)
        if not np.isfinite(nrm) or nrm <= 1e-12 * max(1.0, abs(Mg[i, i])):
            raise Breakdown("non-positive norm in Gram-Schmidt")
        C[i] = v / np.sqrt(nrm)
        done.append(i)
    return C


class PCG:
    def __init__(self, op, Y0, mode=FULL, precond="iter", precond_tol=1e-4,
                 precond_maxit=50, reapply_every=10, restart_every=10, mlp=None, precond_adaptive=False):
        """precond: "iter" (inner CG on Eq. precond), "exact" (Eq. precond solved exactly in the
        Kohn-Sham basis, where it is diagonal), "none", or "learned" with mlp = (parameter vector,
        hidden width) of the atom-block network of ``learned``.
        precond_adaptive: the inner tolerance of a step is min(0.1, max(precond_tol, largest
        residual of the iterate)) -- loose first, tight at the end (suggested in Sec. IV A)."""
        self.op = op
        self.mode = mode
        self.precond = precond
        self.learned = None
        if precond == "learned":
            from .learned import LearnedPreconditioner
            self.learned = LearnedPreconditioner(op.sys, mlp[0], mlp[1], op.mask)
        self.casida = None
        if precond == "exact":
            from .casida import Casida
            self.casida = Casida(op.sys, fxc_kind="none")
        self.precond_tol = precond_tol
        self.precond_adaptive = precond_adaptive
        self.step_tol = precond_tol
        self.precond_maxit = precond_maxit
        self.reapply_every = reapply_every
        self.restart_every = restart_every
        self.trunc = op.sys.kernel_cutoff > 0.0
        m = op.mask
        self.Yp = np.array([m * Y for Y in Y0])
        self.Yq = self.Yp.copy()
        self.k = self.Yp.shape[0]
        self.Pp = np.array([op.project(Y) for Y in self.Yp])
        self.Pq = np.array([op.project(Y) for Y in self.Yq])
        self.fp = np.zeros_like(self.Pp)
        self.fq = np.zeros_like(self.Pq)
        T = self.pq_products(self.Pp, self.Pq)
        self.orthonormalize(T, list(range(self.k)))
        self.reapply()
        self.it = 0
        self.omega_prev = None
        self.prev = None
        self.flipped = False
        self.inner_iters = 0
        self.fallbacks = 0
        self.last_lambda = 0.0

    # ---------------------------------------------------------------------------------------------
    def inner(self, X, Y):
        return self.op.inner(X, Y)

    def reapply(self):
        self.fp, self.fq = self.op.apply(self.Pp, self.Pq, self.mode)

    def pq_products(self, A, B):
        """T_ij = <A_i, B_j> over the states."""
        return np.array([[self.inner(A[i], B[j]) for j in range(self.k)] for i in range(self.k)])

    def orthonormalize(self, T, order):
        """Sign flip (q -> -q where <p_i, q_i> < 0), then Gram-Schmidt in the metric of Eq. ortho.
        T_ij = <p_i, q_j> of the current pairs."""
        T = T.copy()
        flipped = False
        for i in range(self.k):
            if T[i, i] < 0.0:
                self.Pq[i] *= -1.0
                self.Yq[i] *= -1.0
                self.fq[i] *= -1.0
                T[:, i] *= -1.0
                flipped = True
        Mg = 0.5 * (T + T.T)
        C = gram_schmidt_coefficients(Mg, order)
        for arr in (self.Yp, self.Yq, self.Pp, self.Pq, self.fp, self.fq):
            arr[...] = np.einsum("ia,arc->irc", C, arr)
        return flipped

    # ---------------------------------------------------------------------------------------------
    def evaluate(self):
        """Q matrix, its eigenvalues, the gradients and residuals of the current iterate."""
        k = self.k
        a = np.array([[self.inner(self.Pp[j], self.fp[i]) + self.inner(self.Pq[j], self.fq[i])
                       for j in range(k)] for i in range(k)])
        Q = 0.5 * a
        gp = np.array([self.fp[i] - sum(Q[i, j] * self.Pq[j] for j in range(k)) for i in range(k)])
        gq = np.array([self.fq[i] - sum(Q[i, j] * self.Pp[j] for j in range(k)) for i in range(k)])
        if self.trunc:
            self.GLp = np.array([self.op.l_gradient(x) for x in gp])
            self.GLq = np.array([self.op.l_gradient(x) for x in gq])
            res = np.sqrt(np.sum(self.GLp ** 2, axis=(1, 2)) + np.sum(self.GLq ** 2, axis=(1, 2)))
        else:
            res = np.array([np.sqrt(max(self.inner(gp[i], gp[i]) + self.inner(gq[i], gq[i]), 0.0))
                            for i in range(k)])
        omega = np.linalg.eigvalsh(0.5 * (Q + Q.T))
        self.step_tol = (min(0.1, max(self.precond_tol, float(np.max(res)))) if self.precond_adaptive
                         else self.precond_tol)
        return Q, omega, gp, gq, res

    def converged(self, omega, res, tol):
        if self.omega_prev is None:
            return False
        return bool(np.max(res) <= tol and np.max(np.abs(omega - self.omega_prev)) <= 0.1 * tol)

    # ---------------------------------------------------------------------------------------------
    def apply_preconditioner(self, g):
        """Approximate solution G of P^c H^chi G - G H^phi P^v = g (Eq. precond) by CG."""
        if self.precond == "none":
            return g.copy()
        if self.precond == "exact":
            return self.exact_preconditioner(g)
        G = np.zeros_like(g)
        r = g.copy()
        p = r.copy()
        rr = self.inner(r, r)
        r0 = np.sqrt(max(rr, 0.0))
        for _ in range(self.precond_maxit):
            if r0 == 0.0 or np.sqrt(max(rr, 0.0)) <= self.step_tol * r0:
                break
            Lp = self.op.ks_difference(p)
            pLp = self.inner(p, Lp)
            if pLp <= 0.0:
                break
            alpha = rr / pLp
            G = G + alpha * p
            r = r - alpha * Lp
            rr_new = self.inner(r, r)
            p = r + (rr_new / rr) * p
            rr = rr_new
            self.inner_iters += 1
        return G

    def exact_preconditioner(self, g):
        """The exact solution of Eq. precond for g in the conduction x valence subspace: with the
        Kohn-Sham states P^c H^chi d_c = eps_c d_c and H^phi P^v-side c_v, G = D_c X C_v^T turns
        P^c H^chi G - G H^phi P^v into D_c (eps_c X - X eps_v) C_v^T, so X = Y / (eps_c - eps_v)
        with Y = D_c^T S^chi g S^phi C_v the Kohn-Sham coordinates of g."""
        cas = self.casida
        Y = cas.to_ks(g)
        return cas.to_ngwf(Y / (cas.eps_c[:, None] - cas.eps_v[None, :]))

    def search_gradient(self, gp, gq):
        """The gradient the preconditioner acts on: g itself, or P^c G_L P^v with truncation."""
        op = self.op
        if self.trunc:
            # precondition the L-gradient: z = mask * Pinv(P^c G_L P^v), positive in Frobenius
            return (np.array([op.pc_x_pv(G) for G in self.GLp]),
                    np.array([op.pc_x_pv(G) for G in self.GLq]))
        return gp, gq

    def iterative_z(self, hp, hq):
        m = self.op.mask
        return (np.array([m * self.apply_preconditioner(x) for x in hp]),
                np.array([m * self.apply_preconditioner(x) for x in hq]))

    def samples(self):
        """Training rows of the learned preconditioner at the current iterate: inputs from the
        search gradient h, targets from the iterative preconditioner's z = mask * Pinv(h), and
        the row weights."""
        from .learned import Features
        Q, omega, gp, gq, res = self.evaluate()
        hp, hq = self.search_gradient(gp, gq)
        zp, zq = self.iterative_z(hp, hq)
        feat = Features(self.op.sys)
        X, s = feat.rows(hp, hq)
        return X, feat.targets(zp, zq, s, hp, hq), feat.weights(s, self.k)

    def gradient_when_not_descent(self):
        """Whether a non-descent preconditioned direction is replaced by the search gradient
        (no: the dense form's preconditioner is positive definite on the conduction x valence
        space, where its CG stays)."""
        return False

    def gdot(self, gp, gq, zp, zq, Zp, Zq):
        """sum_i <g_i, Z_i>: the slope of the sum functional along Z (z its L-space preimage, not
        needed here)."""
        return sum(self.inner(gp[i], Zp[i]) + self.inner(gq[i], Zq[i]) for i in range(self.k))

    def update(self, Q, omega, gp, gq):
        k = self.k
        op = self.op
        hp, hq = self.search_gradient(gp, gq)
        gz = 0.0
        if self.learned is not None:
            # learned map; the iterative preconditioner stands in when -z is not a descent
            # direction of the sum functional (<g, Z> <= 0)
            zp, zq = self.learned.apply(hp, hq)
            Zp = np.array([op.project(X) for X in zp])
            Zq = np.array([op.project(X) for X in zq])
            gz = self.gdot(gp, gq, zp, zq, Zp, Zq)
            if not gz > 0.0:
                self.fallbacks += 1
        if self.learned is None or not gz > 0.0:
            zp, zq = self.iterative_z(hp, hq)
            Zp = np.array([op.project(X) for X in zp])
            Zq = np.array([op.project(X) for X in zq])
            gz = self.gdot(gp, gq, zp, zq, Zp, Zq)
            if self.learned is None and not gz > 0.0 and self.gradient_when_not_descent():
                # the preconditioned direction does not descend: the step takes the search
                # gradient itself (the form's reading of Eq. precond, see TruncatedPCG)
                self.fallbacks += 1
                m = op.mask if self.trunc else 1.0
                zp, zq = m * hp, m * hq
                Zp = np.array([op.project(X) for X in zp])
                Zq = np.array([op.project(X) for X in zq])
                gz = self.gdot(gp, gq, zp, zq, Zp, Zq)
        restart = self.prev is None or self.it % self.restart_every == 0 or self.flipped
        beta = 0.0
        if not restart:
            pdir_p, pdir_q, pDp, pDq, pzp, pzq, pZp, pZq, pgz = self.prev
            gzp = self.gdot(gp, gq, pzp, pzq, pZp, pZq)
            beta = max(0.0, (gz - gzp) / pgz) if pgz != 0.0 else 0.0
        # descent directions: d = -z + beta d_prev (L space), Delta = its image in P space
        dir_p, dir_q, Dp, Dq = -zp, -zq, -Zp, -Zq
        if beta > 0.0:
            dir_p = dir_p + beta * pdir_p
            dir_q = dir_q + beta * pdir_q
            Dp = Dp + beta * pDp
            Dq = Dq + beta * pDq
            slope = self.gdot(gp, gq, dir_p, dir_q, Dp, Dq)
            if slope >= 0.0:
                beta = 0.0
                dir_p, dir_q, Dp, Dq = -zp, -zq, -Zp, -Zq
        fDp, fDq = op.apply(Dp, Dq, self.mode)
        # k x k blocks of the numerator and metric along the line
        def E(A, B, C, D):
            return np.array([[self.inner(A[i], C[j]) + self.inner(B[i], D[j])
                              for j in range(k)] for i in range(k)])
        N0 = E(self.Pp, self.Pq, self.fp, self.fq)
        Ef = E(Dp, Dq, self.fp, self.fq)
        N1 = Ef + Ef.T
        N2 = E(Dp, Dq, fDp, fDq)
        N0 = 0.5 * (N0 + N0.T)
        N2 = 0.5 * (N2 + N2.T)
        T0 = self.pq_products(self.Pp, self.Pq)
        T1 = self.pq_products(self.Pp, Dq) + self.pq_products(Dp, self.Pq)
        T2 = self.pq_products(Dp, Dq)
        M0, M1, M2 = (0.5 * (T + T.T) for T in (T0, T1, T2))
        lam = line_step(N0, N1, N2, M0, M1, M2)
        self.last_lambda = lam
        self.Yp += lam * dir_p
        self.Yq += lam * dir_q
        self.Pp += lam * Dp
        self.Pq += lam * Dq
        self.fp += lam * fDp
        self.fq += lam * fDq
        T = T0 + lam * T1 + lam * lam * T2
        order = list(np.argsort(np.diag(Q), kind="stable"))
        self.flipped = self.orthonormalize(T, order)
        self.it += 1
        if self.reapply_every > 0 and self.it % self.reapply_every == 0:
            # P afresh from the search variables (equal in exact arithmetic), then f = f(P)
            self.Pp = np.array([op.project(Y) for Y in self.Yp])
            self.Pq = np.array([op.project(Y) for Y in self.Yq])
            self.reapply()
        self.prev = (dir_p, dir_q, Dp, Dq, zp, zq, Zp, Zq, gz)
        self.omega_prev = omega
        return lam

    def step(self):
        """One PCG iteration; returns (omega, residual) of the iterate it started from."""
        Q, omega, gp, gq, res = self.evaluate()
        self.update(Q, omega, gp, gq)
        return omega, res

    def solve(self, tol=1e-6, max_iter=500):
        """Iterate to convergence; returns (omega ascending, residuals, iterations)."""
        for _ in range(max_iter):
            Q, omega, gp, gq, res = self.evaluate()
            if self.converged(omega, res, tol):
                return omega, res, self.it
            self.update(Q, omega, gp, gq)
        Q, omega, gp, gq, res = self.evaluate()
        return omega, res, self.it

    def pairing_errors(self):
        """Per Ritz pair of the converged subspace: |<p, f_p> - omega| and |<q, f_q> - omega|.
        At an eigenpair each half of the Tsiper numerator equals omega (and (-p, q) is the -omega
        partner)."""
        Q = 0.5 * np.array([[self.inner(self.Pp[j], self.fp[i]) + self.inner(self.Pq[j], self.fq[i])
                             for j in range(self.k)] for i in range(self.k)])
        om, U = np.linalg.eigh(0.5 * (Q + Q.T))
        out = []
        for a in range(self.k):
            p = np.einsum("i,irc->rc", U[:, a], self.Pp)
            q = np.einsum("i,irc->rc", U[:, a], self.Pq)
            fp = np.einsum("i,irc->rc", U[:, a], self.fp)
            fq = np.einsum("i,irc->rc", U[:, a], self.fq)
            out.append((abs(self.inner(p, fp) - om[a]), abs(self.inner(q, fq) - om[a])))
        return np.array(out)
