"""Learned atom-block preconditioner (FP64 reference): block features, the 3-layer perceptron,
its mean-squared loss and gradient, one Adam step, and the preconditioner map h -> z.

TEST INFRASTRUCTURE ONLY (see the package docstring): only tests/, the smoke check and the
CPU-baseline leg of the benchmark may import this module.

The paper's preconditioner (Sec. III B, Eq. precond) is the approximate solution z of
P^c H^chi z - z H^phi P^v = h for a gradient h, obtained by an inner CG. Its learned stand-in
maps each atom block of h to the same block of z with a linear map that a small network predicts
from the block's fixed features, so the preconditioner stays linear in h (as the CG solve is):

* Samples. For state i, chi-atom I and phi-atom J (functions grouped by atom, n_c chi and n_v phi
  per atom) the block h^p_IJ = h^p_i[I n_c : (I+1) n_c, J n_v : (J+1) n_v] and h^q_IJ likewise.
  With s = sqrt(|h^p_IJ|^2 + |h^q_IJ|^2) (Frobenius) the input row is
      x = [h^p_IJ / s, h^q_IJ / s, M^c_II, S^chi_II, M^v_JJ, S^phi_JJ, d_IJ / 10]
  (blocks flattened row-major; M^c = P^c H^chi, M^v = H^phi P^v, the two matrices of Eq.
  precond; d_IJ the minimum-image distance of the two atoms in bohr): the block part b of
  n_b = 2 n_c n_v entries, then the feature part f of n_f = 2 n_c^2 + 2 n_v^2 + 1. The model
  learns the correction to the identity map: the target row is
  y = [(z^p_IJ - h^p_IJ) / s, (z^q_IJ - h^q_IJ) / s] (n_b entries)
  and the row weight is w = s^2 / (sum of s^2 over the rows of the same state), the share of the
  state's gradient norm that the block carries. A block with s = 0 has a zero h part, zero
  weight, and its z block is zero. Rows are ordered (i, I, J) with J fastest.
* Model. A 3-layer perceptron maps the features to an n_b x n_b matrix,
  vec(A) = W3^T relu(W2^T relu(W1^T f + b1) + b2) + b3 (row form H1 = relu(F W1 + b1),
  H2 = relu(H1 W2 + b2), vec(A) = H2 W3 + b3, W1 [n_f][w], W2 [w][w], W3 [w][n_b^2], A row-major),
  and the output row is y = A b. The parameter vector is W1, b1, W2, b2, W3, b3, each row-major,
  concatenated.
* Loss. L = sum_r w_r sum_j (y_rj - T_rj)^2 / (n n_b) over the n rows (w = 1 without
  weights), i.e. the weighted squared error of the z blocks themselves.
* Adam (Kingma & Ba 2015): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
  theta -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), b1 = 0.9, b2 = 0.999, eps = 1e-8.
* Inference uses the parameters rounded to bfloat16 (round to nearest, ties to even).
* The map: z_IJ = h_IJ + A_IJ h_IJ (blocks as vectors; s cancels), then the kernel mask as for
  the iterative preconditioner. It is linear in h; an untrained network with small output is
  close to the identity (no preconditioner).
"""
import numpy as np

ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def block_dims(sys):
    """(n_c, n_v, natoms): functions per atom in chi and phi; atoms must carry equal counts."""
    na = sys.pos.shape[0]
    nc_tot, nv_tot = sys.chi.nfun, sys.phi.nfun
    if nc_tot % na or nv_tot % na:
        raise ValueError("the learned preconditioner needs equal function counts on every atom")
    nc, nv = nc_tot // na, nv_tot // na
    if not (np.array_equal(sys.chi.atom, np.repeat(np.arange(na), nc))
            and np.array_equal(sys.phi.atom, np.repeat(np.arange(na), nv))):
        raise ValueError("functions must be grouped by atom")
    return nc, nv, na


def io_sizes(sys):
    """(n_b, n_f): lengths of the block part and the feature part of a row."""
    nc, nv, _ = block_dims(sys)
    return 2 * nc * nv, 2 * nc * nc + 2 * nv * nv + 1


def atom_distances(sys):
    d = sys.pos[:, None, :] - sys.pos[None, :, :]
    d -= sys.cell * np.round(d / sys.cell)
    return np.sqrt(np.sum(d * d, axis=-1))


class Features:
    """The fixed (per-system) parts of the input rows."""

    def __init__(self, sys):
        self.nc, self.nv, self.na = block_dims(sys)
        nc, nv, na = self.nc, self.nv, self.na
        Mc = sys.P_c @ sys.H_chi
        Mv = sys.H_phi @ sys.P_v
        self.fc = np.array([np.concatenate([Mc[I * nc:(I + 1) * nc, I * nc:(I + 1) * nc].ravel(),
                                            sys.S_chi[I * nc:(I + 1) * nc, I * nc:(I + 1) * nc].ravel()])
                            for I in range(na)])
        self.fv = np.array([np.concatenate([Mv[J * nv:(J + 1) * nv, J * nv:(J + 1) * nv].ravel(),
                                            sys.S_phi[J * nv:(J + 1) * nv, J * nv:(J + 1) * nv].ravel()])
                            for J in range(na)])
        self.d = atom_distances(sys) / 10.0

    def rows(self, hp, hq):
        """Input rows X [k na na][n_in] and block scales s [k na na] of the gradients hp, hq
        ([k][N_chi][N_phi]), written out block by block."""
        nc, nv, na = self.nc, self.nv, self.na
        k = hp.shape[0]
        X, s = [], []
        for i in range(k):
            for I in range(na):
                for J in range(na):
                    bp = hp[i, I * nc:(I + 1) * nc, J * nv:(J + 1) * nv].ravel()
                    bq = hq[i, I * nc:(I + 1) * nc, J * nv:(J + 1) * nv].ravel()
                    sc = float(np.sqrt(np.sum(bp * bp) + np.sum(bq * bq)))
                    inv = 1.0 / sc if sc > 0.0 else 0.0
                    X.append(np.concatenate([bp * inv, bq * inv, self.fc[I], self.fv[J], [self.d[I, J]]]))
                    s.append(sc)
        return np.array(X), np.array(s)

    def targets(self, zp, zq, s, hp, hq):
        """Target rows T [k na na][n_out]: (z - h) blocks divided by the scales of the h blocks."""
        nc, nv, na = self.nc, self.nv, self.na
        k = zp.shape[0]
        T = []
        q = 0
        for i in range(k):
            for I in range(na):
                for J in range(na):
                    inv = 1.0 / s[q] if s[q] > 0.0 else 0.0
                    rows, cols = slice(I * nc, (I + 1) * nc), slice(J * nv, (J + 1) * nv)
                    T.append(np.concatenate([(zp[i, rows, cols] - hp[i, rows, cols]).ravel() * inv,
                                             (zq[i, rows, cols] - hq[i, rows, cols]).ravel() * inv]))
                    q += 1
        return np.array(T)

    def weights(self, s, k):
        """Row weights s^2 / (sum of s^2 over the rows of the same state)."""
        s2 = np.asarray(s, dtype=np.float64).reshape(k, -1) ** 2
        tot = s2.sum(axis=1, keepdims=True)
        return np.where(tot > 0.0, s2 / np.where(tot > 0.0, tot, 1.0), 0.0).ravel()

    def scatter(self, Y, s, hp, hq):
        """z^p, z^q [k][N_chi][N_phi] = h + s * Y block by block."""
        nc, nv, na = self.nc, self.nv, self.na
        k = hp.shape[0]
        zp = np.zeros_like(hp)
        zq = np.zeros_like(hq)
        q = 0
        for i in range(k):
            for I in range(na):
                for J in range(na):
                    y = Y[q] * s[q]
                    rows, cols = slice(I * nc, (I + 1) * nc), slice(J * nv, (J + 1) * nv)
                    zp[i, rows, cols] = hp[i, rows, cols] + y[:nc * nv].reshape(nc, nv)
                    zq[i, rows, cols] = hq[i, rows, cols] + y[nc * nv:].reshape(nc, nv)
                    q += 1
        return zp, zq


# ---- the network ---------------------------------------------------------------------------------
def n_params(n_in, w, n_out):
    return n_in * w + w + w * w + w + w * n_out + n_out


def unpack(theta, n_in, w, n_out):
    sizes = [(n_in, w), (w,), (w, w), (w,), (w, n_out), (n_out,)]
    out, o = [], 0
    for sh in sizes:
        m = int(np.prod(sh))
        out.append(np.asarray(theta[o:o + m], dtype=np.float64).reshape(sh))
        o += m
    return out


def mlp_dims(n_b, n_f, width):
    """(inputs, width, outputs) of the perceptron inside the model."""
    return n_f, width, n_b * n_b


def mlp(theta, dims, F):
    """vec(A) rows of the perceptron for feature rows F, and its hidden activations."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, *dims)
    H1 = np.maximum(F @ W1 + b1, 0.0)
    H2 = np.maximum(H1 @ W2 + b2, 0.0)
    return H2 @ W3 + b3, H1, H2


def forward(theta, n_b, width, X):
    """Model output rows y = A(f) b for rows X = [b, f]; also A and the hidden activations."""
    n_f = X.shape[1] - n_b
    A, H1, H2 = mlp(theta, mlp_dims(n_b, n_f, width), X[:, n_b:])
    Am = A.reshape(-1, n_b, n_b)
    return np.einsum("rij,rj->ri", Am, X[:, :n_b]), Am, H1, H2


def loss_grad(theta, n_b, width, X, T, w=None):
    """Weighted mean-squared loss and its gradient with respect to the parameter vector
    (through y = A b, then backpropagation through the three layers; relu'(0) = 0).
    w: row weights (None = 1)."""
    n_f = X.shape[1] - n_b
    dims = mlp_dims(n_b, n_f, width)
    W1, b1, W2, b2, W3, b3 = unpack(theta, *dims)
    Yb, Am, H1, H2 = forward(theta, n_b, width, X)
    n = Yb.shape[0]
    R = Yb - T
    wr = np.ones(n) if w is None else np.asarray(w, dtype=np.float64)
    L = float(np.sum(wr[:, None] * R * R) / (n * n_b))
    dYb = 2.0 * wr[:, None] * R / (n * n_b)
    dY = (dYb[:, :, None] * X[:, None, :n_b]).reshape(n, n_b * n_b)     # d vec(A)
    gW3 = H2.T @ dY
    gb3 = dY.sum(axis=0)
    dH2 = (dY @ W3.T) * (H2 > 0.0)
    gW2 = H1.T @ dH2
    gb2 = dH2.sum(axis=0)
    dH1 = (dH2 @ W2.T) * (H1 > 0.0)
    gW1 = X[:, n_b:].T @ dH1
    gb1 = dH1.sum(axis=0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return L, g


def adam_step(theta, g, m, v, t, lr):
    """One Adam update (step number t >= 1); returns new (theta, m, v)."""
    m = ADAM_B1 * m + (1.0 - ADAM_B1) * g
    v = ADAM_B2 * v + (1.0 - ADAM_B2) * g * g
    mh = m / (1.0 - ADAM_B1 ** t)
    vh = v / (1.0 - ADAM_B2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v


def round_bf16(x):
    """float32 values rounded to the nearest bfloat16 (ties to even), returned as float64."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


class LearnedPreconditioner:
    """z = mask * (h + A h) block by block (inference with bfloat16-rounded parameters)."""

    def __init__(self, sys, theta, width, mask):
        self.feat = Features(sys)
        self.n_b, n_f = io_sizes(sys)
        self.width = width
        if len(theta) != n_params(*mlp_dims(self.n_b, n_f, width)):
            raise ValueError("parameter vector has the wrong length")
        self.theta = round_bf16(theta)
        self.mask = mask

    def apply(self, hp, hq):
        X, s = self.feat.rows(hp, hq)
        Y, _, _, _ = forward(self.theta, self.n_b, self.width, X)
        zp, zq = self.feat.scatter(Y, s, hp, hq)
        return zp * self.mask, zq * self.mask
