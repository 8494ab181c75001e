"""Pins of the learned-preconditioner oracle (oracle/learned.py) against things other than itself:
central finite differences for the backward pass, scalar loops for the forward pass, the closed
form of Adam's first step, torch's bfloat16 conversion for the rounding, the exact round trip of
the block features, homogeneity of the map, and the dense eigenvalues for the learned PCG."""
import numpy as np
import pytest

from oracle import learned, solver
from paper_1507_08157_gb300 import synthetic as sy


def _tiny_net(seed, n_in=5, w=7, n_out=3, n=6):
    rng = np.random.default_rng(seed)
    dims = (n_in, w, n_out)
    theta = rng.normal(size=learned.n_params(*dims))
    X = rng.normal(size=(n, n_in))
    T = rng.normal(size=(n, n_out))
    return dims, theta, X, T


def test_gradient_matches_central_differences():
    dims, theta, X, T = _tiny_net(1)
    L, g = learned.loss_grad(theta, dims, X, T)
    h = 1e-6
    fd = np.empty_like(theta)
    for p in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        fd[p] = (learned.loss_grad(tp, dims, X, T)[0] - learned.loss_grad(tm, dims, X, T)[0]) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-7 * np.max(np.abs(g))
    # a dropped term (say the b1 gradient) would show up here
    assert np.all(np.abs(g) < 1e3) and np.count_nonzero(g) > 0.5 * g.size


def test_forward_equals_scalar_loops():
    dims, theta, X, _ = _tiny_net(2, n=3)
    n_in, w, n_out = dims
    W1, b1, W2, b2, W3, b3 = learned.unpack(theta, *dims)
    Y, _, _ = learned.forward(theta, dims, X)
    for r in range(X.shape[0]):
        h1 = [max(0.0, b1[j] + sum(X[r, i] * W1[i, j] for i in range(n_in))) for j in range(w)]
        h2 = [max(0.0, b2[j] + sum(h1[i] * W2[i, j] for i in range(w))) for j in range(w)]
        y = [b3[j] + sum(h2[i] * W3[i, j] for i in range(w)) for j in range(n_out)]
        assert np.allclose(Y[r], y, rtol=1e-13, atol=1e-13)


def test_adam_constant_gradient_steps_are_sign_steps():
    rng = np.random.default_rng(3)
    theta = rng.normal(size=11)
    g = rng.normal(size=11)
    m = np.zeros(11)
    v = np.zeros(11)
    lr = 1e-3
    th = theta
    for t in (1, 2, 3):
        new, m, v = learned.adam_step(th, g, m, v, t, lr)
        # bias correction makes m_hat = g and v_hat = g^2 for a constant gradient
        assert np.allclose(th - new, lr * g / (np.abs(g) + learned.ADAM_EPS), rtol=1e-12, atol=0)
        th = new


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.normal(size=2000).astype(np.float32),
                        np.float32([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -1.0 - 2 ** -8, 0.0, 1e-30, 3e38])])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(learned.round_bf16(x), ref)
    assert learned.round_bf16(np.float32([1.0 + 2 ** -8]))[0] == 1.0          # tie -> even


def test_features_round_trip_and_fixed_parts(tiny_system):
    s = tiny_system
    feat = learned.Features(s)
    nc, nv, na = learned.block_dims(s)
    n_in, n_out = learned.io_sizes(s)
    hp, hq = sy.random_kernels(s, 2, 9)
    X, sc = feat.rows(hp, hq)
    assert X.shape == (2 * na * na, n_in)
    zp, zq = feat.scatter(X[:, :n_out], sc, 2)
    assert np.allclose(zp, hp, rtol=1e-14, atol=1e-14) and np.allclose(zq, hq, rtol=1e-14, atol=1e-14)
    # one block by hand: state 1, chi-atom 2, phi-atom 0
    q = (1 * na + 2) * na + 0
    bp = hp[1, 2 * nc:3 * nc, 0:nv].ravel()
    bq = hq[1, 2 * nc:3 * nc, 0:nv].ravel()
    assert np.isclose(sc[q], np.sqrt(bp @ bp + bq @ bq))
    Sc_blk = X[q, n_out + nc * nc:n_out + 2 * nc * nc].reshape(nc, nc)
    assert np.allclose(Sc_blk, s.S_chi[2 * nc:3 * nc, 2 * nc:3 * nc])
    d = X[:, -1].reshape(2, na, na)[0]
    assert np.allclose(np.diag(d), 0.0) and np.allclose(d, d.T)
    T = feat.targets(hp, hq, sc)
    assert np.allclose(T, X[:, :n_out])


def test_learned_map_is_homogeneous(tiny_system, tiny_operator):
    s = tiny_system
    n_in, n_out = learned.io_sizes(s)
    theta = sy.mlp_init(n_in, 16, n_out, 5)
    P = learned.LearnedPreconditioner(s, theta, 16, tiny_operator.mask)
    hp, hq = sy.random_kernels(s, 2, 10)
    zp, zq = P.apply(hp, hq)
    zp3, zq3 = P.apply(3.0 * hp, 3.0 * hq)
    assert np.allclose(zp3, 3.0 * zp, rtol=1e-12, atol=1e-14)
    assert np.allclose(zq3, 3.0 * zq, rtol=1e-12, atol=1e-14)


@pytest.mark.slow
def test_learned_pcg_reaches_dense_eigenvalues(tiny_system, tiny_operator, tiny_casida):
    s = tiny_system
    n_in, n_out = learned.io_sizes(s)
    theta = sy.mlp_init(n_in, 16, n_out, 6)          # untrained: the fixed point must not move
    pcg = solver.PCG(tiny_operator, sy.initial_guess(s, 2, 1), precond="learned", mlp=(theta, 16))
    omega, res, it = pcg.solve(tol=1e-7, max_iter=400)
    ref = tiny_casida.omega_symmetric()[:2]
    assert np.max(np.abs(np.sort(omega) - ref)) < 1e-6
