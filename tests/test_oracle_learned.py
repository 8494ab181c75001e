"""Pins of the learned-preconditioner oracle (oracle/learned.py) against things other than itself:
central finite differences for the backward pass, scalar loops for the forward pass, the closed
form of Adam's first step, torch's bfloat16 conversion for the rounding, the exact round trip of
the block features, homogeneity of the map, and the dense eigenvalues for the learned PCG."""
import numpy as np
import pytest

from oracle import learned, solver
from paper_1507_08157_gb300 import synthetic as sy


def _tiny_net(seed, n_b=3, n_f=4, w=7, n=6):
    rng = np.random.default_rng(seed)
    theta = rng.normal(size=learned.n_params(*learned.mlp_dims(n_b, n_f, w)))
    X = rng.normal(size=(n, n_b + n_f))
    T = rng.normal(size=(n, n_b))
    return (n_b, n_f, w), theta, X, T


@pytest.mark.parametrize("weighted", [False, True])
def test_gradient_matches_central_differences(weighted):
    (n_b, n_f, w), theta, X, T = _tiny_net(1)
    rw = np.random.default_rng(11).uniform(0.1, 2.0, size=X.shape[0]) if weighted else None
    L, g = learned.loss_grad(theta, n_b, w, X, T, rw)
    h = 1e-6
    fd = np.empty_like(theta)
    for p in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        fd[p] = (learned.loss_grad(tp, n_b, w, X, T, rw)[0] - learned.loss_grad(tm, n_b, w, X, T, rw)[0]) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-7 * np.max(np.abs(g))
    # a dropped term (say the b1 gradient) would show up here
    assert np.all(np.abs(g) < 1e4) and np.count_nonzero(g) > 0.5 * g.size


def test_forward_equals_scalar_loops():
    (n_b, n_f, w), theta, X, _ = _tiny_net(2, n=3)
    W1, b1, W2, b2, W3, b3 = learned.unpack(theta, *learned.mlp_dims(n_b, n_f, w))
    Y, _, _, _ = learned.forward(theta, n_b, w, X)
    for r in range(X.shape[0]):
        f = X[r, n_b:]
        h1 = [max(0.0, b1[j] + sum(f[i] * W1[i, j] for i in range(n_f))) for j in range(w)]
        h2 = [max(0.0, b2[j] + sum(h1[i] * W2[i, j] for i in range(w))) for j in range(w)]
        a = [b3[j] + sum(h2[i] * W3[i, j] for i in range(w)) for j in range(n_b * n_b)]
        y = [sum(a[i * n_b + j] * X[r, j] for j in range(n_b)) for i in range(n_b)]
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
    n_out, n_f = learned.io_sizes(s)
    n_in = n_out + n_f
    hp, hq = sy.random_kernels(s, 2, 9)
    X, sc = feat.rows(hp, hq)
    assert X.shape == (2 * na * na, n_in)
    # z = h + s * (h / s) = 2 h block by block
    zp, zq = feat.scatter(X[:, :n_out], sc, hp, hq)
    assert np.allclose(zp, 2 * hp, rtol=1e-14, atol=1e-14) and np.allclose(zq, 2 * hq, rtol=1e-14, atol=1e-14)
    # one block by hand: state 1, chi-atom 2, phi-atom 0
    q = (1 * na + 2) * na + 0
    bp = hp[1, 2 * nc:3 * nc, 0:nv].ravel()
    bq = hq[1, 2 * nc:3 * nc, 0:nv].ravel()
    assert np.isclose(sc[q], np.sqrt(bp @ bp + bq @ bq))
    Sc_blk = X[q, n_out + nc * nc:n_out + 2 * nc * nc].reshape(nc, nc)
    assert np.allclose(Sc_blk, s.S_chi[2 * nc:3 * nc, 2 * nc:3 * nc])
    d = X[:, -1].reshape(2, na, na)[0]
    assert np.allclose(np.diag(d), 0.0) and np.allclose(d, d.T)
    T = feat.targets(2 * hp, 2 * hq, sc, hp, hq)
    assert np.allclose(T, X[:, :n_out])
    w = feat.weights(sc, 2)
    assert np.allclose(w.reshape(2, -1).sum(axis=1), 1.0)
    assert np.isclose(w[q], sc[q] ** 2 / np.sum(sc[na * na:] ** 2))


def test_learned_map_is_linear(tiny_system, tiny_operator):
    s = tiny_system
    n_b, n_f = learned.io_sizes(s)
    theta = sy.mlp_init(n_f, 16, n_b * n_b, 5)
    P = learned.LearnedPreconditioner(s, theta, 16, tiny_operator.mask)
    hp, hq = sy.random_kernels(s, 2, 10)
    gp, gq = sy.random_kernels(s, 2, 11)
    zp, zq = P.apply(hp, hq)
    yp, yq = P.apply(gp, gq)
    wp, wq = P.apply(3.0 * hp - 2.0 * gp, 3.0 * hq - 2.0 * gq)
    assert np.allclose(wp, 3.0 * zp - 2.0 * yp, rtol=1e-10, atol=1e-12)
    assert np.allclose(wq, 3.0 * zq - 2.0 * yq, rtol=1e-10, atol=1e-12)


@pytest.mark.slow
def test_learned_pcg_reaches_dense_eigenvalues(tiny_system, tiny_operator, tiny_casida):
    s = tiny_system
    n_b, n_f = learned.io_sizes(s)
    theta = sy.mlp_init(n_f, 16, n_b * n_b, 6)       # untrained: the fixed point must not move
    pcg = solver.PCG(tiny_operator, sy.initial_guess(s, 2, 1), precond="learned", mlp=(theta, 16))
    omega, res, it = pcg.solve(tol=1e-7, max_iter=400)
    ref = tiny_casida.omega_symmetric()[:2]
    assert np.max(np.abs(np.sort(omega) - ref)) < 1e-6
