"""Pins of the surrogate oracle (oracle/surrogate.py) against what mathematics
fixes independently of its own code: brute-force periodic convolution with
explicit index arithmetic, the response to a unit impulse, the adjoint
identity, central finite differences of the loss, the closed form of the first
Adam step, and translation equivariance on the periodic grid."""
import numpy as np
import pytest

from oracle import surrogate as S


def _brute_conv(x, W, b):
    n, ci, ny, nx = x.shape
    co = W.shape[2]
    out = np.zeros((n, co, ny, nx))
    for q in range(n):
        for o in range(co):
            for y in range(ny):
                for xx in range(nx):
                    acc = b[o]
                    for ky in range(3):
                        for kx in range(3):
                            for c in range(ci):
                                acc += W[ky, kx, o, c] * x[q, c, (y + ky - 1) % ny, (xx + kx - 1) % nx]
                    out[q, o, y, xx] = acc
    return out


def test_conv_matches_brute_force_periodic_loops():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 5, 7))
    W = rng.standard_normal((3, 3, 4, 3))
    b = rng.standard_normal(4)
    assert np.allclose(S.conv3x3(x, W, b), _brute_conv(x, W, b), rtol=0, atol=1e-12)


def test_conv_of_unit_impulse_is_the_flipped_kernel():
    # a delta at (y0, x0) reaches output (y0 - ky + 1, x0 - kx + 1) with weight W[ky, kx]
    W = np.arange(9.0).reshape(3, 3, 1, 1) + 1.0
    x = np.zeros((1, 1, 6, 6))
    x[0, 0, 0, 0] = 1.0              # a corner: every tap wraps around somewhere
    out = S.conv3x3(x, W, np.zeros(1))[0, 0]
    for ky in range(3):
        for kx in range(3):
            assert out[(0 - ky + 1) % 6, (0 - kx + 1) % 6] == W[ky, kx, 0, 0]
    assert np.count_nonzero(out) == 9


def test_adjoint_identity():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 3, 6, 5))
    g = rng.standard_normal((2, 4, 6, 5))
    W = rng.standard_normal((3, 3, 4, 3))
    lhs = np.sum(S.conv3x3(x, W, np.zeros(4)) * g)
    rhs = np.sum(x * S.conv3x3_adjoint(g, W))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    # weight gradient: d<conv(x, W), g>/dW
    dW = S.conv3x3_wgrad(g, x)
    E = rng.standard_normal(W.shape)
    assert abs(np.sum(dW * E) - np.sum(S.conv3x3(x, E, np.zeros(4)) * g)) < 1e-10 * abs(lhs) * 10


def test_silu_and_its_derivative():
    z = np.linspace(-8, 8, 101)
    h = 1e-6
    fd = (S.silu(z + h) - S.silu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - S.dsilu(z))) < 1e-8
    assert S.silu(np.array([0.0]))[0] == 0.0
    assert abs(S.silu(np.array([40.0]))[0] - 40.0) < 1e-12


def _tiny_problem(width=4, depth=3, seed=3):
    rng = np.random.default_rng(seed)
    _, real = S.layer_shapes(width, depth)
    layers = [(rng.standard_normal((3, 3, ro, ri)) * 0.4, rng.standard_normal(ro) * 0.1) for ri, ro in real]
    p = S.pack(layers, width, depth)
    X = rng.standard_normal((2, 3, 5, 6))
    Y = X + 0.3 * rng.standard_normal(X.shape)
    return p, X, Y, rng


def test_pack_unpack_round_trip_and_padding_is_zero():
    p, _, _, _ = _tiny_problem()
    assert p.size == S.n_params(4, 3)
    q = S.pack(S.unpack(p, 4, 3), 4, 3)
    assert np.array_equal(p, q)


def test_loss_gradient_matches_central_differences():
    width, depth = 4, 3
    p, X, Y, rng = _tiny_problem(width, depth)
    si, so = [1.5, 0.7, 1.1], [0.5, 2.0, 1.3]
    L, g = S.loss_grad(p, X, Y, si, so, width, depth)
    assert abs(L - S.loss(p, X, Y, si, so, width, depth)) < 1e-14 * max(1.0, L)
    # every real parameter of the first and last layers, a sample of the rest
    stored, real = S.layer_shapes(width, depth)
    mask = S.pack([(np.ones((3, 3, ro, ri)), np.ones(ro)) for ri, ro in real], width, depth) > 0
    idx = np.flatnonzero(mask)
    assert np.all(g[~mask] == 0.0)        # padding receives no gradient
    pick = rng.choice(idx, size=80, replace=False)
    h = 1e-6
    for i in pick:
        e = np.zeros_like(p)
        e[i] = h
        fd = (S.loss(p + e, X, Y, si, so, width, depth) - S.loss(p - e, X, Y, si, so, width, depth)) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1e-3, abs(fd)) + 1e-9, (i, fd, g[i])


def test_first_adam_step_is_the_signed_learning_rate():
    # m_hat = g and v_hat = g^2 after one step: p - lr g / (|g| + eps)
    rng = np.random.default_rng(4)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    lr = 1e-3
    p1, m, v = S.adam(p, g, np.zeros(50), np.zeros(50), 1, lr)
    assert np.allclose(p1, p - lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_network_is_translation_equivariant_on_the_periodic_grid():
    p, X, _, _ = _tiny_problem()
    a = S.apply(p, X, [1, 1, 1], [1, 1, 1], 4, 3)
    b = S.apply(p, np.roll(X, (2, -3), axis=(2, 3)), [1, 1, 1], [1, 1, 1], 4, 3)
    assert np.allclose(np.roll(a, (2, -3), axis=(2, 3)), b, rtol=0, atol=1e-12)


def test_zero_network_is_the_identity_map():
    p = np.zeros(S.n_params(4, 3))
    _, X, _, _ = _tiny_problem()
    assert np.array_equal(S.apply(p, X, [2, 2, 2], [3, 3, 3], 4, 3), X)
