"""Pins of the oracle of the learned preconditioner correction (oracle/mlp.py):
back-propagated gradients against central differences of the loss, the
network's closed forms, Adam's first step and the features' definitions."""
import numpy as np

from oracle import mlp as M
from paper_2605_28637_gb300 import synthetic as syn


def rand_params(seed, scale=0.5):
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, M.NPARAM)


def test_param_count_matches_layout():
    assert M.NPARAM == syn.MLP_NPARAM == 4481
    W1, b1, W2, b2, w3, b3 = M.unpack(np.arange(M.NPARAM, dtype=float))
    assert W1.shape == (64, 3) and W2.shape == (64, 64) and w3.shape == (64,)
    assert W1[0, 0] == 0 and b1[0] == 192 and W2[0, 0] == 256 and b2[0] == 4352 and w3[0] == 4416
    assert b3 == 4480


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    U = rng.normal(size=(40, 3))
    t = rng.normal(size=40)
    w = rng.uniform(0.1, 2.0, 40)
    p = rand_params(2)
    _, g = M.loss_and_grad(p, U, t, w)
    idx = np.concatenate([rng.choice(M.NPARAM, 200, replace=False), [M.NPARAM - 1, 0, 192, 4352, 4416]])
    h = 1e-6
    for i in idx:
        e = np.zeros(M.NPARAM); e[i] = h
        fd = (M.loss_and_grad(p + e, U, t, w)[0] - M.loss_and_grad(p - e, U, t, w)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-7 + 1e-6 * abs(fd), (i, fd, g[i])


def test_zero_weights_give_the_output_bias():
    p = np.zeros(M.NPARAM)
    p[-1] = 0.7
    U = np.random.default_rng(3).normal(size=(5, 3))
    s, h1, h2 = M.forward(p, U)
    assert np.allclose(s, 0.7) and np.all(h1 == 0) and np.all(h2 == 0)
    assert np.allclose(M.multiplier(p, U), np.exp(0.7))
    p[-1] = 10.0
    assert np.allclose(M.multiplier(p, U), np.exp(3.0))   # clipped


def test_single_path_is_nested_tanh():
    """Only W1[0, 1], W2[0, 0] and w3[0] nonzero: s = c tanh(b tanh(a u1))."""
    p = np.zeros(M.NPARAM)
    a, b, c = 0.8, -1.3, 2.1
    p[1] = a
    p[256] = b
    p[4416] = c
    U = np.array([[9.0, 0.4, -2.0], [1.0, -1.5, 3.0]])
    s, _, _ = M.forward(p, U)
    assert np.allclose(s, c * np.tanh(b * np.tanh(a * U[:, 1])), atol=1e-15)


def test_adam_first_step_closed_form():
    """Step 1: the bias-corrected moments are g and g^2, so the update is
    lr g / (|g| + eps)."""
    rng = np.random.default_rng(4)
    p = rng.normal(size=10)
    g = rng.normal(size=10)
    pn, m, v = M.adam_step(p, g, np.zeros(10), np.zeros(10), 1, lr=0.01)
    assert np.allclose(pn, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_features_definitions():
    """Two bands, three coefficients: kinetic energy of the residual, rms and
    the log1p transforms by hand."""
    g2h = np.array([0.0, 1.0, 4.0])
    g = np.array([[1.0, 0.0], [1j, 2.0], [0.0, 2.0j]])
    eps = np.array([-0.5, 0.25])
    U = M.features(g, g2h, eps).reshape(2, 3, 3)
    T0 = (0 * 1 + 1 * 1) / 2.0
    T1 = (1 * 4 + 4 * 4) / 8.0
    rms0, rms1 = np.sqrt(2.0 / 3.0), np.sqrt(8.0 / 3.0)
    assert np.allclose(U[0, :, 0], np.log1p(g2h / T0))
    assert np.allclose(U[1, :, 0], np.log1p(g2h / T1))
    assert np.allclose(U[0, :, 1], np.log1p(np.array([1.0, 1.0, 0.0]) / rms0))
    assert np.allclose(U[1, :, 1], np.log1p(np.array([0.0, 2.0, 2.0]) / rms1))
    assert np.all(U[0, :, 2] == -0.5) and np.all(U[1, :, 2] == 0.25)


def test_initial_params_are_identity_correction():
    p = syn.mlp_initial_params(0).astype(np.float64)
    U = np.random.default_rng(5).normal(size=(7, 3))
    assert np.all(M.multiplier(p, U) == 1.0)
