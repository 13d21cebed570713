"""Pins of the oracle MLP (12 -> 64 -> 64 -> 10, ReLU, MSE) and Adam.

* the backpropagated gradient equals central differences of the loss;
* a network whose weights make it the identity on its first 10 inputs
  (through ReLU on positive inputs) returns them exactly;
* Adam's first step moves every parameter by lr against the sign of its
  gradient (bias correction), and Adam minimises a quadratic.
"""
import numpy as np

import oracle

NI, NH, NO = 12, 64, 10
OFF_W1, OFF_B1 = 0, NH * NI
OFF_W2 = OFF_B1 + NH
OFF_B2 = OFF_W2 + NH * NH
OFF_W3 = OFF_B2 + NH
OFF_B3 = OFF_W3 + NO * NH


def rand_params(seed):
    rng = np.random.default_rng(seed)
    p = np.zeros(oracle.MLP_NPARAM)
    p[OFF_W1:OFF_B1] = rng.standard_normal(NH * NI) * np.sqrt(2.0 / NI)
    p[OFF_B1:OFF_W2] = rng.standard_normal(NH) * 0.1
    p[OFF_W2:OFF_B2] = rng.standard_normal(NH * NH) * np.sqrt(2.0 / NH)
    p[OFF_B2:OFF_W3] = rng.standard_normal(NH) * 0.1
    p[OFF_W3:OFF_B3] = rng.standard_normal(NO * NH) * np.sqrt(1.0 / NH)
    p[OFF_B3:] = rng.standard_normal(NO) * 0.1
    return p


def test_parameter_count():
    assert oracle.lib().or_mlp_nparam() == oracle.MLP_NPARAM == 5642


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    p = rand_params(1)
    X = rng.standard_normal((7, NI))
    T = rng.standard_normal((7, NO))
    loss, g = oracle.mlp_loss_grad(p, X, T)
    idx = np.concatenate([rng.choice(np.arange(s, e), min(12, e - s), replace=False)
                          for s, e in [(OFF_W1, OFF_B1), (OFF_B1, OFF_W2), (OFF_W2, OFF_B2),
                                       (OFF_B2, OFF_W3), (OFF_W3, OFF_B3), (OFF_B3, oracle.MLP_NPARAM)]])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle.mlp_loss_grad(pp, X, T)[0] - oracle.mlp_loss_grad(pm, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9, (i, fd, g[i])
    Y = oracle.mlp_forward(p, X)
    assert abs(loss - np.mean((Y - T) ** 2)) <= 1e-14 * loss


def test_identity_network():
    p = np.zeros(oracle.MLP_NPARAM)
    for i in range(NO):
        p[OFF_W1 + i * NI + i] = 1.0          # h1_i = relu(x_i)
        p[OFF_W2 + i * NH + i] = 1.0          # h2_i = relu(h1_i)
        p[OFF_W3 + i * NH + i] = 1.0          # y_i = h2_i
    X = np.abs(np.random.default_rng(3).standard_normal((5, NI)))
    assert np.array_equal(oracle.mlp_forward(p, X), X[:, :NO])


def test_adam_first_step_and_convergence():
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    m, v = np.zeros(3), np.zeros(3)
    p0 = p.copy()
    oracle.adam_step(p, g, m, v, 1, lr=0.01)
    assert np.allclose(p - p0, -0.01 * np.sign(g), rtol=1e-4)
    x, m, v = np.array([5.0]), np.zeros(1), np.zeros(1)
    for t in range(1, 3001):
        oracle.adam_step(x, 2.0 * (x - 1.5), m, v, t, lr=0.05)
    assert abs(x[0] - 1.5) < 1e-3
