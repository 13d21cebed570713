"""Pins of the oracle MLP (12 -> 64 -> 64 -> 10, ReLU, MSE) and Adam.

* the backpropagated gradient equals central differences of the loss;
* a network whose weights make it the identity on its first 10 inputs
  (through ReLU on positive inputs) returns them exactly;
* Adam's first step moves every parameter by lr against the sign of its
  gradient (bias correction), and Adam minimises a quadratic;
* the BF16-operand form (the tensor-core network's arithmetic): its rounding
  equals the library's float -> bfloat16 conversion, closed forms on one path
  show each operand rounded where the form says (and the output bias not),
  and with BF16-exact operands it equals the exact form bit for bit.
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


# ----------------------------------------------- BF16-operand form (pins)
def _bf16_torch(x):
    """round to bfloat16 by the library's conversion (round to nearest even)"""
    import torch
    return torch.tensor(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def test_bf16_rounding_matches_library_conversion():
    """the oracle's rounding from the definition equals torch's float32 ->
    bfloat16 conversion on random values, exact ties (both directions of
    ties-to-even), powers of two and tiny values"""
    rng = np.random.default_rng(4)
    x = (rng.standard_normal(4000) * 10.0 ** rng.uniform(-30, 30, 4000)).astype(np.float32)
    ties = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 2 ** -20 * (1 + 5 * 2 ** -8),
                     1.0, 0.5, -2.0 ** 40, 1 + 2 ** -9, 1 + 2 ** -8 + 2 ** -20], np.float32)
    v = np.concatenate([x, ties]).astype(np.float64)
    assert np.array_equal(oracle.bf16_round(v), _bf16_torch(v))
    assert oracle.bf16_round(1 + 2 ** -8) == 1.0                      # tie to even (down)
    assert oracle.bf16_round(1 + 3 * 2 ** -8) == 1 + 2 ** -6          # tie to even (up)


def _path_params(w1=1.0, b1=0.0, w2=1.0, b2=0.0, w3=1.0, b3=0.0):
    """one path x0 -> h1_0 -> h2_0 -> y0 through the network"""
    p = np.zeros(oracle.MLP_NPARAM)
    p[OFF_W1], p[OFF_B1], p[OFF_W2], p[OFF_B2], p[OFF_W3], p[OFF_B3] = w1, b1, w2, b2, w3, b3
    return p


def test_bf16_forward_rounds_at_each_operand():
    """closed forms on one path: an input, a weight, a hidden activation
    after its bias and ReLU are rounded (1 + 2^-9 -> 1); the output bias is
    not (y keeps its 2^-9); the exact form keeps 1 + 2^-9 everywhere"""
    e = 2.0 ** -9
    cases = [(1.0 + e, dict(), 1.0),           # input rounded
             (1.0, dict(w1=1 + e), 1.0),        # weight rounded
             (1.0, dict(b1=e), 1.0),            # h1 rounded after its bias
             (1.0, dict(b2=e), 1.0),            # h2 rounded after its bias
             (1.0, dict(b3=e), 1.0 + e)]        # output bias: not rounded
    for x0, kw, want in cases:
        X = np.zeros((1, NI))
        X[0, 0] = x0
        p = _path_params(**kw)
        assert oracle.mlp_forward(p, X, bf16=True)[0, 0] == want, kw
        assert oracle.mlp_forward(p, X)[0, 0] == 1.0 + e, kw


def test_bf16_backward_rounds_each_gradient_operand():
    """one row, one path with weights 3 (so products leave BF16): dY, dH2 and
    dH1 are BF16-rounded, and each gradient is the exact product of its
    rounded operands (closed forms with the library's BF16 rounding)"""
    X = np.zeros((1, NI))
    X[0, 0] = 1.0
    p = _path_params(w1=1.0, w2=3.0, w3=3.0)
    y = 9.0                                   # h1 = 1, h2 = 3, y = 9 (all exact)
    T = np.zeros((1, NO))
    T[0, 0] = y - 0.5                         # e = 0.5, dY = 2 e / 10 = 0.1
    loss, g = oracle.mlp_loss_grad(p, X, T, bf16=True)
    r = lambda v: float(_bf16_torch([v])[0])
    dy = r(0.1)
    dh2 = r(3.0 * dy)
    dh1 = r(3.0 * dh2)
    assert loss == 0.25 / 10
    assert g[OFF_B3] == dy and g[OFF_W3] == dy * 3.0
    assert g[OFF_B2] == dh2 and g[OFF_W2] == dh2 * 1.0
    assert g[OFF_B1] == dh1 and g[OFF_W1] == dh1 * 1.0
    # the exact form differs at each of them
    _, ge = oracle.mlp_loss_grad(p, X, T)
    assert ge[OFF_B3] == 0.1 and ge[OFF_B3] != dy


def test_bf16_form_equals_exact_form_when_operands_are_bf16():
    """permutation-like network, BF16-exact inputs and a target that makes dY
    exact (rows 16: dY = 2 * 5 / 160 = 1/16): forward and gradient agree with
    the exact form bit for bit"""
    rng = np.random.default_rng(8)
    p = np.zeros(oracle.MLP_NPARAM)
    for i in range(NO):
        p[OFF_W1 + i * NI + i] = 1.0
        p[OFF_W2 + i * NH + i] = 2.0
        p[OFF_W3 + i * NH + i] = 0.5
    X = rng.integers(0, 9, (16, NI)) / 4.0
    Y = oracle.mlp_forward(p, X)
    assert np.array_equal(oracle.mlp_forward(p, X, bf16=True), Y)
    T = Y - 5.0
    le, ge = oracle.mlp_loss_grad(p, X, T)
    lq, gq = oracle.mlp_loss_grad(p, X, T, bf16=True)
    assert le == lq and np.array_equal(ge, gq)
