"""Pins of the oracle's per-point MLP (the learned warm start): the gradient
against central finite differences, the forward pass against its layer-by-layer
definition on a case worked with numpy, and the loss at a known optimum."""
import numpy as np

from paper_1904_02108_gb300 import workload as W


def _params(orc, seed, scale=0.3):
    return scale * W.random_array(W.SplitMix64(seed), (orc.mlp_nparam(),))


def test_parameter_count(orc):
    assert orc.mlp_nparam() == 64 * 16 + 64 + 64 * 64 + 64 + 3 * 64 + 3 == 5443


def test_gradient_matches_central_differences(orc):
    P = _params(orc, 71)
    rng = W.SplitMix64(72)
    x = W.random_array(rng, (7, 16))
    t = W.random_array(rng, (7, 3))
    _, g = orc.mlp_loss_grad(P, x, t)
    h = 1e-6
    idx = list(range(0, len(P), 37)) + [len(P) - 1, len(P) - 3, 1024, 1024 + 63]
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (orc.mlp_loss_grad(Pp, x, t)[0] - orc.mlp_loss_grad(Pm, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_zero_weights_give_the_output_bias_and_zero_loss_at_it(orc):
    P = np.zeros(orc.mlp_nparam())
    P[-3:] = [0.5, -1.0, 2.0]
    x = W.random_array(W.SplitMix64(73), (4, 16))
    y = orc.mlp_forward(P, x)
    assert np.array_equal(y, np.tile([0.5, -1.0, 2.0], (4, 1)))
    loss, g = orc.mlp_loss_grad(P, x, y)
    assert loss == 0.0 and np.abs(g).max() == 0.0


def test_single_hidden_unit_path(orc):
    """Only W1[0,0] = a, W2[0,0] = b, W3[c,0] = 1: y_c = silu(b silu(a x0)),
    the SiLU s(v) = v / (1 + e^-v) written out by hand."""
    P = np.zeros(orc.mlp_nparam())
    a, b = 0.7, -1.3
    P[0] = a                         # W1[0][0]
    P[1024 + 64] = b                 # W2[0][0]
    w3 = 1024 + 64 + 4096 + 64
    P[w3 + 0 * 64] = P[w3 + 1 * 64] = P[w3 + 2 * 64] = 1.0  # W3[c][0]
    x = np.zeros((1, 16))
    x[0, 0] = 0.9
    s = lambda v: v / (1.0 + np.exp(-v))
    y = orc.mlp_forward(P, x)
    # hidden units 1..63 of layer 1 are s(0) = 0; layer-2 unit 0 sees b s(a x0)
    ref = s(b * s(a * 0.9))
    assert np.allclose(y, ref, rtol=0, atol=1e-15)
