"""Pins of the oracle's closure network (three 3x3x3 valid convolutions,
3 -> H -> H -> 1 channels, ReLU between): an identity network copies its
input, a ReLU-inactive network equals three cross-correlations computed
independently (scipy.ndimage), and the loss gradient matches central
differences."""
import numpy as np
import pytest

H = 16


def split_params(p, h=H):
    i = 0
    out = []
    for shape in ((h, 3, 27), (h,), (h, h, 27), (h,), (1, h, 27), (1,)):
        n = int(np.prod(shape))
        out.append(p[i:i + n].reshape(shape))
        i += n
    return out


def test_parameter_count(O):
    assert O.closure_num_params(16) == 16 * 3 * 27 + 16 + 16 * 16 * 27 + 16 + 16 * 27 + 1 == 8673


def test_identity_network_copies_channel(O):
    """Unit 0 = relu(u), unit 1 = relu(-u) at the centre tap; layer 2 copies
    them; layer 3 returns unit0 - unit1 = u: out[z] = in[0][z + 3]."""
    p = np.zeros(O.closure_num_params(H))
    W1, b1, W2, b2, W3, b3 = split_params(p)
    c = 13  # centre tap (1, 1, 1)
    W1[0, 0, c], W1[1, 0, c] = 1.0, -1.0
    W2[0, 0, c], W2[1, 1, c] = 1.0, 1.0
    W3[0, 0, c], W3[0, 1, c] = 1.0, -1.0
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 11, 12, 13))
    out = O.closure_forward(p, x)
    np.testing.assert_allclose(out, x[0, 3:-3, 3:-3, 3:-3], rtol=0, atol=1e-14)


def test_relu_inactive_network_is_three_correlations(O):
    """Positive inputs, weights and biases keep every ReLU inactive: the net
    is three cross-correlations with biases, computed here with scipy."""
    from scipy import ndimage
    rng = np.random.default_rng(1)
    h = 4
    p = rng.uniform(0.1, 1.0, O.closure_num_params(h))
    W1, b1, W2, b2, W3, b3 = split_params(p, h)
    x = rng.uniform(0.1, 1.0, (3, 10, 9, 11))

    def corr(inp, W, b):
        co, ci = W.shape[:2]
        out = []
        for o in range(co):
            s = sum(ndimage.correlate(inp[i], W[o, i].reshape(3, 3, 3), mode="constant")
                    for i in range(ci))
            out.append(s[1:-1, 1:-1, 1:-1] + b[o])
        return np.array(out)

    ref = corr(corr(corr(x, W1, b1), W2, b2), W3, b3)[0]
    np.testing.assert_allclose(O.closure_forward(p, x, hidden=h), ref, rtol=1e-12)


@pytest.mark.parametrize("h", [2, 16])
def test_gradient_matches_central_differences(O, h):
    rng = np.random.default_rng(2 + h)
    p = 0.3 * rng.standard_normal(O.closure_num_params(h))
    x = rng.standard_normal((2, 3, 9, 8, 10))
    t = rng.standard_normal((2, 3, 2, 4))
    L0, g = O.closure_loss_grad(p, x, t, hidden=h)
    idx = rng.choice(p.size, size=40, replace=False)
    eps = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = eps
        fd = (O.closure_loss_grad(p + e, x, t, hidden=h, grad=False)[0] -
              O.closure_loss_grad(p - e, x, t, hidden=h, grad=False)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
