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


def test_same_padded_net_interior_equals_valid_net(O):
    """Away from the grid's faces (3 points: the receptive-field radius) the
    zero-padded network equals the valid one, whose pins are above."""
    rng = np.random.default_rng(3)
    p = rng.standard_normal(O.closure_num_params(H)) * 0.2
    x = rng.standard_normal((3, 11, 10, 12))
    same = O.closure_forward_same(p, x)
    assert same.shape == (11, 10, 12)
    np.testing.assert_allclose(same[3:-3, 3:-3, 3:-3], O.closure_forward(p, x), rtol=1e-12, atol=1e-12)


def test_same_padded_net_equals_valid_net_on_zero_extended_grid_when_linear(O):
    """With every ReLU inactive (biases large, weights non-negative, inputs
    non-negative) the network is linear and bias-free outside: then the
    zero-padded net on a grid equals the composition of three zero-padded
    cross-correlations computed independently by scipy.ndimage."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(4)
    p = np.zeros(O.closure_num_params(H))
    W1, b1, W2, b2, W3, b3 = split_params(p)
    W1[:] = rng.uniform(0, 1, W1.shape)
    W2[:] = rng.uniform(0, 1, W2.shape)
    W3[:] = rng.uniform(-1, 1, W3.shape)
    b1[:] = rng.uniform(0.5, 1, b1.shape)
    b2[:] = rng.uniform(0.5, 1, b2.shape)
    b3[:] = 0.3
    x = rng.uniform(0, 1, (3, 7, 8, 9))

    def layer(a, W, b):
        out = []
        for o in range(W.shape[0]):
            acc = np.full(a.shape[1:], b[o])
            for i in range(W.shape[1]):
                k = W[o, i].reshape(3, 3, 3)
                acc += ndimage.correlate(a[i], k, mode="constant", cval=0.0)
            out.append(acc)
        return np.array(out)

    ref = layer(layer(layer(x, W1, b1), W2, b2), W3, b3)[0]
    np.testing.assert_allclose(O.closure_forward_same(p, x), ref, rtol=1e-12, atol=1e-12)


def test_closure_step_with_zero_network_is_the_acoustic_step(O):
    """A network with all parameters zero adds nothing: the closure step is
    the plain step of Algorithm 1 (source included)."""
    rng = np.random.default_rng(5)
    vp = rng.uniform(1500, 3000, (8, 9, 10))
    s = O.Setup(vp, 10.0, 3, 4, 1e-3)
    u, um = rng.standard_normal((2,) + s.shape)
    src = np.array([[40.0, 30.0, 35.0]])
    p = np.zeros(O.closure_num_params(H))
    np.testing.assert_allclose(O.closure_step(s, u, um, vp, p, src, [2.0]),
                               O.acoustic_step(s, u, um, src, [2.0]), rtol=1e-13, atol=1e-13)


def test_closure_step_network_of_velocity_alone_adds_nothing(O):
    """A network that ignores the wavefield channels (here: only biases and
    velocity weights) gives net(x) = net(x0): the closure step is the plain
    step. And a zero wavefield gets no correction whatever the network."""
    rng = np.random.default_rng(6)
    vp = rng.uniform(1500, 3000, (8, 9, 10))
    s = O.Setup(vp, 10.0, 3, 4, 1e-3)
    u, um = rng.standard_normal((2,) + s.shape)
    p = np.zeros(O.closure_num_params(H))
    W1, b1, W2, b2, W3, b3 = split_params(p)
    W1[:, 2] = rng.standard_normal(W1[:, 2].shape)
    W2[:] = rng.standard_normal(W2.shape) * 0.2
    W3[:] = rng.standard_normal(W3.shape) * 0.2
    b1[:], b2[:], b3[:] = 0.1, -0.05, 0.25
    np.testing.assert_allclose(O.closure_step(s, u, um, vp, p), O.acoustic_step(s, u, um),
                               rtol=1e-12, atol=1e-12)
    p2 = rng.standard_normal(p.size) * 0.3
    z = np.zeros(s.shape)
    np.testing.assert_array_equal(O.closure_step(s, z, z, vp, p2), np.zeros(s.shape))


def test_closure_step_linear_network_scales_out(O):
    """A network that is linear in the wavefield channels (ReLUs inactive,
    no velocity weights, positive biases) gives m * (net(x) - net(x0)) =
    the linear map applied to u itself: independent of the normalisation m.
    Checked by scaling u and u_{n-1} together."""
    rng = np.random.default_rng(7)
    vp = rng.uniform(1500, 3000, (8, 9, 10))
    s = O.Setup(vp, 10.0, 3, 4, 1e-3)
    assert s.shape == (14, 15, 16)
    u, um = rng.uniform(0, 1, (2,) + s.shape)
    p = np.zeros(O.closure_num_params(H))
    W1, b1, W2, b2, W3, b3 = split_params(p)
    W1[:, :2] = rng.uniform(0, 0.1, W1[:, :2].shape)
    W2[:] = rng.uniform(0, 0.1, W2.shape)
    W3[:] = rng.uniform(-0.1, 0.1, W3.shape)
    b1[:], b2[:] = 1.0, 1.0
    a = O.closure_step(s, u, um, vp, p) - O.acoustic_step(s, u, um)
    b = O.closure_step(s, 3 * u, 3 * um, vp, p) - O.acoustic_step(s, 3 * u, 3 * um)
    np.testing.assert_allclose(b, 3 * a, rtol=1e-10, atol=1e-14)
    assert np.abs(a).max() > 1e-3
    # the sponge (3 points on every face) and the 3 physical points next to
    # it keep the plain update
    inner = np.zeros(s.shape, bool)
    inner[6:-6, 6:-6, 6:-6] = True
    assert np.all(a[~inner] == 0) and np.all(a[inner] != 0)


def test_correction_loss_gradient_matches_central_differences(O):
    """The correction's loss gradient (two vector-Jacobian products) against
    central differences of its loss, on a few random parameters."""
    rng = np.random.default_rng(8)
    p = rng.standard_normal(O.closure_num_params(H)) * 0.2
    x = rng.standard_normal((2, 3, 8, 8, 8))
    t = rng.standard_normal((2, 2, 2, 2))
    loss, g = O.closure_correction_loss_grad(p, x, t)
    fwd = np.stack([O.closure_correction(p, x[b]) for b in range(2)])
    assert abs(loss - np.mean((fwd - t) ** 2)) < 1e-14
    eps = 1e-6
    for i in rng.choice(p.size, 12, replace=False):
        e = np.zeros_like(p)
        e[i] = eps
        lp, _ = O.closure_correction_loss_grad(p + e, x, t)
        lm, _ = O.closure_correction_loss_grad(p - e, x, t)
        assert abs((lp - lm) / (2 * eps) - g[i]) <= 1e-6 * max(1.0, abs(g[i])), i
