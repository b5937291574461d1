"""Pins of the oracle's spatial operators: convergence order of every
derivative type (Section "Stencil operators"), exactness on quadratics, and
the rotated operators of Eq. DiffOp against the geometry of a rotation."""
import math

import numpy as np
import pytest


def periodic_grid(n, L):
    h = L / n
    x = np.arange(n) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return h, X, Y, Z


@pytest.mark.parametrize("order", [2, 4, 8, 12, 16])
def test_laplacian_convergence_order(O, order):
    """Error of the Laplacian of sin(kx x + ky y + kz z) on a periodic box
    falls like h^order."""
    errs, hs = [], []
    L = 2 * math.pi
    for n in (16, 24, 32) if order < 16 else (16, 20, 24):
        h, X, Y, Z = periodic_grid(n, L)
        u = np.sin(X + 2 * Y + Z)
        exact = -(1 + 4 + 1) * u
        lap = O.laplacian(u, order, h, periodic=True)
        errs.append(np.abs(lap - exact).max())
        hs.append(h)
    slope = math.log(errs[-2] / errs[-1]) / math.log(hs[-2] / hs[-1])
    assert slope > order - 0.5, (order, slope, errs)


@pytest.mark.parametrize("order", [2, 6, 16])
def test_laplacian_symbol_exact(O, order):
    """On a periodic grid sin(k.x) is an eigenfunction of the discrete
    Laplacian with eigenvalue sum_a h^-2 (w0 + 2 sum_j w_j cos(j k_a h)),
    w the textbook central weights."""
    from test_oracle_weights import closed_form
    w2, _ = closed_form(order)
    n = 16
    h, X, Y, Z = periodic_grid(n, 2 * math.pi)
    ks = (1, 3, 2)
    u = np.sin(ks[0] * X + ks[1] * Y + ks[2] * Z)
    sym = sum((w2[0] + 2 * sum(w2[j] * math.cos(j * k * h) for j in range(1, len(w2)))) / h ** 2
              for k in ks)
    np.testing.assert_allclose(O.laplacian(u, order, h, periodic=True), sym * u, atol=1e-11 * abs(sym))


@pytest.mark.parametrize("which,fn,dfn", [
    ("x", lambda X, Y, Z: np.sin(X) * np.cos(Y), lambda X, Y, Z: np.cos(X) * np.cos(Y)),
    ("zz", lambda X, Y, Z: np.sin(2 * Z) * np.cos(X), lambda X, Y, Z: -4 * np.sin(2 * Z) * np.cos(X)),
    ("xy", lambda X, Y, Z: np.sin(X) * np.sin(2 * Y), lambda X, Y, Z: 2 * np.cos(X) * np.cos(2 * Y)),
    ("xz", lambda X, Y, Z: np.sin(X + Z) + np.cos(X) * np.sin(Z), lambda X, Y, Z: -np.sin(X + Z) - np.sin(X) * np.cos(Z)),
    ("yz", lambda X, Y, Z: np.cos(Y) * np.cos(Z), lambda X, Y, Z: np.sin(Y) * np.sin(Z)),
])
@pytest.mark.parametrize("order", [4, 8])
def test_derivative_convergence(O, which, fn, dfn, order):
    errs, hs = [], []
    for n in (12, 16, 24):
        h, X, Y, Z = periodic_grid(n, 2 * math.pi)
        d = O.derivative(fn(X, Y, Z), which, order, h, periodic=True)
        errs.append(np.abs(d - dfn(X, Y, Z)).max())
        hs.append(h)
    slope = math.log(errs[-2] / errs[-1]) / math.log(hs[-2] / hs[-1])
    assert slope > order - 0.5, (which, order, slope, errs)


def rotated_frame(theta, phi):
    """Rotated axes: zbar is the symmetry axis at tilt theta from vertical
    and azimuth phi; xbar lies in the vertical plane containing it; ybar is
    horizontal (the frame of Eq. DiffOp)."""
    zb = np.array([math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi), math.cos(theta)])
    xb = np.array([math.cos(theta) * math.cos(phi), math.cos(theta) * math.sin(phi), -math.sin(theta)])
    yb = np.cross(zb, xb)
    return xb, yb, zb


@pytest.mark.parametrize("order", [2, 4, 8, 12])
@pytest.mark.parametrize("theta,phi", [(0.0, 0.0), (0.3, 1.1), (1.0, 2.5), (0.7, -0.4)])
def test_rotated_operators_on_quadratic(O, order, theta, phi):
    """u = x^T A x / 2: every stencil is exact on quadratics, so at points
    r away from the boundary G_aa u = a^T A a for each rotated axis a."""
    rng = np.random.default_rng(7)
    A = rng.standard_normal((3, 3))
    A = A + A.T
    n, h = 20, 0.7
    g = np.arange(n) * h
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    P = np.stack([X, Y, Z], axis=-1)
    u = 0.5 * np.einsum("...i,ij,...j->...", P, A, P)
    gx, gy, gz = O.rotated(u, theta, phi, order, h)
    r = order // 2
    sl = (slice(r, n - r),) * 3
    xb, yb, zb = rotated_frame(theta, phi)
    for G, a in ((gx, xb), (gy, yb), (gz, zb)):
        np.testing.assert_allclose(G[sl], a @ A @ a, rtol=0, atol=1e-8 * np.abs(A).max() / h ** 0)
    # Gxx + Gyy + Gzz is the Laplacian (trace of A) everywhere
    lap = O.laplacian(u, order, h)
    np.testing.assert_allclose(gx + gy + gz, lap, rtol=1e-11, atol=1e-9 * np.abs(lap).max())


@pytest.mark.parametrize("order", [4, 12])
def test_rotated_sum_is_laplacian_random(O, order):
    """On an arbitrary field with point-wise varying angles the three
    rotated operators add up to the Laplacian (coefficients cancel)."""
    rng = np.random.default_rng(3)
    u = rng.standard_normal((14, 15, 16))
    th = rng.uniform(0, math.pi, u.shape)
    ph = rng.uniform(0, 2 * math.pi, u.shape)
    gx, gy, gz = O.rotated(u, th, ph, order, 1.3)
    lap = O.laplacian(u, order, 1.3)
    np.testing.assert_allclose(gx + gy + gz, lap, rtol=0, atol=1e-11 * np.abs(lap).max())


def test_rotated_vertical_axis_is_vti(O):
    """theta = 0: Gzz is d2/dz2 and Gxx + Gyy the horizontal Laplacian (VTI)."""
    rng = np.random.default_rng(5)
    u = rng.standard_normal((12, 13, 14))
    h = 0.9
    for phi in (0.0, 0.8):
        gx, gy, gz = O.rotated(u, 0.0, phi, 8, h)
        np.testing.assert_allclose(gz, O.derivative(u, "zz", 8, h), atol=1e-12)
        np.testing.assert_allclose(gx + gy, O.derivative(u, "xx", 8, h) + O.derivative(u, "yy", 8, h),
                                   atol=1e-11)


def test_dirichlet_ghosts_symmetric(O):
    """With zero ghosts the Laplacian matrix is symmetric: <Lu, v> = <u, Lv>."""
    rng = np.random.default_rng(11)
    u = rng.standard_normal((9, 10, 11))
    v = rng.standard_normal(u.shape)
    for order in (2, 8, 16):
        a = np.sum(O.laplacian(u, order, 1.0) * v)
        b = np.sum(u * O.laplacian(v, order, 1.0))
        assert abs(a - b) < 1e-10 * abs(a)


@pytest.mark.parametrize("order", [4, 8])
def test_point_updates_equal_the_full_step(O, order):
    """The block point updates used to check full-size GPU runs equal the
    full oracle step at interior points of a grid with a varying medium and
    sponge (acoustic and TTI)."""
    rng = np.random.default_rng(order)
    shape = (14, 15, 16)
    nb = 3
    vp = rng.uniform(1500, 3000, shape)
    eps = rng.uniform(0, 0.3, shape)
    delta = np.minimum(rng.uniform(0, 0.2, shape), eps)
    theta = rng.uniform(0, 1.0, shape)
    phi = rng.uniform(0, 3.0, shape)
    dt = 1e-3
    s = O.Setup(vp, 10.0, nb, order, dt, eps=eps, delta=delta, theta=theta, phi=phi)
    comp = s.shape
    u, um, q, qm = rng.standard_normal((4,) + comp)
    up = O.acoustic_step(s, u, um)
    pp, rp = O.tti_step(s, u, um, q, qm)
    r = order // 2
    gam = lambda k, j, i: s.gx[i] + s.gy[j] + s.gz[k]
    for (k, j, i) in [(r, r, r), (r + 1, 7, 9), (comp[0] - r - 1, comp[1] - r - 1, comp[2] - r - 1),
                      (10, r, 12), (r, r + 1, r + 2)]:
        sl = (slice(k - r, k + r + 1), slice(j - r, j + r + 1), slice(i - r, i + r + 1))
        v_c = np.sqrt(s.c[k, j, i]) / dt
        a = O.acoustic_update_at(u[sl], um[k, j, i], v_c, gam(k, j, i), s.h, order, dt)
        assert abs(a - up[k, j, i]) <= 1e-12 * np.abs(u).max()
        b = O.tti_update_at(u[sl], um[k, j, i], q[sl], qm[k, j, i], v_c, s.eps[k, j, i],
                            s.delta[k, j, i], s.theta[k, j, i], s.phi[k, j, i], gam(k, j, i), s.h,
                            order, dt)
        assert abs(b[0] - pp[k, j, i]) <= 1e-12 * np.abs(u).max()
        assert abs(b[1] - rp[k, j, i]) <= 1e-12 * np.abs(u).max()
