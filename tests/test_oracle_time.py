"""Pins of the oracle's time stepping (Algorithm 1 with Eq. Acou / Eq. TTI):
standing modes against their closed forms, energy conservation, the 3D
Green's function, trilinear sources/receivers, and the sponge."""
import math

import numpy as np
import pytest

from paper_1608_03984_gb300 import synth
from test_oracle_operators import periodic_grid, rotated_frame


def mode_setup(O, n=16, order=8, courant=0.3, v=1.0, **kw):
    h, X, Y, Z = periodic_grid(n, 2 * math.pi)
    dt = courant * h / v
    s = O.Setup(np.full((n, n, n), v), h, 0, order, dt, **kw)
    return s, h, X, Y, Z


@pytest.mark.parametrize("order", [2, 8, 16])
def test_acoustic_standing_mode_closed_form(O, order):
    """u_0 = u_-1 = cos(k.x): u_n = cos(w (n+1/2) dt) / cos(w dt/2) cos(k.x)
    with 2 (1 - cos w dt) = dt^2 v^2 Lambda, Lambda the (measured) symbol."""
    s, h, X, Y, Z = mode_setup(O, order=order)
    u0 = np.cos(X + 2 * Y - Z)
    lam = -(O.laplacian(u0, order, h, periodic=True) / u0)[0, 0, 0]
    wdt = math.acos(1.0 - 0.5 * s.dt ** 2 * lam)
    u, um = u0.copy(), u0.copy()
    for n in range(1, 41):
        u, um = O.acoustic_step(s, u, um, periodic=True, damping=False), u
        a = math.cos(wdt * (n + 0.5)) / math.cos(0.5 * wdt)
        np.testing.assert_allclose(u, a * u0, rtol=0, atol=1e-12)


def test_acoustic_time_order_two(O):
    """At fixed h the discrete frequency tends to v sqrt(Lambda) as dt^2."""
    errs = []
    for courant in (0.4, 0.2, 0.1):
        s, h, X, Y, Z = mode_setup(O, order=8, courant=courant)
        u0 = np.cos(X + Y)
        lam = -(O.laplacian(u0, 8, h, periodic=True) / u0)[0, 0, 0]
        u, um = u0.copy(), u0.copy()
        nsteps = int(round(0.8 / s.dt))
        for _ in range(nsteps):
            u, um = O.acoustic_step(s, u, um, periodic=True, damping=False), u
        w = math.sqrt(lam)  # frequency of the time-continuous, space-discrete problem
        exact = math.cos(w * (nsteps + 0.5) * s.dt) / math.cos(0.5 * w * s.dt)
        errs.append(abs(u[0, 0, 0] / u0[0, 0, 0] - exact))
    assert 3.3 < errs[0] / errs[1] < 4.7 and 3.3 < errs[1] / errs[2] < 4.7, errs


@pytest.mark.parametrize("order", [4, 8])
@pytest.mark.parametrize("theta,phi", [(0.0, 0.0), (0.6, 1.2), (1.2, 2.9)])
def test_tti_standing_mode(O, order, theta, phi):
    """Homogeneous TTI on a periodic box: a mode cos(k.x) in p and r obeys the
    2x2 reduction of Eq. TTI, X+ = 2X - X- + dt^2 v^2 M X with
    M = [[e H, d G], [d H, G]], G = n^T S n, H = tr S - G, S the (measured)
    symbols of the six second derivatives."""
    eps, delta = 0.2, 0.1
    n = 16
    s, h, X, Y, Z = mode_setup(O, n=n, order=order, courant=0.25,
                               eps=np.full((n,) * 3, eps), delta=np.full((n,) * 3, delta),
                               theta=np.full((n,) * 3, theta), phi=np.full((n,) * 3, phi))
    u0 = np.cos(X + 2 * Y + 3 * Z)
    S = np.zeros((3, 3))
    names = {(0, 0): "xx", (1, 1): "yy", (2, 2): "zz", (0, 1): "xy", (0, 2): "xz", (1, 2): "yz"}
    for (i, j), w in names.items():
        S[i, j] = S[j, i] = (O.derivative(u0, w, order, h, periodic=True) / u0)[1, 2, 3]
    _, _, nv = rotated_frame(theta, phi)
    G = nv @ S @ nv
    H = np.trace(S) - G
    e, d = 1 + 2 * eps, math.sqrt(1 + 2 * delta)
    M = np.array([[e * H, d * G], [d * H, G]])
    c = s.dt ** 2
    Xc = np.array([1.0, 0.3])
    Xm = Xc.copy()
    p, pm, r, rm = Xc[0] * u0, Xc[0] * u0, Xc[1] * u0, Xc[1] * u0
    for _ in range(30):
        p2, r2 = O.tti_step(s, p, pm, r, rm, periodic=True, damping=False)
        pm, rm, p, r = p, r, p2, r2
        Xc, Xm = 2 * Xc - Xm + c * (M @ Xc), Xc
        np.testing.assert_allclose(p, Xc[0] * u0, atol=1e-11)
        np.testing.assert_allclose(r, Xc[1] * u0, atol=1e-11)


def test_tti_reduces_to_acoustic(O):
    """eps = delta = 0 and p = r: both fields follow the acoustic step for
    any tilt (H + G is the Laplacian)."""
    rng = np.random.default_rng(2)
    shp = (14, 12, 13)
    vp = 1500 + 500 * rng.random(shp)
    th = rng.uniform(0, 1.5, shp)
    ph = rng.uniform(0, 3, shp)
    sa = O.Setup(vp, 10.0, 3, 8, 1e-3)
    st = O.Setup(vp, 10.0, 3, 8, 1e-3, eps=np.zeros(shp), delta=np.zeros(shp), theta=th, phi=ph)
    u = synth.random_wavefield(sa.shape, 4).astype(np.float64)
    um = synth.random_wavefield(sa.shape, 5).astype(np.float64)
    src = np.array([[40.0, 50.0, 60.0]])
    ua = O.acoustic_step(sa, u, um, src, 2.0)
    pp, rp = O.tti_step(st, u, um, u, um, src, 2.0)
    np.testing.assert_allclose(pp, ua, rtol=1e-12, atol=1e-12 * np.abs(ua).max())
    np.testing.assert_allclose(rp, ua, rtol=1e-12, atol=1e-12 * np.abs(ua).max())


def test_energy_conserved_without_damping(O):
    """gamma = 0, no source, zero ghosts: E_{n+1/2} = sum (u_{n+1}-u_n)^2 / c
    - sum u_{n+1} L u_n is constant (L symmetric)."""
    rng = np.random.default_rng(9)
    shp = (20, 18, 22)
    vp = 1500 + 1000 * synth.smooth_random_field(shp, 3, 17).astype(np.float64) ** 2
    h, order = 10.0, 8
    dt = 0.5 * O.max_stable_dt(order, h, vp.max())
    s = O.Setup(vp, h, 0, order, dt)
    g = synth.smooth_random_field(shp, 2, 21).astype(np.float64)
    g *= np.exp(-((np.indices(shp) - np.array(shp)[:, None, None, None] / 2) ** 2).sum(0) / 20)
    u, um = g.copy(), 0.98 * g
    E = []
    for _ in range(60):
        up = O.acoustic_step(s, u, um, damping=False)
        E.append(np.sum((up - u) ** 2 / s.c) - np.sum(up * O.laplacian(u, order, h)))
        um, u = u, up
    E = np.array(E)
    assert np.abs(E / E[0] - 1).max() < 1e-11, np.abs(E / E[0] - 1).max()


def test_sponge_absorbs(O):
    """The damped run loses most of the energy once the pulse has reached
    the boundary, the undamped one keeps it."""
    shp = (24, 24, 24)
    vp = np.full(shp, 2000.0)
    h, order, nb = 10.0, 4, 10
    dt = 0.4 * h / 2000.0
    g = np.exp(-((np.indices((44,) * 3) - 22.0) ** 2).sum(0) / 8.0)
    s = O.Setup(vp, h, nb, order, dt)
    out = []
    for damping in (False, True):
        u, um = g.copy(), g.copy()
        for _ in range(150):
            u, um = O.acoustic_step(s, u, um, damping=damping), u
        out.append(np.sum(u ** 2))
    assert out[1] < 1e-2 * out[0], out


def test_trilinear_interpolation_exact_on_linear(O):
    shp = (10, 11, 12)
    h, nb = 5.0, 2
    kk, jj, ii = np.indices((14, 15, 16)).astype(np.float64)
    # physical coordinate of computational index i is (i - nb) h
    u = 0.3 + 0.7 * (ii - nb) * h - 0.2 * (jj - nb) * h + 1.1 * (kk - nb) * h
    rng = np.random.default_rng(1)
    xyz = rng.uniform([-nb * h, -nb * h, -nb * h], [(shp[2] - 1 + nb) * h, (shp[1] - 1 + nb) * h,
                                                   (shp[0] - 1 + nb) * h], size=(50, 3))
    got = O.interpolate(u, xyz, h, nb)
    exp = 0.3 + 0.7 * xyz[:, 0] - 0.2 * xyz[:, 1] + 1.1 * xyz[:, 2]
    np.testing.assert_allclose(got, exp, rtol=1e-12, atol=1e-10)


def test_injection_is_scaled_transpose_of_interpolation(O):
    """Injecting amplitude a from zero state adds c a w / h^3 at the corners:
    <u_1, f> = c a / h^3 interp(f) for constant c, any f; the total is c a / h^3."""
    shp = (12, 12, 12)
    h, nb, dt = 4.0, 0, 1e-3
    s = O.Setup(np.full(shp, 1000.0), h, nb, 4, dt)
    z = np.zeros(shp)
    xyz = np.array([[13.3, 21.7, 30.1]])
    u1 = O.acoustic_step(s, z, z, xyz, 2.5)
    c = (dt * 1000.0) ** 2
    assert u1.sum() == pytest.approx(c * 2.5 / h ** 3, rel=1e-13)
    f = np.random.default_rng(0).standard_normal(shp)
    assert np.sum(u1 * f) == pytest.approx(c * 2.5 / h ** 3 * O.interpolate(f, xyz, h, nb)[0],
                                           rel=1e-12)


def test_greens_function(O):
    """Homogeneous medium, point source: u(r, t) = s(t - r/v) / (4 pi r)
    (Eq. Acou with q = delta(x) s(t)); traces before any boundary
    reflection arrives. Order 8 is within 3%, order 2 is visibly worse."""
    v, h, n, nb, f0 = 2000.0, 10.0, 56, 30, 10.0
    dt = 0.4 * h / v
    c0 = 28 * h
    src = np.array([[c0, c0, c0]])
    # receivers on grid points (no interpolation error): axial and oblique
    offs = np.array([[10, 0, 0], [0, 0, -14], [18, 0, 0], [10, 10, 0], [8, 6, 0], [0, 12, 9],
                     [-9, 12, 0]], dtype=np.float64)
    recs = c0 + h * offs
    dist = h * np.linalg.norm(offs, axis=1)
    nt = int((1.0 / f0 + dist.max() / v + 1.2 / f0) / dt)
    w = synth.ricker(f0, dt, nt).reshape(nt, 1)
    errs = {}
    for order in (2, 8):
        s = O.Setup(np.full((n,) * 3, v), h, nb, order, dt)
        tr = O.acoustic_forward(s, src, w, nt, recs)["traces"]
        worst = 0.0
        for i, d in enumerate(dist):
            exact = synth.ricker(f0, dt, nt + 1, t0=1.0 / f0 + d / v) / (4 * math.pi * d)
            e = np.linalg.norm(tr[:, i] - exact) / np.linalg.norm(exact)
            worst = max(worst, e)
        errs[order] = worst
    assert errs[8] < 0.02, errs
    assert errs[2] > 2 * errs[8], errs
