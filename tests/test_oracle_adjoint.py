"""Pins of the oracle's adjoint and FWI gradient (the transpose of the
discrete recurrence of Algorithm 1 / Eq. Acou with the sponge): the
dot-product test and the Taylor test of the gradient."""
import numpy as np
import pytest

from paper_1608_03984_gb300 import synth


def small_problem(O, order=4, nt=60, seed=0):
    rng = np.random.default_rng(seed)
    shp = (14, 16, 15)
    h, nb = 10.0, 5
    vp = 1800 + 600 * synth.smooth_random_field(shp, 3, 100 + seed).astype(np.float64) ** 2
    dt = 0.45 * O.max_stable_dt(order, h, vp.max())
    s = O.Setup(vp, h, nb, order, dt)
    src = np.array([[52.0, 61.5, 40.0], [103.0, 47.0, 93.3]])
    rec = rng.uniform([0, 0, 0], [140, 150, 130], size=(6, 3))
    return s, vp, src, rec, nt


@pytest.mark.parametrize("order", [2, 8])
def test_dot_product(O, order):
    """<F s, d> = <s, F^T d> for the map wavelet -> traces (sponge on)."""
    s, vp, src, rec, nt = small_problem(O, order)
    rng = np.random.default_rng(1)
    w = rng.standard_normal((nt, src.shape[0]))
    d = rng.standard_normal((nt + 1, rec.shape[0]))
    Fs = O.acoustic_forward(s, src, w, nt, rec)["traces"]
    Ftd = O.acoustic_adjoint(s, rec, d, nt, src)["wavelet_adj"]
    a, b = np.sum(Fs * d), np.sum(w * Ftd)
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b)), (a, b)


def objective(O, vp, h, nb, order, dt, gmax_v, src, w, rec, nt, dobs, dm=None, eps=0.0):
    m = 1.0 / vp ** 2
    if dm is not None:
        m = m + eps * dm
    s = O.Setup(1.0 / np.sqrt(m), h, nb, order, dt, gamma_vmax=gmax_v)
    out = O.acoustic_forward(s, src, w, nt, rec, history=True)
    r = out["traces"] - dobs
    return 0.5 * np.sum(r * r), r, out, s


def test_gradient_taylor(O):
    """J(m + e dm) - J(m) - e <g, dm> = O(e^2) for the squared slowness m
    (dm supported away from the physical boundary, sponge fixed)."""
    s0, vp, src, rec, nt = small_problem(O, order=4, nt=70, seed=3)
    h, nb, order, dt = s0.h, s0.nb, s0.order, s0.dt
    gv = float(vp.max())
    w = synth.ricker(15.0, dt, nt).reshape(nt, 1).repeat(2, axis=1)
    vtrue = vp * (1 + 0.05 * np.exp(-((np.indices(vp.shape) - 7.0) ** 2).sum(0) / 6.0))
    dobs = O.acoustic_forward(O.Setup(vtrue, h, nb, order, dt, gamma_vmax=gv), src, w, nt,
                              rec)["traces"]
    J0, r, out, s = objective(O, vp, h, nb, order, dt, gv, src, w, rec, nt, dobs)
    g = O.acoustic_adjoint(s, rec, r, nt, src, history=out["history"])["grad_m"]
    rng = np.random.default_rng(5)
    dm = np.zeros(vp.shape)
    dm[2:-2, 2:-2, 2:-2] = rng.standard_normal(tuple(n - 4 for n in vp.shape))
    dm *= 0.02 / vp.max() ** 2
    gphys = g[nb:-nb, nb:-nb, nb:-nb]
    lin = np.sum(gphys * dm)
    rem = []
    for e in (1.0, 0.5, 0.25, 0.125):
        Je = objective(O, vp, h, nb, order, dt, gv, src, w, rec, nt, dobs, dm, e)[0]
        rem.append(abs(Je - J0 - e * lin))
    ratios = [rem[i] / rem[i + 1] for i in range(3)]
    assert all(3.5 < q < 4.5 for q in ratios), (ratios, rem, lin)
    # central difference agrees with <g, dm> to O(e^2)
    e = 1e-3
    Jp = objective(O, vp, h, nb, order, dt, gv, src, w, rec, nt, dobs, dm, e)[0]
    Jm = objective(O, vp, h, nb, order, dt, gv, src, w, rec, nt, dobs, dm, -e)[0]
    assert (Jp - Jm) / (2 * e) == pytest.approx(lin, rel=1e-6)


def test_gradient_in_sponge(O):
    """The gradient is the exact transpose also where the sponge damps
    (P, Q != 1): a perturbation inside the sponge passes the FD check."""
    s0, vp, src, rec, nt = small_problem(O, order=4, nt=50, seed=4)
    h, nb, order, dt = s0.h, s0.nb, s0.order, s0.dt
    gv = float(vp.max())
    w = synth.ricker(15.0, dt, nt).reshape(nt, 1).repeat(2, axis=1)
    dobs = np.zeros((nt + 1, rec.shape[0]))
    J0, r, out, s = objective(O, vp, h, nb, order, dt, gv, src, w, rec, nt, dobs)
    g = O.acoustic_adjoint(s, rec, r, nt, src, history=out["history"])["grad_m"]
    # perturb c directly in a sponge cell by editing the computational medium
    k, j, i = 2, 9, 10
    base = s.c.copy()
    eps = 1e-4 * base[k, j, i]

    def J_with_c(cval):
        s.c = base.copy()
        s.c[k, j, i] = cval
        t = O.acoustic_forward(s, src, w, nt, rec)["traces"]
        return 0.5 * np.sum((t - dobs) ** 2)

    fd = (J_with_c(base[k, j, i] + eps) - J_with_c(base[k, j, i] - eps)) / (2 * eps)
    s.c = base
    # dJ/dc = dJ/dm * dm/dc with m = dt^2 / c: dm/dc = -dt^2 / c^2
    dJdc = g[k, j, i] * (-dt * dt / base[k, j, i] ** 2)
    assert dJdc == pytest.approx(fd, rel=1e-5), (dJdc, fd)


@pytest.mark.parametrize("nb", [1, 3])
def test_extend_adjoint_dot_product(O, nb):
    """extend_adjoint is the transpose of extend (the medium's continuation
    into the sponge, through which the FWI gradient on the computational
    grid is folded back onto the physical grid): <E a, b> = <a, E^T b> for
    random a, b on a non-cubic grid."""
    rng = np.random.default_rng(7 + nb)
    a = rng.standard_normal((5, 7, 6))
    b = rng.standard_normal((5 + 2 * nb, 7 + 2 * nb, 6 + 2 * nb))
    lhs = np.sum(O.extend(a, nb) * b)
    rhs = np.sum(a * O.extend_adjoint(b, nb))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs)), (lhs, rhs)


@pytest.mark.parametrize("nb", [0, 1, 2])
def test_extend_adjoint_equals_transposed_matrix(O, nb):
    """Brute force on a 4 x 5 x 6 grid: build the matrix of the extension
    column by column (extension of each unit vector), transpose it, apply it
    to a random computational field; extend_adjoint gives the same vector.
    A corner sponge point counts once per physical point it copies, so a
    missed edge or corner contribution fails here."""
    shp = (4, 5, 6)
    ncomp = tuple(k + 2 * nb for k in shp)
    cols = []
    for i in range(int(np.prod(shp))):
        e = np.zeros(int(np.prod(shp)))
        e[i] = 1.0
        cols.append(O.extend(e.reshape(shp), nb).ravel())
    M = np.stack(cols, axis=1)  # computational x physical
    # every computational point copies exactly one physical point
    assert M.shape == (int(np.prod(ncomp)), int(np.prod(shp)))
    assert np.all(M.sum(axis=1) == 1.0)
    g = np.random.default_rng(3).standard_normal(ncomp)
    want = (M.T @ g.ravel()).reshape(shp)
    got = O.extend_adjoint(g, nb)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
