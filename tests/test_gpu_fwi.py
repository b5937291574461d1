"""GPU adjoint and FWI gradient against the FP64 oracle and finite
differences, through the C ABI (fdw_adjoint_*, fdw_history_*) and the
torch.autograd wrapper."""
import math

import numpy as np
import pytest

from paper_1608_03984_gb300 import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def problem(order=4, nt=60, seed=0, shape=(18, 21, 25), nb=6, nsrc=2):
    rng = np.random.default_rng(seed)
    h = 10.0
    vp = (1800 + 600 * synth.smooth_random_field(shape, 3, 300 + seed) ** 2).astype(np.float32)
    dt = 0.45 * h * 0.5 / float(vp.max())
    nz, ny, nx = shape
    src = rng.uniform([20, 20, 20], [(nx - 3) * h, (ny - 3) * h, (nz - 3) * h], size=(nsrc, 3))
    rec = rng.uniform([-nb * h, -nb * h, 0], [(nx - 1) * h, (ny - 1) * h, (nz - 1) * h], size=(7, 3))
    return dict(vp=vp, h=h, nb=nb, order=order, dt=dt, nt=nt, src=src, rec=rec, shape=shape)


def solver(fdw, P, wavelet):
    s = fdw.Solver(P["shape"], P["h"], P["nb"], P["order"])
    s.set_model(P["vp"]).set_dt(P["dt"]).set_sources(P["src"], wavelet).set_receivers(P["rec"], P["nt"])
    return s


@pytest.mark.parametrize("order", [2, 8, 16])
def test_adjoint_dot_product(fdw, order):
    """<F s, d> = <s, F^T d> for the map wavelet -> traces (sponge on)."""
    P = problem(order=order, seed=order)
    rng = np.random.default_rng(1)
    w = rng.standard_normal((P["nt"], 2)).astype(np.float32)
    d = rng.standard_normal((P["nt"] + 1, 7))
    s = solver(fdw, P, w)
    s.step(P["nt"])
    Fs = s.traces()
    s.adjoint_begin(d, gradient=False)
    s.adjoint_step(P["nt"])
    Ftd = s.source_adjoint(P["nt"], 2)
    s.check()
    a, b = np.sum(Fs * d), np.sum(w.astype(np.float64) * Ftd)
    assert abs(a - b) <= 1e-5 * max(abs(a), abs(b)), (a, b)
    s.close()


def test_adjoint_and_gradient_match_oracle(fdw, O):
    """Source-side adjoint and dJ/dm (full forward history) against the
    oracle's transposed recurrence."""
    P = problem(order=8, nt=50, seed=3)
    w = synth.ricker(15.0, P["dt"], P["nt"]).astype(np.float32).reshape(-1, 1).repeat(2, axis=1)
    rng = np.random.default_rng(4)
    res = rng.standard_normal((P["nt"] + 1, 7))
    s = solver(fdw, P, w)
    s.history_begin(P["nt"] + 2)
    s.step(P["nt"])
    s.history_end()
    s.adjoint_begin(res, gradient=True)
    s.adjoint_step(P["nt"])
    g_gpu = s.gradient()
    wadj = s.source_adjoint(P["nt"], 2)
    s.check()
    s.close()
    setup = O.Setup(P["vp"], P["h"], P["nb"], P["order"], P["dt"])
    fwd = O.acoustic_forward(setup, P["src"], w, P["nt"], P["rec"], history=True)
    ref = O.acoustic_adjoint(setup, P["rec"], res, P["nt"], P["src"], history=fwd["history"])
    assert rel(wadj, ref["wavelet_adj"]) <= 1e-4
    g_ref = O.extend_adjoint(ref["grad_m"], P["nb"])
    assert rel(g_gpu, g_ref) <= 1e-4, rel(g_gpu, g_ref)


def test_checkpointed_gradient_equals_full_history(fdw):
    """Segments of 7 steps replayed from checkpoints give the gradient of the
    full-history run."""
    import torch
    P = problem(order=4, nt=45, seed=5)
    w = synth.ricker(15.0, P["dt"], P["nt"]).astype(np.float32).reshape(-1, 1).repeat(2, axis=1)
    res = np.random.default_rng(6).standard_normal((P["nt"] + 1, 7))
    s = solver(fdw, P, w)
    s.history_begin(P["nt"] + 2)
    s.step(P["nt"])
    s.history_end()
    s.adjoint_begin(res)
    s.adjoint_step(P["nt"])
    g_full = s.gradient()
    # checkpointed
    s.reset()
    S = 7
    ck = []
    for t0 in range(0, P["nt"], S):
        ck.append((t0, s.wavefield(0, 0).copy(), s.wavefield(0, 1).copy()))
        s.step(min(S, P["nt"] - t0))
    s.adjoint_begin(res)
    for t0, u, um in reversed(ck):
        t1 = min(t0 + S, P["nt"])
        s.set_wavefield(u, 0, 0)
        s.set_wavefield(um, 0, 1)
        s.set_current_step(t0)
        s.history_begin(S + 2)
        s.step(t1 - t0)
        s.history_end()
        s.adjoint_step(t1 - t0)
    assert s.adjoint_current_step == 1
    g_ck = s.gradient()
    s.check()
    s.close()
    assert rel(g_ck, g_full) <= 1e-6


def test_missing_history_is_an_error(fdw):
    P = problem(order=4, nt=20, seed=7)
    w = np.zeros((P["nt"], 2), np.float32)
    s = solver(fdw, P, w)
    s.step(P["nt"])
    s.adjoint_begin(np.ones((P["nt"] + 1, 7)), gradient=True)
    with pytest.raises(fdw.FdwError) as e:
        s.adjoint_step(1)
    assert e.value.code == -5
    s.close()


def test_fwi_autograd_finite_differences(fdw):
    """torch.autograd gradient of J = 1/2 |F(v) - d_obs|^2 (two shots, 20
    checkpoints) against central differences along 8 random smooth model
    perturbations supported inside the physical grid."""
    import torch
    from paper_1608_03984_gb300 import fwi
    shape, h, nb, order = (26, 24, 28), 15.0, 8, 8
    vt = synth.random_velocity(shape, h, 150.0, 911)
    zz, yy, xx = np.indices(shape)
    anomaly = 1 + 0.1 * np.exp(-((zz - 13) ** 2 + (yy - 12) ** 2 + (xx - 14) ** 2) / 18.0)
    v_true = (vt * anomaly).astype(np.float32)
    v0 = vt.astype(np.float32)
    dt = 0.4 * h / 5000.0
    nt = 120
    src = np.array([[100.0, 120.0, 30.0], [300.0, 200.0, 30.0]])
    gx, gy = np.meshgrid(np.linspace(0, (shape[2] - 1) * h, 6), np.linspace(0, (shape[1] - 1) * h, 6))
    rec = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, 45.0)], axis=1)
    survey = fwi.Survey(shape, h, nb, order, dt, nt, src,
                        synth.ricker(12.0, dt, nt).astype(np.float32), rec, checkpoints=20,
                        sponge_vref=5000.0)
    vt_t = torch.from_numpy(v_true).cuda()
    with torch.no_grad():
        d_obs = fwi.fwi_traces(vt_t, survey)
    v = torch.from_numpy(v0).cuda()
    J0, g = fwi.misfit_and_gradient(v, survey, d_obs)
    assert torch.isfinite(g).all() and float(J0) > 0
    # the torch.autograd path (FwiTraces + a torch loss) gives the same gradient
    va = v.clone().requires_grad_(True)
    Ja = 0.5 * torch.sum((fwi.fwi_traces(va, survey) - d_obs) ** 2)
    Ja.backward()
    assert abs(float(Ja) - float(J0)) <= 1e-9 * float(J0)
    assert float((va.grad - g).norm() / g.norm()) <= 1e-5

    def J(vv):
        with torch.no_grad():
            return float(0.5 * torch.sum((fwi.fwi_traces(vv, survey) - d_obs) ** 2))

    # central differences at eps and eps/2, Richardson-extrapolated to remove
    # the eps^2 term (large here: the misfit is small, so the first derivative
    # of J is small against its third)
    errs, big = [], 0
    for k in range(8):
        dv = synth.smooth_random_field(shape, 3, 1200 + k).astype(np.float64)
        dv[:2] = dv[-2:] = 0
        dv[:, :2] = dv[:, -2:] = 0
        dv[:, :, :2] = dv[:, :, -2:] = 0
        dv *= 20.0 / np.abs(dv).max()
        dvt = torch.from_numpy(dv.astype(np.float32)).cuda()
        lin = float(torch.sum(g.double() * dvt.double()))
        scale = float(g.double().norm()) * float(np.linalg.norm(dv))
        fd = {}
        for eps in (0.5, 0.25):
            fd[eps] = (J(v + eps * dvt) - J(v - eps * dvt)) / (2 * eps)
        rich = (4 * fd[0.25] - fd[0.5]) / 3
        errs.append(abs(rich - lin) / max(abs(lin), 1e-2 * scale))
        big += abs(lin) > 1e-2 * scale
    assert max(errs) < 2e-2, errs
    assert big >= 5


@pytest.mark.parametrize("n", [0, 1, 2047, 2048, 2049, 1_000_003])
def test_misfit_matches_numpy_and_is_deterministic(fdw, n):
    """fdw_misfit: residual d - d_obs exactly, J = 1/2 sum r^2 to FP64
    rounding, and the same bits on every call."""
    import torch
    rng = np.random.default_rng(n)
    d = rng.standard_normal(n)
    o = rng.standard_normal(n)
    dt, ot = torch.from_numpy(d).cuda(), torch.from_numpy(o).cuda()
    res = torch.empty_like(dt)
    J1 = float(fdw.misfit(dt, ot, residual=res))
    J2 = float(fdw.misfit(dt, ot))
    np.testing.assert_array_equal(res.cpu().numpy(), d - o)
    exp = 0.5 * float(np.sum((d - o) ** 2))
    assert J1 == J2
    assert abs(J1 - exp) <= 1e-12 * max(exp, 1e-300)
    with pytest.raises(ValueError):
        fdw.misfit(dt.float(), ot)


def test_full_size_gradient(fdw):
    """The benchmark's FWI workload (256^3 + 40-point sponge, order 8, 2000
    steps) for two of its shots, in the benchmark's configuration: the
    gradient with 20 checkpoints per shot equals the one with 13 (the
    replays recompute the same forward states; only the order of the FP32
    segment sums changes), and along two smooth model perturbations inside
    the physical grid it matches Richardson-extrapolated central
    differences of the misfit."""
    import torch
    from paper_1608_03984_gb300 import fwi
    w = synth.fwi()
    vref = 1.1 * float(max(w.v_true.max(), w.v_start.max()))

    def survey(ck):
        return fwi.Survey(w.n, w.h, w.nb, w.order, w.dt, w.nt, w.src_xyz[5:7], w.wavelet, w.rec_xyz,
                          checkpoints=ck, sponge_vref=vref)

    sv = survey(20)
    with torch.no_grad():
        d_obs = fwi.fwi_traces(torch.from_numpy(w.v_true).cuda(), sv)
    v = torch.from_numpy(w.v_start).cuda()
    J0, g = fwi.misfit_and_gradient(v, sv, d_obs)
    J1, g1 = fwi.misfit_and_gradient(v, survey(13), d_obs)
    assert torch.isfinite(g).all() and float(J0) > 0
    assert abs(float(J1) - float(J0)) <= 1e-12 * float(J0)
    assert float((g1 - g).double().norm() / g.double().norm()) <= 1e-5

    def J(vv):
        with torch.no_grad():
            return float(0.5 * torch.sum((fwi.fwi_traces(vv, sv).double() - d_obs.double()) ** 2))

    n = w.n[0]
    for k in range(2):
        dv = synth.smooth_random_field(w.n, 12, 2100 + k).astype(np.float64)
        ramp = np.minimum(np.arange(n), np.arange(n)[::-1]).astype(np.float64)
        ramp = np.clip(ramp / 16.0, 0.0, 1.0)  # zero at the faces of the physical grid
        dv *= ramp[:, None, None] * ramp[None, :, None] * ramp[None, None, :]
        dv *= 20.0 / np.abs(dv).max()
        dvt = torch.from_numpy(dv.astype(np.float32)).cuda()
        lin = float(torch.sum(g.double() * dvt.double()))
        fd = {}
        for eps in (0.5, 0.25):
            fd[eps] = (J(v + eps * dvt) - J(v - eps * dvt)) / (2 * eps)
        rich = (4 * fd[0.25] - fd[0.5]) / 3
        assert abs(rich - lin) <= 3e-2 * abs(lin), (k, rich, lin)


def test_velocity_gradient_chain_rule(fdw):
    """fdw_velocity_gradient: dJ/dv = -2 v^-3 dJ/dm (m = 1/v^2) elementwise,
    against the same rule in FP64 numpy, also when the output aliases the
    input gradient."""
    import torch
    rng = np.random.default_rng(5)
    v = rng.uniform(1500.0, 4500.0, size=(7, 9, 11)).astype(np.float32)
    gm = rng.standard_normal(v.shape)
    want = -2.0 * gm / v.astype(np.float64) ** 3
    vt, gt = torch.from_numpy(v).cuda(), torch.from_numpy(gm).cuda()
    got = fdw.velocity_gradient(vt, gt).cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=1e-15, atol=0)
    fdw.velocity_gradient(vt, gt, out=gt)
    np.testing.assert_allclose(gt.cpu().numpy(), want, rtol=1e-15, atol=0)
