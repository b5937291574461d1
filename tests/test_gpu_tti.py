"""GPU parity of the TTI step (Eq. TTI with Eq. DiffOp and the sponge)
against the FP64 oracle, through the C ABI. Same tolerances as acoustic."""
import numpy as np
import pytest

from paper_1608_03984_gb300 import synth

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-5
RUN_TOL = 1e-4


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def tti_solver(fdw, w, storage="f32"):
    s = fdw.Solver(w.n, w.h, w.nb, w.order, equation="tti", storage=storage)
    s.set_model(w.vp, w.eps, w.delta, w.theta, w.phi).set_dt(w.dt)
    s.set_sources(w.src_xyz, w.wavelet).set_receivers(w.rec_xyz, w.nt)
    return s


def tti_setup(O, w):
    return O.Setup(w.vp, w.h, w.nb, w.order, w.dt, eps=w.eps, delta=w.delta, theta=w.theta,
                   phi=w.phi)


def small_tti(n=(26, 21, 35), order=8, nt=12, seed=None):
    w = synth.random_tti(n=max(n), nb=5, order=order, nt=nt, nrec_side=5, seed=seed)
    nz, ny, nx = n
    for f in ("vp", "eps", "delta", "theta", "phi"):
        setattr(w, f, np.ascontiguousarray(getattr(w, f)[:nz, :ny, :nx]))
    w.n = n
    w.src_xyz = np.array([[(nx - 1) * w.h * 0.4, (ny - 1) * w.h * 0.6, (nz - 1) * w.h * 0.5]])
    w.rec_xyz = w.rec_xyz[(w.rec_xyz[:, 0] <= (nx - 1) * w.h) & (w.rec_xyz[:, 1] <= (ny - 1) * w.h)]
    return w


@pytest.mark.parametrize("order", [4, 8, 12])
def test_one_step_parity(fdw, O, order):
    w = small_tti(order=order, seed=50 + order)
    s = tti_solver(fdw, w)
    comp = s.comp_shape
    fields = [synth.random_wavefield(comp, 90 + i + order, scale=1e-3) for i in range(4)]
    for (f, lvl), a in zip([(0, 0), (0, 1), (1, 0), (1, 1)], fields):
        s.set_wavefield(a, f, lvl)
    k = 3
    s.set_current_step(k)
    s.step(1)
    got_p, got_r = s.wavefield(0, 0), s.wavefield(1, 0)
    s.check()
    pp, rp = O.tti_step(tti_setup(O, w), fields[0], fields[1], fields[2], fields[3], w.src_xyz,
                        float(w.wavelet[k, 0]))
    assert rel(got_p, pp) <= STEP_TOL, rel(got_p, pp)
    assert rel(got_r, rp) <= STEP_TOL, rel(got_r, rp)
    tr = s.traces()
    np.testing.assert_allclose(tr[k + 1], O.interpolate(pp, w.rec_xyz, w.h, w.nb), rtol=0,
                               atol=1e-5 * np.abs(pp).max())
    s.close()


def test_tti_run(fdw, O):
    w = small_tti(order=8, nt=40, seed=77)
    s = tti_solver(fdw, w)
    s.step(w.nt)
    ref = O.tti_forward(tti_setup(O, w), w.src_xyz, w.wavelet, w.nt, w.rec_xyz)
    assert rel(s.traces(), ref["traces"]) <= RUN_TOL
    assert rel(s.wavefield(0, 0), ref["p"]) <= RUN_TOL
    assert rel(s.wavefield(1, 0), ref["r"]) <= RUN_TOL
    assert rel(s.wavefield(1, 1), ref["rm"]) <= RUN_TOL
    s.close()


@pytest.mark.parametrize("order", [2, 6, 10, 16])
def test_tma_kernel_matches_point_kernel(fdw, O, order):
    """The 2.5D TTI kernel (factored cross derivatives, register queues)
    agrees with the one-thread-per-point kernel (direct tensor-product cross
    stencils) and with the oracle, on a grid with ragged tails."""
    w = small_tti(n=(29, 19, 70), order=order, nt=10, seed=60 + order)
    out = []
    for variant in (0, 1):
        s = tti_solver(fdw, w)
        s.set_kernel_variant(variant)
        s.step(w.nt)
        out.append((s.wavefield(0, 0), s.wavefield(1, 0)))
        s.check()
        s.close()
    assert rel(out[0][0], out[1][0]) <= 1e-5
    assert rel(out[0][1], out[1][1]) <= 1e-5
    ref = O.tti_forward(tti_setup(O, w), w.src_xyz, w.wavelet, w.nt)
    assert rel(out[0][0], ref["p"]) <= RUN_TOL
    assert rel(out[0][1], ref["r"]) <= RUN_TOL


def test_isotropic_tti_equals_acoustic(fdw):
    """eps = delta = 0: p = r = the acoustic solution for any tilt."""
    w = small_tti(order=8, nt=25, seed=78)
    w.eps = np.zeros_like(w.eps)
    w.delta = np.zeros_like(w.delta)
    s = tti_solver(fdw, w)
    s.step(w.nt)
    a = fdw.Solver(w.n, w.h, w.nb, w.order)
    a.set_model(w.vp).set_dt(w.dt).set_sources(w.src_xyz, w.wavelet).step(w.nt)
    ua = a.wavefield(0, 0)
    assert rel(s.wavefield(0, 0), ua) <= 1e-5
    assert rel(s.wavefield(1, 0), ua) <= 1e-5
    s.close()
    a.close()


def test_vti_matches_oracle(fdw, O):
    """VTI (Eq. vVTI, D_xx read as the horizontal Laplacian) through the
    binding's "vti" equation: the TTI step with a vertical axis."""
    w = small_tti(order=8, nt=30, seed=81)
    s = fdw.Solver(w.n, w.h, w.nb, w.order, equation="vti")
    s.set_model(w.vp, w.eps, w.delta).set_dt(w.dt)
    s.set_sources(w.src_xyz, w.wavelet).set_receivers(w.rec_xyz, w.nt)
    s.step(w.nt)
    z = np.zeros_like(w.theta)
    ref = O.tti_forward(O.Setup(w.vp, w.h, w.nb, w.order, w.dt, eps=w.eps, delta=w.delta,
                                theta=z, phi=z), w.src_xyz, w.wavelet, w.nt, w.rec_xyz)
    assert rel(s.traces(), ref["traces"]) <= RUN_TOL
    assert rel(s.wavefield(0, 0), ref["p"]) <= RUN_TOL
    assert rel(s.wavefield(1, 0), ref["r"]) <= RUN_TOL
    s.close()


ROW_PAIR_TILES = (9, 10, 11, 12)  # two rows per thread, orders up to 8
NTILES = 13


@pytest.mark.parametrize("order", [2, 8, 12, 16])
@pytest.mark.parametrize("tile", list(range(NTILES)))
def test_every_tti_configuration(fdw, O, order, tile):
    """Each (warps per CTA, z unrolling, variant) configuration of the TTI
    kernel reproduces the oracle's step (ragged tile tails in x, y and z),
    and a few more steps stay finite. The two-rows-per-thread
    configurations exist up to order 8 and are refused above."""
    w = small_tti(n=(23, 13, 37), order=order, seed=70 + order)
    s = tti_solver(fdw, w)
    if tile in ROW_PAIR_TILES and order > 8:
        with pytest.raises(fdw.FdwError):
            s.set_tile_config(tile)
        s.close()
        return
    s.set_tile_config(tile)
    assert s.tile_config == tile
    comp = s.comp_shape
    fields = [synth.random_wavefield(comp, 110 + i + order, scale=1e-3) for i in range(4)]
    for (f, lvl), a in zip([(0, 0), (0, 1), (1, 0), (1, 1)], fields):
        s.set_wavefield(a, f, lvl)
    s.set_current_step(2)
    s.step(1)
    pp, rp = O.tti_step(tti_setup(O, w), fields[0], fields[1], fields[2], fields[3], w.src_xyz,
                        float(w.wavelet[2, 0]))
    assert rel(s.wavefield(0, 0), pp) <= STEP_TOL
    assert rel(s.wavefield(1, 0), rp) <= STEP_TOL
    s.step(3)
    s.check()
    s.close()


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("order", [6, 12])
def test_16bit_tti_configurations(fdw, storage, order):
    """With 16-bit storage every TTI configuration that exists at the order
    gives the fields of configuration 0 (scalar kernel) up to the storage
    type's rounding where the FP32 sums differ in order (ragged grid,
    several steps)."""
    w = small_tti(n=(23, 13, 37), order=order, seed=170 + order)
    comp = None
    out = {}
    for t in range(13):
        if t in ROW_PAIR_TILES and order > 8:
            continue
        s = tti_solver(fdw, w, storage=storage)
        s.set_tile_config(t)
        comp = s.comp_shape
        for i, (f, lvl) in enumerate([(0, 0), (0, 1), (1, 0), (1, 1)]):
            s.set_wavefield(synth.random_wavefield(comp, 120 + i + order, scale=1e-3), f, lvl)
        s.set_current_step(2)
        s.step(3)
        s.check()
        out[t] = (s.wavefield(0, 0), s.wavefield(1, 0))
        s.close()
    tol = {"bf16": 2e-2, "f16": 3e-3}[storage]
    for t, (p, r) in out.items():
        assert rel(p, out[0][0]) <= tol, (t, rel(p, out[0][0]))
        assert rel(r, out[0][1]) <= tol, (t, rel(r, out[0][1]))


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_row_pair_kernel_same_bits(fdw, order, storage):
    """Two rows per thread and the z unrolling change which thread computes
    a point and when, not its arithmetic: the field-pair configurations give
    the same bits (ragged tails in x, y and z, several steps with a
    source)."""
    w = small_tti(n=(29, 19, 41), order=order, nt=6, seed=90 + order)
    out = {}
    same = ((7, 12), (8, 10), (7, 8), (7, 9))
    for tile in sorted({t for p in same for t in p}):
        s = tti_solver(fdw, w, storage=storage)
        s.set_tile_config(tile)
        s.step(w.nt)
        out[tile] = (s.wavefield(0, 0), s.wavefield(1, 0), s.traces())
        s.check()
        s.close()
    for a, b in same:
        for x, y in zip(out[a], out[b]):
            assert np.array_equal(x, y), (a, b)
    assert np.abs(out[7][0]).max() > 0


@pytest.mark.parametrize("order", [8, 12])
def test_full_size_sampled_step(fdw, O, order):
    """384^3 + 40-point sponge (464^3), orders 8 and 12 in the launch
    configuration of the benchmark's TTI workload: one step from random p,
    r levels, checked at sampled points (interior, sponge, faces, corners)
    by the oracle's TTI point update with that point's medium."""
    import torch
    w = synth.random_tti(n=384, nb=40, order=order, nt=8, nrec_side=16)
    s = tti_solver(fdw, w)
    comp = s.comp_shape
    g = torch.Generator(device="cuda").manual_seed(4321)
    lv = [1e-3 * torch.randn(comp, generator=g, device="cuda", dtype=torch.float32) for _ in range(4)]
    for (f, lvl), a in zip([(0, 0), (0, 1), (1, 0), (1, 1)], lv):
        s.set_wavefield(a, f, lvl)
    s.set_current_step(3)
    s.set_sources(np.zeros((0, 3)), None)
    s.step(1)
    pp = torch.empty_like(lv[0])
    rp = torch.empty_like(lv[0])
    s.wavefield(0, 0, out=pp)
    s.wavefield(1, 0, out=rp)
    s.check()
    torch.cuda.synchronize()
    r = w.order // 2
    rng = np.random.default_rng(1)
    N = np.array(comp)
    pts = [tuple(int(v) for v in rng.integers(0, N)) for _ in range(40)]
    pts += [(0, 0, 0), tuple(int(v) for v in N - 1), (int(N[0]) // 2, int(N[1]) // 2, int(N[2]) // 2),
            (3, int(N[1]) - 2, 40), (int(N[0]) - 1, 0, int(N[2]) // 3), (39, 40, 41), (40, 40, 40)]
    setup = tti_setup(O, w)
    pad = [torch.nn.functional.pad(a.view(1, 1, *comp), (r,) * 6)[0, 0] for a in (lv[0], lv[2])]
    worst = 0.0
    for (k, j, i) in pts:
        sl = (slice(k, k + 2 * r + 1), slice(j, j + 2 * r + 1), slice(i, i + 2 * r + 1))
        pb, rb = (a[sl].double().cpu().numpy() for a in pad)
        v_c = float(np.sqrt(setup.c[k, j, i])) / w.dt
        gam = setup.gx[i] + setup.gy[j] + setup.gz[k]
        ep, er = O.tti_update_at(pb, float(lv[1][k, j, i]), rb, float(lv[3][k, j, i]), v_c,
                                 setup.eps[k, j, i], setup.delta[k, j, i], setup.theta[k, j, i],
                                 setup.phi[k, j, i], gam, w.h, w.order, w.dt)
        scale = max(np.abs(pb).max(), np.abs(rb).max())
        worst = max(worst, abs(float(pp[k, j, i]) - ep) / scale, abs(float(rp[k, j, i]) - er) / scale)
    assert worst < 1e-5, worst
    s.close()


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_full_size_sampled_step_16bit(fdw, O, storage):
    """The 464^3 TTI workload with 16-bit storage (order 8, the benchmark's
    launch configuration): one step from random p, r levels, checked at
    sampled points by the oracle's FP64 TTI point update of the stored
    (rounded) input levels with the exact medium. The bound covers one
    rounding of the stored output and the rounding of the stored medium
    (c, 1 + 2 eps, sqrt(1 + 2 delta), the axis): a few units of 2^-9 (BF16)
    or 2^-12 (FP16) of the largest input, the operator terms being up to
    ~10 times that input at CFL 0.4."""
    import torch
    w = synth.random_tti(n=384, nb=40, order=8, nt=8, nrec_side=16)
    s = tti_solver(fdw, w, storage)
    comp = s.comp_shape
    g = torch.Generator(device="cuda").manual_seed(987)
    for f in (0, 1):
        for lvl in (0, 1):
            s.set_wavefield(1e-3 * torch.randn(comp, generator=g, device="cuda", dtype=torch.float32), f, lvl)
    lv = [torch.empty(comp, device="cuda", dtype=torch.float32) for _ in range(4)]
    for (f, lvl), a in zip([(0, 0), (0, 1), (1, 0), (1, 1)], lv):
        s.wavefield(f, lvl, out=a)  # the stored values, as the kernel reads them
    s.set_current_step(3)
    s.set_sources(np.zeros((0, 3)), None)
    s.step(1)
    pp = torch.empty_like(lv[0])
    rp = torch.empty_like(lv[0])
    s.wavefield(0, 0, out=pp)
    s.wavefield(1, 0, out=rp)
    s.check()
    torch.cuda.synchronize()
    r = w.order // 2
    rng = np.random.default_rng(2)
    N = np.array(comp)
    pts = [tuple(int(v) for v in rng.integers(0, N)) for _ in range(30)]
    pts += [(0, 0, 0), tuple(int(v) for v in N - 1), (int(N[0]) // 2, int(N[1]) // 2, int(N[2]) // 2),
            (39, 40, 41), (40, 40, 40)]
    setup = tti_setup(O, w)
    pad = [torch.nn.functional.pad(a.view(1, 1, *comp), (r,) * 6)[0, 0] for a in (lv[0], lv[2])]
    worst = 0.0
    for (k, j, i) in pts:
        sl = (slice(k, k + 2 * r + 1), slice(j, j + 2 * r + 1), slice(i, i + 2 * r + 1))
        pb, rb = (a[sl].double().cpu().numpy() for a in pad)
        v_c = float(np.sqrt(setup.c[k, j, i])) / w.dt
        gam = setup.gx[i] + setup.gy[j] + setup.gz[k]
        ep, er = O.tti_update_at(pb, float(lv[1][k, j, i]), rb, float(lv[3][k, j, i]), v_c,
                                 setup.eps[k, j, i], setup.delta[k, j, i], setup.theta[k, j, i],
                                 setup.phi[k, j, i], gam, w.h, w.order, w.dt)
        scale = max(np.abs(pb).max(), np.abs(rb).max())
        worst = max(worst, abs(float(pp[k, j, i]) - ep) / scale, abs(float(rp[k, j, i]) - er) / scale)
    tol = {"bf16": 5e-2, "f16": 6e-3}[storage]
    assert worst < tol, worst
    print("worst relative deviation (%s): %.3g" % (storage, worst))
    s.close()
