"""GPU parity of the acoustic step (Algorithm 1 with Eq. Acou and the sponge)
against the FP64 oracle, through the C ABI.

Tolerances (FP32 storage and arithmetic): relative L2 <= 1e-5 for one step
from a given state, <= 1e-4 after a full run.
"""
import math

import numpy as np
import pytest

from paper_1608_03984_gb300 import synth

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-5
RUN_TOL = 1e-4


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def random_problem(shape=(30, 27, 41), nb=6, order=8, h=10.0, seed=0, nt=16):
    vp = synth.random_velocity(shape, h, 60.0, 700 + seed)
    dt = 0.4 * h / float(vp.max())
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    src = np.array([[(nx - 1) * h * 0.43, (ny - 1) * h * 0.57, (nz - 1) * h * 0.31]])
    rec = rng.uniform([-nb * h, -nb * h, -nb * h],
                      [(nx - 1 + nb) * h, (ny - 1 + nb) * h, (nz - 1 + nb) * h], size=(23, 3))
    w = synth.ricker(25.0, dt, nt).astype(np.float32).reshape(nt, 1)
    return dict(vp=vp, h=h, nb=nb, order=order, dt=dt, src=src, rec=rec, w=w, nt=nt)


def make_solver(fdw, P, storage="f32"):
    nz, ny, nx = P["vp"].shape
    s = fdw.Solver((nz, ny, nx), P["h"], P["nb"], P["order"], storage=storage)
    s.set_model(P["vp"]).set_dt(P["dt"]).set_sources(P["src"], P["w"]).set_receivers(P["rec"], P["nt"])
    return s


def oracle_setup(O, P):
    return O.Setup(P["vp"], P["h"], P["nb"], P["order"], P["dt"])


@pytest.mark.parametrize("order", [2, 4, 6, 8, 10, 12, 14, 16])
def test_one_step_parity(fdw, O, order):
    """One step from a random state (several tiles in x/y/z, ragged tails,
    sponge, an injecting source at step k) against the oracle's step."""
    P = random_problem(order=order, seed=order)
    s = make_solver(fdw, P)
    comp = s.comp_shape
    u = synth.random_wavefield(comp, 11 + order, scale=1e-3)
    um = synth.random_wavefield(comp, 12 + order, scale=1e-3)
    k = 5
    s.set_wavefield(u, 0, 0)
    s.set_wavefield(um, 0, 1)
    s.set_current_step(k)
    s.step(1)
    got = s.wavefield(0, 0)
    prev = s.wavefield(0, 1)
    tr = s.traces()
    s.check()
    exp = O.acoustic_step(oracle_setup(O, P), u, um, P["src"], float(P["w"][k, 0]))
    assert rel(got, exp) <= STEP_TOL, rel(got, exp)
    np.testing.assert_array_equal(prev, u)  # level n is untouched
    exp_tr = O.interpolate(exp, P["rec"], P["h"], P["nb"])
    np.testing.assert_allclose(tr[k + 1], exp_tr, rtol=0, atol=1e-5 * np.abs(exp).max())
    s.close()


def test_two_layer_full_run(fdw, O):
    """The 64^3 two-layer workload (order 4, 200 steps, Ricker 15 Hz at the
    centre, 32 receivers at 20 m depth): traces and final wavefield."""
    w = synth.two_layer()
    s = fdw.Solver(w.n, w.h, w.nb, w.order)
    s.set_model(w.vp).set_dt(w.dt).set_sources(w.src_xyz, w.wavelet).set_receivers(w.rec_xyz, w.nt)
    s.step(w.nt)
    tr = s.traces()
    u = s.wavefield(0, 0)
    s.check()
    ref = O.acoustic_forward(O.Setup(w.vp, w.h, w.nb, w.order, w.dt), w.src_xyz, w.wavelet, w.nt,
                             w.rec_xyz)
    assert rel(tr, ref["traces"]) <= RUN_TOL
    assert rel(u, ref["u"]) <= RUN_TOL
    assert s.current_step == w.nt
    s.close()


@pytest.mark.parametrize("order", [4, 16])
def test_random_medium_run(fdw, O, order):
    """40 steps in a random medium with sponge, traces and both levels."""
    P = random_problem(shape=(33, 29, 37), nb=8, order=order, seed=3, nt=40)
    s = make_solver(fdw, P)
    s.step(P["nt"])
    ref = O.acoustic_forward(oracle_setup(O, P), P["src"], P["w"], P["nt"], P["rec"])
    assert rel(s.traces(), ref["traces"]) <= RUN_TOL
    assert rel(s.wavefield(0, 0), ref["u"]) <= RUN_TOL
    assert rel(s.wavefield(0, 1), ref["um"]) <= RUN_TOL
    s.close()


@pytest.mark.parametrize("order", [2, 8, 16])
def test_tma_kernel_matches_point_kernel(fdw, order):
    """The 2.5D TMA kernel and the one-thread-per-point kernel agree."""
    P = random_problem(shape=(45, 38, 70), nb=5, order=order, seed=9, nt=12)
    out = []
    for variant in (0, 1):
        s = make_solver(fdw, P)
        s.set_kernel_variant(variant)
        s.step(P["nt"])
        out.append(s.wavefield(0, 0))
        s.close()
    assert rel(out[0], out[1]) <= 1e-6


def test_zchunks_do_not_change_the_result(fdw):
    P = random_problem(shape=(50, 20, 33), nb=4, order=12, seed=4, nt=6)
    res = []
    for zc in (1, 2, 3, 7, 0):
        s = make_solver(fdw, P)
        s.set_zchunks(zc)
        s.step(P["nt"])
        res.append(s.wavefield(0, 0))
        s.close()
    for r in res[1:]:
        np.testing.assert_array_equal(r, res[0])


@pytest.mark.parametrize("shape,nb,order", [((1, 1, 1), 0, 2), ((3, 2, 5), 0, 16), ((7, 40, 3), 1, 8),
                                            ((2, 2, 70), 3, 4), ((17, 16, 32), 0, 6)])
def test_small_and_degenerate_grids(fdw, O, shape, nb, order):
    """Grids narrower than the stencil, a single point, no sponge."""
    P = random_problem(shape=shape, nb=nb, order=order, seed=5, nt=5)
    P["rec"] = P["rec"][:3]
    s = make_solver(fdw, P)
    s.step(P["nt"])
    ref = O.acoustic_forward(oracle_setup(O, P), P["src"], P["w"], P["nt"], P["rec"])
    assert rel(s.wavefield(0, 0), ref["u"]) <= RUN_TOL
    assert rel(s.traces(), ref["traces"]) <= RUN_TOL
    s.close()


def test_reset_and_replay_bit_identical(fdw):
    P = random_problem(seed=6, nt=20)
    s = make_solver(fdw, P)
    s.step(P["nt"])
    a = s.traces().copy()
    s.reset()
    s.step(P["nt"])
    np.testing.assert_array_equal(s.traces(), a)
    s.close()


def test_errors(fdw):
    P = random_problem(seed=7)
    nz, ny, nx = P["vp"].shape
    with pytest.raises(fdw.FdwError) as e:
        fdw.Solver((nz, ny, nx), 10.0, 2, 5)
    assert e.value.code == -1
    s = fdw.Solver((nz, ny, nx), P["h"], P["nb"], P["order"])
    with pytest.raises(fdw.FdwError) as e:
        s.set_dt(1e-3)
    assert e.value.code == -5                      # dt before model
    s.set_model(P["vp"])
    with pytest.raises(fdw.FdwError) as e:
        s.step(1)
    assert e.value.code == -5                      # step before dt
    with pytest.raises(fdw.FdwError) as e:
        s.set_dt(1.01 * s.max_stable_dt())
    assert e.value.code == -2                      # CFL (Eq. stability)
    s.set_dt(s.max_stable_dt())
    with pytest.raises(fdw.FdwError) as e:
        s.set_receivers([[1e6, 0.0, 0.0]], 10)
    assert e.value.code == -7
    with pytest.raises(fdw.FdwError) as e:
        s.set_sources([[-1e3, 0.0, 0.0]], np.zeros(4, np.float32))
    assert e.value.code == -7
    bad = P["vp"].copy()
    bad[3, 4, 5] = -1.0
    with pytest.raises(fdw.FdwError) as e:
        s.set_model(bad)
    assert e.value.code == -1
    with pytest.raises(fdw.FdwError):
        s.step(1)                                  # the model was rejected
    s.close()


def test_cfl_limit_matches_eq_stability(fdw):
    """fdw_max_stable_dt = h sqrt(4/a2) / vmax with a2 from Table tab:stab."""
    a2 = {2: 12.0, 16: 22.28076431505002}
    for order, val in a2.items():
        s = fdw.Solver((8, 8, 8), 10.0, 1, order)
        s.set_model(np.full((8, 8, 8), 2500.0, np.float32))
        assert s.max_stable_dt() == pytest.approx(10.0 * math.sqrt(4 / val) / 2500.0, rel=1e-12)
        s.close()


def test_divergence_watchdog(fdw):
    """dt at the CFL limit of order 2 with a broken (too large) model after
    set_dt is impossible through the API; a non-finite state is caught."""
    P = random_problem(seed=8)
    s = make_solver(fdw, P)
    u = np.zeros(s.comp_shape, np.float32)
    u[5, 6, 7] = np.inf
    s.set_wavefield(u, 0, 0)
    with pytest.raises(fdw.FdwError) as e:
        s.check(finite=True)
    assert e.value.code == -6
    s.close()


@pytest.mark.parametrize("order", [2, 4, 8, 12, 16])
def test_full_size_sampled_step(fdw, O, order):
    """512^3 + 40-point sponge (592^3), each order of the benchmark in its
    launch configuration (default tile and z chunks): one step from a
    random state, checked at sampled points (interior, sponge, faces,
    corners) by the oracle's point update."""
    import torch
    w = synth.random_acoustic(n=512, order=order, nt=8, nrec_side=16)
    s = fdw.Solver(w.n, w.h, w.nb, w.order)
    s.set_model(w.vp).set_dt(w.dt).set_receivers(w.rec_xyz, w.nt)
    comp = s.comp_shape
    g = torch.Generator(device="cuda").manual_seed(1234)
    u = 1e-3 * torch.randn(comp, generator=g, device="cuda", dtype=torch.float32)
    um = 1e-3 * torch.randn(comp, generator=g, device="cuda", dtype=torch.float32)
    s.set_wavefield(u, 0, 0)
    s.set_wavefield(um, 0, 1)
    s.step(1)
    up = torch.empty_like(u)
    s.wavefield(0, 0, out=up)
    s.check()
    torch.cuda.synchronize()
    r = w.order // 2
    rng = np.random.default_rng(0)
    N = np.array(comp)
    pts = [tuple(int(v) for v in rng.integers(0, N)) for _ in range(48)]
    pts += [(0, 0, 0), tuple(int(v) for v in N - 1), (int(N[0]) // 2, int(N[1]) // 2, int(N[2]) // 2),
            (3, int(N[1]) - 2, 40), (int(N[0]) - 1, 0, int(N[2]) // 3), (39, 40, 41), (40, 40, 40),
            (0, 300, int(N[2]) - 1), (591, 591, 0)]
    gmax = O.sponge_gamma_max(float(w.vp.max()), w.nb, w.h)
    prof = [O.sponge_profile(n, w.nb, gmax) for n in comp]
    upad = torch.nn.functional.pad(u.view(1, 1, *comp), (r, r, r, r, r, r))[0, 0]
    worst = 0.0
    for (k, j, i) in pts:
        blk = upad[k:k + 2 * r + 1, j:j + 2 * r + 1, i:i + 2 * r + 1].double().cpu().numpy()
        pk, pj, pi = (min(max(a - w.nb, 0), n - 1) for a, n in zip((k, j, i), w.n))
        vc = float(w.vp[pk, pj, pi])
        gam = prof[0][k] + prof[1][j] + prof[2][i]
        exp = O.acoustic_update_at(blk, float(um[k, j, i]), vc, gam, w.h, w.order, w.dt)
        got = float(up[k, j, i])
        worst = max(worst, abs(got - exp) / np.abs(blk).max())
    assert worst < 1e-5, worst
    s.close()


def test_profiled_steps_match_graph_steps(fdw):
    """Steps launched one by one under kernel timing, with several solvers
    interleaved on one stream, are bit-identical to the CUDA-graph steps."""
    P = random_problem(seed=10, nt=30)
    orders = (2, 8, 16)
    a = [make_solver(fdw, dict(P, order=o)) for o in orders]
    b = [make_solver(fdw, dict(P, order=o)) for o in orders]
    for s in a + b:
        s.step(5)
    for s in a:
        s.profile_begin(20)
    for _ in range(20):
        for s in a:
            s.step(1)
    for s in a:
        ms, n = s.profile_end()
        assert n == 20 and ms > 0
    for s in b:
        s.step(20)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x.wavefield(0, 0), y.wavefield(0, 0))
        np.testing.assert_array_equal(x.wavefield(0, 1), y.wavefield(0, 1))
        np.testing.assert_array_equal(x.traces(), y.traces())
    for s in a + b:
        s.close()


@pytest.mark.parametrize("order", [2, 6, 8, 12, 16])
@pytest.mark.parametrize("tile", list(range(13)))
def test_every_tile_configuration(fdw, O, order, tile):
    """Each tile configuration of the 2.5D kernel (points per thread, warps
    per CTA, z unrolling) reproduces the oracle's step on a grid with ragged
    tails in x, y and z."""
    P = random_problem(shape=(37, 19, 141), nb=3, order=order, seed=20 + tile, nt=8)
    s = make_solver(fdw, P)
    s.set_tile_config(tile)
    assert s.tile_config == tile
    comp = s.comp_shape
    u = synth.random_wavefield(comp, 31, scale=1e-3)
    um = synth.random_wavefield(comp, 32, scale=1e-3)
    s.set_wavefield(u, 0, 0)
    s.set_wavefield(um, 0, 1)
    s.set_current_step(2)
    s.step(1)
    exp = O.acoustic_step(oracle_setup(O, P), u, um, P["src"], float(P["w"][2, 0]))
    assert rel(s.wavefield(0, 0), exp) <= STEP_TOL
    s.step(3)
    s.check()
    s.close()


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("tile", list(range(1, 13)))
def test_16bit_tile_configurations(fdw, storage, tile):
    """With 16-bit storage every tile configuration gives the fields of
    configuration 0 (one point per thread) up to one rounding of the stored
    type where the FP32 sums differ in order (ragged grid, order 16)."""
    P = random_problem(shape=(37, 19, 141), nb=3, order=16, seed=40 + tile, nt=8)
    out = []
    for t in (0, tile):
        s = make_solver(fdw, P, storage=storage)
        s.set_tile_config(t)
        comp = s.comp_shape
        s.set_wavefield(synth.random_wavefield(comp, 41, scale=1e-3), 0, 0)
        s.set_wavefield(synth.random_wavefield(comp, 42, scale=1e-3), 0, 1)
        s.set_current_step(2)
        s.step(4)
        s.check()
        out.append((s.wavefield(0, 0), s.wavefield(0, 1)))
        s.close()
    tol = {"bf16": 8e-3, "f16": 1e-3}[storage]
    for a, b in zip(out[0], out[1]):
        assert rel(b, a) <= tol
