"""The learned closure on the GPU: training kernels (forward, loss,
parameter gradient, Adam) and the closure step of the time loop against the
FP64 oracle, and the trained network's gain over the coarse solver alone.
What is compared is the correction net(x) - net(x0) (x0: the same input
with the wavefield channels zeroed).

The kernels use BF16 copies of the convolution weights (biases stay FP32)
and accumulate in FP32; the oracle gets the same BF16-rounded weights, so
the remaining difference is FP32 rounding of sums of at most 16*27 = 432
products (relative ~1e-6)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

H = 16
NW = (H * 3 * 27, H, H * H * 27, H, H * 27, 1)  # W1 b1 W2 b2 W3 b3


def bf16_weights(p):
    """Round the convolution weights (not the biases) to BF16, nearest-even."""
    import torch
    p = np.asarray(p, dtype=np.float32).copy()
    i = 0
    for k, n in enumerate(NW):
        if k % 2 == 0:
            p[i:i + n] = torch.from_numpy(p[i:i + n]).to(torch.bfloat16).float().numpy()
        i += n
    return p


def random_params(seed, scale=1.0):
    from paper_1608_03984_gb300 import closure
    p = closure.init_params(seed, last_scale=scale)
    rng = np.random.default_rng(seed + 1)
    # non-zero biases exercise the bias gradients
    i = 0
    for k, n in enumerate(NW):
        if k % 2 == 1:
            p[i:i + n] = 0.1 * rng.standard_normal(n)
        i += n
    return bf16_weights(p)


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("B,S", [(1, 7), (3, 10), (8, 18)])
def test_forward_matches_oracle(fdw, O, torch_mod, B, S):
    torch = torch_mod
    p = random_params(B)
    rng = np.random.default_rng(S)
    x = rng.standard_normal((B, 3, S, S, S)).astype(np.float32)
    net = fdw.Closure()
    net.set_params(p)
    out = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    for b in range(B):
        ref = O.closure_correction(p.astype(np.float64), x[b].astype(np.float64))
        assert rel(out[b], ref) < 1e-5, b
    net.close()


@pytest.mark.parametrize("B,S", [(1, 7), (3, 10), (8, 18)])
def test_loss_and_gradient_match_oracle(fdw, O, torch_mod, B, S):
    """Loss and the full parameter gradient (8673 values) of the correction
    net(x) - net(x0) against the oracle, whose gradient is pinned to central
    differences."""
    torch = torch_mod
    p = random_params(10 + B)
    rng = np.random.default_rng(20 + S)
    x = rng.standard_normal((B, 3, S, S, S)).astype(np.float32)
    t = rng.standard_normal((B, S - 6, S - 6, S - 6)).astype(np.float32)
    net = fdw.Closure()
    net.set_params(p)
    loss, g = net.loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    ref_loss, ref_g = O.closure_correction_loss_grad(p.astype(np.float64), x.astype(np.float64),
                                                     t.astype(np.float64))
    assert abs(float(loss) - ref_loss) <= 2e-6 * ref_loss
    g = g.cpu().numpy()
    assert rel(g, ref_g) < 1e-4
    i = 0
    # every block of the gradient, not only the bulk; b3's gradient is zero
    # (it cancels in net(x) - net(x0)), so blocks are measured against the
    # larger of their own norm and 1e-3 of the whole gradient's
    for k, n in enumerate(NW):
        err = np.linalg.norm(g[i:i + n] - ref_g[i:i + n])
        assert err <= 1e-4 * max(np.linalg.norm(ref_g[i:i + n]), 1e-3 * np.linalg.norm(ref_g)), k
        i += n
    net.close()


def test_patch_size_changes_on_one_network(fdw, O, torch_mod):
    """One network fed many small patches, then one large patch (the second
    needs larger layer buffers although it has fewer input points)."""
    torch = torch_mod
    p = random_params(21)
    net = fdw.Closure()
    net.set_params(p)
    rng = np.random.default_rng(22)
    for B, S in ((8, 9), (1, 18), (2, 11)):
        x = rng.standard_normal((B, 3, S, S, S)).astype(np.float32)
        out = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
        for b in range(B):
            ref = O.closure_correction(p.astype(np.float64), x[b].astype(np.float64))
            assert rel(out[b], ref) < 1e-5, (B, S, b)
    net.close()


def test_loss_gradient_is_deterministic(fdw, torch_mod):
    torch = torch_mod
    p = random_params(3)
    rng = np.random.default_rng(9)
    x = torch.from_numpy(rng.standard_normal((6, 3, 16, 16, 16)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal((6, 10, 10, 10)).astype(np.float32)).cuda()
    net = fdw.Closure()
    net.set_params(p)
    l1, g1 = net.loss_grad(x, t)
    l2, g2 = net.loss_grad(x, t)
    assert torch.equal(l1, l2) and torch.equal(g1, g2)
    net.close()


def test_adam_step_matches_update_rule(fdw, torch_mod):
    """Two Adam steps recomputed in FP64 from the gradients the library
    reports at the same parameters (its gradients are deterministic)."""
    torch = torch_mod
    p0 = random_params(4)
    rng = np.random.default_rng(11)
    x = torch.from_numpy(rng.standard_normal((2, 3, 12, 12, 12)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal((2, 6, 6, 6)).astype(np.float32)).cuda()
    net = fdw.Closure()
    net.set_params(p0)
    p = p0.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    lr = 1e-3
    for it in (1, 2):
        _, g = net.loss_grad(x, t)
        g = g.double().cpu().numpy()
        net.adam_step(x, t, lr)
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g * g
        p = p - lr * (m / (1 - 0.9 ** it)) / (np.sqrt(v / (1 - 0.999 ** it)) + 1e-8)
        got = net.get_params()
        np.testing.assert_allclose(got, p, rtol=1e-6, atol=1e-9)
        p = got.astype(np.float64)  # continue from the library's FP32 parameters
    net.close()


def _coarse_case(fdw, O, seed, storage="f32"):
    from paper_1608_03984_gb300 import synth
    n, nb, h, order = 22, 5, 20.0, 4
    vp = synth.random_velocity((n, n + 2, n + 4), h, 120.0, seed)
    dt = 0.35 * h / 4500.0
    solver = fdw.Solver(vp.shape, h, nb, order, storage=storage)
    # unit storage scale: the O(1) random levels fit FP16's range
    solver.set_model(vp).set_sponge(4500.0).set_field_scale(1.0).set_dt(dt)
    src = np.array([[210.0, 190.0, 200.0]])
    wav = (1e3 * synth.ricker(12.0, dt, 20)).astype(np.float32)
    solver.set_sources(src, wav.reshape(-1, 1))
    comp = solver.comp_shape
    u0 = synth.random_wavefield(comp, seed + 1, smooth_pts=2.0).astype(np.float32)
    um = synth.random_wavefield(comp, seed + 2, smooth_pts=2.0).astype(np.float32)
    solver.set_wavefield(u0, 0, 0)
    solver.set_wavefield(um, 0, 1)
    setup = O.Setup(vp, h, nb, order, dt, gamma_vmax=4500.0)
    return solver, setup, vp, src, wav, u0, um


def test_step_closure_matches_oracle(fdw, O):
    """Five coarse steps with the closure's FP32 inference kernels (order 4,
    22 x 24 x 26 physical, sponge 5, a point source, random initial levels)
    against the oracle's closure step on the same BF16-rounded weights."""
    solver, setup, vp, src, wav, u0, um = _coarse_case(fdw, O, 31)
    p = random_params(7, scale=0.3)
    net = fdw.Closure()
    net.set_variant(1)  # FP32 inference kernels
    net.set_params(p)
    ref_u, ref_um = u0.astype(np.float64), um.astype(np.float64)
    for k in range(5):
        solver.step_closure(net, 1)
        nxt = O.closure_step(setup, ref_u, ref_um, vp, p.astype(np.float64), src, [wav[k]])
        ref_um, ref_u = ref_u, nxt
        got = solver.wavefield(0, 0)
        e = rel(got, ref_u)
        assert e < 1e-5 * (k + 1), (k, e)
    # the correction is not negligible: plain steps end far from it
    pu, pum = u0.astype(np.float64), um.astype(np.float64)
    for k in range(5):
        pu, pum = O.acoustic_step(setup, pu, pum, src, [wav[k]]), pu
    assert rel(pu, ref_u) > 1e-2
    assert solver.current_step == 5
    net.close()
    solver.close()


def test_step_closure_every_second_step_matches_oracle(fdw, O):
    """Closure on every second step with the correction doubled
    (fdw_step_closure_every) against the oracle's sequence closure step with
    the last layer times 2 (exact in BF16), plain step, closure step, plain
    step; FP32 inference kernels."""
    from paper_1608_03984_gb300 import closure
    solver, setup, vp, src, wav, u0, um = _coarse_case(fdw, O, 33)
    p = random_params(9, scale=0.3)
    p2 = closure.scale_last_layer(p, 2.0).astype(np.float64)
    net = fdw.Closure()
    net.set_variant(1)
    net.set_params(p)
    solver.step_closure(net, 4, every=2)
    ref_u, ref_um = u0.astype(np.float64), um.astype(np.float64)
    for k in range(4):
        if k % 2 == 0:
            nxt = O.closure_step(setup, ref_u, ref_um, vp, p2, src, [wav[k]])
        else:
            nxt = O.acoustic_step(setup, ref_u, ref_um, src, [wav[k]])
        ref_um, ref_u = ref_u, nxt
    assert rel(solver.wavefield(0, 0), ref_u) < 4e-5
    assert rel(solver.wavefield(0, 1), ref_um) < 4e-5
    assert solver.current_step == 4
    net.close()
    solver.close()


def test_step_closure_every_phase_follows_the_step_count(fdw, O):
    """The every-k closure corrects the steps whose solver step count is a
    multiple of k: two calls of 2 steps with every = 4 give the levels of
    one call of 4 steps (one correction, at step 0), and a call that starts
    at step 2 corrects nothing until step 4."""
    a, *_ = _coarse_case(fdw, O, 45)
    b, *_ = _coarse_case(fdw, O, 45)
    c, *_ = _coarse_case(fdw, O, 45)
    net = fdw.Closure()
    net.set_variant(1)
    net.set_params(random_params(10, scale=0.3))
    a.step_closure(net, 4, every=4)
    b.step_closure(net, 2, every=4)
    b.step_closure(net, 2, every=4)
    np.testing.assert_array_equal(a.wavefield(0, 0), b.wavefield(0, 0))
    np.testing.assert_array_equal(a.wavefield(0, 1), b.wavefield(0, 1))
    # steps 0, 1 plain, then steps 2, 3 through the closure call: no correction
    d, *_ = _coarse_case(fdw, O, 45)
    c.step(4)
    d.step(2)
    d.step_closure(net, 2, every=4)
    np.testing.assert_array_equal(c.wavefield(0, 0), d.wavefield(0, 0))
    net.close()
    for s in (a, b, c, d):
        s.close()


def test_step_closure_zero_network_equals_plain_step(fdw, O):
    """All-zero parameters: fdw_step_closure gives fdw_step's levels."""
    a, *_ = _coarse_case(fdw, O, 41)
    b, *_ = _coarse_case(fdw, O, 41)
    net = fdw.Closure()
    net.set_params(np.zeros(net.num_params, np.float32))
    a.step(4)
    b.step_closure(net, 4)
    np.testing.assert_array_equal(a.wavefield(0, 0), b.wavefield(0, 0))
    np.testing.assert_array_equal(a.wavefield(0, 1), b.wavefield(0, 1))
    net.close()


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_step_closure_16bit_storage(fdw, O, storage):
    """16-bit wavefield storage: the closure reads and updates the stored
    levels; three steps stay within the storage rounding of the oracle."""
    solver, setup, vp, src, wav, u0, um = _coarse_case(fdw, O, 51, storage)
    p = random_params(8, scale=0.3)
    net = fdw.Closure()
    net.set_variant(1)
    net.set_params(p)
    ref_u, ref_um = solver.wavefield(0, 0).astype(np.float64), solver.wavefield(0, 1).astype(np.float64)
    for k in range(3):
        solver.step_closure(net, 1)
        nxt = O.closure_step(setup, ref_u, ref_um, vp, p.astype(np.float64), src, [wav[k]])
        ref_um, ref_u = ref_u, nxt
    tol = {"bf16": 3e-2, "f16": 4e-3}[storage]
    assert rel(solver.wavefield(0, 0), ref_u) < tol
    net.close()
    solver.close()


def _tc_vs_oracle_correction(fdw, O, seed, pscale, variant=0):
    """(GPU correction, oracle correction) of one closure step from random
    levels: the closure step's u_{n+1} minus the plain step's (the source
    term cancels)."""
    solver, setup, vp, src, wav, u0, um = _coarse_case(fdw, O, seed)
    plain, *_ = _coarse_case(fdw, O, seed)
    p = random_params(seed, scale=pscale)
    net = fdw.Closure()
    net.set_variant(variant)
    net.set_params(p)
    solver.step_closure(net, 1)
    plain.step(1)
    got = solver.wavefield(0, 0).astype(np.float64) - plain.wavefield(0, 0).astype(np.float64)
    u, v = u0.astype(np.float64), um.astype(np.float64)
    ref = O.closure_step(setup, u, v, vp, p.astype(np.float64)) - O.acoustic_step(setup, u, v)
    net.close()
    solver.close()
    plain.close()
    return got, ref


@pytest.mark.parametrize("variant", [0, 2])
@pytest.mark.parametrize("seed", [61, 62])
def test_tensor_core_step_matches_oracle(fdw, O, seed, variant):
    """The fused tensor-core inference (FP16 operands, FP32 accumulation;
    tcgen05 and mma.sync kernels) against the oracle's FP64 closure step:
    the correction agrees to the FP16 rounding of the activations. Bound:
    each activation carries a relative rounding error <= 2^-11; through two
    layers of 432-term sums the correction's relative L2 error stays well
    below 1e-2."""
    got, ref = _tc_vs_oracle_correction(fdw, O, seed, 0.3, variant)
    assert np.linalg.norm(ref) > 0
    assert rel(got, ref) < 1e-2


@pytest.mark.parametrize("variant", [0, 2])
def test_tensor_core_matches_fp32_kernels(fdw, O, variant):
    """Tensor-core and FP32 inference kernels on the same state: the
    corrections agree to FP16 rounding (the grid, 32 x 34 x 36 with the
    sponge, is ragged for both kernels' tiles -- 12 x 28 for tcgen05,
    30 x 14 for mma.sync -- and split into z chunks)."""
    corr = []
    for variant in (variant, 1):
        solver, *_ = _coarse_case(fdw, O, 71)
        plain, *_ = _coarse_case(fdw, O, 71)
        net = fdw.Closure()
        net.set_variant(variant)
        net.set_params(random_params(71, scale=0.3))
        solver.step_closure(net, 1)
        plain.step(1)
        corr.append(solver.wavefield(0, 0).astype(np.float64) - plain.wavefield(0, 0))
        net.close()
        solver.close()
        plain.close()
    assert rel(corr[0], corr[1]) < 1e-2


def test_tensor_core_correction_is_exactly_zero_where_the_field_is(fdw):
    """net(x) - net(x0) is computed by the same deterministic kernel for x
    and x0, so a wavefield that is zero over a point's receptive field gets
    no correction at all: a blob in one corner leaves the far corner exactly
    zero after a closure step, and a zero field stays exactly zero."""
    from paper_1608_03984_gb300 import synth
    n, nb, h = 40, 6, 20.0
    vp = synth.random_velocity((n, n, n), h, 120.0, 81)
    s = fdw.Solver(vp.shape, h, nb, 4)
    s.set_model(vp).set_sponge(4500.0).set_dt(0.35 * h / 4500.0)
    comp = s.comp_shape
    u = np.zeros(comp, np.float32)
    u[8:14, 8:14, 8:14] = synth.random_wavefield((6, 6, 6), 82)
    s.set_wavefield(u, 0, 0)
    s.set_wavefield(u, 0, 1)
    net = fdw.Closure()
    net.set_params(random_params(83, scale=0.3))
    s.step_closure(net, 1)
    out = s.wavefield(0, 0)
    assert np.abs(out[8:14, 8:14, 8:14]).max() > 0
    # beyond the blob + stencil radius 2 + receptive field 3 nothing moved
    assert np.all(out[20:, 20:, 20:] == 0)
    z = fdw.Solver(vp.shape, h, nb, 4)
    z.set_model(vp).set_sponge(4500.0).set_dt(0.35 * h / 4500.0)
    z.step_closure(net, 3)
    assert np.all(z.wavefield(0, 0) == 0) and np.all(z.wavefield(0, 1) == 0)
    net.close()
    s.close()
    z.close()


def test_training_reduces_error_on_held_out_models(fdw):
    """Train on solver-generated pairs from ten random models (fine order 16
    at h = 10 m, coarse order 4 at h = 20 m, 96^3 coarse physical points,
    a 10 Hz Ricker source at the centre, steps after the source has ended),
    then on four held-out models the coarse run with the closure is closer
    to the restricted fine run than the coarse run alone: in the final
    wavefield and in the receiver traces, for every model, and by at least
    15% on average; the same holds with the correction applied on every
    4th step only (times 4), at a quarter of the network's cost."""
    from paper_1608_03984_gb300 import closure as C
    pr = C.Pairing(n_c=96, nb_c=8, src_sigma=1.5)
    nt = pr.steps_to_cross(0.45)
    samplers = []
    for seed in range(100, 110):
        x, t = C.samples(pr, seed, nt, stride=2)
        samplers.append(C.PatchSampler(x, t, P=12, nb=pr.nb_c))
    net = fdw.Closure()
    losses = C.train(net, samplers, iters=8000, batch=32, lr=3e-3)
    assert losses[-1] < 0.5 * losses[0]
    ratios = {(run, key): [] for run in ("closure", "closure_every4") for key in ("field", "traces")}
    for seed in (900, 901, 902, 903):
        r = C.evaluate(pr, net, seed, nt, everies=(1, 4))
        for run, key in ratios:
            assert r[run][key] < r["coarse"][key], (seed, run, r)
            ratios[(run, key)].append(r[run][key] / r["coarse"][key])
    for k, v in ratios.items():
        assert np.mean(v) < 0.85, (k, v)
    net.close()


def test_tensor_core_full_size_sampled(fdw, O):
    """The benchmark's coarse grid (256^3 + 20-point sponge = 296^3, h = 20 m,
    order 4) in the launch configuration of its closure runs (tensor-core
    inference, default chunking): one closure step from random levels. At
    sampled points the correction (closure step minus plain step) matches
    the oracle's net(x) - net(x0) on the 7^3 block around the point, times
    m = max |u_n|; in the sponge and its 3-point margin it is exactly zero.
    Bound: FP16 rounding of the activations, as in the small-grid test."""
    import torch
    from paper_1608_03984_gb300 import synth
    n, nb, h, order = 256, 20, 20.0, 4
    vp = synth.random_velocity((n, n, n), h, 200.0, 91)
    dt = 0.35 * h / 4500.0
    p = random_params(92, scale=0.3)
    runs = []
    for closure in (True, False):
        s = fdw.Solver(vp.shape, h, nb, order)
        s.set_model(vp).set_sponge(4500.0).set_dt(dt)
        comp = s.comp_shape
        g = torch.Generator(device="cuda").manual_seed(93)
        u = torch.randn(comp, generator=g, device="cuda", dtype=torch.float32)
        um = torch.randn(comp, generator=g, device="cuda", dtype=torch.float32)
        s.set_wavefield(u, 0, 0)
        s.set_wavefield(um, 0, 1)
        if closure:
            net = fdw.Closure()
            net.set_params(p)
            s.step_closure(net, 1)
            net.close()
        else:
            s.step(1)
        out = torch.empty_like(u)
        s.wavefield(0, 0, out=out)
        s.check()
        s.close()
        runs.append(out)
    corr = (runs[0].double() - runs[1].double()).cpu().numpy()
    u, um = u.double().cpu().numpy(), um.double().cpu().numpy()
    m = float(np.abs(u).max())
    vn = (O.extend(vp, nb) - 3000.0) / 750.0
    N = comp[0]
    a = nb + 3
    rng = np.random.default_rng(94)
    pts = [tuple(int(v) for v in rng.integers(a, N - a, size=3)) for _ in range(40)]
    pts += [(a, a, a), (N - a - 1,) * 3, (a, N // 2, N - a - 1), (N // 2,) * 3]
    got, ref = [], []
    for (k, j, i) in pts:
        sl = (slice(k - 3, k + 4), slice(j - 3, j + 4), slice(i - 3, i + 4))
        x = np.stack([u[sl] / m, um[sl] / m, vn[sl]])
        ref.append(m * float(O.closure_correction(p.astype(np.float64), x)[0, 0, 0]))
        got.append(corr[k, j, i])
    got, ref = np.array(got), np.array(ref)
    assert np.abs(ref).max() > 0
    assert np.abs(got - ref).max() <= 1e-2 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()
    # no correction in the sponge and its margin
    band = np.ones(comp, bool)
    band[a:N - a, a:N - a, a:N - a] = False
    assert np.all(corr[band] == 0.0)


@pytest.mark.parametrize("shape,nb", [((9, 11, 13), 2), ((17, 30, 7), 3), ((40, 6, 29), 2)])
def test_tcgen05_inference_ragged_grids(fdw, O, shape, nb):
    """The tensor-core kernels (tcgen05 and mma.sync) on grids that are not
    multiples of their output columns, thinner than the z halo of the three
    layers, a single work item, or with no point far enough from the sponge
    to be corrected: the correction of one closure step agrees with the
    FP32 CUDA-core kernels to FP16 rounding, and is exactly zero where the
    receptive field leaves the physical grid."""
    from paper_1608_03984_gb300 import synth
    h, order = 20.0, 4
    vp = synth.random_velocity(shape, h, 120.0, 300 + shape[0])
    corr = []
    for variant in (0, 2, 1):
        s = fdw.Solver(vp.shape, h, nb, order)
        s.set_model(vp).set_sponge(4500.0).set_dt(0.35 * h / 4500.0)
        pl = fdw.Solver(vp.shape, h, nb, order)
        pl.set_model(vp).set_sponge(4500.0).set_dt(0.35 * h / 4500.0)
        comp = s.comp_shape
        u = synth.random_wavefield(comp, 11, smooth_pts=1.5).astype(np.float32)
        um = synth.random_wavefield(comp, 12, smooth_pts=1.5).astype(np.float32)
        for q in (s, pl):
            q.set_wavefield(u, 0, 0)
            q.set_wavefield(um, 0, 1)
        net = fdw.Closure()
        net.set_variant(variant)
        net.set_params(random_params(13, scale=0.3))
        s.step_closure(net, 1)
        pl.step(1)
        s.check()
        corr.append(s.wavefield(0, 0).astype(np.float64) - pl.wavefield(0, 0))
        net.close()
        s.close()
        pl.close()
    if np.linalg.norm(corr[2]) > 0:
        assert rel(corr[0], corr[2]) < 1e-2
        assert rel(corr[1], corr[2]) < 1e-2
    m = np.zeros(corr[0].shape, bool)
    a = nb + 3
    m[a:-a or None, a:-a or None, a:-a or None] = True
    assert np.all(corr[0][~m] == 0.0)
    assert np.all(corr[1][~m] == 0.0)
