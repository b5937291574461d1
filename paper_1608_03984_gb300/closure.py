"""Learned coarse-grid closure: training data from the library's own solvers,
training and evaluation through the library's closure kernels.

A fine solver (order 16, spacing h) and a coarse one (order 4, spacing 2h,
time step 2 dt) share the physical box and the sponge's physical width;
coarse point i is fine point 2i. The source is a Ricker wavelet spread by a
Gaussian of width one coarse spacing around its centre, sampled on each
grid (a point source has no common meaning on two grids: each grid would
inject its own unresolved near field).

From a fine run the restricted levels R u^{2k} give, for coarse step k, the
input (R u^{2k}, R u^{2k-2}, v) and the target defect
    R u^{2k+2} - coarse_step(R u^{2k}, R u^{2k-2}),
both divided by m_k = max |R u^{2k}| (the normalisation fdw_step_closure
applies at run time). Training draws cubic patches with probability growing
with the local defect energy; Adam runs in the library
(fdw_closure_adam_step).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

from . import fdwave, synth

VEL_MEAN, VEL_SCALE = 3000.0, 750.0  # the velocity normalisation of fdw_step_closure


@dataclasses.dataclass
class Pairing:
    """A fine/coarse pair of acoustic solvers on one physical box."""
    n_c: int                 # coarse physical points per axis
    h_c: float = 20.0
    nb_c: int = 20
    order_c: int = 4
    order_f: int = 16
    f0: float = 10.0
    vmin: float = 1500.0
    vmax: float = 4500.0
    corr_m: float = 200.0    # correlation length of the random velocity
    cfl_f: float = 0.35      # dt_f = cfl_f h_f / vmax
    src_sigma: float = 1.0   # source width in coarse spacings

    @property
    def n_f(self):
        return 2 * self.n_c

    @property
    def h_f(self):
        return self.h_c / 2

    @property
    def nb_f(self):
        return 2 * self.nb_c

    @property
    def dt_f(self):
        return self.cfl_f * self.h_f / self.vmax

    @property
    def dt_c(self):
        return 2 * self.dt_f

    @property
    def comp_c(self):
        return self.n_c + 2 * self.nb_c

    def source_steps(self):
        """Coarse steps until the Ricker wavelet has died out (t = 2 / f0:
        the delay 1 / f0 plus 1 / f0, where the wavelet is below 1e-3 of its
        peak)."""
        return int(math.ceil(2.0 / self.f0 / self.dt_c))

    def steps_to_cross(self, frac=0.5):
        """Coarse steps for the wavelet's delay plus a travel of `frac` box
        widths at the mean velocity."""
        t = 1.0 / self.f0 + frac * (self.n_c - 1) * self.h_c / VEL_MEAN
        return int(math.ceil(t / self.dt_c))


def init_params(seed=0, last_scale=0.01):
    """He-normal convolution weights, zero biases, a small last layer (the
    untrained closure starts close to no correction)."""
    r = synth.rng(seed)
    parts = []
    for ci, co, scale in ((3, 16, 1.0), (16, 16, 1.0), (16, 1, last_scale)):
        parts.append(scale * math.sqrt(2.0 / (ci * 27)) * r.standard_normal(co * ci * 27))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def model(pr: Pairing, seed: int):
    """Fine velocity (seeded smooth random field), its restriction, and the
    source centre (a point of both grids within the middle fifth)."""
    v_f = synth.random_velocity((pr.n_f,) * 3, pr.h_f, pr.corr_m, seed, vmin=pr.vmin,
                                vmax=pr.vmax)
    v_c = np.ascontiguousarray(v_f[::2, ::2, ::2])
    r = synth.rng(seed + 7919)
    span = (pr.n_c - 1) * pr.h_c
    src = r.uniform(0.4 * span, 0.6 * span, size=3)
    src = np.round(src / pr.h_c) * pr.h_c
    return v_f, v_c, src


def gaussian_source(center, h, n, sigma, radius_sigmas=4.0):
    """Grid points within radius_sigmas * sigma of `center` (x, y, z metres)
    and weights exp(-r^2 / (2 sigma^2)) scaled to sum to one: injecting
    weight * wavelet at each point spreads a unit source over the Gaussian."""
    rad = radius_sigmas * sigma
    lo = np.maximum(np.floor((center - rad) / h), 0).astype(int)
    hi = np.minimum(np.ceil((center + rad) / h), n - 1).astype(int)
    ax = [np.arange(lo[i], hi[i] + 1) * h for i in range(3)]
    X, Y, Z = np.meshgrid(ax[0], ax[1], ax[2], indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    r2 = np.sum((pts - center) ** 2, axis=1)
    keep = r2 <= rad * rad
    pts, w = pts[keep], np.exp(-r2[keep] / (2 * sigma * sigma))
    return pts, w / w.sum()


def _sources(pr, solver, center, h, n, dt, nt):
    pts, w = gaussian_source(center, h, n, pr.src_sigma * pr.h_c)
    wav = synth.ricker(pr.f0, dt, nt)
    solver.set_sources(pts, (wav[:, None] * w[None, :]).astype(np.float32))


def fine_solver(pr: Pairing, v_f, src, nt_f, rec=None):
    s = fdwave.Solver(v_f.shape, pr.h_f, pr.nb_f, pr.order_f)
    s.set_model(v_f).set_sponge(pr.vmax).set_dt(pr.dt_f)
    _sources(pr, s, src, pr.h_f, pr.n_f, pr.dt_f, nt_f)
    if rec is not None:
        s.set_receivers(rec, nt_f)
    return s


def coarse_solver(pr: Pairing, v_c, src, nt_c, rec=None):
    s = fdwave.Solver(v_c.shape, pr.h_c, pr.nb_c, pr.order_c)
    s.set_model(v_c).set_sponge(pr.vmax).set_dt(pr.dt_c)
    if s.max_stable_dt() < pr.dt_c:
        raise ValueError("coarse step above the stability limit")
    _sources(pr, s, src, pr.h_c, pr.n_c, pr.dt_c, nt_c + 2)
    if rec is not None:
        s.set_receivers(rec, nt_c)
    return s


def restrict(full):
    """Fine computational grid -> coarse (every other point from the first)."""
    return full[::2, ::2, ::2].contiguous()


def velocity_channel(v_c, nb_c):
    """(v - 3000) / 750 on the coarse computational grid, edge-extended."""
    v = torch.from_numpy(np.pad(v_c, nb_c, mode="edge")).cuda()
    return (v - VEL_MEAN) / VEL_SCALE


def samples(pr: Pairing, seed: int, nt_c: int, k0: int | None = None, stride: int = 1):
    """(x [K, 3, N, N, N], target [K, N, N, N]) on the coarse computational
    grid (N = n_c + 2 nb_c) for coarse steps k0, k0 + stride, ... < nt_c;
    k0 defaults to the end of the source (the closure corrects propagation;
    while the source acts the defect is the two grids' different sampling
    of the source, not a property of the wave)."""
    k0 = pr.source_steps() if k0 is None else k0
    v_f, v_c, src = model(pr, seed)
    fs = fine_solver(pr, v_f, src, 2 * nt_c + 2)
    if fs.max_stable_dt() < pr.dt_f:
        raise ValueError("fine step above the stability limit")
    cs = coarse_solver(pr, v_c, src, nt_c)
    if restrict(torch.empty(fs.comp_shape)).shape != cs.comp_shape:
        raise ValueError("grids do not nest")
    vn = velocity_channel(v_c, pr.nb_c)
    full = torch.empty(fs.comp_shape, dtype=torch.float32, device="cuda")
    pred = torch.empty(cs.comp_shape, dtype=torch.float32, device="cuda")
    prev = torch.zeros(cs.comp_shape, dtype=torch.float32, device="cuda")  # R u^{2k-2}
    cur = torch.zeros_like(prev)                                           # R u^{2k}
    xs, ts = [], []
    for k in range(nt_c):
        fs.step(2)
        fs.wavefield(0, 0, out=full)
        nxt = restrict(full)                                               # R u^{2k+2}
        m = float(cur.abs().max())
        if k >= k0 and (k - k0) % stride == 0 and m > 0:
            cs.set_wavefield(cur, 0, 0)
            cs.set_wavefield(prev, 0, 1)
            cs.set_current_step(k)
            cs.step(1)
            cs.wavefield(0, 0, out=pred)
            xs.append(torch.stack([cur / m, prev / m, vn]))
            ts.append((nxt - pred) / m)
        prev, cur = cur, nxt
    fs.close()
    cs.close()
    return torch.stack(xs), torch.stack(ts)


class PatchSampler:
    """Random cubic patches of one (x, target) set: inputs (P+6)^3 on
    physical points, targets the central P^3 (the points the closure
    corrects: 3 or more points from the sponge). The valid convolutions of
    a patch give exactly what the time loop's zero-padded ones give there. Every time step (sample) is
    drawn equally often (the defect while the source acts is ~10x the later
    propagation defect and would otherwise crowd it out); within a step the
    origin is drawn with probability proportional to the patch's defect
    energy, plus `floor` times the uniform probability."""

    def __init__(self, x, t, P, nb, floor=0.2):
        self.P, self.N = P, x.shape[2]
        self.lo = nb                                # first input origin
        side = self.N - 2 * nb - (P + 6) + 1        # origins o: o >= nb, o + P + 6 <= N - nb
        if side < 1:
            raise ValueError("physical region smaller than a patch")
        self.side = side
        self.x, self.t = x, t
        a = self.lo + 3
        w = torch.nn.functional.avg_pool3d(
            t[:, None, a:a + side + P - 1, a:a + side + P - 1, a:a + side + P - 1] ** 2,
            kernel_size=P, stride=1)[:, 0]
        per_step = w.flatten(1).sum(1).clamp_min(1e-300)
        w = w / per_step[:, None, None, None] + floor / w[0].numel()
        self.w = (w / w.sum()).flatten()
        # inverse-CDF sampling (torch.multinomial takes at most 2^24 categories)
        self.cdf = torch.cumsum(self.w.double(), 0)
        self.cdf /= self.cdf[-1].clone()

    def __call__(self, count, gen):
        P, side = self.P, self.side
        u = torch.rand(count, generator=gen, device=self.cdf.device, dtype=torch.float64)
        idx = torch.searchsorted(self.cdf, u).clamp_max(self.cdf.numel() - 1)
        per = side ** 3
        kk, rem = idx // per, idx % per
        zz, yy, xx = (self.lo + rem // (side * side), self.lo + (rem // side) % side,
                      self.lo + rem % side)
        a = torch.arange(P + 6, device=idx.device)
        k4 = kk[:, None, None, None]
        X = self.x[k4, :, (zz[:, None] + a)[:, :, None, None], (yy[:, None] + a)[:, None, :, None],
                   (xx[:, None] + a)[:, None, None, :]]
        X = X.permute(0, 4, 1, 2, 3).contiguous()  # the advanced indices come first
        a = a[3:P + 3]
        T = self.t[k4, (zz[:, None] + a)[:, :, None, None], (yy[:, None] + a)[:, None, :, None],
                   (xx[:, None] + a)[:, None, None, :]].contiguous()
        return X, T


class PatchBank:
    """Patches drawn once from many models' samplers (whose full fields are
    then dropped), served uniformly at random: the training set of many
    models in a fraction of the memory. Callable like a PatchSampler."""

    def __init__(self):
        self.X, self.T = [], []

    def add(self, sampler, count, gen):
        X, T = sampler(count, gen)
        self.X.append(X)
        self.T.append(T)

    def freeze(self):
        self.X, self.T = torch.cat(self.X), torch.cat(self.T)
        return self

    def __len__(self):
        return int(self.X.shape[0])

    def __call__(self, count, gen):
        idx = torch.randint(0, self.X.shape[0], (count,), generator=gen, device=self.X.device)
        return self.X[idx].contiguous(), self.T[idx].contiguous()


def target_scale(samplers, gen, count=512):
    """Power of two K that brings the patches' RMS target near one. The
    defect of one coarse step is ~1e-4 of max |u|: trained on K * target
    the network works with O(1) numbers, and dividing its last layer by K
    afterwards (exact in BF16 and FP32) gives the network of the real
    target."""
    ms = 0.0
    for smp in samplers:
        _, T = smp(count, gen)
        ms += float((T.double() ** 2).mean()) / len(samplers)
    return 2.0 ** round(-0.5 * math.log2(ms)) if ms > 0 else 1.0


def scale_last_layer(params, factor):
    """Multiply W3 and b3 (the last 16 * 27 + 1 parameters) by factor."""
    p = np.array(params, dtype=np.float32, copy=True)
    p[-(16 * 27 + 1):] *= np.float32(factor)
    return p


def train(net: "fdwave.Closure", samplers, iters=1000, batch=32, lr=2e-3, seed=0, init_seed=0,
          log=None):
    """Adam on random patches drawn in turn from the PatchSamplers (targets
    times target_scale; the last layer is divided by it at the end),
    learning rate decaying geometrically to lr / 10. Starts from
    init_params(init_seed) in the scaled problem, or from the network's
    current parameters if init_seed is None. Returns the losses (of the
    scaled targets) every 50 steps."""
    gen = torch.Generator(device="cuda").manual_seed(seed)
    K = target_scale(samplers, gen)
    if init_seed is None:
        net.set_params(scale_last_layer(net.get_params(), K))
    else:
        net.set_params(init_params(init_seed))
    losses = []
    loss = torch.empty((), dtype=torch.float32, device="cuda")
    for it in range(iters):
        X, T = samplers[it % len(samplers)](batch, gen)
        net.adam_step(X, T * K, lr * (0.1 ** (it / max(iters, 1))), loss=loss)
        if it % 50 == 0 or it == iters - 1:
            losses.append(float(loss))
            if log:
                log(it, losses[-1])
    net.set_params(scale_last_layer(net.get_params(), 1.0 / K))
    return losses


def unexplained(net: "fdwave.Closure", sampler, count=512, seed=1):
    """One-step misfit of the closure on `count` patches of a sampler,
    relative to the targets' mean square (1 = no better than no closure)."""
    gen = torch.Generator(device="cuda").manual_seed(seed)
    X, T = sampler(count, gen)
    loss, _ = net.loss_grad(X, T, grad=False)
    return float(loss) / float((T.double() ** 2).mean())


TRACE_DEPTHS = (5, 10, 20)  # receiver depths in coarse spacings; the first is the headline


def receivers(pr: Pairing, nside=8, depths=(5,)):
    """nside x nside grids of receivers at the given depths in coarse
    spacings (5: just below the 3-point band next to the sponge that the
    closure leaves alone), on points of both grids; one grid after the
    other, in the order of `depths`."""
    span = (pr.n_c - 1) * pr.h_c
    g = np.round(np.linspace(0.1 * span, 0.9 * span, nside) / pr.h_c) * pr.h_c
    X, Y = np.meshgrid(g, g)
    return np.concatenate([np.stack([X.ravel(), Y.ravel(), np.full(X.size, dep * pr.h_c)], axis=1)
                           for dep in depths])


def evaluate(pr: Pairing, net, seed: int, nt_c: int, timing=False, closure_from=None, everies=(1,)):
    """Relative L2 errors of the coarse run alone and with the closure
    against the restricted fine run: final level (physical part) and traces
    (receivers of `receivers` at 5 coarse spacings depth, fine traces at
    the coarse times; `traces_by_depth` repeats it for every depth of
    TRACE_DEPTHS). The closure run takes plain steps until `closure_from`
    (default: the end of the source, pr.source_steps()), then closure
    steps: on every step ("closure"), or on every e-th step with the
    correction times e ("closure_every<e>") for each e of `everies`. With
    timing=True also the device milliseconds of each run."""
    k1 = pr.source_steps() if closure_from is None else int(closure_from)
    k1 = min(max(k1, 0), nt_c)
    v_f, v_c, src = model(pr, seed)
    rec = receivers(pr, depths=TRACE_DEPTHS)
    ng = rec.shape[0] // len(TRACE_DEPTHS)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    fs = fine_solver(pr, v_f, src, 2 * nt_c, rec)
    ev[0].record()
    fs.step(2 * nt_c)
    ev[1].record()
    torch.cuda.synchronize()
    ms = {"fine": ev[0].elapsed_time(ev[1])}
    ref_tr = fs.traces()[::2]
    full = torch.empty(fs.comp_shape, dtype=torch.float32, device="cuda")
    fs.wavefield(0, 0, out=full)
    nb = pr.nb_c
    phys = (slice(nb, nb + pr.n_c),) * 3
    ref_u = restrict(full)[phys].double()
    fs.close()
    out = {}
    runs = [("coarse", 0)] + [("closure" if e == 1 else "closure_every%d" % e, e) for e in everies]
    for name, every in runs:
        cs = coarse_solver(pr, v_c, src, nt_c, rec)
        u = torch.empty(cs.comp_shape, dtype=torch.float32, device="cuda")
        ev[0].record()
        if name == "coarse":
            cs.step(nt_c)
        else:
            cs.step(k1)
            cs.step_closure(net, nt_c - k1, every=every)
        ev[1].record()
        torch.cuda.synchronize()
        ms[name] = ev[0].elapsed_time(ev[1])
        cs.wavefield(0, 0, out=u)
        tr = cs.traces()
        cs.close()
        uu = u[phys].double()
        by_depth = {}
        for i, dep in enumerate(TRACE_DEPTHS):
            sl = slice(i * ng, (i + 1) * ng)
            by_depth[dep] = float(np.linalg.norm(tr[:, sl] - ref_tr[:, sl]) / np.linalg.norm(ref_tr[:, sl]))
        out[name] = {"field": float(torch.linalg.vector_norm(uu - ref_u) / torch.linalg.vector_norm(ref_u)),
                     "traces": by_depth[TRACE_DEPTHS[0]], "traces_by_depth": by_depth}
    if timing:
        out["ms"] = ms
    return out
