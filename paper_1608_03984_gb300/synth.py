"""Seeded synthetic inputs shared by the GPU path's tests/bench and the oracle.

This module holds no arithmetic of the solver: it only draws velocity and
anisotropy models, source wavelets and acquisition geometries with fixed
seeds (numpy PCG64), in the shapes of the workloads the solver is measured
on. Both the oracle and the CUDA library receive what it returns as plain
arrays.

Workload recipes (sizes are physical grids; the solver adds the sponge):
  * ``two_layer``: acoustic, 64^3, h = 10 m, v = 1500 m/s above mid-depth and
    2500 m/s below, Ricker 15 Hz at the grid centre, 32 receivers on a line
    at 20 m depth, 10-point sponge, dt at CFL 0.4, 200 steps.
  * ``random_acoustic``: acoustic, 512^3, h = 10 m, Gaussian-smoothed random
    velocity (correlation length 200 m) clipped to 1500-4500 m/s, 40-point
    sponge, Ricker 10 Hz, 256 x 256 receivers at 20 m depth, 1000 steps.
  * ``random_tti``: TTI, 384^3, h = 12.5 m, smooth eps in [0, 0.3],
    delta in [0, 0.2] (delta <= eps), theta in [0, 60 deg], phi in
    [0, 180 deg], velocity 1500-4500 m/s, 800 steps.
Every recipe accepts a reduced ``n`` so tests can run the same structure at
oracle-friendly sizes.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = {"two_layer": 1001, "random_acoustic": 1002, "random_tti": 1003, "fwi": 1004,
             "closure": 5000}


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def ricker(f0: float, dt: float, nt: int, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet of peak frequency f0 sampled at t_n = n dt, n < nt,
    delayed by t0 (default 1/f0), unit peak amplitude."""
    t0 = 1.0 / f0 if t0 is None else t0
    t = np.arange(nt, dtype=np.float64) * dt - t0
    a = (math.pi * f0 * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def smooth_random_field(shape, corr_pts: float, seed: int) -> np.ndarray:
    """Standardised (zero-mean, unit-variance) Gaussian random field with a
    Gaussian correlation of `corr_pts` grid points, float32.

    White noise is drawn on a grid coarser by f = max(1, corr_pts // 4),
    convolved (periodically, via FFT) with a Gaussian of sigma corr_pts / f,
    then trilinearly upsampled by f and cropped: the field is smooth on the
    scale of corr_pts, so the coarse draw loses nothing visible and keeps the
    512^3 recipe cheap."""
    shape = tuple(int(n) for n in shape)
    f = max(1, int(corr_pts // 4))
    cshape = tuple(-(-n // f) + 2 for n in shape)
    w = rng(seed).standard_normal(cshape)
    sig = corr_pts / f
    W = np.fft.rfftn(w)
    kz = np.fft.fftfreq(cshape[0])[:, None, None]
    ky = np.fft.fftfreq(cshape[1])[None, :, None]
    kx = np.fft.rfftfreq(cshape[2])[None, None, :]
    W *= np.exp(-2.0 * (math.pi * sig) ** 2 * (kx * kx + ky * ky + kz * kz))
    s = np.fft.irfftn(W, s=cshape, axes=(0, 1, 2))
    s = (s - s.mean()) / max(s.std(), 1e-30)
    if f > 1:
        s = _upsample_linear(s, f, shape)
    else:
        s = s[: shape[0], : shape[1], : shape[2]]
    s = (s - s.mean()) / max(float(s.std()), 1e-30)
    return s.astype(np.float32)


def _upsample_linear(c: np.ndarray, f: int, shape) -> np.ndarray:
    out = c.astype(np.float32)
    for ax in range(3):
        n = shape[ax]
        pos = np.arange(n, dtype=np.float64) / f
        i0 = np.floor(pos).astype(np.int64)
        t = (pos - i0).astype(np.float32)
        a = np.take(out, i0, axis=ax)
        b = np.take(out, i0 + 1, axis=ax)
        sh = [1, 1, 1]
        sh[ax] = n
        t = t.reshape(sh)
        out = a * (1.0 - t) + b * t
    return out


@dataclasses.dataclass
class Workload:
    name: str
    equation: str            # "acoustic" | "tti"
    n: tuple                 # physical (nz, ny, nx)
    h: float
    nb: int
    order: int
    dt: float
    nt: int
    vp: np.ndarray           # physical velocity, float32 (nz, ny, nx), m/s
    src_xyz: np.ndarray      # (nsrc, 3) metres, float64
    wavelet: np.ndarray      # (nt, nsrc) float32
    rec_xyz: np.ndarray      # (nrec, 3) metres, float64
    eps: np.ndarray | None = None
    delta: np.ndarray | None = None
    theta: np.ndarray | None = None   # radians
    phi: np.ndarray | None = None     # radians
    f0: float = 10.0

    @property
    def n_comp(self):
        return tuple(x + 2 * self.nb for x in self.n)

    @property
    def points(self):
        nz, ny, nx = self.n_comp
        return nz * ny * nx


def _cfl_dt(h, vmax, cfl=0.4):
    """dt at Courant number `cfl` (vmax dt / h = cfl)."""
    return cfl * h / vmax


def two_layer(n: int = 64, h: float = 10.0, nb: int = 10, order: int = 4, nt: int = 200,
              nrec: int = 32, f0: float = 15.0) -> Workload:
    """Two-layer acoustic model at CFL 0.4 (the 64^3 parity workload)."""
    vp = np.full((n, n, n), 1500.0, dtype=np.float32)
    vp[n // 2:, :, :] = 2500.0
    dt = _cfl_dt(h, 2500.0)
    centre = (n - 1) * h / 2.0
    src = np.array([[centre, centre, centre]], dtype=np.float64)
    rec = np.zeros((nrec, 3))
    rec[:, 0] = np.linspace(0.0, (n - 1) * h, nrec)
    rec[:, 1] = centre
    rec[:, 2] = 20.0
    w = ricker(f0, dt, nt).astype(np.float32).reshape(nt, 1)
    return Workload("two_layer", "acoustic", (n, n, n), h, nb, order, dt, nt, vp, src, w, rec,
                    f0=f0)


def random_velocity(shape, h, corr_m, seed, vmin=1500.0, vmax=4500.0, mean=3000.0, sd=750.0):
    z = smooth_random_field(shape, corr_m / h, seed)
    return np.clip(mean + sd * z, vmin, vmax).astype(np.float32)


def random_acoustic(n: int = 512, h: float = 10.0, nb: int = 40, order: int = 8,
                    nt: int = 1000, nrec_side: int = 256, f0: float = 10.0,
                    seed: int | None = None) -> Workload:
    """Smooth random acoustic model (the 512^3 order-sweep workload)."""
    seed = SEED_BASE["random_acoustic"] if seed is None else seed
    vp = random_velocity((n, n, n), h, 200.0, seed)
    dt = _cfl_dt(h, 4500.0)
    centre = (n - 1) * h / 2.0
    src = np.array([[centre, centre, centre]], dtype=np.float64)
    g = np.linspace(0.0, (n - 1) * h, nrec_side)
    X, Y = np.meshgrid(g, g, indexing="xy")
    rec = np.stack([X.ravel(), Y.ravel(), np.full(X.size, min(20.0, (n - 1) * h))], axis=1)
    w = ricker(f0, dt, nt).astype(np.float32).reshape(nt, 1)
    return Workload("random_acoustic", "acoustic", (n, n, n), h, nb, order, dt, nt, vp, src, w,
                    rec, f0=f0)


def random_tti(n: int = 384, h: float = 12.5, nb: int = 40, order: int = 8, nt: int = 800,
               nrec_side: int = 128, f0: float = 10.0, seed: int | None = None) -> Workload:
    """Smooth random TTI model (the 384^3 workload). delta is capped at eps
    pointwise so the system stays hyperbolic."""
    seed = SEED_BASE["random_tti"] if seed is None else seed
    shp = (n, n, n)
    corr = 200.0 / h
    vp = random_velocity(shp, h, 200.0, seed)
    eps = np.clip(0.15 + 0.075 * smooth_random_field(shp, corr, seed + 100), 0.0, 0.3)
    delta = np.clip(0.10 + 0.05 * smooth_random_field(shp, corr, seed + 200), 0.0, 0.2)
    delta = np.minimum(delta, eps)
    theta = np.deg2rad(np.clip(30.0 + 15.0 * smooth_random_field(shp, corr, seed + 300), 0.0, 60.0))
    phi = np.deg2rad(np.clip(90.0 + 45.0 * smooth_random_field(shp, corr, seed + 400), 0.0, 180.0))
    vmax_eff = 4500.0 * math.sqrt(1.0 + 2.0 * 0.3)
    dt = _cfl_dt(h, vmax_eff)
    centre = (n - 1) * h / 2.0
    src = np.array([[centre, centre, centre]], dtype=np.float64)
    g = np.linspace(0.0, (n - 1) * h, nrec_side)
    X, Y = np.meshgrid(g, g, indexing="xy")
    rec = np.stack([X.ravel(), Y.ravel(), np.full(X.size, min(25.0, (n - 1) * h))], axis=1)
    w = ricker(f0, dt, nt).astype(np.float32).reshape(nt, 1)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Workload("random_tti", "tti", shp, h, nb, order, dt, nt, vp, src, w, rec,
                    eps=f32(eps), delta=f32(delta), theta=f32(theta), phi=f32(phi), f0=f0)


def gaussian_smooth(a: np.ndarray, sigma_pts: float) -> np.ndarray:
    """Periodic Gaussian smoothing (FFT) of a 3D array, edge-padded by
    3 sigma first so the model's faces do not wrap into each other."""
    pad = int(min(3 * sigma_pts, max(a.shape)))
    b = np.pad(np.asarray(a, np.float64), pad, mode="edge")
    B = np.fft.rfftn(b)
    kz = np.fft.fftfreq(b.shape[0])[:, None, None]
    ky = np.fft.fftfreq(b.shape[1])[None, :, None]
    kx = np.fft.rfftfreq(b.shape[2])[None, None, :]
    B *= np.exp(-2.0 * (math.pi * sigma_pts) ** 2 * (kx * kx + ky * ky + kz * kz))
    out = np.fft.irfftn(B, s=b.shape, axes=(0, 1, 2))
    return out[pad:pad + a.shape[0], pad:pad + a.shape[1], pad:pad + a.shape[2]]


@dataclasses.dataclass
class FwiWorkload:
    n: tuple
    h: float
    nb: int
    order: int
    dt: float
    nt: int
    v_true: np.ndarray
    v_start: np.ndarray
    src_xyz: np.ndarray      # (nshot, 3)
    wavelet: np.ndarray      # (nt,)
    rec_xyz: np.ndarray      # (nrec, 3)
    checkpoints: int = 20


def fwi(n: int = 256, h: float = 15.0, nb: int = 40, order: int = 8, nt: int = 2000,
        shots_side: int = 4, rec_side: int = 128, f0: float = 8.0, checkpoints: int = 20,
        seed: int | None = None) -> FwiWorkload:
    """FWI workload (256^3, h = 15 m): true model = smooth random velocity
    (correlation length 200 m) plus three Gaussian anomalies of +-10%
    (sigma 150 m, seeded centres); starting model = the true one smoothed
    with sigma = 40 points; 4 x 4 shots at 30 m depth over the middle half,
    128 x 128 receivers at 30 m depth, Ricker 8 Hz, dt at CFL 0.4 of the
    largest velocity."""
    seed = SEED_BASE["fwi"] if seed is None else seed
    shp = (n, n, n)
    v = random_velocity(shp, h, 200.0, seed).astype(np.float64)
    r = rng(seed + 1)
    zz, yy, xx = (np.arange(k, dtype=np.float64) * h for k in shp)
    sig = 150.0
    for sign in (1.0, -1.0, 1.0):
        c = r.uniform(0.25, 0.75, size=3) * (n - 1) * h
        g = (np.exp(-((zz - c[0]) ** 2) / (2 * sig * sig))[:, None, None]
             * np.exp(-((yy - c[1]) ** 2) / (2 * sig * sig))[None, :, None]
             * np.exp(-((xx - c[2]) ** 2) / (2 * sig * sig))[None, None, :])
        v *= 1.0 + sign * 0.1 * g
    v_true = v.astype(np.float32)
    v_start = gaussian_smooth(v, 40.0).astype(np.float32)
    vmax = max(float(v_true.max()), float(v_start.max()))
    dt = _cfl_dt(h, vmax)
    span = (n - 1) * h
    s = np.linspace(0.25 * span, 0.75 * span, shots_side)
    SX, SY = np.meshgrid(s, s, indexing="xy")
    src = np.stack([SX.ravel(), SY.ravel(), np.full(SX.size, 30.0)], axis=1)
    g = np.linspace(0.0, span, rec_side)
    RX, RY = np.meshgrid(g, g, indexing="xy")
    rec = np.stack([RX.ravel(), RY.ravel(), np.full(RX.size, 30.0)], axis=1)
    w = ricker(f0, dt, nt).astype(np.float32)
    return FwiWorkload(shp, h, nb, order, dt, nt, v_true, v_start, src, w, rec, checkpoints)


def random_wavefield(shape, seed, scale=1.0, smooth_pts=2.0):
    """Smooth random field used as a wavefield state for one-step checks."""
    return (scale * smooth_random_field(shape, smooth_pts, seed)).astype(np.float32)
