"""FP64 CPU oracle of the explicit FD wave solvers (arXiv 1608.03984).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. It shares no code
with the GPU library; the C kernels are in ``fdoracle.c`` (plain loops in
the paper's order and notation), this module marshals numpy arrays and holds
the set-up steps the paper states as formulas (CFL limit of Eq. stability,
the sponge-medium extension, c = dt^2 v^2).

Parity unpinned (conventions the paper does not fix; nothing outside the
oracle fixes their values, so only the GPU-vs-oracle parity covers them):
the sponge constants of ``sponge_gamma_max`` / ``sponge_profile`` (reflection
coefficient R = 1e-3, linear ramp; the tests only pin that the sponge
absorbs), the medium extension into the sponge of ``extend`` (edge values),
and the receiver sampling of the forward runs (nt + 1 samples, d[0] = 0).
``extend_adjoint`` is pinned as the transpose of ``extend`` (dot test and
the brute-force transposed matrix in the adjoint tests).

Array convention: numpy arrays of shape (nz, ny, nx), C order, x fastest.
Positions are (x, y, z) metres of the physical grid, whose first point is at
the origin; the computational grid adds ``nb`` sponge points on every face.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdoracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libfdoracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.c_int
_F = ctypes.c_double


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, OpenMP) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "fdoracle.h"))):
        tmp = _SO + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            sig = {
                "or_fornberg": [_I, _D, _F, _I, _D],
                "or_fd_weights": [_I, _D, _D],
                "or_laplacian": [_I, _I, _I, _I, _F, _I, _D, _D],
                "or_derivative": [_I, _I, _I, _I, _F, _I, _I, _D, _D],
                "or_rotated": [_I, _I, _I, _I, _F, _I, _D, _D, _D, _D, _D, _D],
                "or_sponge_profile": [_I, _I, _F, _D],
                "or_interpolate": [_I, _I, _I, _F, _I, _D, _I, _D, _D],
                "or_acoustic_step": [_I, _I, _I, _I, _F, _I, _I, _F, _D, _D, _D, _D, _D, _D,
                                     _I, _D, _D, _D],
                "or_acoustic_forward": [_I, _I, _I, _I, _F, _I, _F, _D, _D, _D, _D, _I, _D, _D,
                                        _I, _I, _D, _D, _D, _D, _D],
                "or_tti_step": [_I, _I, _I, _I, _F, _I, _I, _F, _D, _D, _D, _D, _D, _D, _D, _D,
                                _D, _D, _D, _D, _I, _D, _D, _D, _D],
                "or_tti_forward": [_I, _I, _I, _I, _F, _I, _F, _D, _D, _D, _D, _D, _D, _D, _D,
                                   _I, _D, _D, _I, _I, _D, _D, _D],
                "or_acoustic_adjoint": [_I, _I, _I, _I, _F, _I, _F, _D, _D, _D, _D, _I, _D, _D,
                                        _I, _I, _D, _D, _D, _D],
            }
            for name, args in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = _I
            L.or_sponge_gamma_max.argtypes = [_F, _I, _F, _F]
            L.or_sponge_gamma_max.restype = _F
            _lib = L
    return _lib


def _p(a):
    """double* of a C-contiguous float64 array, or NULL for None."""
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous, (a.dtype, a.flags)
    return a.ctypes.data_as(_D)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _chk(rc, what):
    if rc != 0:
        raise ValueError("oracle %s failed (rc=%d)" % (what, rc))


# --------------------------------------------------------------------------
# weights and operators (Section "Stencil operators")
# --------------------------------------------------------------------------

def fornberg(x, z, mmax):
    """Weights[node, m] of the m-th derivative at z from nodes x (Fornberg 1988)."""
    x = _f64(np.asarray(x))
    out = np.zeros((x.size, mmax + 1))
    _chk(lib().or_fornberg(x.size - 1, _p(x), float(z), mmax, _p(out)), "fornberg")
    return out


def fd_weights(order):
    """(w2, c1): central 2nd/1st-derivative weights at offsets 0..r (unit spacing)."""
    r = order // 2
    w2 = np.zeros(r + 1)
    c1 = np.zeros(r + 1)
    _chk(lib().or_fd_weights(order, _p(w2), _p(c1)), "fd_weights")
    return w2, c1


def laplacian(u, order, h, periodic=False):
    u = _f64(u)
    out = np.empty_like(u)
    nz, ny, nx = u.shape
    _chk(lib().or_laplacian(nx, ny, nz, order, h, int(periodic), _p(u), _p(out)), "laplacian")
    return out


DERIVS = {"x": 0, "y": 1, "z": 2, "xx": 3, "yy": 4, "zz": 5, "xy": 6, "xz": 7, "yz": 8}


def derivative(u, which, order, h, periodic=False):
    u = _f64(u)
    out = np.empty_like(u)
    nz, ny, nx = u.shape
    _chk(lib().or_derivative(nx, ny, nz, order, h, int(periodic), DERIVS[which], _p(u), _p(out)),
         "derivative")
    return out


def rotated(u, theta, phi, order, h, periodic=False):
    """(Gxx u, Gyy u, Gzz u) of Eq. DiffOp, theta/phi per point in radians."""
    u = _f64(u)
    th = _f64(np.broadcast_to(theta, u.shape))
    ph = _f64(np.broadcast_to(phi, u.shape))
    gx, gy, gz = np.empty_like(u), np.empty_like(u), np.empty_like(u)
    nz, ny, nx = u.shape
    _chk(lib().or_rotated(nx, ny, nz, order, h, int(periodic), _p(th), _p(ph), _p(u),
                          _p(gx), _p(gy), _p(gz)), "rotated")
    return gx, gy, gz


# --------------------------------------------------------------------------
# set-up: stability (Eq. stability), sponge, medium on the computational grid
# --------------------------------------------------------------------------

def laplacian_abs_weight_sum(order):
    """a2 of Eq. stability: sum of |weights| of the 3D Laplacian stencil."""
    w2, _ = fd_weights(order)
    return 3.0 * (abs(w2[0]) + 2.0 * np.abs(w2[1:]).sum())


def max_stable_dt(order, h, vmax, a1=4.0):
    """Largest dt with vmax dt / h <= sqrt(a1/a2) (Eq. stability, CFL)."""
    return h * np.sqrt(a1 / laplacian_abs_weight_sum(order)) / vmax


def sponge_gamma_max(vmax, nb, h, R=1e-3):
    return lib().or_sponge_gamma_max(float(vmax), int(nb), float(h), float(R))


def sponge_profile(n_comp, nb, gamma_max):
    out = np.zeros(n_comp)
    _chk(lib().or_sponge_profile(n_comp, nb, float(gamma_max), _p(out)), "sponge_profile")
    return out


def extend(field, nb):
    """Physical field -> computational grid: sponge points take the value of
    the nearest physical point (the medium continues into the sponge)."""
    return np.pad(np.asarray(field, dtype=np.float64), nb, mode="edge")


class Setup:
    """Computational-grid medium and damping for a physical model.

    vp: physical velocity (nz, ny, nx) m/s; eps/delta/theta/phi optional TTI
    fields (physical grid, radians for angles). `gamma_vmax` is the velocity
    scale of the sponge (defaults to max vp)."""

    def __init__(self, vp, h, nb, order, dt, R=1e-3, eps=None, delta=None, theta=None,
                 phi=None, gamma_vmax=None):
        self.h, self.nb, self.order, self.dt = float(h), int(nb), int(order), float(dt)
        v = extend(vp, nb)
        self.shape = v.shape
        self.c = dt * dt * v * v
        vmax = float(np.max(vp)) if gamma_vmax is None else float(gamma_vmax)
        gmax = sponge_gamma_max(vmax, nb, h, R) if nb > 0 else 0.0
        nz, ny, nx = self.shape
        self.gx = sponge_profile(nx, nb, gmax)
        self.gy = sponge_profile(ny, nb, gmax)
        self.gz = sponge_profile(nz, nb, gmax)
        self.eps = None if eps is None else extend(eps, nb)
        self.delta = None if delta is None else extend(delta, nb)
        self.theta = None if theta is None else extend(theta, nb)
        self.phi = None if phi is None else extend(phi, nb)


def _pos(xyz):
    if xyz is None:
        return 0, None
    a = _f64(np.asarray(xyz).reshape(-1, 3))
    return a.shape[0], a


# --------------------------------------------------------------------------
# time stepping (Algorithm 1)
# --------------------------------------------------------------------------

def interpolate(u, rec_xyz, h, nb):
    u = _f64(u)
    nrec, rx = _pos(rec_xyz)
    out = np.zeros(nrec)
    nz, ny, nx = u.shape
    _chk(lib().or_interpolate(nx, ny, nz, h, nb, _p(u), nrec, _p(rx), _p(out)), "interpolate")
    return out


def acoustic_step(s: Setup, u, um, src_xyz=None, amp=None, periodic=False, damping=True):
    u, um = _f64(u), _f64(um)
    up = np.empty_like(u)
    nsrc, sx = _pos(src_xyz)
    a = _f64(np.atleast_1d(amp)) if nsrc else None
    nz, ny, nx = u.shape
    g = (s.gx, s.gy, s.gz) if damping else (None, None, None)
    _chk(lib().or_acoustic_step(nx, ny, nz, s.order, s.h, int(periodic), s.nb, s.dt,
                                _p(_f64(s.c)), _p(g[0]), _p(g[1]), _p(g[2]), _p(u), _p(um),
                                nsrc, _p(sx), _p(a), _p(up)), "acoustic_step")
    return up


def acoustic_forward(s: Setup, src_xyz, wavelet, nt, rec_xyz=None, history=False):
    """Returns dict(traces[(nt+1), nrec], u, um, history?)."""
    nsrc, sx = _pos(src_xyz)
    w = _f64(np.asarray(wavelet).reshape(nt, nsrc)) if nsrc else None
    nrec, rx = _pos(rec_xyz)
    traces = np.zeros((nt + 1, max(nrec, 0)))
    u = np.zeros(s.shape)
    um = np.zeros(s.shape)
    hist = np.zeros((nt + 1,) + s.shape) if history else None
    nz, ny, nx = s.shape
    _chk(lib().or_acoustic_forward(nx, ny, nz, s.order, s.h, s.nb, s.dt, _p(_f64(s.c)),
                                   _p(s.gx), _p(s.gy), _p(s.gz), nsrc, _p(sx), _p(w), nt,
                                   nrec, _p(rx), _p(traces) if nrec else None, _p(u), _p(um),
                                   _p(hist)), "acoustic_forward")
    out = {"traces": traces, "u": u, "um": um}
    if history:
        out["history"] = hist
    return out


def acoustic_adjoint(s: Setup, rec_xyz, res, nt, src_xyz=None, history=None):
    """Adjoint of acoustic_forward: returns dict(wavelet_adj[nt, nsrc], grad_m)."""
    nrec, rx = _pos(rec_xyz)
    res = _f64(np.asarray(res).reshape(nt + 1, nrec))
    nsrc, sx = _pos(src_xyz)
    wadj = np.zeros((nt, nsrc)) if nsrc else None
    grad = np.zeros(s.shape) if history is not None else None
    hist = _f64(history) if history is not None else None
    nz, ny, nx = s.shape
    _chk(lib().or_acoustic_adjoint(nx, ny, nz, s.order, s.h, s.nb, s.dt, _p(_f64(s.c)),
                                   _p(s.gx), _p(s.gy), _p(s.gz), nrec, _p(rx), _p(res), nt,
                                   nsrc, _p(sx), _p(wadj), _p(hist), _p(grad)),
         "acoustic_adjoint")
    return {"wavelet_adj": wadj, "grad_m": grad}


def tti_step(s: Setup, p, pm, r, rm, src_xyz=None, amp=None, periodic=False, damping=True):
    p, pm, r, rm = _f64(p), _f64(pm), _f64(r), _f64(rm)
    pp, rp = np.empty_like(p), np.empty_like(r)
    nsrc, sx = _pos(src_xyz)
    a = _f64(np.atleast_1d(amp)) if nsrc else None
    nz, ny, nx = p.shape
    g = (s.gx, s.gy, s.gz) if damping else (None, None, None)
    _chk(lib().or_tti_step(nx, ny, nz, s.order, s.h, int(periodic), s.nb, s.dt, _p(_f64(s.c)),
                           _p(s.eps), _p(s.delta), _p(s.theta), _p(s.phi), _p(g[0]), _p(g[1]),
                           _p(g[2]), _p(p), _p(pm), _p(r), _p(rm), nsrc, _p(sx), _p(a),
                           _p(pp), _p(rp)), "tti_step")
    return pp, rp


def tti_forward(s: Setup, src_xyz, wavelet, nt, rec_xyz=None):
    """Returns dict(traces, p, pm, r, rm)."""
    nsrc, sx = _pos(src_xyz)
    w = _f64(np.asarray(wavelet).reshape(nt, nsrc)) if nsrc else None
    nrec, rx = _pos(rec_xyz)
    traces = np.zeros((nt + 1, max(nrec, 0)))
    fields = np.zeros((4,) + s.shape)
    nz, ny, nx = s.shape
    _chk(lib().or_tti_forward(nx, ny, nz, s.order, s.h, s.nb, s.dt, _p(_f64(s.c)), _p(s.eps),
                              _p(s.delta), _p(s.theta), _p(s.phi), _p(s.gx), _p(s.gy), _p(s.gz),
                              nsrc, _p(sx), _p(w), nt, nrec, _p(rx),
                              _p(traces) if nrec else None, _p(fields)), "tti_forward")
    return {"traces": traces, "p": fields[0], "pm": fields[1], "r": fields[2], "rm": fields[3]}


class _BlockSetup:
    """Medium of a small block: constant c, damping given per axis."""

    def __init__(self, shape, h, nb, order, dt, c, gx, gy, gz):
        self.shape, self.h, self.nb, self.order, self.dt = shape, h, nb, order, dt
        self.c = np.full(shape, c)
        self.gx, self.gy, self.gz = gx, gy, gz


def acoustic_update_at(u_block, um_c, v_c, gamma_c, h, order, dt):
    """u_{n+1} at the centre of a (2r+1)^3 block of u_n (no source): the
    oracle step run on the block, whose centre stencil stays inside it.
    v_c, um_c, gamma_c: velocity, u_{n-1} and damping gamma at the centre."""
    r = order // 2
    n = 2 * r + 1
    assert u_block.shape == (n, n, n)
    gx = np.full(n, float(gamma_c))
    z = np.zeros(n)
    s = _BlockSetup((n, n, n), h, 0, order, dt, dt * dt * float(v_c) ** 2, gx, z, z)
    um = np.zeros((n, n, n))
    um[r, r, r] = um_c
    return acoustic_step(s, u_block, um)[r, r, r]


class _TtiBlockSetup(_BlockSetup):
    """Medium of a small TTI block: every field constant (the centre's)."""

    def __init__(self, shape, h, order, dt, v, eps, delta, theta, phi, gamma):
        n = shape[0]
        super().__init__(shape, h, 0, order, dt, dt * dt * float(v) ** 2, np.full(n, float(gamma)),
                         np.zeros(n), np.zeros(n))
        self.eps = np.full(shape, float(eps))
        self.delta = np.full(shape, float(delta))
        self.theta = np.full(shape, float(theta))
        self.phi = np.full(shape, float(phi))


def tti_update_at(p_block, pm_c, r_block, rm_c, v_c, eps_c, delta_c, theta_c, phi_c, gamma_c, h,
                  order, dt):
    """(p_{n+1}, r_{n+1}) at the centre of (2r+1)^3 blocks of p_n, r_n (no
    source): the oracle's TTI step run on the blocks with the centre's medium
    everywhere. The centre's operator reads p and r within r points along
    each axis (second derivatives, and cross derivatives with both offsets
    <= r) and the medium at the centre only, so it stays inside the block."""
    r = order // 2
    n = 2 * r + 1
    assert p_block.shape == (n, n, n) and r_block.shape == (n, n, n)
    s = _TtiBlockSetup((n, n, n), h, order, dt, v_c, eps_c, delta_c, theta_c, phi_c, gamma_c)
    pm = np.zeros((n, n, n))
    rm = np.zeros((n, n, n))
    pm[r, r, r], rm[r, r, r] = pm_c, rm_c
    pp, rp = tti_step(s, p_block, pm, r_block, rm)
    return pp[r, r, r], rp[r, r, r]


def extend_adjoint(g, nb):
    """Adjoint of `extend`: each physical point collects the computational
    points that copy its value (separable: per axis, the nb sponge slices
    beyond a face add onto the face slice)."""
    g = np.asarray(g, dtype=np.float64)
    if nb == 0:
        return g.copy()
    for ax in range(3):
        a = np.moveaxis(g, ax, 0)
        inner = a[nb:a.shape[0] - nb].copy()
        inner[0] += a[:nb].sum(axis=0)
        inner[-1] += a[a.shape[0] - nb:].sum(axis=0)
        g = np.moveaxis(inner, 0, ax)
    return np.ascontiguousarray(g)


# --------------------------------------------------------------------------
# learned closure (3x3x3 conv net, fdoracle.c)
# --------------------------------------------------------------------------

def closure_num_params(hidden=16):
    L = lib()
    L.or_closure_num_params.argtypes = [_I]
    L.or_closure_num_params.restype = ctypes.c_long
    return int(L.or_closure_num_params(hidden))


def closure_forward(params, x, hidden=16):
    """x [3, nz, ny, nx] -> out [nz-6, ny-6, nx-6] (valid 3x3x3 convolutions)."""
    L = lib()
    L.or_closure_forward.argtypes = [_I, _I, _I, _I, _D, _D, _D, _D, _D]
    L.or_closure_forward.restype = _I
    params, x = _f64(params), _f64(x)
    _, nz, ny, nx = x.shape
    out = np.zeros((nz - 6, ny - 6, nx - 6))
    _chk(L.or_closure_forward(hidden, nz, ny, nx, _p(params), _p(x), None, None, _p(out)),
         "closure_forward")
    return out


def closure_loss_grad(params, x, target, hidden=16, grad=True):
    """Mean-squared error of a batch x [B, 3, nz, ny, nx] against target
    [B, nz-6, ny-6, nx-6] and its gradient w.r.t. the parameters."""
    L = lib()
    L.or_closure_loss_grad.argtypes = [_I, _I, _I, _I, _I, _D, _D, _D, _D, _D]
    L.or_closure_loss_grad.restype = _I
    params, x, target = _f64(params), _f64(x), _f64(target)
    B, _, nz, ny, nx = x.shape
    loss = np.zeros(1)
    g = np.zeros(params.size) if grad else None
    _chk(L.or_closure_loss_grad(hidden, B, nz, ny, nx, _p(params), _p(x), _p(target), _p(loss),
                                _p(g)), "closure_loss_grad")
    return float(loss[0]), g


def closure_forward_same(params, x, hidden=16):
    """The closure net on a whole grid, as the time loop applies it: every
    3x3x3 convolution keeps the grid's size and reads zeros outside it.
    x [3, nz, ny, nx] -> [nz, ny, nx]. Parameter layout as in fdoracle.c
    (W1[H][3][27], b1, W2[H][H][27], b2, W3[1][H][27], b3; tap (a*3+b)*3+c
    for offsets (a-1, b-1, c-1) along (z, y, x))."""
    p = _f64(params)
    x = _f64(x)
    H = hidden
    layers = []
    off = 0
    for ci, co in ((3, H), (H, H), (H, 1)):
        W = p[off:off + co * ci * 27].reshape(co, ci, 27)
        off += co * ci * 27
        b = p[off:off + co]
        off += co
        layers.append((W, b))
    a = x
    for li, (W, b) in enumerate(layers):
        _, nz, ny, nx = a.shape
        ap = np.pad(a, ((0, 0), (1, 1), (1, 1), (1, 1)))
        out = np.broadcast_to(b[:, None, None, None], (W.shape[0], nz, ny, nx)).copy()
        for ta in range(3):
            for tb in range(3):
                for tc in range(3):
                    tap = (ta * 3 + tb) * 3 + tc
                    out += np.einsum("oi,izyx->ozyx", W[:, :, tap],
                                     ap[:, ta:ta + nz, tb:tb + ny, tc:tc + nx])
        a = np.maximum(out, 0.0) if li < 2 else out
    return a[0]


def closure_correction(params, x, hidden=16):
    """net(x) - net(x0) of a patch x [3, nz, ny, nx] (valid convolutions),
    x0 = x with the two wavefield channels set to zero."""
    x = _f64(x)
    x0 = x.copy()
    x0[:2] = 0.0
    return closure_forward(params, x, hidden) - closure_forward(params, x0, hidden)


def closure_correction_loss_grad(params, x, target, hidden=16):
    """Mean-squared error of net(x) - net(x0) against target for a batch
    x [B, 3, nz, ny, nx], and its gradient w.r.t. the parameters.

    With r = net(x) - net(x0) - target, the gradient is (2/M) sum r (d net(x)
    - d net(x0)). Each half is a vector-Jacobian product, obtained from the
    plain loss gradient: the gradient of mean (net(y) - (net(y) - r))^2 is
    exactly (2/M) sum r d net(y)."""
    params, x, target = _f64(params), _f64(x), _f64(target)
    B = x.shape[0]
    x0 = x.copy()
    x0[:, :2] = 0.0
    f = np.stack([closure_forward(params, x[b], hidden) for b in range(B)])
    f0 = np.stack([closure_forward(params, x0[b], hidden) for b in range(B)])
    r = f - f0 - target
    loss = float(np.mean(r * r))
    _, g1 = closure_loss_grad(params, x, f - r, hidden)
    _, g0 = closure_loss_grad(params, x0, f0 - r, hidden)
    return loss, g1 - g0


def closure_step(s: Setup, u, um, vp, params, src_xyz=None, amp=None, hidden=16):
    """One coarse step with the closure: the acoustic update of Algorithm 1
    plus m * (net(x) - net(x0)), x = (u_n / m, u_{n-1} / m, (v - 3000) / 750),
    x0 = (0, 0, (v - 3000) / 750), m = max |u_n| (1e-30 for a zero level),
    v the physical model extended into the sponge, every convolution
    zero-padded to the grid's size; the correction is added on the physical
    points whose 7^3 receptive field is physical (3 points or more from the
    sponge); elsewhere the plain update stands. Returns u_{n+1}."""
    u, um = _f64(u), _f64(um)
    up = acoustic_step(s, u, um)
    m = float(np.max(np.abs(u)))
    m = m if m > 1e-30 else 1e-30
    vn = (extend(vp, s.nb) - 3000.0) / 750.0
    z = np.zeros_like(u)
    corr = (closure_forward_same(params, np.stack([u / m, um / m, vn]), hidden)
            - closure_forward_same(params, np.stack([z, z, vn]), hidden))
    a = s.nb + 3
    inner = tuple(slice(a, n - a) for n in u.shape)
    up[inner] += m * corr[inner]
    if src_xyz is not None:
        # the source term alone: a step of zero fields injects exactly it
        up = up + acoustic_step(s, z, z, src_xyz, amp)
    return up
