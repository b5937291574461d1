"""ctypes binding of libfdwave (include/fdwave.h): argument marshalling only.

Every compute step runs in the CUDA library; this module converts numpy
arrays / torch tensors into pointers and checks return codes. Importing it
does not load the library; the first call does, and fails loudly when the
library has not been built (``python -c "import __graft_entry__ as g;
g.build()"``) -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

FDW_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "UNSTABLE_DT", -3: "OOM", -4: "CUDA", -5: "STATE",
          -6: "DIVERGED", -7: "OUT_OF_DOMAIN", -8: "DEVICE_TIMEOUT"}
ACOUSTIC, TTI = 0, 1
STORAGE = {"f32": 0, "bf16": 1, "f16": 2}
EQUATION = {"acoustic": ACOUSTIC, "tti": TTI}

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

_SIGS = {
    "fdw_last_error": ([], ctypes.c_char_p),
    "fdw_version": ([], ctypes.c_char_p),
    "fdw_create": ([ctypes.POINTER(_P), _I, _I, _I, _D, _I, _I, _I, _I, _P], _I),
    "fdw_destroy": ([_P], _I),
    "fdw_set_model": ([_P, _P, _P, _P, _P, _P, _I], _I),
    "fdw_max_stable_dt": ([_P], _D),
    "fdw_set_dt": ([_P, _D], _I),
    "fdw_set_sources": ([_P, _I, _P, _P, _I, _I], _I),
    "fdw_set_receivers": ([_P, _I, _P, _I], _I),
    "fdw_reset": ([_P], _I),
    "fdw_current_step": ([_P], _I),
    "fdw_set_current_step": ([_P, _I], _I),
    "fdw_step": ([_P, _I], _I),
    "fdw_gather_receivers": ([_P, _P, _I], _I),
    "fdw_get_wavefield": ([_P, _I, _I, _P, _I], _I),
    "fdw_set_wavefield": ([_P, _I, _I, _P, _I], _I),
    "fdw_check": ([_P, _I], _I),
    "fdw_set_kernel_variant": ([_P, _I], _I),
    "fdw_set_zchunks": ([_P, _I], _I),
    "fdw_get_zchunks": ([_P], _I),
    "fdw_set_tile_config": ([_P, _I], _I),
    "fdw_get_tile_config": ([_P], _I),
    "fdw_set_sponge": ([_P, _D, _D], _I),
    "fdw_set_field_scale": ([_P, _D], _I),
    "fdw_get_field_scale": ([_P], _D),
    "fdw_history_begin": ([_P, _I], _I),
    "fdw_history_end": ([_P], _I),
    "fdw_adjoint_begin": ([_P, _P, _I, _I, _I], _I),
    "fdw_adjoint_step": ([_P, _I], _I),
    "fdw_adjoint_current_step": ([_P], _I),
    "fdw_get_gradient": ([_P, _P, _I], _I),
    "fdw_get_source_adjoint": ([_P, _P, _I], _I),
    "fdw_get_adjoint_wavefield": ([_P, _I, _P, _I], _I),
    "fdw_misfit": ([_P, _P, ctypes.c_longlong, _P, _P, _P], _I),
    "fdw_misfit_noalloc": ([_P, _P, ctypes.c_longlong, _P, _P, _P], _I),
    "fdw_velocity_gradient": ([_P, _P, ctypes.c_longlong, _P, _P], _I),
    "fdw_closure_num_params": ([], ctypes.c_longlong),
    "fdw_closure_create": ([ctypes.POINTER(_P), _P], _I),
    "fdw_closure_destroy": ([_P], _I),
    "fdw_closure_set_variant": ([_P, _I], _I),
    "fdw_closure_set_params": ([_P, _P, _I], _I),
    "fdw_closure_get_params": ([_P, _P, _I], _I),
    "fdw_closure_forward": ([_P, _P, _I, _I, _P], _I),
    "fdw_closure_loss_grad": ([_P, _P, _P, _I, _I, _P, _P], _I),
    "fdw_closure_adam_step": ([_P, _P, _P, _I, _I, ctypes.c_float, _P], _I),
    "fdw_step_closure": ([_P, _P, _I], _I),
    "fdw_step_closure_every": ([_P, _P, _I, _I], _I),
    "fdw_profile_begin": ([_P, _I], _I),
    "fdw_profile_end": ([_P, ctypes.POINTER(_D), ctypes.POINTER(_I)], _I),
}


class FdwError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("fdwave error %d (%s): %s" % (code, ERRORS.get(code, "?"), msg))
        self.code = code


def library_path() -> str:
    return _build.SO


def lib(build_if_missing: bool = False):
    """Load libfdwave.so (raises if it is missing: no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError("libfdwave.so is not built (%s); run "
                                       "`python -c \"import __graft_entry__ as g; g.build()\"`"
                                       % path)
                _build.build()
            L = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def declared_symbols(header: str | None = None):
    """Names of the functions declared in include/fdwave.h."""
    header = header or os.path.join(_build.INCLUDE, "fdwave.h")
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fdw_\w+)\s*\(", text)))


def _chk(rc):
    if rc != FDW_OK:
        raise FdwError(rc, lib().fdw_last_error().decode())
    return rc


def _is_torch(a):
    return type(a).__module__.split(".")[0] == "torch"


def _ptr(a, dtype):
    """(pointer, is_device, keepalive) for a numpy array or torch tensor."""
    if a is None:
        return None, 0, None
    if _is_torch(a):
        import torch
        tdt = {np.float32: torch.float32, np.float64: torch.float64}[dtype]
        t = a.detach().contiguous()
        if t.dtype != tdt:
            t = t.to(tdt)
        return t.data_ptr(), int(t.is_cuda), t
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, 0, arr


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _cuda_f64(t, name):
    import torch
    if not (_is_torch(t) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("%s must be a contiguous float64 CUDA tensor" % name)
    return t.data_ptr()


def misfit(d, d_obs, residual=None, J=None, stream=None):
    """Residual d - d_obs (into `residual` if given) and J = 1/2 sum r^2 by
    fdw_misfit; d, d_obs, residual, J are float64 CUDA tensors. Returns J
    (a 0-d CUDA tensor), asynchronous on the stream."""
    import torch
    n = d.numel()
    if d_obs.numel() != n or (residual is not None and residual.numel() != n):
        raise ValueError("size mismatch")
    if J is None:
        J = torch.empty((), dtype=torch.float64, device=d.device)
    rp = _cuda_f64(residual, "residual") if residual is not None else None
    _chk(lib().fdw_misfit(_cuda_f64(d, "d"), _cuda_f64(d_obs, "d_obs"), n, rp,
                          _cuda_f64(J, "J"), _stream_handle(stream)))
    return J


def velocity_gradient(vp, grad_m, out=None, stream=None):
    """dJ/dv = -2 v^-3 dJ/dm by fdw_velocity_gradient: vp a float32 CUDA
    tensor, grad_m a float64 CUDA tensor of the same size; returns float64
    (into `out` if given), asynchronous on the stream."""
    import torch
    if not (_is_torch(vp) and vp.is_cuda and vp.dtype == torch.float32 and vp.is_contiguous()):
        raise ValueError("vp must be a contiguous float32 CUDA tensor")
    n = vp.numel()
    if grad_m.numel() != n:
        raise ValueError("size mismatch")
    if out is None:
        out = torch.empty_like(grad_m)
    _chk(lib().fdw_velocity_gradient(vp.data_ptr(), _cuda_f64(grad_m, "grad_m"), n,
                                     _cuda_f64(out, "out"), _stream_handle(stream)))
    return out


class Closure:
    """The learned closure network of fdwave.h (3x3x3 convs 3 -> 16 -> 16 -> 1).
    Batches are float32 CUDA tensors [B, 3, S, S, S]; targets [B, S-6, S-6, S-6]."""

    def __init__(self, stream=None):
        self.stream = _stream_handle(stream)
        h = _P()
        _chk(lib().fdw_closure_create(ctypes.byref(h), self.stream))
        self._h = h
        self.num_params = int(lib().fdw_closure_num_params())

    def close(self):
        if getattr(self, "_h", None):
            lib().fdw_closure_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_variant(self, variant):
        """Inference kernels of Solver.step_closure: 0 tcgen05 tensor-core
        kernel (default), 1 FP32 CUDA-core convolutions, 2 mma.sync
        tensor-core kernel."""
        _chk(lib().fdw_closure_set_variant(self._h, int(variant)))

    def set_params(self, p):
        ptr, dev, keep = _ptr(p, np.float32)
        if (keep.numel() if _is_torch(keep) else keep.size) != self.num_params:
            raise ValueError("expected %d parameters" % self.num_params)
        _chk(lib().fdw_closure_set_params(self._h, ptr, dev))

    def get_params(self):
        out = np.zeros(self.num_params, dtype=np.float32)
        _chk(lib().fdw_closure_get_params(self._h, out.ctypes.data, 0))
        return out

    @staticmethod
    def _batch(x):
        import torch
        if not (x.is_cuda and x.dtype == torch.float32 and x.is_contiguous() and x.dim() == 5
                and x.shape[1] == 3 and x.shape[2] == x.shape[3] == x.shape[4]):
            raise ValueError("x must be a contiguous float32 CUDA tensor [B, 3, S, S, S]")
        return x.shape[0], x.shape[2]

    def forward(self, x, out=None):
        import torch
        B, S = self._batch(x)
        if out is None:
            out = torch.empty((B, S - 6, S - 6, S - 6), dtype=torch.float32, device=x.device)
        _chk(lib().fdw_closure_forward(self._h, x.data_ptr(), B, S, out.data_ptr()))
        return out

    def loss_grad(self, x, target, grad=True):
        import torch
        B, S = self._batch(x)
        loss = torch.empty((), dtype=torch.float32, device=x.device)
        g = torch.empty(self.num_params, dtype=torch.float32, device=x.device) if grad else None
        _chk(lib().fdw_closure_loss_grad(self._h, x.data_ptr(), target.contiguous().data_ptr(), B, S,
                                         loss.data_ptr(), g.data_ptr() if grad else None))
        return loss, g

    def adam_step(self, x, target, lr, loss=None):
        import torch
        B, S = self._batch(x)
        if loss is None:
            loss = torch.empty((), dtype=torch.float32, device=x.device)
        _chk(lib().fdw_closure_adam_step(self._h, x.data_ptr(), target.contiguous().data_ptr(), B, S,
                                         float(lr), loss.data_ptr()))
        return loss


class Solver:
    """One wave-equation solver on the current CUDA device.

    shape: physical grid (nz, ny, nx); h metres; nb sponge points per face;
    order: space order 2..16; equation: "acoustic" | "tti";
    storage: "f32" | "bf16" | "f16". Stream: torch stream / raw handle /
    None (torch's current stream)."""

    def __init__(self, shape, h, nb, order, equation="acoustic", storage="f32", stream=None):
        self.shape = tuple(int(n) for n in shape)
        self.h, self.nb, self.order = float(h), int(nb), int(order)
        self.equation, self.storage = equation, storage
        nz, ny, nx = self.shape
        self.comp_shape = (nz + 2 * nb, ny + 2 * nb, nx + 2 * nb)
        self.stream = _stream_handle(stream)
        handle = _P()
        # VTI (Eq. vVTI) is the TTI system with a vertical symmetry axis
        eq = EQUATION["tti" if equation == "vti" else equation]
        _chk(lib().fdw_create(ctypes.byref(handle), nx, ny, nz, self.h, self.nb,
                              eq, self.order, STORAGE[storage], self.stream))
        self._h = handle
        self.nrec = 0
        self.nt_rec = 0

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().fdw_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- set-up -----------------------------------------------------------
    def set_model(self, vp, eps=None, delta=None, theta=None, phi=None):
        if self.equation == "vti":
            if theta is not None or phi is not None:
                raise ValueError("VTI has a vertical axis: no theta/phi")
            if _is_torch(vp):
                import torch
                theta = torch.zeros_like(vp, dtype=torch.float32)
            else:
                theta = np.zeros(np.shape(vp), dtype=np.float32)
            phi = theta
        ptrs = [_ptr(a, np.float32) for a in (vp, eps, delta, theta, phi)]
        dev = ptrs[0][1]
        if any(p[0] is not None and p[1] != dev for p in ptrs):
            raise ValueError("model arrays must all be host or all device")
        _chk(lib().fdw_set_model(self._h, *[p[0] for p in ptrs], dev))
        return self

    def set_sponge(self, vref=0.0, R=1e-3):
        """Fix the sponge's velocity scale (vref <= 0: the model's vmax)."""
        _chk(lib().fdw_set_sponge(self._h, float(vref), float(R)))
        return self

    def set_field_scale(self, scale=0.0):
        """Storage scale of the wavefields (0: automatic, see fdwave.h)."""
        _chk(lib().fdw_set_field_scale(self._h, float(scale)))
        return self

    @property
    def field_scale(self):
        return lib().fdw_get_field_scale(self._h)

    def max_stable_dt(self):
        return lib().fdw_max_stable_dt(self._h)

    def set_dt(self, dt):
        _chk(lib().fdw_set_dt(self._h, float(dt)))
        self.dt = float(dt)
        return self

    def set_sources(self, xyz, wavelet):
        xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
        nsrc = xyz.shape[0]
        if nsrc == 0:
            _chk(lib().fdw_set_sources(self._h, 0, None, None, 0, 0))
            return self
        wp, dev, keep = _ptr(wavelet, np.float32)
        nt = (keep.numel() if _is_torch(keep) else keep.size) // nsrc
        _chk(lib().fdw_set_sources(self._h, nsrc, xyz.ctypes.data, wp, nt, dev))
        return self

    def set_receivers(self, xyz, nt):
        xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
        _chk(lib().fdw_set_receivers(self._h, xyz.shape[0], xyz.ctypes.data if xyz.size else None,
                                     int(nt)))
        self.nrec, self.nt_rec = xyz.shape[0], int(nt)
        return self

    # -- time loop --------------------------------------------------------
    def reset(self):
        _chk(lib().fdw_reset(self._h))
        return self

    @property
    def current_step(self):
        return lib().fdw_current_step(self._h)

    def set_current_step(self, n):
        _chk(lib().fdw_set_current_step(self._h, int(n)))

    def step(self, n=1):
        _chk(lib().fdw_step(self._h, int(n)))
        return self

    def step_closure(self, closure, n=1, every=1):
        """n steps with the learned closure applied after every update, or
        (every > 1) on every `every`-th step with the correction times
        `every` (the others are plain steps)."""
        if int(every) == 1:
            _chk(lib().fdw_step_closure(self._h, closure._h, int(n)))
        else:
            _chk(lib().fdw_step_closure_every(self._h, closure._h, int(n), int(every)))
        return self

    def check(self, finite=True):
        _chk(lib().fdw_check(self._h, int(finite)))

    # -- outputs / state ---------------------------------------------------
    def traces(self, out=None):
        """Receiver traces [(nt+1), nrec] float64 (numpy, or into a torch tensor)."""
        if out is None:
            out = np.zeros((self.nt_rec + 1, self.nrec), dtype=np.float64)
        p, dev, keep = _ptr(out, np.float64)
        _chk(lib().fdw_gather_receivers(self._h, p, dev))
        return keep if not _is_torch(out) or keep is out else out.copy_(keep)

    def wavefield(self, field=0, level=0, out=None):
        """Computational-grid field level as float32 (numpy, or into a torch tensor)."""
        if out is None:
            out = np.zeros(self.comp_shape, dtype=np.float32)
        p, dev, keep = _ptr(out, np.float32)
        _chk(lib().fdw_get_wavefield(self._h, int(field), int(level), p, dev))
        return keep if not _is_torch(out) or keep is out else out.copy_(keep)

    def set_wavefield(self, data, field=0, level=0):
        p, dev, keep = _ptr(data, np.float32)
        _chk(lib().fdw_set_wavefield(self._h, int(field), int(level), p, dev))

    # -- tuning / cross-checks ---------------------------------------------
    def set_kernel_variant(self, variant):
        """0 = 2.5D TMA kernel (default), 1 = one-thread-per-point kernel."""
        _chk(lib().fdw_set_kernel_variant(self._h, int(variant)))

    def set_zchunks(self, zchunks):
        _chk(lib().fdw_set_zchunks(self._h, int(zchunks)))

    def set_tile_config(self, tile):
        """Tile configuration of the 2.5D kernel (acoustic 0..12, TTI 0..12 with
        9..12 up to order 8), -1 = default."""
        _chk(lib().fdw_set_tile_config(self._h, int(tile)))

    @property
    def tile_config(self):
        return lib().fdw_get_tile_config(self._h)

    @property
    def zchunks(self):
        return lib().fdw_get_zchunks(self._h)

    # -- adjoint / FWI gradient --------------------------------------------
    def history_begin(self, nlevels):
        _chk(lib().fdw_history_begin(self._h, int(nlevels)))

    def history_end(self):
        _chk(lib().fdw_history_end(self._h))

    def adjoint_begin(self, residual, gradient=True):
        """residual: [(nt+1), nrec] float64 (numpy or torch, host or device)."""
        p, dev, keep = _ptr(residual, np.float64)
        n = keep.shape[0] - 1
        self._res_keep = keep
        _chk(lib().fdw_adjoint_begin(self._h, p, int(n), dev, int(bool(gradient))))

    def adjoint_step(self, n=1):
        _chk(lib().fdw_adjoint_step(self._h, int(n)))

    @property
    def adjoint_current_step(self):
        return lib().fdw_adjoint_current_step(self._h)

    def gradient(self, out=None):
        """dJ/dm (m = 1/v^2) on the physical grid, float64."""
        if out is None:
            out = np.zeros(self.shape, dtype=np.float64)
        p, dev, keep = _ptr(out, np.float64)
        _chk(lib().fdw_get_gradient(self._h, p, dev))
        return keep if not _is_torch(out) or keep is out else out.copy_(keep)

    def source_adjoint(self, nt, nsrc):
        out = np.zeros((nt, nsrc), dtype=np.float64)
        _chk(lib().fdw_get_source_adjoint(self._h, out.ctypes.data, 0))
        return out

    def adjoint_wavefield(self, level=0):
        out = np.zeros(self.comp_shape, dtype=np.float32)
        _chk(lib().fdw_get_adjoint_wavefield(self._h, int(level), out.ctypes.data, 0))
        return out

    def profile_begin(self, max_launches=65536):
        _chk(lib().fdw_profile_begin(self._h, int(max_launches)))

    def profile_end(self):
        """(summed stencil-kernel milliseconds, number of launches timed)."""
        ms, n = _D(), _I()
        _chk(lib().fdw_profile_end(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value
