"""FWI velocity gradient through torch.autograd, on the library's adjoint.

`fwi_traces(vp, survey)` returns the traces of every shot; its backward pass
runs, per shot, the adjoint of the discrete recurrence (fdw_adjoint_*) with
checkpointing: the forward run keeps (u_n, u_{n-1}) every `segment` steps;
the backward pass, segment by segment from the last, restores the
checkpoint, replays the segment into the library's history ring and runs
that segment's adjoint steps, accumulating dJ/dm (m = 1/v^2) on the device
in FP32 per segment and FP64 overall. The chain rule to velocity is
dJ/dv = -2 v^-3 dJ/dm. This module only orchestrates library calls.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

from . import fdwave


@dataclasses.dataclass
class Survey:
    shape: tuple            # physical (nz, ny, nx)
    h: float
    nb: int
    order: int
    dt: float
    nt: int
    src_xyz: np.ndarray     # (nshot, 3): one source per shot
    wavelet: np.ndarray     # (nt,) float32, shared by the shots
    rec_xyz: np.ndarray     # (nrec, 3), shared by the shots
    checkpoints: int = 20
    keep_checkpoints: bool = True   # False: recompute each shot's forward run in backward
    storage: str = "f32"
    sponge_vref: float = 0.0        # fixed sponge velocity scale (0: the model's vmax)

    @property
    def nshot(self):
        return int(self.src_xyz.shape[0])

    @property
    def segment(self):
        return max(1, math.ceil(self.nt / self.checkpoints))


class _Engine:
    """One solver reused for every shot (buffers stay allocated)."""

    def __init__(self, survey: Survey):
        self.sv = survey
        self.solver = fdwave.Solver(survey.shape, survey.h, survey.nb, survey.order,
                                    storage=survey.storage)
        self.solver.set_receivers(survey.rec_xyz, survey.nt)

    def set_model(self, vp):
        # the gradient holds the sponge fixed: pin its velocity scale
        self.solver.set_model(vp).set_sponge(self.sv.sponge_vref).set_dt(self.sv.dt)

    def forward_shot(self, k, keep):
        """Run shot k; returns (traces [nt+1, nrec] float64 cuda, checkpoints)."""
        s, sv = self.solver, self.sv
        s.set_sources(sv.src_xyz[k:k + 1], sv.wavelet.reshape(-1, 1))
        s.reset()
        ck = []
        comp = s.comp_shape
        for t0 in range(0, sv.nt, sv.segment):
            if keep:
                u = torch.empty(comp, dtype=torch.float32, device="cuda")
                um = torch.empty_like(u)
                s.wavefield(0, 0, out=u)
                s.wavefield(0, 1, out=um)
                ck.append((t0, u, um))
            s.step(min(sv.segment, sv.nt - t0))
        tr = torch.empty((sv.nt + 1, s.nrec), dtype=torch.float64, device="cuda")
        s.traces(out=tr)
        return tr, ck

    def adjoint_shot(self, k, residual, ck):
        """dJ/dm (physical grid, float64 cuda) of shot k for dJ/dtraces = residual."""
        s, sv = self.solver, self.sv
        if not ck:
            _, ck = self.forward_shot(k, keep=True)
        else:
            s.set_sources(sv.src_xyz[k:k + 1], sv.wavelet.reshape(-1, 1))
        s.adjoint_begin(residual.contiguous(), gradient=True)
        for t0, u, um in reversed(ck):
            t1 = min(t0 + sv.segment, sv.nt)
            s.set_wavefield(u, 0, 0)
            s.set_wavefield(um, 0, 1)
            s.set_current_step(t0)
            s.history_begin(sv.segment + 2)
            s.step(t1 - t0)
            s.history_end()
            s.adjoint_step(t1 - t0)
        g = torch.empty(sv.shape, dtype=torch.float64, device="cuda")
        s.gradient(out=g)
        return g

    def close(self):
        self.solver.close()


class FwiTraces(torch.autograd.Function):
    """traces[shot] = F(vp) for every shot; backward gives dJ/dvp."""

    @staticmethod
    def forward(ctx, vp, survey: Survey):
        eng = _Engine(survey)
        eng.set_model(vp.detach().float().contiguous())
        outs, cks = [], []
        for k in range(survey.nshot):
            tr, ck = eng.forward_shot(k, keep=survey.keep_checkpoints)
            outs.append(tr)
            cks.append(ck)
        ctx.eng, ctx.cks = eng, cks
        ctx.save_for_backward(vp)
        return torch.stack(outs)

    @staticmethod
    def backward(ctx, grad_traces):
        (vp,) = ctx.saved_tensors
        eng, cks = ctx.eng, ctx.cks
        gm = torch.zeros(vp.shape, dtype=torch.float64, device="cuda")
        for k in range(eng.sv.nshot):
            gm += eng.adjoint_shot(k, grad_traces[k].double(), cks[k])
            cks[k] = None
        eng.close()
        gv = fdwave.velocity_gradient(vp.detach().float().contiguous(), gm)
        return gv.to(vp.dtype), None


def fwi_traces(vp, survey: Survey):
    return FwiTraces.apply(vp, survey)


def misfit_and_gradient(vp, survey: Survey, d_obs):
    """J = 1/2 sum (F(vp) - d_obs)^2 over shots and its gradient dJ/dvp,
    shot by shot (forward with checkpoints, residual and misfit by
    fdw_misfit, adjoint with checkpoint replay), so only one shot's
    checkpoints are held at a time."""
    eng = _Engine(survey)
    eng.set_model(vp.detach().float().contiguous())
    J = torch.zeros((), dtype=torch.float64, device="cuda")
    Jk = torch.empty_like(J)
    gm = torch.zeros(vp.shape, dtype=torch.float64, device="cuda")
    for k in range(survey.nshot):
        tr, ck = eng.forward_shot(k, keep=True)
        res = torch.empty_like(tr)
        fdwave.misfit(tr, d_obs[k].contiguous(), residual=res, J=Jk)
        J += Jk
        gm += eng.adjoint_shot(k, res, ck)
        del ck
    eng.close()
    return J, fdwave.velocity_gradient(vp.detach().float().contiguous(), gm).to(vp.dtype)
