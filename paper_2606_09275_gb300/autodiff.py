"""The reaction force of a sequence of load steps as a differentiable function
of the per-point Young's modulus and yield stress.

Forward: the load steps of `mpm.step` (Sec. 2.4, with the Sec. 5 re-adaptation),
keeping the point state at the start of every step as a device checkpoint.
Backward: `mpm.adjoint`, the discrete adjoint of those steps, with the
discrete events of the forward run held fixed.  Both directions run in the
library's CUDA kernels; this module only arranges tensors and calls.
"""
import numpy as np
import torch

from . import inputs, mpm


class LoadPath:
    """A load-step sequence: workload parameters, initial points and the Newton
    and Krylov settings used by both the forward run and the adjoint."""

    def __init__(self, ctx, cfg, points, nsteps, capacity=None, tol=1e-12, maxit=30, lin_tol=1e-12,
                 lin_maxit=200000, precision=mpm.FP64, method=0, mg_reuse=0, store_increments=True):
        self.ctx, self.cfg, self.points, self.nsteps = ctx, cfg, points, nsteps
        self.capacity = capacity or 64 * len(points["x"])
        # keep each step's converged increment with its checkpoint, so that the
        # adjoint does not solve the step again (one nodal vector per step)
        self.store_increments = store_increments
        self.kw = dict(tol=tol, maxit=maxit, lin_tol=lin_tol, lin_maxit=lin_maxit,
                       precision=precision, method=method, mg_reuse=mg_reuse)

    def schedule(self, n):
        """(body position, load factor) of load step n (0-based)."""
        bz = inputs.body_z(self.cfg, n + 1) if self.cfg.get("body") else 0.0
        return bz, inputs.load_factor(self.cfg, n + 1)

    def run(self, E, ys, keep=True):
        """Run the steps with the given device E, ys; returns (reaction of the
        last step as a float64 tensor, checkpoints, per-step statistics)."""
        pts = mpm.Points(self.points, capacity=self.capacity)
        n0 = pts.count
        pts.t["E"][:n0] = E.detach().to(pts.t["E"].device, torch.float64)
        pts.t["ys"][:n0] = ys.detach().to(pts.t["ys"].device, torch.float64)
        ckpts, stats = [], []
        # nodal increments: at most 3 per node, and a mesh has fewer active
        # nodes than 8 per point
        du = (torch.empty(24 * self.capacity, dtype=torch.float64, device=pts.t["x"].device)
              if keep and self.store_increments else None)
        for n in range(self.nsteps):
            bz, ld = self.schedule(n)
            if keep:
                start = pts.clone()
            st = mpm.step(self.ctx, self.cfg, pts, body_z=bz, load=ld, du_out=du, **self.kw)
            stats.append(st)
            if keep:
                ckpts.append((start, bz, ld, du[:3 * st["ndof"]].clone()) if du is not None
                             else (start, bz, ld))
        reaction = torch.tensor(stats[-1]["reaction"], dtype=torch.float64)
        return reaction, ckpts, stats

    def gradient(self, ckpts, w):
        kw = dict(self.kw)
        return mpm.adjoint(self.ctx, self.cfg, ckpts, w, **kw)


class _Reaction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, E, ys, path):
        reaction, ckpts, stats = path.run(E, ys)
        fctx.path, fctx.ckpts = path, ckpts
        fctx.last_stats = stats
        return reaction

    @staticmethod
    def backward(fctx, g):
        dE, dys, _ = fctx.path.gradient(fctx.ckpts, g.detach().cpu().numpy().astype(np.float64))
        return dE, dys, None


def reaction(path, E, ys):
    """Reaction force (3,) on the body at the end of the last load step; E and
    ys are device float64 tensors of one entry per initial point."""
    return _Reaction.apply(E, ys, path)
