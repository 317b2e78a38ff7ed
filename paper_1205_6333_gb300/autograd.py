"""torch.autograd.Function wrappers around the C ABI.

``mobility_apply(system, x, F)``   v = mu(x) F                     backward: sd_mobility_vjp
``euler_trajectory(system, x0, F_ext, dt, nsteps, ckpt_every)``
                                    x_T after nsteps Euler steps    backward: sd_adjoint
                                    (Sec. 3.1 with forces F_ext + gravity held fixed)

Both run entirely in the library's kernels; the tensors must be CUDA float64
(positions, F_ext) or CUDA float32/float64 (the apply's forces) on the system's
device.  Gradients flow to x / x0 and to the forces.
"""
from __future__ import annotations

import torch


class _MobilityApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, F, system):
        system.set_positions(x.detach().contiguous())
        V = system.mobility_apply(F.detach().contiguous())
        ctx.system = system
        ctx.save_for_backward(x, F)
        return V

    @staticmethod
    def backward(ctx, gV):
        x, F = ctx.saved_tensors
        s = ctx.system
        s.set_positions(x.detach().contiguous())
        gx, gF = s.vjp(F.detach().contiguous(), gV.to(F.dtype).contiguous())
        return gx.to(x.dtype), gF, None


class _EulerTrajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, fext, system, dt, nsteps, ckpt_every):
        system.set_positions(x0.detach().contiguous())
        system.set_forces(fext.detach().contiguous())
        system.step(dt, nsteps)
        xT = torch.empty_like(x0, dtype=torch.float64)
        system.get_positions(xT)
        system.synchronize()
        ctx.system = system
        ctx.args = (float(dt), int(nsteps), int(ckpt_every))
        ctx.save_for_backward(x0, fext)
        return xT

    @staticmethod
    def backward(ctx, gxT):
        x0, fext = ctx.saved_tensors
        s = ctx.system
        dt, nsteps, ckpt = ctx.args
        s.set_positions(x0.detach().contiguous())
        s.set_forces(fext.detach().contiguous())
        gx0, gF = s.adjoint(dt, nsteps, ckpt, gxT.to(torch.float64).contiguous())
        return gx0, gF, None, None, None, None


def mobility_apply(system, x, F):
    """Differentiable v = mu(x) F on `system` (a paper_1205_6333_gb300.System of len(x) particles)."""
    return _MobilityApply.apply(x, F, system)


def euler_trajectory(system, x0, fext, dt, nsteps, ckpt_every=50):
    """Differentiable x(T) after `nsteps` explicit Euler steps of `system` from x0 with
    per-particle forces fext (+ the system's gravity); backward re-runs the forward
    pass from FP64 checkpoints every `ckpt_every` steps."""
    return _EulerTrajectory.apply(x0, fext, system, dt, nsteps, ckpt_every)
