"""The field energy after N steps as a differentiable function of the initial particles.

``field_energy_after(x0, P0, cfg, q, m, nsteps, every)`` runs the GPU library forward from the
initial positions x0 and canonical momenta P0 (each (np, 3) float64 CUDA tensors; the initial
vector potential is zero, so v0 = P0 / m) and returns W^N, the field energy after nsteps steps,
as a 0-d tensor.  Its backward pass is the library's hand-written adjoint (pic_step_vjp,
pic_energy_vjp, pic_init_vjp), with checkpoint-and-recompute over time steps: the forward keeps
the state every ``every`` steps on the device; the backward recomputes each interval's states
from its checkpoint, then walks the interval backwards, re-running each step (so that the
context holds level n and the accepted iterate) and applying its adjoint.  Checkpoints keep the
positions as stored (cell units, pic_get_positions / pic_set_positions), so a recomputed step
starts from the forward run's state bit for bit: past the two-stream saturation the run is
chaotic, and a state rounded through physical units would linearise about another trajectory.  Every derivative is
computed by the library's kernels; this module only orders the calls and holds the tensors.
"""

from __future__ import annotations

import torch

from . import sim


def _sim(cfg, x0, P0, q, m):
    return sim.PicSim(cfg, x0, P0 / m, q, m)


class FieldEnergyAfter(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, P0, cfg, q, m, nsteps, every):
        s = _sim(cfg, x0, P0, q, m)
        ckpt = {}
        for n in range(nsteps):
            if n % every == 0:
                ckpt[n] = s.checkpoint()
            info = s.step(1)
            if not info.converged:
                raise sim.PicError(4, "a forward step did not converge")
        W = s.energy().W
        s.close()
        ctx.save_for_backward(x0, P0)
        ctx.cfg, ctx.q, ctx.m, ctx.nsteps, ctx.every, ctx.ckpt = cfg, q, m, nsteps, every, ckpt
        ctx.vjp_iterations = []
        return torch.tensor(W, dtype=torch.float64, device=x0.device)

    @staticmethod
    def backward(ctx, gW):
        x0, P0 = ctx.saved_tensors
        cfg, q, m, nsteps, every = ctx.cfg, ctx.q, ctx.m, ctx.nsteps, ctx.every
        s = _sim(cfg, x0, P0, q, m)
        # lambda^N = dW/d(state N), on the state after N steps (recomputed from the last checkpoint)
        last = max(ctx.ckpt)
        s.restore(ctx.ckpt[last])
        for _ in range(last, nsteps):
            s.step(1)
        lam = s.energy_vjp()
        gs = float(gW)
        for k in lam:
            lam[k] *= gs
        for start in sorted(ctx.ckpt, reverse=True):
            end = min(start + every, nsteps)
            states = {start: ctx.ckpt[start]}
            s.restore(ctx.ckpt[start])
            for n in range(start, end - 1):          # the interval's levels, recomputed once
                s.step(1)
                states[n + 1] = s.checkpoint()
            for n in range(end - 1, start - 1, -1):
                s.restore(states[n])
                s.step(1)                             # level n and v* of step n -> n+1
                lam, info = s.step_vjp(lam)
                ctx.vjp_iterations.append(int(info.iterations))
            del states
        s.close()
        # the initial data: a fresh context holds pic_init's state
        s0 = _sim(cfg, x0, P0, q, m)
        lx, lv = s0.init_vjp(lam)
        s0.close()
        npart = x0.shape[0]
        gx = lx[: 3 * npart].reshape(3, npart).t().contiguous()
        gP = (lv[: 3 * npart] / m).reshape(3, npart).t().contiguous()
        return gx, gP, None, None, None, None, None


def field_energy_after(x0, P0, cfg, q, m, nsteps, every=10):
    """W^N of the run from (x0, P0) (CUDA float64 (np, 3) tensors), differentiable in both."""
    return FieldEnergyAfter.apply(x0, P0, cfg, q, m, nsteps, every)
