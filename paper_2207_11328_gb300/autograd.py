"""torch.autograd.Function over the differentiable run of the C ABI.

    x_T = rollout(u0, alpha, sim, pos0, delta0, mass, ptype, T=64, K=8)

runs sph_record (T steps from (pos0, u0, delta0) with dt frozen, a
checkpoint every K steps) and returns the final positions (float64, upload
order); backward calls sph_backward with dL/dx_T and returns dL/du0 and
dL/dalpha.  Argument marshalling only: all arithmetic is in the library.

A context holds one recording at a time: forward stores the generation of
its recording (sph_tape_generation) and backward refuses to run when a later
forward on the same context has replaced it (one context per rollout in a
loss that holds several).  Every library call runs on torch's current
stream, so the upload, the recording and the gradients are ordered against
the caller's work on that stream.
"""
from __future__ import annotations

import torch


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, alpha, sim, pos0, delta0, mass, ptype, T, K):
        dev = u0.device
        stream = torch.cuda.current_stream(dev)
        sim.set_alpha(float(alpha))
        sim.upload_device(pos0.to(dev, torch.float64).contiguous(), u0.detach().to(torch.float32).contiguous(),
                          delta0.to(dev, torch.float32).contiguous(), mass.to(dev, torch.float32).contiguous(),
                          ptype.to(dev, torch.uint8).contiguous(), stream=stream)
        ctx.dt = sim.record(int(T), int(K), stream=stream)
        ctx.gen = sim.tape_generation()
        x_T = torch.empty((pos0.shape[0], 3), dtype=torch.float64, device=dev)
        sim.download_device(x_T, None, None, stream=stream)
        ctx.sim = sim
        ctx.alpha_dtype = alpha.dtype if torch.is_tensor(alpha) else torch.float64
        return x_T

    @staticmethod
    def backward(ctx, grad_x):
        if ctx.sim.tape_generation() != ctx.gen:
            raise RuntimeError("Rollout.backward: the context's recording was replaced by a later forward "
                               "(use one Simulation per rollout held in the graph)")
        stream = torch.cuda.current_stream(grad_x.device)
        _, ubar0, _, ab = ctx.sim.backward(xbar_T=grad_x.to(torch.float32).contiguous(), stream=stream)
        galpha = torch.tensor(ab, dtype=ctx.alpha_dtype, device=grad_x.device)
        return ubar0, galpha, None, None, None, None, None, None, None


def rollout(u0, alpha, sim, pos0, delta0, mass, ptype, T=64, K=8):
    return Rollout.apply(u0, alpha, sim, pos0, delta0, mass, ptype, T, K)
