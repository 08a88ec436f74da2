"""torch.autograd form of the potential (the differentiation form used for
force-matching training).  Every derivative is computed by the library's kernels
(libnnp.so); the Functions below only route tensors and apply the chain-rule
factors handed in by autograd (a per-system scale and a per-system dot product).

  batch = TrainingBatch(nnp, types, starts, boxes)
  E = NNPEnergy.apply(pos, weights, batch)                      # [B], float64
  F = -torch.autograd.grad(E.sum(), pos, create_graph=True)[0]   # forces, differentiable in weights
  loss(E, F).backward()                                          # weights.grad via the double backward

NNPEnergy.backward gives dL/dpos = -dL/dE_b F_m (the forces) and dL/dweights =
sum_b dL/dE_b dE_b/dweights.  The force node (_ForceTerm) has the hand-written
double backward: dL/dweights = sum_m u_m . d(-dL/dE_b F_m)/dweights, computed from
the descriptor tangents along u with dG/dr recomputed.  Second derivatives with
respect to positions (Hessian products) are not formed: the force node returns
no position gradient.

EnergyForces.apply(pos, weights, batch) -> (E, F) is the same computation as one
node, for training loops that need energies and forces together.
"""
from __future__ import annotations

import numpy as np
import torch


class TrainingBatch:
    """Fixed layout of a batch of systems: types, system offsets and boxes."""

    def __init__(self, nnp, types, starts, boxes):
        self.nnp = nnp
        self.types = types
        self.starts = np.ascontiguousarray(np.asarray(starts, np.int32))
        self.boxes = np.ascontiguousarray(np.asarray(boxes, np.float64).reshape(-1, 3))
        n_per = np.diff(self.starts)
        self.sys_of = torch.repeat_interleave(torch.arange(len(n_per), device=types.device),
                                              torch.as_tensor(n_per, device=types.device))
        self.n_systems = len(n_per)

    def _load(self, weights):
        self.nnp.set_weights(weights.detach().contiguous())

    def evaluate(self, pos, weights):
        self._load(weights)
        return self.nnp.compute_batch(pos.detach().contiguous(), self.types, self.starts, self.boxes)

    def grad(self, pos, weights, dLdE=None, dLdF=None):
        self._load(weights)
        return self.nnp.param_grad(pos.detach().contiguous(), self.types, self.starts, self.boxes,
                                   None if dLdE is None else dLdE.detach().to(torch.float64).contiguous(),
                                   None if dLdF is None else dLdF.detach().to(torch.float32).contiguous())

    def per_atom(self, v):
        """Per-system values broadcast to atoms (autograd chain-rule factor)."""
        return v[self.sys_of]

    def per_system_sum(self, v):
        out = torch.zeros(self.n_systems, dtype=v.dtype, device=v.device)
        return out.index_add_(0, self.sys_of, v)


class NNPEnergy(torch.autograd.Function):
    """E_b(pos, weights) for every system of the batch."""

    @staticmethod
    def forward(ctx, pos, weights, batch):
        out = batch.evaluate(pos, weights)
        ctx.save_for_backward(pos, weights, out["F"])
        ctx.batch = batch
        return out["energy"]

    @staticmethod
    def backward(ctx, gE):
        pos, weights, F = ctx.saved_tensors
        batch = ctx.batch
        grad_pos = grad_w = None
        if ctx.needs_input_grad[0]:
            grad_pos = _ForceTerm.apply(pos, weights, gE, F, batch)
        if ctx.needs_input_grad[1]:
            grad_w = batch.grad(pos, weights, dLdE=gE)
        return grad_pos, grad_w, None


class _ForceTerm(torch.autograd.Function):
    """dE/dpos scaled by the upstream gradient: -gE_b F_m (a function of the weights)."""

    @staticmethod
    def forward(ctx, pos, weights, gE, F, batch):
        ctx.save_for_backward(pos, weights, gE, F)
        ctx.batch = batch
        return -batch.per_atom(gE).to(F.dtype)[:, None] * F

    @staticmethod
    def backward(ctx, u):
        pos, weights, gE, F = ctx.saved_tensors
        batch = ctx.batch
        grad_w = grad_gE = None
        if ctx.needs_input_grad[1]:
            v = -batch.per_atom(gE).to(u.dtype)[:, None] * u
            grad_w = batch.grad(pos, weights, dLdF=v)
        if ctx.needs_input_grad[2]:
            grad_gE = -batch.per_system_sum((u * F).sum(1).to(torch.float64)).to(gE.dtype)
        # position second derivatives are not formed
        return None, grad_w, grad_gE, None, None


class EnergyForces(torch.autograd.Function):
    """(E [B], F [N,3]) in one node; backward gives the weight gradient of both."""

    @staticmethod
    def forward(ctx, pos, weights, batch):
        out = batch.evaluate(pos, weights)
        ctx.save_for_backward(pos, weights, out["F"])
        ctx.batch = batch
        return out["energy"], out["F"]

    @staticmethod
    def backward(ctx, gE, gF):
        pos, weights, F = ctx.saved_tensors
        batch = ctx.batch
        grad_pos = grad_w = None
        if ctx.needs_input_grad[1]:
            grad_w = batch.grad(pos, weights, dLdE=gE, dLdF=gF)
        if ctx.needs_input_grad[0]:
            if gF is not None and bool(gF.abs().max() > 0):
                raise NotImplementedError("position gradients through the forces (Hessian) are not formed")
            grad_pos = -batch.per_atom(gE).to(F.dtype)[:, None] * F if gE is not None else None
        return grad_pos, grad_w, None


def force_matching_loss(E, F, E_ref, F_ref, n_atoms, w_force=10.0):
    """(1/B) sum_b ((E_b - E_ref_b)/N_b)^2 + w_force/(3 sum N) sum (F - F_ref)^2."""
    B = E.shape[0]
    le = (((E - E_ref) / n_atoms) ** 2).sum() / B
    lf = ((F.double() - F_ref.double()) ** 2).sum() / (3.0 * float(n_atoms.sum()))
    return le + w_force * lf
