"""torch.autograd bindings of the SNAP library (argument marshalling only).

SnapEnergy.apply(pos, snap, box) returns the per-atom energies E_i; its
backward is the library's adjoint force path: the dE_i/dr_ik of the forward
evaluation gathered with the upstream per-atom weights
(snap_force_weighted), so d(sum_i w_i E_i)/dr is exact for any w.

force_matching_grad() returns the loss sum_k |F_k - F_ref,k|^2 and its
gradient with respect to beta from the bispectrum derivative along
g = 2 (F - F_ref) (snap_bispectrum_deriv): dL/dbeta_l = -sum_i dB_g[i, l];
force_matching_grad_batch() does the same for a batch of configurations with
one batched evaluation and one batched derivative (snap_compute_batch,
snap_bispectrum_deriv_batch).
"""
from __future__ import annotations

import torch

from . import snap as _snap


class SnapEnergy(torch.autograd.Function):
    """Per-atom SNAP energies with the adjoint force kernel as backward."""

    @staticmethod
    def forward(ctx, pos, model: "_snap.Snap", box):
        E, _, _ = model.compute(pos.detach().contiguous(), box)
        ctx.model = model
        ctx.box = box
        ctx.generation = model.generation()
        ctx.save_for_backward(pos)
        return E.clone()

    @staticmethod
    def backward(ctx, grad_e):
        (pos,) = ctx.saved_tensors
        model = ctx.model
        if model.generation() != ctx.generation:
            # the context evaluated something else since: redo this forward
            model.compute(pos.detach().contiguous(), ctx.box)
        grad = model.force_weighted(grad_e.detach().to(torch.float64).contiguous())
        return grad, None, None


def energy(model: "_snap.Snap", pos, box):
    """Differentiable per-atom energies (see SnapEnergy)."""
    return SnapEnergy.apply(pos, model, box)


def force_matching_grad(model: "_snap.Snap", pos, box, f_ref):
    """(L, dL/dbeta) for L = sum_k |F_k - F_ref,k|^2 on one configuration.

    F is linear in beta, F_k = -sum_i sum_l beta_l dB_l(i)/dr_k, so with
    g = 2 (F - F_ref) held fixed, dL/dbeta_l = -sum_i dB_g[i, l] and
    dL/dbeta_0 = 0.  Both are computed on the GPU; the result is a float64
    tensor of length 1 + N_B on the device.
    """
    _, F, _ = model.compute(pos, box)
    r = F - f_ref
    loss = (r * r).sum()
    g = (2.0 * r).contiguous()
    dB = model.bispectrum_deriv(pos, box, g)
    grad = torch.zeros(dB.shape[1] + 1, dtype=torch.float64, device=pos.device)
    grad[1:] = -dB.sum(dim=0)
    return loss, grad


def force_matching_grad_batch(model: "_snap.Snap", pos, natoms, boxes, f_ref):
    """(L, dL/dbeta) for L = sum over all configurations and atoms of
    |F_k - F_ref,k|^2, the configurations concatenated as in
    Snap.compute_batch: one batched force evaluation and one batched
    bispectrum derivative along g = 2 (F - F_ref)."""
    _, F, _ = model.compute_batch(pos, natoms, boxes)
    r = F - f_ref
    loss = (r * r).sum()
    dB = model.bispectrum_deriv_batch(pos, natoms, boxes, (2.0 * r).contiguous())
    grad = torch.zeros(dB.shape[1] + 1, dtype=torch.float64, device=pos.device)
    grad[1:] = -dB.sum(dim=0)
    return loss, grad
