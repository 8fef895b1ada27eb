"""The energy as a differentiable function (torch.autograd), two ways.

``energy(h, eri, e0, ctx, mps)``: E(h, eri, e0) = <psi|H|psi> / <psi|psi> with
H of Eq. (hamil) as a function of the integrals.  E is linear in them, so its
gradient is the pair of density matrices, dE/dh_ij = Re gamma_ij / <psi|psi>,
dE/d(ij|kl) = Re Gamma_ijkl / (2 <psi|psi>) and dE/de0 = 1 (the 1- and 2-RDMs
that the hole densities of Sec. 3.2 are read from).

``state_energy(ctx, mpo, labels, *tensors)``: E as a function of the site
tensors A_i of the MPS (Eq. mps).  Its backward is the library's adjoint of
the effective-Hamiltonian matvec (``tdmps_energy_gradient``):
dE/dconj(A_i) = (H_i A_i - E N_i A_i) / <psi|psi>, the one-site products of
Eq. add_min's local problem taken with psi's own environments, which are
recomputed in the backward pass rather than kept from the forward one.

Every number is computed in the CUDA library (the MPO build, the FP64
chains, the density matrices, the adjoint); this module only moves arrays
between torch and the C ABI and applies the chain rule's upstream factor.
PyTorch's gradient of a real function of a complex tensor is 2 dE/dconj(z).
"""
from __future__ import annotations

import numpy as np
import torch

from . import build_mpo, energy_gradient, integral_gradient, mps_import
from . import energy as _energy


class Energy(torch.autograd.Function):
    """``Energy.apply(h, eri, e0, ctx, mps)`` -> 0-d float64 tensor."""

    @staticmethod
    def forward(fctx, h, eri, e0, ctx, mps):
        hn = h.detach().cpu().numpy().astype(np.float64)
        en = eri.detach().cpu().numpy().astype(np.float64)
        e0v = float(e0.detach().cpu()) if torch.is_tensor(e0) else float(e0)
        L = hn.shape[0]
        mpo = build_mpo(ctx, hn, en, L, mps.info()["n_elec"], e0v)
        e = _energy(ctx, mpo, mps)
        mpo.free()
        fctx.ctx, fctx.mps = ctx, mps
        fctx.e0_is_tensor = torch.is_tensor(e0)
        fctx.dev, fctx.dtype = h.device, h.dtype
        return torch.tensor(e, dtype=torch.float64, device=h.device)

    @staticmethod
    def backward(fctx, g):
        dh, deri = integral_gradient(fctx.ctx, fctx.mps)
        gh = g.to(fctx.dtype) * torch.as_tensor(dh, dtype=fctx.dtype, device=fctx.dev)
        geri = g.to(fctx.dtype) * torch.as_tensor(deri, dtype=fctx.dtype, device=fctx.dev)
        ge0 = g.detach().cpu().to(torch.float64) if fctx.e0_is_tensor else None
        return gh, geri, ge0, None, None


def energy(h, eri, e0, ctx, mps):
    """Differentiable <psi|H(h, eri, e0)|psi> / <psi|psi>."""
    return Energy.apply(h, eri, e0, ctx, mps)


def _vector_order(labels_in, labels_out):
    """Index p with out-vector p[x] = in-vector x: the k-th vector of a
    sector in one list is the k-th vector of that sector in the other."""
    li = np.asarray(labels_in).reshape(-1, 2)
    lo = np.asarray(labels_out).reshape(-1, 2)
    slots: dict = {}
    for y, qy in enumerate(map(tuple, lo.tolist())):
        slots.setdefault(qy, []).append(y)
    seen: dict = {}
    p = np.empty(len(li), dtype=np.int64)
    for x, qx in enumerate(map(tuple, li.tolist())):
        k = seen.get(qx, 0)
        p[x] = slots[qx][k]
        seen[qx] = k + 1
    return p


class StateEnergy(torch.autograd.Function):
    """``StateEnergy.apply(ctx, mpo, labels, stride, *tensors)`` -> 0-d float64
    tensor; ``tensors`` are the dense complex site tensors (D_l, 4, D_r) and
    ``labels`` their bond labels, as for ``mps_import``."""

    @staticmethod
    def forward(fctx, ctx, mpo, labels, stride, *tensors):
        arrs = [t.detach().cpu().numpy().astype(np.complex128) for t in tensors]
        psi = mps_import(ctx, arrs, labels)
        e = _energy(ctx, mpo, psi)
        psi.free()
        fctx.ctx, fctx.mpo, fctx.labels, fctx.stride = ctx, mpo, labels, stride
        fctx.save_for_backward(*tensors)
        return torch.tensor(e, dtype=torch.float64, device=tensors[0].device)

    @staticmethod
    def backward(fctx, g):
        tensors = fctx.saved_tensors
        arrs = [t.detach().cpu().numpy().astype(np.complex128) for t in tensors]
        psi = mps_import(fctx.ctx, arrs, fctx.labels)
        _, G, _ = energy_gradient(fctx.ctx, fctx.mpo, psi, fctx.stride)
        gt, glab = G.export()
        G.free()
        psi.free()
        # the library orders each bond's vectors by sector: back to the caller's order
        perm = [_vector_order(a, b) for a, b in zip(fctx.labels, glab)]
        gt = [x[np.ix_(perm[i], np.arange(4), perm[i + 1])] for i, x in enumerate(gt)]
        scale = 2.0 * g.detach().cpu().to(torch.float64)
        grads = [scale * torch.as_tensor(x, dtype=torch.complex128) for x in gt]
        return (None, None, None, None,
                *[gr.to(device=t.device, dtype=t.dtype) for gr, t in zip(grads, tensors)])


def state_energy(ctx, mpo, labels, tensors, stride=1):
    """Differentiable <psi|H|psi> / <psi|psi> of the MPS with these site tensors."""
    return StateEnergy.apply(ctx, mpo, labels, stride, *tensors)
