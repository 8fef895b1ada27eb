"""Energy as a differentiable function of the integrals (torch.autograd).

E(h, eri, e0) = <psi|H|psi> / <psi|psi> with H of Eq. (hamil) is linear in
the integrals, so its gradient is the pair of density matrices:
dE/dh_ij = Re gamma_ij / <psi|psi> and dE/d(ij|kl) = Re Gamma_ijkl / (2
<psi|psi>), dE/de0 = 1 (gamma, Gamma as in ``one_rdm`` / ``two_rdm``; the
real part because the integrals are real and E is).  Forward and backward
run in the CUDA library: the MPO build and sandwich forward, the two
density matrices backward.
"""
from __future__ import annotations

import numpy as np
import torch

from . import build_mpo, expectation, one_rdm, overlap, two_rdm


class Energy(torch.autograd.Function):
    """``Energy.apply(h, eri, e0, ctx, mps)`` -> 0-d float64 tensor."""

    @staticmethod
    def forward(fctx, h, eri, e0, ctx, mps):
        hn = h.detach().cpu().numpy().astype(np.float64)
        en = eri.detach().cpu().numpy().astype(np.float64)
        e0v = float(e0.detach().cpu()) if torch.is_tensor(e0) else float(e0)
        L = hn.shape[0]
        info = mps.info()
        mpo = build_mpo(ctx, hn, en, L, info["n_elec"], e0v)
        nrm = overlap(ctx, mps, mps).real
        e = expectation(ctx, mpo, mps, mps).real / nrm
        mpo.free()
        fctx.ctx, fctx.mps, fctx.nrm = ctx, mps, nrm
        fctx.e0_is_tensor = torch.is_tensor(e0)
        fctx.dev, fctx.dtype = h.device, h.dtype
        return torch.tensor(e, dtype=torch.float64, device=h.device)

    @staticmethod
    def backward(fctx, g):
        gv = float(g.detach().cpu())
        gamma = one_rdm(fctx.ctx, fctx.mps).real / fctx.nrm
        Gam = two_rdm(fctx.ctx, fctx.mps).real / fctx.nrm
        gh = torch.as_tensor(gv * gamma, dtype=fctx.dtype, device=fctx.dev)
        geri = torch.as_tensor(0.5 * gv * Gam, dtype=fctx.dtype, device=fctx.dev)
        ge0 = torch.tensor(gv, dtype=torch.float64) if fctx.e0_is_tensor else None
        return gh, geri, ge0, None, None


def energy(h, eri, e0, ctx, mps):
    """Differentiable <psi|H(h, eri, e0)|psi> / <psi|psi>."""
    return Energy.apply(h, eri, e0, ctx, mps)
