"""torch.autograd bindings: lhaf(B_n) with gradients from the library's adjoint kernel, and the
GBS log-probability of a pure Gaussian state (App. A) built from it.

lhaf is holomorphic in the entries of B and gamma, so for a real loss L the gradient torch expects
is grad_out * conj(d lhaf / d z). The library reads B from its upper triangle (i <= j), so the
gradient with respect to the B tensor lives on that triangle.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import Context


class LoopHafnian(torch.autograd.Function):
    @staticmethod
    def forward(fctx, B, gamma, reps, lib_ctx):
        Bn = B.detach().cpu().numpy()
        gn = None if gamma is None else gamma.detach().cpu().numpy()
        if fctx.needs_input_grad[0] or fctx.needs_input_grad[1]:
            val, dB, dg = lib_ctx.lhaf_grad(Bn, gn, reps)
            fctx.save_for_backward(torch.from_numpy(np.triu(dB)).to(B.device),
                                   torch.from_numpy(dg if dg is not None else np.zeros(Bn.shape[0], np.complex128))
                                   .to(B.device))
        else:
            val = lib_ctx.lhaf(Bn, gn, reps)
        fctx.has_gamma = gamma is not None
        return torch.tensor(val, dtype=torch.complex128, device=B.device)

    @staticmethod
    def backward(fctx, grad_out):
        dB, dg = fctx.saved_tensors
        gB = grad_out * dB.conj()
        gg = grad_out * dg.conj() if fctx.has_gamma else None
        return gB, gg, None, None


class LoopHafnianBatch(torch.autograd.Function):
    """lhaf(B_{n_i}) for a batch of patterns with one shared B and per-item loop weights, the
    gradients from one lhaf_grad_batched call."""

    @staticmethod
    def forward(fctx, B, gammas, reps, lib_ctx):
        Bn = B.detach().cpu().numpy()
        gn = gammas.detach().cpu().numpy()
        vals, dB, dg, st = lib_ctx.lhaf_grad_batched(Bn, gn, reps)
        if np.any(st != 0):
            raise RuntimeError(f"lhaf_grad_batched item statuses {st[st != 0][:8]}")
        fctx.save_for_backward(torch.from_numpy(np.triu(dB)).to(B.device), torch.from_numpy(dg).to(B.device))
        return torch.from_numpy(vals).to(B.device)

    @staticmethod
    def backward(fctx, grad_out):
        dB, dg = fctx.saved_tensors
        gB = torch.einsum("b,bij->ij", grad_out, dB.conj())
        gg = grad_out[:, None] * dg.conj()
        return gB, gg, None, None


def lhaf_batch_torch(B: torch.Tensor, gammas: torch.Tensor, reps, lib_ctx: Context) -> torch.Tensor:
    """lhaf(B_{n_i}) for reps (batch x M) as a differentiable complex128 vector (B shared, gammas
    batch x M)."""
    return LoopHafnianBatch.apply(B, gammas, np.asarray(reps, dtype=np.int32), lib_ctx)


def lhaf_torch(B: torch.Tensor, gamma, reps, lib_ctx: Context) -> torch.Tensor:
    """lhaf(B_n) as a differentiable complex128 scalar (B, gamma: complex128 tensors)."""
    return LoopHafnian.apply(B, gamma, np.asarray(reps, dtype=np.int32), lib_ctx)


def pure_state_kernel_torch(U: torch.Tensor, r: torch.Tensor, alpha: torch.Tensor):
    """(B, gamma_B, log P0) of the pure state (squeezing r, interferometer U, displacement alpha),
    App. A: sigma = S S^dag / 2, sigma_Q = sigma + I/2, A = X (I - sigma_Q^-1), gamma =
    alpha_full^dag sigma_Q^-1, P0 = exp(-alpha_full^dag sigma_Q^-1 alpha_full / 2) / sqrt(det sigma_Q)."""
    M = r.shape[0]
    ch = torch.diag(torch.cosh(r)).to(torch.complex128)
    sh = torch.diag(torch.sinh(r)).to(torch.complex128)
    Z = torch.zeros((M, M), dtype=torch.complex128, device=U.device)
    Ssq = torch.cat([torch.cat([ch, -sh], 1), torch.cat([-sh, ch], 1)], 0)
    Su = torch.cat([torch.cat([U, Z], 1), torch.cat([Z, U.conj()], 1)], 0)
    S = Su @ Ssq
    I2 = torch.eye(2 * M, dtype=torch.complex128, device=U.device)
    sQ = 0.5 * S @ S.conj().T + 0.5 * I2
    sQi = torch.linalg.inv(sQ)
    B = -sQi[M:, :M]
    af = torch.cat([alpha, alpha.conj()])
    gam = af.conj() @ sQi
    quad = (gam @ af).real
    logdet = torch.linalg.slogdet(sQ)[1]
    return B, gam[:M], -0.5 * quad - 0.5 * logdet


def gbs_log_prob_torch(U, r, alpha, n, lib_ctx: Context) -> torch.Tensor:
    """log P(n) = log P0 + log |lhaf(B_n)|^2 - sum log n_i! (Eq. mixed_prob with Eq. Adef),
    differentiable in U, r and alpha."""
    B, g, logP0 = pure_state_kernel_torch(U, r, alpha)
    lh = lhaf_torch(B, g, n, lib_ctx)
    return logP0 + torch.log((lh * lh.conj()).real) - sum(math.lgamma(int(k) + 1) for k in n)


def gbs_log_prob_batch_torch(U, r, alpha, ns, lib_ctx: Context) -> torch.Tensor:
    """log P(n_i) for a batch of outcomes ns (batch x M) of one pure state, differentiable in U, r
    and alpha; the loop hafnians and their gradients come from one lhaf_grad_batched call."""
    B, g, logP0 = pure_state_kernel_torch(U, r, alpha)
    ns = np.asarray(ns, dtype=np.int32)
    lh = lhaf_batch_torch(B, g.unsqueeze(0).expand(ns.shape[0], -1).contiguous(), ns, lib_ctx)
    fact = torch.tensor([sum(math.lgamma(int(k) + 1) for k in row) for row in ns], dtype=torch.float64,
                        device=lh.device)
    return logP0 + torch.log((lh * lh.conj()).real) - fact
