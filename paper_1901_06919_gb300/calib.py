"""Calibration of view positions and disparities (Sec. V-B) on the GPU.

The objective of Eq. CalibrationProb is minimised over u and d by gradient
descent; each evaluation re-solves the layers at every listed frequency
inside ``fdl_calib_grad`` (the factors are never stored) and returns the
gradient of Eqs. gradP / gradD from the same kernel.  ``CalibLoss`` exposes it
as a ``torch.autograd.Function`` so that any torch optimiser can drive it.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import torch

from . import fdl


class CalibLoss(torch.autograd.Function):
    """loss(u, d) of Eq. CalibrationProb; backward uses the hand-written gradient kernel."""

    @staticmethod
    def forward(ctx, u, d, spectra, lam, reg, bins, precision):
        loss, gu, gd = fdl.calib_grad(spectra, u.detach().contiguous(), d.detach().contiguous(), lam, reg=reg,
                                      bins=bins, precision=precision)
        ctx.save_for_backward(gu, gd)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        gu, gd = ctx.saved_tensors
        return g * gu, g * gd, None, None, None, None, None


def calib_loss(u, d, spectra, lam, reg="layer2", bins=None, precision="df"):
    return CalibLoss.apply(u, d, spectra, lam, reg, bins, precision)


@dataclass
class CalibResult:
    u: torch.Tensor
    d: torch.Tensor
    losses: list = field(default_factory=list)


def calibrate(spectra: torch.Tensor, u0: torch.Tensor, d0: torch.Tensor, lam: float = 1e-2, steps: int = 200,
              lr: float = 1e-2, subset: int | None = 4096, seed: int = 0, reg: str = "layer2",
              rule: str = "adam", alpha: float = 0.2, eps: float = 1e-12, precision: str = "df") -> CalibResult:
    """Estimate u [K][2] and d [N] from the half spectra of the views.

    ``subset``: number of frequencies drawn (seeded, without replacement) from the stored half
    spectrum at every step (4096 in Sec. V-B); None uses all of them.
    ``rule``: "adam" (torch Adam, betas 0.9/0.999) or "paper", the normalised step of
    Sec. V-B: ``u <- u - alpha grad_u / (eps + |grad_u|^2)``, and the same for d.
    """
    dev = spectra.device
    K, C, H, Wh = spectra.shape
    nbins = H * Wh
    u = u0.detach().clone().to(dev).requires_grad_(True)
    d = d0.detach().clone().to(dev).requires_grad_(True)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    opt = torch.optim.Adam([u, d], lr=lr, betas=(0.9, 0.999)) if rule == "adam" else None
    out = CalibResult(u, d)
    for _ in range(steps):
        bins = None
        if subset is not None and subset < nbins:
            bins = torch.randperm(nbins, generator=gen, device=dev)[:subset].to(torch.int32)
        loss = calib_loss(u, d, spectra, lam, reg, bins, precision)
        if opt is not None:
            opt.zero_grad(set_to_none=True)
            loss.backward()
            opt.step()
        else:
            gu, gd = torch.autograd.grad(loss, [u, d])
            with torch.no_grad():
                u -= alpha * gu / (eps + torch.sum(gu * gu))
                d -= alpha * gd / (eps + torch.sum(gd * gd))
        out.losses.append(float(loss.detach()))
    out.u = u.detach()
    out.d = d.detach()
    return out


class CalibLossShifts(torch.autograd.Function):
    """loss(P) of Eq. CalibrationProb with free shifts P [K][N][2]; backward: dL/dP of Eq. gradP."""

    @staticmethod
    def forward(ctx, P, spectra, lam, reg, bins, precision):
        loss, gP = fdl.calib_grad_shifts(spectra, P.detach().contiguous(), lam, reg=reg, bins=bins,
                                         precision=precision)
        ctx.save_for_backward(gP)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (gP,) = ctx.saved_tensors
        return g * gP, None, None, None, None, None


@dataclass
class ShiftCalibResult:
    P: torch.Tensor
    losses: list = field(default_factory=list)


def calibrate_shifts(spectra: torch.Tensor, P0: torch.Tensor, lam: float = 1e-2, steps: int = 200, lr: float = 1e-2,
                     subset: int | None = 4096, seed: int = 0, reg: str = "layer2",
                     precision: str = "df") -> ShiftCalibResult:
    """The relaxed FDL model: the shifts P [K][N][2] searched directly (no rank-1 constraint
    P = u d^T) by gradient descent with dL/dP, from ``P0`` (normally the rank-1 solution of
    :func:`calibrate`, as the paper initialises it), on seeded frequency subsets, Adam steps."""
    dev = spectra.device
    K, C, H, Wh = spectra.shape
    nbins = H * Wh
    P = P0.detach().clone().to(dev).contiguous().requires_grad_(True)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    opt = torch.optim.Adam([P], lr=lr, betas=(0.9, 0.999))
    out = ShiftCalibResult(P)
    for _ in range(steps):
        bins = None
        if subset is not None and subset < nbins:
            bins = torch.randperm(nbins, generator=gen, device=dev)[:subset].to(torch.int32)
        loss = CalibLossShifts.apply(P, spectra, lam, reg, bins, precision)
        opt.zero_grad(set_to_none=True)
        loss.backward()
        opt.step()
        out.losses.append(float(loss.detach()))
    out.P = P.detach()
    return out
