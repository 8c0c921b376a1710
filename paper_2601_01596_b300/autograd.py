"""Differentiable correction: e_K = F(e0) for K forced iterations of Alg. 1.

``FFCzCorrect.apply(e0, eps_s, eps_f, K, ckpt_every)`` runs K iterations
(min_iters = max_iters = K, no certification) in the CUDA library, writing
float32 checkpoints of e every ``ckpt_every`` iterations
(``ffcz_correct_ckpt``); its backward calls ``ffcz_correct_backward_ckpt``,
the vector-Jacobian product built from the clips' active-set masks,
regenerated by replaying each segment from its checkpoint.  One step e <- P_s(IDFT(P_f(DFT(e)))) has the
Jacobian M_s IDFT M_f DFT, and IDFT M_f DFT is symmetric in the real frequency
basis of Sec. IV-A, so the transposed step is g <- IDFT(M_f DFT(M_s g)).
"""
from __future__ import annotations

import torch

from . import Plan

_plans: dict = {}


def _plan(shape, K, m, keep=0):
    key = (tuple(shape), int(K), int(m), int(keep), torch.cuda.current_device())
    p = _plans.get(key)
    if p is None:
        p = Plan([tuple(shape)], min_iters=K, max_iters=K, certify=0, K=K, ckpt_every=m, keep_masks=int(keep))
        _plans[key] = p
    return p


class FFCzCorrect(torch.autograd.Function):
    @staticmethod
    def forward(ctx, e0, eps_s: float, eps_f: float, K: int = 50, ckpt_every: int = 10, keep_masks: int = 0):
        if e0.dtype != torch.float32 or not e0.is_cuda:
            raise TypeError("e0 must be a float32 CUDA tensor")
        e0c = e0.detach().contiguous()
        plan = _plan(e0c.shape, K, ckpt_every, keep_masks)
        e = e0c.clone()
        ckpt = torch.empty(plan.ckpt_floats(), dtype=torch.float32, device=e0c.device)
        plan.correct_ckpt(e.reshape(-1), [eps_s], [eps_f], ckpt)
        ctx.save_for_backward(e0c, ckpt)
        ctx.cfg = (float(eps_s), float(eps_f), int(K), int(ckpt_every), int(keep_masks))
        return e

    @staticmethod
    def backward(ctx, grad_out):
        e0, ckpt = ctx.saved_tensors
        eps_s, eps_f, K, m, keep = ctx.cfg
        plan = _plan(e0.shape, K, m, keep)
        g = grad_out.detach().to(torch.float32).contiguous()
        gin = torch.empty_like(e0)
        plan.backward(e0.reshape(-1), g.reshape(-1), gin.reshape(-1), [eps_s], [eps_f], ckpt=ckpt)
        return gin, None, None, None, None, None


def correct_differentiable(e0, eps_s, eps_f, K=50, ckpt_every=10, keep_masks=0):
    """keep_masks = 1: the forward keeps every step's clip masks in the plan
    and the backward runs the adjoint steps without replaying the segments
    (the masks must belong to this forward: one backward per forward)."""
    return FFCzCorrect.apply(e0, eps_s, eps_f, K, ckpt_every, keep_masks)


_bplans: dict = {}


def _bplan(shapes, K, m):
    key = (tuple(tuple(s) for s in shapes), int(K), int(m), torch.cuda.current_device())
    p = _bplans.get(key)
    if p is None:
        p = Plan([tuple(s) for s in shapes], min_iters=K, max_iters=K, certify=0, K=K, ckpt_every=m)
        _bplans[key] = p
    return p


class FFCzCorrectBatch(torch.autograd.Function):
    """The same for a batch of items of any shapes (2D or 3D), packed back to
    back in one float32 CUDA tensor; eps_s / eps_f one per item."""

    @staticmethod
    def forward(ctx, e0, shapes, eps_s, eps_f, K: int = 50, ckpt_every: int = 10):
        if e0.dtype != torch.float32 or not e0.is_cuda:
            raise TypeError("e0 must be a float32 CUDA tensor")
        e0c = e0.detach().contiguous()
        plan = _bplan(shapes, K, ckpt_every)
        e = e0c.clone()
        ckpt = torch.empty(plan.ckpt_floats(), dtype=torch.float32, device=e0c.device)
        plan.correct_ckpt(e.reshape(-1), list(eps_s), list(eps_f), ckpt)
        ctx.save_for_backward(e0c, ckpt)
        ctx.cfg = (tuple(tuple(s) for s in shapes), tuple(eps_s), tuple(eps_f), int(K), int(ckpt_every))
        return e

    @staticmethod
    def backward(ctx, grad_out):
        e0, ckpt = ctx.saved_tensors
        shapes, eps_s, eps_f, K, m = ctx.cfg
        plan = _bplan(shapes, K, m)
        g = grad_out.detach().to(torch.float32).contiguous()
        gin = torch.empty_like(e0)
        plan.backward(e0.reshape(-1), g.reshape(-1), gin.reshape(-1), list(eps_s), list(eps_f), ckpt=ckpt)
        return gin, None, None, None, None, None


def correct_differentiable_batch(e0, shapes, eps_s, eps_f, K=50, ckpt_every=10):
    return FFCzCorrectBatch.apply(e0, shapes, eps_s, eps_f, K, ckpt_every)


_shell_cache: dict = {}


def _shells(n, device, k_max):
    """Shell index round(|k|) of every half-spectrum bin, the bin weights (2
    for bins standing for k and -k, 1 on the self-conjugate planes) and the
    mask of bins with shell <= k_max, cached per shape and device."""
    key = (tuple(n), str(device), int(k_max))
    hit = _shell_cache.get(key)
    if hit is None:
        import torch
        ks = [torch.fft.fftfreq(s, d=1.0 / s, device=device, dtype=torch.float64) for s in n[:-1]]
        ks.append(torch.arange(n[-1] // 2 + 1, device=device, dtype=torch.float64))
        grids = torch.meshgrid(*ks, indexing="ij")
        kr = torch.sqrt(sum(g * g for g in grids)).round().long()
        w = torch.full(kr.shape, 2.0, dtype=torch.float64, device=device)
        w[..., 0] = 1.0
        if n[-1] % 2 == 0:
            w[..., -1] = 1.0
        mask = kr <= k_max
        hit = (kr[mask], w[mask], mask)
        _shell_cache[key] = hit
    return hit


def power_spectrum_loss(x, e, k_max=None):
    """Squared log power-spectrum mismatch between x + e and x (float64 sums).

    Shell-summed power spectrum of Sec. III on the fluctuation x - mean
    (A13), integer shells round(|k|) in 1..N/2, half-spectrum bins weighted 2
    except the self-conjugate planes.  Test and benchmark use only (torch.fft).
    """
    n = tuple(x.shape)
    km = k_max or min(n) // 2
    kr, w, mask = _shells(n, x.device, km)

    def spectrum(f):
        f = f.to(torch.float64)
        F = torch.fft.rfftn(f - f.mean())
        p = F.real ** 2 + F.imag ** 2
        shells = torch.zeros(km + 1, dtype=torch.float64, device=f.device)
        shells.index_add_(0, kr, w * p[mask])
        return shells[1:]
    return torch.sum((torch.log(spectrum(x + e)) - torch.log(spectrum(x))) ** 2)
