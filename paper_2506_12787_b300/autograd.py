"""Differentiable spectrum synthesis: a torch.autograd.Function over the C ABI.

forward  (Sec. 4.2 Eq. 12-15, Sec. 4.1 Eq. 8-9): residuals of the deformation
         MLP (wrf_deform), projection (wrf_project), tile binning (wrf_bin)
         and the order-free rasteriser (wrf_render).
backward (Sec. 4.4: all parameters are fitted by back-propagation):
         wrf_render_backward recomputes every per-pixel weight from the
         records and tile lists (nothing per pixel is stored by the forward),
         wrf_project_backward maps record gradients to the residual and
         reference-frame gradients, wrf_deform_backward back-propagates
         through the MLP and (unless stop_grad_mean) through gamma(mean).

PyTorch provides memory and the stream only; every step runs in the
library's CUDA kernels.
"""
from __future__ import annotations

import dataclasses

import torch

from . import api


@dataclasses.dataclass
class SpectrumConfig:
    grid: object                 # api.make_grid(...)
    L_mean: int = 6
    L_tx: int = 10
    room_min: tuple = (0.0, 0.0, 0.0)
    room_size: tuple = (5.0, 5.0, 3.0)
    stop_grad_mean: bool = False  # the paper's fine stage freezes position gradients
    renderer: object = None       # reusable api.Renderer (created on first use)
    saved_activation_bytes: int = 16 << 30  # keep the MLP's activations up to this size
    # the forward MLP: api.WRF_FP32 (CUDA cores) or api.WRF_BF16X3 (tensor
    # cores, three BF16 products per FP32 product: FP32-level results)
    mlp_precision: int = api.WRF_FP32
    # the forward does not wait for the key count (no host sync): the caller
    # calls renderer.key_overflow() before using the step's results and
    # recomputes them if it returns True (train.Trainer does)
    defer_key_check: bool = False


class SpectrumFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, cfg, tx, mean, log_scale, rot, opacity_logit, amp, *params):
        dev = tx.device
        scene = api.DeviceScene(mean.detach().contiguous(), log_scale.detach().contiguous(),
                                rot.detach().contiguous(), opacity_logit.detach().contiguous(),
                                amp.detach().contiguous())
        mlp = None  # no MLP parameters: the reference frame G^0 for every query
        if params:
            W = [p.detach().contiguous() for p in params[0::2]]
            b = [p.detach().contiguous() for p in params[1::2]]
            mlp = api.DeviceMLP(W, b, cfg.L_mean, cfg.L_tx, tuple(cfg.room_min),
                                tuple(cfg.room_size), cfg.mlp_precision)
        if cfg.renderer is None:
            cfg.renderer = api.Renderer(cfg.grid, dev, fused=False)
        r = cfg.renderer
        txc = tx.detach().contiguous()
        # the forward keeps its hidden activations for the backward (no
        # recompute there) when they fit in the budget
        acts = None
        if mlp is not None:
            nbytes = (len(W) - 1) * int(txc.shape[0]) * scene.n * 128 * 4
            if nbytes <= cfg.saved_activation_bytes:
                acts = torch.empty((len(W) - 1, int(txc.shape[0]) * scene.n, 128),
                                   dtype=torch.float32, device=dev)
        out = r.forward(scene, mlp, txc, acts=acts, deferred=cfg.defer_key_check).clone()
        last = r.last
        ctx.cfg, ctx.scene, ctx.mlp, ctx.tx = cfg, scene, mlp, txc
        ctx.saved = dict(rec=last["rec"].clone(), gids=last["gids"].clone(),
                         offs=last["offs"].clone(), n_keys=last["n_keys"].clone(),
                         resid=last["resid"].clone() if last["resid"] is not None else None,
                         cap=r.cap, acts=acts)
        ctx.n_params = len(params)
        return out

    @staticmethod
    def backward(ctx, dA):
        cfg, scene, mlp, sv = ctx.cfg, ctx.scene, ctx.mlp, ctx.saved
        Q, N = int(ctx.tx.shape[0]), scene.n
        d_rec = api.wrf_render_backward(sv["rec"], sv["gids"], sv["offs"], sv["n_keys"],
                                        sv["cap"], N, Q, cfg.grid, dA.contiguous())
        g = api.wrf_project_backward(scene, sv["resid"], Q, d_rec)
        if mlp is None:
            return (None, None, g["d_mean"], g["d_log_scale"], g["d_rot"], g["d_opacity"],
                    g["d_amp"])
        dW, db, d_mean = api.wrf_deform_backward(scene, mlp, cfg.grid, ctx.tx, g["d_resid"],
                                                 d_mean=g["d_mean"],
                                                 stop_grad_mean=cfg.stop_grad_mean,
                                                 acts=sv["acts"])
        grads = [None, None, d_mean, g["d_log_scale"], g["d_rot"], g["d_opacity"], g["d_amp"]]
        for w, b in zip(dW, db):
            grads += [w, b]
        return tuple(grads)


def render_spectra(cfg: SpectrumConfig, tx, mean, log_scale, rot, opacity_logit, amp, params):
    """Spectra [Q,H,W] for TX positions tx [Q,3], differentiable in the
    Gaussians and the MLP parameters (params = [W0, b0, W1, b1, ...]; an empty
    list renders the reference frame without deformation)."""
    return SpectrumFunction.apply(cfg, tx, mean, log_scale, rot, opacity_logit, amp, *params)


class SpectrumLossFunction(torch.autograd.Function):
    """Eq. 16: lambda_1 mean|pred - target| + (1 - lambda_1) (1 - mean SSIM),
    value and gradient from wrf_loss in one call."""

    @staticmethod
    def forward(ctx, pred, target, lambda1):
        out, d = api.wrf_loss(pred.detach().contiguous(), target.detach().contiguous(), lambda1,
                              want_grad=pred.requires_grad)
        ctx.save_for_backward(d if d is not None else out)
        ctx.has_grad = d is not None
        return out[0]

    @staticmethod
    def backward(ctx, gL):
        (d,) = ctx.saved_tensors
        return (gL * d if ctx.has_grad else None), None, None


def spectrum_loss(pred, target, lambda1: float = 0.7):
    """Eq. 16 loss of a batch of spectra [Q,H,W] (differentiable in pred)."""
    return SpectrumLossFunction.apply(pred, target, lambda1)
