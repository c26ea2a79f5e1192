"""Training protocol of Sec. 4.4 on the library's kernels.

* Coarse stage: only the Gaussians (mean, log-scale, rotation, opacity,
  amplitude) are fitted, to all training spectra, with the deformation MLP
  frozen and not applied: every query renders the reference frame G^0.
* Fine stage: the MLP is activated and fitted together with the Gaussians,
  except their positions, whose gradients are frozen.  The TX position fed to
  the MLP's encoding carries the anneal-smoothing noise of Eq. 17-18,
    n_i = gamma N3(0,1) (2 / cbrt(N_s)) (1 - i / tau)  for i < tau, else 0,
  on the position normalised to the room's unit cube (i counts fine-stage
  iterations; N_s is the number of training positions).
* Loss: Eq. 16 (wrf_loss: L1 + SSIM), optimiser: Adam (wrf_adam) with the
  learning rates of Table I (1e-2 for the Gaussians, 8e-3 for the MLP).

Readings where the paper is silent: one Adam state per parameter that runs
on across the stages (its step count is the number of updates that parameter
has had); PyTorch's Adam defaults beta = (0.9, 0.999), eps = 1e-8; the
minibatch of TX positions drawn uniformly with replacement every iteration.
Random draws come from a torch.Generator the caller seeds, or are passed in.

A step does not stall the host: host-side draws reach the device through
pinned staging buffers, and the forward's key count is checked only before
the Adam update (SpectrumConfig.defer_key_check); a step whose keys did not
fit is recomputed with the raised capacity before any parameter changes.
On CUDA the forward and the backward replay captured graphs (Trainer.step).
"""
from __future__ import annotations

import dataclasses

import torch

from . import api
from .autograd import SpectrumConfig, render_spectra, spectrum_loss

GAUSS_FIELDS = ("mean", "log_scale", "rot", "opacity_logit", "amp")


@dataclasses.dataclass
class TrainConfig:
    lambda1: float = 0.7       # Table I: L1 weight of Eq. 16
    lr_gauss: float = 1e-2     # Table I
    lr_mlp: float = 8e-3       # Table I
    gamma: float = 1.0         # Table I: anneal smoothing weight
    tau: int = 10000           # Table I: anneal smoothing threshold
    coarse_iters: int = 1000
    batch: int = 64
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8


class Trainer:
    """Coarse-to-fine fitting of a scene and its deformation MLP to measured
    spectra (Sec. 4.4).

    gauss: dict of device FP32 tensors mean [N,2], log_scale [N,2], rot [N],
    opacity_logit [N], amp [N] (updated in place); mlp_params: [W0, b0, W1, b1,
    ...] device FP32 tensors (updated in place); tx_train [N_s,3] metres and
    targets [N_s,H,W] on the device."""

    def __init__(self, gauss: dict, mlp_params: list, spec: SpectrumConfig, tx_train, targets,
                 cfg: TrainConfig = TrainConfig(), generator: torch.Generator | None = None,
                 graph: bool = True):
        self.g = {k: gauss[k] for k in GAUSS_FIELDS}
        self.mlp = list(mlp_params)
        self.spec, self.cfg = spec, cfg
        self.tx_train, self.targets = tx_train, targets
        self.gen = generator
        self.state = {id(p): [torch.zeros_like(p), torch.zeros_like(p), 0]
                      for p in list(self.g.values()) + self.mlp}
        self.it = 0
        spec.defer_key_check = True
        self._ring = [None] * 4  # pinned staging buffers: (buffer, copy-done event)
        self._ring_i = 0
        self.use_graph = graph and tx_train.device.type == "cuda"
        self._graphs = {}  # stage (coarse?) -> captured forward + loss + backward
        self.graph_steps = 0  # steps that replayed a graph

    def _upload(self, t):
        """t on the training device; a host tensor goes through a pinned
        staging buffer (asynchronous copy; a buffer is reused once its previous
        copy has finished), so the host does not wait for the device."""
        dev = self.tx_train.device
        if t.device == dev or dev.type != "cuda":
            return t.to(dev)
        t = t.contiguous()
        nbytes = t.numel() * t.element_size()
        slot = self._ring_i % len(self._ring)
        self._ring_i += 1
        buf, ev = self._ring[slot] or (None, None)
        if ev is not None:
            ev.synchronize()
        if buf is None or buf.numel() < nbytes:
            buf = torch.empty(max(nbytes, 4096), dtype=torch.uint8, pin_memory=True)
        host = buf[:nbytes].view(t.dtype).view(t.shape)
        host.copy_(t)
        out = host.to(dev, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record()
        self._ring[slot] = (buf, ev)
        return out

    @property
    def coarse(self) -> bool:
        return self.it < self.cfg.coarse_iters

    def noisy_tx(self, idx, normals=None):
        """The MLP's TX input at this fine-stage iteration: the training
        positions idx plus the Eq. 18 noise (wrf_anneal_tx), in metres."""
        if normals is None:
            normals = torch.randn(int(idx.numel()), 3, generator=self.gen)
        normals = self._upload(normals.to(torch.float32))
        i = self.it - self.cfg.coarse_iters
        return api.wrf_anneal_tx(self.tx_train, normals, i, self.cfg.gamma, self.cfg.tau,
                                 self.spec.room_size, idx=idx)

    def noise(self, Qb: int, normals=None):
        """Metres added to the MLP's TX input at this fine-stage iteration
        (the noisy positions of rows 0 .. Qb-1 minus the positions)."""
        idx = torch.arange(Qb, device=self.tx_train.device)
        return self.noisy_tx(idx, normals) - self.tx_train[:Qb]

    def step(self, idx=None, normals=None):
        """One iteration; idx [B] (training positions) and normals [B,3] may be
        given, else they are drawn.  Returns the loss (0-dim tensor).

        With graph=True (and a batch of cfg.batch positions on a CUDA
        device) the forward with the loss, and the backward, replay two CUDA
        graphs captured once per stage; the host waits for the forward only
        (its key count) before launching Adam behind the backward.  The
        anneal noise and the Adam update, whose scalar arguments change every
        step, run as ordinary launches."""
        c = self.cfg
        if idx is None:
            idx = torch.randint(self.tx_train.shape[0], (c.batch,), generator=self.gen)
        if not self.coarse and normals is None:
            normals = torch.randn(int(idx.numel()), 3, generator=self.gen)
        if self.use_graph and int(idx.numel()) == c.batch:
            out = self._step_graph(idx, normals)
            if out is not None:
                return out
        return self._step_eager(idx, normals)

    def _step_eager(self, idx, normals):
        c = self.cfg
        idx = self._upload(idx)
        tgt = self.targets[idx]
        coarse = self.coarse
        if not coarse and normals is None:
            normals = torch.randn(int(idx.numel()), 3, generator=self.gen)
        tx = self.noisy_tx(idx, normals) if not coarse else self.tx_train[idx]
        self.spec.stop_grad_mean = not coarse
        leaves = {k: v.detach().requires_grad_(coarse or k != "mean") for k, v in self.g.items()}
        params = [] if coarse else [p.detach().requires_grad_() for p in self.mlp]
        out = render_spectra(self.spec, tx.contiguous(), leaves["mean"], leaves["log_scale"],
                             leaves["rot"], leaves["opacity_logit"], leaves["amp"], params)
        loss = spectrum_loss(out, tgt, c.lambda1)
        loss.backward()
        if self.spec.renderer.key_overflow():
            # the keys did not fit: recompute with the raised capacity (same
            # draws) before any parameter changes
            return self._step_eager(idx, normals)
        groups = []
        for k in GAUSS_FIELDS:
            if leaves[k].grad is not None:
                groups.append((self.g[k], leaves[k].grad, c.lr_gauss))
        for p, lp in zip(self.mlp, params):
            groups.append((p, lp.grad, c.lr_mlp))
        self._adam(groups)
        self.it += 1
        return loss.detach()

    # ---- CUDA-graph path
    def _capture(self, coarse: bool, st: dict):
        """Leaves sharing the parameters' storage and two graphs, forward +
        loss and backward, over the static inputs st (positions, noise
        normals, TX, already holding this step's values)."""
        c, dev = self.cfg, self.tx_train.device
        self.spec.stop_grad_mean = not coarse
        leaves = {k: v.detach().requires_grad_(coarse or k != "mean") for k, v in self.g.items()}
        params = [] if coarse else [p.detach().requires_grad_() for p in self.mlp]

        def fwd():
            tx = self.tx_train[st["idx"]] if coarse else st["tx"]
            out = render_spectra(self.spec, tx, leaves["mean"], leaves["log_scale"],
                                 leaves["rot"], leaves["opacity_logit"], leaves["amp"], params)
            return spectrum_loss(out, self.targets[st["idx"]], c.lambda1)

        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            for _ in range(2):  # warm-up: key capacity, workspaces, pinned buffers
                fwd().backward()
                self.spec.renderer.key_overflow()
                for v in list(leaves.values()) + params:
                    v.grad = None
        torch.cuda.current_stream(dev).wait_stream(side)
        # two graphs sharing one memory pool: the forward (with the binning's
        # key count copied to the host) and the backward, so that a step can
        # check the key count while its backward runs
        g_fwd, g_bwd = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_fwd, stream=side):
            loss = fwd()
        with torch.cuda.graph(g_bwd, stream=side, pool=g_fwd.pool()):
            loss.backward()
        self.spec.renderer._pending = None  # replays are checked with replayed_key_overflow
        return dict(g_fwd=g_fwd, g_bwd=g_bwd, fwd_done=torch.cuda.Event(), static=st,
                    leaves=leaves, params=params, loss=loss.detach(),
                    cap=self.spec.renderer.cap, renderer=self.spec.renderer, stream=side)

    def _step_graph(self, idx, normals):
        coarse = self.coarse
        if self.spec.renderer is None or self.spec.renderer.cap <= 0:
            return None  # the first (eager) step sizes the key capacity
        dev, B = self.tx_train.device, self.cfg.batch
        gr = self._graphs.get(coarse)
        if gr is not None and gr["cap"] != self.spec.renderer.cap:
            gr = None
        if gr is None:
            self._graphs.clear()  # one stage at a time holds graph memory
            st = dict(idx=torch.zeros(B, dtype=torch.int64, device=dev),
                      normals=torch.zeros(B, 3, dtype=torch.float32, device=dev),
                      tx=torch.zeros(B, 3, dtype=torch.float32, device=dev))
        else:
            st = gr["static"]
        st["idx"].copy_(self._upload(idx))
        if not coarse:
            st["normals"].copy_(self._upload(normals.to(torch.float32)))
            i = self.it - self.cfg.coarse_iters
            api.wrf_anneal_tx(self.tx_train, st["normals"], i, self.cfg.gamma, self.cfg.tau,
                              self.spec.room_size, idx=st["idx"], out=st["tx"])
        if gr is None:
            gr = self._graphs[coarse] = self._capture(coarse, st)
        self.spec.stop_grad_mean = not coarse
        gr["g_fwd"].replay()
        gr["fwd_done"].record()
        gr["g_bwd"].replay()
        gr["fwd_done"].synchronize()  # the forward only: the backward keeps running
        if gr["renderer"].replayed_key_overflow(gr["cap"], gr["stream"]):
            # the keys did not fit: the capacity is raised; recapture at the
            # next step and recompute this one without the graph
            self._graphs.pop(coarse, None)
            return None
        c = self.cfg
        groups = []
        for k in GAUSS_FIELDS:
            lv = gr["leaves"][k]
            if lv.grad is not None:
                groups.append((self.g[k], lv.grad, c.lr_gauss))
        for p, lp in zip(self.mlp, gr["params"]):
            groups.append((p, lp.grad, c.lr_mlp))
        self._adam(groups)
        self.it += 1
        self.graph_steps += 1
        return gr["loss"].clone()

    def _adam(self, groups):
        # one launch per distinct step count (all equal except around the
        # stage change, when the MLP starts at step 1)
        by_step = {}
        for p, g, lr in groups:
            st = self.state[id(p)]
            st[2] += 1
            by_step.setdefault(st[2], []).append((p, g.contiguous(), st[0], st[1], lr))
        for step, gs in by_step.items():
            for i in range(0, len(gs), 32):
                api.wrf_adam(gs[i:i + 32], step, self.cfg.beta1, self.cfg.beta2, self.cfg.eps)
