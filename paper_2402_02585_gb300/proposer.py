"""Learned angle proposer: an MLP from an instance's density of states to p
angle pairs, trained and run by the library's own kernels.

The paper observes that optimal angles cluster with the instance size and
clause count (Section III.B, Fig. 2; Appendix D) and suggests determining
angles from statistics of the density of states (Section V). The proposer
reads x = [h[c]/2^n (padded to d_in - 2), n/32, m/128] and outputs
angles = 2 pi sigmoid(MLP(x)), the first p gammas then p betas. It is trained
with the periodic loss 2 (1 - cos(angle - label)) to canonicalised angles that
the batched optimizer
(`optim.AngleOptimizer`) produces; gqaoa_mlp_backward and gqaoa_adam_f32 do
every step. At inference the plain optimizer starts from the proposal and
remains the judge: the proposer only chooses the starting point.
"""

from __future__ import annotations

import numpy as np
import torch

from . import _capi as C
from . import core, instances


class Proposer:
    def __init__(self, p: int = 16, d_in: int = 130, d_h: int = 256, seed: int = 0,
                 device="cuda"):
        self.p = p
        self.dims = (d_in, d_h, 2 * p)
        self.device = torch.device(device)
        params = instances.random_mlp_params(*self.dims, seed=seed)
        self.params = torch.as_tensor(params, device=self.device).contiguous()
        self.count = C.gqaoa_mlp_param_count(*self.dims)
        assert self.count == self.params.numel()
        self.m1 = torch.zeros_like(self.params)
        self.m2 = torch.zeros_like(self.params)
        self.grads = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.t = 0
        self._ws = None
        self.launches = 0  # kernels launched by the library for this proposer

    # ------------------------------------------------------------ features
    def features(self, hists, ns, ms) -> torch.Tensor:
        """x [B, d_in] on the device from per-instance histograms (lists of h[c])."""
        d_in = self.dims[0]
        B = len(hists)
        stride = max(len(h) for h in hists)
        H = np.zeros((B, stride), dtype=np.int64)
        for i, h in enumerate(hists):
            H[i, :len(h)] = np.asarray(h, dtype=np.int64)
        Hd = torch.as_tensor(H, device=self.device)
        nd = torch.as_tensor(np.asarray(ns, dtype=np.int32), device=self.device)
        md = torch.as_tensor(np.asarray(ms, dtype=np.int32), device=self.device)
        x = torch.empty((B, d_in), dtype=torch.float32, device=self.device)
        C.gqaoa_mlp_features(Hd.data_ptr(), stride, nd.data_ptr(), md.data_ptr(), B, d_in,
                             x.data_ptr(), torch.cuda.current_stream().cuda_stream)
        self.launches += 1
        return x

    def _workspace(self, B):
        need = C.gqaoa_mlp_workspace_size(B, *self.dims)
        if self._ws is None or self._ws.numel() < need:
            self._ws = core.workspace(need, self.device)
        return self._ws

    # ------------------------------------------------------------ inference
    def predict(self, x: torch.Tensor) -> torch.Tensor:
        """angles [B, 2p] (float32, in (0, 2 pi))."""
        B = x.shape[0]
        out = torch.empty((B, self.dims[2]), dtype=torch.float32, device=self.device)
        ws = self._workspace(B)
        C.gqaoa_mlp_forward(self.params.data_ptr(), *self.dims, x.data_ptr(), B, out.data_ptr(),
                            ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream)
        self.launches += 4  # three GEMMs with their epilogues, the output head
        return out

    def propose(self, x: torch.Tensor):
        """(gammas [B, p], betas [B, p]) float64 on the device."""
        a = self.predict(x).to(torch.float64)
        return a[:, :self.p].contiguous(), a[:, self.p:].contiguous()

    # ------------------------------------------------------------ training
    def train_step(self, x: torch.Tensor, labels: torch.Tensor, lr: float) -> torch.Tensor:
        """One Adam step on the periodic loss of a batch; returns the loss (device)."""
        B = x.shape[0]
        ws = self._workspace(B)
        s = torch.cuda.current_stream().cuda_stream
        C.gqaoa_mlp_backward(self.params.data_ptr(), *self.dims, x.data_ptr(), labels.data_ptr(), B,
                             self.grads.data_ptr(), self.loss.data_ptr(), ws.data_ptr(), ws.numel(), s)
        self.t += 1
        C.gqaoa_adam_f32(self.params.data_ptr(), self.grads.data_ptr(), self.m1.data_ptr(),
                         self.m2.data_ptr(), self.count, lr, 0.9, 0.999, 1e-8, self.t, 1.0, s)
        # forward GEMMs (3), loss head and its sum (2), per layer the weight
        # GEMM, the two-kernel bias column sum and (but the first) the input
        # GEMM (4 + 4 + 3), Adam (1)
        self.launches += 17
        return self.loss

    def fit(self, x: torch.Tensor, labels: torch.Tensor, epochs: int = 200, batch: int = 512,
            lr: float = 1e-3, seed: int = 0) -> list[float]:
        """Mini-batch Adam over (x, labels) on the device; returns the mean loss per epoch."""
        N = x.shape[0]
        labels = labels.to(torch.float32).contiguous()
        g = torch.Generator(device="cpu")
        g.manual_seed(seed)
        hist = []
        for _ in range(epochs):
            perm = torch.randperm(N, generator=g).to(self.device)
            xs = x[perm].contiguous()
            ys = labels[perm].contiguous()
            tot = torch.zeros(1, dtype=torch.float64, device=self.device)
            nb = 0
            for i in range(0, N, batch):
                xb = xs[i:i + batch].contiguous()
                yb = ys[i:i + batch].contiguous()
                tot += self.train_step(xb, yb, lr)
                nb += 1
            hist.append(float(tot.item()) / nb)
        return hist

    def state_dict(self):
        return {"params": self.params.cpu(), "dims": self.dims, "p": self.p}

    def load_state_dict(self, sd):
        self.params.copy_(sd["params"].to(self.device))
