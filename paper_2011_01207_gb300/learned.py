"""Learned initial guess: training data from the solver, training, checkpoints.

Training pairs come from the solver itself: for configurations along a trajectory the
induced dipoles are converged tightly, and ap_mlp_features() turns each atom into
(features, target) with target = R^T (mu - alpha E) / 0.02 in the atom's frame. The
network is trained with the library's tensor-core gradient kernel and Adam
(ap_mlp_train_step). Checkpoints hold the FP32 parameters and Adam state in a small
binary file with a header.
"""
from __future__ import annotations

import struct

import numpy as np

from . import binding

MAGIC = b"APMLP001"


def init_params(seed: int, nin=16, nh=128, nout=3) -> np.ndarray:
    """Seeded He-style initialisation, flattened in the library's master order."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(size=(nin, nh)) * np.sqrt(2.0 / nin), np.zeros(nh),
             rng.normal(size=(nh, nh)) * np.sqrt(2.0 / nh), np.zeros(nh),
             rng.normal(size=(nh, nout)) * np.sqrt(1.0 / nh), np.zeros(nout)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def collect(ctx: "binding.Context", positions, tol: float = 1e-8, max_iter: int = 500):
    """(features [M,16], targets [M,3]) as CUDA float32 tensors from converged solves at
    each configuration in `positions` (iterable of [n,3] arrays or CUDA tensors)."""
    import torch
    feats, tgts = [], []
    for xyz in positions:
        ctx.set_positions(xyz) if not isinstance(xyz, torch.Tensor) else ctx.xyz.copy_(xyz)
        ctx.permanent_field(out=False)
        ctx.solve(tol=tol, max_iter=max_iter)
        f = torch.empty((ctx.n, 16), dtype=torch.float32, device=ctx.device)
        t = torch.empty((ctx.n, 3), dtype=torch.float32, device=ctx.device)
        binding.ap_mlp_features(ctx.ctx, f, ctx.mu, t)
        feats.append(f)
        tgts.append(t)
    return torch.cat(feats), torch.cat(tgts)


class Trainer:
    """FP32 master parameters, Adam moments and the packed copy the kernels read."""

    def __init__(self, seed: int = 7, device="cuda", params: np.ndarray | None = None):
        import torch
        self.torch = torch
        P = binding.ap_mlp_param_count()
        p0 = init_params(seed) if params is None else np.asarray(params, np.float32)
        assert p0.size == P
        self.params = torch.tensor(p0, device=device)
        self.grad = torch.zeros(P, dtype=torch.float32, device=device)
        self.m = torch.zeros(P, dtype=torch.float32, device=device)
        self.v = torch.zeros(P, dtype=torch.float32, device=device)
        self.packed = torch.zeros(binding.ap_mlp_packed_bytes(), dtype=torch.uint8, device=device)
        self.step = 0
        binding.ap_mlp_pack(self.params, self.packed)

    def fit(self, feat, target, steps: int, batch: int = 8192, lr: float = 2e-3, seed: int = 0,
            lr_final: float | None = None):
        """Adam on contiguous minibatches of a seeded shuffle; returns per-step losses."""
        torch = self.torch
        n = feat.shape[0]
        g = torch.Generator(device="cpu").manual_seed(seed)
        order = torch.randperm(n, generator=g).to(feat.device)
        feat = feat.index_select(0, order).contiguous()
        target = target.index_select(0, order).contiguous()
        losses = []
        nb = max(1, n // batch)
        for k in range(steps):
            b = k % nb
            fb = feat[b * batch:(b + 1) * batch]
            tb = target[b * batch:(b + 1) * batch]
            loss = torch.zeros(1, dtype=torch.float64, device=feat.device)
            self.step += 1
            rate = lr if lr_final is None else lr * (lr_final / lr) ** (k / max(1, steps - 1))
            binding.ap_mlp_train_step(self.params, self.grad, self.m, self.v, self.step, rate, fb, tb, loss,
                                      self.packed)
            losses.append(loss)
        torch.cuda.synchronize()
        binding.ap_mlp_status()
        return np.array([float(x.item()) for x in losses])

    def loss(self, feat, target):
        torch = self.torch
        grad = torch.zeros_like(self.grad)
        loss = torch.zeros(1, dtype=torch.float64, device=feat.device)
        binding.ap_mlp_gradient(self.packed, feat, target, grad, loss)
        torch.cuda.synchronize()
        return float(loss.item())

    def save(self, path: str):
        arrs = [t.detach().cpu().numpy().astype(np.float32) for t in (self.params, self.m, self.v)]
        with open(path, "wb") as fh:
            fh.write(MAGIC + struct.pack("<qq", arrs[0].size, self.step))
            for a in arrs:
                fh.write(a.tobytes())

    @classmethod
    def load(cls, path: str, device="cuda") -> "Trainer":
        with open(path, "rb") as fh:
            if fh.read(8) != MAGIC:
                raise ValueError("not an MLP checkpoint")
            head = fh.read(16)
            if len(head) != 16:
                raise ValueError("truncated MLP checkpoint")
            size, step = struct.unpack("<qq", head)
            if size <= 0 or step < 0:
                raise ValueError("corrupt MLP checkpoint header")
            arrs = [np.frombuffer(fh.read(4 * size), np.float32) for _ in range(3)]
            if any(a.size != size for a in arrs) or fh.read(1):
                raise ValueError("MLP checkpoint size does not match its header")
        tr = cls(device=device, params=arrs[0])
        tr.m.copy_(tr.torch.tensor(arrs[1], device=device))
        tr.v.copy_(tr.torch.tensor(arrs[2], device=device))
        tr.step = step
        return tr
