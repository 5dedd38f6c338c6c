"""Training and use of the MLP surrogate of the per-halo ICM solve.

The host loop here only sequences calls: every forward, loss, backward and Adam step
is one of the library's kernels (bp_mlp_* in include/bp.h).  Training targets come
from the library's FP64 solve.  Checkpoints use a small self-describing binary format
(header + FP32 arrays) so that training can resume.
"""
from __future__ import annotations

import math
import struct

import numpy as np
import torch

from . import _lib as L
from .inputs import SURROGATE_RANGES

MAGIC = b"BPSURR01"


def feature_norm():
    """Means and scales of the 6 features: the centres and half-widths of the sampling
    ranges, so the training set maps onto [-1, 1]."""
    R = SURROGATE_RANGES
    lm = R["log10_M"]
    # log10 c spans the c(M) relation over the mass range, widened by the scatter
    c_lo = math.log10(5.0 * (10 ** lm[1] / 1e14) ** -0.1) + R["dlog10_c"][0]
    c_hi = math.log10(5.0 * (10 ** lm[0] / 1e14) ** -0.1) + R["dlog10_c"][1]
    rng = [lm, (c_lo, c_hi), R["z"], R["eps_star"], R["f_star"], R["eps_dm"]]
    mean = [0.5 * (a + b) for a, b in rng]
    scale = [0.5 * (b - a) for a, b in rng]
    return np.array(mean), np.array(scale)


class Surrogate:
    def __init__(self, params: torch.Tensor, norm: torch.Tensor, hull: torch.Tensor):
        self.params = params  # FP32 [NPARAMS] on the device
        self.norm = norm      # FP32 [18]
        self.hull = hull      # FP32 [12]
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.step = 0
        self.wb = None
        self.history = []

    @staticmethod
    def init(device, seed=0, hull_margin=0.02):
        rng = np.random.default_rng(seed)
        p = np.zeros(L.MLP_NPARAMS, np.float32)
        off = 0
        for fin, fout in ((6, 128), (128, 128), (128, 128), (128, 3)):
            lim = math.sqrt(6.0 / (fin + fout))  # Glorot uniform
            p[off:off + fin * fout] = rng.uniform(-lim, lim, fin * fout)
            off += fin * fout + fout  # biases stay 0
        fm, fs = feature_norm()
        norm = np.concatenate([fm, np.zeros(3), fs, np.ones(3)]).astype(np.float32)
        hull = np.concatenate([np.full(6, -1.0 - hull_margin),
                               np.full(6, 1.0 + hull_margin)]).astype(np.float32)
        t = lambda a: torch.from_numpy(a).to(device)
        return Surrogate(t(p), t(norm), t(hull))

    # ------------------------------------------------------------ training
    def fit(self, ctx, M, c, z, prm, epochs=8, batch=4096, lr=2e-3, lr_min=5e-5,
            log_every=200):
        """Solve the training halos with the FP64 solve, then train with Adam on the
        normalised targets.  Returns the final training loss."""
        model, status = ctx.solve_halos_ex(M, c, z, params=prm, raise_on_noconv=False)
        ok = status == 0
        M, c, z, prm, model = M[ok], c[ok], z[ok], prm[:, ok].contiguous(), model[:, ok]
        model = model.contiguous()
        # target normalisation from the raw targets of the training set
        ident = self.norm.clone()
        ident[6:9] = 0.0
        ident[15:18] = 1.0
        raw = ctx.mlp_targets(model, ident).double().cpu().numpy()
        self.norm[6:9] = torch.from_numpy(raw.mean(0).astype(np.float32))
        self.norm[15:18] = torch.from_numpy(raw.std(0).astype(np.float32) + 1e-6)
        x = ctx.mlp_features(M, c, z, prm, self.norm)
        t = ctx.mlp_targets(model, self.norm)
        n = x.shape[0]
        steps_per_epoch = max(1, n // batch)
        total = epochs * steps_per_epoch
        cache = torch.empty((batch, L.MLP_CACHE_PER_ROW), dtype=torch.float32, device=x.device)
        dy = torch.empty((batch, 3), dtype=torch.float32, device=x.device)
        grad = torch.empty(L.MLP_NPARAMS, dtype=torch.float32, device=x.device)
        loss = float("nan")
        for k in range(total):
            i0 = (k % steps_per_epoch) * batch
            xb, tb = x[i0:i0 + batch], t[i0:i0 + batch]
            y, _ = ctx.mlp_forward(self.params, xb, cache)
            want = (k % log_every == 0) or (k == total - 1)
            _, l = ctx.mlp_mse(y, tb, dy, want_loss=want)
            ctx.mlp_backward(self.params, xb, cache, dy, grad)
            self.step += 1
            frac = k / max(1, total - 1)
            lr_k = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * frac))
            ctx.mlp_adam(self.params, grad, self.m, self.v, self.step, lr_k)
            if want:
                loss = l
                self.history.append((self.step, l))
        self.wb = ctx.mlp_to_bf16(self.params)
        return loss

    def bf16(self, ctx):
        if self.wb is None:
            self.wb = ctx.mlp_to_bf16(self.params)
        return self.wb

    def solve(self, ctx, M, c, z, prm=None, polish_iter=4, gate=1e-4, raise_on_noconv=True):
        return ctx.solve_halos_surrogate(M, c, z, prm, self.bf16(ctx), self.params, self.norm,
                                         self.hull, polish_iter, gate,
                                         raise_on_noconv=raise_on_noconv)

    # ------------------------------------------------------------ checkpoints
    def save(self, path):
        arrays = [self.params, self.norm, self.hull, self.m, self.v]
        with open(path, "wb") as f:
            f.write(MAGIC)
            f.write(struct.pack("<qq", self.step, len(arrays)))
            for a in arrays:
                h = a.detach().float().cpu().numpy()
                f.write(struct.pack("<q", h.size))
                f.write(h.astype("<f4").tobytes())

    @staticmethod
    def load(path, device):
        with open(path, "rb") as f:
            if f.read(8) != MAGIC:
                raise ValueError("not a surrogate checkpoint")
            step, na = struct.unpack("<qq", f.read(16))
            arrs = []
            for _ in range(na):
                (sz,) = struct.unpack("<q", f.read(8))
                arrs.append(torch.from_numpy(np.frombuffer(f.read(4 * sz), "<f4").copy())
                            .to(device))
        s = Surrogate(arrs[0], arrs[1], arrs[2])
        s.m, s.v, s.step = arrs[3], arrs[4], step
        return s
