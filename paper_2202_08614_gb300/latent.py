"""Training the latent decoder with the library's own kernels.

Each leaf gets a 32-dim latent; a shared MLP 32 -> 64 -> 64 -> n1 + 27 n2
(ReLU) decodes its Fourier coefficients.  Training minimises the per-
coefficient weighted squared error to target coefficients (those the Fourier
PlenOctree generation produces); every gradient and update runs in libfpo
(fpo_decoder_grad, fpo_adam).  PyTorch holds the arrays and draws the batches.
Inference casts the latents to FP16 and the weights to BF16 for the
tensor-core decoder (fpo_latent_table / LATENT storage).
"""

from __future__ import annotations

import ctypes as C
import math

from . import fpo


class LatentModel:
    def __init__(self, n_leaves: int, n1: int = 31, n2: int = 5, seed: int = 0, device="cuda"):
        import torch

        self.n, self.n1, self.n2 = n_leaves, n1, n2
        self.nc = n1 + 27 * n2
        g = torch.Generator(device=device).manual_seed(seed)
        rn = lambda *s: torch.randn(*s, generator=g, device=device)
        self.p = {
            "lat": rn(n_leaves, 32) * 0.5,
            "w1": rn(64, 32) * math.sqrt(2 / 32), "b1": torch.zeros(64, device=device),
            "w2": rn(64, 64) * math.sqrt(2 / 64), "b2": torch.zeros(64, device=device),
            "w3": rn(self.nc, 64) * math.sqrt(1 / 64) * 0.1, "b3": torch.zeros(self.nc, device=device),
        }
        self.m = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.g = {k: torch.zeros_like(v) for k, v in self.p.items() if k != "lat"}
        self.step_count = 0

    def state_dict(self):
        """Latents, MLP, Adam moments and step count (host tensors)."""
        return {"n1": self.n1, "n2": self.n2, "step_count": self.step_count,
                "p": {k: v.cpu() for k, v in self.p.items()}, "m": {k: v.cpu() for k, v in self.m.items()},
                "v": {k: v.cpu() for k, v in self.v.items()}}

    def load_state_dict(self, st):
        if (st["n1"], st["n2"]) != (self.n1, self.n2) or tuple(st["p"]["lat"].shape) != tuple(self.p["lat"].shape):
            raise ValueError("state of a different model size")
        for part in ("p", "m", "v"):
            for k, t in getattr(self, part).items():
                t.copy_(st[part][k])
        self.step_count = int(st["step_count"])

    def _mlp(self, d):
        return fpo.Mlp(*(d[k].data_ptr() for k in ("w1", "b1", "w2", "b2", "w3", "b3")))

    def default_weights(self, device, sigma_weight: float = 0.05):
        """Squared-error weights by each coefficient's first-order effect on a
        composited pixel: a density error moves alpha by about delta * d_sigma
        (delta ~ a fine cell), an SH error moves the colour by about
        S'(.) Y_00 d_z ~ 0.07 d_z; both scaled by |IDFT_i| <= 1."""
        import torch

        w = torch.ones(self.nc, device=device)
        w[: self.n1] = sigma_weight
        return (w / self.nc).contiguous()

    def init_output_bias(self, targets):
        self.p["b3"].copy_(targets.mean(0))

    def grad(self, rows, targets, coef_weight, extra_dy=None, stream=None):
        """Accumulates weight gradients into self.g; returns (dlatents, loss tensor)."""
        import torch

        for t in self.g.values():
            t.zero_()
        b = rows.shape[0]
        dl = torch.empty((b, 32), device=rows.device)
        loss = torch.zeros(1, dtype=torch.float64, device=rows.device)
        w, g = self._mlp(self.p), self._mlp(self.g)
        fpo.check(fpo.lib().fpo_decoder_grad(
            C.byref(w), self.n1, self.n2, b, C.c_void_p(rows.data_ptr()),
            C.c_void_p(self.p["lat"].data_ptr()), C.c_void_p(targets.data_ptr()),
            C.c_void_p(coef_weight.data_ptr()),
            C.c_void_p(extra_dy.data_ptr() if extra_dy is not None else None), C.byref(g),
            C.c_void_p(dl.data_ptr()), C.c_void_p(loss.data_ptr()),
            C.c_void_p(fpo._stream_handle(stream))))
        return dl, loss

    def _adam(self, key, grad, lr, rows=None, dim=0, stream=None):
        p, m, v = self.p[key], self.m[key], self.v[key]
        n = grad.numel()
        fpo.check(fpo.lib().fpo_adam(
            C.c_void_p(p.data_ptr()), C.c_void_p(grad.data_ptr()), C.c_void_p(m.data_ptr()),
            C.c_void_p(v.data_ptr()), n, C.c_void_p(rows.data_ptr() if rows is not None else None),
            dim, lr, 0.9, 0.999, 1e-8, self.step_count, C.c_void_p(fpo._stream_handle(stream))))

    def step(self, rows, targets, coef_weight, lr_w=1e-3, lr_lat=1e-2, extra_dy=None):
        dl, loss = self.grad(rows, targets, coef_weight, extra_dy)
        self.step_count += 1
        scale = 1.0 / rows.shape[0]
        for k in self.g:
            self.g[k].mul_(scale)
        dl.mul_(scale)
        for k in ("w1", "b1", "w2", "b2", "w3", "b3"):
            self._adam(k, self.g[k], lr_w)
        self._adam("lat", dl, lr_lat, rows=rows, dim=32)
        return loss

    def fit(self, targets, steps, batch=65536, lr_w=1e-3, lr_lat=1e-2, coef_weight=None, seed=0,
            log_every=0, decay=1.0, decay_from=0.7):
        """Weighted L2 training on `targets` [n, nc]; returns the loss history.
        Learning rates stay at their start value until `decay_from` of the
        steps, then follow a cosine down to `decay` times it."""
        import torch

        dev = targets.device
        if coef_weight is None:
            coef_weight = self.default_weights(dev)
        g = torch.Generator(device=dev).manual_seed(seed)
        perm = torch.randperm(self.n, generator=g, device=dev).to(torch.int32)
        at, hist = 0, []
        batch = min(batch, self.n)
        for s in range(steps):
            if at + batch > self.n:
                perm = torch.randperm(self.n, generator=g, device=dev).to(torch.int32)
                at = 0
            rows = perm[at:at + batch]
            at += batch
            u = max(0.0, (s / max(1, steps - 1) - decay_from) / max(1e-9, 1.0 - decay_from))
            f = decay + (1.0 - decay) * 0.5 * (1.0 + math.cos(math.pi * min(1.0, u)))
            loss = self.step(rows, targets, coef_weight, lr_w * f, lr_lat * f)
            if log_every and (s % log_every == 0 or s == steps - 1):
                hist.append((s, float(loss.item()) / batch))
        return hist

    def inference_arrays(self):
        """FP16 latents and BF16-able weights for the tensor-core decoder."""
        import torch

        return (self.p["lat"].to(torch.float16), self.p["w1"], self.p["b1"], self.p["w2"],
                self.p["b2"], self.p["w3"], self.p["b3"])
