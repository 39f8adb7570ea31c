"""Training the latent decoder with the library's own kernels.

Each leaf gets a 32-dim latent; a shared MLP 32 -> 64 -> 64 -> n1 + 27 n2
(ReLU) decodes its Fourier coefficients.  Training minimises the per-
coefficient weighted squared error to target coefficients (those the Fourier
PlenOctree generation produces) plus, optionally, the rendered-pixel loss
(PixelLoss): the squared error of rays rendered from the decoded coefficients
against rays rendered from the targets, back-propagated through the render
adjoint (the back-propagation of the fine-tuning stage, Sec. 4.3, Eq. 13) into
the decoder.  Every gradient and update runs in libfpo (fpo_decoder_forward,
fpo_render, fpo_render_backward, fpo_decoder_grad, fpo_adam); PyTorch holds the
arrays and draws the batches.  Inference casts the latents to FP16 and the
weights to BF16 for the tensor-core decoder (fpo_latent_table / LATENT storage).
"""

from __future__ import annotations

import ctypes as C
import math

from . import fpo


class LatentModel:
    def __init__(self, n_leaves: int, n1: int = 31, n2: int = 5, seed: int = 0, device="cuda",
                 tensor_cores: bool = False):
        """tensor_cores: take the gradients with fpo_decoder_grad_tc (tcgen05,
        BF16 operands) instead of fpo_decoder_grad (FP32 SIMT)."""
        import torch

        self.tensor_cores = tensor_cores
        self.status = torch.zeros(1, dtype=torch.int32, device=device)  # fpo_decoder_grad_tc's status word
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

    def grad(self, rows, targets, coef_weight, extra_dy=None, stream=None, accumulate=False):
        """Weight gradients into self.g (zeroed first unless `accumulate`);
        returns (dlatents of the batch rows, loss tensor).  With tensor_cores,
        a device-side time-out is reported by check_status() (fit calls it at
        its end)."""
        import torch

        if not accumulate:
            for t in self.g.values():
                t.zero_()
        b = rows.shape[0]
        dl = torch.empty((b, 32), device=rows.device)
        loss = torch.zeros(1, dtype=torch.float64, device=rows.device)
        w, g = self._mlp(self.p), self._mlp(self.g)
        args = (C.byref(w), self.n1, self.n2, b, C.c_void_p(rows.data_ptr()),
                C.c_void_p(self.p["lat"].data_ptr()), C.c_void_p(targets.data_ptr()),
                C.c_void_p(coef_weight.data_ptr()),
                C.c_void_p(extra_dy.data_ptr() if extra_dy is not None else None), C.byref(g),
                C.c_void_p(dl.data_ptr()), C.c_void_p(loss.data_ptr()))
        if self.tensor_cores:
            fpo.check(fpo.lib().fpo_decoder_grad_tc(*args, C.c_void_p(self.status.data_ptr()), 0,
                                                    C.c_void_p(fpo._stream_handle(stream))))
        else:
            fpo.check(fpo.lib().fpo_decoder_grad(*args, C.c_void_p(fpo._stream_handle(stream))))
        return dl, loss

    def check_status(self, stream=None):
        """Waits for the stream and raises FPOError if a tensor-core gradient
        step reported a device-side time-out."""
        fpo.check_status_word(self.status, stream)

    def decode(self, out=None, stream=None):
        """FP32 coefficients of every leaf [n, nc] (fpo_decoder_forward)."""
        import torch

        if out is None:
            out = torch.empty((self.n, self.nc), device=self.p["lat"].device)
        fpo.check(fpo.lib().fpo_decoder_forward(C.byref(self._mlp(self.p)), self.n1, self.n2, self.n,
                                                C.c_void_p(self.p["lat"].data_ptr()), C.c_void_p(out.data_ptr()),
                                                C.c_void_p(fpo._stream_handle(stream))))
        return out

    def _adam(self, key, grad, lr, rows=None, dim=0, stream=None):
        p, m, v = self.p[key], self.m[key], self.v[key]
        n = grad.numel()
        fpo.check(fpo.lib().fpo_adam(
            C.c_void_p(p.data_ptr()), C.c_void_p(grad.data_ptr()), C.c_void_p(m.data_ptr()),
            C.c_void_p(v.data_ptr()), n, C.c_void_p(rows.data_ptr() if rows is not None else None),
            dim, lr, 0.9, 0.999, 1e-8, self.step_count, C.c_void_p(fpo._stream_handle(stream))))

    def step(self, rows, targets, coef_weight, lr_w=1e-3, lr_lat=1e-2, pixel=None):
        """One Adam step on the batch `rows` (mean weighted L2 to `targets`).
        pixel: optional (rows_px, dy) from PixelLoss.gradient: dL/d(decoded
        coefficients) of the pixel loss for the leaves rows_px (dy is indexed
        by leaf, [n, nc], already a mean over rays), added to the gradients."""
        dl, loss = self.grad(rows, targets, coef_weight)
        self.step_count += 1
        scale = 1.0 / rows.shape[0]
        for k in self.g:
            self.g[k].mul_(scale)
        dl.mul_(scale)
        dl_px = None
        if pixel is not None:
            rows_px, dy = pixel
            if rows_px.shape[0]:
                dl_px, _ = self.grad(rows_px, targets, self._zero_weight(targets.device), extra_dy=dy,
                                     accumulate=True)
        for k in ("w1", "b1", "w2", "b2", "w3", "b3"):
            self._adam(k, self.g[k], lr_w)
        self._adam("lat", dl, lr_lat, rows=rows, dim=32)
        if dl_px is not None:
            self._adam("lat", dl_px, lr_lat, rows=pixel[0], dim=32)
        return loss

    def _zero_weight(self, device):
        import torch

        if getattr(self, "_zw", None) is None:
            self._zw = torch.zeros(self.nc, device=device)
        return self._zw

    def fit(self, targets, steps, batch=65536, lr_w=1e-3, lr_lat=1e-2, coef_weight=None, seed=0,
            log_every=0, decay=1.0, decay_from=0.7, pixel=None):
        """Weighted L2 training on `targets` [n, nc]; returns the loss history.
        Learning rates stay at their start value until `decay_from` of the
        steps, then follow a cosine down to `decay` times it.  pixel: an
        optional PixelLoss, applied every pixel.every steps from
        pixel.start * steps on."""
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
            px = None
            if pixel is not None and s >= pixel.start * steps and (s % pixel.every) == 0:
                px = pixel.gradient(self)
            loss = self.step(rows, targets, coef_weight, lr_w * f, lr_lat * f, pixel=px)
            if log_every and (s % log_every == 0 or s == steps - 1):
                hist.append((s, float(loss.item()) / batch))
        if self.tensor_cores:
            self.check_status()
        return hist

    def inference_arrays(self):
        """FP16 latents and BF16-able weights for the tensor-core decoder."""
        import torch

        return (self.p["lat"].to(torch.float16), self.p["w1"], self.p["b1"], self.p["w2"],
                self.p["b2"], self.p["w3"], self.p["b3"])


class PixelLoss:
    """The rendered-pixel term of the decoder's loss: rays drawn over the
    training views and frames are rendered from the decoder's current
    coefficients and from the target coefficients (both FP32 contexts with the
    per-visit IDFT, since every ray has its own frame time); the mean squared
    RGB error, times `weight`, is back-propagated by fpo_render_backward to
    dL/d(coefficients) of the leaves the rays visit, which the decoder's
    gradient takes as its extra dL/dy."""

    def __init__(self, tree, cams, rays=8192, weight=1.0, every=4, start=0.0, seed=0, n_frames=60,
                 bg=(1.0, 1.0, 1.0), stop_T=1e-4, tensor_cores=False):
        """tree: the target Fourier PlenOctree (leaf structure and target
        coefficients, host arrays); cams: the training cameras; tensor_cores:
        decode the current coefficients on tcgen05 with the inference
        decoder's FP16 numerics (else in FP32)."""
        import torch

        self.cams, self.rays, self.weight, self.every, self.start = cams, rays, weight, every, start
        self.tensor_cores = tensor_cores
        self.n_frames, self.bg, self.stop_T = n_frames, tuple(bg), float(stop_T)
        self.ref = fpo.Renderer(n1=tree.n1, n2=tree.n2, idft_mode="fused")
        self.ref.upload(tree)
        self.work = fpo.Renderer(n1=tree.n1, n2=tree.n2, idft_mode="fused")
        self.work.upload(tree)
        from .finetune import camera_basis

        n, nc = tree.coeffs.shape
        self.dy = torch.zeros((n, nc), device="cuda")
        self.rows = None  # the rows of dy the last gradient wrote
        self.mark = torch.zeros(n, dtype=torch.uint8, device="cuda")
        self.gen = torch.Generator(device="cuda").manual_seed(seed)
        self.basis = camera_basis(cams)
        self.last_loss = None

    def gradient(self, model):
        """(rows, dy): the visited leaves and dL/d(coefficients) [n, nc] of
        the pixel loss at the model's current parameters."""
        import torch

        from .finetune import camera_ray_batch

        self.work.set_coeffs_from_decoder(model._mlp(model.p), model.p["lat"], tensor_cores=self.tensor_cores)
        o, d, t = camera_ray_batch(self.cams, self.rays, self.gen, self.n_frames, basis=self.basis)
        kw = dict(rays_o=o, rays_d=d, t_per_ray=t, bg=self.bg, stop_T=self.stop_T)
        y = self.ref.render(**kw)["rgb"]
        rgb = self.work.render(**kw)["rgb"]
        diff = rgb - y
        self.last_loss = (diff * diff).sum(1).mean()
        if self.rows is not None:  # only the last gradient's rows are non-zero
            self.dy.index_fill_(0, self.rows.long(), 0.0)
        self.mark.zero_()
        self.work.render_backward(rgb, diff * (2.0 * self.weight / self.rays), self.dy, leaf_mark=self.mark, **kw)
        self.rows = torch.nonzero(self.mark).flatten().to(torch.int32)
        if self.tensor_cores:
            self.work.status()  # the decode's FP16 range and time-out reports (the stream is idle here)
        return self.rows, self.dy

    def close(self):
        self.ref.close()
        self.work.close()
