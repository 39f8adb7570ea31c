"""Fine-tuning of the leaf coefficients (Sec. 4.3): minimise the squared
pixel error of Eq. 13 over rays drawn from the training views and frames.

One step on a batch of explicit rays with per-ray frame times:
  forward   fpo_render (per-visit IDFT, since every ray has its own t),
  loss      mean over rays of the squared RGB error, dL/drgb = 2 (rgb - y) / B,
  adjoint   fpo_render_backward into a dense gradient buffer, marking the
            leaves it touches,
  update    fpo_adam_leaves: Adam on the marked rows only, written straight
            into the renderer's FP32 records; the gradient rows and marks are
            reset in the same pass.
Nothing in a step waits for the host.  Rows the batch did not visit keep their
moments (a sparse-gradient Adam): with a 3.5M-leaf tree a batch of 65,536
rays touches a small fraction of the rows, and a dense update would move all
of them (16 GB per step) to change a few.
"""

from __future__ import annotations

import numpy as np

from . import fpo


def camera_basis(cams):
    """Eye, forward, right and up vectors of each camera: CUDA float32 [n, 12]."""
    import torch

    basis = []
    for c in cams:
        eye, tgt, up = (np.array(v, np.float64) for v in (c.eye, c.target, c.up))
        f = (tgt - eye) / np.linalg.norm(tgt - eye)
        r = np.cross(f, up)
        r /= np.linalg.norm(r)
        basis.append(np.concatenate([eye, f, r, np.cross(r, f)]))
    return torch.as_tensor(np.stack(basis), dtype=torch.float32, device="cuda")


def camera_ray_batch(cams, n, gen, n_frames=60, basis=None):
    """n training rays drawn uniformly over (camera, integer frame, pixel):
    origins, unit directions (pixel centres of the pinhole model documented
    in fpo.h) and frame times, as CUDA tensors.  `gen`: a CUDA torch.Generator;
    `basis`: camera_basis(cams), if already at hand."""
    import torch

    B = camera_basis(cams) if basis is None else basis
    W, H = cams[0].width, cams[0].height
    th = np.tan(np.radians(cams[0].fov_y_deg) / 2)
    v = torch.randint(0, len(cams), (n,), device="cuda", generator=gen)
    p = torch.randint(0, W * H, (n,), device="cuda", generator=gen)
    t = torch.randint(0, n_frames, (n,), device="cuda", generator=gen).float()
    sx = ((2 * ((p % W).float() + 0.5) / W - 1) * th * W / H)[:, None]
    sy = ((1 - 2 * ((p // W).float() + 0.5) / H) * th)[:, None]
    b = B[v]
    d = b[:, 3:6] + sx * b[:, 6:9] + sy * b[:, 9:12]
    return b[:, 0:3].contiguous(), (d / d.norm(dim=1, keepdim=True)).contiguous(), t


class FineTuner:
    def __init__(self, renderer: "fpo.Renderer", coeffs, lr: float = 1e-2, betas=(0.9, 0.999),
                 eps: float = 1e-8, bg=(1.0, 1.0, 1.0), stop_T: float = 1e-4):
        """renderer: an FP32 context holding the tree; coeffs: CUDA float32
        [n_leaves, n1 + 27 n2] (canonical), copied as the starting parameters
        and written into the renderer."""
        import torch

        self.r = renderer
        self.param = coeffs.detach().clone().float().contiguous()
        self.m = torch.zeros_like(self.param)
        self.v = torch.zeros_like(self.param)
        self.grad = torch.zeros_like(self.param)
        self.mark = torch.zeros(self.param.shape[0], dtype=torch.uint8, device=self.param.device)
        self.lr, self.betas, self.eps = lr, betas, eps
        self.bg, self.stop_T = tuple(bg), float(stop_T)
        self.steps = 0
        self.r.set_coeffs(self.param)

    def state_dict(self):
        """Coefficients, Adam moments and step count (host tensors)."""
        return {"param": self.param.cpu(), "m": self.m.cpu(), "v": self.v.cpu(), "steps": self.steps,
                "lr": self.lr, "betas": tuple(self.betas), "eps": self.eps}

    def load_state_dict(self, st):
        """Restores a state_dict and writes the coefficients into the renderer."""
        if tuple(st["param"].shape) != tuple(self.param.shape):
            raise ValueError(f"state for {tuple(st['param'].shape)} coefficients, tuner has {tuple(self.param.shape)}")
        for name in ("param", "m", "v"):
            getattr(self, name).copy_(st[name])
        self.steps = int(st["steps"])
        self.lr, self.betas, self.eps = st["lr"], tuple(st["betas"]), st["eps"]
        self.grad.zero_()
        self.mark.zero_()
        self.r.set_coeffs(self.param)

    def render(self, rays_o, rays_d, t, out=None):
        return self.r.render(rays_o=rays_o, rays_d=rays_d, t_per_ray=t, bg=self.bg, stop_T=self.stop_T,
                             out=out)["rgb"]

    def step(self, rays_o, rays_d, t, target, events=None):
        """One optimiser step; returns the batch loss (a CUDA scalar, before the
        update).  events: optional 4 CUDA events recorded between the phases."""
        rec = (lambda i: events[i].record()) if events else (lambda i: None)
        rec(0)
        rgb = self.render(rays_o, rays_d, t)
        diff = rgb - target
        loss = (diff * diff).sum(1).mean()
        dl = diff * (2.0 / max(1, rgb.shape[0]))
        rec(1)
        self.r.render_backward(rgb, dl, self.grad, rays_o=rays_o, rays_d=rays_d, t_per_ray=t, bg=self.bg,
                               stop_T=self.stop_T, leaf_mark=self.mark)
        rec(2)
        self.steps += 1
        self.r.adam_leaves(self.param, self.grad, self.m, self.v, self.mark, self.steps, lr=self.lr,
                           betas=self.betas, eps=self.eps)
        rec(3)
        return loss
