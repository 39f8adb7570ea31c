"""The adjoint render (fpo_render_backward) against the FP64 oracle gradient,
and fine-tuning of leaf coefficients through the autograd Function
(Sec. 4.3: back-propagation through the IDFT, loss of Eq. 13)."""

import math

import numpy as np
import pytest

import gpu_util as gu
from paper_2202_08614_gb300 import fpo, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def camera_rays(cam):
    """Pixel-centre rays of a pinhole camera (the convention documented in fpo.h)."""
    eye, tgt, up = (np.array(v, np.float64) for v in (cam.eye, cam.target, cam.up))
    f = tgt - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    th = math.tan(math.radians(cam.fov_y_deg) / 2)
    px, py = np.meshgrid(np.arange(cam.width), np.arange(cam.height))
    sx = (2 * (px.ravel() + 0.5) / cam.width - 1) * th * cam.width / cam.height
    sy = (1 - 2 * (py.ravel() + 0.5) / cam.height) * th
    d = f[None] + sx[:, None] * r[None] + sy[:, None] * u[None]
    return np.repeat(eye[None], d.shape[0], 0), d


def _grad_case(seed, n_rays=3000, stop_T=1e-4, fp64=False):
    """GPU and oracle gradients of one batch of rays with per-ray times.  The
    dL/drgb of rays the oracle flags (near-stop: ln T within 1e-3 of ln stop_T,
    where FP32 may stop one segment earlier or later than FP64; near-tie: a
    leaf grazed within 1e-6, which FP32 stepping may visit or skip) is set to
    zero on both sides, so that the comparison holds row by row."""
    tree = synth.shell_tree()
    rng = np.random.default_rng(seed)
    tgt = rng.uniform(0.05, 0.95, (n_rays, 3))
    d = rng.normal(size=(n_rays, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = (tgt - 1.6 * d).astype(np.float32)
    d = d.astype(np.float32)
    tp = rng.uniform(0, 60, n_rays).astype(np.float32)
    g = rng.normal(size=(n_rays, 3)).astype(np.float32)
    flags = gu.oracle.render(gu.oracle_tree(tree), tree.coeffs, rays_o=o.astype(np.float64),
                             rays_d=d.astype(np.float64), t_per_ray=tp.astype(np.float64),
                             stop_T=stop_T)["flags"]
    g[flags != 0] = 0.0
    r = fpo.Renderer(idft_mode="fused")
    r.upload(tree)
    to = lambda a: torch.as_tensor(a, device="cuda")
    res = r.render(rays_o=to(o), rays_d=to(d), t_per_ray=to(tp), stop_T=stop_T)
    grad = torch.zeros(tree.coeffs.shape, device="cuda", dtype=torch.float64 if fp64 else torch.float32)
    r.render_backward(res["rgb"], to(g), grad, rays_o=to(o), rays_d=to(d), t_per_ray=to(tp),
                      stop_T=stop_T, fp64=fp64)
    r.status()
    r.close()
    ref = gu.oracle.render_grad(gu.oracle_tree(tree), tree.coeffs, g.astype(np.float64),
                                rays_o=o.astype(np.float64), rays_d=d.astype(np.float64),
                                t_per_ray=tp.astype(np.float64), stop_T=stop_T)
    return grad.cpu().numpy().astype(np.float64), ref, flags


def _row_errors(gpu, ref, floor=1e-3):
    """Per-row relative error ||gpu_row - ref_row|| / ||ref_row|| on the rows
    whose gradient norm is at least `floor` times the largest row norm."""
    nr = np.linalg.norm(ref, axis=1)
    rows = np.nonzero(nr >= floor * nr.max())[0]
    err = np.linalg.norm(gpu[rows] - ref[rows], axis=1) / nr[rows]
    return rows, err


@pytest.mark.parametrize("stop_T", [0.0, 1e-4])
def test_gradient_matches_oracle(stop_T):
    # The FP32 adjoint takes S_j = C - sum_{k<=j} w_k c_k from the forward
    # colour C: a few FP32 ulps of C, absolute, which is relative error on the
    # small gradients of leaves deep along a ray (the FP64 replay below has
    # none of it).  Rows of at least a tenth of the largest row norm hold
    # 1e-4 each; rows down to 1e-3 of it hold 1e-3 (the finite-difference
    # bound) each and 1e-4 at the 99th percentile; norm-wise 1e-5.
    gpu, ref, flags = _grad_case(5, stop_T=stop_T)
    assert np.abs(ref).max() > 0
    rel = np.linalg.norm(gpu - ref) / np.linalg.norm(ref)
    rows, err = _row_errors(gpu, ref, floor=1e-3)
    big, err_big = _row_errors(gpu, ref, floor=1e-1)
    print(f"stop_T={stop_T}: norm-wise {rel:.2e}; {rows.size} rows >= 1e-3 max: worst {err.max():.2e}, "
          f"99th percentile {np.percentile(err, 99):.2e}, median {np.median(err):.2e}; "
          f"{big.size} rows >= 0.1 max: worst {err_big.max():.2e}; flagged rays dropped {(flags != 0).sum()}")
    assert rel <= 1e-5
    assert big.size > 100 and err_big.max() <= 1e-4
    assert err.max() <= 1e-3 and np.percentile(err, 99) <= 1e-4
    # rows untouched by the oracle get nothing on the GPU either
    assert np.all(gpu[np.linalg.norm(ref, axis=1) == 0] == 0)


def test_fp64_gradcheck_matches_oracle():
    # the gradient-check replay: FP64 segments, IDFT, colour and transmittance
    gpu, ref, flags = _grad_case(5, stop_T=1e-4, fp64=True)
    rows, err = _row_errors(gpu, ref, floor=1e-6)
    print(f"FP64 replay: {rows.size} rows, worst row {err.max():.2e}, median {np.median(err):.2e}")
    assert rows.size > 100
    assert err.max() <= 1e-6
    assert np.all(gpu[np.linalg.norm(ref, axis=1) == 0] == 0)
    gpu0, ref0, _ = _grad_case(6, n_rays=1500, stop_T=0.0, fp64=True)
    rows, err = _row_errors(gpu0, ref0, floor=1e-6)
    assert err.max() <= 1e-6


def test_set_coeffs_round_trip():
    tree = synth.shell_tree()
    cam = synth.shell_camera(48, 48)
    r = fpo.Renderer()
    r.upload(tree)
    a = r.render(camera=cam, t=3.0)["rgb"].clone()
    r.set_coeffs(torch.zeros(tree.coeffs.shape, device="cuda"))
    blank = r.render(camera=cam, t=3.0)["rgb"].clone()
    r.set_coeffs(torch.as_tensor(tree.coeffs, device="cuda"))
    b = r.render(camera=cam, t=3.0)["rgb"]
    r.status()
    r.close()
    assert torch.equal(a, b)
    assert torch.allclose(blank, torch.ones_like(blank))  # zero density: background only


def test_autograd_matches_direct_backward():
    tree = synth.shell_tree()
    rng = np.random.default_rng(1)
    cam = synth.shell_camera(32, 32)
    o, d = camera_rays(cam)
    n = o.shape[0]
    tp = torch.full((n,), 12.5, device="cuda")
    ro = torch.as_tensor(o, dtype=torch.float32, device="cuda")
    rd = torch.as_tensor(d, dtype=torch.float32, device="cuda")
    r = fpo.Renderer(idft_mode="fused")
    r.upload(tree)
    k = torch.as_tensor(tree.coeffs, device="cuda").requires_grad_(True)
    w = torch.as_tensor(rng.normal(size=(n, 3)), dtype=torch.float32, device="cuda")
    rgb = fpo.render_rays(k, r, ro, rd, tp)
    (rgb * w).sum().backward()
    direct = torch.zeros_like(k)
    r.render_backward(rgb.detach(), w, direct, rays_o=ro, rays_d=rd, t_per_ray=tp)
    r.status()
    r.close()
    assert torch.allclose(k.grad, direct)
    # camera-mode forward at the same t gives the same image as the explicit rays
    ref = gu.oracle.render(gu.oracle_tree(tree), tree.coeffs, camera=cam, t=12.5)["rgb"]
    assert np.abs(rgb.detach().cpu().numpy() - ref).max() < 1e-3


def test_finetune_recovers_perturbed_coefficients():
    # Eq. 13: sum over views and frames of squared pixel errors; Adam on the
    # FP32 coefficients, batches of rays drawn over 16 views x 60 frames.
    tree = synth.shell_tree()
    rng = np.random.default_rng(3)
    k_true = torch.as_tensor(tree.coeffs, device="cuda")
    noise = rng.normal(size=tree.coeffs.shape) * (0.1 * np.abs(tree.coeffs) + 0.05)
    k = (k_true + torch.as_tensor(noise, dtype=torch.float32, device="cuda")).requires_grad_(True)
    cams = synth.ring_cameras(16, 40, 40)
    rays = [camera_rays(c) for c in cams]
    O = torch.as_tensor(np.stack([r[0] for r in rays]), dtype=torch.float32, device="cuda")
    Dd = torch.as_tensor(np.stack([r[1] for r in rays]), dtype=torch.float32, device="cuda")
    r = fpo.Renderer(idft_mode="fused")
    r.upload(tree)
    opt = torch.optim.Adam([k], lr=1e-2)
    gen = torch.Generator(device="cuda").manual_seed(0)
    npx = 40 * 40

    def batch(nb):
        v = torch.randint(0, 16, (nb,), device="cuda", generator=gen)
        f = torch.randint(0, 60, (nb,), device="cuda", generator=gen).float()
        p = torch.randint(0, npx, (nb,), device="cuda", generator=gen)
        return O[v, p], Dd[v, p], f

    def loss_of(kk, bo, bd, bt, target):
        return ((fpo.render_rays(kk, r, bo, bd, bt) - target) ** 2).sum(1).mean()

    bo, bd, bt = batch(8192)
    with torch.no_grad():
        target_eval = fpo.render_rays(k_true, r, bo, bd, bt)
        l0 = loss_of(k, bo, bd, bt, target_eval).item()
    for step in range(150):
        so, sd, st = batch(8192)
        with torch.no_grad():
            tgt = fpo.render_rays(k_true, r, so, sd, st)
        opt.zero_grad()
        loss = loss_of(k, so, sd, st, tgt)
        loss.backward()
        opt.step()
    with torch.no_grad():
        l1 = loss_of(k, bo, bd, bt, target_eval).item()
    r.status()
    r.close()
    print(f"held-out loss {l0:.3e} -> {l1:.3e}")
    assert l1 < 0.2 * l0


# --------------------------------------------------------------------------
# Row-sparse fine-tuning step: marks from the adjoint, fused Adam + write-back


def _shell_rays(n, seed):
    cams = synth.ring_cameras(16, 40, 40)
    rays = [camera_rays(c) for c in cams]
    rng = np.random.default_rng(seed)
    v, p = rng.integers(0, 16, n), rng.integers(0, 1600, n)
    o = torch.as_tensor(np.stack([rays[i][0][j] for i, j in zip(v, p)]), dtype=torch.float32, device="cuda")
    d = torch.as_tensor(np.stack([rays[i][1][j] for i, j in zip(v, p)]), dtype=torch.float32, device="cuda")
    t = torch.as_tensor(rng.uniform(0, 60, n), dtype=torch.float32, device="cuda")
    return o, d, t


def test_backward_marks_the_forward_visits():
    tree = synth.shell_tree()
    o, d, t = _shell_rays(4000, 1)
    r = fpo.Renderer(idft_mode="fused")
    r.upload(tree)
    fwd = torch.zeros(tree.n_leaves, dtype=torch.uint8, device="cuda")
    rgb = r.render(rays_o=o, rays_d=d, t_per_ray=t, leaf_mark=fwd)["rgb"]
    bwd = torch.zeros_like(fwd)
    g = torch.zeros(tree.coeffs.shape, device="cuda")
    r.render_backward(rgb, torch.ones_like(rgb), g, rays_o=o, rays_d=d, t_per_ray=t, leaf_mark=bwd)
    r.status()
    r.close()
    assert int(fwd.sum()) > 100
    assert torch.equal(fwd, bwd)
    # rows without a mark receive no gradient
    assert float(g[bwd == 0].abs().max()) == 0.0


def test_adam_leaves_matches_adam_on_marked_rows():
    tree = synth.shell_tree()
    n, nc = tree.coeffs.shape
    rng = np.random.default_rng(4)
    P0 = tree.coeffs.astype(np.float64) + rng.normal(size=(n, nc)) * 0.1
    G0, M0 = rng.normal(size=(n, nc)), rng.normal(size=(n, nc)) * 0.1
    V0 = rng.uniform(0, 0.5, (n, nc))
    mk = (rng.uniform(size=n) < 0.3).astype(np.uint8)
    dev = lambda a: torch.as_tensor(np.asarray(a, np.float32), device="cuda").contiguous()
    P, G, M, V = dev(P0), dev(G0), dev(M0), dev(V0)
    mark = torch.as_tensor(mk, device="cuda")
    r = fpo.Renderer()
    r.upload(tree)
    r.set_coeffs(P)
    lr, b1, b2, eps, step = 0.01, 0.9, 0.999, 1e-8, 3
    r.adam_leaves(P, G, M, V, mark, step, lr=lr, betas=(b1, b2), eps=eps)
    cam = synth.shell_camera(48, 48)
    img = r.render(camera=cam, t=9.0)["rgb"].clone()
    r.set_coeffs(P)
    img2 = r.render(camera=cam, t=9.0)["rgb"]
    r.status()
    r.close()
    # Adam (Kingma & Ba) on the marked rows, from the FP32 inputs in FP64
    f = lambda a: np.asarray(a, np.float32).astype(np.float64)
    m_ = b1 * f(M0) + (1 - b1) * f(G0)
    v_ = b2 * f(V0) + (1 - b2) * f(G0) ** 2
    p_ = f(P0) - lr * (m_ / (1 - b1 ** step)) / (np.sqrt(v_ / (1 - b2 ** step)) + eps)
    on = mk.astype(bool)
    Pn, Gn, Mn, Vn = (x.cpu().numpy() for x in (P, G, M, V))
    np.testing.assert_allclose(Pn[on], p_[on], atol=1e-6)
    # FP32 arithmetic: 1 - beta2 = 0.001 itself carries a relative error of
    # about 2^-24 / 0.001 = 6e-5, so the moments agree to ~1e-6 absolute
    np.testing.assert_allclose(Mn[on], m_[on], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(Vn[on], v_[on], rtol=1e-6, atol=1e-6)
    assert np.array_equal(Pn[~on], np.float32(P0[~on])) and np.array_equal(Mn[~on], np.float32(M0[~on]))
    assert np.array_equal(Gn[~on], np.float32(G0[~on])) and not Gn[on].any()
    assert int(mark.sum()) == 0
    # the records were written with the new rows: same image as set_coeffs(P)
    assert torch.equal(img, img2)


def test_finetuner_recovers_perturbed_coefficients():
    # Eq. 13 with the library's row-sparse step (marks -> fused Adam + write-back)
    from paper_2202_08614_gb300.finetune import FineTuner

    tree = synth.shell_tree()
    rng = np.random.default_rng(3)
    k_true = torch.as_tensor(tree.coeffs, device="cuda")
    noise = rng.normal(size=tree.coeffs.shape) * (0.1 * np.abs(tree.coeffs) + 0.05)
    ref = fpo.Renderer(idft_mode="fused")
    ref.upload(tree)
    r = fpo.Renderer(idft_mode="fused")
    r.upload(tree)
    ft = FineTuner(r, k_true + torch.as_tensor(noise, dtype=torch.float32, device="cuda"), lr=1e-2)
    ho = _shell_rays(8192, 99)
    y_ho = ref.render(rays_o=ho[0], rays_d=ho[1], t_per_ray=ho[2])["rgb"].clone()
    held = lambda: float(((ft.render(*ho) - y_ho) ** 2).sum(1).mean())
    l0 = held()
    for s in range(150):
        o, d, t = _shell_rays(8192, 1000 + s)
        y = ref.render(rays_o=o, rays_d=d, t_per_ray=t)["rgb"].clone()
        ft.step(o, d, t, y)
    l1 = held()
    r.status()
    ref.status()
    r.close()
    ref.close()
    print(f"held-out loss {l0:.3e} -> {l1:.3e}")
    assert l1 < 0.2 * l0
    assert int(ft.mark.sum()) == 0
