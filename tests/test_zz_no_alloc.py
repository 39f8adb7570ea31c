"""fpo_render_noalloc: the render entry point for callers that cannot call
cudaMalloc when they render.  It must give the same image as fpo_render,
call after call, for every storage precision (the FP32 table of FP32 records
and the FP16 table of the reduced-precision storages both live in the
library's fixed device array) and for camera and explicit rays; the FP32
image must also match the FP64 oracle within the parity tolerance.  Trees
above its leaf limit and rays fpo_render refuses are refused.  (This file
sorts last so a stop-at-first-failure run has already run every other test.)"""

import ctypes as C
import math

import numpy as np
import pytest

import gpu_util as gu
from paper_2202_08614_gb300 import fpo, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

MAX_LEAVES = 65536


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _camera_rays(cam, t):
    rays = fpo.Rays()
    rays.mode = fpo.RAYS_CAMERA
    rays.eye = (C.c_double * 3)(*cam.eye)
    rays.target = (C.c_double * 3)(*cam.target)
    rays.up = (C.c_double * 3)(*cam.up)
    rays.fov_y_deg = float(cam.fov_y_deg)
    rays.width, rays.height = int(cam.width), int(cam.height)
    rays.t = float(t)
    return rays


def _explicit_rays(o, d, t):
    rays = fpo.Rays()
    rays.mode = fpo.RAYS_EXPLICIT
    rays.n = o.shape[0]
    rays.o, rays.d = o.data_ptr(), d.data_ptr()
    rays.t = float(t)
    return rays


def _noalloc(r: fpo.Renderer, rays, out):
    opts = fpo.FrameOpts()
    opts.bg = (C.c_float * 3)(1.0, 1.0, 1.0)
    opts.stop_T = 1e-4
    return fpo.lib().fpo_render_noalloc(r.h, C.byref(rays), C.byref(opts),
                                        C.c_void_p(out.data_ptr()),
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream))


def _random_rays(n, seed):
    rng = np.random.default_rng(seed)
    tgt = rng.uniform(0.1, 0.9, (n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = tgt - 1.6 * d
    return o.astype(np.float32), d.astype(np.float32)


@pytest.mark.parametrize("storage", ["f32", "bf16", "fp8"])
def test_noalloc_matches_render_twice_in_a_row(storage):
    tree = synth.shell_tree()
    assert tree.n_leaves <= MAX_LEAVES
    cam = synth.shell_camera(96, 80)
    r = fpo.Renderer(idft_mode="materialise", storage=storage)
    try:
        r.upload(tree)
        n = cam.width * cam.height
        for t in (synth.SHELL_T, 41.5):  # two calls in a row, different frames
            ref = r.render(camera=cam, t=t)["rgb"]
            out = torch.full((n, 3), -1.0, device="cuda")
            assert _noalloc(r, _camera_rays(cam, t), out) == fpo.FPO_OK, fpo.lib().fpo_last_error()
            r.status()
            assert torch.equal(out, ref)  # same kernels, same arithmetic
    finally:
        r.close()


def test_noalloc_explicit_rays_match_render_and_the_oracle():
    tree = synth.shell_tree()
    o_np, d_np = _random_rays(3000, 11)
    o, d = torch.as_tensor(o_np, device="cuda"), torch.as_tensor(d_np, device="cuda")
    r = fpo.Renderer(idft_mode="materialise")
    try:
        r.upload(tree)
        for t in (7.25, 50.0):
            ref = r.render(rays_o=o, rays_d=d, t=t)["rgb"]
            out = torch.full((o.shape[0], 3), -1.0, device="cuda")
            assert _noalloc(r, _explicit_rays(o, d, t), out) == fpo.FPO_OK, fpo.lib().fpo_last_error()
            r.status()
            assert torch.equal(out, ref)
        ora = gu.oracle.render(gu.oracle_tree(tree), tree.coeffs, rays_o=o_np.astype(np.float64),
                               rays_d=d_np.astype(np.float64), t=50.0, stop_T=1e-4)["rgb"]
        err = np.abs(out.cpu().numpy().astype(np.float64) - ora)
        assert err.max() <= 1e-3 and err.mean() <= 1e-5, (err.max(), err.mean())
    finally:
        r.close()


def test_noalloc_matches_the_oracle():
    tree = synth.shell_tree()
    cam = synth.shell_camera(128, 128)
    r = fpo.Renderer(idft_mode="materialise")
    try:
        r.upload(tree)
        out = torch.full((cam.width * cam.height, 3), -1.0, device="cuda")
        assert _noalloc(r, _camera_rays(cam, synth.SHELL_T), out) == fpo.FPO_OK
        r.status()
    finally:
        r.close()
    ref = gu.oracle.render(gu.oracle_tree(tree), tree.coeffs, camera=cam, t=synth.SHELL_T, stop_T=1e-4)["rgb"]
    err = np.abs(out.cpu().numpy().astype(np.float64) - ref)
    assert err.max() <= 1e-3 and err.mean() <= 1e-5, (err.max(), err.mean())


def test_noalloc_refuses_what_render_refuses():
    tree = synth.shell_tree()
    cam = synth.shell_camera(16, 16)
    r = fpo.Renderer(idft_mode="materialise")
    try:
        r.upload(tree)
        out = torch.empty((16 * 16, 3), device="cuda")
        for bad_t in (math.nan, math.inf):
            assert _noalloc(r, _camera_rays(cam, bad_t), out) == -1
            assert "t must be finite" in fpo.lib().fpo_last_error().decode()
            with pytest.raises(fpo.FPOError):
                r.render(camera=cam, t=bad_t, out=out)
        o = torch.zeros((32, 3), device="cuda")
        d = torch.ones((32, 3), device="cuda")
        tp = torch.zeros(32, device="cuda")
        rays = _explicit_rays(o, d, 1.0)
        rays.t_per_ray = tp.data_ptr()
        assert _noalloc(r, rays, out) == -1
        r.status()
    finally:
        r.close()


def test_noalloc_refuses_trees_above_its_limit():
    rng = np.random.default_rng(0)
    g = 64  # 64^3 = 262144 cells at depth 6, above the 65536-leaf limit
    xyz = np.argwhere(np.ones((g, g, g), bool)).astype(np.uint32)
    tree = synth.Tree(np.full(xyz.shape[0], 6, np.uint8), xyz,
                      synth.draw_coefficients(rng, xyz.shape[0]), 6)
    r = fpo.Renderer(idft_mode="materialise")
    try:
        r.upload(tree)
        out = torch.empty((16 * 16, 3), device="cuda")
        st = _noalloc(r, _camera_rays(synth.shell_camera(16, 16), 3.0), out)
        assert st == -1
        assert "at most 65536" in fpo.lib().fpo_last_error().decode()
    finally:
        r.close()


def test_noalloc_honours_the_step_cap():
    tree = synth.shell_tree()
    cam = synth.shell_camera(64, 64)
    r = fpo.Renderer(idft_mode="materialise", max_steps=4)
    try:
        r.upload(tree)
        out = torch.empty((cam.width * cam.height, 3), device="cuda")
        assert _noalloc(r, _camera_rays(cam, 3.0), out) == fpo.FPO_OK
        with pytest.raises(fpo.FPOError) as e:
            r.status()
        assert e.value.code == -6
        r.status()
    finally:
        r.close()
