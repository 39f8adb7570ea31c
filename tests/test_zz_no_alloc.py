"""fpo_render_noalloc: the render entry point for callers that cannot call
cudaMalloc when they render.  It must give the same image as fpo_render,
call after call, while keeping its IDFT table in the library's fixed device
array; trees above its leaf limit are refused.  (This file sorts last so a
stop-at-first-failure run has already run every other test.)"""

import ctypes as C

import numpy as np
import pytest

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


def _noalloc(r: fpo.Renderer, cam, t, out):
    rays = fpo.Rays()
    rays.mode = fpo.RAYS_CAMERA
    rays.eye = (C.c_double * 3)(*cam.eye)
    rays.target = (C.c_double * 3)(*cam.target)
    rays.up = (C.c_double * 3)(*cam.up)
    rays.fov_y_deg = float(cam.fov_y_deg)
    rays.width, rays.height = int(cam.width), int(cam.height)
    rays.t = float(t)
    opts = fpo.FrameOpts()
    opts.bg = (C.c_float * 3)(1.0, 1.0, 1.0)
    opts.stop_T = 1e-4
    return fpo.lib().fpo_render_noalloc(r.h, C.byref(rays), C.byref(opts),
                                        C.c_void_p(out.data_ptr()),
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_render_twice_in_a_row():
    tree = synth.shell_tree()
    assert tree.n_leaves <= MAX_LEAVES
    cam = synth.shell_camera(96, 80)
    r = fpo.Renderer(idft_mode="materialise")
    try:
        r.upload(tree)
        n = cam.width * cam.height
        for t in (synth.SHELL_T, 41.5):  # two calls in a row, different frames
            ref = r.render(camera=cam, t=t)["rgb"]
            out = torch.full((n, 3), -1.0, device="cuda")
            assert _noalloc(r, cam, t, out) == fpo.FPO_OK, fpo.lib().fpo_last_error()
            r.status()
            d = (out - ref).abs()
            assert d.max().item() <= 1e-3 and d.mean().item() <= 1e-5
            assert torch.equal(out, ref)  # same kernels, same arithmetic
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
        st = _noalloc(r, synth.shell_camera(16, 16), 3.0, out)
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
        assert _noalloc(r, cam, 3.0, out) == fpo.FPO_OK
        with pytest.raises(fpo.FPOError) as e:
            r.status()
        assert e.value.code == -6
        r.status()
    finally:
        r.close()
