"""Pipelined multi-frame rendering (fpo_render_frames): the IDFT table of
frame k+1 is computed on a second stream while frame k is traversed, both
kernels resident on every SM with their own launch shapes (the warp-
cooperative form of the IDFT pass for every storage).  The images must equal,
bit for bit, those of one fpo_render call per frame (same per-leaf and per-ray
arithmetic), and one of them is checked against the FP64 oracle."""

import numpy as np
import pytest

import gpu_util as gu
from paper_2202_08614_gb300 import fpo, synth
from paper_2202_08614_gb300.latent import LatentModel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _per_frame(r, cams, times):
    return torch.stack([r.render(camera=c, t=t)["rgb"].clone() for c, t in zip(cams, times)])


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16", "fp8"])
@pytest.mark.parametrize("n_frames", [1, 2, 4, 7, 9])
def test_frames_equal_single_renders(storage, n_frames):
    tree = synth.random_tree(11, max_depth=7, p_split=0.6, p_empty=0.3)
    cams = synth.ring_cameras(8, 160, 96)
    times = [3.0 + 7.7 * i for i in range(n_frames)]
    cs = [cams[i % 8] for i in range(n_frames)]
    r = fpo.Renderer(storage=storage)
    try:
        r.upload(tree)
        a = r.render_frames(cs, times)
        b = _per_frame(r, cs, times)
        r.status()
        assert torch.equal(a, b)
        # a second batch reuses the tables and streams
        a2 = r.render_frames(cs[::-1], times[::-1])
        r.status()
        assert torch.equal(a2, b.flip(0))
    finally:
        r.close()
    if storage == "f32":
        ref = gu.oracle.render(gu.oracle_tree(tree), tree.coeffs, camera=cs[-1], t=times[-1])["rgb"]
        d = np.abs(a[-1].cpu().numpy() - ref)
        assert d.mean() <= 1e-5


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("n_frames", [2, 5, 9])
def test_views_of_one_frame_time(storage, n_frames):
    # every frame at the same t: one table pass serves all the call's
    # traversals; each view equals its own single-frame render, and a
    # following call at another t recomputes the table
    tree = synth.random_tree(17, max_depth=7, p_split=0.6, p_empty=0.3)
    cams = synth.ring_cameras(12, 160, 96)
    cs = [cams[i % 12] for i in range(n_frames)]
    r = fpo.Renderer(storage=storage)
    try:
        r.upload(tree)
        for t in (12.5, 40.25):
            a = r.render_frames(cs, [t] * n_frames)
            b = _per_frame(r, cs, [t] * n_frames)
            r.status()
            assert torch.equal(a, b)
    finally:
        r.close()


@pytest.mark.parametrize("n_frames", [3, 11])
def test_frame_done_events_cover_their_frame(n_frames):
    # each frame read back on a copy stream that waits only for that frame's
    # completion event (as an end-to-end caller does) equals its own
    # single-frame render
    tree = synth.random_tree(13, max_depth=7, p_split=0.6, p_empty=0.3)
    cams = synth.ring_cameras(8, 320, 180)
    times = [1.0 + 5.3 * i for i in range(n_frames)]
    cs = [cams[i % 8] for i in range(n_frames)]
    r = fpo.Renderer()
    try:
        r.upload(tree)
        ref = _per_frame(r, cs, times)
        r.status()
        out = torch.empty_like(ref)
        host = torch.empty(ref.shape, dtype=torch.float32, pin_memory=True)
        evs = [torch.cuda.Event() for _ in range(n_frames)]
        copy = torch.cuda.Stream()
        torch.cuda.synchronize()
        r.render_frames(cs, times, out=out, frame_events=evs)
        with torch.cuda.stream(copy):
            for k in range(n_frames):
                copy.wait_event(evs[k])
                host[k].copy_(out[k], non_blocking=True)
        copy.synchronize()
        r.status()
        assert torch.equal(host, ref.cpu())
    finally:
        r.close()


@pytest.mark.parametrize("depth", [5, 7])
def test_frames_latent_storage(depth):
    # LATENT frames in the pipeline: the two-warpgroup decoder CTA beside the
    # traversal gives the same table, bit for bit, as the eight-warpgroup one
    # of single-frame renders (depth 7: 325k leaves, many tiles per group)
    xyz = synth.shell_leaves(depth)
    n = xyz.shape[0]
    d = np.full(n, depth, np.uint8)
    m = LatentModel(n, seed=4)
    m.p["b3"][0] = 20.0
    lat, *w = m.inference_arrays()
    r = fpo.Renderer(storage="latent")
    try:
        r.upload(synth.Tree(d, xyz, np.zeros((0, 166), np.float32), depth))
        r.set_latents(lat, *w)
        cams = synth.ring_cameras(4, 64, 48)
        times = [1.0, 30.5, 59.0, 12.25]
        a = r.render_frames(cams, times)
        b = _per_frame(r, cams, times)
        r.status()
        assert torch.equal(a, b)
    finally:
        r.close()


def test_frames_rejects_mixed_sizes():
    tree = synth.shell_tree()
    r = fpo.Renderer()
    try:
        r.upload(tree)
        cams = [synth.Camera(eye=synth.sphere_eye(10, 10), width=32, height=32),
                synth.Camera(eye=synth.sphere_eye(10, 10), width=32, height=16)]
        with pytest.raises(fpo.FPOError) as e:
            r.render_frames(cams, [1.0, 2.0], out=torch.empty((2, 1024, 3), device="cuda"))
        assert e.value.code == -1
        assert r.render_frames([], []).shape[0] == 0
    finally:
        r.close()
