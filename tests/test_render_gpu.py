"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances: max |dRGB| <= 1e-3 and mean |dRGB| <= 1e-5 per image; leaf visit
sequences bit-exact for every ray the oracle does not flag as a near tie
(a leaf grazed within 1e-6, or ln T within 1e-3 of ln stop_T).
"""

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


@pytest.mark.parametrize("mode", ["materialise", "fused"])
def test_shell_128_full_frame(mode):
    tree = synth.shell_tree()
    gpu, ref = gu.render_both(tree, camera=synth.shell_camera(), t=synth.SHELL_T, visit_cap=96,
                              idft_mode=mode)
    near = gu.compare(gpu, ref)
    assert near < 0.01 * 128 * 128
    np.testing.assert_allclose(gpu["T"], ref["T"], atol=2e-6, rtol=1e-3)


def test_shell_sweep_32_eyes():
    tree = synth.shell_tree()
    ot = gu.oracle_tree(tree)
    r = fpo.Renderer()
    r.upload(tree)
    try:
        near = 0
        for i, cam in enumerate(synth.sweep_cameras(seed=7, n=32, width=48, height=40)):
            t = float(np.random.default_rng(i).uniform(0, 60))
            gpu, ref = gu.render_both(tree, camera=cam, t=t, visit_cap=96, renderer=r, ot=ot)
            near += gu.compare(gpu, ref)
        assert near < 0.01 * 32 * 48 * 40
    finally:
        r.close()


@pytest.mark.parametrize("seed,depth", [(1, 3), (2, 4), (3, 5), (4, 6), (5, 6)])
@pytest.mark.parametrize("mode", ["materialise", "fused"])
def test_random_mixed_trees_camera(seed, depth, mode):
    tree = synth.random_tree(seed, max_depth=depth)
    cam = synth.Camera(eye=synth.sphere_eye(17 * seed, 35 - 11 * seed), width=53, height=37)
    gpu, ref = gu.render_both(tree, camera=cam, t=1.7 * seed, visit_cap=256, idft_mode=mode)
    gu.compare(gpu, ref)


@pytest.mark.parametrize("seed", [11, 12])
def test_explicit_rays_inside_and_outside(seed):
    tree = synth.random_tree(seed, max_depth=5)
    rng = np.random.default_rng(seed)
    n = 3000
    o = rng.uniform(-0.5, 1.5, (n, 3))  # many origins inside the cube
    d = rng.normal(size=(n, 3))
    gpu, ref = gu.render_both(tree, rays_o=o, rays_d=d, t=12.5, visit_cap=256, bg=(0.2, 0.3, 0.4))
    gu.compare(gpu, ref)


def test_per_ray_times_fused():
    tree = synth.shell_tree()
    rng = np.random.default_rng(3)
    n = 4096
    tgt = rng.uniform(0.1, 0.9, (n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = tgt - 1.5 * d
    tp = rng.uniform(0, 60, n)
    gpu, ref = gu.render_both(tree, rays_o=o, rays_d=d, t_per_ray=tp, visit_cap=96)
    gu.compare(gpu, ref)


@pytest.mark.parametrize("n1,n2", [(11, 5), (21, 5), (31, 11), (7, 3)])
def test_fourier_sizes(n1, n2):
    tree = synth.shell_tree(n1=n1, n2=n2)
    cam = synth.shell_camera(40, 40)
    gpu, ref = gu.render_both(tree, camera=cam, t=31.0, visit_cap=96, idft_mode="materialise")
    gu.compare(gpu, ref)
    if (n1, n2) != (7, 3):
        gpu2, _ = gu.render_both(tree, camera=cam, t=31.0, visit_cap=96, idft_mode="fused")
        gu.compare(gpu2, ref)
    else:
        with pytest.raises(fpo.FPOError) as e:
            gu.render_both(tree, camera=cam, t=31.0, idft_mode="fused")
        assert e.value.code == -8


def test_no_early_stop_and_background():
    tree = synth.shell_tree()
    gpu, ref = gu.render_both(tree, camera=synth.shell_camera(64, 64), t=5.0, stop_T=0.0,
                              bg=(0.0, 0.5, 1.0), visit_cap=96)
    gu.compare(gpu, ref)


def test_empty_tree_and_misses():
    tree = synth.Tree(np.zeros(0, np.uint8), np.zeros((0, 3), np.uint32),
                      np.zeros((0, 166), np.float32), 4)
    gpu, ref = gu.render_both(tree, camera=synth.shell_camera(33, 17), bg=(0.1, 0.2, 0.3))
    assert np.all(gpu["rgb"] == np.float32([0.1, 0.2, 0.3]))
    assert np.all(gpu["T"] == 1.0)
    tree = synth.shell_tree()
    o = np.array([[-1, 2, 2], [0.5, 0.5, -1], [2, 2, 2]], np.float64)
    d = np.array([[1, 0, 0], [0, 1, 0], [1, 1, 1]], np.float64)
    gpu, ref = gu.render_both(tree, rays_o=o, rays_d=d, bg=(0.1, 0.2, 0.3), visit_cap=4)
    assert np.all(gpu["rgb"] == np.float32([0.1, 0.2, 0.3])) and np.all(gpu["visit_count"] == 0)


def test_root_leaf_and_single_deep_leaf():
    rng = np.random.default_rng(0)
    for depth, xyz in [(0, (0, 0, 0)), (7, (40, 77, 90)), (12, (2048, 2047, 2049))]:
        co = synth.draw_coefficients(rng, 1)
        co[0, 0] = 400.0
        tree = synth.Tree(np.array([depth], np.uint8), np.array([xyz], np.uint32), co, depth)
        c = (np.array(xyz) + 0.5) / (1 << depth)
        n = 512
        d = rng.normal(size=(n, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        o = c - 2.0 * d + rng.uniform(-0.3, 0.3, (n, 3)) / (1 << depth)
        gpu, ref = gu.render_both(tree, rays_o=o, rays_d=d, t=3.0, visit_cap=4)
        gu.compare(gpu, ref)
        assert (ref["visit_count"] == 1).sum() > n // 4


def test_cluster_at_the_maximum_depth():
    # 8^3 adjacent depth-12 leaves (the deepest level) inside an otherwise
    # empty depth-3 cell, surrounded by depth-3 leaves: rays aimed at the
    # cluster walk from coarse leaves into it and step between neighbours at
    # the maximum stack depth
    rng = np.random.default_rng(12)
    c0 = 7 * 256 + 120  # depth-12 coordinate of the cluster's corner, inside depth-3 cell (3, 3, 3)
    g = np.arange(8)
    deep = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + c0
    coarse = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    coarse = coarse[(coarse != 3).any(1) & (rng.uniform(size=len(coarse)) < 0.3)]
    d = np.concatenate([np.full(len(deep), 12), np.full(len(coarse), 3)]).astype(np.uint8)
    xyz = np.concatenate([deep, coarse]).astype(np.uint32)
    co = synth.draw_coefficients(rng, len(d))
    co[: len(deep), 0] += 1200.0  # sigma delta about 0.3 per 1/4096 cell: translucent
    tree = synth.Tree(d, xyz, co, 12)
    centre = (c0 + 4.0) / 4096.0
    n = 2048
    dirs = rng.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    o = centre - 1.2 * dirs + rng.uniform(-4.5, 4.5, (n, 3)) / 4096.0
    gpu, ref = gu.render_both(tree, rays_o=o, rays_d=dirs, t=21.0, visit_cap=96)
    gu.compare(gpu, ref)
    assert (ref["visit_count"] >= 8).sum() > n // 8  # many rays cross several deep leaves


def test_ragged_and_tiny_images():
    tree = synth.shell_tree()
    for w, h in [(1, 1), (7, 3), (37, 23), (130, 5)]:
        cam = synth.shell_camera(w, h)
        gpu, ref = gu.render_both(tree, camera=cam, t=9.0, visit_cap=96)
        gu.compare(gpu, ref)


def test_zero_rays():
    tree = synth.shell_tree()
    r = fpo.Renderer()
    r.upload(tree)
    out = r.render(camera=synth.shell_camera(0, 0))
    r.status()
    assert out["rgb"].numel() == 0
    out = r.render(rays_o=torch.zeros(0, 3), rays_d=torch.zeros(0, 3))
    r.status()
    r.close()


def test_non_unit_aabb():
    tree = synth.random_tree(8, max_depth=4)
    tree.aabb_min = (-2.0, 1.0, 0.5)
    tree.aabb_size = 3.0
    cam = synth.Camera(eye=(-5.0, 6.0, 4.0), target=(-0.5, 2.5, 2.0), width=48, height=32)
    gpu, ref = gu.render_both(tree, camera=cam, t=2.0, visit_cap=256)
    gu.compare(gpu, ref)


def test_permuted_upload_order_same_image():
    tree = synth.random_tree(9, max_depth=5)
    perm = np.random.default_rng(1).permutation(tree.n_leaves)
    t2 = synth.Tree(tree.leaf_depth[perm], tree.leaf_xyz[perm], tree.coeffs[perm], tree.max_depth)
    cam = synth.Camera(eye=synth.sphere_eye(50, 10), width=40, height=40)
    a, _ = gu.render_both(tree, camera=cam, t=1.0, visit_cap=128)
    b, _ = gu.render_both(t2, camera=cam, t=1.0, visit_cap=128)
    assert np.array_equal(a["rgb"], b["rgb"])
    la = a["visit_log"].astype(np.int64)
    lb = b["visit_log"].astype(np.int64)
    m = lb >= 0
    assert np.array_equal(np.where(m, perm[np.where(m, lb, 0)], -1), la)


def test_leaf_marks_equal_visited_set():
    tree = synth.shell_tree()
    r = fpo.Renderer()
    r.upload(tree)
    mark = torch.zeros(tree.n_leaves, dtype=torch.uint8, device="cuda")
    res = r.render(camera=synth.shell_camera(64, 64), t=4.0, visit_cap=96, leaf_mark=mark)
    r.status()
    log = res["visit_log"].cpu().numpy()
    seen = np.zeros(tree.n_leaves, bool)
    seen[log[log >= 0]] = True
    assert np.array_equal(mark.cpu().numpy().astype(bool), seen)
    r.close()


def test_visit_overflow_is_reported():
    tree = synth.shell_tree()
    r = fpo.Renderer()
    r.upload(tree)
    r.render(camera=synth.shell_camera(32, 32), t=4.0, visit_cap=2)
    with pytest.raises(fpo.FPOError) as e:
        r.status()
    assert e.value.code == -7
    r.status()  # cleared
    r.close()


def test_errors_before_upload_and_bad_tree():
    r = fpo.Renderer()
    with pytest.raises(fpo.FPOError) as e:
        r.render(camera=synth.shell_camera(8, 8))
    assert e.value.code == -5
    bad = synth.Tree(np.array([1, 2], np.uint8), np.array([[0, 0, 0], [1, 1, 1]], np.uint32),
                     np.zeros((2, 166), np.float32), 2)
    with pytest.raises(fpo.FPOError) as e:
        r.upload(bad)
    assert e.value.code == -4
    cam = synth.Camera(eye=(0.5, 0.5, 3.0), up=(0.0, 0.0, 1.0))  # up parallel to the view
    r.upload(synth.shell_tree())
    with pytest.raises(fpo.FPOError) as e:
        r.render(camera=cam)
    assert e.value.code == -1
    r.close()


def test_materialise_and_fused_agree():
    tree = synth.shell_tree()
    cam = synth.shell_camera()
    a, ref = gu.render_both(tree, camera=cam, t=synth.SHELL_T, idft_mode="materialise")
    b, _ = gu.render_both(tree, camera=cam, t=synth.SHELL_T, idft_mode="fused")
    assert np.abs(a["rgb"] - b["rgb"]).max() <= 2e-5


# ---------------------------------------------------------------------------
# the paper-scale body tree, in the bench's launch configuration


@pytest.fixture(scope="module")
def body():
    tree = synth.body_tree()
    ot = gu.oracle_tree(tree)
    return tree, ot


@pytest.mark.parametrize("mode", ["materialise", "fused"])
def test_body_1080p_sampled_pixels(body, mode):
    tree, ot = body
    assert 2_000_000 <= tree.n_leaves <= 4_000_000
    cams = synth.ring_cameras(16, 1920, 1080)
    r = fpo.Renderer(idft_mode=mode)
    r.upload(tree)
    try:
        import oracle

        for k, t in [(0, 0.0), (5, 22.0), (11, 47.0)]:
            cam = cams[k]
            res = r.render(camera=cam, t=t, visit_cap=512, want_T=True)
            r.status()
            rng = np.random.default_rng(k)
            sel = np.concatenate([rng.integers(0, 1920 * 1080, 3000),
                                  540 * 1920 + np.arange(0, 1920, 3)])
            ref = oracle.render(ot, tree.coeffs, camera=cam, t=t, sel=sel, visit_cap=512)
            gpu = {"rgb": res["rgb"].cpu().numpy()[sel], "visit_log": res["visit_log"].cpu().numpy()[sel],
                   "visit_count": res["visit_count"].cpu().numpy()[sel]}
            gu.compare(gpu, ref)
            assert (ref["visit_count"] > 0).sum() > 150  # the sample sees the body
    finally:
        r.close()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_body_1080p_pipelined_frames(body, storage):
    # the timed launch configuration: fpo_render_frames, the IDFT pass of the
    # next frame beside the traversal on every SM.  Bit-equal to single-frame
    # renders; FP32 sampled pixels within the parity bounds of the oracle.
    tree, ot = body
    cams = synth.ring_cameras(16, 1920, 1080)
    picks = [(3, 5.0), (8, 31.0), (14, 58.0), (1, 17.0)]
    r = fpo.Renderer(storage=storage)
    r.upload(tree)
    try:
        import oracle

        imgs = r.render_frames([cams[k] for k, _ in picks], [t for _, t in picks])
        r.status()
        for i, (k, t) in enumerate(picks):
            single = r.render(camera=cams[k], t=t)["rgb"]
            r.status()
            assert torch.equal(imgs[i], single)
        if storage == "f32":
            for i, (k, t) in enumerate(picks[:2]):
                rng = np.random.default_rng(100 + k)
                sel = rng.integers(0, 1920 * 1080, 3000)
                ref = oracle.render(ot, tree.coeffs, camera=cams[k], t=t, sel=sel)
                gu.compare({"rgb": imgs[i].cpu().numpy()[sel]}, ref)
    finally:
        r.close()


def test_table_reuse_for_views_of_one_frame_time():
    # FPO_FLAG_REUSE_TABLE: views of one t share an IDFT pass; a new t, or new
    # coefficients, rebuild it (the images equal fresh renders bit for bit)
    tree = synth.random_tree(21, max_depth=5, p_split=0.6, p_empty=0.3)
    cams = synth.ring_cameras(4, 48, 40)
    r = fpo.Renderer()
    fresh = fpo.Renderer()
    try:
        r.upload(tree)
        fresh.upload(tree)
        ref = lambda cam, t: fresh.render(camera=cam, t=t)["rgb"].clone()
        r.render(camera=cams[0], t=5.0)
        assert torch.equal(r.render(camera=cams[1], t=5.0, reuse_table=True)["rgb"], ref(cams[1], 5.0))
        assert torch.equal(r.render(camera=cams[2], t=6.5, reuse_table=True)["rgb"], ref(cams[2], 6.5))
        co = torch.as_tensor(tree.coeffs, device="cuda") * 0.5
        r.set_coeffs(co)
        fresh.set_coeffs(co)
        assert torch.equal(r.render(camera=cams[3], t=6.5, reuse_table=True)["rgb"], ref(cams[3], 6.5))
        r.status()
        fresh.status()
    finally:
        r.close()
        fresh.close()


@pytest.mark.parametrize("mode", ["materialise", "fused"])
def test_step_cap_is_reported_and_the_context_stays_usable(mode):
    # device-side failure path without a fault: a cap of 4 steps stops the
    # long rays, the call reports FPO_ERR_TRAVERSAL_LIMIT through the status
    # word, and the same context then renders normally again
    tree = synth.shell_tree()
    cam = synth.shell_camera(64, 64)
    capped = fpo.Renderer(idft_mode=mode, max_steps=4)
    normal = fpo.Renderer(idft_mode=mode)
    try:
        capped.upload(tree)
        normal.upload(tree)
        capped.render(camera=cam, t=3.0)
        with pytest.raises(fpo.FPOError) as e:
            capped.status()
        assert e.value.code == -6
        capped.status()  # the status word was cleared
        ref = normal.render(camera=cam, t=3.0)["rgb"].clone()
        normal.status()
        # rays that needed at most 4 steps are complete and equal
        out = capped.render(camera=cam, t=3.0)["rgb"]
        with pytest.raises(fpo.FPOError):
            capped.status()
        same = (out == ref).all(dim=1)
        assert 0 < int(same.sum()) < same.numel()
    finally:
        capped.close()
        normal.close()


@pytest.mark.parametrize("storage", ["f32", "bf16", "fp8"])
def test_bounded_wait_timeout_is_reported_and_the_context_stays_usable(storage):
    # device-side failure path without a fault: FPO_FLAG_TEST_DEVICE_TIMEOUT
    # makes the IDFT pass's first wait (on a barrier nothing signals) run out
    # after 1 ms; the pass drains its bulk copies in flight, the call reports
    # FPO_ERR_DEVICE_TIMEOUT, and the same context then renders normally
    tree = synth.shell_tree()
    cam = synth.shell_camera(64, 64)
    r = fpo.Renderer(storage=storage)
    try:
        r.upload(tree)
        ref = r.render(camera=cam, t=3.0)["rgb"].clone()
        r.status()
        r.render(camera=cam, t=3.0, test_timeout=True)
        with pytest.raises(fpo.FPOError) as e:
            r.status()
        assert e.value.code == -9
        r.status()  # cleared
        # the failed pass left no valid table behind: REUSE_TABLE rebuilds it
        again = r.render(camera=cam, t=3.0, reuse_table=True)["rgb"]
        r.status()
        assert torch.equal(again, ref)
    finally:
        r.close()
