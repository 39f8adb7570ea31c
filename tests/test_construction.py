"""Fourier PlenOctree generation (Sec. 4.2): the union of per-frame octree
structures (host, library vs the plain oracle) and the per-leaf DFT of
Eq. 10-12 (GPU vs the FP64 oracle), then the whole chain: frames -> union ->
DFT -> render at a frame == that frame's own octree rendered directly."""

import numpy as np
import pytest

import oracle
from oracle import union as ounion
from paper_2202_08614_gb300 import build as fbuild
from paper_2202_08614_gb300 import fpo, synth

N1, N2 = 31, 5
NCOEF = N1 + 27 * N2


@pytest.fixture(scope="module")
def L():
    fbuild.build()
    return fpo.lib()


def _frames(seed, T=4, depth=4):
    rng = np.random.default_rng(seed)
    out = []
    for f in range(T):
        d, xyz = synth.random_mixed_leaves(rng, depth, p_split=0.5, p_empty=0.3)
        out.append((d, xyz, rng.normal(size=(d.shape[0], 28)).astype(np.float32)))
    return out


def _sorted(depth, xyz, vals):
    keys = [(int(d), *map(int, c)) for d, c in zip(depth, xyz)]
    order = sorted(range(len(keys)), key=lambda i: keys[i])
    return [keys[i] for i in order], vals[:, order]


def test_union_hand_example(L):
    # frame A: one depth-1 leaf at the origin octant; frame B: one depth-2
    # leaf in its corner.  A's leaf is divided into 8 depth-2 union leaves
    # carrying A's value; B's value sits in one of them, zeros elsewhere.
    va, vb = np.full((1, 28), 2.0, np.float32), np.full((1, 28), 5.0, np.float32)
    frames = [(np.array([1], np.uint8), np.array([[0, 0, 0]], np.uint32), va),
              (np.array([2], np.uint8), np.array([[1, 1, 1]], np.uint32), vb)]
    depth, xyz, vals = fpo.union_trees(frames, 2)
    assert list(depth) == [2] * 8
    assert sorted(map(tuple, xyz.tolist())) == [(x, y, z) for x in (0, 1) for y in (0, 1) for z in (0, 1)]
    assert np.all(vals[0] == 2.0)
    b_rows = [i for i, c in enumerate(xyz.tolist()) if c == [1, 1, 1]]
    assert np.all(vals[1, b_rows] == 5.0) and np.count_nonzero(vals[1]) == 28


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_union_matches_oracle(L, seed):
    frames = _frames(seed)
    a = _sorted(*fpo.union_trees(frames, 4))
    b = _sorted(*ounion.union_trees(frames))
    assert a[0] == b[0]
    np.testing.assert_array_equal(a[1], b[1])


def test_union_rejects_overlapping_frame(L):
    bad = [(np.array([1, 2], np.uint8), np.array([[0, 0, 0], [1, 1, 1]], np.uint32),
            np.zeros((2, 28), np.float32))]
    with pytest.raises(fpo.FPOError) as e:
        fpo.union_trees(bad, 2)
    assert e.value.code == -4


def _dc_coeffs(values):
    """Coefficients whose IDFT is constant in t: sigma and every z from `values`."""
    co = np.zeros((values.shape[0], NCOEF), np.float32)
    co[:, 0] = values[:, 0]
    co[:, N1::N2] = values[:, 1:]
    return co


def test_union_parent_copy_keeps_every_frame_image():
    # oracle pin of the union: each frame rendered from its own octree equals
    # the frame rendered from the union octree with that frame's values
    frames = _frames(7, T=3)
    for f in frames:
        f[2][:, 0] = np.abs(f[2][:, 0]) * 3
    depth, xyz, vals = ounion.union_trees(frames)
    cam = synth.Camera(eye=synth.sphere_eye(35, 25), width=24, height=24)
    ut = oracle.OracleTree(depth, xyz, 4)
    for f, (d, x, v) in enumerate(frames):
        own = oracle.render(oracle.OracleTree(d, x, 4), _dc_coeffs(v), camera=cam, stop_T=0.0)
        uni = oracle.render(ut, _dc_coeffs(vals[f]), camera=cam, stop_T=0.0)
        np.testing.assert_allclose(uni["rgb"], own["rgb"], atol=1e-12)


# --------------------------------------------------------------------------
# GPU: Eq. 10-12 and the whole chain


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    return torch


@pytest.mark.gpu
@pytest.mark.parametrize("n1,n2,T,n", [(31, 5, 60, 3000), (11, 5, 37, 70), (31, 11, 60, 500), (21, 5, 8, 32)])
def test_dft_leaves_matches_oracle(n1, n2, T, n):
    # (n1, 5): the tiled kernel (full and partial leaf tiles and frame chunks);
    # other n2: the one-thread-per-coefficient kernel
    torch = _cuda()
    rng = np.random.default_rng(n)
    vals = rng.normal(size=(T, n, 28)).astype(np.float32)
    got = fpo.dft_leaves(torch.as_tensor(vals, device="cuda"), n1, n2).cpu().numpy()
    k_sig = oracle.dft(vals[:, :, 0].astype(np.float64), n1)  # [n, n1]
    k_z = oracle.dft(vals[:, :, 1:].reshape(T, -1).astype(np.float64), n2).reshape(n, 27 * n2)
    ref = np.concatenate([k_sig, k_z], axis=1)
    assert np.abs(got - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


@pytest.mark.gpu
@pytest.mark.parametrize("n1,T,n", [(31, 60, 3000), (31, 37, 70), (11, 256, 100), (31, 5, 1)])
def test_dft_bulk_copy_and_tiled_kernels_agree(n1, T, n):
    # a 16-byte aligned values array takes the bulk-copy kernel, one shifted
    # by a float the tiled kernel: same lanes, same summation order
    torch = _cuda()
    rng = np.random.default_rng(T + n)
    vals = torch.as_tensor(rng.normal(size=(T, n, 28)).astype(np.float32), device="cuda")
    shifted = torch.empty(T * n * 28 + 1, device="cuda")
    shifted[1:] = vals.flatten()
    mis = shifted[1:].view(T, n, 28)
    assert vals.data_ptr() % 16 == 0 and mis.data_ptr() % 16 != 0
    a = fpo.dft_leaves(vals, n1, 5)
    b = fpo.dft_leaves(mis, n1, 5)
    whole = torch.full((n + 3, n1 + 135), float("nan"), device="cuda")
    fpo.dft_leaves(vals, n1, 5, out=whole[2:n + 2])  # into rows of a larger array
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(whole[2:n + 2], a)
    assert whole[:2].isnan().all() and whole[n + 2:].isnan().all()
    k_sig = oracle.dft(vals[:, :, 0].double().cpu().numpy(), n1)
    k_z = oracle.dft(vals[:, :, 1:].reshape(T, -1).double().cpu().numpy(), 5).reshape(n, 135)
    ref = np.concatenate([k_sig, k_z], axis=1)
    assert np.abs(a.cpu().numpy() - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


@pytest.mark.gpu
def test_dft_full_chunk_sampled_leaves():
    # a generation-sized chunk (256K leaves x 60 frames: 1.8 GB of values, far
    # more than L2) through the bulk-copy kernel; 64 leaves spread over it,
    # the first and the last included, against the FP64 DFT
    torch = _cuda()
    T, n = 60, 1 << 18
    g = torch.Generator(device="cuda").manual_seed(3)
    vals = torch.randn((T, n, 28), generator=g, device="cuda")
    got = fpo.dft_leaves(vals)
    pick = np.unique(np.concatenate([[0, n - 1], np.random.default_rng(3).integers(0, n, 62)]))
    x = vals[:, torch.as_tensor(pick, device="cuda"), :].double().cpu().numpy()  # [T, m, 28]
    m = len(pick)
    ref = np.concatenate([oracle.dft(x[:, :, 0], 31), oracle.dft(x[:, :, 1:].reshape(T, -1), 5).reshape(m, 135)], 1)
    g_np = got[torch.as_tensor(pick, device="cuda")].double().cpu().numpy()
    assert np.abs(g_np - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


@pytest.mark.gpu
def test_dft_copy_wait_timeout_is_reported():
    # every CTA's first wait runs on a barrier nothing signals (1 ms): the
    # status word gets the time-out bit, every coefficient is NaN, the copies
    # in flight are drained, and the next call on the same device is exact
    torch = _cuda()
    rng = np.random.default_rng(9)
    T, n = 60, 5000
    vals = torch.as_tensor(rng.normal(size=(T, n, 28)).astype(np.float32), device="cuda")
    good = fpo.dft_leaves(vals)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros((n, 166), device="cuda")
    fpo.dft_leaves(vals, out=out, status=st, test_timeout=True)
    torch.cuda.synchronize()
    assert int(st.item()) == fpo.DFT_STATUS_DEVICE_TIMEOUT
    assert out.isnan().all()
    with pytest.raises(fpo.FPOError) as e:
        fpo.dft_leaves(vals, test_timeout=True)
    assert e.value.code == -9
    again = fpo.dft_leaves(vals)
    assert torch.equal(again, good)


@pytest.mark.gpu
def test_generation_chain_reproduces_frames():
    # per-leaf values that are band-limited in time (frequency <= 2 for z,
    # <= 15 for sigma) go through union -> DFT -> IDFT exactly, so a frame
    # rendered from the Fourier PlenOctree equals its own octree rendered
    torch = _cuda()
    rng = np.random.default_rng(5)
    T = 60
    d, xyz = synth.random_mixed_leaves(rng, 4, p_split=0.5, p_empty=0.3)
    n = d.shape[0]
    t = np.arange(1, T + 1)[:, None]
    frames = []
    phase = rng.uniform(0, 2 * np.pi, (n, 28))
    amp = rng.uniform(0.1, 0.5, (n, 28))
    base = np.concatenate([rng.uniform(5, 20, (n, 1)), rng.normal(size=(n, 27))], axis=1)
    for f in range(T):
        freq = np.concatenate([np.full((n, 1), 7.0), np.full((n, 27), 2.0)], axis=1)
        v = base + amp * np.sin(2 * np.pi * freq * (f + 1) / T + phase)
        frames.append((d, xyz, v.astype(np.float32)))
    ud, uxyz, uvals = fpo.union_trees(frames, 4)
    assert ud.shape[0] == n  # identical structures: the union is the frame tree
    coeffs = fpo.dft_leaves(torch.as_tensor(uvals, device="cuda"), N1, N2).cpu().numpy()
    tree = synth.Tree(ud, uxyz, coeffs, 4)
    cam = synth.Camera(eye=synth.sphere_eye(20, 30), width=32, height=32)
    r = fpo.Renderer()
    r.upload(tree)
    for f in (1, 17, 60):
        img = r.render(camera=cam, t=float(f), stop_T=0.0)["rgb"].cpu().numpy()
        own = oracle.render(oracle.OracleTree(ud, uxyz, 4), _dc_coeffs(uvals[f - 1]), camera=cam,
                            stop_T=0.0)["rgb"]
        assert np.abs(img - own).max() < 2e-4
    r.status()
    r.close()
