"""Reduced-precision coefficient storage (BF16, FP16, FP8-E4M3 with a per-leaf
FP32 scale); the IDFT, SH and compositing stay FP32, the per-frame table is
FP16 with these storages unless FP32 is asked for.

1. Encoding: storing coefficients in format X must give exactly the image of
   the FP32 renderer fed with the coefficients rounded to X by torch / numpy
   (round to nearest even), so the library's encoders agree with those
   library conversions code for code.
2. Error against the FP64 oracle (on the original FP32 coefficients), as PSNR:
   BF16 and FP16 at >= 45 dB; FP8 is reported with a looser floor.
"""

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


def _round(coeffs: np.ndarray, storage: str) -> np.ndarray:
    """What the library should store, decoded back to FP32, via torch/numpy."""
    c = torch.from_numpy(coeffs.copy())
    if storage == "bf16":
        return c.to(torch.bfloat16).to(torch.float32).numpy()
    if storage == "f16":
        return coeffs.astype(np.float16).astype(np.float32)
    if storage == "fp8":
        mx = np.abs(coeffs).max(axis=1, keepdims=True)
        sc = np.where(mx > 0, mx / np.float32(448.0), np.float32(1.0)).astype(np.float32)
        q = torch.from_numpy((coeffs / sc).astype(np.float32)).to(torch.float8_e4m3fn).to(torch.float32)
        return q.numpy(), sc
    return coeffs


def _render(tree, storage, cam, t, table="auto"):
    r = fpo.Renderer(storage=storage, idft_mode="materialise", table=table)
    try:
        r.upload(tree)
        out = r.render(camera=cam, t=t)["rgb"].cpu().numpy()
        r.status()
        info = r.info()
    finally:
        r.close()
    return out, info


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_16bit_encoding_matches_library_rounding(storage):
    tree = synth.shell_tree()
    cam = synth.shell_camera(64, 64)
    a, info = _render(tree, storage, cam, 17.0, table="f32")  # same table precision as the FP32 render
    rounded = synth.Tree(tree.leaf_depth, tree.leaf_xyz, _round(tree.coeffs, storage), tree.max_depth)
    b, _ = _render(rounded, "f32", cam, 17.0)
    assert np.array_equal(a, b)
    assert info["leaf_record_bytes"] == 336


def test_fp8_encoding_matches_library_rounding():
    tree = synth.shell_tree()
    cam = synth.shell_camera(64, 64)
    a, info = _render(tree, "fp8", cam, 17.0, table="f32")
    q, sc = _round(tree.coeffs, "fp8")
    rounded = synth.Tree(tree.leaf_depth, tree.leaf_xyz, (q * sc).astype(np.float32), tree.max_depth)
    b, _ = _render(rounded, "f32", cam, 17.0)
    # scale applied after the sums instead of to every coefficient: rounding only
    assert np.abs(a - b).max() <= 2e-5
    assert info["leaf_record_bytes"] == 32 + 144 + 4


def _psnr(x, ref):
    mse = np.mean((x.astype(np.float64) - ref) ** 2)
    return float("inf") if mse == 0 else 10 * np.log10(1.0 / mse)


@pytest.mark.parametrize("storage,floor", [("bf16", 45.0), ("f16", 45.0), ("fp8", 25.0), ("f32", 80.0)])
def test_psnr_against_fp64_oracle_shell(storage, floor):
    tree = synth.shell_tree()
    cam = synth.shell_camera()
    gpu, _ = _render(tree, storage, cam, synth.SHELL_T)
    ref = gu.oracle.render(gu.oracle_tree(tree), tree.coeffs, camera=cam, t=synth.SHELL_T)["rgb"]
    p = _psnr(gpu, ref)
    print(f"{storage}: PSNR {p:.2f} dB, max|d| {np.abs(gpu - ref).max():.2e}")
    assert p >= floor


def test_fused_mode_needs_fp32_records():
    tree = synth.shell_tree()
    r = fpo.Renderer(storage="bf16", idft_mode="fused")
    try:
        r.upload(tree)
        with pytest.raises(fpo.FPOError) as e:
            r.render(camera=synth.shell_camera(8, 8))
        assert e.value.code == -8
    finally:
        r.close()


@pytest.mark.parametrize("storage,floor", [("bf16", 45.0), ("f16", 45.0)])
def test_psnr_body_1080p_sampled(storage, floor):
    tree = synth.body_tree()
    ot = gu.oracle_tree(tree)
    cam = synth.ring_cameras(16, 1920, 1080)[4]
    gpu, _ = _render(tree, storage, cam, 33.0)
    rng = np.random.default_rng(4)
    sel = np.concatenate([rng.integers(0, 1920 * 1080, 4000), 540 * 1920 + np.arange(0, 1920, 2)])
    ref = gu.oracle.render(ot, tree.coeffs, camera=cam, t=33.0, sel=sel)["rgb"]
    assert _psnr(gpu[sel], ref) >= floor


@pytest.mark.parametrize("storage", ["f32", "bf16", "fp8"])
def test_fp16_table_against_fp32_table(storage):
    # the FP16 table rounds sigma(t) and z(t) to 11 significant bits: a few
    # 1e-4 in RGB on the shell (cells 1/32 wide, sigma up to ~60)
    tree = synth.shell_tree()
    cam = synth.shell_camera()
    a, info16 = _render(tree, storage, cam, synth.SHELL_T, table="f16")
    b, info32 = _render(tree, storage, cam, synth.SHELL_T, table="f32")
    d = np.abs(a - b)
    print(f"{storage}: FP16 vs FP32 table max|d| {d.max():.2e}, mean {d.mean():.2e}")
    assert d.max() <= 5e-3 and d.mean() <= 1e-4
    assert info16["table_bytes"] * 2 == info32["table_bytes"] == tree.n_leaves * 128
    ref = gu.oracle.render(gu.oracle_tree(tree), tree.coeffs, camera=cam, t=synth.SHELL_T)["rgb"]
    pa, pb = _psnr(a, ref), _psnr(b, ref)
    print(f"{storage}: PSNR vs FP64 oracle {pa:.2f} dB (FP16 table), {pb:.2f} dB (FP32 table)")
    assert pa >= min(60.0, pb - 1.0)
