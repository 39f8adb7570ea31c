"""What the learned part gains, on a generated body: the latent decoder is
trained by the library's own kernels (coefficient L2 plus the rendered-pixel
loss through the render adjoint) on the coefficients the Fourier PlenOctree
generation produces for a depth-8 capsule body (smooth animated fields ->
union leaves -> per-leaf DFT), then rendered with LATENT storage.  Gates:
every one of 16 frames (one per ring camera, t = 3.75 k) at PSNR >= 45 dB
against the FP64 oracle of the generated coefficients; a tenth of the bytes
per leaf of the plain FP32 FPO; and more frames per second than the plain
FP32 FPO of the same coefficients through fpo_render_frames."""

import numpy as np
import pytest

import gpu_util as gu
from paper_2202_08614_gb300 import fpo, synth
from paper_2202_08614_gb300.latent import LatentModel, PixelLoss

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

DEPTH = 8
W, H = 384, 216


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _frames_per_s(r, cams, frames, reps=4):
    out = torch.empty((len(frames), W * H, 3), device="cuda")
    args = ([cams[k] for k, _ in frames], [t for _, t in frames])
    r.render_frames(*args, out=out)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        r.render_frames(*args, out=out)
    b.record()
    torch.cuda.synchronize()
    r.status()
    return reps * len(frames) / (a.elapsed_time(b) * 1e-3)


def test_latent_decoder_quality_and_gain_on_a_generated_body():
    body = synth.capsule_body(np.random.default_rng(0))
    xyz = synth.capsule_union_leaves(*body, depth=DEPTH)
    d = np.full(xyz.shape[0], DEPTH, np.uint8)
    n = d.shape[0]
    coeffs = fpo.dft_leaves(synth.smooth_frame_values(d, xyz, body))
    gen = synth.Tree(d, xyz, coeffs.cpu().numpy(), DEPTH)
    cams = synth.ring_cameras(16, W, H)

    m = LatentModel(n, seed=0, tensor_cores=True)
    m.init_output_bias(coeffs)
    pixel = PixelLoss(gen, cams, rays=8192, weight=10.0, every=4, start=0.1, tensor_cores=True)
    try:
        hist = m.fit(coeffs, steps=4000, batch=65536, lr_w=1e-3, lr_lat=1e-1, decay=0.05,
                     coef_weight=m.default_weights(coeffs.device, sigma_weight=0.2),
                     log_every=1000, pixel=pixel)
    finally:
        pixel.close()
    print("training loss", hist)

    lat = fpo.Renderer(storage="latent")
    plain = fpo.Renderer()
    try:
        lat.upload(synth.Tree(d, xyz, np.zeros((0, gen.n_coeffs), np.float32), DEPTH))
        lat.set_latents(*m.inference_arrays())
        plain.upload(gen)
        ot = gu.oracle_tree(gen)
        frames = [(k, 3.75 * k) for k in range(16)]
        db = []
        for k, t in frames:
            img = lat.render(camera=cams[k], t=t)["rgb"].cpu().numpy().astype(np.float64)
            ref = gu.oracle.render(ot, gen.coeffs, camera=cams[k], t=t)["rgb"]
            db.append(10 * np.log10(1.0 / np.mean((img - ref) ** 2)))
        lat.status()
        print("latent PSNR per frame vs the FP64 oracle:", np.round(db, 2))
        assert min(db) >= 45.0

        # storage: one FP16 latent per leaf against the FP32 records
        assert lat.info()["leaf_record_bytes"] == 64 and plain.info()["leaf_record_bytes"] == 672
        # speed: the decoder reads 64 B per leaf where the IDFT pass reads 672 B
        fps_lat = _frames_per_s(lat, cams, frames)
        fps_plain = _frames_per_s(plain, cams, frames)
        print(f"frames/s: latent {fps_lat:.0f}, plain FP32 {fps_plain:.0f}")
        assert fps_lat > 1.05 * fps_plain
    finally:
        lat.close()
        plain.close()
