"""Training kernels of the latent decoder (fpo_decoder_grad, fpo_adam)
against the FP64 reference, the LATENT storage render path, and a small
training run on coefficients produced by the Fourier PlenOctree generation
(smooth animated fields -> per-leaf DFT)."""

import ctypes as C

import numpy as np
import pytest

import gpu_util as gu
from oracle import latent as olat
from paper_2202_08614_gb300 import fpo, synth
from paper_2202_08614_gb300.latent import LatentModel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

N1, N2 = 31, 5
NC = N1 + 27 * N2


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def test_decoder_grad_matches_reference():
    rng = np.random.default_rng(0)
    n, b = 2000, 333
    m = LatentModel(n, seed=1)
    m.p["b1"].copy_(torch.as_tensor(rng.normal(size=64) * 0.1))
    m.p["b3"].copy_(torch.as_tensor(rng.normal(size=NC)))
    tgt = torch.as_tensor(rng.normal(size=(n, NC)), dtype=torch.float32, device="cuda")
    cw = torch.as_tensor(rng.uniform(0.5, 2, NC), dtype=torch.float32, device="cuda")
    extra = torch.as_tensor(rng.normal(size=(n, NC)) * 0.01, dtype=torch.float32, device="cuda")
    rows = torch.as_tensor(rng.permutation(n)[:b], dtype=torch.int32, device="cuda")
    dl, loss = m.grad(rows, tgt, cw, extra_dy=extra)
    torch.cuda.synchronize()
    P = {k: v.double().cpu().numpy() for k, v in m.p.items()}
    r = rows.cpu().numpy()
    L, dx, g = olat.loss_grad(P["lat"][r], P["w1"], P["b1"], P["w2"], P["b2"], P["w3"], P["b3"],
                              tgt.double().cpu().numpy()[r], cw.double().cpu().numpy())
    # the extra dL/dy enters like the L2 term's 2 cw (y - t)
    Lx, dxx, gx = olat.loss_grad(P["lat"][r], P["w1"], P["b1"], P["w2"], P["b2"], P["w3"], P["b3"],
                                 np.zeros((b, NC)), np.ones(NC))
    y = olat.decode(P["lat"][r], P["w1"], P["b1"], P["w2"], P["b2"], P["w3"], P["b3"])
    e = extra.double().cpu().numpy()[r]
    assert abs(loss.item() - L) <= 1e-4 * L
    # linear term: gradients of sum(e . y) = back-propagate dy = e
    _, dxe, ge = _backprop_dy(P, r, e)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(dl.double().cpu().numpy(), dx + dxe) <= 1e-4
    for k in ("w1", "b1", "w2", "b2", "w3", "b3"):
        assert rel(m.g[k].double().cpu().numpy(), g[k] + ge[k]) <= 1e-4, k


def _backprop_dy(P, r, dy):
    x = P["lat"][r]
    z1 = x @ P["w1"].T + P["b1"]
    h1 = np.maximum(z1, 0)
    z2 = h1 @ P["w2"].T + P["b2"]
    h2 = np.maximum(z2, 0)
    g = {"w3": dy.T @ h2, "b3": dy.sum(0)}
    d2 = (dy @ P["w3"]) * (z2 > 0)
    g["w2"], g["b2"] = d2.T @ h1, d2.sum(0)
    d1 = (d2 @ P["w2"]) * (z1 > 0)
    g["w1"], g["b1"] = d1.T @ x, d1.sum(0)
    return None, d1 @ P["w1"], g


def test_adam_dense_and_rows():
    rng = np.random.default_rng(2)
    p0 = rng.normal(size=(50, 8)).astype(np.float32)
    dev = lambda a: torch.as_tensor(np.asarray(a, np.float32), device="cuda")
    p, m, v = dev(p0), dev(np.zeros_like(p0)), dev(np.zeros_like(p0))
    pr, mr, vr = p0.astype(np.float64), np.zeros_like(p0, np.float64), np.zeros_like(p0, np.float64)
    for step in (1, 2, 3):
        g = rng.normal(size=p0.shape).astype(np.float32)
        gd = dev(g)  # kept alive until the kernel has run
        fpo.check(fpo.lib().fpo_adam(C.c_void_p(p.data_ptr()), C.c_void_p(gd.data_ptr()),
                                     C.c_void_p(m.data_ptr()), C.c_void_p(v.data_ptr()), p0.size, None,
                                     0, 0.01, 0.9, 0.999, 1e-8, step, None))
        torch.cuda.synchronize()
        mr = 0.9 * mr + 0.1 * g
        vr = 0.999 * vr + 0.001 * g * g
        pr -= 0.01 * (mr / (1 - 0.9 ** step)) / (np.sqrt(vr / (1 - 0.999 ** step)) + 1e-8)
    np.testing.assert_allclose(p.cpu().numpy(), pr, atol=1e-5)
    rows = np.array([3, 17, 40], np.int32)
    q = dev(p0)
    g = rng.normal(size=(3, 8)).astype(np.float32)
    mq, vq = dev(np.zeros_like(p0)), dev(np.zeros_like(p0))
    gd, rd = dev(g), torch.as_tensor(rows, device="cuda")
    fpo.check(fpo.lib().fpo_adam(C.c_void_p(q.data_ptr()), C.c_void_p(gd.data_ptr()),
                                 C.c_void_p(mq.data_ptr()), C.c_void_p(vq.data_ptr()), 24,
                                 C.c_void_p(rd.data_ptr()), 8, 0.01, 0.9, 0.999, 1e-8, 1, None))
    torch.cuda.synchronize()
    qn = q.cpu().numpy()
    untouched = np.setdiff1d(np.arange(50), rows)
    assert np.array_equal(qn[untouched], p0[untouched])
    np.testing.assert_allclose(qn[rows], p0[rows] - 0.01 * np.sign(g), atol=1e-5)


def _smooth_tree(depth=6, seed=0):
    rng = np.random.default_rng(seed)
    body = synth.capsule_body(rng)
    xyz = synth.capsule_union_leaves(*body, depth=depth)
    d = np.full(xyz.shape[0], depth, np.uint8)
    vals = synth.smooth_frame_values(d, xyz, body)
    coeffs = fpo.dft_leaves(vals, N1, N2)
    return d, xyz, coeffs


def test_latent_storage_render_matches_decoded_coefficients():
    d, xyz, _ = _smooth_tree(5)
    n = d.shape[0]
    m = LatentModel(n, seed=3)
    m.p["b3"][0] = 30.0
    lat, w1, b1, w2, b2, w3, b3 = m.inference_arrays()
    # what the tensor-core decoder sees: FP16 latents, BF16 weights
    P = [x.double().cpu().numpy() for x in (lat.float(), w1.bfloat16().float(), b1, w2.bfloat16().float(),
                                             b2, w3.bfloat16().float(), b3)]
    co = olat.decode(*P).astype(np.float32)
    tree = synth.Tree(d, xyz, co, 5)
    cam = synth.Camera(eye=synth.sphere_eye(60, 15), width=64, height=48)
    r = fpo.Renderer(storage="latent")
    r.upload(synth.Tree(d, xyz, np.zeros((0, NC), np.float32), 5))
    r.set_latents(lat, w1, b1, w2, b2, w3, b3)
    img = r.render(camera=cam, t=21.0)["rgb"].cpu().numpy()
    r.status()
    r.close()
    ref = gu.oracle.render(gu.oracle_tree(tree), co, camera=cam, t=21.0)["rgb"]
    assert np.abs(img - ref).max() < 2e-2  # FP16 activations in the decoder
    assert np.mean((img - ref) ** 2) < 1e-5


def test_training_fits_generated_coefficients():
    d, xyz, coeffs = _smooth_tree(6)
    n = d.shape[0]
    m = LatentModel(n, seed=0)
    m.init_output_bias(coeffs)
    hist = m.fit(coeffs, steps=1500, batch=8192, lr_w=2e-3, lr_lat=2e-2, log_every=500)
    print("training loss", hist)
    assert hist[-1][1] < 0.05 * hist[0][1]
    lat, *w = m.inference_arrays()
    r = fpo.Renderer(storage="latent")
    r.upload(synth.Tree(d, xyz, np.zeros((0, NC), np.float32), 6))
    r.set_latents(lat, *w)
    cam = synth.ring_cameras(16, 96, 64)[3]
    img = r.render(camera=cam, t=17.0)["rgb"].cpu().numpy()
    r.status()
    r.close()
    ref = gu.oracle.render(gu.oracle_tree(synth.Tree(d, xyz, coeffs.cpu().numpy(), 6)),
                           coeffs.cpu().numpy(), camera=cam, t=17.0)["rgb"]
    psnr = 10 * np.log10(1.0 / np.mean((img - ref) ** 2))
    print(f"latent render PSNR vs FP64 oracle of the generated FPO: {psnr:.2f} dB")
    assert psnr > 25.0


def test_decoder_timeout_is_reported_and_the_context_stays_usable():
    # the tensor-core decoder's failure path: each warpgroup's first wait for
    # its MMAs (on a barrier nothing signals) runs out after 1 ms; the group
    # waits for the MMAs it committed before TMEM is freed, the call reports
    # FPO_ERR_DEVICE_TIMEOUT, and the context then renders normally
    d, xyz, _ = _smooth_tree(5)
    n = d.shape[0]
    m = LatentModel(n, seed=3)
    m.p["b3"][0] = 30.0
    cam = synth.Camera(eye=synth.sphere_eye(60, 15), width=64, height=48)
    r = fpo.Renderer(storage="latent")
    try:
        r.upload(synth.Tree(d, xyz, np.zeros((0, NC), np.float32), 5))
        r.set_latents(*m.inference_arrays())
        ref = r.render(camera=cam, t=21.0)["rgb"].clone()
        r.status()
        r.render(camera=cam, t=21.0, test_timeout=True)
        with pytest.raises(fpo.FPOError) as e:
            r.status()
        assert e.value.code == -9
        r.status()
        again = r.render(camera=cam, t=21.0)["rgb"]
        r.status()
        assert torch.equal(again, ref)
    finally:
        r.close()


def test_decoder_forward_matches_reference():
    # fpo_decoder_forward (FP32 SIMT decode of every leaf) against the FP64
    # reference, element by element; 3001 leaves: a ragged last tile
    rng = np.random.default_rng(4)
    n = 3001
    m = LatentModel(n, seed=9)
    m.p["b1"].copy_(torch.as_tensor(rng.normal(size=64) * 0.1))
    m.p["b2"].copy_(torch.as_tensor(rng.normal(size=64) * 0.1))
    m.p["b3"].copy_(torch.as_tensor(rng.normal(size=NC)))
    y = m.decode().double().cpu().numpy()
    P = {k: v.double().cpu().numpy() for k, v in m.p.items()}
    ref = olat.decode(P["lat"], P["w1"], P["b1"], P["w2"], P["b2"], P["w3"], P["b3"])
    # FP32 sums of at most 64 products: a few ulp of the largest partial sums
    np.testing.assert_allclose(y, ref, rtol=0, atol=2e-5 * max(1.0, np.abs(ref).max()))


def test_set_coeffs_from_decoder_equals_decode_then_set_coeffs():
    # the fused decode into the context's records writes what
    # fpo_decoder_forward + fpo_set_coeffs write: renders are bit-equal; the
    # decoded values themselves match the FP64 reference (a ragged last tile)
    rng = np.random.default_rng(6)
    d, xyz, _ = _smooth_tree(5)
    n = d.shape[0]
    m = LatentModel(n, seed=11)
    m.p["b1"].copy_(torch.as_tensor(rng.normal(size=64) * 0.1))
    m.p["b3"].copy_(torch.as_tensor(rng.normal(size=NC)))
    m.p["b3"][0] = 30.0
    empty = synth.Tree(d, xyz, np.zeros((n, NC), np.float32), 5)
    a, b = fpo.Renderer(idft_mode="fused"), fpo.Renderer(idft_mode="fused")
    try:
        a.upload(empty)
        b.upload(empty)
        dec = m.decode()
        a.set_coeffs(dec)
        b.set_coeffs_from_decoder(m._mlp(m.p), m.p["lat"])
        cam = synth.Camera(eye=synth.sphere_eye(75, 25), width=64, height=48)
        ia = a.render(camera=cam, t=13.0)["rgb"]
        ib = b.render(camera=cam, t=13.0)["rgb"]
        a.status()
        b.status()
        assert torch.equal(ia, ib)
        P = {k: v.double().cpu().numpy() for k, v in m.p.items()}
        ref = olat.decode(P["lat"], P["w1"], P["b1"], P["w2"], P["b2"], P["w3"], P["b3"])
        assert n % 64 != 0  # a ragged last tile
        np.testing.assert_allclose(dec.double().cpu().numpy(), ref, rtol=0, atol=2e-5 * np.abs(ref).max())
        with pytest.raises(AssertionError):
            b.set_coeffs_from_decoder(m._mlp(m.p), m.p["lat"].half())
        with pytest.raises(fpo.FPOError) as e:
            fpo.check(fpo.lib().fpo_set_coeffs_from_decoder(b.h, C.byref(m._mlp(m.p)), None, 0, None))
        assert e.value.code == -1
    finally:
        a.close()
        b.close()
    c = fpo.Renderer(storage="bf16")
    try:
        c.upload(empty)
        with pytest.raises(fpo.FPOError) as e:
            c.set_coeffs_from_decoder(m._mlp(m.p), m.p["lat"])
        assert e.value.code == -8
    finally:
        c.close()


def _bf16(a):
    """Round-to-nearest-even to BF16, as FP64 (host)."""
    x = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    x = (x + 0x7FFF + ((x >> 16) & 1)) & 0xFFFF0000
    return x.astype(np.uint32).view(np.float32).astype(np.float64)


def _tc_emulation(P, r, tgt, cw, extra):
    """The tensor-core step in FP64 with BF16 operands where the kernel rounds
    them: latents, weights, hidden activations, dL/dy, d2, d1 (biases exact)."""
    x = _bf16(P["lat"][r])
    w1, w2, w3 = _bf16(P["w1"]), _bf16(P["w2"]), _bf16(P["w3"])
    z1 = x @ w1.T + P["b1"]
    h1 = _bf16(np.maximum(z1, 0))
    z2 = h1 @ w2.T + P["b2"]
    h2 = _bf16(np.maximum(z2, 0))
    y = h2 @ w3.T + P["b3"]
    e = y - tgt[r]
    L = float((cw * e * e).sum())
    dy = _bf16(2 * cw * e + (extra[r] if extra is not None else 0))
    d2 = _bf16((dy @ w3) * (z2 > 0))
    d1 = _bf16((d2 @ w2) * (z1 > 0))
    g = {"w3": dy.T @ h2, "b3": dy.sum(0), "w2": d2.T @ h1, "b2": d2.sum(0), "w1": d1.T @ x, "b1": d1.sum(0),
         "dx": d1 @ w1}
    # sum of |terms| of every element: a BF16 operand that rounds the other way
    # (its FP32 sum landed on the other side of a rounding point) moves an
    # element by about 2^-8 of the terms it enters
    a = np.abs
    terms = {"w3": a(dy).T @ a(h2), "b3": a(dy).sum(0), "w2": a(d2).T @ a(h1), "b2": a(d2).sum(0),
             "w1": a(d1).T @ a(x), "b1": a(d1).sum(0), "dx": a(d1) @ a(w1)}
    return L, g, terms


@pytest.mark.parametrize("b", [1, 333, 20000])
def test_decoder_grad_tensor_cores(b):
    # fpo_decoder_grad_tc against an FP64 reference that rounds the operands
    # to BF16 where the kernel does (element-wise, within 2^-6 of the element's
    # sum of |terms|: FP32 accumulation order, and the odd BF16 rounding that
    # goes the other way, compounded over the layers), and against the FP64
    # gradient itself (the BF16 operand error)
    rng = np.random.default_rng(b)
    n = max(2000, b + 10)
    m = LatentModel(n, seed=2, tensor_cores=True)
    m.p["b1"].copy_(torch.as_tensor(rng.normal(size=64) * 0.1))
    m.p["b2"].copy_(torch.as_tensor(rng.normal(size=64) * 0.1))
    m.p["b3"].copy_(torch.as_tensor(rng.normal(size=NC)))
    tgt = torch.as_tensor(rng.normal(size=(n, NC)), dtype=torch.float32, device="cuda")
    cw = torch.as_tensor(rng.uniform(0.5, 2, NC), dtype=torch.float32, device="cuda")
    extra = torch.as_tensor(rng.normal(size=(n, NC)) * 0.01, dtype=torch.float32, device="cuda")
    rows = torch.as_tensor(rng.permutation(n)[:b], dtype=torch.int32, device="cuda")
    dl, loss = m.grad(rows, tgt, cw, extra_dy=extra)
    m.check_status()
    P = {k: v.double().cpu().numpy() for k, v in m.p.items()}
    r = rows.cpu().numpy()
    T, CW, E = tgt.double().cpu().numpy(), cw.double().cpu().numpy(), extra.double().cpu().numpy()
    L, g, terms = _tc_emulation(P, r, T, CW, E)
    got = {k: v.double().cpu().numpy() for k, v in m.g.items()}
    got["dx"] = dl.double().cpu().numpy()
    assert abs(loss.item() - L) <= 1e-3 * L
    for k in ("w1", "b1", "w2", "b2", "w3", "b3", "dx"):
        excess = np.abs(got[k] - g[k]) - (2.0 ** -6 * terms[k] + 1e-6 * np.abs(g[k]).max())
        assert excess.max() <= 0, (k, excess.max())
    # against the FP64 gradient: BF16 operands (and the ReLU masks they flip)
    # move every matrix by a few 2^-8; the kernel is no further from it than
    # exact arithmetic on the same BF16 operands is
    L64, dx64, g64 = olat.loss_grad(P["lat"][r], P["w1"], P["b1"], P["w2"], P["b2"], P["w3"], P["b3"],
                                    T[r], CW)
    _, dxe, ge = _backprop_dy(P, r, E[r])
    g64 = {k: g64[k] + ge[k] for k in ge}
    g64["dx"] = dx64 + dxe
    for k in ("w1", "b1", "w2", "b2", "w3", "b3", "dx"):
        nrm = np.linalg.norm(g64[k])
        rel_gpu, rel_emu = np.linalg.norm(got[k] - g64[k]) / nrm, np.linalg.norm(g[k] - g64[k]) / nrm
        print(f"{k}: |tc - fp64| / |fp64| = {rel_gpu:.2e} (BF16 emulation {rel_emu:.2e})")
        assert rel_emu <= 0.1 and rel_gpu <= 1.05 * rel_emu + 1e-3, (k, rel_gpu, rel_emu)


def test_decoder_grad_tensor_cores_timeout_is_reported():
    # each CTA's first wait (on a barrier nothing signals) runs out after 1 ms:
    # the status word gets the time-out bit, the weight gradients stay as they
    # were, and the next call is exact
    rng = np.random.default_rng(5)
    n, b = 3000, 1000
    m = LatentModel(n, seed=4, tensor_cores=True)
    tgt = torch.as_tensor(rng.normal(size=(n, NC)), dtype=torch.float32, device="cuda")
    cw = torch.ones(NC, device="cuda")
    rows = torch.as_tensor(rng.permutation(n)[:b], dtype=torch.int32, device="cuda")
    ref_dl, _ = m.grad(rows, tgt, cw)
    ref_g = {k: v.clone() for k, v in m.g.items()}
    m.check_status()
    for v in m.g.values():
        v.zero_()
    dl = torch.empty((b, 32), device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    w, g = m._mlp(m.p), m._mlp(m.g)
    fpo.check(fpo.lib().fpo_decoder_grad_tc(
        C.byref(w), N1, N2, b, C.c_void_p(rows.data_ptr()), C.c_void_p(m.p["lat"].data_ptr()),
        C.c_void_p(tgt.data_ptr()), C.c_void_p(cw.data_ptr()), None, C.byref(g), C.c_void_p(dl.data_ptr()),
        C.c_void_p(loss.data_ptr()), C.c_void_p(m.status.data_ptr()), fpo.FLAG_TEST_DEVICE_TIMEOUT, None))
    with pytest.raises(fpo.FPOError) as e:
        m.check_status()
    assert e.value.code == -9
    assert all(int(torch.count_nonzero(v)) == 0 for v in m.g.values())
    m.status.zero_()
    dl2, _ = m.grad(rows, tgt, cw)
    m.check_status()
    assert torch.equal(dl2, ref_dl)
    for k in ref_g:  # float atomics: the sums' order may differ between runs
        assert torch.allclose(m.g[k], ref_g[k], rtol=1e-5, atol=1e-6 * float(ref_g[k].abs().max()))


def _f16(a):
    return np.asarray(a, np.float64).astype(np.float16).astype(np.float64)


def test_decode_into_records_on_the_tensor_cores():
    # fpo_set_coeffs_from_decoder(FPO_FLAG_TENSOR_CORES) against an FP64 decode
    # with the kernel's roundings (FP16 latents, weights through BF16 to FP16,
    # FP16 hidden activations; exact biases): both coefficient sets rendered
    # through the fused per-visit IDFT agree to FP32 accumulation order and
    # the odd FP16 rounding that goes the other way; against the FP32 decode
    # they differ by the FP16 operands
    rng = np.random.default_rng(8)
    d, xyz, _ = _smooth_tree(5)
    n = d.shape[0]
    m = LatentModel(n, seed=12)
    m.p["b1"].copy_(torch.as_tensor(rng.normal(size=64) * 0.1))
    m.p["b3"].copy_(torch.as_tensor(rng.normal(size=NC)))
    m.p["b3"][0] = 30.0
    P = {k: v.double().cpu().numpy() for k, v in m.p.items()}
    wq = {k: _f16(_bf16(P[k])) for k in ("w1", "w2", "w3")}
    z1 = _f16(P["lat"]) @ wq["w1"].T + P["b1"]
    z2 = _f16(np.maximum(z1, 0)) @ wq["w2"].T + P["b2"]
    emu = _f16(np.maximum(z2, 0)) @ wq["w3"].T + P["b3"]
    empty = synth.Tree(d, xyz, np.zeros((n, NC), np.float32), 5)
    cams = [synth.Camera(eye=synth.sphere_eye(a, 20), width=64, height=48) for a in (15, 135, 255)]
    rs = [fpo.Renderer(idft_mode="fused") for _ in range(3)]
    try:
        for r in rs:
            r.upload(empty)
        rs[0].set_coeffs_from_decoder(m._mlp(m.p), m.p["lat"], tensor_cores=True)
        rs[1].set_coeffs(torch.as_tensor(emu, dtype=torch.float32, device="cuda"))
        rs[2].set_coeffs_from_decoder(m._mlp(m.p), m.p["lat"])
        for cam in cams:
            img = [r.render(camera=cam, t=27.0)["rgb"].double().cpu().numpy() for r in rs]
            for r in rs:
                r.status()
            assert np.abs(img[0] - img[1]).max() <= 1e-4
            assert np.abs(img[0] - img[2]).max() <= 2e-2 and np.mean((img[0] - img[2]) ** 2) <= 1e-5
        # the failure path: every group's first wait runs out (1 ms)
        rs[0].set_coeffs_from_decoder(m._mlp(m.p), m.p["lat"], tensor_cores=True, test_timeout=True)
        with pytest.raises(fpo.FPOError) as e:
            rs[0].status()
        assert e.value.code == -9
        # an operand beyond the FP16 range is reported
        big = {k: v.clone() for k, v in m.p.items()}
        big["w2"][3, 5] = 1.0e6
        rs[0].set_coeffs_from_decoder(m._mlp(big), m.p["lat"], tensor_cores=True)
        with pytest.raises(fpo.FPOError) as e:
            rs[0].status()
        assert e.value.code == -10
        rs[0].set_coeffs_from_decoder(m._mlp(m.p), m.p["lat"], tensor_cores=True)
        again = rs[0].render(camera=cams[0], t=27.0)["rgb"].double().cpu().numpy()
        rs[0].status()
        ref = rs[1].render(camera=cams[0], t=27.0)["rgb"].double().cpu().numpy()
        assert np.abs(again - ref).max() <= 1e-4
    finally:
        for r in rs:
            r.close()
