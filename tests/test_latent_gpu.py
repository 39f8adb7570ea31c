"""Latent decoder on the tensor cores (fpo_latent_table): the per-frame table
decoded from FP16 latents by the BF16 MLP with the IDFT folded into the last
layer, against (a) a numpy emulation that rounds the operands to FP16 where
the kernel does, tightly, and (b) the plain FP64 reference, within the FP16
operand error."""

import numpy as np
import pytest

from oracle import latent as olat
from paper_2202_08614_gb300 import fpo

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


def _net(seed):
    rng = np.random.default_rng(seed)
    bf = lambda a: torch.as_tensor(a, dtype=torch.float32).to(torch.bfloat16).float().numpy()
    w1 = bf(rng.normal(size=(64, 32)) / np.sqrt(32))
    w2 = bf(rng.normal(size=(64, 64)) / np.sqrt(64))
    w3 = bf(rng.normal(size=(NC, 64)) / np.sqrt(64))
    b1 = rng.normal(size=64).astype(np.float32) * 0.1
    b2 = rng.normal(size=64).astype(np.float32) * 0.1
    b3 = rng.normal(size=NC).astype(np.float32) * 0.1
    b3[0] += 5.0  # a positive density on average
    return w1, b1, w2, b2, w3, b3


def _f16(a):
    return np.asarray(a, np.float32).astype(np.float16).astype(np.float64)


def _emulate(lat, w1, b1, w2, b2, w3, b3, t):
    """The kernel's rounding points: FP16 operands, FP32 accumulation."""
    import oracle

    b = oracle.basis(N1, t, 60.0).astype(np.float32).astype(np.float64)
    w3f = np.zeros((32, 64))
    w3f[0] = b[:N1] @ w3[:N1]
    w3f[1:28] = np.einsum("i,qih->qh", b[:N2], w3[N1:].reshape(27, N2, 64))
    b3f = np.zeros(32)
    b3f[0] = b[:N1] @ b3[:N1]
    b3f[1:28] = b3[N1:].reshape(27, N2) @ b[:N2]
    h1 = _f16(np.maximum(_f16(lat) @ _f16(w1).T + b1, 0))
    h2 = _f16(np.maximum(h1 @ _f16(w2).T + b2, 0))
    o = h2 @ _f16(w3f).T + b3f
    o[:, 0] = np.maximum(o[:, 0], 0)
    o[:, 28:] = 0
    return o


def _fp16_bound(lat, w1, b1, w2, b2, w3, b3, t):
    """Element-wise bound on |kernel table - FP64 table| from the FP16
    operands: W3'(t) and each hidden activation are rounded to FP16 (relative
    error <= 2^-11), the first hidden layer's error passes through |W2| and
    |W3'(t)|; twice the first-order sum, plus a few FP32 ulps of the terms."""
    import oracle

    x = np.asarray(lat, np.float64)
    a1 = np.maximum(x @ w1.T + b1, 0)
    a2 = np.maximum(a1 @ w2.T + b2, 0)
    b = oracle.basis(N1, t, 60.0)
    w3f = np.zeros((28, 64))
    w3f[0] = b[:N1] @ w3[:N1]
    w3f[1:28] = np.einsum("i,qih->qh", b[:N2], w3[N1:].reshape(27, N2, 64))
    u = 2.0 ** -11
    terms = np.abs(a2) @ np.abs(w3f).T
    first = u * (2 * terms + (np.abs(a1) @ np.abs(w2).T) @ np.abs(w3f).T)
    out = np.zeros((x.shape[0], 32))
    out[:, :28] = 2 * first + 1e-6 * (terms + 1.0)
    return out


@pytest.mark.parametrize("n", [1, 128, 129, 1000, 70000, 2_000_003])
def test_latent_table_matches_references(n):
    w1, b1, w2, b2, w3, b3 = _net(n)
    rng = np.random.default_rng(100 + n)
    lat = rng.normal(size=(n, 32)).astype(np.float16)
    t = 13.7
    dev = lambda a: torch.as_tensor(np.asarray(a), device="cuda")
    got, status = fpo.latent_table(dev(lat), dev(w1), dev(b1), dev(w2), dev(b2), dev(w3), dev(b3), t)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    got = got.cpu().numpy().astype(np.float64)
    emu = _emulate(lat.astype(np.float64), w1, b1, w2, b2, w3, b3, t)
    err = np.abs(got - emu)
    assert err.max() <= 2e-3 * max(1.0, np.abs(emu).max()), err.max()
    # element by element against the plain FP64 table, within the FP16
    # operand bound (rows sampled for the largest case)
    rows = np.arange(n) if n <= 70000 else np.random.default_rng(n).choice(n, 70000, replace=False)
    exact = olat.table(olat.decode(lat[rows].astype(np.float64), w1, b1, w2, b2, w3, b3), t)
    bound = _fp16_bound(lat[rows], w1, b1, w2, b2, w3, b3, t)
    d = np.abs(got[rows] - exact)
    worst = (d / np.maximum(bound, 1e-30))[:, :28].max()
    print(f"n={n}: max |table - FP64| {d.max():.2e}, worst / bound {worst:.3f}")
    assert np.all(d <= bound)


def test_latent_table_reports_fp16_range():
    # a hidden activation beyond 65504 rounds to +inf in the FP16 operands:
    # the table is wrong, and the status word says so
    w1, b1, w2, b2, w3, b3 = _net(3)
    lat = np.full((300, 32), 30.0, np.float16)
    dev = lambda a: torch.as_tensor(np.asarray(a), device="cuda")
    big = w1 * 0 + np.float32(100.0)  # every first-layer output is 32 * 30 * 100 = 96000
    _, status = fpo.latent_table(dev(lat), dev(big), dev(b1), dev(w2), dev(b2), dev(w3), dev(b3), 5.0)
    torch.cuda.synchronize()
    assert int(status.item()) & 8
    # a weight beyond the range (BF16 holds it, FP16 does not)
    w2b = w2.copy()
    w2b[3, 7] = 1.0e5
    _, status = fpo.latent_table(dev(lat * 0), dev(w1), dev(b1), dev(w2b), dev(b2), dev(w3), dev(b3), 5.0)
    torch.cuda.synchronize()
    assert int(status.item()) & 8
    # in range: nothing reported
    _, status = fpo.latent_table(dev(lat * 0), dev(w1), dev(b1), dev(w2), dev(b2), dev(w3), dev(b3), 5.0)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
