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
    exact = olat.table(olat.decode(lat.astype(np.float64), w1, b1, w2, b2, w3, b3), t)
    rel = np.linalg.norm(got - exact) / np.linalg.norm(exact)
    assert rel <= 1e-2, rel
