"""The multi-rank bench path with real renders: two gloo ranks (spawned), each
on its own device ordinal when the machine has two GPUs, else both on GPU 0
(two independent processes whose kernels never wait on one another).  Each
rank takes its rank / world / local ordinal from the launcher's environment
the way bench.py does, renders its own frames of the shell through the C ABI,
and reduces its time with the other rank; the parent checks every image
against the FP64 oracle."""

import os
import sys

import numpy as np
import pytest

import gpu_util as gu
from paper_2202_08614_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
W, H = 48, 36
N_FRAMES = 2


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _rank_main(rank, world, port, q):
    import time

    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench
    from paper_2202_08614_gb300 import fpo

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    r_, w_, local = bench.dist_env()
    dev = local % torch.cuda.device_count()
    torch.cuda.set_device(dev)
    dist.init_process_group("gloo", rank=r_, world_size=w_)
    try:
        tree = synth.shell_tree()
        cams = synth.ring_cameras(16, W, H)
        frames = bench.frames_for_rank(r_, N_FRAMES)
        r = fpo.Renderer(device=dev)
        try:
            r.upload(tree)
            t0 = time.perf_counter()
            imgs = [r.render(camera=cams[k], t=t)["rgb"].cpu().numpy() for k, t in frames]
            r.status()
            el = time.perf_counter() - t0
        finally:
            r.close()
        t_max = bench.max_over_ranks(el, dist, "cpu")
        q.put((r_, dev, frames, imgs, el, t_max))
    finally:
        dist.destroy_process_group()


def test_two_ranks_render_their_own_frames_on_their_own_devices():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29700 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        rank, dev, frames, imgs, el, t_max = q.get(timeout=300)
        res[rank] = (dev, frames, imgs, el, t_max)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    if torch.cuda.device_count() >= 2:
        assert res[0][0] == 0 and res[1][0] == 1
    assert res[0][1] != res[1][1]
    assert res[0][4] == res[1][4] == max(res[0][3], res[1][3])
    tree = synth.shell_tree()
    ot = gu.oracle_tree(tree)
    cams = synth.ring_cameras(16, W, H)
    for rank in (0, 1):
        for (k, t), img in zip(res[rank][1], res[rank][2]):
            ref = gu.oracle.render(ot, tree.coeffs, camera=cams[k], t=t)["rgb"]
            d = np.abs(img.astype(np.float64) - ref)
            assert d.max() <= 1e-3 and d.mean() <= 1e-5, (rank, k, t, d.max())
