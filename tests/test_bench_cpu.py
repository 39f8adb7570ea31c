"""CPU checks of bench.py: the multi-rank logic under gloo (world size 2) and
the reference arm's JSON line (the FP64 oracle on a small sample)."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(10.0 + rank, dist, "cpu")
        frames = bench.frames_for_rank(rank, 8)
        q.put((rank, t, frames))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo_max_time_and_own_frames():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict()
    for _ in range(2):
        rank, t, frames = q.get(timeout=120)
        res[rank] = (t, frames)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][0] == res[1][0] == 11.0  # slowest rank's time on every rank
    assert res[0][1] != res[1][1]  # each rank renders its own frames
    sys.path.insert(0, ROOT)
    import bench

    # whole-job throughput counts both ranks' frames
    assert bench.mrays_per_s(2, 10, 1_000_000, 1000.0) == 2 * bench.mrays_per_s(1, 10, 1_000_000, 1000.0)


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "Mrays/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["higher_is_better"] is True
    # the GPU arm's default workload
    assert line["config"]["idft"] == "materialise" and line["config"]["table"] == "f32"
    assert line["config"]["storage"] == "f32" and line["config"]["frames_per_call"] == 32


def test_frame_roofline_bytes():
    sys.path.insert(0, ROOT)
    import bench

    # 10 leaves of 664 B, 4 visited, 128 B table rows, 3 nodes, 5 rays, 1 ms
    fr = bench.frame_roofline(1.0, 10, 4, 664, 128, 3, 5, 1000.0)
    assert fr["bytes_visited"] == 4 * 664 + 3 * 32 + 5 * 12
    assert fr["bytes_materialised"] == 10 * (664 + 128) + 4 * 128 + 3 * 32 + 5 * 12
    assert fr["bytes_min"] == fr["bytes_visited"]
    assert abs(fr["achieved"] - fr["bytes_min"] / 1e-3 / 1e9) < 1e-12
    assert abs(fr["frac"] - fr["achieved"] / 1000.0) < 1e-12
    # distinct visited leaves never outnumber the leaves, so the visited count
    # is the minimum even when every leaf is reached
    fr = bench.frame_roofline(1.0, 10, 10, 664, 128, 0, 0, 1000.0)
    assert fr["bytes_min"] == fr["bytes_visited"] == 6640


def test_clock_sampler_summary_flags_throttling():
    sys.path.insert(0, ROOT)
    import bench

    c = bench.ClockSampler(0)
    # index, sm, max sm, power, active reasons, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    c.out = ("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
             "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
             "0, 2070, 2070, 1100.5, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.out = "0, 1500, 2070, 700.0, 0x8, Active, Not Active, Not Active, Not Active\n"
    assert c.summary()["reasons"] == ["hw_slowdown"]
    c.out = ""
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_gpus_flag_must_match_the_launched_ranks():
    # --gpus 2 without a launcher would silently time one GPU: refused
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--steps", "1"],
                         capture_output=True, text=True, timeout=120, cwd=ROOT, env=env)
    assert out.returncode != 0
    assert "WORLD_SIZE=1" in out.stderr


def test_both_arms_name_the_same_workload():
    sys.path.insert(0, ROOT)
    import argparse

    import bench

    class T:
        n_leaves = 3506408

    args = argparse.Namespace(width=1920, height=1080, idft="auto", storage="f32", frames_per_call=32,
                              refill_min=0, inner_steps=0)
    cfg = bench.workload_config(T(), args)
    assert cfg["idft"] == "materialise" and cfg["table"] == "f32" and cfg["storage"] == "f32"
    assert cfg["frames_per_call"] == 32 and cfg["resolution"] == [1920, 1080] and cfg["schedule"] == "plain"
    args.storage = "bf16"
    assert bench.workload_config(T(), args)["table"] == "f16"
    args.idft = "fused"
    assert bench.workload_config(T(), args)["table"] is None
