"""Throughput benchmark of the FPO renderer: one step = one full frame.

Workload: the depth-9 union octree of the animated 14-capsule body (about
3.5M leaves, n1 = 31, n2 = 5, i.i.d. coefficients, seed 0), rendered at
1920x1080 from the 16 ring cameras at integer frame times: by default the
960 timed frames are each (camera, t) of the 16 x 60 grid once, in a seeded
order.  The tree (2.4 GB of coefficient records) is larger
than L2, so no flush is needed between frames.  The timed region renders the
frames through fpo_render_frames, 32 frames a call (the IDFT pass of frame
k + 1 overlaps the traversal of frame k); a single-frame pass beforehand
times each kernel on its own.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU
oracle instead, on a bounded sample of pixels per step.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2202_08614_gb300 import synth  # noqa: E402

METRIC = "FPO render Mrays/s, 1080p fps; plain FP32 vs BF16/latent at PSNR≥45dB vs FP64"
ALG_READ_PER_LEAF = 4 * (31 + 135)   # coefficient bytes of one leaf (FP32)
STORED_PER_LEAF = {"f32": 4 * 166, "bf16": 2 * 166, "f16": 2 * 166, "fp8": 166 + 4}  # + FP8 scale
TABLE_VALUES_PER_LEAF = 28           # sigma(t) + 27 z(t), FP32 or FP16 (the table precision)
OUT_BYTES_PER_RAY = 12               # FP32 RGB
E2E_WINDOWS = 5                      # end-to-end windows of K steps; the median is reported


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=960)  # every (camera, t) of the 16 x 60 grid once
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="fpo", choices=["fpo", "reference"])
    ap.add_argument("--idft", default="auto", choices=["auto", "materialise", "fused"])
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f16", "fp8"])
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle sample budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the BF16 and latent-decoder variant measurements")
    ap.add_argument("--variant-frames", type=int, default=100)
    ap.add_argument("--frames-per-call", type=int, default=32,
                    help="frames per fpo_render_frames call in the timed region (1: fpo_render per frame)")
    ap.add_argument("--latent-steps", type=int, default=20000)
    ap.add_argument("--finetune-steps", type=int, default=200)
    ap.add_argument("--refill-min", type=int, default=0,
                    help="traversal schedule: warp-level ray compaction once this many lanes are idle (0: plain)")
    ap.add_argument("--inner-steps", type=int, default=0,
                    help="steps a lane takes between two compaction checks (0: to the end of its ray)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def frames_for_rank(rank: int, n: int):
    """Each rank renders its own frames: a seeded order over the 16 x 60 grid."""
    return synth.frame_schedule(n, seed=1000 + rank)


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The slowest rank's time (all_reduce MAX); x itself on one process."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def mrays_per_s(world: int, steps: int, rays_per_frame: int, elapsed_ms: float) -> float:
    """Whole-job throughput: every rank renders `steps` frames in `elapsed_ms`."""
    return world * steps * rays_per_frame / (elapsed_ms * 1e-3) / 1e6


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal (context for the measured peak)
NODE_BYTES = 32


def frame_roofline(frame_ms: float, n_leaves: int, n_vis: float, s_leaf: int, table_bytes: int,
                   n_nodes: int, n_px: int, peak: float) -> dict:
    """Whole-frame roofline on the bytes the method must move per frame.

    visited: every distinct leaf reached before early stop read once (its
    stored record), the nodes on the way (counted as all nodes, an upper
    bound under 1% of the total) and the output.  materialised: the per-frame
    IDFT pass reads every record and writes every table row, the traversal
    reads the visited rows.  The smaller of the two is the method's minimum.
    """
    out = n_px * OUT_BYTES_PER_RAY
    nodes = n_nodes * NODE_BYTES
    b_vis = n_vis * s_leaf + nodes + out
    b_mat = n_leaves * (s_leaf + table_bytes) + n_vis * table_bytes + nodes + out
    b_min = min(b_vis, b_mat)
    achieved = b_min / (frame_ms * 1e-3) / 1e9
    return {"bytes_visited": b_vis, "bytes_materialised": b_mat, "bytes_min": b_min,
            "frame_ms": frame_ms, "achieved": achieved, "unit": "GB/s", "peak": peak,
            "frac": achieved / peak, "frac_of_nominal": achieved / NOMINAL_HBM_GBS}


# ---------------------------------------------------------------------------
# oracle timing (CPU baseline and the reference arm)


def oracle_sample_rate(tree, cams, frames, budget_s, stride=61, threads=None):
    """Times the FP64 oracle on strided pixel samples of successive frames
    until `budget_s` seconds of wall time; returns (Mrays/s, rays, seconds, threads)."""
    import oracle

    ot = oracle.OracleTree(tree.leaf_depth, tree.leaf_xyz, tree.max_depth)
    threads = threads or os.cpu_count() or 1
    rays, spent, i = 0, 0.0, 0
    while spent < budget_s:
        k, t = frames[i % len(frames)]
        cam = cams[k]
        n = cam.width * cam.height
        sel = np.arange(i % stride, n, stride, dtype=np.int64)
        t0 = time.perf_counter()
        oracle.render(ot, tree.coeffs, camera=cam, t=t, sel=sel, threads=threads)
        spent += time.perf_counter() - t0
        rays += sel.size
        i += 1
    return rays / spent / 1e6, rays, spent, threads


def run_reference(args, rank, world):
    if rank != 0:
        return
    tree = synth.body_tree()
    cams = synth.ring_cameras(16, args.width, args.height)
    frames = frames_for_rank(0, args.steps + args.warmup)
    import oracle

    ot = oracle.OracleTree(tree.leaf_depth, tree.leaf_xyz, tree.max_depth)
    threads = os.cpu_count() or 1
    stride = 256  # each step renders every 256th pixel of its frame
    times, rays = [], 0
    for i, (k, t) in enumerate(frames):
        cam = cams[k]
        sel = np.arange(i % stride, cam.width * cam.height, stride, dtype=np.int64)
        t0 = time.perf_counter()
        oracle.render(ot, tree.coeffs, camera=cam, t=t, sel=sel, threads=threads)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            rays += sel.size
    total = sum(times)
    value = rays / total / 1e6
    sample = (f"every {stride}th pixel of one {args.width}x{args.height} frame per step "
              f"({rays // max(len(times), 1)} rays), {len(times)} steps")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mrays/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / max(len(times), 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(tree, args),
        "cpu_baseline": {"value": value, "unit": "Mrays/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------


def workload_config(tree, args):
    """The workload, derived from the arguments alone, so that the oracle arm
    and the GPU arm name the same one."""
    return {
        "workload": (f"body union octree (14 animated capsules, 60 frames), depth 9, "
                     f"{tree.n_leaves} leaves, n1=31 n2=5 SH deg 2, {args.width}x{args.height}, "
                     f"16 ring cameras x 60 integer t"),
        "leaves": tree.n_leaves,
        "resolution": [args.width, args.height],
        "idft": "fused" if args.idft == "fused" else "materialise",
        "storage": args.storage,
        "table": None if args.idft == "fused" else ("f32" if args.storage == "f32" else "f16"),
        "frames_per_call": max(1, args.frames_per_call),
        "l2": "inputs larger than L2 (2.4 GB of leaf records)",
        "early_stop_T": 1e-4,
        "schedule": ("plain" if args.refill_min in (0, 32) else
                     f"compaction: refill_min {args.refill_min}, inner_steps {args.inner_steps or 'to the end'}"),
    }


class ClockSampler:
    """nvidia-smi sampling (every 20 ms) of SM clocks and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        # nvidia-smi's start-up stays out of the timed region: wait (at most
        # 5 s) for its first sample, taken before the region and not counted
        if self.proc is not None:
            import select

            if select.select([self.proc.stdout], [], [], 5.0)[0]:
                self.proc.stdout.readline()
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(", ") for r in getattr(self, "out", "").strip().splitlines() if r.strip()]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def time_frames(r, cams, frames, out, torch, per_call=1):
    """Mean CUDA-event time (ms) per frame of rendering `frames` (after
    warm-up): fpo_render_frames calls of `per_call` frames, or one fpo_render
    call per frame when per_call is 1."""
    outb = torch.empty((per_call, out.shape[0], 3), dtype=torch.float32, device=out.device) if per_call > 1 else None

    def run(fr):
        if per_call <= 1:
            for k, t in fr:
                r.render(camera=cams[k], t=t, out=out)
            return
        for i in range(0, len(fr), per_call):
            b = fr[i:i + per_call]
            r.render_frames([cams[k] for k, _ in b], [t for _, t in b], out=outb[:len(b)])

    run(frames[:max(3, min(per_call, len(frames)))])
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    run(frames)
    b.record()
    torch.cuda.synchronize()
    r.status()
    return a.elapsed_time(b) / len(frames)


PSNR_FRAMES = [(k, 3.75 * k) for k in range(16)]  # one frame per ring camera, t = 3.75 k


def frame_psnr(r, ot, coeffs, cams, out, torch, refs=None):
    """Per-frame PSNR (and max |dRGB|) of whole rendered frames against the
    FP64 oracle over the 16 frames of PSNR_FRAMES.  `refs` caches the oracle
    images of one coefficient set."""
    import oracle

    if refs is None:
        refs = [oracle.render(ot, coeffs, camera=cams[k], t=t)["rgb"] for k, t in PSNR_FRAMES]
    db, mx = [], []
    for (k, t), ref in zip(PSNR_FRAMES, refs):
        img = r.render(camera=cams[k], t=t, out=out)["rgb"].cpu().numpy().astype(np.float64)
        mse = float(np.mean((img - ref) ** 2))
        db.append(10 * np.log10(1.0 / mse) if mse > 0 else float("inf"))
        mx.append(float(np.abs(img - ref).max()))
    r.status()
    return {"min_db": min(db), "mean_db": float(np.mean(db)), "per_frame_db": db, "max_abs_rgb": max(mx),
            "frames": "camera k at t = 3.75 k, k = 0..15, whole frames"}, refs


def variants(args, tree, cams, frames, out, torch, fpo, n_px, fp32_ms, n_vis, peak, fma_peak=None):
    """BF16 storage on the same tree, and the latent decoder (trained on
    coefficients produced by the generation: smooth animated fields -> per-
    leaf DFT) against the plain FP32 renderer of those coefficients."""
    import oracle
    from paper_2202_08614_gb300.latent import LatentModel, PixelLoss

    res = {}
    nf = frames[: args.variant_frames]
    ot = oracle.OracleTree(tree.leaf_depth, tree.leaf_xyz, tree.max_depth)
    r = fpo.Renderer(storage="bf16")
    r.upload(tree)
    B = args.frames_per_call
    ms = time_frames(r, cams, nf, out, torch, B)
    ms1 = time_frames(r, cams, nf, out, torch)
    res["bf16"] = {"Mrays_s": n_px / ms / 1e3, "fps": 1e3 / ms, "fp32_Mrays_s": n_px / fp32_ms / 1e3,
                   "single_frame_Mrays_s": n_px / ms1 / 1e3,
                   "psnr_vs_fp64_oracle": frame_psnr(r, ot, tree.coeffs, cams, out, torch)[0],
                   "bytes_per_leaf": r.info()["leaf_record_bytes"]}
    # the FP16 table of reduced-precision storage: 28 values x 2 B per leaf
    res["bf16"]["frame_roofline"] = frame_roofline(ms, tree.n_leaves, n_vis, STORED_PER_LEAF["bf16"],
                                                   2 * TABLE_VALUES_PER_LEAF, r.info()["n_nodes"], n_px, peak)
    r.close()
    # multi-view rendering of one frame time: the 16 ring views of each t share
    # one IDFT pass, in one fpo_render_frames call per t (the views' traversals
    # overlap), or as fpo_render calls with FPO_FLAG_REUSE_TABLE
    r = fpo.Renderer()
    r.upload(tree)
    ts = [float(t) for t in range(0, 60, 6)]
    outv = torch.empty((len(cams), n_px, 3), dtype=torch.float32, device="cuda")
    r.render_frames(cams, [ts[0]] * len(cams), out=outv)
    for cam in cams[:3]:
        r.render(camera=cam, t=ts[0], out=out, reuse_table=True)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for t in ts:
        r.render_frames(cams, [t] * len(cams), out=outv)
    b.record()
    c, d = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c.record()
    for t in ts:
        for cam in cams:
            r.render(camera=cam, t=t, out=out, reuse_table=True)
    d.record()
    torch.cuda.synchronize()
    r.status()
    r.close()
    mv = a.elapsed_time(b) / (len(ts) * len(cams))
    mv1 = c.elapsed_time(d) / (len(ts) * len(cams))
    res["multiview_16_views_per_t"] = {"ms_per_view": mv, "Mrays_s": n_px / mv / 1e3, "fps": 1e3 / mv,
                                       "frame_times": len(ts), "views_per_t": len(cams),
                                       "calls": "one fpo_render_frames call per t",
                                       "single_view_calls": {"ms_per_view": mv1, "Mrays_s": n_px / mv1 / 1e3,
                                                             "calls": "fpo_render with the table reused"}}
    # the Fourier sizes of the paper's ablation (Tab. 3) on the same leaves and
    # coefficient distributions: frame rate and bytes per leaf (the (31, 5)
    # entry is the headline measurement)
    pad4 = lambda k: (k + 3) & ~3  # record strides: n1 and 27 n2 floats, each rounded up to 4
    dims = {"31,5": {"Mrays_s": n_px / fp32_ms / 1e3, "fps": 1e3 / fp32_ms, "bytes_per_leaf": 4 * (pad4(31) + pad4(135))}}
    for n1, n2 in ((11, 5), (21, 5), (31, 11)):
        co = synth.draw_coefficients_blocked(1, tree.n_leaves, n1, n2)
        r = fpo.Renderer(n1=n1, n2=n2)
        r.upload(synth.Tree(tree.leaf_depth, tree.leaf_xyz, co, tree.max_depth, n1, n2))
        del co
        ms_d = time_frames(r, cams, nf, out, torch, B)
        dims[f"{n1},{n2}"] = {"Mrays_s": n_px / ms_d / 1e3, "fps": 1e3 / ms_d,
                              "bytes_per_leaf": r.info()["leaf_record_bytes"]}
        r.close()
    res["fourier_dims"] = dims
    if args.finetune_steps > 0:
        res["finetune"] = finetune_variant(args, tree, torch, fpo)
    # latent decoder on generated coefficients (same leaves)
    body = synth.capsule_body(np.random.default_rng(0))
    n = tree.n_leaves
    coeffs = torch.empty((n, 166), dtype=torch.float32, device="cuda")
    ch = 1 << 19
    dft_ms = 0.0
    dft_status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for s0 in range(0, n, ch):
        vals = synth.smooth_frame_values(tree.leaf_depth[s0:s0 + ch], tree.leaf_xyz[s0:s0 + ch], body)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fpo.dft_leaves(vals, out=coeffs[s0:s0 + ch], status=dft_status)
        e1.record()
        torch.cuda.synchronize()
        dft_ms += e0.elapsed_time(e1)
        del vals
    fpo.check_status_word(dft_status)
    # Eq. 10-12 over the whole tree: 60 frames x 28 values in, 166 coefficients out per leaf
    dft_bytes = n * (60 * 28 + 166) * 4
    res["generation_dft"] = {"ms": dft_ms, "leaves": n, "frames": 60, "alg_bytes": dft_bytes,
                             "GB_s": dft_bytes / (dft_ms * 1e-3) / 1e9}
    co_np = coeffs.cpu().numpy()
    gen = synth.Tree(tree.leaf_depth, tree.leaf_xyz, co_np, tree.max_depth)
    r = fpo.Renderer()
    r.upload(gen)
    ms32 = time_frames(r, cams, nf, out, torch, B)
    r.close()
    # training: coefficient L2 (density weight 0.2) plus the rendered-pixel
    # loss every 4th step (8192 rays over the 16 ring views x 60 frames,
    # weight 10) through the render adjoint
    m = LatentModel(n, seed=0, tensor_cores=True)
    m.init_output_bias(coeffs)
    pixel_cfg = dict(rays=8192, weight=10.0, every=4, start=0.1, tensor_cores=True)
    pixel = PixelLoss(gen, cams, **pixel_cfg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = m.fit(coeffs, steps=args.latent_steps, batch=65536, lr_w=1e-3, lr_lat=1e-1, decay=0.05,
                 coef_weight=m.default_weights(coeffs.device, sigma_weight=0.2),
                 log_every=max(1, args.latent_steps // 4), pixel=pixel)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    pixel_loss = float(pixel.last_loss)
    # the training kernels' FP32 rates (flop per leaf: forward 2 (32*64 + 64*64
    # + 64*166); the gradient three times that)
    fwd = 2 * (32 * 64 + 64 * 64 + 64 * 166)
    rows = torch.randperm(n, device="cuda")[:65536].to(torch.int32)
    cw = m.default_weights(coeffs.device, sigma_weight=0.2)

    def rate(f, flop, reps, tensor=False):
        f()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            f()
        b.record()
        torch.cuda.synchronize()
        ms_k = a.elapsed_time(b) / reps
        tf = flop / (ms_k * 1e-3) / 1e12
        if tensor:  # BF16 tensor cores: the measured dense BF16 rate
            return {"ms": ms_k, "tflops": tf, "frac_of_bf16_tensor_peak": tf / bf16_peak if bf16_peak else None}
        return {"ms": ms_k, "tflops": tf, "frac_of_fp32_fma_peak": tf / fma_peak if fma_peak else None}

    bf16_peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16_peak = float(json.load(f)["bf16_tflops"])
    except (OSError, ValueError, KeyError):
        pass
    tc = m.tensor_cores
    m.tensor_cores = True
    k_tc = rate(lambda: m.grad(rows, coeffs, cw), 3 * fwd * 65536, 10, tensor=True)
    m.check_status()
    m.tensor_cores = False
    k_simt = rate(lambda: m.grad(rows, coeffs, cw), 3 * fwd * 65536, 10)
    m.tensor_cores = tc
    train_kernels = {
        "training_gradient": "tcgen05 (fpo_decoder_grad_tc, BF16 operands)" if tc else "FP32 SIMT (fpo_decoder_grad)",
        "decoder_grad_tc_65536_leaves": k_tc,
        "decoder_grad_simt_65536_leaves": k_simt,
        "decode_into_records_all_leaves": rate(
            lambda: pixel.work.set_coeffs_from_decoder(m._mlp(m.p), m.p["lat"]), fwd * n, 3),
        "decode_into_records_tc_all_leaves": rate(
            lambda: pixel.work.set_coeffs_from_decoder(m._mlp(m.p), m.p["lat"], tensor_cores=True), fwd * n, 3,
            tensor=True),
    }
    pixel.work.status()
    pixel.close()
    r = fpo.Renderer(storage="latent")
    r.upload(synth.Tree(tree.leaf_depth, tree.leaf_xyz, np.zeros((0, 166), np.float32), tree.max_depth))
    r.set_latents(*m.inference_arrays())
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    msl = time_frames(r, cams, nf, out, torch, B)
    msl1 = time_frames(r, cams, nf, out, torch)
    k, t = nf[0]
    r.render(camera=cams[k], t=t, out=out, events=ev)
    torch.cuda.synchronize()
    res["latent"] = {
        "Mrays_s": n_px / msl / 1e3, "fps": 1e3 / msl, "fp32_same_tree_Mrays_s": n_px / ms32 / 1e3,
        "single_frame_Mrays_s": n_px / msl1 / 1e3,
        "psnr_vs_fp64_oracle": frame_psnr(r, ot, co_np, cams, out, torch)[0],
        "decode_ms": ev[0].elapsed_time(ev[1]), "train_steps": args.latent_steps, "train_batch": 65536,
        "train_s": train_s, "train_loss": hist, "training_kernels": train_kernels,
        "bytes_per_leaf": r.info()["leaf_record_bytes"],
        "fp32_bytes_per_leaf": 672, "pixel_loss": dict(pixel_cfg, last_batch_mse=pixel_loss),
        "coefficients": "per-leaf DFT (Eq. 10-12) of smooth animated fields over the same leaves"}
    r.close()
    return res


def finetune_variant(args, tree, torch, fpo):
    """The fine-tuning stage (Sec. 4.3, Eq. 13) at full scale: coefficients
    perturbed by N(0, 0.1|k| + 0.05), targets rendered by the FP32 path from
    the original ones at 800x800 over 16 ring views x 60 frames, batches of
    65,536 rays, Adam lr 1e-2 (row-sparse, fused with the write-back)."""
    from paper_2202_08614_gb300.finetune import FineTuner, camera_ray_batch

    B, steps, warm = 65536, args.finetune_steps, 5
    cams = synth.ring_cameras(16, 800, 800)
    gen = torch.Generator(device="cuda").manual_seed(7)
    k_true = torch.as_tensor(tree.coeffs, device="cuda")
    noise = torch.randn(k_true.shape, device="cuda", generator=gen) * (0.1 * k_true.abs() + 0.05)
    ref = fpo.Renderer(idft_mode="fused")
    ref.upload(tree)
    r = fpo.Renderer(idft_mode="fused")
    r.upload(tree)
    ft = FineTuner(r, k_true + noise, lr=1e-2)
    del noise
    batches = []
    for _ in range(warm + steps + 1):
        o, d, t = camera_ray_batch(cams, B, gen)
        batches.append((o, d, t, ref.render(rays_o=o, rays_d=d, t_per_ray=t)["rgb"].clone()))
    ref.status()
    ref.close()
    del k_true
    ho = batches.pop()
    held = lambda: float(((ft.render(*ho[:3]) - ho[3]) ** 2).sum(1).mean())
    l0 = held()
    for b in batches[:warm]:
        ft.step(*b)
    torch.cuda.synchronize()
    # rows one batch touches (an untimed count on the next batch's adjoint)
    o, d, t, y = batches[warm]
    rgb = ft.render(o, d, t)
    g = torch.zeros_like(ft.grad)
    mk = torch.zeros_like(ft.mark)
    r.render_backward(rgb, rgb - y, g, rays_o=o, rays_d=d, t_per_ray=t, leaf_mark=mk)
    rows = int(mk.sum())
    del g, mk
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for i, b in enumerate(batches[warm:]):
        ft.step(*b, events=ev[i])
    z.record()
    torch.cuda.synchronize()
    r.status()
    l1 = held()
    ms = a.elapsed_time(z) / steps
    phase = lambda j: statistics.mean(e[j].elapsed_time(e[j + 1]) for e in ev)
    out = {"ms_per_step": ms, "Mrays_s": B / ms / 1e3, "batch_rays": B, "steps": steps,
           "forward_and_loss_ms": phase(0), "adjoint_ms": phase(1), "adam_writeback_ms": phase(2),
           "rows_touched_per_batch": rows, "held_out_loss": [l0, l1], "resolution": [800, 800],
           "optimizer": "Adam lr 1e-2 on the visited rows (sparse-gradient Adam), FP32"}
    r.close()
    del ft, batches
    torch.cuda.empty_cache()
    return out


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("fpo_kernels.cu", "fpo_internal.h"):
        with open(os.path.join(ROOT, "paper_2202_08614_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None
    when the kernel source changed since those counters were taken."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(kernel)
    if not e or e.get("source_sha") != kernel_source_sha():
        return None
    return e.get("dram_bytes_per_launch_full_workload")


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.gpus != world:
        # one process per GPU: N > 1 needs a launcher (torchrun) that starts N ranks
        print(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={world}; launch N ranks with "
              f"torch.distributed.run --nproc-per-node {args.gpus}", file=sys.stderr)
        sys.exit(2)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch

    from paper_2202_08614_gb300 import fpo

    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    tree = synth.body_tree()
    cams = synth.ring_cameras(16, args.width, args.height)
    K, W = args.steps, args.warmup
    frames = frames_for_rank(rank, K + W)
    r = fpo.Renderer(idft_mode=args.idft, storage=args.storage, device=local, refill_min=args.refill_min,
                     inner_steps=args.inner_steps)
    r.upload(tree)
    info = r.info()
    n_px = args.width * args.height
    out = torch.empty((n_px, 3), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    mat = args.idft in ("auto", "materialise")

    B = max(1, args.frames_per_call)
    timed = frames[W:]
    batches = [timed[i:i + B] for i in range(0, K, B)]
    outb = torch.empty((min(B, K), n_px, 3), dtype=torch.float32, device="cuda")

    def render_batch(bt, dst, events=None):
        r.render_frames([cams[k] for k, _ in bt], [t for _, t in bt], out=dst[:len(bt)], frame_events=events)

    # clocks and throttle reasons are sampled over the whole GPU phase (warm-up,
    # the per-kernel pass, the timed region and the end-to-end pass): the
    # timed region alone can be shorter than the sampling period
    clk = ClockSampler(local).__enter__()
    # warm-up: single-frame calls, then pipelined calls (allocates the second table)
    for k, t in frames[:W]:
        r.render(camera=cams[k], t=t, out=out)
    for i in range(0, W, B):
        render_batch(frames[i:min(i + B, W)], outb)
    r.status()

    # single-frame calls with events around each kernel: the launch durations
    # of the IDFT pass and the traversal (the pipelined calls overlap them)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    for e3 in ev:
        for e in e3:
            e.record(stream)
    torch.cuda.synchronize()
    for i, (k, t) in enumerate(timed):
        r.render(camera=cams[k], t=t, out=out, events=ev[i])
    torch.cuda.synchronize()
    r.status()
    frame_ms = [ev[i][0].elapsed_time(ev[i][2]) for i in range(K)]
    mat_ms = [ev[i][0].elapsed_time(ev[i][1]) for i in range(K)]
    trav_ms = [ev[i][1].elapsed_time(ev[i][2]) for i in range(K)]

    # timed region: the K frames through fpo_render_frames, B frames a call
    bev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in batches]
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    start.record(stream)
    for j, bt in enumerate(batches):
        bev[j][0].record(stream)
        render_batch(bt, outb)
        bev[j][1].record(stream)
    stop.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if pg:
        pg.barrier()
    r.status()
    elapsed_ms = start.elapsed_time(stop)
    t_max = max_over_ranks(elapsed_ms, pg, "cuda")
    batch_frame_ms = [bev[j][0].elapsed_time(bev[j][1]) / len(bt) for j, bt in enumerate(batches)]

    # visited leaves per timed frame (a marking pass outside the timed region)
    mark = torch.zeros(tree.n_leaves, dtype=torch.uint8, device="cuda")
    n_vis = []
    for k, t in timed:
        mark.zero_()
        r.render(camera=cams[k], t=t, out=out, leaf_mark=mark)
        n_vis.append(int(mark.sum().item()))
    r.status()

    # end to end through the public API: every frame is read back into pinned
    # host memory inside the timed region.  Frame i of a call is copied on a
    # copy stream as soon as its pixels are written (the call's per-frame
    # events), while the later frames render; two device and two host buffers
    # alternate between calls, and before a call reuses a pair the host waits
    # until the pair's previous frames are in host memory.
    outs = [outb, torch.empty_like(outb)]
    hosts = [torch.empty(outb.shape, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    fev = [[torch.cuda.Event() for _ in range(outb.shape[0])] for _ in range(2)]
    landed = [torch.cuda.Event(), torch.cuda.Event()]

    def e2e_batch(b, bt):
        render_batch(bt, outs[b], fev[b][:len(bt)])
        with torch.cuda.stream(copy_stream):
            for i in range(len(bt)):
                copy_stream.wait_event(fev[b][i])
                hosts[b][i].copy_(outs[b][i], non_blocking=True)
            landed[b].record(copy_stream)

    # warm-up of this path (first copies into the pinned buffers, events)
    for b in range(2):
        e2e_batch(b, frames[:min(B, W)])
    torch.cuda.synchronize()
    # the K-step window is a host wall clock of a few ms on shared host cores:
    # it is taken E2E_WINDOWS times and the median window is reported
    e2e_windows = []
    for _ in range(E2E_WINDOWS):
        t0 = time.perf_counter()
        for j, bt in enumerate(batches):
            if j >= 2:
                landed[j & 1].synchronize()
            e2e_batch(j & 1, bt)
        torch.cuda.synchronize()
        e2e_windows.append(time.perf_counter() - t0)
    e2e_s = statistics.median(e2e_windows)
    r.status()
    clk.__exit__(None, None, None)

    value = mrays_per_s(world, K, n_px, t_max)
    res = {
        "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": t_max / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(tree, args),
    }
    res["fps"] = 1e3 * K / t_max
    res["frame_ms"] = {"p10": float(np.percentile(batch_frame_ms, 10)), "p50": statistics.median(batch_frame_ms),
                       "p90": float(np.percentile(batch_frame_ms, 90)),
                       "over": f"{len(batches)} calls of fpo_render_frames (time per call / frames per call)"}
    res["single_frame"] = {"Mrays_s": n_px / statistics.median(frame_ms) / 1e3,
                           "fps": 1e3 / statistics.median(frame_ms),
                           "frame_ms": {"p10": float(np.percentile(frame_ms, 10)),
                                        "p50": statistics.median(frame_ms),
                                        "p90": float(np.percentile(frame_ms, 90))},
                           "over": f"{K} fpo_render calls, events from the IDFT pass to the traversal's end"}
    # roofline of the dominant kernel
    avg_mat = statistics.mean(mat_ms) if mat else 0.0
    avg_trav = statistics.mean(trav_ms)
    mean_vis = statistics.mean(n_vis)
    # bytes of sigma(t) and z(t) per leaf: FP16 table rows are 64 B, FP32 128 B
    table_bytes = TABLE_VALUES_PER_LEAF * (2 if r.info()["table_bytes"] == 64 * tree.n_leaves else 4)
    assert res["config"]["table"] == (("f16" if table_bytes == 2 * TABLE_VALUES_PER_LEAF else "f32") if mat else None)
    if mat:
        kernels = {
            "materialise_kernel": (avg_mat, tree.n_leaves * (STORED_PER_LEAF[args.storage] + table_bytes)),
            "traverse_kernel": (avg_trav, mean_vis * table_bytes + n_px * OUT_BYTES_PER_RAY),
        }
    else:
        kernels = {"traverse_kernel": (avg_trav, mean_vis * ALG_READ_PER_LEAF + n_px * OUT_BYTES_PER_RAY)}
    dom = max(kernels, key=lambda k: kernels[k][0])
    ms, nbytes = kernels[dom]
    peak = 6791.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["hbm_gbs"])
        peak_src = "measured"
    except (OSError, ValueError, KeyError):
        peak_src = "fallback"
        peak = 6800.0
    achieved = nbytes / (ms * 1e-3) / 1e9
    res["roofline"] = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                       "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                       "traffic": ncu_traffic(dom), "alg_bytes_per_launch": nbytes,
                       "launch_ms": ms,
                       "launches": "single-frame fpo_render calls (the pipelined calls overlap the two kernels)"}
    res["kernels_ms"] = {k: v[0] for k, v in kernels.items()}
    res["visited_leaves_per_frame"] = mean_vis
    res["frame_roofline"] = frame_roofline(t_max / K, tree.n_leaves, mean_vis,
                                           STORED_PER_LEAF[args.storage], table_bytes, info["n_nodes"],
                                           n_px, peak)
    res["single_frame"]["frame_roofline_frac"] = frame_roofline(
        statistics.median(frame_ms), tree.n_leaves, mean_vis, STORED_PER_LEAF[args.storage], table_bytes,
        info["n_nodes"], n_px, peak)["frac"]
    res["e2e"] = {"value": mrays_per_s(world, K, n_px, 1e3 * max_over_ranks(e2e_s, pg, "cuda")),
                  "unit": "Mrays/s",
                  "h2d_bytes_per_step": int(fpo.C.sizeof(fpo.Rays) + fpo.C.sizeof(fpo.FrameOpts)),
                  "d2h_bytes_per_step": int(n_px * 3 * 4),
                  "windows_Mrays_s": [mrays_per_s(1, K, n_px, 1e3 * w) for w in e2e_windows],
                  "over": f"median of {E2E_WINDOWS} windows of the {K} steps (this rank's), max over ranks"}
    res["gpu_launches"] = K * (2 if mat else 1)
    res["clocks"] = clk.summary()
    res["clocks"]["window"] = "the whole GPU phase: warm-up, per-kernel pass, timed region, end-to-end pass"
    res["tree"] = info
    if not args.no_variants:
        # the second resolution of the workload: 800x800 from the same ring
        cams8 = synth.ring_cameras(16, 800, 800)
        out8 = torch.empty((800 * 800, 3), dtype=torch.float32, device="cuda")
        ev8 = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in frames[W:]]
        for k, t in frames[:W]:
            r.render(camera=cams8[k], t=t, out=out8)
        torch.cuda.synchronize()
        for i, (k, t) in enumerate(frames[W:]):
            ev8[i][0].record(stream)
            r.render(camera=cams8[k], t=t, out=out8)
            ev8[i][1].record(stream)
        torch.cuda.synchronize()
        r.status()
        ms8 = [e[0].elapsed_time(e[1]) for e in ev8]
        msp = time_frames(r, cams8, frames[W:], out8, torch, B)
        res["res_800x800"] = {"Mrays_s": 800 * 800 / msp / 1e3, "fps": 1e3 / msp,
                              "frames_per_call": B,
                              "single_frame": {"Mrays_s": 800 * 800 / statistics.median(ms8) / 1e3,
                                               "fps": 1e3 / statistics.median(ms8),
                                               "frame_ms": {"p10": float(np.percentile(ms8, 10)),
                                                            "p50": statistics.median(ms8),
                                                            "p90": float(np.percentile(ms8, 90))}}}
    # the FP32 FMA rate of this GPU: the denominator of the SIMT FP32 kernels' roofline
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    res["fp32_fma_peak"] = {"tflops": fpo.fma_peak_tflops(),
                            "nominal_tflops_at_max_clock": sms * 128 * 2 * 2.07e9 / 1e12,
                            "how": "fpo_fma_peak: two 1024-thread CTAs per SM, 16 independent FMA chains "
                                   "per thread, 4096 steps, best of 5 launches (CUDA events)"}
    if not args.no_variants and args.storage == "f32" and args.idft == "auto":
        res["variants"] = variants(args, tree, cams, frames[W:], out, torch, fpo, n_px, t_max / K,
                                   mean_vis, peak, res["fp32_fma_peak"]["tflops"])
    if rank == 0 and not args.no_cpu_baseline:
        v, rays, secs, thr = oracle_sample_rate(tree, cams, frames[W:], args.cpu_seconds)
        res["cpu_baseline"] = {"value": v, "unit": "Mrays/s", "cores": thr, "kind": "oracle",
                               "sample": f"{rays} rays: every 61st pixel of successive timed "
                                         f"frames, {secs:.1f} s"}
        # the same oracle on one core, and the full 128x128 shell frame (the
        # parity case) on all cores
        v1, rays1, secs1, _ = oracle_sample_rate(tree, cams, frames[W:], args.cpu_seconds / 4, stride=997, threads=1)
        res["cpu_baseline"]["one_core"] = {"value": v1, "cores": 1, "sample": f"{rays1} rays, {secs1:.1f} s"}
        import oracle

        # four whole frames per resolution (seeded picks from the timed frames)
        ot = oracle.OracleTree(tree.leaf_depth, tree.leaf_xyz, tree.max_depth)
        picks = [frames[W:][i] for i in np.random.default_rng(7).choice(K, size=min(4, K), replace=False)]
        res["cpu_baseline"]["full_frames"] = {}
        for w, h in ((args.width, args.height), (800, 800)):
            cams_r = synth.ring_cameras(16, w, h)
            secs = []
            for k, t in picks:
                t0 = time.perf_counter()
                oracle.render(ot, tree.coeffs, camera=cams_r[k], t=t, threads=thr)
                secs.append(time.perf_counter() - t0)
            res["cpu_baseline"]["full_frames"][f"{w}x{h}"] = {
                "frames": len(picks), "s_per_frame": statistics.mean(secs),
                "Mrays_s": w * h * len(secs) / sum(secs) / 1e6, "cores": thr}
        shell = synth.shell_tree()
        t0 = time.perf_counter()
        oracle.render(oracle.OracleTree(shell.leaf_depth, shell.leaf_xyz, shell.max_depth), shell.coeffs,
                      camera=synth.shell_camera(), t=synth.SHELL_T, threads=thr)
        res["cpu_baseline"]["shell_128_full_frame_s"] = time.perf_counter() - t0
    r.close()
    if rank == 0:
        print(json.dumps(res), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
