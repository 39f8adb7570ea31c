"""ctypes binding of libfpo.so (include/fpo.h).

Argument marshalling only: every step of rendering runs in the CUDA library.
PyTorch supplies device memory (tensor.data_ptr()) and streams
(torch.cuda.current_stream().cuda_stream).  When the compiled library is
missing, loading it raises instead of falling back to anything else.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libfpo.so")

FPO_OK = 0
ERRORS = {
    -1: "FPO_ERR_INVALID_ARG", -2: "FPO_ERR_OOM", -3: "FPO_ERR_CUDA", -4: "FPO_ERR_BAD_TREE",
    -5: "FPO_ERR_NO_TREE", -6: "FPO_ERR_TRAVERSAL_LIMIT", -7: "FPO_ERR_VISIT_OVERFLOW",
    -8: "FPO_ERR_UNSUPPORTED", -9: "FPO_ERR_DEVICE_TIMEOUT", -10: "FPO_ERR_RANGE",
}
STORAGE = {"f32": 0, "bf16": 1, "f16": 2, "fp8": 3, "latent": 4}
IDFT = {"auto": 0, "fused": 1, "materialise": 2}
TABLE = {"auto": 0, "f32": 1, "f16": 2}
RAYS_CAMERA, RAYS_EXPLICIT = 0, 1
FLAG_RECORD_VISITS, FLAG_OUT_T, FLAG_MARK_LEAVES, FLAG_STATS, FLAG_REUSE_TABLE = 1, 2, 4, 8, 16
FLAG_FP64_GRADCHECK, FLAG_TEST_DEVICE_TIMEOUT, FLAG_TENSOR_CORES = 32, 64, 128

# Every symbol include/fpo.h declares.
EXPORTS = ["fpo_create", "fpo_validate_tree", "fpo_upload_tree", "fpo_render",
           "fpo_render_backward", "fpo_status_sync", "fpo_tree_info_get", "fpo_destroy",
           "fpo_last_error", "fpo_version", "fpo_render_noalloc", "fpo_set_coeffs",
           "fpo_dft_leaves", "fpo_union_trees", "fpo_latent_table", "fpo_decoder_grad",
           "fpo_adam", "fpo_set_latents", "fpo_render_frames", "fpo_adam_leaves",
           "fpo_decoder_forward", "fpo_set_coeffs_from_decoder", "fpo_fma_peak", "fpo_decoder_grad_tc"]


class FPOError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [("n1", C.c_int32), ("n2", C.c_int32), ("sh_degree", C.c_int32),
                ("period_T", C.c_double), ("storage", C.c_int32), ("idft_mode", C.c_int32),
                ("device", C.c_int32), ("traverse_threads", C.c_int32), ("refill_min", C.c_int32),
                ("inner_steps", C.c_int32), ("table_precision", C.c_int32), ("max_steps", C.c_int32)]


class TreeDesc(C.Structure):
    _fields_ = [("n_leaves", C.c_uint32), ("max_depth", C.c_uint32), ("leaf_depth", C.c_void_p),
                ("leaf_xyz", C.c_void_p), ("coeffs", C.c_void_p), ("aabb_min", C.c_double * 3),
                ("aabb_size", C.c_double)]


class Rays(C.Structure):
    _fields_ = [("mode", C.c_int32), ("eye", C.c_double * 3), ("target", C.c_double * 3),
                ("up", C.c_double * 3), ("fov_y_deg", C.c_double), ("width", C.c_uint32),
                ("height", C.c_uint32), ("t", C.c_double), ("n", C.c_uint32), ("o", C.c_void_p),
                ("d", C.c_void_p), ("t_per_ray", C.c_void_p)]


class FrameOpts(C.Structure):
    _fields_ = [("bg", C.c_float * 3), ("stop_T", C.c_float), ("flags", C.c_uint32),
                ("visit_log", C.c_void_p), ("visit_cap", C.c_uint32), ("visit_count", C.c_void_p),
                ("out_T", C.c_void_p), ("leaf_mark", C.c_void_p), ("stats", C.c_void_p),
                ("events", C.c_void_p * 3)]


class FrameTree(C.Structure):
    _fields_ = [("n_leaves", C.c_uint32), ("leaf_depth", C.c_void_p), ("leaf_xyz", C.c_void_p),
                ("values", C.c_void_p)]


class Decoder(C.Structure):
    _fields_ = [("w1", C.c_void_p), ("b1", C.c_void_p), ("w2", C.c_void_p), ("b2", C.c_void_p),
                ("w3", C.c_void_p), ("b3", C.c_void_p)]


class Mlp(C.Structure):
    _fields_ = [("w1", C.c_void_p), ("b1", C.c_void_p), ("w2", C.c_void_p), ("b2", C.c_void_p),
                ("w3", C.c_void_p), ("b3", C.c_void_p)]


class TreeInfo(C.Structure):
    _fields_ = [("n_leaves", C.c_uint32), ("n_nodes", C.c_uint32), ("max_depth", C.c_uint32),
                ("n_smem_nodes", C.c_uint32), ("node_bytes", C.c_uint64),
                ("leaf_bytes", C.c_uint64), ("leaf_record_bytes", C.c_uint64),
                ("table_bytes", C.c_uint64)]


_lib = None


def lib():
    """Loads libfpo.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libfpo.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.fpo_create.argtypes = [C.POINTER(P), C.POINTER(Config)]
        L.fpo_validate_tree.argtypes = [C.POINTER(TreeDesc), C.POINTER(Config)]
        L.fpo_upload_tree.argtypes = [P, C.POINTER(TreeDesc)]
        L.fpo_render.argtypes = [P, C.POINTER(Rays), C.POINTER(FrameOpts), P, P]
        L.fpo_render_backward.argtypes = [P, C.POINTER(Rays), C.POINTER(FrameOpts), P, P, P, P]
        L.fpo_render_noalloc.argtypes = [P, C.POINTER(Rays), C.POINTER(FrameOpts), P, P]
        L.fpo_set_coeffs.argtypes = [P, P, P]
        L.fpo_dft_leaves.argtypes = [C.c_int32, C.c_int32, C.c_uint32, C.c_uint32, P, P, P, C.c_uint32, P]
        L.fpo_latent_table.argtypes = [C.POINTER(Decoder), C.c_int32, C.c_int32, C.c_double,
                                       C.c_double, C.c_uint32, P, P, P, P]
        L.fpo_decoder_grad.argtypes = [C.POINTER(Mlp), C.c_int32, C.c_int32, C.c_uint32, P, P, P, P,
                                       P, C.POINTER(Mlp), P, P, P]
        L.fpo_decoder_grad_tc.argtypes = [C.POINTER(Mlp), C.c_int32, C.c_int32, C.c_uint32, P, P, P, P,
                                          P, C.POINTER(Mlp), P, P, P, C.c_uint32, P]
        L.fpo_decoder_forward.argtypes = [C.POINTER(Mlp), C.c_int32, C.c_int32, C.c_uint32, P, P, P]
        L.fpo_set_coeffs_from_decoder.argtypes = [P, C.POINTER(Mlp), P, C.c_uint32, P]
        L.fpo_fma_peak.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, P, C.POINTER(C.c_double), P]
        L.fpo_adam.argtypes = [P, P, P, P, C.c_uint64, P, C.c_uint32, C.c_float, C.c_float,
                               C.c_float, C.c_float, C.c_uint32, P]
        L.fpo_set_latents.argtypes = [P, P, C.POINTER(Decoder), P]
        L.fpo_render_frames.argtypes = [P, P, C.c_uint32, C.POINTER(FrameOpts), P, P, P]
        L.fpo_adam_leaves.argtypes = [P, P, P, P, P, P, C.c_float, C.c_float, C.c_float, C.c_float,
                                      C.c_uint32, P]
        L.fpo_union_trees.argtypes = [C.c_uint32, P, C.c_uint32, C.POINTER(C.c_uint32), P, P, P,
                                      C.c_uint32]
        L.fpo_status_sync.argtypes = [P, P]
        L.fpo_tree_info_get.argtypes = [P, C.POINTER(TreeInfo)]
        L.fpo_destroy.argtypes = [P]
        L.fpo_destroy.restype = None
        L.fpo_last_error.restype = C.c_char_p
        L.fpo_last_error.argtypes = []
        L.fpo_version.argtypes = []
        _lib = L
    return _lib


DFT_STATUS_DEVICE_TIMEOUT = 4  # the bit fpo_dft_leaves ORs into its status word


def check_status_word(status, stream=None):
    """Waits for the stream and raises FPOError if a fpo_dft_leaves status
    word (CUDA int32 [1]) reports a device-side time-out."""
    import torch

    (stream or torch.cuda.current_stream()).synchronize()
    if int(status.item()) & DFT_STATUS_DEVICE_TIMEOUT:
        raise FPOError(-9, "a device-side wait of the per-leaf DFT gave up after its time limit")


def check(code: int):
    if code != FPO_OK:
        raise FPOError(code, lib().fpo_last_error().decode())
    return code


def make_config(n1=31, n2=5, period_T=60.0, storage="f32", idft_mode="auto", device=0,
                traverse_threads=0, refill_min=0, inner_steps=0, table="auto", max_steps=0):
    return Config(n1, n2, 2, float(period_T), STORAGE[storage], IDFT[idft_mode], device,
                  traverse_threads, refill_min, inner_steps, TABLE[table], max_steps)


def make_tree_desc(leaf_depth, leaf_xyz, coeffs, max_depth, aabb_min=(0.0, 0.0, 0.0),
                   aabb_size=1.0):
    """Returns (TreeDesc, keepalive) for host numpy arrays."""
    d = np.ascontiguousarray(leaf_depth, np.uint8)
    x = np.ascontiguousarray(leaf_xyz, np.uint32).reshape(-1, 3)
    c = np.ascontiguousarray(coeffs, np.float32)
    desc = TreeDesc(d.shape[0], int(max_depth), d.ctypes.data, x.ctypes.data, c.ctypes.data,
                    (C.c_double * 3)(*aabb_min), float(aabb_size))
    return desc, (d, x, c)


def validate_tree(tree, n1=31, n2=5) -> None:
    """Host-only validation (no GPU needed); raises FPOError."""
    desc, keep = make_tree_desc(tree.leaf_depth, tree.leaf_xyz, tree.coeffs, tree.max_depth,
                                tree.aabb_min, tree.aabb_size)
    cfg = make_config(n1, n2)
    check(lib().fpo_validate_tree(C.byref(desc), C.byref(cfg)))
    del keep


def _stream_handle(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Renderer:
    """One fpo_ctx: a tree resident on one GPU, rendered frame by frame."""

    def __init__(self, n1=31, n2=5, period_T=60.0, storage="f32", idft_mode="auto", device=0,
                 traverse_threads=0, refill_min=0, inner_steps=0, table="auto", max_steps=0):
        """table: precision of the per-frame table ("auto": FP32 with FP32
        storage, FP16 with the reduced-precision and latent storages)."""
        self.cfg = make_config(n1, n2, period_T, storage, idft_mode, device, traverse_threads,
                               refill_min, inner_steps, table, max_steps)
        self.device = device
        self.n1, self.n2 = n1, n2
        h = C.c_void_p()
        check(lib().fpo_create(C.byref(h), C.byref(self.cfg)))
        self.h = h
        self.n_leaves = 0

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().fpo_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def upload(self, tree):
        desc, keep = make_tree_desc(tree.leaf_depth, tree.leaf_xyz, tree.coeffs, tree.max_depth,
                                    tree.aabb_min, tree.aabb_size)
        check(lib().fpo_upload_tree(self.h, C.byref(desc)))
        self.n_leaves = int(desc.n_leaves)
        del keep

    def info(self) -> dict:
        inf = TreeInfo()
        check(lib().fpo_tree_info_get(self.h, C.byref(inf)))
        return {k: int(getattr(inf, k)) for k, _ in TreeInfo._fields_}

    def status(self, stream=None):
        """Waits for the stream and raises FPOError on a device-side error."""
        check(lib().fpo_status_sync(self.h, C.c_void_p(_stream_handle(stream))))

    def render(self, camera=None, t=0.0, rays_o=None, rays_d=None, t_per_ray=None,
               bg=(1.0, 1.0, 1.0), stop_T=1e-4, out=None, visit_cap=None, want_T=False,
               leaf_mark=None, stats=None, stream=None, events=None, reuse_table=False,
               test_timeout=False):
        """Renders one frame; returns a dict of device tensors.

        camera: an object with eye/target/up/fov_y_deg/width/height (pixel
        index = row * width + column), or explicit rays as CUDA float32
        tensors rays_o, rays_d [n, 3] and optional t_per_ray [n].
        visit_cap: if not None, also returns visit_log [n, cap] and
        visit_count [n] (leaf ids in upload order).  leaf_mark: optional CUDA
        uint8 tensor [n_leaves] set to 1 for visited leaves.  reuse_table:
        skip the IDFT pass when the last table was built for the same t.
        test_timeout: the failure-path test (FPO_FLAG_TEST_DEVICE_TIMEOUT).
        """
        import torch

        dev = torch.device("cuda", self.device)
        r, keep, n = self._rays(camera, t, rays_o, rays_d, t_per_ray)
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float32, device=dev)
        return self._render_into(r, keep, n, out, bg, stop_T, visit_cap, want_T, leaf_mark, stats,
                                 stream, events, reuse_table, test_timeout)

    def _rays(self, camera, t, rays_o, rays_d, t_per_ray):
        import torch

        dev = torch.device("cuda", self.device)
        r = Rays()
        keep = []
        if camera is not None:
            r.mode = RAYS_CAMERA
            r.eye = (C.c_double * 3)(*camera.eye)
            r.target = (C.c_double * 3)(*camera.target)
            r.up = (C.c_double * 3)(*camera.up)
            r.fov_y_deg = float(camera.fov_y_deg)
            r.width, r.height = int(camera.width), int(camera.height)
            n = int(camera.width) * int(camera.height)
        else:
            o = rays_o.to(dev, torch.float32).contiguous()
            d = rays_d.to(dev, torch.float32).contiguous()
            keep += [o, d]
            r.mode = RAYS_EXPLICIT
            n = o.shape[0]
            r.n = n
            r.o, r.d = o.data_ptr() if n else None, d.data_ptr() if n else None
            if t_per_ray is not None:
                tp = t_per_ray.to(dev, torch.float32).contiguous()
                keep.append(tp)
                r.t_per_ray = tp.data_ptr() if n else None
        r.t = float(t)
        return r, keep, n

    def _render_into(self, r, keep, n, out, bg, stop_T, visit_cap, want_T, leaf_mark, stats,
                     stream, events, reuse_table=False, test_timeout=False):
        import torch

        dev = torch.device("cuda", self.device)
        res = {"rgb": out}
        opts = FrameOpts()
        opts.bg = (C.c_float * 3)(*bg)
        opts.stop_T = float(stop_T)
        flags = 0
        if visit_cap is not None:
            res["visit_log"] = torch.full((n, max(visit_cap, 1)), -1, dtype=torch.int32, device=dev)
            res["visit_count"] = torch.zeros(n, dtype=torch.int32, device=dev)
            opts.visit_log = res["visit_log"].data_ptr()
            opts.visit_cap = int(visit_cap)
            opts.visit_count = res["visit_count"].data_ptr()
            flags |= FLAG_RECORD_VISITS
        if want_T:
            res["T"] = torch.empty(n, dtype=torch.float32, device=dev)
            opts.out_T = res["T"].data_ptr()
            flags |= FLAG_OUT_T
        if leaf_mark is not None:
            opts.leaf_mark = leaf_mark.data_ptr()
            flags |= FLAG_MARK_LEAVES
        if stats is not None:  # CUDA int64 tensor [3], accumulated
            opts.stats = stats.data_ptr()
            flags |= FLAG_STATS
        if reuse_table:
            flags |= FLAG_REUSE_TABLE
        if test_timeout:
            flags |= FLAG_TEST_DEVICE_TIMEOUT
        opts.flags = flags
        if events is not None:
            for i, ev in enumerate(events):
                if ev is None:
                    continue
                if not ev.cuda_event:  # torch creates the CUDA event at its first record
                    ev.record(stream)
                opts.events[i] = ev.cuda_event
        check(lib().fpo_render(self.h, C.byref(r), C.byref(opts),
                               C.c_void_p(out.data_ptr() if n else None),
                               C.c_void_p(_stream_handle(stream))))
        res["_keep"] = keep
        return res

    def render_frames(self, cameras, times, bg=(1.0, 1.0, 1.0), stop_T=1e-4, out=None, stream=None,
                      frame_events=None):
        """Renders camera frames (same size) into out [n_frames, W*H, 3] with the
        pipelined fpo_render_frames.  frame_events: optional torch.cuda.Event
        per frame, recorded once that frame's pixels are written."""
        import torch

        n = len(cameras)
        arr = (Rays * max(n, 1))()
        keep = []
        for i, (cam, t) in enumerate(zip(cameras, times)):
            r, k, npx = self._rays(cam, t, None, None, None)
            arr[i] = r
            keep += k
        npx = cameras[0].width * cameras[0].height if n else 0
        if out is None:
            out = torch.empty((n, npx, 3), dtype=torch.float32, device=torch.device("cuda", self.device))
        opts = FrameOpts()
        opts.bg = (C.c_float * 3)(*bg)
        opts.stop_T = float(stop_T)
        done = None
        if frame_events is not None:
            assert len(frame_events) == n
            done = (C.c_void_p * max(n, 1))()
            for i, ev in enumerate(frame_events):
                if ev is None:
                    continue
                if not ev.cuda_event:  # torch creates the CUDA event at its first record
                    ev.record(stream)
                done[i] = ev.cuda_event
        check(lib().fpo_render_frames(self.h, arr, n, C.byref(opts),
                                      C.c_void_p(out.data_ptr() if out.numel() else None),
                                      done, C.c_void_p(_stream_handle(stream))))
        return out

    def set_coeffs(self, coeffs, stream=None):
        """Replaces the tree's coefficients from a CUDA float32 tensor [n_leaves, n1 + 27 n2]."""
        c = coeffs.detach()
        assert c.is_cuda and c.dtype.is_floating_point and c.is_contiguous()
        check(lib().fpo_set_coeffs(self.h, C.c_void_p(c.data_ptr()),
                                   C.c_void_p(_stream_handle(stream))))

    def set_coeffs_from_decoder(self, mlp, latents, stream=None, tensor_cores=False, test_timeout=False):
        """Replaces the tree's coefficients with the decoder's decode of every
        leaf's latent (mlp: an Mlp of FP32 device weights; latents: a CUDA
        float32 tensor [n_leaves, 32] in upload order): in FP32, or with
        tensor_cores on tcgen05 with the inference decoder's FP16 numerics
        (errors then through status())."""
        import torch

        lat = latents.detach()
        assert lat.is_cuda and lat.dtype == torch.float32 and lat.is_contiguous()
        flags = (FLAG_TENSOR_CORES if tensor_cores else 0) | (FLAG_TEST_DEVICE_TIMEOUT if test_timeout else 0)
        check(lib().fpo_set_coeffs_from_decoder(self.h, C.byref(mlp), C.c_void_p(lat.data_ptr()), flags,
                                                C.c_void_p(_stream_handle(stream))))

    def set_latents(self, latents_f16, w1, b1, w2, b2, w3, b3, stream=None):
        """LATENT storage: per-leaf FP16 latents [n_leaves, 32] (CUDA, upload
        order) and the decoder (weights cast to BF16, biases FP32)."""
        import torch

        lat = latents_f16.contiguous()
        assert lat.dtype == torch.float16 and lat.is_cuda
        ws = [w.detach().to(torch.bfloat16).contiguous() for w in (w1, w2, w3)]
        bs = [b.detach().float().contiguous() for b in (b1, b2, b3)]
        dec = Decoder(ws[0].data_ptr(), bs[0].data_ptr(), ws[1].data_ptr(), bs[1].data_ptr(),
                      ws[2].data_ptr(), bs[2].data_ptr())
        check(lib().fpo_set_latents(self.h, C.c_void_p(lat.data_ptr()), C.byref(dec),
                                    C.c_void_p(_stream_handle(stream))))
        torch.cuda.current_stream().synchronize()  # the copies read ws/bs

    def render_backward(self, out_rgb, dL_drgb, dL_dcoeffs, camera=None, t=0.0, rays_o=None,
                        rays_d=None, t_per_ray=None, bg=(1.0, 1.0, 1.0), stop_T=1e-4, leaf_mark=None,
                        stream=None, fp64=False):
        """Accumulates dL/d(coefficients) [n_leaves, n1 + 27 n2] (canonical) into
        dL_dcoeffs; sets leaf_mark[id] = 1 (uint8 CUDA tensor) for visited leaves.
        fp64: the gradient-check replay (dL_dcoeffs is then a float64 tensor)."""
        import torch

        r, keep, n = self._rays(camera, t, rays_o, rays_d, t_per_ray)
        opts = FrameOpts()
        opts.bg = (C.c_float * 3)(*bg)
        opts.stop_T = float(stop_T)
        flags = 0
        if fp64:
            assert dL_dcoeffs.dtype == torch.float64
            flags |= FLAG_FP64_GRADCHECK
        else:
            assert dL_dcoeffs.dtype == torch.float32
        if leaf_mark is not None:
            flags |= FLAG_MARK_LEAVES
            opts.leaf_mark = leaf_mark.data_ptr()
        opts.flags = flags
        g = dL_drgb.contiguous()
        o = out_rgb.contiguous()
        check(lib().fpo_render_backward(self.h, C.byref(r), C.byref(opts),
                                        C.c_void_p(o.data_ptr() if n else None),
                                        C.c_void_p(g.data_ptr() if n else None),
                                        C.c_void_p(dL_dcoeffs.data_ptr()),
                                        C.c_void_p(_stream_handle(stream))))
        del keep


    def adam_leaves(self, param, grad, m, v, leaf_mark, step, lr=1e-2, betas=(0.9, 0.999), eps=1e-8,
                    stream=None):
        """Adam step on the marked leaves' rows, written back into the tree (fpo_adam_leaves)."""
        check(lib().fpo_adam_leaves(self.h, C.c_void_p(param.data_ptr()), C.c_void_p(grad.data_ptr()),
                                    C.c_void_p(m.data_ptr()), C.c_void_p(v.data_ptr()),
                                    C.c_void_p(leaf_mark.data_ptr()), float(lr), float(betas[0]),
                                    float(betas[1]), float(eps), int(step),
                                    C.c_void_p(_stream_handle(stream))))


def union_trees(frames, max_depth):
    """Sec. 4.2 union of per-frame octrees (host).  frames: list of
    (leaf_depth uint8 [n], leaf_xyz uint32 [n, 3], values float32 [n, 28]).
    Returns (depth [m], xyz [m, 3], values [n_frames, m, 28])."""
    keep = []
    arr = (FrameTree * max(len(frames), 1))()
    for i, (d, x, v) in enumerate(frames):
        d = np.ascontiguousarray(d, np.uint8)
        x = np.ascontiguousarray(x, np.uint32).reshape(-1, 3)
        v = np.ascontiguousarray(v, np.float32).reshape(-1, 28)
        keep += [d, x, v]
        arr[i] = FrameTree(d.shape[0], d.ctypes.data, x.ctypes.data, v.ctypes.data)
    n = C.c_uint32(0)
    check(lib().fpo_union_trees(len(frames), arr, int(max_depth), C.byref(n), None, None, None, 0))
    m = n.value
    depth = np.zeros(m, np.uint8)
    xyz = np.zeros((m, 3), np.uint32)
    vals = np.zeros((len(frames), m, 28), np.float32)
    if m:
        check(lib().fpo_union_trees(len(frames), arr, int(max_depth), C.byref(n), depth.ctypes.data,
                                    xyz.ctypes.data, vals.ctypes.data, m))
    return depth, xyz, vals


def latent_table(latents, w1, b1, w2, b2, w3, b3, t, period_T=60.0, n1=31, n2=5, stream=None):
    """Per-frame table [n, 32] from FP16 latents [n, 32] and a BF16 MLP (tcgen05)."""
    import torch

    lat = latents.contiguous()
    assert lat.dtype == torch.float16 and lat.is_cuda and lat.shape[1] == 32
    ws = [w.to(torch.bfloat16).contiguous() for w in (w1, w2, w3)]
    bs = [b.float().contiguous() for b in (b1, b2, b3)]
    dec = Decoder(ws[0].data_ptr(), bs[0].data_ptr(), ws[1].data_ptr(), bs[1].data_ptr(),
                  ws[2].data_ptr(), bs[2].data_ptr())
    n = lat.shape[0]
    out = torch.empty((n, 32), dtype=torch.float32, device=lat.device)
    status = torch.zeros(1, dtype=torch.int32, device=lat.device)
    check(lib().fpo_latent_table(C.byref(dec), n1, n2, float(t), float(period_T), n,
                                 C.c_void_p(lat.data_ptr() if n else None),
                                 C.c_void_p(out.data_ptr() if n else None),
                                 C.c_void_p(status.data_ptr()), C.c_void_p(_stream_handle(stream))))
    return out, status


def fma_peak_tflops(iters=4096, reps=5):
    """The device's FP32 FMA rate (TFLOP/s, best of `reps` launches of
    fpo_fma_peak: two 1024-thread CTAs per SM), timed with CUDA events."""
    import torch

    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks, threads = 2 * sms, 1024
    sink = torch.empty(blocks * threads, device="cuda")
    flops = C.c_double(0.0)
    best = float("inf")
    for rep in range(reps + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        check(lib().fpo_fma_peak(blocks, threads, iters, C.c_void_p(sink.data_ptr()), C.byref(flops),
                                 C.c_void_p(_stream_handle(None))))
        b.record()
        torch.cuda.synchronize()
        if rep:  # the first launch warms up
            best = min(best, a.elapsed_time(b))
    return flops.value / (best * 1e-3) / 1e12


def dft_leaves(values, n1=31, n2=5, stream=None, out=None, status=None, test_timeout=False):
    """Eq. 10-12 on the GPU: values [T, n_leaves, 28] (CUDA float32) ->
    coefficients [n_leaves, n1 + 27 n2] (canonical), into `out` if given
    (a contiguous CUDA float32 tensor of that shape).  status: a CUDA int32
    tensor of one element that a timed-out copy wait ORs its bit into (the
    caller reads it after the stream); without one the call waits for the
    stream and raises FPOError(FPO_ERR_DEVICE_TIMEOUT) itself."""
    import torch

    v = values.contiguous()
    T, n, w = v.shape
    assert w == 28 and v.is_cuda and v.dtype == torch.float32
    if out is None:
        out = torch.empty((n, n1 + 27 * n2), dtype=torch.float32, device=v.device)
    assert out.shape == (n, n1 + 27 * n2) and out.dtype == torch.float32 and out.is_cuda and out.is_contiguous()
    own = status is None
    if own:
        status = torch.zeros(1, dtype=torch.int32, device=v.device)
    assert status.is_cuda and status.dtype == torch.int32 and status.numel() == 1
    check(lib().fpo_dft_leaves(n1, n2, T, n, C.c_void_p(v.data_ptr() if n else None),
                               C.c_void_p(out.data_ptr() if n else None), C.c_void_p(status.data_ptr()),
                               FLAG_TEST_DEVICE_TIMEOUT if test_timeout else 0,
                               C.c_void_p(_stream_handle(stream))))
    if own:
        check_status_word(status, stream)
    return out


def _autograd_function():
    import torch

    class FPORender(torch.autograd.Function):
        """Differentiable render of explicit rays with respect to the leaf
        coefficients (canonical [n_leaves, n1 + 27 n2]): forward sets them and
        renders through fpo_render, backward calls fpo_render_backward."""

        @staticmethod
        def forward(ctx, coeffs, renderer, rays_o, rays_d, t_per_ray, bg, stop_T):
            renderer.set_coeffs(coeffs)
            rgb = renderer.render(rays_o=rays_o, rays_d=rays_d, t_per_ray=t_per_ray, bg=bg,
                                  stop_T=stop_T)["rgb"]
            ctx.renderer, ctx.bg, ctx.stop_T = renderer, bg, stop_T
            ctx.shape = coeffs.shape
            ctx.save_for_backward(rays_o, rays_d, t_per_ray, rgb)
            return rgb

        @staticmethod
        def backward(ctx, g):
            rays_o, rays_d, t_per_ray, rgb = ctx.saved_tensors
            grad = torch.zeros(ctx.shape, dtype=torch.float32, device=g.device)
            ctx.renderer.render_backward(rgb, g.float(), grad, rays_o=rays_o, rays_d=rays_d,
                                         t_per_ray=t_per_ray, bg=ctx.bg, stop_T=ctx.stop_T)
            return grad, None, None, None, None, None, None

    return FPORender


_FPORender = None


def render_rays(coeffs, renderer, rays_o, rays_d, t_per_ray, bg=(1.0, 1.0, 1.0), stop_T=1e-4):
    """Differentiable render: rgb [n, 3] of explicit rays, gradients to `coeffs`."""
    global _FPORender
    if _FPORender is None:
        _FPORender = _autograd_function()
    return _FPORender.apply(coeffs, renderer, rays_o, rays_d, t_per_ray, tuple(bg), float(stop_T))
