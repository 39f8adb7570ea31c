"""FP64 CPU oracle for Fourier PlenOctree rendering (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product path never imports this
package.  The C source (fpo_oracle.c) is plain FP64 code written from the
paper's definitions; it shares nothing with the CUDA library.

Functions and the passages they follow (Wang et al., CVPR 2022):
  basis(n, t, T)     Eq. 8, the real Fourier basis IDFT_i(t)            (Sec. 4.1)
  sh(d, degree)      Eq. 1, real SH Y_{m,l}(d), l <= 2                  (Sec. 3)
  render(...)        Eq. 7, 9 and 1 per leaf segment, then
                     emission-absorption compositing with early stop   (Sec. 4.1, 3)
  render_grad(...)   dL/d(coefficients) of render for a given dL/d(rgb):
                     the back-propagation of the fine-tuning stage     (Sec. 4.3, Eq. 13)
  dft(x, n)          per-series DFT of frames t = 1..T                 (Sec. 4.2, Eq. 10-12)
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fpo_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (FP64, no FMA contraction, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                           "-pthread", "-ffp-contract=off", "-Wall", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Scene(C.Structure):
    _fields_ = [("n1", C.c_int32), ("n2", C.c_int32), ("sh_degree", C.c_int32),
                ("period_T", C.c_double), ("coeffs", C.c_void_p),
                ("aabb_min", C.c_double * 3), ("aabb_size", C.c_double),
                ("bg", C.c_double * 3), ("stop_T", C.c_double)]


class Rays(C.Structure):
    _fields_ = [("mode", C.c_int32), ("eye", C.c_double * 3), ("target", C.c_double * 3),
                ("up", C.c_double * 3), ("fov_y_deg", C.c_double),
                ("width", C.c_int32), ("height", C.c_int32), ("t", C.c_double),
                ("n", C.c_int64), ("o", C.c_void_p), ("d", C.c_void_p),
                ("t_per_ray", C.c_void_p), ("n_sel", C.c_int64), ("sel", C.c_void_p)]


class Out(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("T", C.c_void_p), ("visit_log", C.c_void_p),
                ("visit_cap", C.c_uint32), ("visit_count", C.c_void_p),
                ("visit_delta", C.c_void_p), ("visit_weight", C.c_void_p),
                ("flags", C.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        L.oracle_basis.argtypes = [C.c_int, C.c_double, C.c_double, C.c_void_p]
        L.oracle_sh.argtypes = [C.c_int, C.c_void_p, C.c_void_p]
        L.oracle_tree_new.restype = C.c_void_p
        L.oracle_tree_new.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                      C.POINTER(C.c_int)]
        L.oracle_tree_free.argtypes = [C.c_void_p]
        L.oracle_render.argtypes = [C.c_void_p, C.POINTER(Scene), C.POINTER(Rays),
                                    C.POINTER(Out), C.c_int]
        L.oracle_render_grad.argtypes = [C.c_void_p, C.POINTER(Scene), C.POINTER(Rays),
                                         C.c_void_p, C.c_void_p]
        L.oracle_dft.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def basis(n: int, t: float, period: float = 60.0) -> np.ndarray:
    """Eq. 8: [IDFT_0(t) .. IDFT_{n-1}(t)] in FP64."""
    out = np.empty(n, np.float64)
    if lib().oracle_basis(n, float(t), float(period), _ptr(out)) != 0:
        raise ValueError("bad basis arguments")
    return out


def sh(d, degree: int = 2) -> np.ndarray:
    """Eq. 1: real SH values Y_k(d), k = l(l+1)+m, for a unit vector d."""
    dd = np.ascontiguousarray(d, np.float64)
    out = np.zeros(9, np.float64)
    if lib().oracle_sh(degree, _ptr(dd), _ptr(out)) != 0:
        raise ValueError("bad SH arguments")
    return out[: (degree + 1) ** 2]


class OracleTree:
    """The oracle's own octree built from a leaf list (validated)."""

    def __init__(self, leaf_depth, leaf_xyz, max_depth: int):
        self.leaf_depth = np.ascontiguousarray(leaf_depth, np.uint8)
        self.leaf_xyz = np.ascontiguousarray(leaf_xyz, np.uint32).reshape(-1, 3)
        st = C.c_int(0)
        self.h = lib().oracle_tree_new(self.leaf_depth.shape[0], int(max_depth),
                                       _ptr(self.leaf_depth), _ptr(self.leaf_xyz), C.byref(st))
        self.status = st.value
        if not self.h:
            raise ValueError(f"oracle rejected the tree (status {st.value})")

    def __del__(self):
        if getattr(self, "h", None):
            lib().oracle_tree_free(self.h)
            self.h = None


def render(tree, coeffs, *, n1=31, n2=5, sh_degree=2, period=60.0, aabb_min=(0, 0, 0),
           aabb_size=1.0, bg=(1.0, 1.0, 1.0), stop_T=1e-4, camera=None, t=0.0, rays_o=None,
           rays_d=None, t_per_ray=None, sel=None, visit_cap=0, want_delta=False,
           want_weight=False, threads=None):
    """Renders with the FP64 oracle.

    tree: an OracleTree.  coeffs: float32 [n_leaves, n1 + 3*(deg+1)^2*n2]
    canonical.  Either `camera` (object with eye/target/up/fov_y_deg/width/
    height) or explicit rays (rays_o, rays_d [n, 3]).  `sel` renders a subset
    of ray (pixel) indices.  Returns a dict with rgb [n,3], T [n], flags [n]
    and, when visit_cap > 0, visit_log [n, cap] and visit_count [n].
    """
    sc, r, keep, n = _setup(coeffs, n1, n2, sh_degree, period, aabb_min, aabb_size, bg, stop_T,
                            camera, t, rays_o, rays_d, t_per_ray, sel)
    L = lib()
    res = {"rgb": np.zeros((n, 3), np.float64), "T": np.zeros(n, np.float64),
           "flags": np.zeros(n, np.uint8)}
    o = Out(_ptr(res["rgb"]), _ptr(res["T"]), None, 0, None, None, None, _ptr(res["flags"]))
    if visit_cap:
        res["visit_log"] = np.full((n, visit_cap), 0xFFFFFFFF, np.uint32)
        res["visit_count"] = np.zeros(n, np.uint32)
        o.visit_log, o.visit_cap = _ptr(res["visit_log"]), visit_cap
        o.visit_count = _ptr(res["visit_count"])
        if want_delta:
            res["visit_delta"] = np.zeros((n, visit_cap), np.float64)
            o.visit_delta = _ptr(res["visit_delta"])
        if want_weight:
            res["visit_weight"] = np.zeros((n, visit_cap), np.float64)
            o.visit_weight = _ptr(res["visit_weight"])
    if threads is None:
        threads = os.cpu_count() or 1
    st = L.oracle_render(tree.h, C.byref(sc), C.byref(r), C.byref(o), int(threads))
    if st != 0:
        raise RuntimeError(f"oracle_render failed with status {st}")
    return res


def render_grad(tree, coeffs, dL_drgb, *, n1=31, n2=5, sh_degree=2, period=60.0,
                aabb_min=(0, 0, 0), aabb_size=1.0, bg=(1.0, 1.0, 1.0), stop_T=1e-4, camera=None,
                t=0.0, rays_o=None, rays_d=None, t_per_ray=None, sel=None):
    """Sec. 4.3: dL/dk [n_leaves, ncoef] (FP64, canonical order) for dL/drgb [n, 3]."""
    sc, r, keep, n = _setup(coeffs, n1, n2, sh_degree, period, aabb_min, aabb_size, bg, stop_T,
                            camera, t, rays_o, rays_d, t_per_ray, sel)
    g = np.ascontiguousarray(dL_drgb, np.float64).reshape(n, 3)
    coeffs = keep[0]
    grad = np.zeros(coeffs.shape, np.float64)
    st = lib().oracle_render_grad(tree.h, C.byref(sc), C.byref(r), _ptr(g), _ptr(grad))
    if st != 0:
        raise RuntimeError(f"oracle_render_grad failed with status {st}")
    return grad


def dft(x, n_coef: int) -> np.ndarray:
    """Eq. 10-12: x [T, n_series] sampled at frames 1..T -> k [n_series, n_coef] (FP64)."""
    x = np.ascontiguousarray(x, np.float64)
    if x.ndim == 1:
        x = x[:, None]
    T, ns = x.shape
    k = np.zeros((ns, n_coef), np.float64)
    if lib().oracle_dft(T, ns, _ptr(x), n_coef, _ptr(k)) != 0:
        raise ValueError("bad DFT arguments")
    return k


def _setup(coeffs, n1, n2, sh_degree, period, aabb_min, aabb_size, bg, stop_T, camera, t,
           rays_o, rays_d, t_per_ray, sel):
    coeffs = np.ascontiguousarray(coeffs, np.float32)
    sc = Scene(n1, n2, sh_degree, float(period), _ptr(coeffs) if coeffs.size else None,
               (C.c_double * 3)(*aabb_min), float(aabb_size), (C.c_double * 3)(*bg),
               float(stop_T))
    keep = [coeffs]
    r = Rays()
    if camera is not None:
        r.mode = 0
        r.eye = (C.c_double * 3)(*camera.eye)
        r.target = (C.c_double * 3)(*camera.target)
        r.up = (C.c_double * 3)(*camera.up)
        r.fov_y_deg = float(camera.fov_y_deg)
        r.width, r.height = int(camera.width), int(camera.height)
        n_all = int(camera.width) * int(camera.height)
    else:
        o = np.ascontiguousarray(rays_o, np.float64).reshape(-1, 3)
        d = np.ascontiguousarray(rays_d, np.float64).reshape(-1, 3)
        keep += [o, d]
        r.mode = 1
        r.n = o.shape[0]
        r.o, r.d = _ptr(o), _ptr(d)
        if t_per_ray is not None:
            tp = np.ascontiguousarray(t_per_ray, np.float64)
            keep.append(tp)
            r.t_per_ray = _ptr(tp)
        n_all = o.shape[0]
    r.t = float(t)
    if sel is not None:
        s = np.ascontiguousarray(sel, np.int64)
        keep.append(s)
        r.n_sel, r.sel = s.shape[0], _ptr(s)
        n = s.shape[0]
    else:
        n = n_all
    return sc, r, keep, n
