"""Seeded synthetic inputs for Fourier PlenOctree rendering.

This module only draws inputs: leaf cells of union octrees, Fourier
coefficients and camera parameters.  It holds none of the rendering
arithmetic (no basis, no spherical harmonics, no ray generation, no
compositing), so the CUDA path and the FP64 oracle can both consume what it
produces without sharing any of the method.

Shapes follow the paper's FPO setting: a union octree over the unit cube with
leaves at depth up to 9 (a 512^3 grid, Sec. 5), per leaf n1 = 31 density
Fourier coefficients and n2 = 5 Fourier coefficients for each of the
(l_max+1)^2 * 3 = 27 SH coefficients with l_max = 2 (Sec. 4.1, Eq. 6; Tab. 3).

Canonical coefficient order of one leaf (used at the library boundary):
``[k_sigma_0 .. k_sigma_{n1-1}] [c = 0..2][k = 0..8][i = 0..n2-1]`` with the SH
index k = l(l+1) + m.

Every generator takes an explicit seed and uses numpy's PCG64
(``numpy.random.default_rng``).  Draw order is fixed and documented per
function so that a tree can be regenerated bit-for-bit.
"""

from __future__ import annotations

import dataclasses
import math
import os

import numpy as np

N_SH = 9  # (l_max + 1)^2 with l_max = 2
PERIOD_T = 60.0  # frames in the sequence; the IDFT period (Eq. 8)


@dataclasses.dataclass
class Tree:
    """A union octree described by its leaves (what the library uploads)."""

    leaf_depth: np.ndarray  # uint8 [n]
    leaf_xyz: np.ndarray  # uint32 [n, 3], integer cell coordinates at leaf_depth
    coeffs: np.ndarray  # float32 [n, n1 + 3 * 9 * n2], canonical order
    max_depth: int
    n1: int = 31
    n2: int = 5
    aabb_min: tuple = (0.0, 0.0, 0.0)
    aabb_size: float = 1.0

    @property
    def n_leaves(self) -> int:
        return int(self.leaf_depth.shape[0])

    @property
    def n_coeffs(self) -> int:
        return self.n1 + 3 * N_SH * self.n2


@dataclasses.dataclass
class Camera:
    """Pinhole camera: eye, look-at target, up vector, vertical field of view."""

    eye: tuple
    target: tuple = (0.5, 0.5, 0.5)
    up: tuple = (0.0, 0.0, 1.0)
    fov_y_deg: float = 40.0
    width: int = 128
    height: int = 128


# --------------------------------------------------------------------------
# coefficients


def draw_coefficients(rng: np.random.Generator, n: int, n1: int = 31, n2: int = 5) -> np.ndarray:
    """I.i.d. Fourier coefficients in canonical order, float32 [n, n1 + 27*n2].

    Density: k_sigma_0 ~ U(0, 50); k_sigma_i ~ N(0, 5/(i+1)) for i >= 1.
    SH: k_{c,k,0} ~ N(0, 0.5); k_{c,k,i} ~ N(0, 0.2/(i+1)) for i >= 1.
    The second argument of N(.,.) is the standard deviation.
    Draw order: the n density DC values, then the n x (n1-1) density
    terms, then the n x 3 x 9 x n2 SH terms (all standard normals, scaled).
    """
    out = np.empty((n, n1 + 3 * N_SH * n2), dtype=np.float32)
    out[:, 0] = rng.uniform(0.0, 50.0, size=n).astype(np.float32)
    if n1 > 1:
        std = (5.0 / (np.arange(1, n1) + 1.0)).astype(np.float32)
        out[:, 1:n1] = rng.standard_normal((n, n1 - 1), dtype=np.float32) * std
    std_z = np.empty(n2, dtype=np.float32)
    std_z[0] = 0.5
    if n2 > 1:
        std_z[1:] = 0.2 / (np.arange(1, n2) + 1.0)
    z = rng.standard_normal((n, 3, N_SH, n2), dtype=np.float32) * std_z
    out[:, n1:] = z.reshape(n, -1)
    return out


def draw_coefficients_blocked(seed: int, n: int, n1: int = 31, n2: int = 5,
                              block: int = 1 << 16, workers: int | None = None) -> np.ndarray:
    """Same distributions as draw_coefficients for large n, drawn in blocks.

    Leaves [b * block, (b + 1) * block) come from
    draw_coefficients(default_rng(SeedSequence(seed, spawn_key=(b,))), ...);
    blocks are independent, so the result does not depend on `workers`.
    """
    import concurrent.futures as cf

    out = np.empty((n, n1 + 3 * N_SH * n2), dtype=np.float32)
    nblk = (n + block - 1) // block

    def one(b):
        lo, hi = b * block, min(n, (b + 1) * block)
        rng = np.random.default_rng(np.random.SeedSequence(seed, spawn_key=(b,)))
        out[lo:hi] = draw_coefficients(rng, hi - lo, n1, n2)

    with cf.ThreadPoolExecutor(workers or min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(one, range(nblk)))
    return out


# --------------------------------------------------------------------------
# leaf sets


def morton_key(xyz: np.ndarray, depth: int) -> np.ndarray:
    """Interleaved-bit (Morton) key of integer cell coordinates, x lowest."""
    key = np.zeros(xyz.shape[0], dtype=np.uint64)
    for b in range(depth):
        for a in range(3):
            bit = (xyz[:, a].astype(np.uint64) >> np.uint64(b)) & np.uint64(1)
            key |= bit << np.uint64(3 * b + a)
    return key


def shell_leaves(depth: int = 5, r_in: float = 0.30, r_out: float = 0.40):
    """Cells at `depth` whose centre lies at distance [r_in, r_out] from the
    cube centre, sorted by Morton key.  Returns uint32 [n, 3]."""
    g = 1 << depth
    ax = (np.arange(g) + 0.5) / g
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    m = (r >= r_in) & (r <= r_out)
    idx = np.argwhere(m).astype(np.uint32)
    order = np.argsort(morton_key(idx, depth), kind="stable")
    return idx[order]


def random_mixed_leaves(rng: np.random.Generator, max_depth: int = 4, p_split: float = 0.55,
                        p_empty: float = 0.35, min_depth: int = 1):
    """Random union octree with leaves at mixed depths (disjoint by construction).

    Recursive subdivision from the root: a cell at depth < max_depth splits
    with probability p_split (always below min_depth); an unsplit cell is
    empty with probability p_empty, else a leaf.  Returns (depth uint8 [n],
    xyz uint32 [n, 3]) in depth-first order.
    """
    depths, coords = [], []

    def rec(d, x, y, z):
        if d < max_depth and (d < min_depth or rng.random() < p_split):
            for c in range(8):
                rec(d + 1, 2 * x + (c & 1), 2 * y + ((c >> 1) & 1), 2 * z + ((c >> 2) & 1))
            return
        if d > 0 and rng.random() < p_empty:
            return
        depths.append(d)
        coords.append((x, y, z))

    rec(0, 0, 0, 0)
    return np.array(depths, dtype=np.uint8), np.array(coords, dtype=np.uint32).reshape(-1, 3)


def _segment_dist(p, a, b):
    """Distance from points p [..., 3] to segments a-b ([F, 3] broadcast)."""
    ab = b - a
    ap = p - a
    t = np.clip(np.sum(ap * ab, axis=-1) / np.sum(ab * ab, axis=-1), 0.0, 1.0)
    q = ap - t[..., None] * ab
    return np.sqrt(np.sum(q * q, axis=-1))


# Base figure for the animated body: 14 capsules between joint positions.
_JOINTS = {
    "head_top": (0.50, 0.50, 0.78), "neck": (0.50, 0.50, 0.67),
    "chest": (0.50, 0.50, 0.60), "pelvis": (0.50, 0.50, 0.45),
    "sh_l": (0.39, 0.50, 0.62), "sh_r": (0.61, 0.50, 0.62),
    "el_l": (0.31, 0.48, 0.51), "el_r": (0.69, 0.48, 0.51),
    "wr_l": (0.27, 0.44, 0.40), "wr_r": (0.73, 0.44, 0.40),
    "hip_l": (0.45, 0.50, 0.44), "hip_r": (0.55, 0.50, 0.44),
    "kn_l": (0.43, 0.47, 0.32), "kn_r": (0.57, 0.47, 0.32),
    "an_l": (0.43, 0.51, 0.21), "an_r": (0.57, 0.51, 0.21),
    "toe_l": (0.43, 0.40, 0.20), "toe_r": (0.57, 0.40, 0.20),
}
_BONES = [
    ("head_top", "neck"), ("chest", "pelvis"), ("sh_l", "sh_r"),
    ("sh_l", "el_l"), ("sh_r", "el_r"), ("el_l", "wr_l"), ("el_r", "wr_r"),
    ("hip_l", "hip_r"), ("hip_l", "kn_l"), ("hip_r", "kn_r"),
    ("kn_l", "an_l"), ("kn_r", "an_r"), ("an_l", "toe_l"), ("an_r", "toe_r"),
]
# capsule radii per bone, all within [0.02, 0.08]
_RADII = (0.06, 0.08, 0.04, 0.035, 0.035, 0.03, 0.03, 0.05, 0.05, 0.05, 0.04, 0.04, 0.02, 0.02)


def capsule_body(rng: np.random.Generator, n_frames: int = 60, period: float = PERIOD_T,
                 amp_lo: float = 0.01, amp_hi: float = 0.04):
    """Animated 14-capsule body (radii 0.02..0.08 per bone, fixed table).

    Draw order: per capsule and endpoint (14 x 2) per-axis amplitudes
    A ~ U(amp_lo, amp_hi), then phases ~ U(0, 2 pi).
    Endpoint p(f) = p0 + A * sin(2 pi f / period + phase), f = 0..n_frames-1.
    With the defaults the depth-9 union over 60 frames has about 3.5M cells.
    Returns (a [14, F, 3], b [14, F, 3], radii [14]) in float64.
    """
    radii = np.array(_RADII, dtype=np.float64)
    amp = rng.uniform(amp_lo, amp_hi, size=(len(_BONES), 2, 3))
    phase = rng.uniform(0.0, 2.0 * np.pi, size=(len(_BONES), 2, 3))
    f = np.arange(n_frames, dtype=np.float64)
    s = np.sin(2.0 * np.pi * f[None, None, :, None] / period + phase[:, :, None, :])
    p0 = np.array([[_JOINTS[u], _JOINTS[v]] for u, v in _BONES], dtype=np.float64)
    p = p0[:, :, None, :] + amp[:, :, None, :] * s  # [C, 2, F, 3]
    return p[:, 0], p[:, 1], radii


def capsule_union_leaves(a: np.ndarray, b: np.ndarray, radii: np.ndarray, depth: int = 9,
                         coarse: int = 5):
    """Cells at `depth` whose centre lies inside any capsule at any frame.

    Coarse-to-fine: candidate blocks at level `coarse` are classified per
    frame as fully in (every cell centre inside), fully out, or straddling,
    using the block's centre distance +- the half diagonal spanned by its
    cell centres; straddling blocks are split until `depth`.  The result is
    the exact per-cell test, done on fewer cells.  Returns uint32 [n, 3]
    sorted by Morton key.
    """
    import concurrent.futures as cf

    g = 1 << depth
    occ = np.zeros((g, g, g), dtype=bool)
    h_fine = 1.0 / g

    def one(c):
        A, B, r = a[c], b[c], float(radii[c])
        lo = np.minimum(A.min(0), B.min(0)) - r
        hi = np.maximum(A.max(0), B.max(0)) + r
        gl = 1 << coarse
        i0 = np.clip(np.floor(lo * gl).astype(int), 0, gl - 1)
        i1 = np.clip(np.floor(hi * gl).astype(int), 0, gl - 1)
        rng_axes = [np.arange(i0[k], i1[k] + 1) for k in range(3)]
        cand = np.stack(np.meshgrid(*rng_axes, indexing="ij"), -1).reshape(-1, 3)
        live = np.ones((cand.shape[0], A.shape[0]), dtype=bool)  # frames still undecided
        level = coarse
        while cand.shape[0]:
            h = 1.0 / (1 << level)
            ctr = (cand + 0.5) * h
            span = math.sqrt(3.0) * 0.5 * (h - h_fine)
            dist = np.empty(live.shape)
            for s0 in range(0, cand.shape[0], 1 << 15):
                sl = slice(s0, s0 + (1 << 15))
                dist[sl] = _segment_dist(ctr[sl, None, :], A[None], B[None])
            full = np.any(live & (dist + span <= r), axis=1)
            live = live & ~(dist - span > r)
            # fully covered blocks: mark all their finest cells
            sh = depth - level
            for q in cand[full]:
                x, y, z = (int(v) << sh for v in q)
                occ[x:x + (1 << sh), y:y + (1 << sh), z:z + (1 << sh)] = True
            keep = ~full & np.any(live, axis=1)
            if level == depth:
                break
            cand = cand[keep]
            live = live[keep]
            # split into 8 children
            kids = (cand[:, None, :] * 2 + np.array(
                [[(k >> 0) & 1, (k >> 1) & 1, (k >> 2) & 1] for k in range(8)])[None]).reshape(-1, 3)
            live = np.repeat(live, 8, axis=0)
            cand = kids
            level += 1

    # capsules are independent; concurrent writes only ever store True
    with cf.ThreadPoolExecutor(min(a.shape[0], os.cpu_count() or 1)) as ex:
        list(ex.map(one, range(a.shape[0])))
    idx = np.argwhere(occ).astype(np.uint32)
    order = np.argsort(morton_key(idx, depth), kind="stable")
    return idx[order]


# --------------------------------------------------------------------------
# cameras


def sphere_eye(azimuth_deg: float, elevation_deg: float, radius: float = 1.5,
               center=(0.5, 0.5, 0.5)):
    az, el = math.radians(azimuth_deg), math.radians(elevation_deg)
    return (center[0] + radius * math.cos(el) * math.cos(az),
            center[1] + radius * math.cos(el) * math.sin(az),
            center[2] + radius * math.sin(el))


def ring_cameras(n: int = 16, width: int = 1920, height: int = 1080, radius: float = 1.5,
                 fov_y_deg: float = 40.0):
    """n cameras on a ring of `radius` in the plane z = 0.5, azimuth 2 pi k / n."""
    return [Camera(eye=sphere_eye(360.0 * k / n, 0.0, radius), fov_y_deg=fov_y_deg,
                   width=width, height=height) for k in range(n)]


def sweep_cameras(seed: int, n: int = 32, width: int = 48, height: int = 48, radius: float = 1.5):
    """n seeded eyes on the sphere of `radius` (azimuth U(0,360), elevation U(-60,60))."""
    rng = np.random.default_rng(seed)
    az = rng.uniform(0.0, 360.0, size=n)
    el = rng.uniform(-60.0, 60.0, size=n)
    return [Camera(eye=sphere_eye(float(a), float(e), radius), width=width, height=height)
            for a, e in zip(az, el)]


# --------------------------------------------------------------------------
# the named workloads


def shell_tree(seed: int = 0, depth: int = 5, n1: int = 31, n2: int = 5) -> Tree:
    """Depth-5 spherical shell r in [0.30, 0.40] with i.i.d. coefficients (128x128 parity case)."""
    xyz = shell_leaves(depth)
    rng = np.random.default_rng(seed)
    coeffs = draw_coefficients(rng, xyz.shape[0], n1, n2)
    return Tree(np.full(xyz.shape[0], depth, np.uint8), xyz, coeffs, depth, n1, n2)


def shell_camera(width: int = 128, height: int = 128) -> Camera:
    """Eye on the radius-1.5 sphere at azimuth 30 deg, elevation 20 deg; 40 deg vertical FOV."""
    return Camera(eye=sphere_eye(30.0, 20.0), width=width, height=height)


SHELL_T = 0.37 * PERIOD_T  # frame time of the 128x128 parity case


def body_tree(seed: int = 0, depth: int = 9, n1: int = 31, n2: int = 5,
              cache_dir: str | None = None) -> Tree:
    """Depth-9 union over 60 frames of the animated 14-capsule body, i.i.d. coefficients.

    default_rng(seed) draws the capsule body (capsule_body); the coefficients
    of the Morton-sorted leaves come from draw_coefficients_blocked(seed + 1).
    With `cache_dir` (or $FPO_SYNTH_CACHE) the result is kept in .npy files.
    """
    cache_dir = cache_dir or os.environ.get("FPO_SYNTH_CACHE")
    key = f"body_s{seed}_d{depth}_n{n1}_{n2}"
    if cache_dir:
        fx, fc = (os.path.join(cache_dir, f"{key}_{w}.npy") for w in ("xyz", "coef"))
        if os.path.exists(fx) and os.path.exists(fc):
            xyz = np.load(fx)
            coeffs = np.load(fc, mmap_mode="r")
            return Tree(np.full(xyz.shape[0], depth, np.uint8), xyz, np.ascontiguousarray(coeffs),
                        depth, n1, n2)
    rng = np.random.default_rng(seed)
    a, b, r = capsule_body(rng)
    xyz = capsule_union_leaves(a, b, r, depth)
    coeffs = draw_coefficients_blocked(seed + 1, xyz.shape[0], n1, n2)
    if cache_dir:
        os.makedirs(cache_dir, exist_ok=True)
        np.save(fx, xyz)
        np.save(fc, coeffs)
    return Tree(np.full(xyz.shape[0], depth, np.uint8), xyz, coeffs, depth, n1, n2)


def random_tree(seed: int, max_depth: int = 4, n1: int = 31, n2: int = 5, **kw) -> Tree:
    rng = np.random.default_rng(seed)
    d, xyz = random_mixed_leaves(rng, max_depth, **kw)
    coeffs = draw_coefficients(rng, d.shape[0], n1, n2)
    return Tree(d, xyz, coeffs, max_depth, n1, n2)


def frame_schedule(n_frames: int, seed: int = 0, n_cams: int = 16, n_t: int = 60):
    """Seeded order over the (camera, integer t) grid of n_cams x n_t frames."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n_cams * n_t)
    return [(int(p % n_cams), float(p // n_cams)) for p in perm[:n_frames]] if n_frames <= perm.size \
        else [(int(p % n_cams), float(p // n_cams)) for p in np.resize(perm, n_frames)]


# --------------------------------------------------------------------------
# smooth animated fields (per-frame values of the leaves, for generation)


def smooth_frame_values(leaf_depth, leaf_xyz, body, n_frames: int = 60, seed: int = 0,
                        chunk: int = 1 << 17, device=None):
    """Per-frame values [n_frames, n, 28] (sigma, z_{c,k}) of the leaves of a
    union octree under the animated capsule body `body` = (a, b, radii)
    (from capsule_body): the values a per-frame octree would hold.

    sigma(p, f) = 50 smoothstep(-sdf_f(p) / w), sdf_f the signed distance to
    the union of capsules at frame f (f = 1..n_frames, frame f uses the body
    at f mod 60), w = 2 finest cells.  Colour: four shared travelling waves
    g_m(p, f) = sin(2 pi a_m . p + 2 pi nu_m f / T + phi_m) (nu = 1, 1, 2, 2)
    mixed per SH slot, z_{c,k} = s_k sum_m M[c,k,m] g_m with s_0 = 1.5 and
    s_k = 0.3 for k >= 1: the SH coefficients of a radiance field are
    correlated across colour channels and SH bands, and at most two temporal
    cycles keep them exact in n2 = 5 Fourier terms.
    Draw order (default_rng(seed)): a [4, 3] ~ N(0, 1.5), phi [4] ~ U(0, 2 pi),
    M [3, 9, 4] ~ N(0, 1/2).
    Returns a torch tensor on `device` (default: CUDA if available).
    """
    import torch

    dev = torch.device(device or ("cuda" if torch.cuda.is_available() else "cpu"))
    rng = np.random.default_rng(seed)
    freq = torch.as_tensor(rng.normal(0.0, 1.5, size=(4, 3)), dtype=torch.float32, device=dev)
    phase = torch.as_tensor(rng.uniform(0.0, 2 * np.pi, size=4), dtype=torch.float32, device=dev)
    mix = torch.as_tensor(rng.normal(0.0, np.sqrt(0.5), size=(3, 9, 4)), dtype=torch.float32, device=dev)
    nu = torch.tensor([1.0, 1.0, 2.0, 2.0], device=dev)
    amp = torch.full((9,), 0.3, device=dev)
    amp[0] = 1.5
    mix = mix * amp[None, :, None]
    A, B, R = (torch.as_tensor(np.asarray(v), dtype=torch.float32, device=dev) for v in body)
    depth = int(np.max(leaf_depth)) if len(leaf_depth) else 0
    w = 2.0 / (1 << max(depth, 1))
    n = len(leaf_depth)
    out = torch.empty((n_frames, n, 28), dtype=torch.float32, device=dev)
    for s0 in range(0, n, chunk):
        xyz = torch.as_tensor(np.asarray(leaf_xyz[s0:s0 + chunk], np.float64), dtype=torch.float32, device=dev)
        dd = torch.as_tensor(np.asarray(leaf_depth[s0:s0 + chunk], np.int64), device=dev)
        p = (xyz + 0.5) / (2.0 ** dd.float())[:, None]  # [m, 3]
        spatial = 2 * np.pi * (p @ freq.T) + phase  # [m, 4]
        for f in range(1, n_frames + 1):
            fi = f % A.shape[1]
            a, b = A[:, fi], B[:, fi]  # [C, 3]
            ab = b - a
            ap = p[:, None, :] - a[None]
            tt = torch.clamp((ap * ab).sum(-1) / (ab * ab).sum(-1), 0.0, 1.0)
            dist = torch.linalg.norm(ap - tt[..., None] * ab, dim=-1) - R  # [m, C]
            sdf = dist.min(dim=1).values
            u = torch.clamp((-sdf / w + 1.0) * 0.5, 0.0, 1.0)
            out[f - 1, s0:s0 + chunk, 0] = 50.0 * u * u * (3.0 - 2.0 * u)
            g = torch.sin(spatial + 2 * np.pi * nu * f / n_frames)  # [m, 4]
            out[f - 1, s0:s0 + chunk, 1:] = torch.einsum("mw,ckw->mck", g, mix).reshape(-1, 27)
    return out
