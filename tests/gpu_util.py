"""Helpers shared by the GPU parity tests (compare the CUDA path with the oracle)."""

import numpy as np

import oracle
from paper_2202_08614_gb300 import fpo


def oracle_tree(tree):
    return oracle.OracleTree(tree.leaf_depth, tree.leaf_xyz, tree.max_depth)


def render_both(tree, *, camera=None, t=0.0, rays_o=None, rays_d=None, t_per_ray=None,
                bg=(1.0, 1.0, 1.0), stop_T=1e-4, visit_cap=None, idft_mode="auto", renderer=None,
                ot=None):
    """Renders on the GPU (through the C ABI) and with the oracle on the same inputs."""
    import torch

    own = renderer is None
    r = renderer or fpo.Renderer(n1=tree.n1, n2=tree.n2, idft_mode=idft_mode)
    try:
        if own:
            r.upload(tree)
        kw = dict(bg=bg, stop_T=stop_T, t=t, want_T=True)
        if camera is not None:
            g = r.render(camera=camera, visit_cap=visit_cap, **kw)
        else:
            g = r.render(rays_o=torch.as_tensor(rays_o, dtype=torch.float32),
                         rays_d=torch.as_tensor(rays_d, dtype=torch.float32),
                         t_per_ray=None if t_per_ray is None else torch.as_tensor(t_per_ray, dtype=torch.float32),
                         visit_cap=visit_cap, **kw)
        r.status()
        gpu = {k: v.cpu().numpy() for k, v in g.items() if not k.startswith("_")}
    finally:
        if own:
            r.close()
    ot = ot or oracle_tree(tree)
    ref = oracle.render(ot, tree.coeffs, n1=tree.n1, n2=tree.n2, camera=camera, t=t,
                        rays_o=None if rays_o is None else np.asarray(rays_o, np.float32).astype(np.float64),
                        rays_d=None if rays_d is None else np.asarray(rays_d, np.float32).astype(np.float64),
                        t_per_ray=None if t_per_ray is None else np.asarray(t_per_ray, np.float32).astype(np.float64),
                        bg=bg, stop_T=stop_T, visit_cap=visit_cap or 0,
                        aabb_min=tree.aabb_min, aabb_size=tree.aabb_size)
    return gpu, ref


def compare(gpu, ref, max_tol=1e-3, mean_tol=1e-5, check_visits=True):
    """Element-wise RGB check and exact visit sequences for non-near-tie rays.

    Returns the number of rays excluded from the visit check (near ties)."""
    err = np.abs(gpu["rgb"].astype(np.float64) - ref["rgb"])
    assert err.max() <= max_tol, f"max |dRGB| = {err.max():.3e}"
    assert err.mean() <= mean_tol, f"mean |dRGB| = {err.mean():.3e}"
    near = ref["flags"] != 0
    if check_visits and "visit_log" in gpu:
        gc = gpu["visit_count"].astype(np.int64)
        rc = ref["visit_count"].astype(np.int64)
        cap = ref["visit_log"].shape[1]
        ok = ~near
        bad = np.nonzero(ok & (gc != rc))[0]
        assert bad.size == 0, f"{bad.size} rays differ in visit count, e.g. ray {bad[:5]}: gpu {gc[bad[:5]]} oracle {rc[bad[:5]]}"
        gl = gpu["visit_log"][:, :cap].astype(np.int64) & 0xFFFFFFFF
        rl = ref["visit_log"].astype(np.int64)
        n = np.minimum(rc, cap)
        mask = np.arange(cap)[None, :] < n[:, None]
        diff = np.nonzero(ok[:, None] & mask & (gl != rl))
        assert diff[0].size == 0, f"visit sequences differ for rays {np.unique(diff[0])[:10]}"
    return int(near.sum())
