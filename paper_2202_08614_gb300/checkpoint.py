"""Saving and restoring what the method builds and trains.

- A Fourier PlenOctree (the union octree's leaves and their canonical
  coefficients) as one .npz file: what fpo_upload_tree takes.
- The state of the fine-tuning stage (coefficients, Adam moments, step) and
  of the latent-decoder training (latents, MLP, Adam moments, step), so a run
  resumes where it stopped: the next step after a restore equals the step
  the uninterrupted run would have taken.
"""

from __future__ import annotations

import numpy as np

from . import synth

_TREE_KEYS = ("leaf_depth", "leaf_xyz", "coeffs", "max_depth", "n1", "n2", "aabb_min", "aabb_size")


def save_tree(path, tree: "synth.Tree") -> None:
    np.savez(path, leaf_depth=np.asarray(tree.leaf_depth, np.uint8), leaf_xyz=np.asarray(tree.leaf_xyz, np.uint32),
             coeffs=np.asarray(tree.coeffs, np.float32), max_depth=np.int64(tree.max_depth), n1=np.int64(tree.n1),
             n2=np.int64(tree.n2), aabb_min=np.asarray(tree.aabb_min, np.float64),
             aabb_size=np.float64(tree.aabb_size))


def load_tree(path) -> "synth.Tree":
    with np.load(path) as z:
        missing = [k for k in _TREE_KEYS if k not in z]
        if missing:
            raise ValueError(f"{path}: not a Fourier PlenOctree file (missing {missing})")
        return synth.Tree(z["leaf_depth"].copy(), z["leaf_xyz"].copy(), z["coeffs"].copy(), int(z["max_depth"]),
                          int(z["n1"]), int(z["n2"]), tuple(float(a) for a in z["aabb_min"]), float(z["aabb_size"]))


def save_state(path, obj) -> None:
    """FineTuner or LatentModel state (tensors moved to the host)."""
    import torch

    torch.save(obj.state_dict(), path)


def load_state(path, obj) -> None:
    import torch

    obj.load_state_dict(torch.load(path, map_location="cpu"))
