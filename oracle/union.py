"""Union of per-frame octree structures (Sec. 4.2), written out plainly.

TEST INFRASTRUCTURE ONLY.  A cell is divided in the union when any frame
divides it (holds a leaf strictly inside it); the union leaves are the
undivided children of divided cells (or the root) that some frame's leaf
covers; each frame's value is the value of its leaf covering the union leaf
(the parent copy of Sec. 4.2), zero where it has none.
"""

import numpy as np


def union_trees(frames):
    """frames: list of (depth [n], xyz [n, 3], values [n, 28]).
    Returns (depth [m], xyz [m, 3], values [T, m, 28]) sorted by cell."""
    leaf_of = []  # per frame: {(d, x, y, z): row}
    divided = set()
    for d, xyz, _ in frames:
        m = {}
        for j, (dd, c) in enumerate(zip(d, xyz)):
            dd = int(dd)
            x, y, z = (int(v) for v in c)
            m[(dd, x, y, z)] = j
            for k in range(1, dd + 1):
                divided.add((dd - k, x >> k, y >> k, z >> k))
        leaf_of.append(m)

    def covering(f, cell):
        d, x, y, z = cell
        for k in range(0, d + 1):
            key = (d - k, x >> k, y >> k, z >> k)
            if key in leaf_of[f]:
                return leaf_of[f][key]
        return None

    cands = set()
    if not divided:
        if any(len(m) for m in leaf_of):
            cands.add((0, 0, 0, 0))
    for (d, x, y, z) in divided:
        for c in range(8):
            kid = (d + 1, 2 * x + (c & 1), 2 * y + ((c >> 1) & 1), 2 * z + ((c >> 2) & 1))
            if kid not in divided:
                cands.add(kid)
    leaves = []
    for cell in sorted(cands):
        rows = [covering(f, cell) for f in range(len(frames))]
        if any(r is not None for r in rows):
            leaves.append((cell, rows))
    T = len(frames)
    depth = np.array([c[0] for c, _ in leaves], np.uint8)
    xyz = np.array([c[1:] for c, _ in leaves], np.uint32).reshape(-1, 3)
    vals = np.zeros((T, len(leaves), 28), np.float32)
    for u, (_, rows) in enumerate(leaves):
        for f, r in enumerate(rows):
            if r is not None:
                vals[f, u] = frames[f][2][r]
    return depth, xyz, vals
