"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test ties one part of the oracle to a closed form, a library routine, a
textbook table or a brute-force computation, chosen so that a dropped term,
a wrong sign or index, or a transposed operand fails at least one of them.
CPU only.
"""

import math

import numpy as np
import pytest
import scipy.special as sps

import oracle
from paper_2202_08614_gb300 import synth

PERIOD = 60.0
N1, N2, NSH = 31, 5, 9
NCOEF = N1 + 3 * NSH * N2


def _tree(depths, xyz, max_depth):
    return oracle.OracleTree(np.array(depths, np.uint8), np.array(xyz, np.uint32).reshape(-1, 3),
                             max_depth)


def _coef_index(c, k, i, n1=N1, n2=N2):
    return n1 + (c * NSH + k) * n2 + i


# --------------------------------------------------------------------------
# Eq. 8 (basis)


def test_basis_dc_and_period():
    rng = np.random.default_rng(1)
    for t in rng.uniform(-100, 100, 20):
        b = oracle.basis(N1, t, PERIOD)
        assert b[0] == 1.0
        np.testing.assert_allclose(oracle.basis(N1, t + PERIOD, PERIOD), b, atol=1e-12)


def test_basis_discrete_orthogonality():
    # sum over one period of IDFT_i IDFT_j: T for i=j=0, T/2 for i=j>0, else 0
    B = np.stack([oracle.basis(N1, t, PERIOD) for t in range(60)])
    G = B.T @ B
    want = np.diag([60.0] + [30.0] * (N1 - 1))
    np.testing.assert_allclose(G, want, atol=1e-9)


def test_basis_reproduces_numpy_rfft():
    # A real signal band-limited to frequencies m <= 15 is reproduced by the
    # Eq. 8 series whose coefficients come from numpy's FFT:
    # k_0 = X_0/T, k_{2m} = 2 Re X_m / T, k_{2m-1} = -2 Im X_m / T.
    rng = np.random.default_rng(2)
    T = 60
    spec = np.zeros(T // 2 + 1, complex)
    spec[:16] = rng.normal(size=16) + 1j * rng.normal(size=16)
    spec[0] = spec[0].real
    x = np.fft.irfft(spec, n=T)
    X = np.fft.rfft(x)
    k = np.zeros(N1)
    k[0] = X[0].real / T
    for m in range(1, 16):
        k[2 * m] = 2 * X[m].real / T
        k[2 * m - 1] = -2 * X[m].imag / T
    for t in range(T):
        assert abs(oracle.basis(N1, t, T) @ k - x[t]) < 1e-12


# --------------------------------------------------------------------------
# Eq. 1 (real SH)


def test_sh_textbook_constants(golden_dir):
    rows = [l.split() for l in open(f"{golden_dir}/real_sh_constants.txt") if l.strip() and l[0] != "#"]
    for r in rows:
        k = int(r[0])
        d = np.array([float(v) for v in r[3:6]])
        assert abs(abs(oracle.sh(d)[k]) - float(r[6])) < 5e-7, r


def test_sh_matches_scipy_complex_sh_with_condon_shortley():
    # real Y_{l,m} = sqrt2 Re Y_l^m (m>0), Y_l^0 (m=0), sqrt2 Im Y_l^{|m|} (m<0),
    # with scipy's Y_l^m including the Condon-Shortley phase.
    rng = np.random.default_rng(3)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        y = oracle.sh(d)
        for l in range(3):
            for m in range(-l, l + 1):
                Yc = sps.sph_harm_y(l, abs(m), theta, phi)
                ref = Yc.real if m == 0 else (math.sqrt(2) * (Yc.real if m > 0 else Yc.imag))
                assert abs(y[l * (l + 1) + m] - ref) < 1e-12, (l, m)


def test_sh_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) (8 nodes) x uniform phi (16 nodes) is exact
    # for the degree-<=4 products of two l<=2 harmonics.
    xs, ws = np.polynomial.legendre.leggauss(8)
    G = np.zeros((9, 9))
    for x, w in zip(xs, ws):
        s = math.sqrt(1 - x * x)
        for j in range(16):
            ph = 2 * math.pi * j / 16
            y = oracle.sh(np.array([s * math.cos(ph), s * math.sin(ph), x]))
            G += w * (2 * math.pi / 16) * np.outer(y, y)
    np.testing.assert_allclose(G, np.eye(9), atol=1e-13)


# --------------------------------------------------------------------------
# compositing closed forms


def _one_leaf(depth=2, xyz=(1, 1, 1)):
    return _tree([depth], [xyz], depth)


def _render_ray(tree, coeffs, o, d, **kw):
    return oracle.render(tree, coeffs, rays_o=np.array([o], float), rays_d=np.array([d], float),
                         visit_cap=8, want_delta=True, **kw)


def test_single_leaf_closed_form():
    # one leaf [0.25, 0.5]^3; DC-only coefficients: sigma = k_sigma_0,
    # colour = S(k_{c,0,0} * Y_00) with Y_00 = 1/(2 sqrt(pi)).
    tree = _one_leaf()
    co = np.zeros((1, NCOEF), np.float32)
    co[0, 0] = 7.5
    zc = [0.75, -1.25, 2.0]
    for c in range(3):
        co[0, _coef_index(c, 0, 0)] = zc[c]
    bg = (0.2, 0.5, 0.9)
    for d, L in [((1, 0, 0), 0.25), ((1, 0.1, 0), 0.25 * math.sqrt(1.01))]:
        dn = np.array(d, float) / np.linalg.norm(d)
        o = np.array([0.375, 0.375, 0.375]) - 2.0 * dn  # through the box centre
        r = _render_ray(tree, co, o, d, bg=bg, stop_T=0.0, t=13.0)
        sigma = 7.5
        col = 1 / (1 + np.exp(-np.array(zc, float) * 0.5 / math.sqrt(math.pi)))
        a = 1 - math.exp(-sigma * L)
        want = a * col + (1 - a) * np.array(bg)
        np.testing.assert_allclose(r["rgb"][0], want, atol=1e-14)
        assert abs(r["T"][0] - math.exp(-sigma * L)) < 1e-15
        assert abs(r["visit_delta"][0, 0] - L) < 1e-14
        assert r["visit_count"][0] == 1


def test_density_time_series_follows_rfft():
    # a time-varying density given by FFT-derived coefficients (Eq. 7 with
    # Eq. 8) gives T(t) = exp(-x(t) L) at every integer frame.
    rng = np.random.default_rng(4)
    T = 60
    spec = np.zeros(31, complex)
    spec[:16] = 0.3 * (rng.normal(size=16) + 1j * rng.normal(size=16))
    spec[0] = 40.0 * T  # x(t) ~ 40 + small wiggle, positive
    x = np.fft.irfft(spec, n=T)
    assert x.min() > 0
    X = np.fft.rfft(x)
    co = np.zeros((1, NCOEF), np.float32)
    k = np.zeros(N1)
    k[0] = X[0].real / T
    for m in range(1, 16):
        k[2 * m] = 2 * X[m].real / T
        k[2 * m - 1] = -2 * X[m].imag / T
    co[0, :N1] = k
    tree = _one_leaf()
    xs = np.array(co[0, :N1], float)  # what the oracle actually sees (float32)
    for t in (0, 7, 22, 59):
        r = _render_ray(tree, co, (-1.0, 0.375, 0.375), (1, 0, 0), stop_T=0.0, t=float(t))
        # reference density: the float32-rounded coefficients through the FFT
        # synthesis of numpy (irfft of the rounded spectrum)
        Xr = np.zeros(31, complex)
        Xr[0] = xs[0] * T
        for m in range(1, 16):
            Xr[m] = (xs[2 * m] - 1j * xs[2 * m - 1]) * T / 2
        xt = np.fft.irfft(Xr, n=T)[t]
        assert abs(r["T"][0] - math.exp(-xt * 0.25)) < 1e-12


def test_sh_coefficient_time_series_and_index():
    # Eq. 9: one SH slot k, channel c, with n2 = 5 coefficients from the FFT of
    # a band-limited z(t) (m <= 2); colour of an opaque leaf is S(z(t) Y_k(d)),
    # Y_k from scipy.  Checks the canonical index (c, k, i) and the i-range.
    rng = np.random.default_rng(5)
    T = 60
    d = np.array([0.8, -0.36, 0.48])
    d /= np.linalg.norm(d)
    o = np.array([0.375, 0.375, 0.375]) - 2.0 * d
    theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
    tree = _one_leaf()
    for c, kk in [(0, 0), (1, 5), (2, 8), (1, 3)]:
        spec = np.zeros(31, complex)
        spec[:3] = rng.normal(size=3) + 1j * rng.normal(size=3)
        spec[0] = spec[0].real
        z = np.fft.irfft(spec, n=T) * 20
        X = np.fft.rfft(z)
        co = np.zeros((1, NCOEF), np.float32)
        co[0, 0] = 1e4  # opaque: the leaf's colour is the pixel's colour
        kz = [X[0].real / T, -2 * X[1].imag / T, 2 * X[1].real / T, -2 * X[2].imag / T,
              2 * X[2].real / T]
        for i in range(5):
            co[0, _coef_index(c, kk, i)] = kz[i]
        l = int(math.isqrt(kk))
        m = kk - l * (l + 1)
        Yc = sps.sph_harm_y(l, abs(m), theta, phi)
        yk = Yc.real if m == 0 else math.sqrt(2) * (Yc.real if m > 0 else Yc.imag)
        zf = np.array([co[0, _coef_index(c, kk, i)] for i in range(5)], float)
        for t in (3, 31):
            r = _render_ray(tree, co, o, d, stop_T=0.0, t=float(t), bg=(0.0, 0.0, 0.0))
            Xr = np.zeros(31, complex)
            Xr[0] = zf[0] * T
            Xr[1] = (zf[2] - 1j * zf[1]) * T / 2
            Xr[2] = (zf[4] - 1j * zf[3]) * T / 2
            zt = np.fft.irfft(Xr, n=T)[t]
            want = np.full(3, 0.5)
            want[c] = 1 / (1 + math.exp(-zt * yk))
            np.testing.assert_allclose(r["rgb"][0], want, atol=1e-12)


def test_empty_space_gives_background():
    bg = (0.3, 0.6, 0.1)
    tree = _tree([], np.zeros((0, 3)), 3)
    r = oracle.render(tree, np.zeros((0, NCOEF), np.float32), camera=synth.shell_camera(16, 16),
                      bg=bg)
    assert np.all(r["rgb"] == np.array(bg)) and np.all(r["T"] == 1.0)
    tr = synth.shell_tree()
    ot = oracle.OracleTree(tr.leaf_depth, tr.leaf_xyz, tr.max_depth)
    miss = oracle.render(ot, tr.coeffs, rays_o=[[-1, 2, 2], [0.5, 0.5, -1]],
                         rays_d=[[1, 0, 0], [0, 1, 0]], bg=bg, visit_cap=4)
    assert np.all(miss["rgb"] == np.array(bg)) and np.all(miss["visit_count"] == 0)


def test_dc_only_is_constant_in_time():
    tr = synth.shell_tree()
    co = tr.coeffs.copy()
    co[:, 1:N1] = 0
    z = co[:, N1:].reshape(-1, 3, NSH, N2)
    z[..., 1:] = 0
    co[:, N1:] = z.reshape(co.shape[0], -1)
    ot = oracle.OracleTree(tr.leaf_depth, tr.leaf_xyz, tr.max_depth)
    cam = synth.shell_camera(32, 32)
    ref = oracle.render(ot, co, camera=cam, t=0.0)["rgb"]
    for t in (1.0, 22.2, 59.5, 123.4):
        assert np.array_equal(oracle.render(ot, co, camera=cam, t=t)["rgb"], ref)


# --------------------------------------------------------------------------
# segments and traversal order against brute-force marching


def _locate(leaf_map, max_depth, p):
    """Leaf id containing point p (plain dictionary lookup per depth) or -1."""
    for dep in range(max_depth + 1):
        g = 1 << dep
        key = (dep, int(p[0] * g), int(p[1] * g), int(p[2] * g))
        if key in leaf_map:
            return leaf_map[key]
    return -1


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_segments_match_midpoint_marching(seed):
    depth = 4
    rng = np.random.default_rng(seed)
    d_leaf, xyz = synth.random_mixed_leaves(rng, depth)
    leaf_map = {(int(dd), *map(int, c)): i for i, (dd, c) in enumerate(zip(d_leaf, xyz))}
    ot = oracle.OracleTree(d_leaf, xyz, depth)
    n = d_leaf.shape[0]
    co = np.zeros((n, NCOEF), np.float32)
    co[:, 0] = rng.uniform(0.5, 3.0, n)  # DC density only, small: no early stop
    for c in range(3):
        co[:, _coef_index(c, 0, 0)] = rng.normal(size=n)
    n_rays = 40
    tgt = rng.uniform(0.05, 0.95, (n_rays, 3))
    dirs = rng.normal(size=(n_rays, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    org = tgt - 2.0 * dirs
    bg = np.array([0.1, 0.2, 0.3])
    res = oracle.render(ot, co, rays_o=org, rays_d=dirs, stop_T=0.0, bg=tuple(bg), visit_cap=256,
                        want_delta=True)
    y00 = 0.5 / math.sqrt(math.pi)
    col = 1 / (1 + np.exp(-co[:, N1::N2 * NSH][:, :3].astype(float) * y00))  # k=0,i=0 per c
    errs = {}
    for h in (4e-4, 2e-4):
        worst_len, worst_rgb = 0.0, 0.0
        for r in range(n_rays):
            if res["flags"][r] & 1:
                continue
            ts = np.arange(0.0, 4.0, h) + 0.5 * h
            pts = org[r] + ts[:, None] * dirs[r]
            inside = np.all((pts >= 0) & (pts < 1), axis=1)
            ids = np.array([_locate(leaf_map, depth, p) if ok else -1
                            for p, ok in zip(pts, inside)])
            # order of first appearance and total length per leaf
            seq, length = [], {}
            for i in ids:
                if i < 0:
                    continue
                if i not in length:
                    seq.append(i)
                    length[i] = 0.0
                length[i] += h
            nv = res["visit_count"][r]
            o_seq = list(res["visit_log"][r, :nv])
            o_len = dict(zip(o_seq, res["visit_delta"][r, :nv]))
            long_o = [i for i in o_seq if o_len[i] > 4 * h]
            long_m = [i for i in seq if length[i] > 6 * h]
            assert [i for i in long_o if i in length] == long_o
            assert [i for i in seq if i in o_len and o_len[i] > 4 * h] == long_o
            assert set(long_m) <= set(o_seq)
            for i in o_seq:
                worst_len = max(worst_len, abs(length.get(i, 0.0) - o_len[i]))
            # continuous emission-absorption integral by the midpoint rule
            sig = np.where(ids >= 0, co[np.maximum(ids, 0), 0].astype(float), 0.0)
            cc = np.where(ids[:, None] >= 0, col[np.maximum(ids, 0)], 0.0)
            Tm = np.exp(-np.concatenate([[0.0], np.cumsum(sig * h)]))
            C = np.sum((Tm[:-1] * (1 - np.exp(-sig * h)))[:, None] * cc, axis=0) + Tm[-1] * bg
            worst_rgb = max(worst_rgb, np.max(np.abs(C - res["rgb"][r])))
        assert worst_len <= 2.01 * h
        errs[h] = worst_rgb
        assert worst_rgb < 20 * h
    assert errs[2e-4] < errs[4e-4] or errs[4e-4] < 1e-9


# --------------------------------------------------------------------------
# invariants


def test_union_split_invariance():
    # Sec. 4.2: a divided leaf copies its value into its 8 children; the image
    # must not change (only the visit log does).
    tr = synth.random_tree(21, max_depth=3)
    ot = oracle.OracleTree(tr.leaf_depth, tr.leaf_xyz, tr.max_depth)
    j = int(np.argmin(tr.leaf_depth))
    d0, (x, y, z) = int(tr.leaf_depth[j]), tr.leaf_xyz[j]
    kids = [(2 * x + (c & 1), 2 * y + ((c >> 1) & 1), 2 * z + ((c >> 2) & 1)) for c in range(8)]
    keep = np.arange(tr.n_leaves) != j
    depth2 = np.concatenate([tr.leaf_depth[keep], np.full(8, d0 + 1, np.uint8)])
    xyz2 = np.concatenate([tr.leaf_xyz[keep], np.array(kids, np.uint32)])
    co2 = np.concatenate([tr.coeffs[keep], np.repeat(tr.coeffs[j:j + 1], 8, 0)])
    ot2 = oracle.OracleTree(depth2, xyz2, max(tr.max_depth, d0 + 1))
    cam = synth.Camera(eye=synth.sphere_eye(40, 25), width=40, height=40)
    a = oracle.render(ot, tr.coeffs, camera=cam, t=5.0, stop_T=0.0)
    b = oracle.render(ot2, co2, camera=cam, t=5.0, stop_T=0.0)
    np.testing.assert_allclose(a["rgb"], b["rgb"], atol=1e-12)


def test_weights_sum_to_one_and_range():
    tr = synth.shell_tree()
    ot = oracle.OracleTree(tr.leaf_depth, tr.leaf_xyz, tr.max_depth)
    cam = synth.shell_camera(32, 32)
    r = oracle.render(ot, tr.coeffs, camera=cam, t=9.0, stop_T=0.0, visit_cap=128,
                      want_weight=True, bg=(0.25, 0.5, 1.0))
    assert r["visit_count"].max() < 128
    s = r["visit_weight"].sum(1) + r["T"]
    np.testing.assert_allclose(s, 1.0, atol=1e-12)
    assert r["rgb"].min() >= 0 and r["rgb"].max() <= 1


def test_permuted_upload_order():
    tr = synth.random_tree(31, max_depth=4)
    perm = np.random.default_rng(0).permutation(tr.n_leaves)
    cam = synth.Camera(eye=synth.sphere_eye(100, -30), width=32, height=24)
    a = oracle.render(oracle.OracleTree(tr.leaf_depth, tr.leaf_xyz, 4), tr.coeffs, camera=cam,
                      t=3.0, visit_cap=64)
    b = oracle.render(oracle.OracleTree(tr.leaf_depth[perm], tr.leaf_xyz[perm], 4),
                      tr.coeffs[perm], camera=cam, t=3.0, visit_cap=64)
    assert np.array_equal(a["rgb"], b["rgb"])
    for r in range(a["rgb"].shape[0]):
        n = a["visit_count"][r]
        assert np.array_equal(perm[b["visit_log"][r, :n]], a["visit_log"][r, :n])


def test_early_stop_effect_bounded():
    tr = synth.shell_tree()
    ot = oracle.OracleTree(tr.leaf_depth, tr.leaf_xyz, tr.max_depth)
    cam = synth.shell_camera(48, 48)
    a = oracle.render(ot, tr.coeffs, camera=cam, t=synth.SHELL_T, stop_T=1e-4)
    b = oracle.render(ot, tr.coeffs, camera=cam, t=synth.SHELL_T, stop_T=0.0)
    assert np.abs(a["rgb"] - b["rgb"]).max() <= 1e-4
    assert np.all(a["T"][a["T"] < 1e-4] > 0)


def test_camera_orientation():
    # one small leaf up and to the left of the target as seen from the eye:
    # it must show in the upper-left quadrant (row 0 = top, column 0 = left).
    eye = (0.5, -1.0, 0.5)  # looking along +y; up = +z; right = f x up = +x
    leaf = (3, 12, 12)  # depth 4 cell near x=0.22, z=0.78
    tree = _tree([4], [leaf], 4)
    co = np.zeros((1, NCOEF), np.float32)
    co[0, 0] = 1e3
    cam = synth.Camera(eye=eye, target=(0.5, 0.5, 0.5), width=64, height=64)
    r = oracle.render(tree, co, camera=cam, bg=(1, 1, 1))
    hit = np.argwhere(r["T"].reshape(64, 64) < 0.5)
    assert hit.size
    assert hit[:, 0].max() < 32 and hit[:, 1].max() < 32
    # the centre of an odd image looks exactly at the target
    cam2 = synth.Camera(eye=eye, target=(0.5, 0.5, 0.5), width=33, height=33)
    c_tree = _tree([6], [(32, 32, 32)], 6)  # cell [0.5, 0.5156)^3 touches the target corner
    r2 = oracle.render(c_tree, co, camera=cam2, sel=[16 * 33 + 16], visit_cap=2, want_delta=True)
    assert r2["visit_count"][0] == 1  # the ray enters the cell at its corner edge
    assert r2["flags"][0] & 1  # ... along an edge: flagged as a near tie


def test_tree_validation():
    with pytest.raises(ValueError):
        _tree([2, 1], [(0, 0, 0), (0, 0, 0)], 2)  # leaf inside another leaf
    with pytest.raises(ValueError):
        _tree([1, 1], [(1, 0, 0), (1, 0, 0)], 1)  # duplicate
    with pytest.raises(ValueError):
        _tree([2], [(4, 0, 0)], 2)  # out of range
    with pytest.raises(ValueError):
        _tree([3], [(0, 0, 0)], 2)  # deeper than max depth


# --------------------------------------------------------------------------
# Sec. 4.3 gradient, pinned by central differences of the forward render


@pytest.mark.parametrize("stop_T", [0.0, 1e-4])
def test_gradient_matches_finite_differences(stop_T):
    tree = synth.shell_tree()
    ot = oracle.OracleTree(tree.leaf_depth, tree.leaf_xyz, tree.max_depth)
    cam = synth.shell_camera(20, 16)
    t = 22.2
    bg = (0.3, 0.6, 0.9)
    rng = np.random.default_rng(9)
    g = rng.normal(size=(cam.width * cam.height, 3))
    base = oracle.render(ot, tree.coeffs, camera=cam, t=t, stop_T=stop_T, bg=bg)
    G = oracle.render_grad(ot, tree.coeffs, g, camera=cam, t=t, stop_T=stop_T, bg=bg)
    touched = np.nonzero(np.abs(G).sum(1))[0]
    assert touched.size > 50
    b = oracle.basis(N1, t, PERIOD)
    sraw = tree.coeffs[:, :N1].astype(np.float64) @ b
    picks = []
    for leaf in rng.choice(touched, 40, replace=False):
        for j in rng.choice(NCOEF, 5, replace=False):
            if j < N1 and abs(sraw[leaf]) < 0.05:
                continue  # the ReLU kink of the density
            picks.append((leaf, j))
    checked = 0
    for leaf, j in picks:
        k0 = tree.coeffs[leaf, j]
        eps = 1e-3 * max(1.0, abs(float(k0)))
        kp, km = np.float32(k0 + eps), np.float32(k0 - eps)
        co = tree.coeffs.copy()
        co[leaf, j] = kp
        rp = oracle.render(ot, co, camera=cam, t=t, stop_T=stop_T, bg=bg)
        co[leaf, j] = km
        rm = oracle.render(ot, co, camera=cam, t=t, stop_T=stop_T, bg=bg)
        if stop_T > 0 and not (np.array_equal(rp["T"] < stop_T, base["T"] < stop_T)
                               and np.array_equal(rm["T"] < stop_T, base["T"] < stop_T)):
            continue  # the perturbation moved an early stop: not differentiable there
        fd = np.sum(g * (rp["rgb"] - rm["rgb"])) / (float(kp) - float(km))
        assert abs(G[leaf, j] - fd) <= 1e-3 * abs(fd) + 1e-7, (leaf, j, G[leaf, j], fd)
        checked += 1
    assert checked > 100


# --------------------------------------------------------------------------
# Eq. 10-12 (per-leaf DFT) with the 2/T reading


def test_dft_round_trip_band_limited():
    # frequencies 0..15 < T/2: the Eq. 8 series of the DFT coefficients gives
    # back the samples at every frame t = 1..60 (and matches numpy's FFT)
    rng = np.random.default_rng(11)
    T = 60
    spec = np.zeros(T // 2 + 1, complex)
    spec[:16] = rng.normal(size=16) + 1j * rng.normal(size=16)
    spec[0] = spec[0].real
    x = np.fft.irfft(spec, n=T)  # x[t] for t = 0..59; frame t = 1..60 -> x[t % 60]
    frames = np.array([x[t % T] for t in range(1, T + 1)])
    k = oracle.dft(frames, N1)[0]
    for t in range(1, T + 1):
        assert abs(oracle.basis(N1, t, T) @ k - frames[t - 1]) < 1e-12
    X = np.fft.rfft(x)
    assert abs(k[0] - X[0].real / T) < 1e-12
    for m in range(1, 16):
        assert abs(k[2 * m] - 2 * X[m].real / T) < 1e-12
        assert abs(k[2 * m - 1] + 2 * X[m].imag / T) < 1e-12


def test_dft_of_constant_and_single_tone():
    T = 60
    k = oracle.dft(np.full(T, 3.5), 5)[0]
    np.testing.assert_allclose(k, [3.5, 0, 0, 0, 0], atol=1e-13)
    t = np.arange(1, T + 1)
    k = oracle.dft(0.7 * np.sin(2 * np.pi * 2 * t / T), 7)[0]  # frequency 2 -> odd index 3
    np.testing.assert_allclose(k, [0, 0, 0, 0.7, 0, 0, 0], atol=1e-13)


# --------------------------------------------------------------------------
# latent decoder reference: its gradient against central differences


def test_latent_loss_gradient_matches_finite_differences():
    from oracle import latent as olat

    rng = np.random.default_rng(12)
    nc = 13
    w = [rng.normal(size=(64, 32)) / 6, rng.normal(size=64) * 0.1, rng.normal(size=(64, 64)) / 8,
         rng.normal(size=64) * 0.1, rng.normal(size=(nc, 64)) / 8, rng.normal(size=nc)]
    x = rng.normal(size=(5, 32))
    tgt = rng.normal(size=(5, nc))
    cw = rng.uniform(0.5, 2.0, nc)
    L, dx, g = olat.loss_grad(x, *w, tgt, cw)
    names = ["w1", "b1", "w2", "b2", "w3", "b3"]

    def f(ws, xx):
        return olat.loss_grad(xx, *ws, tgt, cw)[0]

    eps = 1e-6
    for k, name in enumerate(names):
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in w[k].shape)
            wp = [a.copy() for a in w]
            wm = [a.copy() for a in w]
            wp[k][idx] += eps
            wm[k][idx] -= eps
            fd = (f(wp, x) - f(wm, x)) / (2 * eps)
            assert abs(g[name][idx] - fd) <= 1e-6 * max(1.0, abs(fd)), name
    for _ in range(10):
        idx = tuple(rng.integers(0, s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += eps
        xm[idx] -= eps
        fd = (f(w, xp) - f(w, xm)) / (2 * eps)
        assert abs(dx[idx] - fd) <= 1e-6 * max(1.0, abs(fd))


def _one_hot_net(nc=NCOEF):
    """A decoder whose outputs are known ReLU chains of single latent entries:
    h1 = [relu(x + 0.25), relu(0.25 - x)], h2 = relu(h1[perm] - 0.5) with a
    permutation that is not its own inverse, y_o = (o + 1) h2[o % 64] + o."""
    w1 = np.zeros((64, 32))
    for j in range(32):
        w1[j, j] = 1.0
        w1[32 + j, j] = -1.0
    perm = (np.arange(64) * 5 + 3) % 64
    w2 = np.zeros((64, 64))
    w2[np.arange(64), perm] = 1.0
    w3 = np.zeros((nc, 64))
    w3[np.arange(nc), np.arange(nc) % 64] = np.arange(nc) + 1.0
    return w1, np.full(64, 0.25), w2, np.full(64, -0.5), w3, np.arange(nc, dtype=float), perm


def test_latent_decode_of_a_one_hot_network():
    # decode() against the ReLU chains written out by hand: catches a missing
    # ReLU (the -0.5 bias makes h2 negative without the second one, and
    # relu(-x) without the first), a transposed weight (W1 is 64 x 32 and the
    # permutation in W2 is not symmetric) and a dropped bias.
    from oracle import latent as olat

    w1, b1, w2, b2, w3, b3, perm = _one_hot_net()
    x = np.random.default_rng(3).normal(size=(7, 32)) * 2.0
    y = olat.decode(x, w1, b1, w2, b2, w3, b3)
    for r in range(x.shape[0]):
        h1 = [max(x[r, j] + 0.25, 0.0) for j in range(32)] + [max(0.25 - x[r, j], 0.0) for j in range(32)]
        h2 = [max(h1[perm[i]] - 0.5, 0.0) for i in range(64)]
        want = [(o + 1) * h2[o % 64] + o for o in range(NCOEF)]
        np.testing.assert_allclose(y[r], want, rtol=0, atol=1e-12)
    # a latent of -1 everywhere drives the first half of h1 to 0 and the
    # second half to 1.25
    yn = olat.decode(-np.ones((1, 32)), w1, b1, w2, b2, w3, b3)[0]
    h2n = np.where(perm >= 32, 0.75, 0.0)
    np.testing.assert_allclose(yn, [(o + 1) * h2n[o % 64] + o for o in range(NCOEF)], atol=1e-12)


def test_latent_loss_forward_is_decode():
    # loss_grad's own forward must be decode(): L = sum_j cw_j (decode - target)^2
    from oracle import latent as olat

    rng = np.random.default_rng(21)
    nc = 17
    w = [rng.normal(size=(64, 32)) / 6, rng.normal(size=64) * 0.1, rng.normal(size=(64, 64)) / 8,
         rng.normal(size=64) * 0.1, rng.normal(size=(nc, 64)) / 8, rng.normal(size=nc)]
    x = rng.normal(size=(9, 32))
    tgt = rng.normal(size=(9, nc))
    cw = rng.uniform(0.5, 2.0, nc)
    L = olat.loss_grad(x, *w, tgt, cw)[0]
    y = olat.decode(x, *w)
    assert abs(L - float(np.sum(cw * (y - tgt) ** 2))) <= 1e-12 * max(1.0, abs(L))
    w1, b1, w2, b2, w3, b3, _ = _one_hot_net(nc)
    L1 = olat.loss_grad(x, w1, b1, w2, b2, w3, b3, tgt, cw)[0]
    y1 = olat.decode(x, w1, b1, w2, b2, w3, b3)
    assert abs(L1 - float(np.sum(cw * (y1 - tgt) ** 2))) <= 1e-12 * max(1.0, abs(L1))


def test_latent_table_against_the_oracle_render():
    # table() holds [max(0, sigma(t)), z_{c,k}(t)] of Eq. 7 and Eq. 9; the
    # pinned C oracle renders a one-leaf tree from the same coefficients, and
    # along a ray of length L through the leaf the pixel is
    # (1 - e^{-sigma L}) S(sum_k z_{c,k} Y_k(d)) + e^{-sigma L} bg.  A
    # transposed (n2, 27) reshape or a wrong density row fails it.
    from oracle import latent as olat

    rng = np.random.default_rng(8)
    co = synth.draw_coefficients(rng, 3)  # i.i.d. draws of the parity recipe
    co[2, :N1] *= -1.0                    # a leaf whose density clamps at 0
    tree = _one_leaf()
    bg = np.array([0.2, 0.5, 0.9])
    for t in (0.0, 13.37, 44.0):
        tab = olat.table(co, t)
        assert np.all(tab[:, 28:] == 0.0)
        for j in range(co.shape[0]):
            sigma, z = tab[j, 0], tab[j, 1:28].reshape(3, 9)
            assert sigma >= 0.0
            for d in ((1.0, 0.0, 0.0), (0.6, -0.48, 0.64), (-0.36, 0.8, 0.48)):
                dn = np.array(d) / np.linalg.norm(d)
                o = np.array([0.375, 0.375, 0.375]) - 2.0 * dn
                r = _render_ray(tree, co[j:j + 1], o, dn, bg=tuple(bg), stop_T=0.0, t=t)
                L = r["visit_delta"][0, 0]
                Y = oracle.sh(dn, 2)
                col = 1.0 / (1.0 + np.exp(-(z @ Y)))
                a = 1.0 - math.exp(-sigma * L)
                np.testing.assert_allclose(r["rgb"][0], a * col + (1 - a) * bg, rtol=0, atol=1e-12)
