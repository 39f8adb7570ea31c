"""Checkpoints: a Fourier PlenOctree file round-trips exactly; fine-tuning and
latent training resume where they stopped (the restored state is bit-equal to
the saved one, and the next step agrees with the uninterrupted run up to the
order of the gradient atomics)."""

import numpy as np
import pytest

from paper_2202_08614_gb300 import checkpoint, synth


def test_tree_file_round_trip(tmp_path):
    tree = synth.random_tree(3, max_depth=4, p_split=0.6, p_empty=0.2)
    tree = synth.Tree(tree.leaf_depth, tree.leaf_xyz, tree.coeffs, tree.max_depth, aabb_min=(-1.0, 0.5, 2.0),
                      aabb_size=3.0)
    p = tmp_path / "fpo.npz"
    checkpoint.save_tree(p, tree)
    t2 = checkpoint.load_tree(p)
    assert np.array_equal(t2.leaf_depth, tree.leaf_depth) and t2.leaf_depth.dtype == np.uint8
    assert np.array_equal(t2.leaf_xyz, tree.leaf_xyz) and t2.leaf_xyz.dtype == np.uint32
    assert np.array_equal(t2.coeffs, tree.coeffs) and t2.coeffs.dtype == np.float32
    assert (t2.max_depth, t2.n1, t2.n2, t2.aabb_min, t2.aabb_size) == (4, 31, 5, (-1.0, 0.5, 2.0), 3.0)


def test_not_a_tree_file(tmp_path):
    p = tmp_path / "x.npz"
    np.savez(p, a=np.zeros(3))
    with pytest.raises(ValueError):
        checkpoint.load_tree(p)


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__

    __graft_entry__.build()
    return torch


@pytest.mark.gpu
def test_finetuner_resumes(tmp_path):
    torch = _cuda()
    from paper_2202_08614_gb300 import fpo
    from paper_2202_08614_gb300.finetune import FineTuner

    tree = synth.shell_tree()
    rng = np.random.default_rng(2)
    k0 = torch.as_tensor(tree.coeffs * 1.05, device="cuda")
    o = torch.as_tensor(rng.uniform(-0.5, 1.5, (2048, 3)), dtype=torch.float32, device="cuda")
    d = torch.as_tensor(0.5 - o.cpu().numpy() + rng.normal(size=(2048, 3)) * 0.2, dtype=torch.float32, device="cuda")
    t = torch.as_tensor(rng.uniform(0, 60, 2048), dtype=torch.float32, device="cuda")
    ref = fpo.Renderer(idft_mode="fused")
    ref.upload(tree)
    y = ref.render(rays_o=o, rays_d=d, t_per_ray=t)["rgb"].clone()
    runs = []
    for resume in (False, True):
        r = fpo.Renderer(idft_mode="fused")
        r.upload(tree)
        ft = FineTuner(r, k0, lr=1e-2)
        for _ in range(3):
            ft.step(o, d, t, y)
        if resume:
            checkpoint.save_state(tmp_path / "ft.pt", ft)
            saved = ft.state_dict()
            r2 = fpo.Renderer(idft_mode="fused")
            r2.upload(tree)
            ft = FineTuner(r2, torch.zeros_like(k0))
            checkpoint.load_state(tmp_path / "ft.pt", ft)
            st = ft.state_dict()
            assert st["steps"] == 3 and all(torch.equal(st[k], saved[k]) for k in ("param", "m", "v"))
            # the renderer holds the restored coefficients
            assert torch.equal(ft.render(o, d, t), r.render(rays_o=o, rays_d=d, t_per_ray=t)["rgb"])
        ft.step(o, d, t, y)
        runs.append((ft.param.clone(), ft.render(o, d, t).clone()))
    assert torch.allclose(runs[0][0], runs[1][0], rtol=1e-5, atol=1e-6)
    assert torch.allclose(runs[0][1], runs[1][1], rtol=1e-5, atol=1e-6)
    ref.close()


@pytest.mark.gpu
def test_latent_training_resumes(tmp_path):
    torch = _cuda()
    from paper_2202_08614_gb300.latent import LatentModel

    n = 5000
    tgt = torch.as_tensor(np.random.default_rng(0).normal(size=(n, 166)), dtype=torch.float32, device="cuda")
    runs = []
    for resume in (False, True):
        m = LatentModel(n, seed=1)
        m.fit(tgt, steps=6, batch=1024, seed=3)
        if resume:
            checkpoint.save_state(tmp_path / "lat.pt", m)
            saved = {k: v.clone() for k, v in m.p.items()}
            m = LatentModel(n, seed=9)
            checkpoint.load_state(tmp_path / "lat.pt", m)
            assert m.step_count == 6 and all(torch.equal(m.p[k], saved[k]) for k in saved)
        m.fit(tgt, steps=1, batch=1024, seed=4)
        runs.append({k: v.clone() for k, v in m.p.items()})
    for k in runs[0]:
        assert torch.allclose(runs[0][k], runs[1][k], rtol=1e-4, atol=1e-5), k
