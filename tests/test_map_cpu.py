"""Host-side map management: Z-order permutation and its application to the
packed parameter / gradient / moment buffers (CPU tensors)."""
import numpy as np
import torch

from paper_2409_13055_gb300 import mapping, scenes


def test_morton_order_is_a_locality_preserving_permutation():
    rng = np.random.default_rng(2)
    pts = torch.tensor(rng.uniform(size=(4096, 3)))
    perm = mapping.morton_order(pts)
    assert sorted(perm.tolist()) == list(range(4096))
    q = pts[perm]
    step = (q[1:] - q[:-1]).norm(dim=1)
    rnd = (pts[1:] - pts[:-1]).norm(dim=1)
    assert step.mean() < 0.25 * rnd.mean()  # neighbours in index are near in space


def test_permute_moves_every_group_and_buffer():
    p, _ = scenes.tiny_scene(37, 32, 24, seed=4, sh_degree=3)
    gm = mapping.GaussianMap(p, device="cpu")
    gm.m.copy_(torch.arange(gm.total, dtype=torch.float32))
    before = gm.to_numpy()
    m_before = {k: t.clone() for k, t in gm._views(gm.m).items()}
    perm = torch.tensor(np.random.default_rng(5).permutation(37))
    gm.permute(perm)
    after = gm.to_numpy()
    for k in ("means", "log_scales", "quats", "opacity_logits"):
        np.testing.assert_array_equal(after[k], before[k][perm.numpy()])
    np.testing.assert_array_equal(after["sh"], before["sh"][:, perm.numpy()])
    for k, t in gm._views(gm.m).items():
        want = m_before[k][:, perm] if k == "sh" else m_before[k][perm]
        assert torch.equal(t, want)
