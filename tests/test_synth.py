"""The seeded generators: shapes, ranges, determinism and recipe bookkeeping."""
import numpy as np

import synth


def test_tiny_and_early_shapes():
    t = synth.tiny()
    assert t.pos.shape == (32 ** 3, 3) and t.pos.dtype == np.float32
    assert t.cpd == 9 and t.R == 2
    assert np.all(t.pos >= 0) and np.all(t.pos < 1)
    assert np.isclose(t.eps, (1 / 32) / 40) and np.isclose(t.gm, 1 / 32 ** 3)
    e = synth.early(n_side=32, cpd=9)
    assert e.pos.shape == (32 ** 3, 3) and np.all(e.pos < 1) and np.all(e.pos >= 0)


def test_deterministic():
    a = synth.tiny()
    b = synth.tiny()
    assert np.array_equal(a.pos, b.pos)
    c = synth.tiny(seed=1)
    assert not np.array_equal(a.pos, c.pos)


def test_clustered_recipe_counts():
    pos, info = synth.clustered_box(64 ** 3, 5, n_halos=40)
    n = 64 ** 3
    assert pos.shape == (n, 3) and pos.dtype == np.float32
    assert np.all(pos >= 0) and np.all(pos < 1)
    assert info["n_lattice"] + info["n_halo_particles"] == n
    assert info["n_halo_particles"] == round(0.4 * n)
    assert info["max_halo"] >= 100


def test_rescale_largest_remainder_sums_exactly():
    raw = np.array([1.5, 2.5, 3.3, 100.7])
    out = synth._rescale_counts(raw, 1001)
    assert out.sum() == 1001 and np.all(out >= 0)


def test_batched_box_sizes():
    boxes = synth.batched(n_boxes=3, lo_side=16, hi_side=24)
    for b in boxes:
        assert 16 ** 3 <= b.n <= 24 ** 3
        assert b.cpd == max(5, round((b.n / 60) ** (1 / 3)))
        assert np.all(b.pos < 1) and np.all(b.pos >= 0)


def test_cotangent():
    w = synth.cotangent(1000, 4)
    assert w.shape == (1000, 3) and w.dtype == np.float32
    assert abs(w.mean()) < 0.1 and abs(w.std() - 1) < 0.1
