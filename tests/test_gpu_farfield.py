"""GPU far field (multipoles, derivatives tensor, Taylor series of order p;
Maksimova et al. 2021, Sec. 3.1) against the FP64 oracle of the same method,
and near + far against the Ewald sum of the periodic 1/r^2 force.

The GPU forms the multipoles from the FP32 cell-relative records and
evaluates the Taylor series in FP32 (the tensor and the convolution are
FP64), so it agrees with the FP64 oracle of the same method to about the
FP32 rounding of the far field; the method itself is within 1e-5 of the
Ewald force at p = 8.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2110_11398_gb300 import build
    build.build()
    return torch.device("cuda", 0)


def rel(got, ref):
    return np.linalg.norm(np.asarray(got, np.float64) - ref, axis=1) / np.linalg.norm(ref, axis=1)


def far_gpu(pos, L, cpd, eps, dev, p=8, mass=None, gm=None, R=2):
    from paper_2110_11398_gb300 import NearField
    nf = NearField(L, cpd, eps, radius=R, capacity=len(pos), device=dev)
    nf.far_init(p)
    m = None if mass is None else torch.from_numpy(mass.astype(np.float32)).to(dev)
    nf.bin(torch.from_numpy(pos.astype(np.float32)).to(dev), m, gm=gm)
    far = nf.far().cpu().numpy()
    near = nf.accel().cpu().numpy()
    nf.close()
    return far, near


@pytest.mark.parametrize("p", [4, 8])
def test_far_matches_the_oracle(dev, p):
    rng = np.random.default_rng(1)
    n, L, cpd = 3000, 1.0, 7
    pos = rng.random((n, 3)).astype(np.float32)
    mass = (rng.uniform(0.5, 1.5, n) / n).astype(np.float32)
    got, _ = far_gpu(pos, L, cpd, 1e-3, dev, p=p, mass=mass)
    ref = oracle.far_accel(pos.astype(np.float64), L, cpd, 2, p, mass=mass.astype(np.float64))
    e = rel(got, ref)
    assert np.median(e) < 2e-6 and np.quantile(e, 0.999) < 1e-4, (np.median(e), np.quantile(e, 0.999))


def test_far_equal_masses_clustered_box(dev):
    pos, _ = synth.clustered_box(24 ** 3, 3, n_halos=8)
    L, cpd = 1.0, 8
    gm = 1.0 / len(pos)
    got, _ = far_gpu(pos, L, cpd, 1e-4, dev, p=8, gm=gm)
    idx = np.arange(0, len(pos), 5)
    ref = oracle.far_accel(pos.astype(np.float64), L, cpd, 2, 8, m0=gm)[idx]
    e = rel(got[idx], ref)
    assert np.median(e) < 2e-6 and np.quantile(e, 0.999) < 1e-4, (np.median(e), np.quantile(e, 0.999))


def test_near_plus_far_is_the_ewald_force(dev):
    """With (almost) no softening, near field + far field at p = 8 is the
    total periodic force."""
    rng = np.random.default_rng(2)
    n, L, cpd = 600, 1.0, 7
    pos = rng.random((n, 3)).astype(np.float32)
    mass = (rng.uniform(0.5, 1.5, n) / n).astype(np.float32)
    far, near = far_gpu(pos, L, cpd, 1e-7, dev, p=8, mass=mass)
    tot = oracle.ewald_accel(pos.astype(np.float64), L, mass=mass.astype(np.float64))
    e = rel(far.astype(np.float64) + near, tot)
    assert np.median(e) < 2e-6 and e.max() < 1e-3, (np.median(e), e.max())


def test_far_accumulates_onto_the_near_field(dev):
    from paper_2110_11398_gb300 import NearField
    box = synth.tiny()
    nf = NearField(box.L, box.cpd, box.eps, capacity=box.n, device=dev)
    nf.far_init(6)
    nf.bin(torch.from_numpy(box.pos).to(dev), gm=box.gm)
    near = nf.accel()
    far = nf.far()
    both = nf.far(out=near.clone(), accumulate=True)
    assert torch.equal(both, near + far)
    st = nf.stats()
    assert st["far_ms"] > 0 and 0 < st["far_conv_ms"] <= st["far_ms"]
    nf.close()


def test_far_is_deterministic_and_follows_a_cell_shift(dev):
    rng = np.random.default_rng(4)
    n, L, cpd = 2000, 1.0, 8
    pos = rng.random((n, 3)).astype(np.float32)
    a1, _ = far_gpu(pos, L, cpd, 1e-3, dev, p=6, gm=1.0 / n)
    a2, _ = far_gpu(pos, L, cpd, 1e-3, dev, p=6, gm=1.0 / n)
    assert np.array_equal(a1, a2)
    # a whole-cell shift by a power-of-two fraction of the box moves the far field along
    shifted = np.mod(pos.astype(np.float64) + np.array([3, 1, 6]) / cpd, L).astype(np.float32)
    a3, _ = far_gpu(shifted, L, cpd, 1e-3, dev, p=6, gm=1.0 / n)
    scale = np.abs(a1).max()
    assert np.abs(a3 - a1).max() <= 1e-5 * scale


def test_far_argument_errors(dev):
    from paper_2110_11398_gb300 import NearField, NFError
    box = synth.tiny()
    nf = NearField(box.L, box.cpd, box.eps, capacity=box.n, device=dev)
    nf.bin(torch.from_numpy(box.pos).to(dev), gm=box.gm)
    with pytest.raises(NFError, match="NF_ESTATE"):
        nf.far()
    with pytest.raises(NFError, match="NF_EINVAL"):
        nf.far_init(9)
    with pytest.raises(NFError, match="NF_EINVAL"):
        nf.far_init(0)
    nf.close()


def test_batched_far_field_equals_each_box_alone(dev):
    """Several boxes in one context (two share a CPD, so they share a tensor):
    each box's far field equals that of its own one-box context bit for bit,
    and the oracle's."""
    from paper_2110_11398_gb300 import NearField
    rng = np.random.default_rng(30)
    specs = [(1.0, 7, 900), (2.0, 5, 600), (1.0, 7, 1200)]
    pos = [(rng.random((n, 3)) * L).astype(np.float32) for L, _, n in specs]
    offs = np.cumsum([0] + [n for _, _, n in specs])
    gms = [1.0 / n for _, _, n in specs]
    nb = NearField([L for L, _, _ in specs], [c for _, c, _ in specs], [1e-3] * 3, capacity=int(offs[-1]),
                   device=dev)
    nb.far_init(6)
    nb.bin(torch.from_numpy(np.concatenate(pos)).to(dev), gm=gms, box_offsets=offs)
    fb = nb.far().cpu().numpy()
    nb.close()
    for (L, cpd, n), x, gm, o0, o1 in zip(specs, pos, gms, offs[:-1], offs[1:]):
        got, _ = far_gpu(x, L, cpd, 1e-3, dev, p=6, gm=gm)
        assert np.array_equal(fb[o0:o1].view(np.uint32), got.view(np.uint32))
        ref = oracle.far_accel(x.astype(np.float64), L, cpd, 2, 6, m0=gm)
        e = rel(got, ref)
        assert np.median(e) < 2e-6, np.median(e)


@pytest.mark.parametrize("cpd,R", [(5, 1), (8, 3)])
def test_far_matches_the_oracle_other_radii(dev, cpd, R):
    rng = np.random.default_rng(20 + R)
    n, L = 1500, 1.0
    pos = rng.random((n, 3)).astype(np.float32)
    got, _ = far_gpu(pos, L, cpd, 1e-3, dev, p=6, gm=1.0 / n, R=R)
    ref = oracle.far_accel(pos.astype(np.float64), L, cpd, R, 6, m0=1.0 / n)
    e = rel(got, ref)
    assert np.median(e) < 2e-6 and np.quantile(e, 0.999) < 1e-4, (np.median(e), np.quantile(e, 0.999))


def test_far_field_properties_at_full_early_size(dev):
    """The 16.8M-particle early box (CPD 65) at p = 8, in the configuration the
    benchmark times, checked by properties that hold at any size: the far
    momentum sum_i m a_i cancels (each pair's two far terms are opposite, up
    to the truncation); a shift of every particle by whole cells moves the far
    field with them; and p = 6 is within the truncation error of p = 8."""
    from paper_2110_11398_gb300 import NearField
    box = synth.early()
    nf = NearField(box.L, box.cpd, box.eps, capacity=box.n, device=dev)
    pos = torch.from_numpy(box.pos).to(dev)
    nf.far_init(8)
    nf.bin(pos, gm=box.gm)
    a8 = nf.far()
    mom = a8.double().sum(0).abs().max().item()
    assert mom <= 1e-5 * a8.double().norm(dim=1).sum().item(), mom
    # whole-cell shift (3, 5, 1) cells, wrapped; float32 shifts are exact here
    # up to the rounding of x + k h, about 1e-7 cells
    shift = torch.tensor([3.0, 5.0, 1.0], dtype=torch.float64, device=dev) * (box.L / box.cpd)
    moved = torch.remainder(pos.double() + shift, box.L).float()
    nf.bin(moved, gm=box.gm)
    a8s = nf.far()
    d = (a8s - a8).double().norm(dim=1) / a8.double().norm(dim=1)
    assert d.median().item() < 1e-5, d.median().item()
    nf.far_init(6)
    nf.bin(pos, gm=box.gm)
    a6 = nf.far()
    d6 = (a6 - a8).double().norm(dim=1) / a8.double().norm(dim=1)
    assert d6.median().item() < 1e-4, d6.median().item()
    nf.close()


@pytest.mark.parametrize("p", [1, 2, 3, 5, 7])
def test_far_matches_the_oracle_every_order(dev, p):
    """Every order the library takes (the templated Taylor kernel has one
    instance per order), on an even CPD."""
    rng = np.random.default_rng(40 + p)
    n, L, cpd = 1500, 1.0, 6
    pos = rng.random((n, 3)).astype(np.float32)
    got, _ = far_gpu(pos, L, cpd, 1e-3, dev, p=p, gm=1.0 / n)
    ref = oracle.far_accel(pos.astype(np.float64), L, cpd, 2, p, m0=1.0 / n)
    e = rel(got, ref)
    assert np.median(e) < 2e-6 and np.quantile(e, 0.999) < 1e-4, (np.median(e), np.quantile(e, 0.999))
