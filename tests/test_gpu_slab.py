"""Slab decomposition on one GPU: several slab contexts, one per rank of a
ring, with their ghost slabs copied between them (Maksimova et al. 2021,
Sec. 3.2: each node owns a contiguous range of x slabs and receives the R
slabs beyond either end of it; Sec. 3.1: R is the near-field radius).

Each rank bins its owned particles in their global order, so every cell
holds the same particles in the same order as in a whole-box context, and
the per-sink sums run over the same sources in the same order: the
accelerations must equal the whole box's bit for bit (and so match the
oracle), the interaction counts must add up, and so must the FP64 momentum.
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
    oracle.build()
    return torch.device("cuda", 0)


def whole_box(box, dev, mass=None, precision="fp32"):
    from paper_2110_11398_gb300 import NearField
    nf = NearField(box.L, box.cpd, box.eps, radius=box.R, precision=precision, capacity=box.n, device=dev)
    pos = torch.from_numpy(box.pos).to(dev)
    nf.bin(pos, mass, gm=None if mass is not None else box.gm)
    a = nf.accel()
    st = nf.stats()
    out = a.cpu().numpy()
    nf.close()
    return out, st


def slab_run(box, dev, world, mass=None, precision="fp32", pos=None):
    from paper_2110_11398_gb300.slab import (SlabNearField, exchange_local, owners, slab_capacity,
                                             slab_of, slab_ranges)
    pos = torch.from_numpy(box.pos).to(dev) if pos is None else pos
    ranges = slab_ranges(box.cpd, world, box.R)
    own = owners(pos, box.L, box.cpd, ranges)
    slabs = slab_of(pos, box.L, box.cpd)
    fields = []
    for r, (x0, nx) in enumerate(ranges):
        idx = torch.nonzero(own == r).squeeze(1)
        sf = SlabNearField(box.L, box.cpd, box.eps, x0, nx, radius=box.R, precision=precision,
                           capacity=slab_capacity(slabs, x0, nx, box.R, box.cpd), device=dev)
        m = None if mass is None else mass[idx].contiguous()
        sf.bin(pos[idx].contiguous(), m, gm=None if m is not None else box.gm)
        fields.append((sf, idx))
    exchange_local([f for f, _ in fields])
    acc = torch.empty((box.n, 3), dtype=torch.float32, device=dev)
    stats = []
    for sf, idx in fields:
        acc[idx] = sf.accel()
        stats.append(sf.stats())
    for sf, _ in fields:
        sf.close()
    return acc.cpu().numpy(), stats


def assert_same_bits(a, b):
    assert np.array_equal(np.asarray(a, np.float32).view(np.uint32), np.asarray(b, np.float32).view(np.uint32))


@pytest.mark.parametrize("world", [1, 2, 3, 4])
def test_slabs_reproduce_the_whole_box_bit_for_bit(dev, world):
    pos, _ = synth.clustered_box(48 ** 3, 41, n_halos=20)
    box = synth.Box("cl48", pos, 1.0, 13, (1 / 48) / 40, 1 / 48 ** 3)
    ref, st = whole_box(box, dev)
    got, sts = slab_run(box, dev, world)
    assert_same_bits(got, ref)
    assert sum(s["interactions"] for s in sts) == st["interactions"]
    assert sum(s["n_particles"] for s in sts) == box.n
    P = np.sum([s["momentum"] for s in sts], axis=0)
    S = sum(s["abs_momentum"] for s in sts)
    assert abs(S - st["abs_momentum"]) <= 1e-12 * S
    assert np.all(np.abs(P - np.array(st["momentum"])) <= 1e-12 * S)
    idx = np.arange(0, box.n, 13)
    oref = oracle.accel(box.pos, box.L, box.cpd, box.R, box.eps, m0=box.gm, sinks=idx)
    e = np.linalg.norm(got[idx] - oref, axis=1) / np.linalg.norm(oref, axis=1)
    assert np.median(e) <= 1e-6 and np.quantile(e, 0.999) <= 1e-4


@pytest.mark.parametrize("R,cpd,world", [(1, 6, 3), (2, 5, 2), (3, 14, 4), (2, 8, 4)])
def test_slabs_other_radii_and_narrow_ranks(dev, R, cpd, world):
    """Ranks owning exactly R slabs (both exports are then the same slabs),
    two ranks that are each other's left and right neighbour, R = 1 and 3."""
    rng = np.random.default_rng(R * 31 + cpd)
    n = 12000
    pos = rng.random((n, 3)).astype(np.float32)
    box = synth.Box("r", pos, 1.0, cpd, 0.05 / cpd, 1.0 / n, R)
    ref, _ = whole_box(box, dev)
    got, _ = slab_run(box, dev, world)
    assert_same_bits(got, ref)


@pytest.mark.parametrize("precision", ["fp32_comp", "fp32_comp_pair"])
def test_slabs_unequal_masses_and_compensated(dev, precision):
    box = synth.tiny(seed=12)
    mass = torch.from_numpy(np.random.default_rng(2).uniform(0.2, 3.0, box.n).astype(np.float32) / box.n).to(dev)
    ref, _ = whole_box(box, dev, mass=mass, precision=precision)
    got, _ = slab_run(box, dev, 3, mass=mass, precision=precision)
    assert_same_bits(got, ref)


def test_slabs_after_a_drift(dev):
    """Positions move, particles change slabs: re-route, re-bin, re-exchange."""
    from paper_2110_11398_gb300 import NearField
    box = synth.tiny(seed=4)
    nf = NearField(box.L, box.cpd, box.eps, capacity=box.n, device=dev)
    pos = torch.from_numpy(box.pos).to(dev)
    vel = torch.from_numpy((np.random.default_rng(5).standard_normal((box.n, 3)) * 0.3).astype(np.float32)).to(dev)
    nf.bin(pos, gm=box.gm)
    nf.drift(pos, vel, 0.2)
    nf.bin(pos, gm=box.gm)
    ref = nf.accel().cpu().numpy()
    nf.close()
    got, _ = slab_run(box, dev, 3, pos=pos)
    assert_same_bits(got, ref)


def test_slab_context_errors(dev):
    from paper_2110_11398_gb300 import NFError
    from paper_2110_11398_gb300.slab import SlabNearField
    box = synth.tiny(seed=1)
    pos = torch.from_numpy(box.pos).to(dev)
    with pytest.raises(NFError, match="NF_EINVAL"):          # fewer than R slabs
        SlabNearField(1.0, 9, box.eps, 0, 1, capacity=box.n, device=dev)
    with pytest.raises(NFError, match="NF_EINVAL"):          # FP64 has no FP32 ghost records
        SlabNearField(1.0, 9, box.eps, 0, 3, precision="fp64", capacity=box.n, device=dev)
    sf = SlabNearField(1.0, 9, box.eps, 3, 3, capacity=box.n, device=dev)
    with pytest.raises(NFError, match="NF_ERANGE"):          # particles of other slabs
        sf.bin(pos, gm=box.gm)
    xs = np.floor(box.pos[:, 0].astype(np.float64) * 9).astype(int)
    mine = torch.from_numpy(np.nonzero((xs >= 3) & (xs < 6))[0]).to(dev)
    sf.bin(pos[mine].contiguous(), gm=box.gm)
    with pytest.raises(NFError, match="NF_ESTATE"):          # no ghosts yet
        sf.accel()
    c0, r0 = sf.export(0)
    c1, r1 = sf.export(1)
    bad = c0.clone()
    bad[5] += 1                                              # counts do not add up
    with pytest.raises(NFError, match="NF_EINVAL"):
        sf.import_ghosts((c1, r1), (bad, r0))
    neg = c0.clone()
    neg[1] += neg[0] + 1
    neg[0] = -1                                              # same total, one count negative
    with pytest.raises(NFError, match="NF_EINVAL"):
        sf.import_ghosts((c1, r1), (neg, r0))
    with pytest.raises(NFError, match="NF_ESTATE"):          # a failed import leaves no ghosts
        sf.accel()
    sf.import_ghosts((c1, r1), (c0, r0))
    sf.accel()
    with pytest.raises(NFError, match="NF_EINVAL"):
        sf.vjp(torch.zeros((sf.n, 3), device=dev))
    with pytest.raises(NFError, match="NF_EINVAL"):
        sf.far_init(4)
    sf.close()


def test_slab_of_matches_the_binning(dev):
    from paper_2110_11398_gb300.slab import slab_of
    for L, cpd in ((1.0, 129), (3.7, 17), (250.0, 64)):
        rng = np.random.default_rng(cpd)
        x = (rng.random((50000, 3)) * L).astype(np.float32)
        x[x >= np.float32(L)] = 0
        faces = np.array([k * L / cpd for k in range(cpd)], np.float32)
        x[:cpd, 0] = faces
        x[cpd:2 * cpd, 0] = np.nextafter(faces, np.float32(0))
        x[cpd:2 * cpd, 0][x[cpd:2 * cpd, 0] < 0] = 0
        x[-1, 0] = np.float32(L)                              # outside
        got = slab_of(torch.from_numpy(x).to(dev), L, cpd).cpu().numpy()
        cid = oracle.bin_particles(x[:-1], L, cpd)["cid"]
        assert np.array_equal(got[:-1], cid // (cpd * cpd))
        assert got[-1] == -1
