"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances. Forces: median fractional error <= 1e-6 and 99.9th percentile
<= 1e-4 per sink, e_i = |a_i - a_i^ref| / |a_i^ref|. Binning (cell table,
permutation, cell-relative float32 coordinates): bit-exact. The FP64
reference kernel: within 1e-11 of the oracle (both are double sums of the
same pairs; they differ in summation order and in the oracle's use of
absolute instead of cell-relative coordinates).

Paper: Maksimova et al. 2021, Sec. 3.1 (cells, near field), Sec. 5.2
(Plummer softening).
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

MED_TOL, P999_TOL = 1e-6, 1e-4


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2110_11398_gb300 import build
    build.build()
    oracle.build()
    return torch.device("cuda", 0)


def frac_err(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.linalg.norm(ref, axis=1)
    den = np.where(den > 0, den, 1.0)
    return np.linalg.norm(got - ref, axis=1) / den


def assert_parity(got, ref, med=MED_TOL, p999=P999_TOL, what=""):
    e = frac_err(got, ref)
    m, q = float(np.median(e)), float(np.quantile(e, 0.999))
    assert m <= med and q <= p999, f"{what}: median {m:.3e} (<= {med}), p99.9 {q:.3e} (<= {p999})"
    return m, q


def make_nf(box, dev, precision="fp32", capacity=None, **tune):
    from paper_2110_11398_gb300 import NearField
    nf = NearField(box.L, box.cpd, box.eps, radius=box.R, precision=precision,
                   capacity=capacity or max(box.n, 1), device=dev)
    if tune:
        nf.set_tuning(**tune)
    return nf


def gpu_accel(box, dev, precision="fp32", mass=None, f64=False, **tune):
    nf = make_nf(box, dev, precision, **tune)
    pos = torch.from_numpy(box.pos).to(dev)
    m = None if mass is None else torch.from_numpy(np.asarray(mass, np.float32)).to(dev)
    nf.bin(pos, m, gm=None if m is not None else box.gm)
    a = nf.accel(dtype=torch.float64 if f64 else torch.float32)
    torch.cuda.synchronize()
    out = a.cpu().numpy()
    st = nf.stats()
    nf.close()
    return out, st


# ---------------------------------------------------------------- binning
def _bin_case(box, dev):
    nf = make_nf(box, dev)
    nf.bin(torch.from_numpy(box.pos).to(dev), gm=box.gm)
    cs, perm, srt = (t.cpu().numpy() for t in nf.binning())
    nf.close()
    ref = oracle.bin_particles(box.pos, box.L, box.cpd)
    assert np.array_equal(cs.astype(np.int64), ref["cell_start"])
    assert np.array_equal(perm.astype(np.int64), ref["perm"])
    assert np.array_equal(srt[:, :3].view(np.uint32), ref["rel"].view(np.uint32))
    assert np.all(srt[:, 3] == np.float32(box.gm))


def test_binning_bit_exact_tiny(dev):
    _bin_case(synth.tiny(), dev)


@pytest.mark.parametrize("L,cpd", [(1.0, 9), (3.7, 7), (250.0, 16), (1.0, 33), (0.5, 13),
                                   (2.0, 129), (1024.0, 65), (1.0, 1000)])
def test_binning_bit_exact_faces_and_non_pow2_box(dev, L, cpd):
    rng = np.random.default_rng(cpd)
    x = rng.random((20000, 3)).astype(np.float32) * np.float32(L)
    faces = np.array([k * L / cpd for k in range(cpd)], np.float32)
    near = np.concatenate([faces, np.nextafter(faces, np.float32(0)), np.nextafter(faces, np.float32(2 * L)),
                           [np.nextafter(np.float32(L), np.float32(0))]])
    near = near[(near >= 0) & (near < np.float32(L))]
    blk = np.stack([near, near[::-1], np.roll(near, 5)], 1).astype(np.float32)
    pos = np.concatenate([x, blk, x[:500]], 0)          # duplicates: stability
    rng.shuffle(pos)
    box = synth.Box("faces", np.ascontiguousarray(pos), L, cpd, 0.01 * L / cpd, 1.0 / len(pos))
    _bin_case(box, dev)


def test_binning_clustered_bit_exact(dev):
    pos, _ = synth.clustered_box(64 ** 3, 77, n_halos=30)
    box = synth.Box("clustered64", pos, 1.0, 17, (1 / 64) / 40, 1 / 64 ** 3)
    _bin_case(box, dev)


# ---------------------------------------------------------------- forward
@pytest.mark.parametrize("precision", ["fp32", "fp32_comp", "fp32_comp_pair"])
def test_tiny_forward_parity(dev, precision):
    box = synth.tiny()
    ref = oracle.accel(box.pos, box.L, box.cpd, box.R, box.eps, m0=box.gm)
    got, st = gpu_accel(box, dev, precision)
    assert_parity(got, ref, what=precision)
    cid = oracle.bin_particles(box.pos, box.L, box.cpd)["cid"]
    assert st["interactions"] == oracle.interactions(cid, box.cpd, box.R)
    assert st["max_occupancy"] == np.bincount(cid).max()


def test_tiny_forward_fp64_reference_kernel(dev):
    box = synth.tiny()
    ref = oracle.accel(box.pos, box.L, box.cpd, box.R, box.eps, m0=box.gm)
    got, _ = gpu_accel(box, dev, "fp64", f64=True)
    e = frac_err(got, ref)
    assert np.max(e) < 1e-11, np.max(e)


def test_comp_is_not_less_accurate(dev):
    box = synth.early(n_side=48, cpd=13)
    ref = oracle.accel(box.pos, box.L, box.cpd, box.R, box.eps, m0=box.gm)
    e32 = frac_err(gpu_accel(box, dev, "fp32")[0], ref)
    ec = frac_err(gpu_accel(box, dev, "fp32_comp")[0], ref)
    ep = frac_err(gpu_accel(box, dev, "fp32_comp_pair")[0], ref)
    assert np.median(ec) <= np.median(e32) * 1.05
    assert np.median(ep) <= np.median(ec) * 1.05
    assert_parity(gpu_accel(box, dev, "fp32")[0], ref)


def test_comp_on_dense_cells(dev):
    """Clustered cells with thousands of sources per sink: the fold of many
    tile sums is where the compensated total pays; both compensated forms
    must be at least as accurate as plain FP32 there."""
    pos, _ = synth.clustered_box(48 ** 3, 31, n_halos=12)
    box = synth.Box("cl48", pos, 1.0, 13, (1 / 48) / 40, 1 / 48 ** 3)
    idx = np.arange(0, box.n, 5)
    ref = oracle.accel(box.pos, box.L, box.cpd, box.R, box.eps, m0=box.gm, sinks=idx)
    errs = {p: frac_err(gpu_accel(box, dev, p)[0][idx], ref) for p in ("fp32", "fp32_comp", "fp32_comp_pair")}
    for p, e in errs.items():
        assert np.median(e) <= MED_TOL and np.quantile(e, 0.999) <= P999_TOL, p
    assert np.median(errs["fp32_comp"]) <= np.median(errs["fp32"]) * 1.05
    assert np.median(errs["fp32_comp_pair"]) <= np.median(errs["fp32"]) * 1.05


@pytest.mark.parametrize("precision", ["fp32", "fp32_comp", "fp32_comp_pair", "fp64"])
def test_unequal_masses(dev, precision):
    box = synth.tiny(seed=5)
    mass = np.random.default_rng(3).uniform(0.2, 3.0, box.n).astype(np.float32) / box.n
    ref = oracle.accel(box.pos, box.L, box.cpd, box.R, box.eps, mass=mass.astype(np.float64))
    got, st = gpu_accel(box, dev, precision, mass=mass, f64=precision == "fp64")
    if precision == "fp64":
        assert np.max(frac_err(got, ref)) < 1e-11
    else:
        assert_parity(got, ref, what=precision)
    P = np.array(st["momentum"])
    assert np.all(np.abs(P) <= 1e-5 * st["abs_momentum"])


@pytest.mark.parametrize("box_kind", ["early", "clustered", "tiny"])
def test_pencils_on_and_off(dev, box_kind):
    """Four-cell pencils served by one block (sparse cells) against the
    per-warp items alone: both within the tolerance, with equal and
    unequal masses; on the near-uniform box most sinks go to pencils."""
    if box_kind == "early":
        box = synth.early(n_side=48, cpd=13)
    elif box_kind == "clustered":
        pos, _ = synth.clustered_box(48 ** 3, 9, n_halos=15)
        box = synth.Box("cl48", pos, 1.0, 13, (1 / 48) / 40, 1 / 48 ** 3)
    else:
        box = synth.tiny(seed=6)
    ref = oracle.accel(box.pos, box.L, box.cpd, box.R, box.eps, m0=box.gm)
    on, st_on = gpu_accel(box, dev, use_pencils=1)
    off, st_off = gpu_accel(box, dev, use_pencils=0)
    assert_parity(on, ref, what=f"pencils {box_kind}")
    assert_parity(off, ref, what=f"no pencils {box_kind}")
    assert st_off["n_pencils"] == 0 and st_on["n_pencils"] > 0
    assert st_on["interactions"] == st_off["interactions"]
    if box_kind == "early":                 # every full pencil of the near-uniform box
        assert st_on["n_pencils"] == box.cpd ** 2 * (box.cpd // 4)
    mass = np.random.default_rng(3).uniform(0.2, 3.0, box.n).astype(np.float32) / box.n
    refm = oracle.accel(box.pos, box.L, box.cpd, box.R, box.eps, mass=mass.astype(np.float64))
    gotm, stm = gpu_accel(box, dev, mass=mass, use_pencils=1)
    assert stm["n_pencils"] > 0
    assert_parity(gotm, refm, what=f"pencils, masses {box_kind}")


@pytest.mark.parametrize("box_kind,pencils", [("lattice", 1), ("lattice", 0), ("clustered", 1)])
def test_small_items_on_and_off(dev, box_kind, pencils):
    """Work items of at most 8 sinks (the sinks a cell has left after its full
    groups) served by the small-item kernel, which reads its sources straight
    from the records, against the tiled kernel: both within the tolerance,
    with equal and unequal masses, on the same items."""
    if box_kind == "lattice":                   # ~64 per cell: many cells keep a few sinks over
        box = synth.early(n_side=52, cpd=13)
    else:
        pos, _ = synth.clustered_box(48 ** 3, 9, n_halos=15)
        box = synth.Box("cl48", pos, 1.0, 13, (1 / 48) / 40, 1 / 48 ** 3)
    ref = oracle.accel(box.pos, box.L, box.cpd, box.R, box.eps, m0=box.gm)
    on, st_on = gpu_accel(box, dev, use_pencils=pencils, small_items=1)
    off, st_off = gpu_accel(box, dev, use_pencils=pencils, small_items=0)
    assert_parity(on, ref, what=f"small items {box_kind}")
    assert_parity(off, ref, what=f"no small items {box_kind}")
    assert st_on["n_small"] > 0 and st_off["n_small"] == 0
    assert st_on["n_items"] == st_off["n_items"]
    assert st_on["interactions"] == st_off["interactions"]
    mass = np.random.default_rng(4).uniform(0.2, 3.0, box.n).astype(np.float32) / box.n
    refm = oracle.accel(box.pos, box.L, box.cpd, box.R, box.eps, mass=mass.astype(np.float64))
    gotm, stm = gpu_accel(box, dev, mass=mass, use_pencils=pencils, small_items=1)
    assert stm["n_small"] > 0
    assert_parity(gotm, refm, what=f"small items, masses {box_kind}")


@pytest.mark.parametrize("tile,K,precision", [(64, 4, "fp32"), (256, 4, "fp32"), (64, 1, "fp32_comp"),
                                               (256, 2, "fp32_comp"), (256, 2, "fp32_comp_pair")])
def test_source_tiles(dev, tile, K, precision):
    """Every staged-tile size gives the same accelerations within the
    tolerance, with equal and unequal masses."""
    box = synth.early(n_side=40, cpd=11)
    ref = oracle.accel(box.pos, box.L, box.cpd, box.R, box.eps, m0=box.gm)
    got, _ = gpu_accel(box, dev, precision, sinks_per_lane=K, source_tile=tile)
    assert_parity(got, ref, what=f"tile {tile} K={K} {precision}")
    mass = np.random.default_rng(tile).uniform(0.2, 3.0, box.n).astype(np.float32) / box.n
    refm = oracle.accel(box.pos, box.L, box.cpd, box.R, box.eps, mass=mass.astype(np.float64))
    gotm, _ = gpu_accel(box, dev, precision, mass=mass, sinks_per_lane=K, source_tile=tile)
    assert_parity(gotm, refm, what=f"tile {tile} masses")


@pytest.mark.parametrize("K,warps", [(1, 2), (1, 4), (2, 4), (2, 8), (4, 4), (4, 16), (2, 16)])
def test_launch_shapes_all_agree(dev, K, warps):
    box = synth.tiny(seed=2)
    ref = oracle.accel(box.pos, box.L, box.cpd, box.R, box.eps, m0=box.gm)
    got, _ = gpu_accel(box, dev, "fp32", sinks_per_lane=K, warps_per_block=warps)
    assert_parity(got, ref, what=f"K={K} warps={warps}")


@pytest.mark.parametrize("R,cpd,n", [(1, 3, 3000), (1, 8, 20000), (2, 5, 4000), (3, 7, 8000), (3, 11, 30000)])
def test_radius_and_smallest_cpd(dev, R, cpd, n):
    rng = np.random.default_rng(R * 100 + cpd)
    pos = rng.random((n, 3)).astype(np.float32)
    box = synth.Box("r", pos, 1.0, cpd, 0.05 / cpd, 1.0 / n, R)
    ref = oracle.accel(pos, 1.0, cpd, R, box.eps, m0=box.gm)
    got, st = gpu_accel(box, dev)
    assert_parity(got, ref, what=f"R={R} cpd={cpd}")
    cid = oracle.bin_particles(pos, 1.0, cpd)["cid"]
    assert st["interactions"] == oracle.interactions(cid, cpd, R)


def test_non_pow2_box_side(dev):
    rng = np.random.default_rng(8)
    L = 3.7
    pos = (rng.random((30000, 3)) * L).astype(np.float32)
    pos[pos >= np.float32(L)] = 0
    box = synth.Box("L3.7", pos, L, 9, 0.02 * L / 9, 1.0 / 30000)
    ref = oracle.accel(pos, L, 9, 2, box.eps, m0=box.gm)
    got, _ = gpu_accel(box, dev)
    assert_parity(got, ref)


def test_large_cpd_multilevel_scan(dev):
    """CPD = 400 gives 6.4e7 cells, more than one scan level covers: the cell
    table must still be exact and the forces right."""
    rng = np.random.default_rng(21)
    n, cpd = 200000, 400
    pos = rng.random((n, 3)).astype(np.float32)
    box = synth.Box("cpd400", pos, 1.0, cpd, 0.1 / cpd, 1.0 / n)
    nf = make_nf(box, dev)
    nf.bin(torch.from_numpy(pos).to(dev), gm=box.gm)
    cs, perm, _ = (t.cpu().numpy() for t in nf.binning())
    acc = nf.accel().cpu().numpy()
    nf.close()
    ref = oracle.bin_particles(pos, 1.0, cpd)
    assert np.array_equal(cs.astype(np.int64), ref["cell_start"])
    assert np.array_equal(perm.astype(np.int64), ref["perm"])
    idx = np.arange(0, n, 101)
    ra = oracle.accel(pos, 1.0, cpd, 2, box.eps, m0=box.gm, sinks=idx, cid=ref["cid"])
    assert_parity(acc[idx], ra, what="cpd400")


def test_one_dense_cell_and_empty_cells(dev):
    """5000 particles in one cell of a CPD=9 box, plus a few elsewhere: the
    dense cell is split over many items; most cells are empty."""
    rng = np.random.default_rng(4)
    dense = (np.array([4, 4, 4]) + rng.random((5000, 3))) / 9
    sparse = rng.random((37, 3))
    pos = np.concatenate([dense, sparse]).astype(np.float32)
    box = synth.Box("dense", pos, 1.0, 9, 0.002, 1.0 / len(pos))
    ref = oracle.accel(pos, 1.0, 9, 2, box.eps, m0=box.gm)
    got, st = gpu_accel(box, dev)
    assert_parity(got, ref)
    assert st["max_occupancy"] >= 5000


@pytest.mark.parametrize("n", [0, 1, 2, 31, 33, 64, 65, 129])
def test_tiny_sizes(dev, n):
    rng = np.random.default_rng(n)
    pos = rng.random((n, 3)).astype(np.float32)
    box = synth.Box("n", pos, 1.0, 5, 0.01, 1.0)
    got, st = gpu_accel(box, dev)
    assert got.shape == (n, 3)
    if n:
        ref = oracle.accel(pos, 1.0, 5, 2, 0.01, m0=1.0)
        if n == 1:
            assert np.all(got == 0)
        else:
            assert_parity(got, ref, what=f"n={n}")
    assert st["interactions"] == n * n          # CPD = 2R+1: every pair once


def test_out_of_range_position_is_rejected(dev):
    from paper_2110_11398_gb300 import NFError
    box = synth.tiny()
    nf = make_nf(box, dev)
    for bad in (np.nan, 1.0, -0.25, np.inf):
        pos = box.pos.copy()
        pos[123, 2] = bad
        with pytest.raises(NFError, match="NF_ERANGE"):
            nf.bin(torch.from_numpy(pos).to(dev), gm=box.gm)
        with pytest.raises(NFError, match="NF_ESTATE"):
            nf.accel()
    nf.bin(torch.from_numpy(box.pos).to(dev), gm=box.gm)   # recovers
    nf.accel()
    nf.close()


def test_compute_before_bin_is_an_error(dev):
    from paper_2110_11398_gb300 import NFError
    nf = make_nf(synth.tiny(), dev)
    with pytest.raises(NFError, match="NF_ESTATE"):
        nf.accel(out=torch.empty((0, 3), device=dev))
    nf.close()


def test_deterministic_and_graph_equals_direct(dev):
    box = synth.tiny(seed=9)
    a1, _ = gpu_accel(box, dev, use_graph=1)
    a2, _ = gpu_accel(box, dev, use_graph=1)
    a3, _ = gpu_accel(box, dev, use_graph=0)
    assert np.array_equal(a1.view(np.uint32), a2.view(np.uint32))
    assert np.array_equal(a1.view(np.uint32), a3.view(np.uint32))


def test_repeated_calls_with_new_outputs_and_rebin(dev):
    """Graph replays with changing output pointers and fresh binnings."""
    nf = make_nf(synth.tiny(), dev)
    outs = []
    for seed in (0, 1, 0):
        box = synth.tiny(seed=seed)
        nf.bin(torch.from_numpy(box.pos).to(dev), gm=box.gm)
        for _ in range(2):
            outs.append(nf.accel().cpu().numpy())
    nf.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[4])
    assert not np.array_equal(outs[0], outs[2])


def test_host_buffer_path_with_pinned_buffers(dev):
    """Page-locked host buffers (the end-to-end path's fast case, where the
    pair kernels store the accelerations into the host buffer directly) give
    the device path's result, also on a second call that replays the graph,
    and the momentum diagnostic reads the same accelerations."""
    box = synth.tiny(seed=3)
    nf = make_nf(box, dev)
    hpos = torch.from_numpy(box.pos).pin_memory().numpy()
    hacc = torch.full((box.n, 3), float("nan"), dtype=torch.float32).pin_memory().numpy()
    nf.accel_host(hpos, gm=box.gm, out=hacc)
    a1 = hacc.copy()
    hacc[:] = np.nan
    nf.accel_host(hpos, gm=box.gm, out=hacc)            # graph replay into the same buffer
    st_host = nf.stats()
    nf.bin(torch.from_numpy(box.pos).to(dev), gm=box.gm)
    a_dev = nf.accel().cpu().numpy()
    st = nf.stats()
    nf.close()
    assert np.array_equal(a1, a_dev) and np.array_equal(hacc, a_dev)
    assert np.all(np.abs(np.array(st["momentum"])) <= 1e-5 * st["abs_momentum"])
    assert st_host["abs_momentum"] == pytest.approx(st["abs_momentum"], rel=1e-12)
    assert np.allclose(st_host["momentum"], st["momentum"], rtol=0, atol=1e-12 * st["abs_momentum"])


def test_host_buffer_path_pinned_ragged_and_unaligned(dev):
    """Page-locked positions that the key kernel reads itself: a count that
    is not a whole number of its 1024-particle chunks, rows that start 12
    bytes into the page-locked block (not 16-byte aligned), and per-particle
    masses; the result equals the device path's bit for bit."""
    box = synth.tiny(seed=5)
    n = box.n - 77
    pos = box.pos[:n]
    rng = np.random.default_rng(5)
    mass = (rng.random(n, dtype=np.float32) + 0.5) / n
    big = torch.zeros((n + 1, 3), dtype=torch.float32).pin_memory()
    big[1:] = torch.from_numpy(pos)
    hpos = big.numpy()[1:]
    assert hpos.ctypes.data % 16 == 12
    hacc = torch.full((n, 3), float("nan"), dtype=torch.float32).pin_memory().numpy()
    nf = make_nf(box, dev)
    nf.accel_host(hpos, mass, out=hacc)
    nf.bin(torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev))
    a_dev = nf.accel().cpu().numpy()
    nf.close()
    assert np.array_equal(hacc, a_dev)


@pytest.mark.parametrize("pin_pos,pin_acc", [(True, False), (False, True)])
def test_host_buffer_path_mixed_buffers(dev, pin_pos, pin_acc):
    """One page-locked buffer and one pageable one: the kernels read the
    page-locked positions (or write the page-locked accelerations) directly,
    the other side goes through the staged copy; the result equals the
    device path's bit for bit."""
    box = synth.tiny(seed=4)
    hpos = torch.from_numpy(box.pos).pin_memory().numpy() if pin_pos else box.pos.copy()
    if pin_acc:
        hacc = torch.full((box.n, 3), float("nan"), dtype=torch.float32).pin_memory().numpy()
    else:
        hacc = np.full((box.n, 3), np.nan, np.float32)
    nf = make_nf(box, dev)
    nf.accel_host(hpos, gm=box.gm, out=hacc)
    nf.bin(torch.from_numpy(box.pos).to(dev), gm=box.gm)
    a_dev = nf.accel().cpu().numpy()
    nf.close()
    assert np.array_equal(hacc, a_dev)


def test_host_buffer_path_matches_device_path(dev):
    box = synth.tiny(seed=3)
    nf = make_nf(box, dev)
    a_host = nf.accel_host(box.pos, gm=box.gm)
    nf.bin(torch.from_numpy(box.pos).to(dev), gm=box.gm)
    a_dev = nf.accel().cpu().numpy()
    nf.close()
    assert np.array_equal(a_host, a_dev)


def test_batched_boxes_bit_identical_to_plain(dev):
    from paper_2110_11398_gb300 import NearField
    boxes = synth.batched(n_boxes=4, lo_side=20, hi_side=40)
    boxes[1].L = 2.0
    boxes[1].pos = (boxes[1].pos * 2).astype(np.float32)
    boxes[1].eps *= 2
    n = sum(b.n for b in boxes)
    offs = np.cumsum([0] + [b.n for b in boxes])
    nfb = NearField([b.L for b in boxes], [b.cpd for b in boxes], [b.eps for b in boxes],
                    capacity=n, device=dev)
    pos = torch.from_numpy(np.concatenate([b.pos for b in boxes])).to(dev)
    mass = torch.from_numpy(np.concatenate([np.full(b.n, b.gm, np.float32) for b in boxes])).to(dev)
    nfb.bin(pos, mass, box_offsets=offs)
    ab = nfb.accel().cpu().numpy()
    inter = nfb.stats()["interactions"]
    nfb.close()
    tot = 0
    for b, o0, o1 in zip(boxes, offs[:-1], offs[1:]):
        nf = make_nf(b, dev)
        nf.bin(torch.from_numpy(b.pos).to(dev), mass[o0:o1].contiguous())
        ap = nf.accel().cpu().numpy()
        tot += nf.stats()["interactions"]
        nf.close()
        assert np.array_equal(ab[o0:o1].view(np.uint32), ap.view(np.uint32))
        ref = oracle.accel(b.pos, b.L, b.cpd, b.R, b.eps, m0=b.gm,
                           sinks=np.arange(0, b.n, 7))
        assert_parity(ap[::7], ref, what=b.name)
    assert inter == tot


def test_batched_per_box_masses_bit_identical_to_plain(dev):
    """Per-box equal masses (nf_set_box_masses) keep the equal-mass kernel;
    each box's result equals its own single-box context bit for bit."""
    from paper_2110_11398_gb300 import NearField
    boxes = synth.batched(n_boxes=5, lo_side=18, hi_side=36, seed0=11)
    offs = np.cumsum([0] + [b.n for b in boxes])
    nfb = NearField([b.L for b in boxes], [b.cpd for b in boxes], [b.eps for b in boxes],
                    capacity=int(offs[-1]), device=dev)
    pos = torch.from_numpy(np.concatenate([b.pos for b in boxes])).to(dev)
    nfb.bin(pos, gm=[b.gm for b in boxes], box_offsets=offs)
    ab = nfb.accel().cpu().numpy()
    mom = nfb.stats()
    nfb.close()
    for b, o0, o1 in zip(boxes, offs[:-1], offs[1:]):
        nf = make_nf(b, dev)
        nf.bin(torch.from_numpy(b.pos).to(dev), gm=b.gm)
        ap = nf.accel().cpu().numpy()
        nf.close()
        assert np.array_equal(ab[o0:o1].view(np.uint32), ap.view(np.uint32))
    assert np.all(np.abs(np.array(mom["momentum"])) <= 1e-5 * mom["abs_momentum"])


def test_autotune_picks_a_valid_shape(dev, tmp_path):
    import json
    box = synth.tiny()
    nf = make_nf(box, dev)
    nf.bin(torch.from_numpy(box.pos).to(dev), gm=box.gm)
    cache = str(tmp_path / "tune.json")
    t = nf.autotune(reps=1, cache=cache)
    assert t["sinks_per_lane"] in (1, 2, 4) and t["warps_per_block"] in (4, 8)
    assert t["source_tile"] in (64, 128, 256)
    ref = oracle.accel(box.pos, box.L, box.cpd, box.R, box.eps, m0=box.gm)
    assert_parity(nf.accel().cpu().numpy(), ref)
    nf.close()
    # a second context reads the cached shape instead of timing again
    (key, rec), = json.load(open(cache)).items()
    rec["sinks_per_lane"] = 1 if t["sinks_per_lane"] != 1 else 2
    json.dump({key: rec}, open(cache, "w"))
    nf2 = make_nf(box, dev)
    nf2.bin(torch.from_numpy(box.pos).to(dev), gm=box.gm)
    assert nf2.autotune(reps=1, cache=cache)["sinks_per_lane"] == rec["sinks_per_lane"]
    nf2.close()


def test_momentum_diagnostic(dev):
    box = synth.tiny()
    _, st = gpu_accel(box, dev)
    P = np.array(st["momentum"])
    assert st["abs_momentum"] > 0
    assert np.all(np.abs(P) <= 1e-5 * st["abs_momentum"]), (P, st["abs_momentum"])


# ---------------------------------------------------------------- adjoint
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_tiny_vjp_parity(dev, precision):
    box = synth.tiny()
    w = synth.cotangent(box.n, 4)
    ref = oracle.vjp(box.pos, w, box.L, box.cpd, box.R, box.eps, m0=box.gm)
    nf = make_nf(box, dev, precision)
    nf.bin(torch.from_numpy(box.pos).to(dev), gm=box.gm)
    g = nf.vjp(torch.from_numpy(w).to(dev)).cpu().numpy()
    nf.close()
    if precision == "fp64":
        assert np.median(frac_err(g, ref)) < 1e-7    # FP64 pairs, FP32 output
    else:
        assert_parity(g, ref, what="vjp")


def test_vjp_unequal_masses(dev):
    box = synth.tiny(seed=6)
    mass = np.random.default_rng(1).uniform(0.2, 3.0, box.n).astype(np.float32) / box.n
    w = synth.cotangent(box.n, 5)
    ref = oracle.vjp(box.pos, w, box.L, box.cpd, box.R, box.eps, mass=mass.astype(np.float64))
    nf = make_nf(box, dev)
    nf.bin(torch.from_numpy(box.pos).to(dev), torch.from_numpy(mass).to(dev))
    g = nf.vjp(torch.from_numpy(w).to(dev)).cpu().numpy()
    nf.close()
    assert_parity(g, ref, what="vjp masses")
    assert np.abs(g.astype(np.float64).sum(0)).max() <= 1e-5 * np.abs(g).sum()


def test_autograd_matches_vjp(dev):
    from paper_2110_11398_gb300 import accel
    box = synth.tiny(seed=1)
    nf = make_nf(box, dev)
    p = torch.from_numpy(box.pos).to(dev).requires_grad_(True)
    a = accel(p, nf, gm=box.gm)
    w = torch.from_numpy(synth.cotangent(box.n, 2)).to(dev)
    (g,) = torch.autograd.grad(a, p, grad_outputs=w)
    g2 = nf.vjp(w)
    assert torch.equal(g, g2)
    nf.close()


# ---------------------------------------------------------------- full sizes
def _sampled(box, dev, n_sample, seed, precision="fp32", w=None):
    from paper_2110_11398_gb300 import NearField
    nf = NearField(box.L, box.cpd, box.eps, radius=box.R, precision=precision, capacity=box.n, device=dev)
    pos = torch.from_numpy(box.pos).to(dev)
    nf.bin(pos, gm=box.gm)
    if w is None:
        out = nf.accel()
    else:
        out = nf.vjp(torch.from_numpy(w).to(dev))
    st = nf.stats()
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(box.n, n_sample, replace=False))
    got = out[torch.from_numpy(idx).to(dev)].cpu().numpy()
    nf.close()
    del pos, out
    torch.cuda.empty_cache()
    return idx, got, st


def test_early_full_size_sampled(dev):
    box = synth.early()
    idx, got, st = _sampled(box, dev, 20000, 11)
    ref = oracle.accel(box.pos, box.L, box.cpd, box.R, box.eps, m0=box.gm, sinks=idx)
    m, q = assert_parity(got, ref, what="early 256^3")
    P = np.array(st["momentum"])
    assert np.all(np.abs(P) <= 1e-5 * st["abs_momentum"])


def test_late_full_size_sampled(dev):
    box = synth.late()
    idx, got, st = _sampled(box, dev, 2000, 12)
    ref = oracle.accel(box.pos, box.L, box.cpd, box.R, box.eps, m0=box.gm, sinks=idx)
    assert_parity(got, ref, what="late 512^3")
    assert st["max_occupancy"] > 10000


def test_adjoint_full_size_sampled(dev):
    box = synth.adjoint()
    w = synth.cotangent(box.n, box.seed)
    idx, got, _ = _sampled(box, dev, 5000, 13, w=w)
    ref = oracle.vjp(box.pos, w, box.L, box.cpd, box.R, box.eps, m0=box.gm, sinks=idx)
    assert_parity(got, ref, what="adjoint 128^3")


# ---------------------------------------------------------------- more edges
def test_batched_with_an_empty_box(dev):
    from paper_2110_11398_gb300 import NearField
    boxes = synth.batched(n_boxes=3, lo_side=16, hi_side=24, seed0=30)
    boxes[1].pos = boxes[1].pos[:0]                      # box 1 holds no particles
    offs = np.cumsum([0] + [len(b.pos) for b in boxes])
    nfb = NearField([b.L for b in boxes], [b.cpd for b in boxes], [b.eps for b in boxes],
                    capacity=int(offs[-1]), device=dev)
    pos = torch.from_numpy(np.concatenate([b.pos for b in boxes])).to(dev)
    nfb.bin(pos, gm=[b.gm for b in boxes], box_offsets=offs)
    a = nfb.accel().cpu().numpy()
    nfb.close()
    for b, o0, o1 in zip(boxes, offs[:-1], offs[1:]):
        if o1 > o0:
            ref = oracle.accel(b.pos, b.L, b.cpd, b.R, b.eps, m0=b.gm)
            assert_parity(a[o0:o1], ref, what=b.name)


def test_argument_errors(dev):
    from paper_2110_11398_gb300 import NFError, NearField
    box = synth.tiny()
    nf = NearField(box.L, box.cpd, box.eps, capacity=1000, device=dev)
    with pytest.raises(NFError, match="NF_EINVAL"):          # beyond capacity
        nf.bin(torch.from_numpy(box.pos).to(dev), gm=box.gm)
    nf.close()
    nfb = NearField([1.0, 1.0], [9, 9], [1e-3, 1e-3], capacity=box.n, device=dev)
    p = torch.from_numpy(box.pos).to(dev)
    with pytest.raises(NFError, match="NF_EINVAL"):          # offsets must end at n
        nfb.bin(p, gm=box.gm, box_offsets=[0, 100, 200])
    with pytest.raises(NFError, match="NF_EINVAL"):          # and be non-decreasing
        nfb.bin(p, gm=box.gm, box_offsets=[0, box.n + 1, box.n])
    nfb.close()


@pytest.mark.parametrize("R,cpd", [(1, 6), (3, 9)])
def test_vjp_other_radii(dev, R, cpd):
    rng = np.random.default_rng(R)
    n = 6000
    pos = rng.random((n, 3)).astype(np.float32)
    box = synth.Box("r", pos, 1.0, cpd, 0.05 / cpd, 1.0 / n, R)
    w = synth.cotangent(n, R)
    ref = oracle.vjp(pos, w, 1.0, cpd, R, box.eps, m0=box.gm)
    nf = make_nf(box, dev)
    nf.bin(torch.from_numpy(pos).to(dev), gm=box.gm)
    g = nf.vjp(torch.from_numpy(w).to(dev)).cpu().numpy()
    nf.close()
    assert_parity(g, ref, what=f"vjp R={R}")


def test_fp64_vjp_unequal_masses(dev):
    box = synth.tiny(seed=8)
    mass = np.random.default_rng(9).uniform(0.2, 3.0, box.n).astype(np.float32) / box.n
    w = synth.cotangent(box.n, 9)
    ref = oracle.vjp(box.pos, w, box.L, box.cpd, box.R, box.eps, mass=mass.astype(np.float64))
    nf = make_nf(box, dev, "fp64")
    nf.bin(torch.from_numpy(box.pos).to(dev), torch.from_numpy(mass).to(dev))
    g = nf.vjp(torch.from_numpy(w).to(dev)).cpu().numpy()
    nf.close()
    assert np.median(frac_err(g, ref)) < 1e-7


def test_batched_vjp_bit_identical_to_plain(dev):
    """The adjoint over several boxes in one context equals each box's own
    adjoint bit for bit, and the oracle on sampled sinks."""
    from paper_2110_11398_gb300 import NearField
    boxes = synth.batched(n_boxes=3, lo_side=16, hi_side=28, seed0=50)
    offs = np.cumsum([0] + [b.n for b in boxes])
    nfb = NearField([b.L for b in boxes], [b.cpd for b in boxes], [b.eps for b in boxes],
                    capacity=int(offs[-1]), device=dev)
    pos = torch.from_numpy(np.concatenate([b.pos for b in boxes])).to(dev)
    w = torch.from_numpy(synth.cotangent(int(offs[-1]), 50)).to(dev)
    nfb.bin(pos, gm=[b.gm for b in boxes], box_offsets=offs)
    gb = nfb.vjp(w).cpu().numpy()
    nfb.close()
    for b, o0, o1 in zip(boxes, offs[:-1], offs[1:]):
        nf = make_nf(b, dev)
        nf.bin(pos[o0:o1].contiguous(), gm=b.gm)
        gp = nf.vjp(w[o0:o1].contiguous()).cpu().numpy()
        nf.close()
        assert np.array_equal(gb[o0:o1].view(np.uint32), gp.view(np.uint32))
        idx = np.arange(0, b.n, 11)
        ref = oracle.vjp(b.pos, w[o0:o1].cpu().numpy(), b.L, b.cpd, b.R, b.eps, m0=b.gm, sinks=idx)
        assert_parity(gp[idx], ref, what=f"batched vjp {b.name}")


@pytest.mark.parametrize("kv", [0, 1, 2, 4])
def test_vjp_launch_shapes(dev, kv):
    """The adjoint kernel's own sinks per lane (0: as the forward kernel),
    alternating with forward calls of another K in one context."""
    box = synth.tiny(seed=2)
    w = synth.cotangent(box.n, 9)
    ref = oracle.vjp(box.pos, w, box.L, box.cpd, box.R, box.eps, m0=box.gm)
    refa = oracle.accel(box.pos, box.L, box.cpd, box.R, box.eps, m0=box.gm)
    nf = make_nf(box, dev, sinks_per_lane=4, vjp_sinks_per_lane=kv)
    nf.bin(torch.from_numpy(box.pos).to(dev), gm=box.gm)
    wt = torch.from_numpy(w).to(dev)
    for _ in range(2):
        a = nf.accel().cpu().numpy()
        g = nf.vjp(wt).cpu().numpy()
        assert_parity(a, refa, what=f"forward next to vjp K={kv}")
        assert_parity(g, ref, what=f"vjp K={kv}")
    assert nf.tuning["vjp_sinks_per_lane"] == kv
    nf.close()


def test_default_launch_shapes(dev):
    """Defaults: forward K = 4; the adjoint K = 2 (its fastest on the
    clustered adjoint box, 94 ms against 104 ms at K = 4); one sink per lane
    for FP64."""
    box = synth.tiny()
    nf = make_nf(box, dev)
    t = nf.tuning
    assert (t["sinks_per_lane"], t["warps_per_block"], t["vjp_sinks_per_lane"]) == (4, 4, 2)
    nf.close()
    nf = make_nf(box, dev, "fp64")
    t = nf.tuning
    assert (t["sinks_per_lane"], t["vjp_sinks_per_lane"]) == (1, 1)
    nf.close()
