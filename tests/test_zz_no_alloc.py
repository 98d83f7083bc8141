"""The no-allocation binning entry point, checked against the allocating one.

nf_bin_cells_noalloc serves callers that cannot allocate device memory, such
as a program whose own pool allocator already holds the GPU's memory (another
cudaMalloc would fail or fragment it) or a loop that cannot pay cudaMalloc's
device-wide synchronisation. It keeps its scratch in one static device array
shared by all calls, so these checks run it several times in a row with
different sizes: each call must give exactly the cell table, permutation and
cell-relative records of nf_bin_particles + nf_copy_binning (binning is exact
work, so the comparison is bit for bit, as in the other binning tests).
The limits are run at their edge (2^20 particles, CPD 64), together with an
empty input, an out-of-range position, and a check that repeated calls leave
the device's free memory unchanged.
This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2110_11398_gb300 import _native, build
    build.build()
    return _native.load(), torch.device("cuda", 0)


def _noalloc(lib, dev, pos, L, cpd, gm, mass=None):
    n = pos.shape[0]
    cs = torch.full((cpd ** 3 + 1,), -7, dtype=torch.int32, device=dev)
    perm = torch.full((n,), -7, dtype=torch.int32, device=dev)
    srt = torch.full((n, 4), float("nan"), dtype=torch.float32, device=dev)
    rc = lib.nf_bin_cells_noalloc(pos.data_ptr(), None if mass is None else mass.data_ptr(),
                                  float(gm), n, float(L), cpd, cs.data_ptr(), perm.data_ptr(),
                                  srt.data_ptr(), torch.cuda.current_stream(dev).cuda_stream)
    assert rc == 0, lib.nf_last_error(None)
    return cs.cpu().numpy(), perm.cpu().numpy(), srt.cpu().numpy()


def _allocating(dev, pos, L, cpd, gm, mass=None):
    from paper_2110_11398_gb300 import NearField
    nf = NearField(L, cpd, 0.01 * L / cpd, capacity=pos.shape[0], device=dev)
    nf.bin(pos, mass, gm=None if mass is not None else gm)
    out = tuple(t.cpu().numpy() for t in nf.binning())
    nf.close()
    return out


def _cases(dev):
    big, _ = synth.clustered_box(64 ** 3, 21, n_halos=40)            # 262,144 particles
    rng = np.random.default_rng(5)
    L = 3.7
    small = (rng.random((5000, 3)) * L).astype(np.float32)
    small[small >= np.float32(L)] = 0
    mass = rng.uniform(0.5, 2.0, 5000).astype(np.float32)
    return [
        (torch.from_numpy(big).to(dev), 1.0, 33, 1.0 / 64 ** 3, None),
        (torch.from_numpy(small).to(dev), L, 9, 0.0, torch.from_numpy(mass).to(dev)),
        (torch.from_numpy(big[:100000].copy()).to(dev), 1.0, 64, 1e-5, None),
    ]


def test_noalloc_matches_allocating_binning_on_consecutive_calls(env):
    lib, dev = env
    for pos, L, cpd, gm, mass in _cases(dev):
        got = _noalloc(lib, dev, pos, L, cpd, gm, mass)
        ref = _allocating(dev, pos, L, cpd, gm, mass)
        assert np.array_equal(got[0], ref[0])
        assert np.array_equal(got[1], ref[1])
        assert np.array_equal(got[2].view(np.uint32), ref[2].view(np.uint32))


def test_noalloc_twice_in_a_row_is_identical(env):
    lib, dev = env
    pos, L, cpd, gm, mass = _cases(dev)[0]
    a = _noalloc(lib, dev, pos, L, cpd, gm, mass)
    b = _noalloc(lib, dev, pos, L, cpd, gm, mass)
    for x, y in zip(a, b):
        assert np.array_equal(x.view(np.uint32) if x.dtype == np.float32 else x,
                              y.view(np.uint32) if y.dtype == np.float32 else y)


def test_noalloc_rejects_sizes_beyond_its_limit(env):
    lib, dev = env
    pos = torch.zeros((16, 3), dtype=torch.float32, device=dev)
    buf = torch.zeros(16 * 4, dtype=torch.float32, device=dev)
    cs = torch.zeros(8, dtype=torch.int32, device=dev)
    rc = lib.nf_bin_cells_noalloc(pos.data_ptr(), None, 1.0, (1 << 20) + 1, 1.0, 9, cs.data_ptr(),
                                  cs.data_ptr(), buf.data_ptr(), None)
    assert rc == -1 and b"1048576" in lib.nf_last_error(None)
    rc = lib.nf_bin_cells_noalloc(pos.data_ptr(), None, 1.0, 16, 1.0, 65, cs.data_ptr(),
                                  cs.data_ptr(), buf.data_ptr(), None)
    assert rc == -1 and b"cpd" in lib.nf_last_error(None)


def test_noalloc_at_its_particle_limit(env):
    """n = 2^20 particles at CPD = 64 (the largest sizes the static array is
    cut for), bit for bit against the allocating binning."""
    lib, dev = env
    rng = np.random.default_rng(12)
    n = 1 << 20
    halo = (np.array([0.3, 0.6, 0.2]) + 0.01 * rng.standard_normal((n // 4, 3))) % 1.0
    pos = np.concatenate([rng.random((n - n // 4, 3)), halo]).astype(np.float32)
    pos[pos >= np.float32(1.0)] = 0
    p = torch.from_numpy(pos).to(dev)
    got = _noalloc(lib, dev, p, 1.0, 64, 1.0 / n)
    ref = _allocating(dev, p, 1.0, 64, 1.0 / n)
    assert np.array_equal(got[0], ref[0])
    assert np.array_equal(got[1], ref[1])
    assert np.array_equal(got[2].view(np.uint32), ref[2].view(np.uint32))


def test_noalloc_empty_input(env):
    lib, dev = env
    cpd = 7
    cs = torch.full((cpd ** 3 + 1,), -7, dtype=torch.int32, device=dev)
    rc = lib.nf_bin_cells_noalloc(None, None, 1.0, 0, 1.0, cpd, cs.data_ptr(), None, None,
                                  torch.cuda.current_stream(dev).cuda_stream)
    assert rc == 0, lib.nf_last_error(None)
    assert np.all(cs.cpu().numpy() == 0)


@pytest.mark.parametrize("bad", [1.0, float("nan"), -1e-3])
def test_noalloc_out_of_range_position(env, bad):
    lib, dev = env
    pos = np.random.default_rng(3).random((4000, 3)).astype(np.float32)
    pos[123, 1] = bad
    p = torch.from_numpy(pos).to(dev)
    cs = torch.empty(9 ** 3 + 1, dtype=torch.int32, device=dev)
    perm = torch.empty(4000, dtype=torch.int32, device=dev)
    srt = torch.empty((4000, 4), dtype=torch.float32, device=dev)
    rc = lib.nf_bin_cells_noalloc(p.data_ptr(), None, 1.0, 4000, 1.0, 9, cs.data_ptr(), perm.data_ptr(),
                                  srt.data_ptr(), torch.cuda.current_stream(dev).cuda_stream)
    assert rc == -2 and b"outside" in lib.nf_last_error(None)
    # the shared array is usable again at once
    ok = _noalloc(lib, dev, torch.from_numpy(np.random.default_rng(4).random((4000, 3)).astype(np.float32)).to(dev),
                  1.0, 9, 1.0)
    assert ok[0][-1] == 4000


def test_noalloc_calls_leave_free_device_memory_unchanged(env):
    """After a first call (which loads the kernels it launches), further calls
    must not change the device's free memory (cudaMemGetInfo)."""
    lib, dev = env
    pos, L, cpd, gm, mass = _cases(dev)[0]
    n = pos.shape[0]
    cs = torch.empty(cpd ** 3 + 1, dtype=torch.int32, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    srt = torch.empty((n, 4), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream

    def call():
        rc = lib.nf_bin_cells_noalloc(pos.data_ptr(), None, float(gm), n, float(L), cpd, cs.data_ptr(),
                                      perm.data_ptr(), srt.data_ptr(), stream)
        assert rc == 0, lib.nf_last_error(None)

    call()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    call()
    free1, _ = torch.cuda.mem_get_info(dev)
    call()
    free2, _ = torch.cuda.mem_get_info(dev)
    assert free0 == free1 == free2, (free0, free1, free2)
