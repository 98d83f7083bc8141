"""The FP64 momentum diagnostic of nf_compute_accel against a host FP64 sum.

Newton's third law makes the near-field force of a pair antisymmetric, so
P = sum_i m_i a_i vanishes up to rounding (Maksimova et al. 2021, Sec. 3.1:
every pair within the near-field radius is summed from both ends). The
library reduces P, and the scale S = sum_i m_i |a_i|, on the GPU in FP64
(k_momentum / k_momentum_eq, a two-level fixed-order reduction). These tests
recompute both on the host from the accelerations the library returned and
the masses it binned, and require agreement to 1e-12 of S:

  - both sides sum the same FP64 terms m_i a_i (a product of two floats is
    exact in FP64), in different orders, so they differ by summation
    rounding only: about sqrt(N) 1e-16 S; with one mass for the whole box
    the GPU sums a_i and multiplies by G m once, which differs from the
    per-term products by rounding of the same size;
  - |a_i| is formed the same way on both sides: for float32 accelerations
    the float32 sum (x^2 + y^2) + z^2 of the float32 squares, each step
    rounded, for float64 ones the FP64 sum of squares rounded once to
    float32; then a correctly rounded float32 square root.

A reduction that dropped one of its 512 block partials would move S by
about 1/512 of itself and P by the sum of about N/512 terms that do not
cancel; one that skipped the mass factor would change S by a factor 1/m.
Either breaks the 1e-12 bound by many orders of magnitude.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

REL = 1e-12


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2110_11398_gb300 import build
    build.build()
    return torch.device("cuda", 0)


def host_momentum(acc, mass):
    """(P, S) from the returned accelerations (N,3) and the binned masses (N,)."""
    a = np.asarray(acc, np.float64)
    m = np.asarray(mass, np.float32).astype(np.float64)
    P = np.sum(m[:, None] * a, axis=0)
    if acc.dtype == np.float32:
        x, y, z = acc[:, 0], acc[:, 1], acc[:, 2]
        a2 = (x * x + y * y) + z * z                 # float32 operations
    else:
        a2 = np.sum(a * a, axis=1).astype(np.float32)
    assert a2.dtype == np.float32
    S = float(np.sum(m * np.sqrt(a2).astype(np.float64)))
    return P, S


def check(st, acc, mass):
    P, S = host_momentum(acc, mass)
    Pg, Sg = np.array(st["momentum"]), st["abs_momentum"]
    assert S > 0
    assert abs(Sg - S) <= REL * S, (Sg, S)
    assert np.all(np.abs(Pg - P) <= REL * S), (Pg, P, S)
    # and the diagnostic itself: Newton's third law up to FP32 pair rounding
    assert np.all(np.abs(Pg) <= 1e-5 * Sg), (Pg, Sg)


def run_one(box, dev, mass=None, f64=False, precision="fp32"):
    from paper_2110_11398_gb300 import NearField
    nf = NearField(box.L, box.cpd, box.eps, radius=box.R, precision=precision,
                   capacity=max(box.n, 1), device=dev)
    pos = torch.from_numpy(box.pos).to(dev)
    if mass is None:
        nf.bin(pos, gm=box.gm)
        m = np.full(box.n, np.float32(box.gm), np.float32)
    else:
        nf.bin(pos, torch.from_numpy(mass).to(dev))
        m = mass
    acc = nf.accel(dtype=torch.float64 if f64 else torch.float32)
    st = nf.stats()
    out = acc.cpu().numpy()
    nf.close()
    return st, out, m


def test_momentum_equal_masses(dev):
    st, acc, m = run_one(synth.tiny(), dev)
    check(st, acc, m)


def test_momentum_unequal_masses(dev):
    box = synth.tiny(seed=5)
    mass = np.random.default_rng(3).uniform(0.2, 3.0, box.n).astype(np.float32) / box.n
    st, acc, m = run_one(box, dev, mass=mass)
    check(st, acc, m)


@pytest.mark.parametrize("precision", ["fp32_comp", "fp64"])
def test_momentum_other_precisions(dev, precision):
    box = synth.tiny(seed=7)
    st, acc, m = run_one(box, dev, f64=precision == "fp64", precision=precision)
    check(st, acc, m)


def test_momentum_batched_per_box_masses(dev):
    from paper_2110_11398_gb300 import NearField
    boxes = synth.batched(n_boxes=5, lo_side=18, hi_side=36, seed0=11)
    offs = np.cumsum([0] + [b.n for b in boxes])
    nf = NearField([b.L for b in boxes], [b.cpd for b in boxes], [b.eps for b in boxes],
                   capacity=int(offs[-1]), device=dev)
    pos = torch.from_numpy(np.concatenate([b.pos for b in boxes])).to(dev)
    nf.bin(pos, gm=[b.gm for b in boxes], box_offsets=offs)
    acc = nf.accel().cpu().numpy()
    st = nf.stats()
    nf.close()
    m = np.concatenate([np.full(b.n, np.float32(b.gm), np.float32) for b in boxes])
    check(st, acc, m)


def test_momentum_early_full_size(dev):
    box = synth.early()
    st, acc, m = run_one(box, dev)
    check(st, acc, m)
    torch.cuda.empty_cache()
