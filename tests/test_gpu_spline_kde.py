"""GPU parity for the spline pair law and the in-pass kernel density estimate.

Spline law: exactly Newtonian for r >= eps_s (Maksimova et al. 2021, Sec. 2.5
and Sec. 5.2), r (10 - 15u + 6u^2)/eps_s^3 inside (the reading pinned in
tests/test_oracle_spline_kde.py). Density: sum_j G m_j (1 - r^2/b^2)_+ over
the near field, b = 0.4 of the mean spacing (Sec. 3.3). Tolerances as for the
forces: median fractional error <= 1e-6, 99.9th percentile <= 1e-4.
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


def frac(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    if got.ndim == 1:
        return np.abs(got - ref) / np.abs(ref)
    return np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)


def check(got, ref, what):
    e = frac(got, ref)
    m, q = np.median(e), np.quantile(e, 0.999)
    assert m <= 1e-6 and q <= 1e-4, f"{what}: median {m:.3e} p99.9 {q:.3e}"


def run(box, dev, law, kde_b=None, mass=None, eps=None, **tune):
    from paper_2110_11398_gb300 import NearField
    nf = NearField(box.L, box.cpd, eps or box.eps, radius=box.R, capacity=box.n, device=dev,
                   softening=law)
    if tune:
        nf.set_tuning(**tune)
    m = None if mass is None else torch.from_numpy(mass.astype(np.float32)).to(dev)
    nf.bin(torch.from_numpy(box.pos).to(dev), m, gm=None if m is not None else box.gm)
    if kde_b is None:
        a, d = nf.accel(), None
    else:
        a, d = nf.accel_density(kde_b)
    torch.cuda.synchronize()
    out = (a.cpu().numpy(), None if d is None else d.cpu().numpy())
    nf.close()
    return out


def spacing(box):
    return box.L / box.n ** (1 / 3)


@pytest.mark.parametrize("K", [1, 2, 4])
def test_spline_forward(dev, K):
    box = synth.tiny()
    eps_s = 2.5 * box.eps
    ref = oracle.accel_ex(box.pos, box.L, box.cpd, box.R, eps_s, law="spline", m0=box.gm)
    got, _ = run(box, dev, "spline", eps=eps_s, sinks_per_lane=K)
    check(got, ref, f"spline K={K}")


@pytest.mark.parametrize("law", ["plummer", "spline"])
@pytest.mark.parametrize("K", [2, 4])
def test_density_with_forces(dev, law, K):
    box = synth.tiny(seed=4)
    eps = 2.5 * box.eps if law == "spline" else box.eps
    b = 0.4 * spacing(box)
    ref_a, ref_d = oracle.accel_ex(box.pos, box.L, box.cpd, box.R, eps, law=law, kde_b=b, m0=box.gm)
    got_a, got_d = run(box, dev, law, kde_b=b, eps=eps, sinks_per_lane=K)
    check(got_a, ref_a, f"{law} acc with density")
    check(got_d, ref_d, f"{law} density")
    assert np.all(got_d >= np.float32(box.gm) * (1 - 1e-6))      # the self term


def test_density_unequal_masses_clustered(dev):
    pos, _ = synth.clustered_box(40 ** 3, 8, n_halos=20)
    box = synth.Box("cl40", pos, 1.0, 11, (1 / 40) / 40, 1 / 40 ** 3)
    mass = np.random.default_rng(2).uniform(0.3, 3.0, box.n) / box.n
    b = 0.4 * spacing(box)
    ref_a, ref_d = oracle.accel_ex(box.pos, box.L, box.cpd, box.R, 2.5 * box.eps, law="spline",
                                   kde_b=b, mass=mass.astype(np.float32).astype(np.float64))
    got_a, got_d = run(box, dev, "spline", kde_b=b, mass=mass, eps=2.5 * box.eps)
    check(got_a, ref_a, "spline acc, masses")
    check(got_d, ref_d, "density, masses")


def test_density_early_full_size_sampled(dev):
    box = synth.early()
    b = 0.4 * spacing(box)
    got_a, got_d = run(box, dev, "plummer", kde_b=b)
    idx = np.sort(np.random.default_rng(3).choice(box.n, 5000, replace=False))
    ref_a, ref_d = oracle.accel_ex(box.pos, box.L, box.cpd, box.R, box.eps, kde_b=b, m0=box.gm,
                                   sinks=idx)
    check(got_a[idx], ref_a, "early acc")
    check(got_d[idx], ref_d, "early density")


def test_spline_and_density_argument_checks(dev):
    from paper_2110_11398_gb300 import NearField, NFError
    box = synth.tiny()
    with pytest.raises(NFError, match="NF_EINVAL"):
        NearField(box.L, box.cpd, box.eps, capacity=box.n, device=dev, softening="spline",
                  precision="fp32_comp")
    nf = NearField(box.L, box.cpd, box.eps, capacity=box.n, device=dev, softening="spline")
    nf.bin(torch.from_numpy(box.pos).to(dev), gm=box.gm)
    assert not torch.any(nf.vjp(torch.zeros((box.n, 3), device=dev)))   # zero cotangent
    with pytest.raises(NFError, match="NF_EINVAL"):          # b beyond the near field
        nf.accel_density(2.5 * box.L / box.cpd)
    with pytest.raises(NFError, match="NF_EINVAL"):
        nf.accel_density(0.0)
    nf.close()


# ---------------------------------------------------------------- spline adjoint
def run_vjp(box, dev, eps_s, w, mass=None, **tune):
    from paper_2110_11398_gb300 import NearField
    nf = NearField(box.L, box.cpd, eps_s, radius=box.R, capacity=box.n, device=dev,
                   softening="spline")
    if tune:
        nf.set_tuning(**tune)
    m = None if mass is None else torch.from_numpy(mass.astype(np.float32)).to(dev)
    nf.bin(torch.from_numpy(box.pos).to(dev), m, gm=None if m is not None else box.gm)
    g = nf.vjp(torch.from_numpy(w).to(dev)).cpu().numpy()
    nf.close()
    return g


@pytest.mark.parametrize("K", [1, 2, 4])
@pytest.mark.parametrize("radius", ["production", "wide"])
def test_spline_vjp(dev, K, radius):
    """Adjoint of the spline law against the oracle's, with eps_s = 2.5 eps
    (few pairs inside) and eps_s = 0.8 spacing (many pairs on the polynomial
    branch)."""
    box = synth.tiny()
    eps_s = 2.5 * box.eps if radius == "production" else 0.8 * spacing(box)
    w = synth.cotangent(box.n, 11)
    ref = oracle.vjp(box.pos, w, box.L, box.cpd, box.R, eps_s, m0=box.gm, law="spline")
    got = run_vjp(box, dev, eps_s, w, vjp_sinks_per_lane=K)
    check(got, ref, f"spline vjp K={K} {radius}")
    assert np.abs(got.astype(np.float64).sum(0)).max() <= 1e-5 * np.abs(got).sum()


def test_spline_vjp_unequal_masses_clustered(dev):
    pos, _ = synth.clustered_box(40 ** 3, 6, n_halos=15)
    box = synth.Box("cl40", pos, 1.0, 11, (1 / 40) / 40, 1 / 40 ** 3)
    mass = np.random.default_rng(2).uniform(0.2, 3.0, box.n) / box.n
    eps_s = 0.5 * spacing(box)
    w = synth.cotangent(box.n, 12)
    ref = oracle.vjp(box.pos, w, box.L, box.cpd, box.R, eps_s,
                     mass=mass.astype(np.float32).astype(np.float64), law="spline")
    check(run_vjp(box, dev, eps_s, w, mass=mass), ref, "spline vjp masses")


def test_spline_autograd(dev):
    """torch.autograd through the spline accelerations calls the spline adjoint."""
    from paper_2110_11398_gb300 import NearField, accel
    box = synth.tiny(seed=4)
    eps_s = 0.6 * spacing(box)
    nf = NearField(box.L, box.cpd, eps_s, radius=box.R, capacity=box.n, device=dev,
                   softening="spline")
    pos = torch.from_numpy(box.pos).to(dev).requires_grad_(True)
    w = synth.cotangent(box.n, 13)
    loss = (accel(pos, nf, gm=box.gm) * torch.from_numpy(w).to(dev)).sum()
    loss.backward()
    ref = oracle.vjp(box.pos, w, box.L, box.cpd, box.R, eps_s, m0=box.gm, law="spline")
    check(pos.grad.cpu().numpy(), ref, "spline autograd")
    nf.close()
