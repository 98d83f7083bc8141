"""Seeded synthetic particle sets shaped like the paper's workloads.

This module is shared by the tests, the oracle's checks and ``bench.py``. It
holds no part of the near-field method itself: no binning, no force law, no
neighbourhood logic. It only draws particle positions (and, for the adjoint,
cotangent weights) from fixed recipes with ``numpy.random.default_rng(seed)``.

The AbacusSummit particle snapshots are not available, so these recipes stand
in for them, keeping the shapes the paper describes:

* about 60 particles per cell (the paper's base boxes use CPD=1701 for 6912^3
  particles, 67 per cell; Sec. 2.5);
* Plummer-equivalent softening at 1/40 of the mean interparticle spacing (the
  paper's 7.2 kpc/h proper for a 2 Gpc/h, 6912^3 box; Sec. 2.5);
* early times: particles close to a lattice (the initial grid; Sec. 2.4);
* late times: strongly clustered, with most of the pair work inside halos
  (the paper's late-epoch timing is dominated by the near field; Sec. 4.3).

All positions are float32 in the half-open box [0, L) with L = 1, and G*m is
folded into a single equal mass 1/N.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Box",
    "uniform_box",
    "perturbed_lattice",
    "clustered_box",
    "tiny",
    "early",
    "late",
    "batched",
    "adjoint",
    "cotangent",
    "make",
]


@dataclass
class Box:
    """One periodic box: positions plus the parameters of the near-field sum."""

    name: str
    pos: np.ndarray            # (N, 3) float32 in [0, L)
    L: float                   # box side
    cpd: int                   # cells per dimension
    eps: float                 # Plummer softening length (same units as L)
    gm: float                  # G * m per particle (equal masses)
    R: int = 2                 # near-field radius in cells
    seed: int = 0
    info: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _to_box_f32(x: np.ndarray, L: float = 1.0) -> np.ndarray:
    """Wrap float64 coordinates into [0, L) and round to float32.

    A value that rounds up to L in float32 lies within one float32 ulp of the
    face, i.e. at the same place as 0 in the periodic box; it is wrapped to 0.
    """
    x = np.mod(x, L)
    x32 = x.astype(np.float32)
    x32[x32 >= np.float32(L)] = np.float32(0.0)
    return x32


def uniform_box(n: int, seed: int, L: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return _to_box_f32(rng.random((n, 3)) * L, L)


def _lattice_sites(n_side: int) -> np.ndarray:
    """Cell-centred lattice (i + 0.5) / n_side, x slowest, as float64 (n_side^3, 3)."""
    g = (np.arange(n_side, dtype=np.float64) + 0.5) / n_side
    gx, gy, gz = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)


def perturbed_lattice(n_side: int, sigma_spacing: float, seed: int,
                      keep: int | None = None, rng=None) -> np.ndarray:
    """Lattice of n_side^3 sites displaced by iid N(0, sigma) per axis.

    ``keep`` selects that many sites uniformly at random (without replacement)
    before the displacement; the selected sites stay in lattice order.
    Returns float64 positions (unwrapped).
    """
    rng = np.random.default_rng(seed) if rng is None else rng
    n_sites = n_side ** 3
    if keep is None or keep >= n_sites:
        idx = None
        m = n_sites
    else:
        idx = np.sort(rng.permutation(n_sites)[:keep])
        m = keep
    sites = _lattice_sites(n_side)
    if idx is not None:
        sites = sites[idx]
    sites += rng.normal(0.0, sigma_spacing / n_side, size=(m, 3))
    return sites


def _power_law_counts(n_halos: int, slope: float, lo: float, hi: float, rng) -> np.ndarray:
    """Draw halo particle counts from dN/dM ~ M^-slope on [lo, hi] by inverse CDF."""
    u = rng.random(n_halos)
    a = 1.0 - slope
    return (lo ** a + u * (hi ** a - lo ** a)) ** (1.0 / a)


def _rescale_counts(raw: np.ndarray, total: int) -> np.ndarray:
    """Largest-remainder rounding of ``raw`` rescaled to sum exactly to ``total``."""
    t = raw * (total / raw.sum())
    base = np.floor(t).astype(np.int64)
    short = int(total - base.sum())
    if short > 0:
        frac = t - base
        order = np.argsort(-frac, kind="stable")[:short]
        base[order] += 1
    return base


def _nfw_radii(counts_total: int, conc: float, rng, ngrid: int = 8192) -> np.ndarray:
    """Radii in units of r200 for an NFW profile truncated at r200.

    The enclosed-mass fraction is mu(x)/mu(c) with mu(x) = ln(1+x) - x/(1+x),
    x = r / r_s, r_s = r200 / c; it is inverted by interpolation on a table.
    """
    x = np.concatenate([[0.0], np.geomspace(1e-6, conc, ngrid)])
    mu = np.log1p(x) - x / (1.0 + x)
    cdf = mu / mu[-1]
    u = rng.random(counts_total)
    return np.interp(u, cdf, x) / conc


def _isotropic(n: int, rng) -> np.ndarray:
    v = rng.normal(size=(n, 3))
    nrm = np.sqrt((v * v).sum(axis=1, keepdims=True))
    nrm[nrm == 0] = 1.0
    return v / nrm


def clustered_box(n_total: int, seed: int, *, lattice_frac: float = 0.6,
                  sigma_spacing: float = 0.5, n_halos: int = 20000,
                  conc: float = 5.0, slope: float = 1.9, mlo: float = 100.0,
                  mhi: float = 2e6, overdensity: float = 200.0):
    """Late-time clustered recipe.

    * ``lattice_frac`` of the particles sit on randomly chosen sites of the
      lattice of side round(cbrt(N)), displaced by N(0, sigma_spacing) spacings;
    * the rest are in ``n_halos`` NFW halos (concentration ``conc``) with
      particle counts drawn from dN/dM ~ M^-slope on [mlo, mhi], rescaled by
      largest remainder to sum exactly to the halo share of N; halo centres
      are uniform in the box; each halo is truncated at r200, the radius
      inside which its mean density is ``overdensity`` times the box mean.

    Returns (float32 positions, info dict).
    """
    rng = np.random.default_rng(seed)
    n_halo_p = int(round((1.0 - lattice_frac) * n_total))
    n_lat = n_total - n_halo_p
    n_side = int(round(n_total ** (1.0 / 3.0)))
    while n_side ** 3 < n_lat:
        n_side += 1
    lat = perturbed_lattice(n_side, sigma_spacing, seed, keep=n_lat, rng=rng)

    counts = _rescale_counts(_power_law_counts(n_halos, slope, mlo, mhi, rng), n_halo_p)
    centres = rng.random((n_halos, 3))
    r200 = (3.0 * counts / (4.0 * math.pi * overdensity * n_total)) ** (1.0 / 3.0)
    owner = np.repeat(np.arange(n_halos), counts)
    rad = _nfw_radii(n_halo_p, conc, rng) * r200[owner]
    halo = centres[owner] + _isotropic(n_halo_p, rng) * rad[:, None]

    pos = _to_box_f32(np.concatenate([lat, halo], axis=0))
    info = {
        "n_lattice": n_lat,
        "n_halo_particles": n_halo_p,
        "n_halos": n_halos,
        "max_halo": int(counts.max()) if n_halos else 0,
        "lattice_side": n_side,
    }
    return pos, info


def _eps(n: int, L: float = 1.0) -> float:
    """Plummer softening at 1/40 of the mean interparticle spacing."""
    return (L / n ** (1.0 / 3.0)) / 40.0


def tiny(seed: int = 0) -> Box:
    """32^3 uniform particles, CPD=9 (about 45 per cell)."""
    n = 32 ** 3
    return Box("tiny_32c_cpd9", uniform_box(n, seed), 1.0, 9, _eps(n), 1.0 / n, 2, seed)


def early(seed: int = 1, n_side: int = 256, cpd: int = 65) -> Box:
    """Early-time box: 256^3 lattice displaced by N(0, 0.3 spacing), CPD=65."""
    n = n_side ** 3
    pos = _to_box_f32(perturbed_lattice(n_side, 0.3, seed))
    return Box(f"early_{n_side}c_cpd{cpd}", pos, 1.0, cpd, _eps(n), 1.0 / n, 2, seed)


def late(seed: int = 2, n_side: int = 512, cpd: int = 129, n_halos: int = 20000) -> Box:
    """Late-time clustered box: 512^3 particles, CPD=129, 20000 NFW halos."""
    n = n_side ** 3
    pos, info = clustered_box(n, seed, n_halos=n_halos)
    return Box(f"late_{n_side}c_cpd{cpd}", pos, 1.0, cpd, _eps(n), 1.0 / n, 2, seed, info)


def _scaled_halos(n: int) -> int:
    """Halo count scaled with N from the 20000 halos of the 512^3 box."""
    return max(1, int(round(20000 * n / 512 ** 3)))


def batched(n_boxes: int = 64, seed0: int = 3, lo_side: int = 64, hi_side: int = 192,
            workers: int | None = None) -> list[Box]:
    """Independent clustered boxes with N log-uniform in [lo_side^3, hi_side^3].

    Box b uses seed ``seed0 + b``; CPD_b = round(cbrt(N_b / 60)). Boxes are
    drawn on ``workers`` threads (default: the host's cores, at most 16);
    each box has its own generator, so the result does not depend on it.
    """
    def one(b):
        rng = np.random.default_rng(seed0 + b)
        n = int(round(math.exp(rng.uniform(math.log(lo_side ** 3), math.log(hi_side ** 3)))))
        cpd = max(5, int(round((n / 60.0) ** (1.0 / 3.0))))
        pos, info = clustered_box(n, seed0 + b + 1000, n_halos=_scaled_halos(n))
        return Box(f"batched_box{b}", pos, 1.0, cpd, _eps(n), 1.0 / n, 2, seed0 + b, info)

    if workers is None:
        workers = min(16, os.cpu_count() or 1)
    if workers <= 1 or n_boxes <= 1:
        return [one(b) for b in range(n_boxes)]
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(workers) as ex:
        return list(ex.map(one, range(n_boxes)))


def adjoint(seed: int = 4, n_side: int = 128, cpd: int = 33) -> Box:
    """Clustered 128^3 box for the vector-Jacobian product, CPD=33."""
    n = n_side ** 3
    pos, info = clustered_box(n, seed, n_halos=_scaled_halos(n))
    return Box(f"adjoint_{n_side}c_cpd{cpd}", pos, 1.0, cpd, _eps(n), 1.0 / n, 2, seed, info)


def cotangent(n: int, seed: int) -> np.ndarray:
    """iid N(0, 1) float32 weights w_i (the cotangent of the accelerations)."""
    return np.random.default_rng(seed + 7919).standard_normal((n, 3)).astype(np.float32)


def make(name: str, **kw):
    """Build a named workload: tiny, early, late, batched or adjoint."""
    fn = {"tiny": tiny, "early": early, "late": late, "batched": batched, "adjoint": adjoint}[name]
    return fn(**kw)
