"""Pins for the FP64 oracle against facts that do not depend on it.

Each check below is chosen so that a plausible slip in the oracle (a dropped
softening term, a wrong sign, a wrong periodic image, a transposed index, a
wrong neighbourhood, an unstable sort) fails at least one of them:

* binning: exact rational containment of each point in its cell, sortedness,
  stability, and counts equal to an independent histogram;
* the cell-neighbourhood sum against a brute-force all-pairs x 27-images sum
  with the inclusion rule written per pair (a different loop structure);
* the two-body closed form inside and outside the softening length, across a
  periodic face, with unequal masses;
* the open-boundary reduction: a cluster inside a 3x3x3 block of cells away
  from the faces equals the textbook open direct sum;
* Newton's third law (net momentum change zero) and lattice symmetry zeros;
* invariance under whole-cell shifts of every particle;
* the adjoint against central finite differences of the oracle's own forward
  sum, and sum_k g_k = 0.

Paper: Maksimova et al. 2021, Sec. 3.1 (cells, near/far split, near-field
direct sum) and Sec. 5.2 (Plummer softening potential).
"""
from fractions import Fraction

import numpy as np
import pytest

import synth


# ---------------------------------------------------------------- helpers
def brute_accel(pos, L, cpd, R, eps, mass):
    """All pairs x all 27 images; a pair (i, j, image n) is near iff the cell
    offset c_j + n*CPD - c_i lies in [-R, R] on every axis (Sec. 3.1)."""
    pos = np.asarray(pos, np.float64)
    n = len(pos)
    c = np.floor(pos * cpd / L).astype(np.int64)
    c = np.minimum(c, cpd - 1)
    acc = np.zeros((n, 3))
    imgs = np.array([(a, b, d) for a in (-1, 0, 1) for b in (-1, 0, 1) for d in (-1, 0, 1)])
    for i in range(n):
        for im in imgs:
            off = c + im * cpd - c[i]
            ok = np.all(np.abs(off) <= R, axis=1)
            if not ok.any():
                continue
            D = pos[ok] + im * L - pos[i]
            s = (D * D).sum(1) + eps * eps
            acc[i] += ((mass[ok] / s ** 1.5)[:, None] * D).sum(0)
    return acc, c


def brute_count(pos, L, cpd, R):
    c = np.minimum(np.floor(np.asarray(pos, np.float64) * cpd / L).astype(np.int64), cpd - 1)
    tot = 0
    for i in range(len(pos)):
        for a in (-1, 0, 1):
            for b in (-1, 0, 1):
                for d in (-1, 0, 1):
                    off = c + np.array([a, b, d]) * cpd - c[i]
                    tot += int(np.all(np.abs(off) <= R, axis=1).sum())
    return tot


def open_direct(pos, eps, mass):
    """Textbook open-boundary direct sum."""
    D = pos[None, :, :] - pos[:, None, :]
    s = (D * D).sum(-1) + eps * eps
    return ((mass[None, :] / s ** 1.5)[:, :, None] * D).sum(1)


# ---------------------------------------------------------------- binning
def _adversarial_positions(rng, cpd, L, n):
    """Random points plus points on and next to every cell face."""
    x = rng.random((n, 3)).astype(np.float32) * np.float32(L)
    faces = np.array([k * L / cpd for k in range(cpd)], np.float32)
    extra = []
    for f in faces:
        for v in (f, np.nextafter(f, np.float32(0)), np.nextafter(f, np.float32(2 * L))):
            if 0 <= v < L:
                extra.append(v)
    extra.append(np.nextafter(np.float32(L), np.float32(0)))
    extra = np.array(extra, np.float32)
    m = len(extra)
    block = np.stack([extra, extra[::-1], np.roll(extra, 3)], axis=1)
    out = np.concatenate([x, block], axis=0)
    rng.shuffle(out)
    return out


@pytest.mark.parametrize("cpd,L", [(9, 1.0), (5, 1.0), (7, 3.7), (33, 1.0), (16, 250.0)])
def test_binning_exact_containment_and_stability(oracle_mod, cpd, L):
    rng = np.random.default_rng(11 + cpd)
    pos = _adversarial_positions(rng, cpd, L, 3000)
    # duplicate some points so stability matters
    pos = np.concatenate([pos, pos[:200]], axis=0)
    b = oracle_mod.bin_particles(pos, L, cpd)
    cid, cs, perm, rel = b["cid"], b["cell_start"], b["perm"], b["rel"]
    n = len(pos)
    c3 = np.stack([cid // (cpd * cpd), (cid // cpd) % cpd, cid % cpd], axis=1)
    Lq = Fraction(L)
    for i in range(0, n, 7):
        for a in range(3):
            u = Fraction(float(pos[i, a])) * cpd / Lq          # exact x*CPD/L
            k = int(c3[i, a])
            if k <= u < k + 1:
                continue
            # only a point within one double rounding of a face may land on
            # the other side of it (the binning rounds x*CPD/L to double)
            face = k if u < k else k + 1
            assert abs(u - face) <= Fraction(cpd, 2 ** 50), (i, a, float(u), k)
    # counts and prefix sum against an independent histogram
    counts = np.bincount(cid, minlength=cpd ** 3)
    assert cs[0] == 0 and cs[-1] == n
    assert np.array_equal(np.diff(cs), counts)
    # perm is a permutation; sorted cells non-decreasing; stable within cells
    assert np.array_equal(np.sort(perm), np.arange(n))
    sc = cid[perm]
    assert np.all(np.diff(sc) >= 0)
    same = sc[1:] == sc[:-1]
    assert np.all(perm[1:][same] > perm[:-1][same])
    # cell-relative coordinates: within one float32 rounding of the exact value
    for k in range(0, n, 13):
        i = perm[k]
        for a in range(3):
            exact = Fraction(float(pos[i, a])) * cpd / Lq - c3[i, a] - Fraction(1, 2)
            assert abs(Fraction(float(rel[k, a])) - exact) <= Fraction(1, 2 ** 25) + Fraction(1, 2 ** 48)
            assert -0.5 <= rel[k, a] <= 0.5


@pytest.mark.parametrize("bad", [np.nan, np.inf, -1e-7, 1.0, 1.5, -np.inf])
def test_binning_rejects_out_of_range(oracle_mod, bad):
    pos = np.random.default_rng(0).random((50, 3)).astype(np.float32)
    pos[17, 1] = bad
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.bin_particles(pos, 1.0, 9)


# ---------------------------------------------------------------- forward sum
@pytest.mark.parametrize("cpd,R,n,masses", [(5, 2, 400, False), (7, 2, 600, True),
                                             (9, 2, 700, False), (3, 1, 300, True),
                                             (6, 1, 500, False), (11, 3, 600, True)])
def test_accel_matches_brute_force_images(oracle_mod, cpd, R, n, masses):
    rng = np.random.default_rng(cpd * 100 + R)
    L = 1.0
    pos = rng.random((n, 3)).astype(np.float32)
    mass = rng.uniform(0.5, 2.0, n) if masses else np.full(n, 1.0 / n)
    eps = 0.3 / cpd
    ref, c = brute_accel(pos, L, cpd, R, eps, mass)
    b = oracle_mod.bin_particles(pos, L, cpd)
    c_lin = (c[:, 0] * cpd + c[:, 1]) * cpd + c[:, 2]
    assert np.array_equal(c_lin, b["cid"])
    got = oracle_mod.accel(pos, L, cpd, R, eps, mass=mass if masses else None, m0=1.0 / n)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-13 * scale)
    # the interaction count of the same inclusion rule
    assert oracle_mod.interactions(b["cid"], cpd, R) == brute_count(pos, L, cpd, R)


@pytest.mark.parametrize("r_over_eps", [0.05, 0.5, 1.0, 2.0, 10.0, 60.0])
def test_two_body_closed_form_across_face(oracle_mod, r_over_eps):
    """|a| = G m r / (r^2 + eps^2)^(3/2) along the separation, for the pair's
    nearest image across the periodic x face (CPD = 2R+1 = 5, so each pair
    is near exactly once)."""
    L, cpd, R = 1.0, 5, 2
    eps = 0.004
    r = r_over_eps * eps
    u = np.array([0.8, -0.36, 0.48])        # unit vector
    a_pos = np.array([0.001, 0.52, 0.43])
    b_pos = a_pos - r * u                    # crosses x = 0
    b_pos = np.mod(b_pos, L)
    pos = np.stack([a_pos, b_pos])
    m1, m2 = 0.7, 1.9
    got = oracle_mod.accel(pos, L, cpd, R, eps, mass=np.array([m1, m2]),
                           cid=_cells(pos, L, cpd))
    D = -r * u                               # b - a through the image
    mag = r / (r * r + eps * eps) ** 1.5
    np.testing.assert_allclose(got[0], m2 * mag * D / r, rtol=1e-12, atol=0)
    np.testing.assert_allclose(got[1], -m1 * mag * D / r, rtol=1e-12, atol=0)


def _cells(pos, L, cpd):
    c = np.minimum(np.floor(np.asarray(pos, np.float64) * cpd / L).astype(np.int64), cpd - 1)
    return ((c[:, 0] * cpd + c[:, 1]) * cpd + c[:, 2]).astype(np.int32)


def test_golden_two_body_values(oracle_mod):
    """Hand-derived values stored in tests/golden/two_body.txt."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "two_body.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for row in rows:
        L, cpd, R, eps, m1, m2 = map(float, row[:6])
        p = np.array(list(map(float, row[6:12]))).reshape(2, 3)
        exp = np.array(list(map(float, row[12:18]))).reshape(2, 3)
        got = oracle_mod.accel(p, L, int(cpd), int(R), eps, mass=np.array([m1, m2]),
                               cid=_cells(p, L, int(cpd)))
        np.testing.assert_allclose(got, exp, rtol=1e-12, atol=1e-300)


def test_open_boundary_reduction(oracle_mod):
    """All particles inside cells 3..5 of a CPD=9 box: every pair is near with
    no wrap, so the sum is the textbook open direct sum."""
    rng = np.random.default_rng(5)
    cpd, L, R = 9, 1.0, 2
    n = 900
    pos = (3.0 + 3.0 * rng.random((n, 3))) / cpd
    mass = rng.uniform(0.1, 3.0, n)
    eps = 0.01
    got = oracle_mod.accel(pos, L, cpd, R, eps, mass=mass, cid=_cells(pos, L, cpd))
    ref = open_direct(pos, eps, mass)
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())


def test_newton_third_law(oracle_mod):
    box = synth.tiny()
    rng = np.random.default_rng(2)
    for mass in (None, rng.uniform(0.2, 5.0, box.n) / box.n):
        a = oracle_mod.accel(box.pos, box.L, box.cpd, box.R, box.eps, mass=mass, m0=box.gm)
        m = np.full(box.n, box.gm) if mass is None else mass
        P = (m[:, None] * a).sum(0)
        scale = np.abs(m[:, None] * a).sum()
        assert np.all(np.abs(P) <= 1e-13 * scale), (P, scale)


def test_lattice_symmetry_zero(oracle_mod):
    """One particle per cell at the same cell-relative offset: each sink sees
    the symmetric set {d h} of sources, so its near-field force is zero."""
    cpd, L, R = 7, 1.0, 2
    h = L / cpd
    g = np.arange(cpd)
    cx, cy, cz = np.meshgrid(g, g, g, indexing="ij")
    off = np.array([0.13, 0.71, 0.42])
    pos = (np.stack([cx.ravel(), cy.ravel(), cz.ravel()], 1) + off) * h
    eps = 0.02 * h
    a = oracle_mod.accel(pos, L, cpd, R, eps, m0=1.0, cid=_cells(pos, L, cpd))
    pair = 1.0 / h ** 2
    assert np.abs(a).max() <= 1e-12 * pair


def test_whole_cell_shift_invariance(oracle_mod):
    """Shifting every particle by whole cells (wrapped) permutes cells but not
    the force on any particle. L = CPD so that shifts are exact."""
    rng = np.random.default_rng(9)
    cpd = 9
    L = float(cpd)
    n = 3000
    pos = np.floor(rng.random((n, 3)) * cpd * 2 ** 16) / 2 ** 16
    eps = 0.02
    a0 = oracle_mod.accel(pos.astype(np.float32), L, cpd, 2, eps, m0=1.0)
    for k in ([1, 0, 0], [3, 5, 8], [8, 8, 8], [0, 4, 0]):
        sp = np.mod(pos + np.array(k, float), L)
        a1 = oracle_mod.accel(sp.astype(np.float32), L, cpd, 2, eps, m0=1.0)
        np.testing.assert_allclose(a1, a0, rtol=1e-11, atol=1e-12 * np.abs(a0).max())


def test_softening_matters_inside_eps(oracle_mod):
    """Inside the softening length the force falls below the bare 1/r^2 law by
    the closed-form factor (r^2/(r^2+eps^2))^(3/2); far outside it agrees."""
    L, cpd, R, eps = 1.0, 5, 2, 0.01
    for r, expect_ratio in ((0.001, (0.001 ** 2 / (0.001 ** 2 + eps ** 2)) ** 1.5),
                            (0.09, (0.09 ** 2 / (0.09 ** 2 + eps ** 2)) ** 1.5)):
        pos = np.array([[0.5, 0.5, 0.5], [0.5 + r, 0.5, 0.5]])
        a = oracle_mod.accel(pos, L, cpd, R, eps, m0=1.0, cid=_cells(pos, L, cpd))
        assert a[0, 0] > 0 and a[1, 0] < 0
        np.testing.assert_allclose(a[0, 0] * r * r, expect_ratio, rtol=1e-12)


# ---------------------------------------------------------------- adjoint
def test_vjp_central_differences(oracle_mod):
    rng = np.random.default_rng(17)
    cpd, L, R = 6, 1.0, 2
    n = 250
    pos = rng.random((n, 3))
    mass = rng.uniform(0.5, 2.0, n)
    spacing = L / n ** (1 / 3)
    eps = spacing / 10
    cid = _cells(pos, L, cpd)
    w = rng.standard_normal((n, 3))
    g = oracle_mod.vjp(pos, w, L, cpd, R, eps, mass=mass, cid=cid)

    def lw(p):
        return float((w * oracle_mod.accel(p, L, cpd, R, eps, mass=mass, cid=cid)).sum())

    h = 1e-4 * spacing
    gscale = np.abs(g).max()
    for k in rng.choice(n, 25, replace=False):
        for a in range(3):
            pp = pos.copy(); pp[k, a] += h
            pm = pos.copy(); pm[k, a] -= h
            fd = (lw(pp) - lw(pm)) / (2 * h)
            assert abs(fd - g[k, a]) <= 2e-5 * gscale + 1e-6 * abs(g[k, a]), (k, a, fd, g[k, a])
    # translating every particle leaves sum_i w_i . a_i unchanged
    assert np.abs(g.sum(0)).max() <= 1e-12 * np.abs(g).sum()


def test_vjp_two_body_finite_difference(oracle_mod):
    """Two bodies across a face, inside and outside eps, equal and unequal masses."""
    L, cpd, R = 1.0, 5, 2
    eps = 0.01
    rng = np.random.default_rng(3)
    for r in (0.003, 0.01, 0.05):
        u = rng.standard_normal(3); u /= np.linalg.norm(u)
        a = np.array([0.002, 0.5, 0.5])
        b = np.mod(a - r * u, L)
        pos = np.stack([a, b])
        mass = np.array([1.3, 0.4])
        w = rng.standard_normal((2, 3))
        cid = _cells(pos, L, cpd)
        g = oracle_mod.vjp(pos, w, L, cpd, R, eps, mass=mass, cid=cid)
        hh = 1e-7
        for k in range(2):
            for ax in range(3):
                pp = pos.copy(); pp[k, ax] += hh
                pm = pos.copy(); pm[k, ax] -= hh
                fp = (w * oracle_mod.accel(pp, L, cpd, R, eps, mass=mass, cid=cid)).sum()
                fm = (w * oracle_mod.accel(pm, L, cpd, R, eps, mass=mass, cid=cid)).sum()
                fd = (fp - fm) / (2 * hh)
                assert abs(fd - g[k, ax]) <= 1e-5 * np.abs(g).max(), (r, k, ax, fd, g[k, ax])


def test_sink_subset_matches_full(oracle_mod):
    box = synth.tiny()
    full = oracle_mod.accel(box.pos, box.L, box.cpd, box.R, box.eps, m0=box.gm)
    sub = np.array([0, 5, 77, box.n - 1, 1234])
    part = oracle_mod.accel(box.pos, box.L, box.cpd, box.R, box.eps, m0=box.gm, sinks=sub)
    assert np.array_equal(part, full[sub])


def test_golden_file_is_what_its_script_writes():
    import os
    import subprocess
    import sys
    here = os.path.join(os.path.dirname(__file__), "golden")
    out = subprocess.run([sys.executable, os.path.join(here, "make_two_body.py")],
                         capture_output=True, text=True, check=True).stdout
    assert out == open(os.path.join(here, "two_body.txt")).read()
