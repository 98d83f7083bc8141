"""Pins for the oracle's spline force law and kernel density estimate.

Spline law: the near-field force returns to exactly 1/r^2 beyond a finite
radius (Maksimova et al. 2021, Sec. 2.5 and Sec. 5.2). The reading used here
is the lowest-order law F = r P(r/eps) that meets 1/r^2 at r = eps with
continuous first and second derivatives. The checks below fix it from the
outside: 1/r^2 beyond eps, continuity of F, F' and F'' at eps measured from
one-sided differences of the oracle's own two-body forces, the slope of F at
r -> 0, and the central potential obtained by integrating the force.

Density estimate: weight 1 - r^2/b^2 inside b (Sec. 3.3), summed over the
same cells as the near-field force, self included.
"""
import numpy as np
import pytest

import synth


def _cells(pos, L, cpd):
    c = np.minimum(np.floor(np.asarray(pos, np.float64) * cpd / L).astype(np.int64), cpd - 1)
    return ((c[:, 0] * cpd + c[:, 1]) * cpd + c[:, 2]).astype(np.int32)


def _F(oracle_mod, r, eps, L=1.0, cpd=5):
    """Pair force magnitude on body 1 from body 2 (unit mass) at distance r."""
    p = np.array([[0.5, 0.5, 0.5], [0.5 + r, 0.5, 0.5]])
    a = oracle_mod.accel_ex(p, L, cpd, 2, eps, law="spline", m0=1.0, cid=_cells(p, L, cpd))
    return a[0, 0]


def test_spline_is_newtonian_beyond_eps(oracle_mod):
    eps = 0.02
    for r in (eps, 1.0001 * eps, 1.5 * eps, 3 * eps, 0.15):
        np.testing.assert_allclose(_F(oracle_mod, r, eps), 1.0 / r ** 2, rtol=1e-12)


def test_spline_smooth_at_eps(oracle_mod):
    eps = 0.02
    h = 1e-3 * eps
    # values and one-sided derivatives from inside and from outside
    fin = [_F(oracle_mod, eps - k * h, eps) for k in (0, 1, 2, 3)]
    fout = [_F(oracle_mod, eps + k * h, eps) for k in (0, 1, 2, 3)]
    d1_in = (3 * fin[0] - 4 * fin[1] + fin[2]) / (2 * h)
    d1_out = (-3 * fout[0] + 4 * fout[1] - fout[2]) / (2 * h)
    d2_in = (2 * fin[0] - 5 * fin[1] + 4 * fin[2] - fin[3]) / h ** 2
    d2_out = (2 * fout[0] - 5 * fout[1] + 4 * fout[2] - fout[3]) / h ** 2
    F0 = 1 / eps ** 2
    assert abs(fin[0] - F0) <= 1e-12 * F0
    assert abs(d1_in - d1_out) <= 1e-4 * abs(d1_out)
    assert abs(d2_in - d2_out) <= 2e-2 * abs(d2_out)
    # and those derivatives are the Newtonian ones
    np.testing.assert_allclose(d1_out, -2 / eps ** 3, rtol=1e-4)


def test_spline_linear_core_and_central_potential(oracle_mod):
    eps = 0.02
    r = 1e-7 * eps
    np.testing.assert_allclose(_F(oracle_mod, r, eps) / r, 10.0 / eps ** 3, rtol=1e-5)
    # phi(0) = -int_0^inf F dr; inside eps by Gauss-Legendre on the oracle's
    # force, outside 1/eps exactly
    xs, ws = np.polynomial.legendre.leggauss(12)
    rr = 0.5 * eps * (xs + 1)
    inner = 0.5 * eps * sum(w * _F(oracle_mod, r_, eps) for r_, w in zip(rr, ws))
    np.testing.assert_allclose(inner + 1 / eps, 2.5 / eps, rtol=1e-12)


def _brute_spline_kde(pos, L, cpd, R, eps, b, mass):
    pos = np.asarray(pos, np.float64)
    n = len(pos)
    c = np.minimum(np.floor(pos * cpd / L).astype(np.int64), cpd - 1)
    acc = np.zeros((n, 3))
    rho = np.zeros(n)
    for i in range(n):
        for im in [(a, bb, d) for a in (-1, 0, 1) for bb in (-1, 0, 1) for d in (-1, 0, 1)]:
            im = np.array(im)
            ok = np.all(np.abs(c + im * cpd - c[i]) <= R, axis=1)
            D = pos[ok] + im * L - pos[i]
            r = np.sqrt((D * D).sum(1))
            u = r / eps
            with np.errstate(divide="ignore", invalid="ignore"):
                f = np.where(r >= eps, 1 / np.maximum(r, 1e-300) ** 3,
                             (10 - 15 * u + 6 * u * u) / eps ** 3)
            acc[i] += ((mass[ok] * f)[:, None] * D).sum(0)
            rho[i] += (mass[ok] * np.clip(1 - r * r / b ** 2, 0, None)).sum()
    return acc, rho


@pytest.mark.parametrize("cpd,R", [(5, 2), (7, 2), (6, 1)])
def test_spline_and_density_match_brute_force(oracle_mod, cpd, R):
    rng = np.random.default_rng(40 + cpd)
    n = 500
    pos = rng.random((n, 3))
    mass = rng.uniform(0.5, 2.0, n)
    eps, b = 0.4 / cpd, 0.6 / cpd
    ref_a, ref_r = _brute_spline_kde(pos, 1.0, cpd, R, eps, b, mass)
    a, rho = oracle_mod.accel_ex(pos, 1.0, cpd, R, eps, law="spline", kde_b=b, mass=mass,
                                 cid=_cells(pos, 1.0, cpd))
    np.testing.assert_allclose(a, ref_a, rtol=1e-10, atol=1e-12 * np.abs(ref_a).max())
    np.testing.assert_allclose(rho, ref_r, rtol=1e-12)


def test_spline_newton_third_law(oracle_mod):
    box = synth.tiny()
    a = oracle_mod.accel_ex(box.pos, box.L, box.cpd, box.R, 2.5 * box.eps, law="spline", m0=box.gm)
    P = (box.gm * a).sum(0)
    assert np.all(np.abs(P) <= 1e-13 * np.abs(box.gm * a).sum())


def test_density_isolated_and_two_body(oracle_mod):
    L, cpd, b = 1.0, 5, 0.05
    for r in (0.01, 0.049, 0.051, 0.3):
        p = np.array([[0.001, 0.5, 0.5], [np.mod(0.001 - r, 1.0), 0.5, 0.5]])   # across x = 0
        m = np.array([1.5, 0.25])
        _, rho = oracle_mod.accel_ex(p, L, cpd, 2, 0.01, kde_b=b, mass=m, cid=_cells(p, L, cpd))
        w = max(0.0, 1 - r * r / b ** 2)
        np.testing.assert_allclose(rho, [1.5 + 0.25 * w, 0.25 + 1.5 * w], rtol=1e-12)


def test_density_on_a_lattice(oracle_mod):
    """One particle per cell of a cubic lattice of spacing a: with b = 1.2 a
    only the 6 face neighbours (at a) fall inside b (the next shell is at
    1.414 a), so every density is m (1 + 6 (1 - 1/1.44))."""
    cpd = 8
    a = 1.0 / cpd
    g = (np.arange(cpd) + 0.37) * a
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    _, rho = oracle_mod.accel_ex(pos, 1.0, cpd, 2, 0.1 * a, kde_b=1.2 * a, m0=2.0,
                                 cid=_cells(pos, 1.0, cpd))
    np.testing.assert_allclose(rho, 2.0 * (1 + 6 * (1 - 1 / 1.44)), rtol=1e-12)


# ---------------------------------------------------------------- spline adjoint
def test_spline_vjp_central_differences(oracle_mod):
    """The spline adjoint against central differences of the forward spline
    sum (binning frozen), with eps chosen so that both branches of the law
    are common; translation leaves sum_i w_i . a_i unchanged, so the
    gradient sums to zero."""
    rng = np.random.default_rng(23)
    cpd, L, R = 6, 1.0, 2
    n = 250
    pos = rng.random((n, 3))
    mass = rng.uniform(0.5, 2.0, n)
    spacing = L / n ** (1 / 3)
    eps = 0.8 * spacing
    cid = _cells(pos, L, cpd)
    w = rng.standard_normal((n, 3))
    g = oracle_mod.vjp(pos, w, L, cpd, R, eps, mass=mass, cid=cid, law="spline")

    def lw(p):
        return float((w * oracle_mod.accel_ex(p, L, cpd, R, eps, law="spline", mass=mass,
                                              cid=cid)).sum())

    h = 1e-5 * spacing
    gscale = np.abs(g).max()
    for k in rng.choice(n, 25, replace=False):
        for a in range(3):
            pp = pos.copy(); pp[k, a] += h
            pm = pos.copy(); pm[k, a] -= h
            fd = (lw(pp) - lw(pm)) / (2 * h)
            assert abs(fd - g[k, a]) <= 2e-5 * gscale + 1e-6 * abs(g[k, a]), (k, a, fd, g[k, a])
    assert np.abs(g.sum(0)).max() <= 1e-12 * np.abs(g).sum()


def test_spline_vjp_two_body_symbolic(oracle_mod):
    """Two bodies, inside and outside the spline radius and across a periodic
    face: the adjoint equals the Jacobian of the pair force obtained by
    symbolic differentiation of F(r) = r (10 - 15u + 6u^2)/eps^3 (u < 1) and
    1/r^2 (u >= 1), the law the forward pins fix."""
    sp = pytest.importorskip("sympy")
    L, cpd, R, eps = 1.0, 5, 2, 0.02
    x, y, z, e = sp.symbols("x y z e", positive=True)
    r = sp.sqrt(x * x + y * y + z * z)
    u = r / e
    inside = sp.Matrix([x, y, z]) * (10 - 15 * u + 6 * u * u) / e ** 3
    outside = sp.Matrix([x, y, z]) / r ** 3
    J_in = sp.lambdify((x, y, z, e), inside.jacobian([x, y, z]), "numpy")
    J_out = sp.lambdify((x, y, z, e), outside.jacobian([x, y, z]), "numpy")
    rng = np.random.default_rng(8)
    for dist in (0.004, 0.013, 0.0199, 0.0201, 0.05):
        d = rng.standard_normal(3); d *= dist / np.linalg.norm(d)
        a = np.array([0.001, 0.5, 0.5])
        b = np.mod(a + d, L)
        pos = np.stack([a, b])
        m = np.array([1.3, 0.4])
        w = rng.standard_normal((2, 3))
        g = oracle_mod.vjp(pos, w, L, cpd, R, eps, mass=m, cid=_cells(pos, L, cpd), law="spline")
        J = np.array((J_in if dist < eps else J_out)(*d, eps), dtype=np.float64)   # J(D_01) = J(D_10)
        g0 = J @ (m[0] * w[1] - m[1] * w[0])
        np.testing.assert_allclose(g[0], g0, rtol=1e-9, atol=1e-12 * np.abs(g0).max())
        np.testing.assert_allclose(g[1], -g0, rtol=1e-9, atol=1e-12 * np.abs(g0).max())


def test_spline_vjp_coincident_bodies(oracle_mod):
    """At r = 0 the pair Jacobian is f(0) I = (10/eps^3) I: the D D^T term
    vanishes with D."""
    L, cpd, R, eps = 1.0, 5, 2, 0.02
    pos = np.array([[0.3, 0.3, 0.3], [0.3, 0.3, 0.3]])
    m = np.array([2.0, 0.5])
    w = np.array([[1.0, -2.0, 0.5], [0.25, 3.0, -1.0]])
    g = oracle_mod.vjp(pos, w, L, cpd, R, eps, mass=m, cid=_cells(pos, L, cpd), law="spline")
    g0 = 10.0 / eps ** 3 * (m[0] * w[1] - m[1] * w[0])
    np.testing.assert_allclose(g[0], g0, rtol=1e-13)
    np.testing.assert_allclose(g[1], -g0, rtol=1e-13)


def test_plummer_vjp_unchanged_by_the_law_switch(oracle_mod):
    box = synth.tiny()
    w = synth.cotangent(box.n, 3)
    idx = np.arange(0, box.n, 97)
    a = oracle_mod.vjp(box.pos, w, box.L, box.cpd, box.R, box.eps, m0=box.gm, sinks=idx)
    b = oracle_mod.vjp(box.pos, w, box.L, box.cpd, box.R, box.eps, m0=box.gm, sinks=idx, law="plummer")
    assert np.array_equal(a, b)
