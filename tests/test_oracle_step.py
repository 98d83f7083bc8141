"""Pins for the oracle's particle update: the timestep criterion and the
kick-drift-kick leapfrog step (Maksimova et al. 2021, Sec. 2.5).

The criterion is checked on hand-built cells. The step is checked by
properties a leapfrog must have: time reversibility, bounded energy error
on a circular two-body orbit, and second-order convergence.
"""
import math

import numpy as np

import oracle


def _cells(pos, L, cpd):
    c = np.minimum(np.floor(np.asarray(pos, np.float64) * cpd / L).astype(np.int64), cpd - 1)
    return ((c[:, 0] * cpd + c[:, 1]) * cpd + c[:, 2]).astype(np.int32)


def test_timestep_on_hand_built_cells():
    cpd, L = 5, 1.0
    h = L / cpd
    pos = np.array([
        [0.5, 0.5, 0.5], [0.55, 0.5, 0.5],            # cell A: two bodies
        [0.1, 0.1, 0.1], [0.12, 0.1, 0.1], [0.14, 0.1, 0.1],   # cell B: three bodies
        [0.9, 0.9, 0.9],                               # a lone body: no bound
        [0.5, 0.1, 0.9], [0.52, 0.1, 0.9],             # zero accelerations: no bound
    ])
    vel = np.array([[1, 0, 0], [-1, 0, 0],
                    [0, 2, 0], [0, -2, 0], [0, 0, 0],
                    [0, 0, 0],
                    [5, 0, 0], [-5, 0, 0]], float)
    acc = np.array([[0, 4, 0], [0, 1, 0],
                    [1, 0, 0], [0, 0.5, 0], [0, 0, 0.25],
                    [0, 1e-9, 0],
                    [0, 0, 0], [0, 0, 0]], float)
    cid = _cells(pos, L, cpd)
    assert len(set(cid[:2])) == 1 and len(set(cid[2:5])) == 1
    # A: sigma = 1 (deviations of length 1), max|a| = 4 -> 0.25
    # B: deviations (0,2,0), (0,-2,0), (0,0,0): sigma^2 = 8/3, max|a| = 1
    expect = 0.25 * min(1 / 4, math.sqrt(8 / 3) / 1)
    assert oracle.cell_timestep(vel, acc, cid, cpd, 0.25) == expect


def _two_body(d, eps, m):
    """Circular orbit of two equal masses at separation d (Plummer law)."""
    com = np.array([0.5, 0.5, 0.5])
    x = np.stack([com - [d / 2, 0, 0], com + [d / 2, 0, 0]])
    g = m * d / (d * d + eps * eps) ** 1.5           # pull on each body
    v = math.sqrt(g * d / 2)
    vel = np.array([[0, -v, 0], [0, v, 0]])
    period = 2 * math.pi * (d / 2) / v
    return x.astype(np.float32), vel.astype(np.float32), period


def _energy(x, v, eps, m, L):
    D = (x[1].astype(np.float64) - x[0]) - L * np.round((x[1].astype(np.float64) - x[0]) / L)
    return 0.5 * m * (v.astype(np.float64) ** 2).sum() - m * m / math.sqrt((D * D).sum() + eps * eps)


def test_kdk_reversible():
    L, cpd, R, eps, m = 1.0, 5, 2, 0.01, 1e-3
    rng = np.random.default_rng(1)
    x = rng.random((60, 3)).astype(np.float32)
    v = (rng.standard_normal((60, 3)) * 0.01).astype(np.float32)
    dt = 0.05
    x1, v1, a1 = oracle.kdk_step(x, v, dt, L, cpd, R, eps, m0=m)
    x0, v0, _ = oracle.kdk_step(x1, v1, -dt, L, cpd, R, eps, m0=m, acc0=a1)
    np.testing.assert_allclose(v0, v, rtol=0, atol=1e-6 * np.abs(v).max())
    D = (x0.astype(np.float64) - x) - L * np.round((x0.astype(np.float64) - x) / L)
    assert np.abs(D).max() < 1e-6


def test_kdk_energy_on_a_circular_orbit():
    L, cpd, R, eps, m = 1.0, 5, 2, 0.002, 1e-3
    x, v, T = _two_body(0.1, eps, m)
    e0 = _energy(x, v, eps, m, L)
    dt = T / 200
    a = None
    errs = []
    for step in range(400):
        x, v, a = oracle.kdk_step(x, v, dt, L, cpd, R, eps, m0=m, acc0=a)
        errs.append(abs(_energy(x, v, eps, m, L) / e0 - 1))
    assert max(errs) < 2e-3
    # no secular drift: the error over the second orbit is like the first
    assert max(errs[200:]) < 2 * max(errs[:200]) + 1e-6


def test_kdk_second_order():
    L, cpd, R, eps, m = 1.0, 5, 2, 0.002, 1e-3
    x0, v0, T = _two_body(0.1, eps, m)

    def orbit(nsteps):
        x, v, a = x0, v0, None
        for _ in range(nsteps):
            x, v, a = oracle.kdk_step(x, v, T / nsteps, L, cpd, R, eps, m0=m, acc0=a)
        D = (x.astype(np.float64) - x0) - L * np.round((x.astype(np.float64) - x0) / L)
        return np.abs(D).max()

    e1, e2 = orbit(100), orbit(200)
    assert 3.0 < e1 / e2 < 5.0, (e1, e2)


def test_kdk_with_the_far_field_kicks_with_the_total_force():
    """With the far field on, the step's force is near + far, which for
    (almost) unsoftened particles is the Ewald force of the periodic box: the
    acceleration the step returns at its new positions matches the Ewald sum
    there to the far field's truncation error, and the velocity follows the
    leapfrog with those forces. Without the far field it misses the other
    images by far more."""
    L, cpd, R, eps = 1.0, 7, 2, 1e-7
    rng = np.random.default_rng(3)
    n = 80
    m = 1.0 / n
    x = rng.random((n, 3)).astype(np.float32)
    v = (rng.standard_normal((n, 3)) * 0.01).astype(np.float32)
    dt = 1e-3
    x1, v1, a1 = oracle.kdk_step(x, v, dt, L, cpd, R, eps, m0=m, far_order=8)
    a0e = oracle.ewald_accel(x.astype(np.float64), L, m0=m)
    a1e = oracle.ewald_accel(x1.astype(np.float64), L, m0=m)
    e = np.linalg.norm(a1 - a1e, axis=1) / np.linalg.norm(a1e, axis=1)
    assert np.median(e) < 1e-5, np.median(e)
    v_half = (v.astype(np.float64) + 0.5 * dt * a0e).astype(np.float32)
    v_e = v_half.astype(np.float64) + 0.5 * dt * a1e
    scale = dt * np.abs(a1e).max()
    assert np.abs(v1 - v_e).max() < 1e-5 * scale + 1e-6 * np.abs(v).max()
    _, _, a1n = oracle.kdk_step(x, v, dt, L, cpd, R, eps, m0=m)
    en = np.linalg.norm(a1n - a1e, axis=1) / np.linalg.norm(a1e, axis=1)
    assert np.median(en) > 100 * np.median(e), (np.median(en), np.median(e))
