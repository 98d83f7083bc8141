"""Pins for the far-field oracle (oracle/farfield.c): the derivatives tensor,
the Ewald total force and the multipole / Taylor far field of Sec. 3.1.

The far field is an approximation (Taylor series of order p), so it is pinned
against an exact definition: the Ewald sum of the periodic 1/r^2 force, which
equals near field + far field with no approximation. The pieces are pinned
on their own: the tensor against a textbook lattice constant, against the
plain image sum where that converges absolutely, against finite differences
of itself and against a change of the Ewald splitting parameter; the Ewald
force against a change of that parameter and against lattice symmetry.
"""
import numpy as np
import pytest

import oracle

# Regularised lattice sum of 1/|n| over the simple cubic lattice with a
# uniform neutralising background, sum_{n != 0} 1/|n| -> -2.8372974794806
# (the Ewald "self" constant of a point in a cubic periodic box, xi/L; e.g.
# Nijboer and de Wette 1957; Hummer, Pratt and Garcia 1995).
XI_SC = -2.8372974794806


def _per_order(Q):
    return oracle.far_multi_indices(Q).sum(1)


@pytest.mark.parametrize("P", [1, 5, 7])
def test_tensor_origin_value_is_the_cubic_lattice_constant(P):
    for alpha in (2.5 / P, 3.5 / P):
        D = oracle.far_dtensor([0, 0, 0], P, 0, alpha, 2)
        assert abs(D[0] * P - XI_SC) < 1e-12
        # second derivatives at the origin: isotropic by cubic symmetry, with
        # trace 4 pi / V from the uniform background (lap psi = -4 pi delta + 4 pi / V)
        mi = oracle.far_multi_indices(2)
        for i in range(4, 10):
            diag = tuple(mi[i]) in ((2, 0, 0), (0, 2, 0), (0, 0, 2))
            expect = 4 * np.pi / (3 * P ** 3) if diag else 0.0
            assert abs(D[i] - expect) < 1e-12, (tuple(mi[i]), D[i], expect)


@pytest.mark.parametrize("d", [(0, 0, 0), (1, 2, 2), (2, 0, 0), (3, 1, 0), (3, 3, 3), (-2, 3, 1)])
def test_tensor_does_not_depend_on_the_splitting(d):
    P, R, Q = 7, 2, 16
    deg = _per_order(Q)
    a = oracle.far_dtensor(d, P, R, 2.5 / P, Q)
    b = oracle.far_dtensor(d, P, R, 3.5 / P, Q)
    noise = 1e-15 * np.abs(a).max()   # for orders that vanish by symmetry
    for t in range(Q + 1):
        sel = deg == t
        tol = max(2e-9 * np.abs(a[sel]).max(), noise)
        assert np.abs(a[sel] - b[sel]).max() <= tol, (d, t)


def test_tensor_has_the_parity_of_its_order():
    """1/r is even, and both the image sum and the near block it leaves out
    are symmetric, so D_q(-d) = (-1)^|q| D_q(d), and D is periodic in d with
    period CPD. Its discrete transform over the grid is therefore i^|q| times a
    real function (what the GPU keeps of it)."""
    P, R, Q = 5, 2, 10
    deg = _per_order(Q)
    for d in ((1, 2, 0), (2, 2, 1), (0, 0, 3), (4, 1, 3)):
        a = oracle.far_dtensor(d, P, R, 3.5 / P, Q)
        b = oracle.far_dtensor([-x for x in d], P, R, 3.5 / P, Q)
        c = oracle.far_dtensor([(-x) % P for x in d], P, R, 3.5 / P, Q)
        scale = np.abs(a).max()
        assert np.abs(b - (-1.0) ** deg * a).max() <= 1e-12 * scale, d
        assert np.abs(c - b).max() <= 1e-12 * scale, d
    Q = 4
    deg = _per_order(Q)
    D = np.zeros((len(deg), P, P, P))
    for x in range(P):
        for y in range(P):
            for z in range(P):
                D[:, x, y, z] = oracle.far_dtensor([x, y, z], P, R, 3.5 / P, Q)
    E = (1j ** -deg)[:, None, None, None] * np.fft.rfftn(D, axes=(1, 2, 3))
    assert np.abs(E.imag).max() <= 1e-13 * np.abs(E.real).max()


def test_tensor_is_its_own_derivative():
    """d^(q + e_x) D = d/dx d^q D, by central differences at a non-lattice point."""
    P, Q, h = 7, 10, 1e-5
    d0 = np.array([2.3, -1.1, 0.7])
    mi = oracle.far_multi_indices(Q)
    lut = {tuple(x): i for i, x in enumerate(mi)}
    base = oracle.far_dtensor(d0, P, -1, 3.5 / P, Q)
    deg = mi.sum(1)
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        dp = oracle.far_dtensor(d0 + e, P, -1, 3.5 / P, Q)
        dm = oracle.far_dtensor(d0 - e, P, -1, 3.5 / P, Q)
        for i, q in enumerate(mi):
            if q.sum() >= Q:
                continue
            q2 = q.copy()
            q2[ax] += 1
            exact = base[lut[tuple(q2)]]
            scale = np.abs(base[deg == q2.sum()]).max()
            assert abs((dp[i] - dm[i]) / (2 * h) - exact) <= 1e-6 * scale, (ax, tuple(q))


def test_high_orders_equal_the_plain_image_sum():
    """For |q| >= 6 the lattice sum of d^q (1/r) converges absolutely, and the
    Ewald value must equal it: derivatives from sympy, summed over a cube of
    images directly (no splitting), near image left out. The cube's tail
    falls as M^-(|q|-2)."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z", real=True)
    f = 1 / sp.sqrt(x * x + y * y + z * z)
    P, R, M = 5, 2, 24
    qs = [(6, 0, 0), (2, 2, 2), (3, 1, 3), (0, 7, 0), (4, 3, 1), (2, 0, 6), (1, 1, 6)]
    mi = oracle.far_multi_indices(8)
    lut = {tuple(v): i for i, v in enumerate(mi)}
    n = np.arange(-M, M + 1)
    NX, NY, NZ = np.meshgrid(n, n, n, indexing="ij")
    for d in ((2, 1, 0), (0, 0, 0), (1, 2, 2)):
        D = oracle.far_dtensor(d, P, R, 3.5 / P, 8)
        X, Y, Z = d[0] + P * NX, d[1] + P * NY, d[2] + P * NZ
        near = (np.abs(X) <= R) & (np.abs(Y) <= R) & (np.abs(Z) <= R)
        X, Y, Z = X[~near].astype(float), Y[~near].astype(float), Z[~near].astype(float)
        for q in qs:
            fn = sp.lambdify((x, y, z), sp.diff(f, x, q[0], y, q[1], z, q[2]), "numpy")
            direct = float(np.sum(fn(X, Y, Z)))
            assert abs(direct - D[lut[q]]) <= 1e-7 * max(abs(D[lut[q]]), 1e-3), (d, q, direct, D[lut[q]])


def _box(seed, n=300):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)).astype(np.float32).astype(np.float64)
    mass = rng.uniform(0.5, 1.5, n) / n
    return pos, mass


def test_ewald_does_not_depend_on_the_splitting():
    pos, mass = _box(3, 150)
    a = oracle.ewald_accel(pos, 1.0, mass=mass, alpha=3.0)
    b = oracle.ewald_accel(pos, 1.0, mass=mass, alpha=4.5)
    assert np.abs(a - b).max() <= 1e-11 * np.abs(a).max()


def test_ewald_lattice_and_pair_symmetry():
    g = (np.arange(4) + 0.25) / 4
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    lat = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    assert np.abs(oracle.ewald_accel(lat, 1.0, m0=1.0)).max() < 1e-12
    # two bodies: equal and opposite, and along the separation for a pair on an axis
    pair = np.array([[0.3, 0.5, 0.5], [0.45, 0.5, 0.5]])
    a = oracle.ewald_accel(pair, 1.0, m0=1.0)
    assert np.allclose(a[0], -a[1], rtol=0, atol=1e-13)
    assert a[0, 0] > 0 and abs(a[0, 1]) < 1e-13 and abs(a[0, 2]) < 1e-13
    # at small separation it is Newton plus the background's (4 pi / 3) r pull
    r = 0.15
    assert abs(a[0, 0] - (1 / r ** 2 - 4 * np.pi / 3 * r)) < 2e-3 * (1 / r ** 2)


def test_far_plus_near_equals_ewald_and_converges_with_order():
    """near (unsoftened, one image per cell offset) + far (order p) = Ewald
    total. The error falls geometrically with p; at p = 8 it is at the 1e-6
    level (Sec. 6 of the paper quotes typical errors of 1e-5)."""
    pos, mass = _box(5, 300)
    L, cpd, R = 1.0, 7, 2
    cid = oracle.bin_particles(pos.astype(np.float32), L, cpd)["cid"]
    tot = oracle.ewald_accel(pos, L, mass=mass)
    near = oracle.accel(pos, L, cpd, R, 1e-12, mass=mass, cid=cid)
    med = {}
    for p in (4, 6, 8):
        far = oracle.far_accel(pos, L, cpd, R, p, mass=mass, cid=cid)
        e = np.linalg.norm(far + near - tot, axis=1) / np.linalg.norm(tot, axis=1)
        med[p] = np.median(e)
        if p == 8:
            assert med[p] < 2e-6 and e.max() < 5e-4, (med[p], e.max())
    assert med[4] > 8 * med[6] > 64 * med[8]


def test_far_field_follows_a_whole_cell_shift():
    """Shifting every particle by whole cells (wrapped) moves the far field
    with them: the tensor depends on cell offsets only."""
    pos, mass = _box(9, 200)
    L, cpd, R = 1.0, 7, 2
    far = oracle.far_accel(pos, L, cpd, R, 6, mass=mass)
    shifted = np.mod(pos + np.array([2, 5, 1]) / cpd, L)
    far2 = oracle.far_accel(shifted, L, cpd, R, 6, mass=mass)
    assert np.abs(far2 - far).max() <= 1e-9 * np.abs(far).max()


@pytest.mark.parametrize("cpd,R", [(5, 1), (8, 3)])
def test_far_plus_near_equals_ewald_other_radii(cpd, R):
    """The near-field radius moves images between the two parts; their sum
    is the Ewald force whatever R is."""
    pos, mass = _box(11 + R, 200)
    L = 1.0
    cid = oracle.bin_particles(pos.astype(np.float32), L, cpd)["cid"]
    tot = oracle.ewald_accel(pos, L, mass=mass)
    near = oracle.accel(pos, L, cpd, R, 1e-12, mass=mass, cid=cid)
    far = oracle.far_accel(pos, L, cpd, R, 8, mass=mass, cid=cid)
    e = np.linalg.norm(far + near - tot, axis=1) / np.linalg.norm(tot, axis=1)
    # the error falls with the separation of the nearest far cells, R + 1:
    # about 3e-5 at R = 1 and 4e-8 at R = 3 (p = 8)
    assert np.median(e) < (1e-4 if R == 1 else 2e-7), np.median(e)


def test_far_field_of_a_perfect_lattice_vanishes():
    """One particle per cell at the same offset from every cell centre: the
    periodic force on each is zero by symmetry, and so is its near field
    (every pair is a lattice vector, matched by its opposite), so the far
    field is zero too, up to the truncation of the series, which falls
    geometrically with p. A wrong sign on the odd moments, a missing
    factorial or a lopsided near block leaves a force of the order of the
    far field of a random box."""
    cpd, L, R = 5, 1.0, 2
    g = (np.arange(cpd) + 0.5) / cpd
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    lat = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1) + np.array([0.1, -0.2, 0.3]) / cpd
    m0 = 1.0 / len(lat)
    rng = np.random.default_rng(0)
    scale = np.median(np.linalg.norm(oracle.far_accel(rng.random((len(lat), 3)), L, cpd, R, 6, m0=m0), axis=1))
    big = [np.abs(oracle.far_accel(lat, L, cpd, R, p, m0=m0)).max() for p in (4, 6, 8)]
    assert big[2] < 1e-7 * scale, (big, scale)
    assert big[0] > 10 * big[1] > 100 * big[2], big
