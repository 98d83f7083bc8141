"""FP64 CPU oracle for the near-field direct sum (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this package. The product library never imports it, and it
imports nothing from the product: the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, double precision, OpenMP over
sinks). This module compiles it with gcc into ``oracle/_build/liboracle.so``
and marshals numpy arrays through ctypes. Each function cites the passage of
Maksimova et al. 2021 ("AbacusSummit", arXiv 2110.11398) that it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "farfield.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_EINVAL, ORC_ERANGE, ORC_ENOMEM = 0, -1, -2, -3


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` and ``farfield.c`` with gcc (-O2, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < max(os.path.getmtime(f) for f in _SRCS):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
               "-shared", *_SRCS, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            lib.orc_bin.argtypes = [i64, vp, dbl, i32, vp, vp, vp, vp]
            lib.orc_bin.restype = i32
            lib.orc_accel.argtypes = [i64, vp, vp, vp, dbl, dbl, i32, i32, dbl, vp, i64, vp]
            lib.orc_accel.restype = i32
            lib.orc_vjp.argtypes = [i64, vp, vp, vp, dbl, dbl, i32, i32, dbl, vp, vp, i64, vp]
            lib.orc_vjp_ex.argtypes = [i64, vp, vp, vp, dbl, dbl, i32, i32, dbl, i32, vp, vp, i64, vp]
            lib.orc_vjp_ex.restype = i32
            lib.orc_accel_ex.argtypes = [i64, vp, vp, vp, dbl, dbl, i32, i32, dbl, i32, dbl, vp, i64, vp, vp]
            lib.orc_accel_ex.restype = i32
            lib.orc_vjp.restype = i32
            lib.orc_cell_timestep.argtypes = [i64, vp, vp, vp, i32, dbl]
            lib.orc_cell_timestep.restype = dbl
            lib.orc_interactions.argtypes = [i64, vp, i32, i32, vp]
            lib.orc_interactions.restype = i64
            lib.orc_far_dtensor.argtypes = [vp, i32, i32, dbl, i32, vp]
            lib.orc_far_dtensor.restype = i32
            lib.orc_far_multi_indices.argtypes = [i32, vp]
            lib.orc_far_multi_indices.restype = i32
            lib.orc_ewald_accel.argtypes = [i64, vp, vp, dbl, dbl, dbl, vp]
            lib.orc_ewald_accel.restype = i32
            lib.orc_far_accel.argtypes = [i64, vp, vp, vp, dbl, dbl, i32, i32, i32, dbl, vp]
            lib.orc_far_accel.restype = i32
            lib.orc_num_threads.argtypes = []
            lib.orc_num_threads.restype = i32
            lib.orc_set_num_threads.argtypes = [i32]
            lib.orc_set_num_threads.restype = None
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _check(rc: int, what: str):
    if rc != ORC_OK:
        raise OracleError(f"{what} failed with code {rc}")


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(t: int) -> None:
    _load().orc_set_num_threads(int(t))


def bin_particles(pos32: np.ndarray, L: float, cpd: int):
    """Cell binning and stable counting sort (Sec. 3.1, cubic lattice of cells).

    Returns dict with ``cid`` (int32 linear cell id, x slowest), ``cell_start``
    (int64, CPD^3+1), ``perm`` (int64; sorted slot -> input index, stable) and
    ``rel`` (float32 (N,3) cell-relative coordinates in cell units, sorted).
    """
    pos32 = np.ascontiguousarray(pos32, dtype=np.float32)
    n = pos32.shape[0]
    ncell = cpd ** 3
    cid = np.empty(n, np.int32)
    cs = np.empty(ncell + 1, np.int64)
    perm = np.empty(n, np.int64)
    rel = np.empty((n, 3), np.float32)
    _check(_load().orc_bin(n, _ptr(pos32), float(L), int(cpd), _ptr(cid), _ptr(cs),
                           _ptr(perm), _ptr(rel)), "orc_bin")
    return {"cid": cid, "cell_start": cs, "perm": perm, "rel": rel}


def _prep(pos, cid, mass, sinks):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    cid = np.ascontiguousarray(cid, dtype=np.int32)
    mass = None if mass is None else np.ascontiguousarray(mass, dtype=np.float64)
    sinks = None if sinks is None else np.ascontiguousarray(sinks, dtype=np.int64)
    return pos, cid, mass, sinks


def accel(pos, L: float, cpd: int, R: int, eps: float, *, mass=None, m0: float = 1.0,
          sinks=None, cid=None) -> np.ndarray:
    """Near-field Plummer-softened accelerations in FP64 (Sec. 3.1; Sec. 5.2).

    ``pos`` may be float32 or float64 (N,3). If ``cid`` is None the cells come
    from :func:`bin_particles` on float32 positions; pass ``cid`` to hold the
    binning fixed. Returns (len(sinks) or N, 3) float64.
    """
    if cid is None:
        cid = bin_particles(np.asarray(pos, np.float32), L, cpd)["cid"]
    pos, cid, mass, sinks = _prep(pos, cid, mass, sinks)
    n = pos.shape[0]
    ns = n if sinks is None else sinks.shape[0]
    out = np.empty((ns, 3), np.float64)
    _check(_load().orc_accel(n, _ptr(pos), _ptr(cid), _ptr(mass), float(m0), float(L),
                             int(cpd), int(R), float(eps), _ptr(sinks), ns, _ptr(out)),
           "orc_accel")
    return out


LAWS = {"plummer": 0, "spline": 1}


def accel_ex(pos, L: float, cpd: int, R: int, eps: float, *, law: str = "plummer",
             kde_b: float = 0.0, mass=None, m0: float = 1.0, sinks=None, cid=None):
    """Near-field accelerations with the Plummer law (Sec. 5.2) or the spline
    law that returns to 1/r^2 at r >= eps (Sec. 2.5, 5.2), and, for kde_b > 0,
    the kernel density estimate sum_j m_j (1 - r^2/b^2)_+ (Sec. 3.3).
    Returns acc, or (acc, density) when kde_b > 0."""
    if cid is None:
        cid = bin_particles(np.asarray(pos, np.float32), L, cpd)["cid"]
    pos, cid, mass, sinks = _prep(pos, cid, mass, sinks)
    n = pos.shape[0]
    ns = n if sinks is None else sinks.shape[0]
    out = np.empty((ns, 3), np.float64)
    dens = np.empty(ns, np.float64) if kde_b > 0 else None
    _check(_load().orc_accel_ex(n, _ptr(pos), _ptr(cid), _ptr(mass), float(m0), float(L), int(cpd),
                                int(R), float(eps), LAWS[law], float(kde_b), _ptr(sinks), ns,
                                _ptr(out), _ptr(dens)), "orc_accel_ex")
    return (out, dens) if kde_b > 0 else out


def vjp(pos, w, L: float, cpd: int, R: int, eps: float, *, mass=None, m0: float = 1.0,
        sinks=None, cid=None, law: str = "plummer") -> np.ndarray:
    """Vector-Jacobian product d(sum_i w_i . a_i)/dx with the binning held fixed.

    g_k = sum_j J(Delta_kj)(m_k w_j - m_j w_k) with J(D) = f I + (f'(r)/r) D D^T
    for the pair law a = m D f(r): for Plummer J = s^-3/2 I - 3 s^-5/2 D D^T
    (derivative of the near-field sum of Sec. 3.1 / Sec. 5.2); ``law="spline"``
    differentiates the spline law of accel_ex, eps being its radius.
    """
    if cid is None:
        cid = bin_particles(np.asarray(pos, np.float32), L, cpd)["cid"]
    pos, cid, mass, sinks = _prep(pos, cid, mass, sinks)
    w = np.ascontiguousarray(w, dtype=np.float64)
    n = pos.shape[0]
    ns = n if sinks is None else sinks.shape[0]
    out = np.empty((ns, 3), np.float64)
    if law == "plummer":
        _check(_load().orc_vjp(n, _ptr(pos), _ptr(cid), _ptr(mass), float(m0), float(L),
                               int(cpd), int(R), float(eps), _ptr(w), _ptr(sinks), ns, _ptr(out)),
               "orc_vjp")
    else:
        _check(_load().orc_vjp_ex(n, _ptr(pos), _ptr(cid), _ptr(mass), float(m0), float(L),
                                  int(cpd), int(R), float(eps), LAWS[law], _ptr(w), _ptr(sinks), ns,
                                  _ptr(out)), "orc_vjp_ex")
    return out


def interactions(cid, cpd: int, R: int, per_sink: bool = False):
    """Pairwise interaction count of the near-field sum ("directs", Sec. 4.3).

    sum_c n_c * sum_{|d|<=R} n_{c+d}, self pairs included. With ``per_sink``
    also returns the number of sources seen by each particle.
    """
    cid = np.ascontiguousarray(cid, dtype=np.int32)
    n = cid.shape[0]
    nsrc = np.empty(n, np.int64) if per_sink else None
    tot = int(_load().orc_interactions(n, _ptr(cid), int(cpd), int(R), _ptr(nsrc)))
    if tot < 0:
        raise OracleError("orc_interactions: out of memory")
    return (tot, nsrc) if per_sink else tot


def cell_timestep(vel, acc, cid, cpd: int, eta: float = 0.25) -> float:
    """Small-scale timestep criterion (Sec. 2.5): eta times the minimum over
    cells of velocity dispersion / maximum particle acceleration."""
    vel = np.ascontiguousarray(vel, dtype=np.float64)
    acc = np.ascontiguousarray(acc, dtype=np.float64)
    cid = np.ascontiguousarray(cid, dtype=np.int32)
    r = float(_load().orc_cell_timestep(vel.shape[0], _ptr(vel), _ptr(acc), _ptr(cid), int(cpd),
                                        float(eta)))
    if r < 0:
        raise OracleError("orc_cell_timestep failed")
    return r


def wrap_f32(x, L: float):
    """Positions wrapped into [0, L) in double, then rounded to float32; a value
    that rounds up to L is the periodic image of 0."""
    x = np.mod(np.asarray(x, np.float64), L)
    x32 = x.astype(np.float32)
    x32[x32 >= np.float32(L)] = np.float32(0)
    return x32


def kdk_step(pos32, vel32, dt: float, L: float, cpd: int, R: int, eps: float, *, m0: float,
             acc0=None, far_order: int = 0):
    """One second-order kick-drift-kick leapfrog step with a global timestep
    (Sec. 2.5): v += a(x) dt/2; x += v dt (wrapped); v += a(x') dt/2, with the
    near-field accelerations re-binned at x' (plus the far field of order
    ``far_order`` when it is > 0: the total force). Positions and velocities
    are float32 as on the device; the arithmetic is double. Returns
    (pos, vel, acc at the new positions)."""
    def total(x):
        a = accel(x, L, cpd, R, eps, m0=m0)
        if far_order:
            a = a + far_accel(np.asarray(x, np.float64), L, cpd, R, far_order, m0=m0)
        return a
    a0 = total(pos32) if acc0 is None else np.asarray(acc0, np.float64)
    v_half = (np.asarray(vel32, np.float64) + 0.5 * dt * a0).astype(np.float32)
    x1 = wrap_f32(np.asarray(pos32, np.float64) + dt * v_half.astype(np.float64), L)
    a1 = total(x1)
    v1 = (v_half.astype(np.float64) + 0.5 * dt * a1).astype(np.float32)
    return x1, v1, a1


# ---------------------------------------------------------------- far field
def far_multi_indices(Q: int) -> np.ndarray:
    """The (a, b, c) multi-indices with a + b + c <= Q in the far-field
    oracle's order (total degree, then a, then b descending)."""
    n = (Q + 1) * (Q + 2) * (Q + 3) // 6
    out = np.empty((n, 3), np.int32)
    _check(_load().orc_far_multi_indices(int(Q), _ptr(out)), "orc_far_multi_indices")
    return out


def far_dtensor(d, P: int, R: int, alpha: float, Q: int) -> np.ndarray:
    """Ewald sum of the Cartesian derivatives d^q of the periodic 1/r at the
    point ``d`` (cell units, period P), |q| <= Q (order of far_multi_indices);
    with R >= 0 the near-field image of an integer offset is left out (the
    derivatives tensor of Sec. 3.1), with R = -1 nothing is."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    n = (Q + 1) * (Q + 2) * (Q + 3) // 6
    out = np.empty(n, np.float64)
    _check(_load().orc_far_dtensor(_ptr(d), int(P), int(R), float(alpha), int(Q), _ptr(out)),
           "orc_far_dtensor")
    return out


def ewald_accel(pos, L: float, *, mass=None, m0: float = 1.0, alpha: float | None = None) -> np.ndarray:
    """Total periodic acceleration (Ewald sum, uniform background): near plus
    far field, unsoftened. ``alpha`` in 1/box units (default 3.5 / L)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = pos.shape[0]
    if mass is not None:
        mass = np.ascontiguousarray(mass, dtype=np.float64)
    out = np.empty((n, 3), np.float64)
    _check(_load().orc_ewald_accel(n, _ptr(pos), _ptr(mass), float(m0), float(L),
                                   float(alpha or 3.5 / L), _ptr(out)), "orc_ewald_accel")
    return out


def far_accel(pos, L: float, cpd: int, R: int, p: int = 8, *, mass=None, m0: float = 1.0,
              cid=None, alpha: float | None = None) -> np.ndarray:
    """Far-field acceleration by cell multipoles, the periodic derivatives
    tensor and Taylor series of order p (Sec. 3.1). ``alpha`` in 1/cell units
    (default 3.5 / CPD)."""
    if cid is None:
        cid = bin_particles(np.asarray(pos, np.float32), L, cpd)["cid"]
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    cid = np.ascontiguousarray(cid, dtype=np.int32)
    n = pos.shape[0]
    if mass is not None:
        mass = np.ascontiguousarray(mass, dtype=np.float64)
    out = np.empty((n, 3), np.float64)
    _check(_load().orc_far_accel(n, _ptr(pos), _ptr(cid), _ptr(mass), float(m0), float(L), int(cpd),
                                 int(R), int(p), float(alpha or 3.5 / cpd), _ptr(out)), "orc_far_accel")
    return out
