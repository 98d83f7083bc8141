"""GPU particle update (kick, drift, timestep criterion, kick-drift-kick step)
against the oracle (Maksimova et al. 2021, Sec. 2.5: second-order leapfrog
with a global timestep; the timestep is eta times the minimum over cells of
velocity dispersion / maximum acceleration)."""
import math

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


def _setup(box, dev, sigma_v=0.05, seed=1):
    from paper_2110_11398_gb300 import NearField
    nf = NearField(box.L, box.cpd, box.eps, radius=box.R, capacity=box.n, device=dev)
    vel = (np.random.default_rng(seed).standard_normal((box.n, 3)) * sigma_v).astype(np.float32)
    pos_t = torch.from_numpy(box.pos.copy()).to(dev)
    vel_t = torch.from_numpy(vel.copy()).to(dev)
    nf.bin(pos_t, gm=box.gm)
    acc_t = nf.accel()
    return nf, pos_t, vel_t, acc_t, vel


def test_kick_and_drift_match_the_oracle_arithmetic(dev):
    box = synth.tiny()
    nf, pos, vel, acc, vel0 = _setup(box, dev, sigma_v=3.0)
    a = acc.cpu().numpy()
    nf.kick(vel, acc, 0.013)
    ref_v = (vel0.astype(np.float64) + 0.013 * a.astype(np.float64)).astype(np.float32)
    assert np.array_equal(vel.cpu().numpy(), ref_v)      # same unfused double sequence
    v1 = vel.cpu().numpy()
    nf.drift(pos, vel, 0.21)                     # moves many particles across the faces
    ref_x = oracle.wrap_f32(box.pos.astype(np.float64) + 0.21 * v1.astype(np.float64), box.L)
    got = pos.cpu().numpy()
    assert np.all(got >= 0) and np.all(got < box.L)
    crossed = np.mean((box.pos.astype(np.float64) + 0.21 * v1.astype(np.float64) < 0)
                      | (box.pos.astype(np.float64) + 0.21 * v1.astype(np.float64) >= box.L))
    assert crossed > 0.05                        # the wrap is exercised
    assert np.array_equal(got, ref_x)            # bit for bit, wrapped ones included
    nf.close()


def test_timestep_criterion(dev):
    pos, _ = synth.clustered_box(40 ** 3, 6, n_halos=15)
    box = synth.Box("cl40", pos, 1.0, 11, (1 / 40) / 40, 1 / 40 ** 3)
    nf, p, vel, acc, vel0 = _setup(box, dev)
    dt = nf.timestep(vel, acc, 0.25)
    cid = oracle.bin_particles(box.pos, box.L, box.cpd)["cid"]
    ref = oracle.cell_timestep(vel0, acc.cpu().numpy(), cid, box.cpd, 0.25)
    assert math.isfinite(dt) and dt > 0
    np.testing.assert_allclose(dt, ref, rtol=1e-6)
    nf.close()


def test_kdk_steps_match_the_oracle(dev):
    box = synth.tiny(seed=7)
    nf, pos, vel, acc, vel0 = _setup(box, dev, sigma_v=0.05)
    dt = nf.timestep(vel, acc, 0.25)
    x_ref, v_ref, a_ref = box.pos.copy(), vel0.copy(), None
    for _ in range(3):
        nf.kdk_step(pos, vel, acc, dt, gm=box.gm)
        x_ref, v_ref, a_ref = oracle.kdk_step(x_ref, v_ref, dt, box.L, box.cpd, box.R, box.eps,
                                              m0=box.gm, acc0=a_ref)
    xg, vg = pos.cpu().numpy(), vel.cpu().numpy()
    D = (xg.astype(np.float64) - x_ref) - box.L * np.round((xg.astype(np.float64) - x_ref) / box.L)
    assert np.abs(D).max() < 1e-6
    dv = np.linalg.norm(vg.astype(np.float64) - v_ref, axis=1)
    kick = np.linalg.norm(v_ref.astype(np.float64) - vel0, axis=1)
    assert np.median(dv / kick) < 1e-5, np.median(dv / kick)
    # the context's binning is that of the new positions
    cs, perm, _ = (t.cpu().numpy() for t in nf.binning())
    ref_bin = oracle.bin_particles(xg, box.L, box.cpd)
    assert np.array_equal(perm.astype(np.int64), ref_bin["perm"])
    nf.close()


def test_two_body_orbit_energy_on_gpu(dev):
    from paper_2110_11398_gb300 import NearField
    L, cpd, eps, m, d = 1.0, 5, 0.002, 1e-3, 0.1
    x = np.array([[0.45, 0.5, 0.5], [0.55, 0.5, 0.5]], np.float32)
    v = math.sqrt(m * d / (d * d + eps * eps) ** 1.5 * d / 2)
    vel = np.array([[0, -v, 0], [0, v, 0]], np.float32)
    T = 2 * math.pi * (d / 2) / v
    nf = NearField(L, cpd, eps, capacity=2, device=dev)
    pos_t, vel_t = torch.from_numpy(x).to(dev), torch.from_numpy(vel).to(dev)
    nf.bin(pos_t, gm=m)
    acc_t = nf.accel()

    def energy():
        xx, vv = pos_t.cpu().numpy().astype(np.float64), vel_t.cpu().numpy().astype(np.float64)
        D = (xx[1] - xx[0]) - L * np.round((xx[1] - xx[0]) / L)
        return 0.5 * m * (vv ** 2).sum() - m * m / math.sqrt((D * D).sum() + eps * eps)

    e0 = energy()
    worst = 0.0
    for _ in range(400):
        nf.kdk_step(pos_t, vel_t, acc_t, T / 200, gm=m)
        worst = max(worst, abs(energy() / e0 - 1))
    nf.close()
    assert worst < 3e-3, worst


def test_kdk_steps_with_the_far_field(dev):
    """With the far field enabled the step kicks with the total force."""
    from paper_2110_11398_gb300 import NearField
    box = synth.tiny(seed=8)
    vel0 = (np.random.default_rng(3).standard_normal((box.n, 3)) * 0.05).astype(np.float32)
    nf = NearField(box.L, box.cpd, box.eps, radius=box.R, capacity=box.n, device=dev)
    nf.far_init(4)
    pos = torch.from_numpy(box.pos.copy()).to(dev)
    vel = torch.from_numpy(vel0.copy()).to(dev)
    nf.bin(pos, gm=box.gm)
    acc = nf.far(out=nf.accel(), accumulate=True)
    dt = nf.timestep(vel, acc, 0.25)
    x_ref, v_ref, a_ref = box.pos.copy(), vel0.copy(), None
    for _ in range(2):
        nf.kdk_step(pos, vel, acc, dt, gm=box.gm)
        x_ref, v_ref, a_ref = oracle.kdk_step(x_ref, v_ref, dt, box.L, box.cpd, box.R, box.eps,
                                              m0=box.gm, acc0=a_ref, far_order=4)
    xg, vg, ag = pos.cpu().numpy(), vel.cpu().numpy(), acc.cpu().numpy()
    D = (xg.astype(np.float64) - x_ref) - box.L * np.round((xg.astype(np.float64) - x_ref) / box.L)
    assert np.abs(D).max() < 1e-6
    ea = np.linalg.norm(ag.astype(np.float64) - a_ref, axis=1) / np.linalg.norm(a_ref, axis=1)
    assert np.median(ea) < 1e-6, np.median(ea)
    dv = np.linalg.norm(vg.astype(np.float64) - v_ref, axis=1)
    kick = np.linalg.norm(v_ref.astype(np.float64) - vel0, axis=1)
    assert np.median(dv / kick) < 1e-5, np.median(dv / kick)
    nf.close()
