"""Pins of the oracle's rigid-body step (Eq. (3), a body integrated with the
contact impulses of a time step): closed forms of free fall and of a constant
torque about a principal axis, the velocity jump of a given impulse, locked
degrees of freedom, and conservation of the world angular momentum of a
torque-free body (which fixes the sign of the gyroscopic term)."""
import numpy as np

import oracle as O
from paper_2503_05046_gb300 import scenes

G = np.array([0.0, 0.0, -9.81])


def _rot(axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def _dyn(**kw):
    d = dict(mass=2.0, inertia=[0.1, 0.2, 0.3], force=[0, 0, 0], torque=[0, 0, 0], dof_mask=63,
             gravity=1)
    d.update(kw)
    return d


def test_free_fall_is_semi_implicit_euler():
    b = scenes.body(scenes.SPHERE, (0.05,), p=(0.0, 0.0, 1.0), v=(0.3, 0.0, 0.0))
    dt, n = 1e-3, 50
    for _ in range(n):
        b = O.rigid_dynamics_step(b, _dyn(), G, np.zeros(6), dt)
    assert np.allclose(b["v"], [0.3, 0.0, -9.81 * n * dt], atol=1e-12)
    z = 1.0 - 9.81 * dt * dt * n * (n + 1) / 2
    assert np.allclose(b["p"], [0.3 * n * dt, 0.0, z], atol=1e-12)


def test_impulse_gives_velocity_jump():
    R = _rot([1, 2, 3], 0.7)
    b = scenes.body(scenes.BOX, (0.1, 0.1, 0.1), R=R)
    J = np.array([0.4, -0.2, 0.1])
    L = np.array([0.01, 0.03, -0.02])
    d = _dyn(gravity=0)
    b2 = O.rigid_dynamics_step(b, d, G, np.concatenate([J, L]), 1e-3)
    assert np.allclose(b2["v"], J / d["mass"], atol=1e-14)
    Iw = R @ np.diag(d["inertia"]) @ R.T
    assert np.allclose(Iw @ b2["omega"], L, atol=1e-14)


def test_constant_torque_about_a_principal_axis():
    b = scenes.body(scenes.BOX, (0.1, 0.1, 0.1))
    d = _dyn(gravity=0, torque=[0.0, 0.0, 0.6])
    dt, n = 1e-3, 100
    for _ in range(n):
        b = O.rigid_dynamics_step(b, d, G, np.zeros(6), dt)
    assert np.allclose(b["omega"], [0.0, 0.0, 0.6 / 0.3 * n * dt], atol=1e-12)


def test_locked_degrees_of_freedom_stay_at_rest():
    b = scenes.body(scenes.BOX, (0.1, 0.1, 0.1), v=(1.0, 1.0, 1.0), omega=(1.0, 1.0, 1.0))
    d = _dyn(dof_mask=0b001001, force=[1.0, 2.0, 3.0])  # translation x, rotation about x
    b2 = O.rigid_dynamics_step(b, d, G, np.ones(6), 1e-2)
    assert b2["v"][1] == 0.0 and b2["v"][2] == 0.0 and b2["v"][0] != 0.0
    assert b2["omega"][1] == 0.0 and b2["omega"][2] == 0.0 and b2["omega"][0] != 0.0
    assert b2["p"][1] == 0.0 and b2["p"][2] == 0.0


def test_torque_free_body_keeps_its_world_angular_momentum():
    def drift(dt, T=0.05):
        b = scenes.body(scenes.BOX, (0.1, 0.1, 0.1), R=_rot([0, 1, 1], 0.3), omega=(3.0, 5.0, -4.0))
        d = _dyn(gravity=0, inertia=[0.1, 0.25, 0.4])
        L0 = np.asarray(b["R"]) @ np.diag(d["inertia"]) @ np.asarray(b["R"]).T @ np.asarray(b["omega"])
        for _ in range(int(round(T / dt))):
            b = O.rigid_dynamics_step(b, d, G, np.zeros(6), dt)
        R = np.asarray(b["R"])
        L = R @ np.diag(d["inertia"]) @ R.T @ np.asarray(b["omega"])
        return np.linalg.norm(L - L0) / np.linalg.norm(L0)
    e1, e2 = drift(1e-4), drift(5e-5)
    # first-order scheme: small and halving with dt (a flipped gyroscopic term
    # would turn L by about 2 |w| T, i.e. ~70%)
    assert e1 < 5e-3
    assert e2 < 0.7 * e1
