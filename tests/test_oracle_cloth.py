"""Pins of the oracle's cloth (the paper's cloth results, Sec. VI; reading: a
corotated membrane energy per mesh triangle, psi = mu |F - R|^2 +
lam/2 (J - 1)^2 with F = Ds Dm^-1, times the rest volume, its forces on the
vertex particles added
to their P2G momentum): checked against what mechanics fixes, not against its
own formula: a rest shape has no energy or force, forces are minus the
gradient of the energy (central differences), rigid motions change neither
energy nor force magnitudes, forces conserve momentum and angular momentum,
a uniaxial stretch has the closed-form energy, and a substep conserves
momentum while the cloth's particles keep F = I."""
import numpy as np
import pytest

import oracle as O

RNG = np.random.default_rng(7)


def _tri(seed=0):
    r = np.random.default_rng(seed)
    X = r.normal(size=(3, 3)) * 0.01
    return X


def _rot(axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def test_rest_shape_has_no_energy_or_force():
    X = _tri(1)
    dmi, area = O.cloth_rest(*X)
    assert area == pytest.approx(0.5 * np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0])))
    e, f = O.cloth_triangle(*X, dmi, area * 1e-3, 1e3, 2e3)
    assert abs(e) < 1e-20 and np.max(np.abs(f)) < 1e-12


@pytest.mark.parametrize("seed", range(4))
def test_forces_are_minus_the_energy_gradient(seed):
    X = _tri(seed)
    dmi, area = O.cloth_rest(*X)
    r = np.random.default_rng(100 + seed)
    x = X + 0.2 * 0.01 * r.normal(size=(3, 3))  # a generic deformation
    mu, lam = 1.3e3, 2.1e3
    e, f = O.cloth_triangle(*x, dmi, area, mu, lam)
    h = 1e-8
    for k in range(3):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[k, c] += h
            xm[k, c] -= h
            d = (O.cloth_triangle(*xp, dmi, area, mu, lam)[0] -
                 O.cloth_triangle(*xm, dmi, area, mu, lam)[0]) / (2 * h)
            assert abs(-d - f[k, c]) <= 1e-6 * np.max(np.abs(f)) + 1e-14, (k, c)


def test_rigid_motion_invariance_and_balance():
    X = _tri(5)
    dmi, area = O.cloth_rest(*X)
    x = X + 0.003 * RNG.normal(size=(3, 3))
    mu, lam = 1e3, 4e3
    e, f = O.cloth_triangle(*x, dmi, area, mu, lam)
    Q = _rot([0.3, -1.0, 0.4], 1.1)
    y = x @ Q.T + np.array([0.5, -0.2, 0.1])
    e2, f2 = O.cloth_triangle(*y, dmi, area, mu, lam)
    assert e2 == pytest.approx(e, rel=1e-10)
    assert np.allclose(f2, f @ Q.T, atol=1e-10 * np.max(np.abs(f)))
    # no net force or moment
    assert np.max(np.abs(f.sum(0))) <= 1e-10 * np.max(np.abs(f))
    moment = sum(np.cross(x[k], f[k]) for k in range(3))
    assert np.max(np.abs(moment)) <= 1e-10 * np.max(np.abs(f)) * np.max(np.abs(x))


def test_uniaxial_stretch_closed_form():
    # right triangle in the xy plane, stretched by s along x: F = diag(s, 1)
    # in the triangle's frame, R = I, J = s: psi = mu (s-1)^2 + lam/2 (s-1)^2
    X = np.array([[0.0, 0.0, 0.0], [0.02, 0.0, 0.0], [0.0, 0.03, 0.0]])
    dmi, area = O.cloth_rest(*X)
    assert area == pytest.approx(0.5 * 0.02 * 0.03)
    for s in (0.7, 1.05, 1.6):
        x = X * np.array([s, 1.0, 1.0])
        mu, lam = 2e3, 5e3
        e, _ = O.cloth_triangle(*x, dmi, area, mu, lam)
        assert e == pytest.approx(area * (mu + 0.5 * lam) * (s - 1) ** 2, rel=1e-12)


def _sheet(n=6, spacing=0.004, z=0.05):
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x = np.stack([i.ravel() * spacing, j.ravel() * spacing, np.full(n * n, z)], 1) - \
        np.array([(n - 1) * spacing / 2, (n - 1) * spacing / 2, 0.0])
    tris = []
    for a in range(n - 1):
        for b in range(n - 1):
            v0, v1, v2, v3 = a * n + b, (a + 1) * n + b, a * n + b + 1, (a + 1) * n + b + 1
            tris += [(v0, v1, v3), (v0, v3, v2)]
    return x, np.array(tris)


def test_substep_conserves_momentum_and_keeps_cloth_unstressed():
    x0, tris = _sheet()
    n = len(x0)
    grid = {"dx": 0.004, "res": (24, 24, 40), "origin": (-0.048, -0.048, 0.0),
            "gravity": (0.0, 0.0, 0.0), "bc_layers": 3}
    mats = [{"model": O.CLOTH, "E": 1e5, "nu": 0.3, "friction_angle_deg": 0.0}]
    scene = {"groups": [{"x": x0, "tris": tris, "thickness": 1e-3}]}
    cloth = O.cloth_from_scene(scene)
    # stretch the sheet and give it a random velocity field
    x = x0 * np.array([1.15, 0.9, 1.0])
    x[:, 2] += 0.002 * np.sin(40 * x0[:, 0])
    v = RNG.normal(size=(n, 3)) * 0.01
    st = O.Sim.state({"x": x, "v": v, "mass": np.full(n, 1e-5), "vol": np.full(n, 1e-8),
                      "mat": np.zeros(n, np.int32)})
    sim = O.Sim(grid)
    sim.set_cloth(cloth)
    p0 = (st["mass"][:, None] * st["v"]).sum(0)
    code, info = sim.substep(st, mats, [], 1e-5, O.solver())
    assert code == O.OK
    p1 = (st["mass"][:, None] * st["v"]).sum(0)
    assert np.max(np.abs(p1 - p0)) <= 1e-12
    assert np.allclose(st["F"], np.eye(3))
    # the stretched sheet pulls inward along x: the mesh forces did act
    fx = np.sign(x0[:, 0]) * (st["v"][:, 0] - v[:, 0])
    assert np.mean(fx[np.abs(x0[:, 0]) > 0.005]) < 0
    sim.close()
