"""Pins of the oracle's full substep (Eq. (5)-(8)) against closed forms and
invariants: symplectic-Euler free fall, APIC mass / momentum / angular-momentum
conservation, exact round trip of affine velocity fields, zero-contact
behaviour, momentum balance with contact impulses, and basic contact physics
(a block coming to rest on the ground; sticking below and sliding at
g (sin t - mu cos t) above the friction angle on an incline)."""
import numpy as np
import pytest

import oracle as O
from paper_2503_05046_gb300 import scenes

S_TIGHT = O.solver(eps_r=1e-10, eps_a=0.0, max_iters=5000)


def _small_scene(v0=(0.3, -0.2, 0.1), n_side=6, gravity=(0.0, 0.0, -9.81), bodies=None,
                 center=(0.0, 0.0, 0.25), jitter=True):
    rng = np.random.default_rng(1)
    g = scenes.cube_group(n_side, 0.005, center, v0, scenes.elastic(1e5, 0.3, 1000.0),
                          jitter=2e-4 if jitter else 0.0, rng=rng)
    grid = {"dx": 0.01, "res": (32, 32, 48), "origin": (-0.16, -0.16, -0.04),
            "gravity": gravity, "bc_layers": 3}
    return {"grid": grid, "groups": [g], "bodies": bodies or [], "h": 1e-4, "substeps": 10}


def _run(scene, n_sub, S=S_TIGHT, st=None, mats=None):
    sim = O.Sim(scene["grid"])
    if st is None:
        st, mats = O.from_scene(scene)
    imp = np.zeros(6 * max(len(scene["bodies"]), 1))
    infos = []
    for _ in range(n_sub):
        code, info = sim.substep(st, mats, [O.make_body(b) for b in scene["bodies"]],
                                 scene["h"], S, imp)
        assert code == O.OK, code
        infos.append(info)
    return sim, st, imp, infos


def test_free_fall_closed_form():
    """F = I, no contact: every particle follows the symplectic Euler closed
    form v_n = v0 + n h g, x_n = x0 + n h v0 + h^2 g n(n+1)/2."""
    sc = _small_scene()
    st0, _ = O.from_scene(sc)
    n = 100
    sim, st, imp, _ = _run(sc, n)
    h = sc["h"]
    g = np.array(sc["grid"]["gravity"])
    v0 = st0["v"]  # the scene's float32 velocities, widened
    assert np.allclose(st["v"], v0 + n * h * g, rtol=0, atol=1e-12)
    assert np.allclose(st["x"], st0["x"] + n * h * v0 + h * h * g * n * (n + 1) / 2, atol=1e-12)
    assert np.max(np.abs(st["C"])) < 1e-9
    assert np.allclose(st["F"], np.eye(3), atol=1e-12)


def _angular(x, v, C, m, dx):
    L = np.sum(np.cross(x, m[:, None] * v), 0)
    # affine part: m dx^2/4 eps_abc C_cb
    Cs = C
    L += np.sum(m[:, None] * (dx * dx / 4) * np.stack(
        [Cs[:, 2, 1] - Cs[:, 1, 2], Cs[:, 0, 2] - Cs[:, 2, 0], Cs[:, 1, 0] - Cs[:, 0, 1]], 1), 0)
    return L


def test_p2g_g2p_conservation():
    """No gravity, no contact: P2G conserves mass, momentum and (APIC) angular
    momentum with the stress term included; G2P conserves them back."""
    sc = _small_scene(gravity=(0.0, 0.0, 0.0))
    st, mats = O.from_scene(sc)
    rng = np.random.default_rng(3)
    n = len(st["x"])
    st["v"] = rng.normal(size=(n, 3))
    A = rng.normal(size=(n, 3, 3))
    st["C"] = 10 * A
    st["F"] = np.eye(3) + 0.05 * rng.normal(size=(n, 3, 3))
    x0, v0, C0 = st["x"].copy(), st["v"].copy(), st["C"].copy()
    m = st["mass"]
    dx = sc["grid"]["dx"]
    sim = O.Sim(sc["grid"])
    code, info = sim.substep(st, mats, [], sc["h"], S_TIGHT)
    assert code == O.OK
    ids, mi, vs, vg = sim.last_grid()
    res = sc["grid"]["res"]
    idx = np.stack([ids % res[0], (ids // res[0]) % res[1], ids // (res[0] * res[1])], 1)
    xi = np.asarray(sc["grid"]["origin"]) + dx * idx
    assert abs(mi.sum() - m.sum()) < 1e-14 * m.sum()
    P_p = np.sum(m[:, None] * v0, 0)
    P_g = np.sum(mi[:, None] * vg, 0)
    assert np.allclose(P_g, P_p, atol=1e-12 * np.abs(m[:, None] * v0).sum())
    L_p = _angular(x0, v0, C0, m, dx)
    L_g = np.sum(np.cross(xi, mi[:, None] * vg), 0)
    scale = np.abs(np.cross(x0, m[:, None] * v0)).sum() + 1e-30
    assert np.allclose(L_g, L_p, atol=1e-11 * scale)
    # G2P back to particles (positions before advection)
    xb = st["x"] - sc["h"] * st["v"]
    assert np.allclose(np.sum(m[:, None] * st["v"], 0), P_g, atol=1e-12 * scale)
    assert np.allclose(_angular(xb, st["v"], st["C"], m, dx), L_g, atol=1e-11 * scale)


def test_affine_field_round_trip():
    """APIC transfers reproduce an affine velocity field exactly: particles with
    v_p = b + A x_p and C_p = A come back with the same v and C."""
    sc = _small_scene(gravity=(0.0, 0.0, 0.0))
    st, mats = O.from_scene(sc)
    rng = np.random.default_rng(4)
    A = rng.normal(size=(3, 3))
    b = rng.normal(size=3)
    st["v"] = b + st["x"] @ A.T
    st["C"] = np.tile(A, (len(st["x"]), 1, 1))
    x0 = st["x"].copy()
    sim = O.Sim(sc["grid"])
    code, _ = sim.substep(st, mats, [], sc["h"], S_TIGHT)
    assert code == O.OK
    assert np.allclose(st["v"], b + x0 @ A.T, atol=1e-12)
    assert np.allclose(st["C"], A, atol=1e-10)


def test_far_body_registers_no_contact():
    far = scenes.body(scenes.SPHERE, (0.05,), p=(0.5, 0.5, 0.5))
    sc = _small_scene(bodies=[far])
    sim, st, imp, infos = _run(sc, 3)
    assert all(i.n_contacts == 0 and i.iters == 0 for i in infos)
    assert np.all(imp == 0)


def test_contact_momentum_balance():
    """With contact, grid momentum changes by exactly the impulses on the
    particles (sum_p R_p gamma_p) and the bodies receive the opposite."""
    ground = scenes.body(scenes.HALFSPACE, mu=0.5)
    sc = _small_scene(v0=(0.0, 0.0, -0.5), bodies=[ground], center=(0.0, 0.0, 0.0124))
    st, mats = O.from_scene(sc)
    sim = O.Sim(sc["grid"])
    imp = np.zeros(6)
    code, info = sim.substep(st, mats, [O.make_body(b) for b in sc["bodies"]], sc["h"], S_TIGHT, imp)
    assert code == O.OK and info.n_contacts > 0 and info.converged
    ids, mi, vs, vg = sim.last_grid()
    p, bidx, gam, phi0, n0 = sim.last_contacts()
    dP = np.sum(mi[:, None] * (vg - vs), 0)
    assert np.allclose(dP, gam.sum(0), rtol=1e-8, atol=1e-14)
    assert np.allclose(imp[:3], -gam.sum(0), rtol=1e-12, atol=1e-18)
    assert gam[:, 2].min() >= 0  # the ground only pushes up
    assert np.all(phi0 > 0) and np.all(n0 >= 0)


def _centroid_velocity(st):
    return np.sum(st["mass"][:, None] * st["v"], 0) / st["mass"].sum()


@pytest.mark.slow
def test_block_comes_to_rest_on_ground():
    ground = scenes.body(scenes.HALFSPACE, mu=0.5)
    # bottom particle layer on the ground, moving down at 5 cm/s
    sc = _small_scene(v0=(0.0, 0.0, -0.05), bodies=[ground], center=(0.0, 0.0, 0.0075), n_side=4)
    S = O.solver(eps_r=1e-4, eps_a=0.0, max_iters=20000)
    sim, st, imp, infos = _run(sc, 1500, S)
    v = st["v"]
    assert np.max(np.abs(v)) < 2e-3
    assert abs(_centroid_velocity(st)[2]) < 2e-4
    # the ground carries the weight: impulse per substep -> m g h
    M = st["mass"].sum()
    imp2 = np.zeros(6)
    sim2 = O.Sim(sc["grid"])
    for _ in range(50):
        sim2.substep(st, O.from_scene(sc)[1], [O.make_body(b) for b in sc["bodies"]], sc["h"], S, imp2)
    assert abs(imp2[2] / (50 * sc["h"]) + M * 9.81) < 0.03 * M * 9.81


@pytest.mark.slow
@pytest.mark.parametrize("theta,mu,slides", [(30.0, 0.3, True), (20.0, 0.5, False)])
def test_incline_stick_and_slide(theta, mu, slides):
    """Block on a tilted half-space: above the friction angle the centroid
    accelerates at g (sin t - mu cos t) (within 1%); below it the block sticks
    with creep of the order of the regularisation velocity eps_s."""
    sc = scenes.incline_block(theta, mu)
    st, mats = O.from_scene(sc)
    S = O.solver(eps_r=1e-4, eps_a=0.0, max_iters=5000)
    sim = O.Sim(sc["grid"])
    bodies = [O.make_body(b) for b in sc["bodies"]]
    t = np.radians(theta)
    down = np.array([np.cos(t), 0.0, -np.sin(t)])
    vel = []
    n_sub = 1200
    for k in range(n_sub):
        code, info = sim.substep(st, mats, bodies, sc["h"], S)
        assert code == O.OK
        vel.append(_centroid_velocity(st) @ down)
    vel = np.array(vel)
    k0 = n_sub // 3
    if slides:
        a_exact = 9.81 * (np.sin(t) - mu * np.cos(t))
        a = (vel[-1] - vel[k0]) / ((n_sub - 1 - k0) * sc["h"])
        assert abs(a - a_exact) < 0.01 * a_exact
    else:
        assert np.max(np.abs(vel[k0:])) < 5 * 1e-4


@pytest.mark.parametrize("bc", [0, 1, 3])
def test_dirichlet_layers_counted_by_hand(bc):
    """Domain walls (the reading taken where the paper is silent): the nodes
    within bc_layers of a face are held at v* = 0. On a 12^3 grid whose every
    node has mass, particles at rest under gravity leave exactly
    (12 - 2 bc)^3 nodes moving: 1728, 1000 and 6^3 = 216 for 0, 1 and 3
    layers, and those are the nodes with bc <= i, j, k < 12 - bc."""
    sc = scenes.filled_box(bc=bc)
    sim, st, imp, infos = _run(sc, 1)
    ids, m, vs, v = sim.last_grid()
    assert len(ids) == 12 ** 3 and np.all(m > 0)
    moving = np.any(vs != 0.0, axis=1)
    assert int(moving.sum()) == (12 - 2 * bc) ** 3
    i, j, k = ids % 12, (ids // 12) % 12, ids // 144
    inner = (i >= bc) & (i < 12 - bc) & (j >= bc) & (j < 12 - bc) & (k >= bc) & (k < 12 - bc)
    assert np.array_equal(moving, inner)
    # free nodes fall with gravity (the particles are at rest and stress-free)
    assert np.allclose(vs[inner], [0.0, 0.0, -9.81e-4], rtol=0, atol=1e-12)
