"""Pins of the oracle's pinned particles (the held cloth corners of the paper's
cloth experiment, Sec. VI; reading: a Dirichlet condition on the particle, which
enters each substep with its prescribed velocity and C = 0, has the mesh forces
on it dropped, and is put back on x_start + h v_pin after G2P). Checked against
what the condition and mechanics fix: a pinned particle follows its path
exactly whatever acts on it; releasing every pin gives back the unpinned
substep bit for bit; an unpinned sheet under gravity falls with the
semi-implicit Euler closed form of its centre of mass, and pinning its corners
holds them exactly and slows the fall; bad pin sets are refused."""
import numpy as np
import pytest

import oracle as O

GRID = {"dx": 0.004, "res": (32, 32, 48), "origin": (-0.064, -0.064, 0.0),
        "gravity": (0.0, 0.0, -9.81), "bc_layers": 3}


def _sheet(n=9, spacing=0.004, z=0.12):
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x = np.stack([i.ravel() * spacing, j.ravel() * spacing, np.full(n * n, z)], 1) - \
        np.array([(n - 1) * spacing / 2, (n - 1) * spacing / 2, 0.0])
    tris = []
    for a in range(n - 1):
        for b in range(n - 1):
            v0, v1, v2, v3 = a * n + b, (a + 1) * n + b, a * n + b + 1, (a + 1) * n + b + 1
            tris += [(v0, v1, v3), (v0, v3, v2)]
    return x, np.array(tris)


def _cloth_case(n=9):
    x0, tris = _sheet(n)
    mats = [{"model": O.CLOTH, "E": 3.2e6, "nu": 0.4, "friction_angle_deg": 0.0}]
    cloth = O.cloth_from_scene({"groups": [{"x": x0, "tris": tris, "thickness": 5e-4}]})
    st = O.Sim.state({"x": x0, "v": np.zeros_like(x0), "mass": np.full(len(x0), 2.4e-5),
                      "vol": np.full(len(x0), 1.6e-8), "mat": np.zeros(len(x0), np.int32)})
    return x0, tris, mats, cloth, st


def _block(n_side=6, spacing=0.002, z=0.08, seed=3):
    r = np.random.default_rng(seed)
    g = np.arange(n_side) * spacing
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    x = x - x.mean(0) + np.array([0.0, 0.0, z]) + r.uniform(-2e-4, 2e-4, x.shape)
    n = len(x)
    F = np.tile(np.eye(3).reshape(1, 9), (n, 1)) + 0.02 * r.normal(size=(n, 9))
    st = O.Sim.state({"x": x, "v": 0.05 * r.normal(size=(n, 3)), "F": F,
                      "mass": np.full(n, 8e-6), "vol": np.full(n, 8e-9),
                      "mat": np.zeros(n, np.int32)})
    mats = [{"model": O.COROTATED, "E": 2e5, "nu": 0.3, "friction_angle_deg": 0.0}]
    return st, mats


def test_pinned_particles_follow_their_path_exactly():
    st, mats = _block()
    sim = O.Sim(GRID)
    ids = np.array([0, 17, 101], np.int32)
    vp = np.array([[0.1, -0.2, 0.05], [0.0, 0.0, 0.0], [-0.3, 0.1, 0.2]])
    sim.set_pins(ids, vp)
    x0 = st["x"][ids].copy()
    h = 1e-5
    for k in range(1, 6):
        code, _ = sim.substep(st, mats, [], h, O.solver())
        assert code == O.OK
        assert np.allclose(st["x"][ids], x0 + k * h * vp, rtol=0, atol=1e-15)
        assert np.array_equal(st["v"][ids], vp)
        assert not np.any(st["C"][ids])
    # the free particles moved under the stress and gravity
    free = np.setdiff1d(np.arange(len(st["x"])), ids)
    assert np.all(np.linalg.norm(st["v"][free], axis=1) > 0)
    sim.close()


def test_releasing_every_pin_restores_the_unpinned_substep():
    st_a, mats = _block()
    st_b, _ = _block()
    sa, sb = O.Sim(GRID), O.Sim(GRID)
    sb.set_pins([4, 9], np.ones((2, 3)))
    sb.set_pins([], np.zeros((0, 3)))
    for _ in range(3):
        assert sa.substep(st_a, mats, [], 1e-5, O.solver())[0] == O.OK
        assert sb.substep(st_b, mats, [], 1e-5, O.solver())[0] == O.OK
    for k in ("x", "v", "C", "F"):
        assert np.array_equal(st_a[k], st_b[k])
    sa.close()
    sb.close()


def test_free_sheet_falls_with_the_closed_form_and_pinned_corners_hold():
    h, K = 2e-5, 40
    g = -9.81
    x0, tris, mats, cloth, st = _cloth_case()
    sim = O.Sim(GRID)
    sim.set_cloth(cloth)
    m = st["mass"]
    z0 = (m * st["x"][:, 2]).sum() / m.sum()
    for _ in range(K):
        assert sim.substep(st, mats, [], h, O.solver())[0] == O.OK
    # semi-implicit Euler of the centre of mass: v_k = k h g, z_K = z0 + h^2 g K(K+1)/2
    zK = (m * st["x"][:, 2]).sum() / m.sum()
    vK = (m * st["v"][:, 2]).sum() / m.sum()
    assert vK == pytest.approx(K * h * g, rel=1e-12)
    assert zK - z0 == pytest.approx(h * h * g * K * (K + 1) / 2, rel=1e-9)
    sim.close()

    x0, tris, mats, cloth, st = _cloth_case()
    n = int(round(np.sqrt(len(x0))))
    corners = np.array([0, n - 1, n * (n - 1), n * n - 1], np.int32)
    sim = O.Sim(GRID)
    sim.set_cloth(cloth)
    sim.set_pins(corners, np.zeros((4, 3)))
    for _ in range(K):
        assert sim.substep(st, mats, [], h, O.solver())[0] == O.OK
    assert np.array_equal(st["x"][corners], x0[corners])
    assert not np.any(st["v"][corners])
    zp = (m * st["x"][:, 2]).sum() / m.sum()
    assert z0 > zp > zK  # it sags, held at the corners
    # the sag is largest at the middle and the mesh pulls the corners' neighbours up
    c = (n // 2) * n + n // 2
    assert st["x"][c, 2] < st["x"][1, 2] < x0[1, 2]
    sim.close()


def test_a_pinned_vertex_lends_the_grid_only_its_prescribed_momentum():
    # a stretched triangle with edges of 6 dx: no node is shared between its
    # vertices' stencils; vertex 0 is pinned, so its nodes get v* = v_pin + h g
    # exactly (no mesh force through it), while the free vertices' nodes feel
    # the membrane
    dx, h = GRID["dx"], 2e-5
    X = np.array([[0.0, 0.0, 0.1], [6 * dx, 0.0, 0.1], [0.0, 6 * dx, 0.1]]) + 0.3 * dx
    tri = np.array([[0, 1, 2]])
    cloth = O.cloth_from_scene({"groups": [{"x": X, "tris": tri, "thickness": 5e-4}]})
    mats = [{"model": O.CLOTH, "E": 3.2e6, "nu": 0.4, "friction_angle_deg": 0.0}]
    x = X * np.array([1.05, 1.02, 1.0])
    st = O.Sim.state({"x": x, "v": np.zeros((3, 3)), "mass": np.full(3, 1e-5),
                      "vol": np.full(3, 1e-8), "mat": np.zeros(3, np.int32)})
    vp = np.array([[0.02, -0.01, 0.03]])
    sim = O.Sim(GRID)
    sim.set_cloth(cloth)
    sim.set_pins([0], vp)
    assert sim.substep(st, mats, [], h, O.solver())[0] == O.OK
    ids, m, vs, _ = sim.last_grid()
    res = GRID["res"]

    def stencil(p):
        b, _, _ = O.bspline(dx, GRID["origin"], p)
        return {int(b[0] + a + res[0] * (b[1] + c + res[1] * (b[2] + e)))
                for a in range(3) for c in range(3) for e in range(3)}

    s0, s1 = stencil(x[0]), stencil(x[1]) | stencil(x[2])
    assert not (s0 & s1)
    gvec = np.array(GRID["gravity"])
    at0 = np.isin(ids, list(s0))
    assert at0.sum() == 27
    assert np.allclose(vs[at0], vp[0] + h * gvec, rtol=0, atol=1e-15)
    at1 = np.isin(ids, list(s1))
    assert np.max(np.abs(vs[at1] - h * gvec)) > 1e-6  # the membrane acted there
    sim.close()


def test_bad_pin_sets_are_refused():
    sim = O.Sim(GRID)
    with pytest.raises(ValueError):
        sim.set_pins([3, 3], np.zeros((2, 3)))
    with pytest.raises(ValueError):
        sim.set_pins([-1], np.zeros((1, 3)))
    st, mats = _block()
    sim.set_pins([len(st["x"])], np.zeros((1, 3)))  # beyond the particles
    code, _ = sim.substep(st, mats, [], 1e-5, O.solver())
    assert code == O.ERR_ARG
    sim.close()
