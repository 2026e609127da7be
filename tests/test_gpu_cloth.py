"""Cloth (mpm_add_cloth; the paper's cloth results, Sec. VI): a triangle mesh
whose vertices are MPM particles, its corotated membrane forces added in P2G,
against the FP64 oracle's substep from the same float32 state.

The parity case: a 13 x 13 sheet lying on the ground (every vertex 2e-5 m
inside it), pre-stretched in its plane by 0.6% and 0.4% so the membrane pulls,
sliding at 3 cm/s, with a static sphere resting on its centre; per substep
the particle velocities, positions, contacts and impulses must match the
oracle at the tolerances of the other parity tests. Then the drape scene (a
sheet falling onto a sphere) steps stably and keeps its mesh intact."""
import numpy as np
import pytest

import oracle as O
from paper_2503_05046_gb300 import scenes
from gpu_helpers import oracle_substep, rel_linf

pytestmark = pytest.mark.gpu

SOLVER_GPU = dict(eps_r=1e-6, eps_a=0.0, max_iters=200000, ls_rel_tol=1e-5, ls_max_iters=50)
SOLVER_ORC = O.solver(eps_r=1e-10, eps_a=0.0, max_iters=200000)


@pytest.fixture(scope="module")
def native():
    import torch
    assert torch.cuda.is_available()
    from paper_2503_05046_gb300 import native as N
    return N


def _parity_scene(n_side=13, spacing=4e-3, h=2e-5, radius=0.01):
    g = scenes.cloth_sheet(n_side, spacing, (0.0, 0.0, -2e-5), v0=(0.03, 0.0, 0.0))
    m_p = g["material"]["rho"] * g["vol"]
    k = 0.8 * m_p / h ** 2
    bodies = [scenes.body(scenes.HALFSPACE, mu=0.3, k=k),
              scenes.body(scenes.SPHERE, (radius, 0, 0, 0), p=(0.0, 0.0, radius - 3e-5), mu=0.3, k=k)]
    dx = 2 * spacing
    res = 4 * int(np.ceil(((n_side - 1) * spacing * 1.2 / dx + 16) / 4))
    grid = {"dx": dx, "res": (res, res, 16), "origin": (-res * dx / 2, -res * dx / 2, -6 * dx),
            "gravity": (0.0, 0.0, -9.81), "bc_layers": 3}
    return {"name": "cloth_parity", "grid": grid, "groups": [g], "bodies": bodies, "h": h,
            "substeps": 1}


def test_cloth_substeps_match_the_oracle(native):
    sc = _parity_scene()
    sim = native.Sim(sc)
    st = sim.get_particles()
    x = st["x"].copy()
    # pre-stretched in the plane: the membrane pulls inward (a strain e
    # releases at about e sqrt(E / rho), 0.3 m/s here: larger in-plane speeds
    # would bury the contact impulses under float32 rounding of the momenta)
    x[:, 0] *= 1.006
    x[:, 1] *= 1.004
    sim.set_particles(x, st["v"], st["C"], st["F"])
    sgpu = native.solver_params(**SOLVER_GPU)
    for k in range(3):
        st = sim.get_particles()
        bodies = sim.bodies()
        ost, info, osim, oimp, code = oracle_substep(sc, st, bodies, SOLVER_ORC)
        assert code == O.OK
        sim.impulses(reset=True)
        stats = sim.step(n_substeps=1, solver=sgpu)
        out = sim.get_particles()
        assert stats.contacts_max == info.n_contacts > len(x) // 2
        ev = rel_linf(out["v"], ost["v"])
        assert ev < 1e-5, "cloth v mismatch %.3e at substep %d" % (ev, k)
        assert np.max(np.abs(out["x"] - ost["x"])) < 1e-7
        vmax = np.max(np.abs(ost["v"]))
        assert np.max(np.abs(out["C"] - ost["C"])) / (vmax / sc["grid"]["dx"]) < 1e-4
        assert np.allclose(out["F"], np.eye(3))  # cloth carries no deformation gradient
        imp = sim.impulses()
        iscale = np.max(np.abs(oimp[:, :3]))
        assert np.max(np.abs(imp[:, :3] - oimp[:, :3])) < 1e-4 * iscale
    # the membrane acted: the sheet contracts in x relative to a sheet without it
    assert np.mean(np.sign(x[:, 0]) * (out["v"][:, 0] - 0.03)) < 0
    sim.close()


def _pinned_drape(n_side=13):
    # the cradle of the paper's cloth experiment in miniature: the drape
    # sheet held at its four corners, one of them moving inward
    sc = scenes.cloth_drape(n_side=n_side, v0=(0.0, 0.0, 0.0))
    n = n_side
    corners = [0, n - 1, n * (n - 1), n * n - 1]
    v = np.zeros((4, 3), np.float32)
    v[3] = (-0.05, -0.05, 0.02)
    sc["groups"][0]["pins"] = {"ids": corners, "v": v}
    return sc, np.array(corners), v


def test_pinned_cloth_substeps_match_the_oracle(native):
    sc, corners, vp = _pinned_drape()
    sim = native.Sim(sc)
    sgpu = native.solver_params(**SOLVER_GPU)
    h = sc["h"]
    x_c = sim.get_particles()["x"][corners].astype(np.float64)
    for k in range(4):
        st = sim.get_particles()
        ost, info, osim, oimp, code = oracle_substep(sc, st, sim.bodies(), SOLVER_ORC)
        assert code == O.OK
        stats = sim.step(n_substeps=1, solver=sgpu)
        out = sim.get_particles()
        assert stats.contacts_max == info.n_contacts > 0
        assert rel_linf(out["v"], ost["v"]) < 1e-5
        assert np.max(np.abs(out["x"] - ost["x"])) < 1e-7
        # the pins: on their prescribed paths, C = 0
        x_c = x_c + h * vp
        assert np.max(np.abs(out["x"][corners] - x_c)) < 1e-8
        assert np.array_equal(out["v"][corners], vp)
        assert not np.any(out["C"][corners])
    # released: the corners fall with the rest of the sheet
    sim.set_pins([], np.zeros((0, 3)))
    sim.step(n_substeps=20, solver=native.solver_params(eps_r=1e-4, max_iters=2000))
    assert np.all(sim.get_particles()["v"][corners[:3], 2] < -1e-3)
    sim.close()


def test_box_bagging_step_matches_the_oracle(native):
    """The cloth cradle (corners pinned) with the dynamic 8 cm box coming
    down on it at 5 cm/s and sliding at 2 cm/s. Each of the step's 10
    substeps (the box frozen) from the GPU's own state against the oracle's;
    then one whole step of the library, whose rigid step (Eq. (3)) moves the
    box with the step's impulses, against the oracle's rollout of the same
    step."""
    sc, dyn = scenes.box_bagging()
    sc["bodies"][1]["v"] = np.array([0.02, 0.0, -0.05])
    sgpu = native.solver_params(**SOLVER_GPU)
    sim = native.Sim(sc)
    bodies = sim.bodies()
    contacts = 0
    for k in range(sc["substeps"]):
        st = sim.get_particles()
        ost, info, osim, oimp, code = oracle_substep(sc, st, bodies, SOLVER_ORC)
        assert code == O.OK
        sim.impulses(reset=True)
        stats = sim.step(n_substeps=1, solver=sgpu)
        sim.set_bodies(bodies)  # frozen for the whole step (no rigid update here)
        out = sim.get_particles()
        assert stats.contacts_max == info.n_contacts
        contacts = max(contacts, info.n_contacts)
        assert rel_linf(out["v"], ost["v"]) < 1e-5, k
        assert np.max(np.abs(out["x"] - ost["x"])) < 1e-7
        if info.n_contacts:
            imp = sim.impulses()
            iscale = np.max(np.abs(oimp[:, :3]))
            assert np.max(np.abs(imp[:, :3] - oimp[:, :3])) < 1e-4 * iscale
    assert contacts > 20
    sim.close()

    sim = native.Sim(sc)
    sim.set_dynamics(1, dyn)
    st = sim.get_particles()
    sim.step(solver=sgpu)
    gb = sim.bodies()
    cur, imp_total = st, np.zeros((len(bodies), 6))
    for k in range(sc["substeps"]):
        ost, info, osim, oimp, code = oracle_substep(sc, cur, bodies, SOLVER_ORC)
        assert code == O.OK
        imp_total += oimp
        cur = {key: ost[key].astype(np.float32) for key in ("x", "v", "C", "F")}
    dt = sc["h"] * sc["substeps"]
    ob = O.rigid_dynamics_step(O.bodies_from_scene({"bodies": bodies})[1], dyn,
                               sc["grid"]["gravity"], imp_total[1], dt)
    dv_scale = np.linalg.norm(np.asarray(ob["v"]) - np.asarray(bodies[1]["v"]))
    assert np.max(np.abs(np.asarray(gb[1]["v"]) - ob["v"])) <= 1e-4 * dv_scale + 1e-7
    assert np.max(np.abs(np.asarray(gb[1]["p"]) - ob["p"])) < 1e-7
    # the cloth pushed back: the box gained less downward speed than in free fall
    assert gb[1]["v"][2] > bodies[1]["v"][2] - 9.81 * dt
    sim.close()


def test_cloth_drape_is_stable(native):
    sc = scenes.cloth_drape(n_side=24, spacing=4e-3, v0=(0.0, 0.0, -0.2))
    sim = native.Sim(sc)
    solver = native.solver_params(eps_r=5e-2, max_iters=2000)
    rest = np.asarray(sc["groups"][0]["x"], np.float64)
    tris = sc["groups"][0]["tris"]
    contacts = 0
    for _ in range(20):  # 200 substeps, 4 ms
        st = sim.step(solver=solver)
        contacts = max(contacts, st.contacts_max)
    x = sim.get_particles()["x"].astype(np.float64)
    assert np.all(np.isfinite(x)) and contacts > 0
    # edges neither tear nor collapse: within 15% of their rest length
    for a, b in ((0, 1), (1, 2), (2, 0)):
        l0 = np.linalg.norm(rest[tris[:, a]] - rest[tris[:, b]], axis=1)
        l1 = np.linalg.norm(x[tris[:, a]] - x[tris[:, b]], axis=1)
        assert np.all(np.abs(l1 / l0 - 1.0) < 0.15)
    # draped: the sphere (top at z = 0.04) holds the vertex above its axis
    # (0.2 mm in after the fall), the corners fall on (0.8 mm at 0.2 m/s)
    r = np.linalg.norm(rest[:, :2], axis=1)
    c, corners = np.argmin(r), r > r.max() - 1e-6
    assert 0.0395 < x[c, 2] < 0.0400
    assert np.all(x[corners, 2] < x[c, 2] - 5e-4)
    sim.close()


def test_cloth_refusals(native):
    sc = _parity_scene(n_side=4)
    sim = native.Sim(sc)
    with pytest.raises(native.MpmError):
        sim.tape_begin()  # the adjoints do not cover cloth
    with pytest.raises(native.MpmError):
        native.mpm_batch_create([sim.ctx])
    with pytest.raises(native.MpmError):
        sim.set_pins([1, 1], np.zeros((2, 3)))
    with pytest.raises(native.MpmError):
        sim.set_pins([sim.n], np.zeros((1, 3)))
    g = sc["groups"][0]
    bad = np.array([[0, 1, 99]], np.int32)
    with pytest.raises(native.MpmError):
        native.mpm_add_cloth(sim.ctx, g["x"], g["v"], bad, 1e-3, native.make_material(g["material"]))
    sim.close()
    # pins on plain particles: no tape, no batch
    sim = native.Sim(scenes.cube_drop(n_side=8))
    sim.set_pins([0, 5], np.zeros((2, 3)))
    with pytest.raises(native.MpmError):
        sim.tape_begin()
    with pytest.raises(native.MpmError):
        native.mpm_batch_create([sim.ctx])
    sim.set_pins([], np.zeros((0, 3)))
    sim.tape_begin()
    sim.tape_end()
    sim.close()
