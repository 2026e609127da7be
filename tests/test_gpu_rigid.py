"""Dynamic rigid bodies integrated by the library with the contact impulses
of each time step (Eq. (3)): one step against the oracle (its substeps with
the body frozen, then its rigid step), and the panel squeeze of Sec. VI-A
(Fig. 2) reaching the analytic steady state."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2503_05046_gb300 import scenes
from gpu_helpers import oracle_substep, rel_linf

pytestmark = pytest.mark.gpu

TIGHT = dict(eps_r=1e-6, eps_a=0.0, max_iters=200000, ls_rel_tol=1e-5, ls_max_iters=50)
SOLVER_ORC = O.solver(eps_r=1e-10, eps_a=0.0, max_iters=200000)


@pytest.fixture(scope="module")
def native():
    import torch
    assert torch.cuda.is_available()
    from paper_2503_05046_gb300 import native as N
    return N


def test_dynamic_body_step_matches_oracle(native):
    """The cube at touch-down with the side sphere made dynamic (0.5 kg,
    gravity on): one rigid step of 10 substeps."""
    sc = scenes.cube_contact(n_side=10, v0=(0.0, 0.0, -0.05))
    r = 0.05
    dyn = dict(mass=0.5, inertia=[0.4 * 0.5 * r * r] * 3, force=[0.0, 0.0, 0.0],
               torque=[0.0, 0.0, 0.0], dof_mask=63, gravity=1)
    sim = native.Sim(sc)
    sim.set_dynamics(1, dyn)
    st = sim.get_particles()
    bodies = sim.bodies()
    sp = native.solver_params(**TIGHT)
    stats = sim.step(solver=sp)
    assert stats.contacts_max > 0
    out = sim.get_particles()
    gb = sim.bodies()
    # the oracle: N substeps with the bodies frozen, impulses accumulated,
    # then the rigid step of Eq. (3) for the dynamic sphere
    cur = st
    imp_total = np.zeros((len(bodies), 6))
    for k in range(sc["substeps"]):
        ost, info, osim, oimp, code = oracle_substep(sc, cur, bodies, SOLVER_ORC)
        assert code == O.OK
        imp_total += oimp
        cur = {key: ost[key].astype(np.float32) for key in ("x", "v", "C", "F")}
    assert rel_linf(out["v"], ost["v"]) < 1e-5
    dt = sc["h"] * sc["substeps"]
    ob = O.rigid_dynamics_step(O.bodies_from_scene({"bodies": bodies})[1], dyn,
                               sc["grid"]["gravity"], imp_total[1], dt)
    # the body's velocity change is mostly gravity plus the contact impulse:
    # compare against the scale of the change
    dv_scale = np.linalg.norm(np.asarray(ob["v"]) - np.asarray(bodies[1]["v"]))
    assert np.max(np.abs(np.asarray(gb[1]["v"]) - ob["v"])) <= 1e-4 * dv_scale + 1e-7
    dw_scale = np.linalg.norm(np.asarray(ob["omega"]) - np.asarray(bodies[1]["omega"])) + 1e-12
    assert np.max(np.abs(np.asarray(gb[1]["omega"]) - ob["omega"])) <= 1e-3 * dw_scale + 1e-6
    assert np.max(np.abs(np.asarray(gb[1]["p"]) - ob["p"])) < 1e-7
    # the static ground did not move
    assert np.allclose(gb[0]["p"], bodies[0]["p"])
    sim.close()


def _golden(name):
    vals = {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            key, val = line.split()
            vals[key] = float(val)
    return vals


def test_panel_squeeze_reaches_the_analytic_steady_state(native):
    """Two panels pushed together with 10 N each hold an elastic cube against
    gravity by friction (Sec. VI-A, Fig. 2): after the transient each panel
    feels the normal force 10 N and a vertical friction force of half the
    cube's weight (dt = 0.1 ms, one substep per step, eps_r = 5e-2)."""
    gold = _golden("panel_squeeze_steady_state.txt")
    f_e = gold["applied_normal_force_N"]
    sc, dyn = scenes.panel_squeeze(force=f_e)
    sim = native.Sim(sc)
    for i, d in enumerate(dyn):
        sim.set_dynamics(i, d)
    sp = native.solver_params(eps_r=5e-2, max_iters=2000)
    n_steps = 15000
    window = 1000  # the last 0.1 s, about two and a half periods of the panel
    hist = np.zeros((window, 2, 3))
    sim.impulses(reset=True)
    for k in range(n_steps):
        code, _ = sim.step(solver=sp, check=False)
        assert code == native.OK
        imp = sim.impulses(reset=True)
        if k >= n_steps - window:
            hist[k - (n_steps - window)] = imp[:, :3] / sc["h"]
    m_box = scenes.n_particles(sc) * float(np.float32(sc["groups"][0]["vol"])) * 1000.0
    half_weight = gold["friction_fraction_of_weight_per_panel"] * m_box * 9.81
    f_left, f_right = hist[:, 0].mean(0), hist[:, 1].mean(0)
    # the cube pushes each panel outwards with the applied 10 N
    assert abs(f_left[0] + f_e) < 0.02 * f_e and abs(f_right[0] - f_e) < 0.02 * f_e
    # and drags each down with half its weight; no sideways force
    assert abs(f_left[2] + half_weight) < 0.05 * half_weight
    assert abs(f_right[2] + half_weight) < 0.05 * half_weight
    assert abs(f_left[1]) < 0.02 and abs(f_right[1]) < 0.02
    # the cube hangs still between the panels
    st = sim.get_particles()
    assert abs(float(st["v"][:, 2].mean())) < 2e-3
    sim.close()
