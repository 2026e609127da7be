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


def test_device_rigid_update_matches_the_host_path(native):
    """After each step the bodies move on the device (one warp per body:
    kinematic ones by their velocity, dynamic ones by Eq. (3) with the step's
    impulses), except while a tape records the steps, when the host
    integrates them. The same five steps with a dynamic sphere and a static
    ground, one context recording a tape and one not, give the same bodies
    and particles (FP32 rounding of the same FP64 update), and the device
    path does not need the host between steps."""
    sc = scenes.cube_contact(n_side=8, v0=(0.0, 0.0, -0.05))
    r = 0.05
    dyn = dict(mass=0.5, inertia=[0.4 * 0.5 * r * r, 0.3 * 0.5 * r * r, 0.5 * 0.5 * r * r],
               force=[0.1, 0.0, 0.0], torque=[0.0, 1e-4, 0.0], dof_mask=0b111011, gravity=1)
    sp = native.solver_params(eps_r=1e-6, eps_a=0.0, max_iters=200000)
    out = []
    for taped in (False, True):
        sim = native.Sim(sc)
        sim.set_dynamics(1, dyn)
        if taped:
            sim.tape_begin()
        for _ in range(5):
            native.mpm_step(sim.ctx, sc["h"], sc["substeps"], sp, want_stats=False)
        if taped:
            sim.tape_end()
        assert native.mpm_synchronize(sim.ctx) == native.OK
        out.append((sim.bodies(), sim.get_particles()))
        sim.close()
    (ba, pa), (bb, pb) = out
    for key in ("R", "p", "v", "omega"):
        for b0, b1 in zip(ba, bb):
            scale = max(np.max(np.abs(b1[key])), 1e-6)
            assert np.max(np.abs(np.asarray(b0[key]) - np.asarray(b1[key]))) <= 1e-6 * scale, key
    assert np.max(np.abs(ba[1]["v"] - sc["bodies"][1]["v"])) > 1e-4  # the sphere did move
    assert ba[1]["v"][2] == 0.0 and ba[1]["omega"][2] == 0.0     # locked DoFs
    assert np.max(np.abs(pa["x"] - pb["x"])) <= 1e-6
