"""mpm_backward against the FP64 oracle: directional derivatives of a linear
functional of the final state of a short rollout (the differentiation
workload in miniature: a lattice cube of elastic material or of
Drucker-Prager sand on the ground, pushed by a kinematic box; 2 rigid steps
of 5 substeps) with respect to the initial state, E, nu and each body's mu,
and the bodies' linear velocity and position, by central differences of the
oracle's rollout (Eq. (3)-(8), FP64, tightly solved), compared with the inner
product of the CUDA path's adjoint and the same direction."""
import numpy as np
import pytest

import oracle as O
from paper_2503_05046_gb300 import scenes

pytestmark = pytest.mark.gpu

SCENE = dict(side=0.04, dx=0.01, lattice_side=8, substeps=5, sink=1e-5, box_overlap=1e-5,
             v0=(0.02, 0.0, -0.02))
STEPS = 2
GPU_SOLVER = dict(eps_r=1e-7, eps_a=0.0, max_iters=100000, ls_rel_tol=1e-6, ls_max_iters=60)
ORC_SOLVER = dict(eps_r=1e-10, eps_a=0.0, max_iters=50000, ls_rel_tol=1e-12)


def _initial_state(sc, sand):
    """The scene's particles; for sand a generic start away from the return
    map's kinks: F = I with uniform velocity makes C' = 0 inside the cube, so
    tr(log s) sits exactly on the tension/compression boundary of the return
    map, where the rollout has no derivative (the one-sided slopes differ).
    Sand starts instead slightly compressed with a random shear and velocity
    spread (float32 values, shared by both sides)."""
    st0, _ = O.from_scene(sc)
    st = {k: np.array(v) for k, v in st0.items()}
    if sand:
        n = len(st["x"])
        rng = np.random.default_rng(21)
        F = np.tile(np.eye(3) * (1.0 - 2e-3), (n, 1, 1)) + 5e-4 * rng.normal(size=(n, 3, 3))
        st["F"] = F.astype(np.float32).astype(np.float64)
        st["v"] = (st["v"] + 5e-3 * rng.normal(size=(n, 3))).astype(np.float32).astype(np.float64)
    return st


@pytest.fixture(scope="module", params=["elastic", "sand"])
def case(request):
    import torch
    assert torch.cuda.is_available()
    from paper_2503_05046_gb300 import native
    sand = request.param == "sand"
    sc, _ = scenes.push_cube(**SCENE, material=scenes.SAND if sand else None)
    sc["bodies"][1]["omega"] = np.array([0.0, 0.0, 0.5])  # the box also turns
    sc["init"] = _initial_state(sc, sand)
    n = scenes.n_particles(sc)
    rng = np.random.default_rng(11)
    cot = {"x": rng.normal(size=(n, 3)), "v": rng.normal(size=(n, 3)) * 1e-2,
           "C": rng.normal(size=(n, 3, 3)) * 1e-4, "F": rng.normal(size=(n, 3, 3)) * 1e-3}
    sim = native.Sim(sc)
    init = sc["init"]
    sim.set_particles(init["x"].astype(np.float32), init["v"].astype(np.float32),
                      init["C"].astype(np.float32), init["F"].astype(np.float32))
    sim.tape_begin()
    for _ in range(STEPS):
        sim.step(n_substeps=sc["substeps"], solver=native.solver_params(**GPU_SOLVER))
    sim.tape_end()
    out = sim.backward(x_bar=cot["x"].astype(np.float32), v_bar=cot["v"].astype(np.float32),
                       C_bar=cot["C"].astype(np.float32), F_bar=cot["F"].astype(np.float32))
    final = sim.get_particles()
    sim.close()
    return native, sc, cot, out, final


def _loss(sc, cot, state=None, materials=None, bodies=None):
    st, code = O.rollout(sc, STEPS, O.solver(**ORC_SOLVER), materials=materials, bodies=bodies,
                         state=sc["init"] if state is None else state)
    assert code == O.OK
    return sum(float(np.sum(cot[k] * st[k])) for k in ("x", "v", "C", "F"))


def _fd_state(sc, cot, key, delta, eps):
    st0 = sc["init"]
    plus, minus = dict(st0), dict(st0)
    plus[key] = st0[key] + eps * delta
    minus[key] = st0[key] - eps * delta
    return (_loss(sc, cot, state=plus) - _loss(sc, cot, state=minus)) / (2 * eps)


def _fd_material(sc, cot, key, eps):
    _, mats = O.from_scene(sc)
    p, m = [dict(x) for x in mats], [dict(x) for x in mats]
    p[0][key] += eps
    m[0][key] -= eps
    return (_loss(sc, cot, materials=p) - _loss(sc, cot, materials=m)) / (2 * eps)


def _fd_mu(sc, cot, b, eps):
    bp, bm = O.bodies_from_scene(sc), O.bodies_from_scene(sc)
    bp[b]["mu"] += eps
    bm[b]["mu"] -= eps
    return (_loss(sc, cot, bodies=bp) - _loss(sc, cot, bodies=bm)) / (2 * eps)


def _fd_body(sc, cot, b, key, c, eps):
    bp, bm = O.bodies_from_scene(sc), O.bodies_from_scene(sc)
    if key == "R":  # a world-frame rotation of the orientation about axis c
        def turned(R, t):
            k = np.zeros(3)
            k[c] = 1.0
            K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
            Q = np.eye(3) + np.sin(t) * K + (1 - np.cos(t)) * K @ K
            return Q @ np.asarray(R, np.float64).reshape(3, 3)
        bp[b]["R"] = turned(bp[b]["R"], eps)
        bm[b]["R"] = turned(bm[b]["R"], -eps)
    else:
        bp[b][key] = np.array(bp[b][key], np.float64)
        bm[b][key] = np.array(bm[b][key], np.float64)
        bp[b][key][c] += eps
        bm[b][key][c] -= eps
    return (_loss(sc, cot, bodies=bp) - _loss(sc, cot, bodies=bm)) / (2 * eps)


def test_forward_matches_oracle(case):
    native, sc, cot, out, final = case
    st, code = O.rollout(sc, STEPS, O.solver(**ORC_SOLVER), state=sc["init"])
    assert code == O.OK
    assert np.max(np.abs(final["x"] - st["x"])) < 1e-6


@pytest.mark.parametrize("key,eps", [("v", 1e-6), ("x", 1e-8), ("F", 1e-7), ("C", 1e-5)])
def test_state_adjoint(case, key, eps):
    native, sc, cot, out, final = case
    n = scenes.n_particles(sc)
    shape = (n, 3) if key in "xv" else (n, 3, 3)
    delta = np.random.default_rng({"v": 1, "x": 2, "F": 3, "C": 4}[key]).normal(size=shape)
    fd = _fd_state(sc, cot, key, delta, eps)
    got = float(np.sum(out[key].astype(np.float64) * delta))
    print("d/d%s0: fd %.6e adjoint %.6e rel %.2e" % (key, fd, got, abs(got - fd) / abs(fd)))
    assert abs(got - fd) <= 1e-3 * abs(fd)


def test_parameter_adjoint(case):
    native, sc, cot, out, final = case
    E = float(np.float32(sc["groups"][0]["material"]["E"]))
    rows = [("E", _fd_material(sc, cot, "E", 1e-6 * E), out["E"][0]),
            ("nu", _fd_material(sc, cot, "nu", 1e-6), out["nu"][0])]
    for b in range(len(sc["bodies"])):
        rows.append(("mu%d" % b, _fd_mu(sc, cot, b, 1e-6), out["mu"][b]))
    # the pushing box (kinematic: its position advances with v) and the
    # ground's velocity (static: it enters the contacts' bias only)
    for c in (0, 2):
        rows.append(("v1_%d" % c, _fd_body(sc, cot, 1, "v", c, 1e-6), out["body_v"][1][c]))
        rows.append(("p1_%d" % c, _fd_body(sc, cot, 1, "p", c, 1e-8), out["body_p"][1][c]))
    rows.append(("v0_0", _fd_body(sc, cot, 0, "v", 0, 1e-6), out["body_v"][0][0]))
    # angular velocity and orientation of the turning box; a tilt of the ground
    for c in (0, 2):
        rows.append(("w1_%d" % c, _fd_body(sc, cot, 1, "omega", c, 1e-6), out["body_w"][1][c]))
        rows.append(("R1_%d" % c, _fd_body(sc, cot, 1, "R", c, 1e-7), out["body_R"][1][c]))
    rows.append(("R0_0", _fd_body(sc, cot, 0, "R", 0, 1e-7), out["body_R"][0][0]))
    for name, fd, got in rows:
        print("d/d%s: fd %.6e adjoint %.6e rel %.2e" % (name, fd, got, abs(got - fd) / max(abs(fd), 1e-300)))
    scale = max(abs(fd) for _, fd, _ in rows if _ is not None)
    for name, fd, got in rows:
        # (a derivative that vanishes by symmetry is compared absolutely)
        assert abs(got - fd) <= 1e-3 * abs(fd) or abs(got - fd) <= 1e-9 * scale, name


def test_autograd_rollout(case):
    """The torch.autograd binding: a nonlinear loss (squared centroid
    distance plus a velocity term) through the rollout; E.grad, nu.grad,
    mu.grad, the pushing box's velocity gradient and a direction of v0.grad
    against central differences of the oracle's rollout."""
    import torch
    from paper_2503_05046_gb300 import autograd
    native, sc, cot, out, final = case
    if sc["groups"][0]["material"]["model"] != scenes.COROTATED:
        pytest.skip("the binding starts from F = I, where sand sits on the return map's kink")
    n = scenes.n_particles(sc)
    target = np.array([0.01, 0.0, 0.02])
    wv = np.random.default_rng(12).normal(size=(n, 3)) * 1e-2

    def loss_np(st):
        c = st["x"].mean(0)
        return float(np.sum((c - target) ** 2) + np.sum(wv * st["v"]))

    mat = sc["groups"][0]["material"]
    x0 = torch.tensor(sc["groups"][0]["x"], dtype=torch.float32, device="cuda")
    v0 = torch.tensor(sc["groups"][0]["v"], dtype=torch.float32, device="cuda", requires_grad=True)
    E = torch.tensor([float(np.float32(mat["E"]))], dtype=torch.float64, requires_grad=True)
    nu = torch.tensor([float(np.float32(mat["nu"]))], dtype=torch.float64, requires_grad=True)
    mu = torch.tensor([float(np.float32(b["mu"])) for b in sc["bodies"]], dtype=torch.float64,
                      requires_grad=True)
    bv = torch.tensor(np.array([np.float32(b["v"]) for b in sc["bodies"]], np.float64),
                      requires_grad=True)
    sim = native.Sim(sc)
    xf, vf = autograd.rollout(sim, STEPS, x0, v0, E, nu, mu,
                              solver=native.solver_params(**GPU_SOLVER), body_v=bv)
    L = ((xf.double().mean(0) - torch.tensor(target, device="cuda")) ** 2).sum() + \
        (vf.double() * torch.tensor(wv, device="cuda")).sum()
    L.backward()
    sim.close()
    S = O.solver(**ORC_SOLVER)

    def orc(materials=None, bodies=None, state=None):
        st, code = O.rollout(sc, STEPS, S, materials=materials, bodies=bodies,
                             state=sc["init"] if state is None else state)
        assert code == O.OK
        return loss_np(st)

    _, mats = O.from_scene(sc)
    hE = 1e-6 * mats[0]["E"]
    p, m = [dict(mats[0], E=mats[0]["E"] + hE)], [dict(mats[0], E=mats[0]["E"] - hE)]
    assert abs(E.grad.item() - (orc(materials=p) - orc(materials=m)) / (2 * hE)) <= \
        1e-3 * abs((orc(materials=p) - orc(materials=m)) / (2 * hE))
    p, m = [dict(mats[0], nu=mats[0]["nu"] + 1e-6)], [dict(mats[0], nu=mats[0]["nu"] - 1e-6)]
    fd = (orc(materials=p) - orc(materials=m)) / 2e-6
    assert abs(nu.grad.item() - fd) <= 1e-3 * abs(fd)
    for b in range(len(sc["bodies"])):
        bp, bm = O.bodies_from_scene(sc), O.bodies_from_scene(sc)
        bp[b]["mu"] += 1e-6
        bm[b]["mu"] -= 1e-6
        fd = (orc(bodies=bp) - orc(bodies=bm)) / 2e-6
        assert abs(mu.grad[b].item() - fd) <= 1e-3 * abs(fd), b
    bp, bm = O.bodies_from_scene(sc), O.bodies_from_scene(sc)
    bp[1]["v"] = np.array(bp[1]["v"]) + np.array([1e-6, 0.0, 0.0])
    bm[1]["v"] = np.array(bm[1]["v"]) - np.array([1e-6, 0.0, 0.0])
    fd = (orc(bodies=bp) - orc(bodies=bm)) / 2e-6
    assert abs(bv.grad[1, 0].item() - fd) <= 1e-3 * abs(fd)
    st0 = sc["init"]
    dv = np.random.default_rng(13).normal(size=(n, 3))
    sp, sm = dict(st0), dict(st0)
    sp["v"] = st0["v"] + 1e-6 * dv
    sm["v"] = st0["v"] - 1e-6 * dv
    fd = (orc(state=sp) - orc(state=sm)) / 2e-6
    got = float(np.sum(v0.grad.double().cpu().numpy() * dv))
    assert abs(got - fd) <= 1e-3 * abs(fd)


def test_backward_error_paths():
    """mpm_backward refuses what it cannot differentiate, with MPM_ERR_STATE
    and without touching the state: no tape, a body that changed kind
    (kinematic, then dynamic) within the tape, particles added after the
    tape began, particles or bodies set between two recorded steps;
    mpm_set_material is refused while recording. Setting them after the tape
    begins and before its first step is allowed."""
    from paper_2503_05046_gb300 import native
    sc, _ = scenes.push_cube(**SCENE)
    sim = native.Sim(sc, max_particles=2 * scenes.n_particles(sc))
    with pytest.raises(native.MpmError) as e:
        sim.backward(x_bar=np.zeros((sim.n, 3), np.float32))
    assert e.value.code == native.ERR_STATE
    sim.tape_begin()
    with pytest.raises(native.MpmError) as e:
        native.mpm_set_material(sim.ctx, 0, sc["groups"][0]["material"])
    assert e.value.code == native.ERR_STATE
    sim.step(n_substeps=2)
    before = sim.get_particles()
    sim.set_dynamics(1, {"mass": 1.0, "inertia": [1e-3, 1e-3, 1e-3]})
    sim.step(n_substeps=2)
    sim.tape_end()
    after = sim.get_particles()
    with pytest.raises(native.MpmError) as e:
        sim.backward(x_bar=np.zeros((sim.n, 3), np.float32))
    assert e.value.code == native.ERR_STATE
    assert np.array_equal(sim.get_particles()["x"], after["x"])
    sim.set_dynamics(1, None)
    sim.tape_begin()
    native.mpm_add_particles(sim.ctx, before["x"][:4] + np.float32([0, 0, 0.05]),
                             before["v"][:4], sc["groups"][0]["vol"],
                             native.make_material(sc["groups"][0]["material"]))
    with pytest.raises(native.MpmError) as e:
        sim.step(n_substeps=1)
    assert e.value.code == native.ERR_STATE
    sim.close()
    sim = native.Sim(sc)
    start, bodies = sim.get_particles(), sim.bodies()
    for reset in ("particles", "bodies", None):
        sim.tape_begin()
        sim.set_particles(start["x"], start["v"], start["C"], start["F"])
        sim.set_bodies(bodies)
        sim.step(n_substeps=1)
        if reset == "particles":
            sim.set_particles(start["x"], start["v"], start["C"], start["F"])
        elif reset == "bodies":
            sim.set_bodies(bodies)
        sim.step(n_substeps=1)
        sim.tape_end()
        if reset is None:
            sim.backward(x_bar=np.ones((sim.n, 3), np.float32))
            continue
        with pytest.raises(native.MpmError) as e:
            sim.backward(x_bar=np.ones((sim.n, 3), np.float32))
        assert e.value.code == native.ERR_STATE
    sim.close()


def test_backward_without_taped_solutions_agrees():
    """With the solution pool switched off (MPM_OPT_TAPE_SOLUTIONS = 0) every
    replayed solve starts from v*; the gradients equal those of the default
    warm-started backward (both solve the same substeps to the same
    tolerance)."""
    from paper_2503_05046_gb300 import native
    sc, _ = scenes.push_cube(**SCENE)
    n = scenes.n_particles(sc)
    xbar = np.random.default_rng(31).normal(size=(n, 3)).astype(np.float32)
    out = []
    for pool in (1 << 24, 0):
        sim = native.Sim(sc)
        native.mpm_set_option(sim.ctx, native.OPT_TAPE_SOLUTIONS, pool)
        sim.tape_begin()
        for _ in range(STEPS):
            sim.step(n_substeps=sc["substeps"], solver=native.solver_params(**GPU_SOLVER))
        sim.tape_end()
        out.append(sim.backward(x_bar=xbar))
        sim.close()
    for key in ("x", "v", "F"):
        a, b = out[0][key].astype(np.float64), out[1][key].astype(np.float64)
        assert np.max(np.abs(a - b)) <= 1e-3 * np.max(np.abs(b)), key
    for key in ("E", "nu", "mu"):
        assert np.allclose(out[0][key], out[1][key], rtol=1e-3, atol=0), key


DYN = {"mass": 0.05, "inertia": [2e-5, 3e-5, 4e-5], "force": [0.0, 0.0, 0.0],
       "torque": [0.0, 0.0, 0.0], "dof_mask": 63, "gravity": 0}


def _vee_log(Rn, Rref):
    M = np.asarray(Rn).reshape(3, 3) @ np.asarray(Rref).reshape(3, 3).T
    S = 0.5 * (M - M.T)
    return np.array([S[2, 1], S[0, 2], S[1, 0]])


def test_backward_through_a_dynamic_body():
    """The pushing box is a free rigid body (Eq. (3); no gravity, turning at
    0.5 rad/s): the loss reads the particles and the box's final state; the
    gradients in E, mu, the box's initial velocity, angular velocity,
    position and orientation and the particles' initial velocity against
    central differences of the oracle's rollout with the same rigid steps."""
    from paper_2503_05046_gb300 import native
    sc, _ = scenes.push_cube(**SCENE)
    sc["bodies"][1]["omega"] = np.array([0.0, 0.0, 0.5])
    sc["init"] = _initial_state(sc, False)
    n = scenes.n_particles(sc)
    rng = np.random.default_rng(41)
    cot = {"x": rng.normal(size=(n, 3)), "v": rng.normal(size=(n, 3)) * 1e-2,
           "C": np.zeros((n, 3, 3)), "F": np.zeros((n, 3, 3))}
    sbar = np.zeros((2, 12))
    sbar[1] = rng.normal(size=12) * np.repeat([1.0, 30.0, 0.1, 1.0], 3)
    sim = native.Sim(sc)
    sim.set_dynamics(1, DYN)
    sim.tape_begin()
    for _ in range(STEPS):
        sim.step(n_substeps=sc["substeps"], solver=native.solver_params(**GPU_SOLVER))
    sim.tape_end()
    out = sim.backward(x_bar=cot["x"].astype(np.float32), v_bar=cot["v"].astype(np.float32),
                       body_state_bar=sbar)
    final_bodies = sim.bodies()
    sim.close()
    S = O.solver(**ORC_SOLVER)
    st_ref, code, b_ref = O.rollout(sc, STEPS, S, state=sc["init"], dynamics={1: DYN},
                                    with_bodies=True)
    assert code == O.OK
    assert np.allclose(np.float32(b_ref[1]["v"]), final_bodies[1]["v"], rtol=1e-4, atol=1e-6)
    R_ref = b_ref[1]["R"]

    def loss(state=None, materials=None, bodies=None):
        st, c, bds = O.rollout(sc, STEPS, S, materials=materials, bodies=bodies,
                               state=sc["init"] if state is None else state,
                               dynamics={1: DYN}, with_bodies=True)
        assert c == O.OK
        b = bds[1]
        return (float(np.sum(cot["x"] * st["x"]) + np.sum(cot["v"] * st["v"])) +
                float(sbar[1, 0:3] @ b["v"] + sbar[1, 3:6] @ b["p"] + sbar[1, 6:9] @ b["omega"] +
                      sbar[1, 9:12] @ _vee_log(b["R"], R_ref)))

    rows = []
    _, mats = O.from_scene(sc)
    hE = 1e-6 * mats[0]["E"]
    rows.append(("E", (loss(materials=[dict(mats[0], E=mats[0]["E"] + hE)]) -
                       loss(materials=[dict(mats[0], E=mats[0]["E"] - hE)])) / (2 * hE), out["E"][0]))

    def body_fd(key, c, eps):
        bp, bm = O.bodies_from_scene(sc), O.bodies_from_scene(sc)
        if key == "R":
            k = np.zeros(3)
            k[c] = 1.0
            K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
            Q = lambda t: np.eye(3) + np.sin(t) * K + (1 - np.cos(t)) * K @ K
            bp[1]["R"] = Q(eps) @ np.asarray(bp[1]["R"]).reshape(3, 3)
            bm[1]["R"] = Q(-eps) @ np.asarray(bm[1]["R"]).reshape(3, 3)
        elif key == "mu":
            bp[1]["mu"] += eps
            bm[1]["mu"] -= eps
        else:
            bp[1][key] = np.array(bp[1][key], np.float64)
            bm[1][key] = np.array(bm[1][key], np.float64)
            bp[1][key][c] += eps
            bm[1][key][c] -= eps
        return (loss(bodies=bp) - loss(bodies=bm)) / (2 * eps)

    rows.append(("mu1", body_fd("mu", 0, 1e-6), out["mu"][1]))
    for c in (0, 2):
        rows.append(("v1_%d" % c, body_fd("v", c, 1e-6), out["body_v"][1][c]))
        rows.append(("p1_%d" % c, body_fd("p", c, 1e-8), out["body_p"][1][c]))
        rows.append(("w1_%d" % c, body_fd("omega", c, 1e-6), out["body_w"][1][c]))
        rows.append(("R1_%d" % c, body_fd("R", c, 1e-7), out["body_R"][1][c]))
    dv = rng.normal(size=(n, 3))
    sp, sm = dict(sc["init"]), dict(sc["init"])
    sp["v"] = sc["init"]["v"] + 1e-6 * dv
    sm["v"] = sc["init"]["v"] - 1e-6 * dv
    rows.append(("v0", (loss(state=sp) - loss(state=sm)) / 2e-6,
                 float(np.sum(out["v"].astype(np.float64) * dv))))
    scale = max(abs(fd) for _, fd, _ in rows)
    for name, fd, got in rows:
        print("d/d%s: fd %.6e adjoint %.6e rel %.2e" % (name, fd, got, abs(got - fd) / max(abs(fd), 1e-300)))
    for name, fd, got in rows:
        assert abs(got - fd) <= 1e-3 * abs(fd) or abs(got - fd) <= 1e-9 * scale, name


def test_backward_two_materials_uneven_steps():
    """Two particle groups (the elastic lattice cube and a sand copy beside
    it, started compressed and sheared) and recorded steps of 3 and 5
    substeps: dL/dE and dL/dnu of each group and a direction of v0 against
    central differences of the oracle's rollout."""
    from paper_2503_05046_gb300 import native
    sc, _ = scenes.push_cube(**SCENE)
    g0 = sc["groups"][0]
    g1 = dict(g0, x=(g0["x"] + np.float32([0.045, 0.0, 0.0])).astype(np.float32),
              material=dict(scenes.SAND))
    sc["groups"] = [g0, g1]
    st0, _ = O.from_scene(sc)
    st = {k: np.array(v) for k, v in st0.items()}
    n0, n = len(g0["x"]), len(st["x"])
    rng = np.random.default_rng(51)
    F = np.tile(np.eye(3), (n, 1, 1))
    F[n0:] = np.eye(3) * (1.0 - 2e-3) + 5e-4 * rng.normal(size=(n - n0, 3, 3))
    st["F"] = F.astype(np.float32).astype(np.float64)
    st["v"] = (st["v"] + 5e-3 * rng.normal(size=(n, 3))).astype(np.float32).astype(np.float64)
    steps = [3, 5]
    cot_x = rng.normal(size=(n, 3))
    sim = native.Sim(sc)
    sim.set_particles(st["x"].astype(np.float32), st["v"].astype(np.float32),
                      st["C"].astype(np.float32), st["F"].astype(np.float32))
    sim.tape_begin()
    for k in steps:
        sim.step(n_substeps=k, solver=native.solver_params(**GPU_SOLVER))
    sim.tape_end()
    out = sim.backward(x_bar=cot_x.astype(np.float32))
    sim.close()
    S = O.solver(**ORC_SOLVER)

    def loss(materials=None, state=None):
        fin, c = O.rollout(sc, len(steps), S, materials=materials,
                           state=st if state is None else state, substeps=steps)
        assert c == O.OK
        return float(np.sum(cot_x * fin["x"]))

    _, mats = O.from_scene(sc)
    rows = []
    for gi in (0, 1):
        for key, rel in (("E", 1e-6), ("nu", None)):
            h = rel * mats[gi][key] if rel else 1e-6
            p, m = [dict(x) for x in mats], [dict(x) for x in mats]
            p[gi][key] += h
            m[gi][key] -= h
            rows.append(("%s%d" % (key, gi), (loss(materials=p) - loss(materials=m)) / (2 * h),
                         out[key][gi]))
    dv = rng.normal(size=(n, 3))
    sp, sm = dict(st), dict(st)
    sp["v"] = st["v"] + 1e-6 * dv
    sm["v"] = st["v"] - 1e-6 * dv
    rows.append(("v0", (loss(state=sp) - loss(state=sm)) / 2e-6,
                 float(np.sum(out["v"].astype(np.float64) * dv))))
    for name, fd, got in rows:
        print("d/d%s: fd %.6e adjoint %.6e rel %.2e" % (name, fd, got, abs(got - fd) / abs(fd)))
    for name, fd, got in rows:
        assert abs(got - fd) <= 1e-3 * abs(fd), name
