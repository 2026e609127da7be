"""Pins of the oracle's rollout under the asynchronous splitting (Sec. IV-A)
and of central differences taken through it, the machinery the gradient
tests compare the adjoint against."""
import numpy as np

import oracle as O
from paper_2503_05046_gb300 import scenes


def _free_scene(n_side=3):
    sc = scenes.cube_drop(n_side=n_side, drop_height=0.2, v0=(0.1, 0.0, 0.0))
    sc["bodies"] = []
    sc["substeps"] = 3
    return sc


def test_rollout_free_fall_closed_form():
    """No bodies, F = I: every particle follows symplectic Euler under gravity,
    x_n = x_0 + n h v_0 + h^2 g n (n + 1) / 2 (stress-free, APIC exact)."""
    sc = _free_scene()
    st0, _ = O.from_scene(sc)
    st, code = O.rollout(sc, 2, O.solver())
    assert code == O.OK
    n, h = 6, sc["h"]
    g = np.asarray(sc["grid"]["gravity"])
    want = st0["x"] + n * h * st0["v"] + h * h * g * n * (n + 1) / 2.0
    assert np.allclose(st["x"], want, rtol=0, atol=1e-12)


def test_central_difference_of_the_centroid():
    """d centroid_n / d v0 = n h I exactly in free fall, so the central
    difference of L = |c - t|^2 in a uniform change of v0 is 2 (c - t) . d n h."""
    sc = _free_scene()
    st0, _ = O.from_scene(sc)
    t = np.array([0.01, 0.02, 0.1])
    d = np.array([0.3, -0.2, 0.5])

    def L(eps):
        s = dict(st0)
        s["v"] = st0["v"] + eps * d
        st, code = O.rollout(sc, 2, O.solver(), state=s)
        assert code == O.OK
        return float(np.sum((st["x"].mean(0) - t) ** 2))

    st, _ = O.rollout(sc, 2, O.solver())
    c = st["x"].mean(0)
    fd = (L(1e-6) - L(-1e-6)) / 2e-6
    assert abs(fd - 2.0 * np.dot(c - t, d) * 6 * sc["h"]) <= 1e-8


def test_kinematic_bodies_advance_between_steps():
    """A kinematic body far from the material moves by n_substeps h v per
    step and never touches the particles: the rollout equals free fall."""
    sc = _free_scene()
    sc["bodies"] = [scenes.body(scenes.SPHERE, (0.01,), p=(0.2, 0.2, 0.2), v=(0.1, 0.0, 0.0),
                                kinematic=1)]
    st_a, _ = O.rollout(sc, 2, O.solver())
    sc_free = _free_scene()
    st_b, _ = O.rollout(sc_free, 2, O.solver())
    assert np.array_equal(st_a["x"], st_b["x"])
    b = O.advance_kinematic(O.bodies_from_scene(sc), 3 * sc["h"])
    assert np.allclose(b[0]["p"], np.float32([0.2, 0.2, 0.2]) + np.array([0.1, 0, 0]) * 3 * sc["h"])


def test_dynamic_body_free_motion():
    """A dynamic body far from the material, without gravity, force or
    torque, spinning about a principal axis: the rigid steps of Eq. (3) keep
    v and omega, p advances by T v and R by exp(T [omega]x) (no gyroscopic
    torque about a principal axis)."""
    sc = _free_scene()
    w = np.array([0.0, 0.0, 1.5])
    sc["bodies"] = [scenes.body(scenes.BOX, (0.01, 0.02, 0.03), p=(0.2, 0.2, 0.2),
                                v=(0.1, -0.05, 0.02), omega=w)]
    dyn = {0: {"mass": 0.3, "inertia": [1e-3, 2e-3, 3e-3], "gravity": 0, "dof_mask": 63}}
    st, code, bds = O.rollout(sc, 3, O.solver(), dynamics=dyn, with_bodies=True)
    assert code == O.OK
    b0 = O.bodies_from_scene(sc)[0]
    T = 3 * sc["substeps"] * sc["h"]
    assert np.allclose(bds[0]["v"], b0["v"], rtol=0, atol=1e-15)
    assert np.allclose(bds[0]["omega"], b0["omega"], rtol=0, atol=1e-12)
    assert np.allclose(bds[0]["p"], b0["p"] + T * np.asarray(b0["v"]), rtol=0, atol=1e-14)
    th = T * float(np.float32(1.5))
    Rz = np.array([[np.cos(th), -np.sin(th), 0.0], [np.sin(th), np.cos(th), 0.0], [0.0, 0.0, 1.0]])
    assert np.allclose(np.asarray(bds[0]["R"]).reshape(3, 3), Rz @ np.asarray(b0["R"]).reshape(3, 3),
                       rtol=0, atol=1e-12)


def test_per_step_substep_counts():
    """Steps of 2 and 5 substeps: free fall reaches the closed form at n = 7
    (not 2 x 3, the scene's default), and a kinematic body far away has
    advanced by 7 h v."""
    sc = _free_scene()
    sc["bodies"] = [scenes.body(scenes.SPHERE, (0.01,), p=(0.2, 0.2, 0.2), v=(0.1, 0.0, 0.0),
                                kinematic=1)]
    st0, _ = O.from_scene(sc)
    st, code, bds = O.rollout(sc, 2, O.solver(), substeps=[2, 5], with_bodies=True)
    assert code == O.OK
    n, h = 7, sc["h"]
    g = np.asarray(sc["grid"]["gravity"])
    want = st0["x"] + n * h * st0["v"] + h * h * g * n * (n + 1) / 2.0
    assert np.allclose(st["x"], want, rtol=0, atol=1e-12)
    b0 = O.bodies_from_scene(sc)[0]
    assert np.allclose(bds[0]["p"], np.asarray(b0["p"]) + n * h * np.asarray(b0["v"]),
                       rtol=0, atol=1e-15)
