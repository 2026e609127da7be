"""Per-substep parity of the CUDA path (called through the C ABI) with the FP64
oracle, from identical float32 states: particle state, grid mass / free-motion
/ post-contact velocities, the contact set, impulses and the solve residual.

Tolerances: the CUDA path is FP32 and solves the contact problem to a relative
residual of 1e-6 (Alg. 1's stopping test); the oracle solves to 1e-10. With a
solve residual r the particle-velocity error is of order r (the oracle measures
7e-5 at r = 1e-4, 8e-7 at r = 1e-6 on these scenes), so particle velocities
must agree to 1e-5 relative (L-infinity over particles, relative to the
largest speed). Post-contact grid velocities are compared in the M-norm (the
norm of the solve's error bound) and pointwise on nodes holding at least half
a particle mass; lighter nodes sit at the edge of a stencil and carry the
residual divided by sqrt(m_i).
"""
import numpy as np
import pytest

import oracle as O
from paper_2503_05046_gb300 import scenes
from gpu_helpers import align_grids, oracle_substep, rel_linf

pytestmark = pytest.mark.gpu

TOL_V = 1e-5
SOLVER_GPU = dict(eps_r=1e-6, eps_a=0.0, max_iters=200000, ls_rel_tol=1e-5, ls_max_iters=50)
SOLVER_ORC = O.solver(eps_r=1e-10, eps_a=0.0, max_iters=200000)


@pytest.fixture(scope="module")
def native():
    import torch
    assert torch.cuda.is_available()
    from paper_2503_05046_gb300 import native as N
    return N


def run_parity(native, sc, n_sub=2, warm_steps=0, warm_solver=None, tol_v=TOL_V, check_grid=True,
               options=()):
    sim = native.Sim(sc)
    for opt, val in options:
        native.mpm_set_option(sim.ctx, opt, val)
    if warm_steps:
        for _ in range(warm_steps):
            sim.step(solver=warm_solver or native.solver_params(eps_r=1e-4, max_iters=20000),
                     check=False)
    sgpu = native.solver_params(**SOLVER_GPU)
    mass_p = min(np.float32(g["vol"]) * np.float32(g["material"]["rho"]) for g in sc["groups"])
    report = []
    for k in range(n_sub):
        st = sim.get_particles()
        bodies = sim.bodies()
        ost, info, osim, oimp, code = oracle_substep(sc, st, bodies, SOLVER_ORC)
        assert code == O.OK, "oracle substep status %d" % code
        sim.impulses(reset=True)
        stats = sim.step(n_substeps=1, solver=sgpu)
        out = sim.get_particles()
        # particle state
        ev = rel_linf(out["v"], ost["v"])
        assert ev < tol_v, "particle v mismatch %.3e at substep %d" % (ev, k)
        ex = np.max(np.abs(out["x"] - ost["x"]))
        assert ex < 1e-6 * sc["grid"]["dx"] * 100 + 1e-7, "x mismatch %.3e" % ex
        # C measures velocity differences over a cell: error ~ 6 dv / dx
        vmax = np.max(np.abs(ost["v"]))
        eC = np.max(np.abs(out["C"] - ost["C"])) / (vmax / sc["grid"]["dx"])
        assert eC < 1e-4, "C mismatch %.3e" % eC
        eF = np.max(np.abs(out["F"] - ost["F"]))
        assert eF < 1e-5, "F mismatch %.3e" % eF
        # contacts: same (particle, body) pairs
        p, b, gam, phi0, n0 = sim.contacts()
        op, ob, ogam, ophi, on0 = osim.last_contacts()
        assert info.n_contacts == len(p)
        gk = {(int(a), int(c)): i for i, (a, c) in enumerate(zip(p, b))}
        ok = {(int(a), int(c)): i for i, (a, c) in enumerate(zip(op, ob))}
        assert set(gk) == set(ok)
        if len(p):
            gi = np.array([gk[key] for key in ok])
            oi = np.array([ok[key] for key in ok])
            assert np.allclose(phi0[gi], ophi[oi], rtol=1e-3, atol=1e-7 * sc["grid"]["dx"])
            gscale = np.max(np.abs(ogam))
            assert np.max(np.abs(gam[gi] - ogam[oi])) < 1e-3 * gscale + 1e-12
            assert stats.residual_max <= 1e-6
            imp = sim.impulses()
            iscale = np.max(np.abs(oimp[:, :3])) + 1e-30
            assert np.max(np.abs(imp[:, :3] - oimp[:, :3])) < 1e-4 * iscale
        # grid
        if check_grid:
            (m, vs, v), (om, ovs, ov) = align_grids(sim.grid(), osim.last_grid(), 1e-6 * mass_p)
            # FP32 sums of B-spline-weighted masses: 1e-5 relative, plus the
            # absolute FP32 error of small weights (about 1e-7 of a particle mass)
            assert np.all(np.abs(m - om) <= 1e-5 * om + 1e-6 * mass_p)
            # free-motion velocity on nodes holding >= 1e-2 of a particle mass
            # (lighter nodes carry v* - v = h f / m with m a small fraction of
            # a particle's: FP32 rounding of the stress term is amplified by
            # m_p / m there)
            # (lighter nodes get B-spline weights below 1e-3, whose FP32 value
            # has a relative error above 1e-5)
            mid = om >= 1e-2 * mass_p
            assert rel_linf(vs[mid], ovs[mid]) < 1e-5
            # post-contact velocity: the objective is M-strongly convex, so the
            # stopping test of Alg. 1 bounds the solve's error in the M-norm,
            # ||v - v_opt||_M <= ||M^-1/2 grad|| <= r * scale with r the
            # relative residual (1e-6) and scale >= ||M^1/2 v||; node i may
            # thus deviate by r * scale / sqrt(m_i) (about 2x for the FP32
            # evaluation of the stopping norms). Checked in the M-norm over all
            # nodes and pointwise with that bound.
            sm = np.sqrt(om)[:, None]
            dm = sm * (v - ov)
            scale = np.linalg.norm(sm * ov)
            assert np.linalg.norm(dm) <= 1e-5 * scale
            vmax_g = np.max(np.abs(ov))
            bound = 1e-5 * vmax_g + 2.0 * 1e-6 * scale / np.sqrt(np.maximum(om, 1e-300))
            assert np.all(np.abs(v - ov).max(1) <= bound)
        report.append((k, info.n_contacts, info.iters, stats.iters_total, ev,
                       stats.ls_split_substeps, stats.cluster_substeps))
    sim.close()
    return report


def test_free_fall_matches_closed_form_and_oracle(native):
    sc = scenes.cube_drop(n_side=8)
    sim = native.Sim(sc)
    st0 = sim.get_particles()
    n = 20
    stats = sim.step(n_substeps=n)
    out = sim.get_particles()
    h, g = sc["h"], np.array(sc["grid"]["gravity"])
    v0 = st0["v"].astype(np.float64)
    assert np.allclose(out["v"], v0 + n * h * g, rtol=0, atol=2e-6)
    assert np.allclose(out["x"], st0["x"] + n * h * v0 + h * h * g * n * (n + 1) / 2, atol=2e-6)
    assert stats.contacts_max == 0 and stats.iters_total == 0
    sim.close()
    run_parity(native, sc, n_sub=2)


def test_normal_contact_parity(native):
    rep = run_parity(native, scenes.cube_contact(n_side=10, v0=(0.0, 0.0, -0.05)), n_sub=3)
    assert all(r[1] > 0 for r in rep)
    # a few hundred contacts: one thread-block cluster, each block line-searching alone
    assert all(r[6] == 1 and r[5] == 0 for r in rep), rep


def test_normal_contact_parity_cooperative_launch(native):
    """The same substeps through the cooperative kernel (device-wide barriers)
    instead of the cluster."""
    rep = run_parity(native, scenes.cube_contact(n_side=10, v0=(0.0, 0.0, -0.05)), n_sub=2,
                     options=((native.OPT_CLUSTER_CONTACTS, 0),))
    assert all(r[1] > 0 and r[6] == 0 for r in rep), rep


# P2G (form, particles per block): MPM_P2G_GATHER at 256 and 1,024, MPM_P2G_SCATTER at 256
P2G_SHAPES = [(0, 256), (0, 1024), (1, 256)]


def p2g_options(native, shape):
    return ((native.OPT_P2G_FORM, shape[0]), (native.OPT_P2G_CHUNK, shape[1]))


@pytest.mark.parametrize("shape", P2G_SHAPES)
def test_sliding_contact_parity(native, shape):
    rep = run_parity(native, scenes.cube_contact(n_side=8, v0=(0.05, 0.0, -0.05)), n_sub=2,
                     options=p2g_options(native, shape))
    assert all(r[1] > 0 for r in rep)


def test_sand_paddle_parity(native):
    sc = scenes.sand_column(n_side=12)
    rep = run_parity(native, sc, n_sub=2, warm_steps=2)
    assert any(r[1] > 0 for r in rep)


@pytest.mark.parametrize("shape", P2G_SHAPES)
def test_ragged_sizes_and_two_materials(native, shape):
    rng = np.random.default_rng(5)
    sc = scenes.cube_contact(n_side=7, v0=(0.0, 0.0, -0.05))
    sand = scenes.cube_group(5, 0.005, (-0.06, 0.0, 0.012), (0.0, 0.0, -0.02), dict(scenes.SAND),
                             jitter=1e-4, rng=rng)
    sc["groups"].append(sand)  # 343 + 125 particles: not a multiple of any tile
    run_parity(native, sc, n_sub=2, options=p2g_options(native, shape))


def test_empty_context_steps(native):
    sc = scenes.cube_drop(n_side=4)
    sc["groups"] = []
    sim = native.Sim(sc, max_particles=16)
    stats = sim.step(n_substeps=3)
    assert stats.substeps == 3 and stats.contacts_max == 0
    assert sim.impulses().shape == (2, 6)
    sim.close()


def test_sort_only_step_keeps_state_bit_exact(native):
    """n_substeps = 0 runs only the radix sort and permutation; state read back
    in id order must be bit-identical."""
    sc = scenes.sand_column(n_side=14)
    sim = native.Sim(sc)
    sim.step(n_substeps=2)
    a = sim.get_particles()
    sim.step(n_substeps=0)
    b = sim.get_particles()
    for key in a:
        assert np.array_equal(a[key], b[key])
    sim.close()


@pytest.mark.parametrize("shape", P2G_SHAPES)
@pytest.mark.parametrize("ppc", [1.0, 4.0])
def test_random_sparse_sand_parity(native, ppc, shape):
    """Sand sampled at random at about one (and four) particles per cell, as in
    the granular scooping benchmark, with the lowest particles starting in
    contact with the ground: both P2G forms on short and long same-cell runs,
    and G2P's Drucker-Prager update, off the lattice."""
    sc = scenes.sand_random(n_particles=8000, ppc=ppc, penetration=0.02 * 0.01)
    rep = run_parity(native, sc, n_sub=3, options=p2g_options(native, shape))
    assert any(r[1] > 0 for r in rep)


def test_split_line_search_parity(native):
    """More contacts than one thread block line-searches alone (4,096): the
    solve splits each line-search pass over its blocks and ends it in a
    device-wide reduction (Alg. 1's exact line search, Sec. V-B). A sand slab
    whose whole bottom layer (72 x 72 particles) is inside the ground, with a
    paddle on one side: particle and grid velocities, contacts, impulses and
    the residual against the oracle, substep by substep, and the statistics
    must show that the split path ran."""
    sc = scenes.sand_slab()
    rep = run_parity(native, sc, n_sub=2, options=((native.OPT_CLUSTER_CONTACTS, 4096),))
    assert all(r[1] > 4096 for r in rep), [r[1] for r in rep]
    assert all(r[5] == 1 and r[6] == 0 for r in rep), "the split line search did not run: %s" % rep


def test_cluster_split_line_search_parity(native):
    """The same slab (5,000+ contacts) solved by one thread-block cluster: the
    line-search passes split over the cluster's blocks and reduced through
    distributed shared memory, against the oracle."""
    sc = scenes.sand_slab()
    rep = run_parity(native, sc, n_sub=2, options=((native.OPT_CLUSTER_CONTACTS, 1 << 16),))
    assert all(r[1] > 4096 for r in rep), [r[1] for r in rep]
    assert all(r[5] == 1 and r[6] == 1 for r in rep), "the cluster solve did not run: %s" % rep


def _support(shape, params, R, d):
    """Offset from a body's origin to its point farthest along d (unit)."""
    u = R.T @ d  # d in the body frame
    if shape == scenes.BOX:
        return R @ (np.sign(u) * np.asarray(params[:3]))
    if shape == scenes.CAPSULE:
        return R @ np.array([0.0, 0.0, np.sign(u[2]) * params[0]]) + params[1] * d
    return params[0] * d  # sphere


def _random_rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    return q if np.linalg.det(q) > 0 else -q


def extremes_scene(depth=8e-3, v0=(0.0, 0.0, 0.0)):
    """A 14^3-particle elastic cube at 5 mm spacing (dx = 1 cm, the scale of
    the other parity scenes) with rigid bodies whose extreme points (two
    randomly rotated boxes' corners, a tilted capsule's end cap, a sphere's
    pole) reach `depth` into four of its faces: the contacts sit where the
    geometry is farthest from each body's origin. The bodies are frictionless:
    deep contacts of a cube at rest stick, and the oracle's solve to 1e-10 then
    takes over 10^5 iterations."""
    rng = np.random.default_rng(31)
    dx, spacing, n_side = 1e-2, 5e-3, 14
    centre = np.array([0.0, 0.0, 0.06])
    half = n_side * spacing / 2.0
    g = scenes.cube_group(n_side, spacing, centre, v0, scenes.elastic(1.0e5, 0.3, 1000.0),
                          jitter=1e-2 * spacing, rng=rng)
    bodies = [scenes.body(scenes.HALFSPACE, mu=0.4)]
    faces = [  # (direction into the cube, a point of the face, shape, params, rotation)
        (np.array([-1.0, 0.0, 0.0]), centre + [half, 0.008, -0.004], scenes.BOX, (0.02, 0.03, 0.04),
         _random_rotation(rng)),
        (np.array([1.0, 0.0, 0.0]), centre + [-half, -0.008, 0.008], scenes.BOX, (0.015, 0.025, 0.035),
         _random_rotation(rng)),
        (np.array([0.0, 1.0, 0.0]), centre + [0.012, -half, 0.0], scenes.CAPSULE, (0.02, 0.01),
         _random_rotation(rng)),
        (np.array([0.0, 0.0, -1.0]), centre + [-0.008, 0.004, half], scenes.SPHERE, (0.015,), np.eye(3)),
    ]
    for d, face, shape, params, R in faces:
        target = face + depth * d  # the extreme point, `depth` inside the face
        p = target - _support(shape, params, R, d)
        bodies.append(scenes.body(shape, params, p=p, R=R, mu=0.0))
    grid = {"dx": dx, "res": (40, 40, 32), "origin": (-0.2, -0.2, -0.06),
            "gravity": (0.0, 0.0, -9.81), "bc_layers": 3}
    return {"name": "extremes_%d" % len(g["x"]), "grid": grid, "groups": [g], "bodies": bodies,
            "h": 1e-4, "substeps": 1}


@pytest.mark.parametrize("shape", P2G_SHAPES)
def test_contacts_at_body_extremes_parity(native, shape):
    """Contact detection skips a body for a warp whose particles all lie
    outside a ball around the body's origin; the contact set must still be the
    oracle's where the geometry is farthest from that origin."""
    sc = extremes_scene()
    rep = run_parity(native, sc, n_sub=1, options=p2g_options(native, shape))
    assert rep[0][1] > 0
    sim = native.Sim(sc)
    for opt, val in p2g_options(native, shape):
        native.mpm_set_option(sim.ctx, opt, val)
    sim.step(n_substeps=1, solver=native.solver_params(**SOLVER_GPU))
    _, b, _, _, _ = sim.contacts()
    sim.close()
    assert set(int(x) for x in b) >= {1, 2, 3, 4}, "every body has contacts"
