"""Batches of scenes (mpm_batch_*): one launch per phase per substep over all
scenes, each scene's contact solve in a block of its own, the bodies moved on
the device at the end of the step. Every scene of the batch is compared with
the FP64 oracle's substep from the same float32 state (not with the
single-scene path), at the tolerances of the single-scene parity tests:
particle velocities to 1e-5 relative, x, C and F, contact sets, impulses.

The scenes are cubes of uneven size at touch-down, elastic and Drucker-Prager
sand, each pressed by a kinematic gripper jaw (the batch workload of the
benchmark, at sizes the oracle finishes in seconds).
"""
import numpy as np
import pytest

import oracle as O
from paper_2503_05046_gb300 import scenes
from gpu_helpers import oracle_substep, rel_linf

pytestmark = pytest.mark.gpu

SOLVER_GPU = dict(eps_r=1e-6, eps_a=0.0, max_iters=200000, ls_rel_tol=1e-5, ls_max_iters=50)
SOLVER_ORC = O.solver(eps_r=1e-10, eps_a=0.0, max_iters=200000)
TOL_V = 1e-5
# sand 2,744 and 3,375 particles, elastic 1,000 and 2,744
SCENE_IDS = (0, 1, 2, 3)


@pytest.fixture(scope="module")
def native():
    import torch
    assert torch.cuda.is_available()
    from paper_2503_05046_gb300 import native as N
    return N


def small_scenes(ids=SCENE_IDS):
    scs = [scenes.batch_scene(i, n_min=500, n_max=4000) for i in ids]
    models = {sc["groups"][0]["material"]["model"] for sc in scs}
    assert models == {0, 1}, "the batch mixes elastic and sand"
    assert len({scenes.n_particles(sc) for sc in scs}) >= 3, "uneven sizes"
    return scs


def compare_with_oracle(sc, st, bodies, out, imp, stats):
    ost, info, osim, oimp, code = oracle_substep(sc, st, bodies, SOLVER_ORC)
    assert code == O.OK, "oracle substep status %d" % code
    ev = rel_linf(out["v"], ost["v"])
    assert ev < TOL_V, "particle v mismatch %.3e in %s" % (ev, sc["name"])
    assert np.max(np.abs(out["x"] - ost["x"])) < 1e-4 * sc["grid"]["dx"] + 1e-7
    vmax = np.max(np.abs(ost["v"]))
    assert np.max(np.abs(out["C"] - ost["C"])) / (vmax / sc["grid"]["dx"]) < 1e-4
    assert np.max(np.abs(out["F"] - ost["F"])) < 1e-5
    assert stats["contacts_max"] == info.n_contacts > 0
    assert stats["residual_max"] <= 1e-6
    iscale = np.max(np.abs(oimp[:, :3])) + 1e-30
    assert np.max(np.abs(imp[:, :3] - oimp[:, :3])) < 1e-4 * iscale
    return ev


def run_batch_parity(native, batch, scs, steps=2, options=None):
    sgpu = native.solver_params(**SOLVER_GPU)
    errs = []
    for k in range(steps):
        for opt, val in (options or {}).get(k, ()):
            batch.set_option(opt, val)
        starts = []
        for sim in batch.sims:
            starts.append((sim.get_particles(), sim.bodies()))
            sim.impulses(reset=True)
        batch.step(scs[0]["h"], 1, sgpu)
        code, codes, stats = batch.synchronize()
        assert code == native.OK and not np.any(codes), codes
        for sim, sc, (st, bodies), s in zip(batch.sims, scs, starts, stats):
            assert s["substeps"] == 1
            errs.append(compare_with_oracle(sc, st, bodies, sim.get_particles(), sim.impulses(), s))
            # the kinematic jaw moved on the device by h v (Eq. (4)); the
            # ground stayed
            moved = sim.bodies()
            assert np.allclose(moved[0]["p"], bodies[0]["p"])
            want = np.asarray(bodies[1]["p"]) + sc["h"] * np.asarray(bodies[1]["v"])
            assert np.max(np.abs(np.asarray(moved[1]["p"]) - want)) < 1e-7
    return errs


def test_batched_scenes_match_the_oracle(native):
    scs = small_scenes()
    batch = native.Batch(scs)
    errs = run_batch_parity(native, batch, scs, steps=2)
    assert len(errs) == 2 * len(scs)
    batch.close()


def test_batched_launch_options_keep_parity(native):
    """Other work lists (64 and 128 particles per P2G warp tile, 128- and
    512-thread G2P blocks, several grid blocks per scene) and each scene's
    contact solve in a cluster of 4, then 2 blocks re-record the step's graph
    and give the same results as the oracle."""
    scs = small_scenes()
    batch = native.Batch(scs)
    opts = {0: [(native.BATCH_OPT_P2G_CHUNK, 512), (native.BATCH_OPT_G2P_THREADS, 128),
                (native.BATCH_OPT_GRID_PARTICLES, 256), (native.BATCH_OPT_SOLVE_BLOCKS, 4)],
            1: [(native.BATCH_OPT_P2G_CHUNK, 1024), (native.BATCH_OPT_G2P_THREADS, 512),
                (native.BATCH_OPT_GRID_PARTICLES, 100000), (native.BATCH_OPT_SOLVE_BLOCKS, 2),
                (native.BATCH_OPT_GRAPHS, 0)]}
    run_batch_parity(native, batch, scs, steps=2, options=opts)
    batch.close()


def test_batched_dynamic_body_matches_oracle(native):
    """A member whose jaw is dynamic: after a batch step of the scene's 10
    substeps the jaw follows Eq. (3) with the impulses of those substeps
    (the oracle's substeps chained from the same start, then its rigid step)."""
    scs = small_scenes((2, 3, 1))
    batch = native.Batch(scs)
    sim, sc = batch.sims[0], scs[0]
    dyn = dict(mass=0.05, inertia=[1e-5, 1e-5, 1e-5], force=[0.0, 0.0, 0.0],
               torque=[0.0, 0.0, 0.0], dof_mask=63, gravity=0)
    sim.set_dynamics(1, dyn)
    st = sim.get_particles()
    bodies = sim.bodies()
    sim.impulses(reset=True)
    batch.step(sc["h"], sc["substeps"], native.solver_params(**SOLVER_GPU))
    code, codes, stats = batch.synchronize()
    assert code == native.OK and not np.any(codes), codes
    assert stats[0]["substeps"] == sc["substeps"]
    cur = st
    imp_total = np.zeros((len(bodies), 6))
    for _ in range(sc["substeps"]):
        ost, info, osim, oimp, ocode = oracle_substep(sc, cur, bodies, SOLVER_ORC)
        assert ocode == O.OK
        imp_total += oimp
        cur = {key: ost[key].astype(np.float32) for key in ("x", "v", "C", "F")}
    out = sim.get_particles()
    assert rel_linf(out["v"], ost["v"]) < 1e-5
    gb = sim.bodies()
    ob = O.rigid_dynamics_step(O.bodies_from_scene({"bodies": bodies})[1], dyn,
                               sc["grid"]["gravity"], imp_total[1], sc["h"] * sc["substeps"])
    dv_scale = np.linalg.norm(np.asarray(ob["v"]) - np.asarray(bodies[1]["v"]))
    assert dv_scale > 0
    assert np.max(np.abs(np.asarray(gb[1]["v"]) - ob["v"])) <= 1e-4 * dv_scale + 1e-7
    assert np.max(np.abs(np.asarray(gb[1]["p"]) - ob["p"])) < 1e-7
    batch.close()


def test_member_calls_between_batch_steps(native):
    """Per-context calls stay valid on members between batch steps: bodies
    set on one member take effect at the next batch step, and a member
    stepped on its own (mpm_step, which sorts) rejoins the batch on its new
    particle buffer."""
    scs = small_scenes()
    batch = native.Batch(scs)
    sgpu = native.solver_params(**SOLVER_GPU)
    batch.step(scs[0]["h"], 1, sgpu)
    code, codes, _ = batch.synchronize(stats=False)
    assert code == native.OK
    # lift the jaw of member 1 out of contact, step member 2 alone
    lifted = batch.sims[1].bodies()
    lifted[1]["p"] = np.asarray(lifted[1]["p"]) + np.array([-0.05, 0.0, 0.0])
    batch.sims[1].set_bodies(lifted)
    batch.sims[2].step(n_substeps=1, solver=sgpu)
    run_batch_parity(native, batch, scs, steps=1)
    assert not np.any(batch.sims[1].contacts()[1] == 1), "the lifted jaw has no contacts"
    batch.close()
