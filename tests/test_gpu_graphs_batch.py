"""CUDA-graph replay of a step and concurrently stepped contexts (batched
scenes) give the results of plain launches, to the solver's tolerance."""
import numpy as np
import pytest

from paper_2503_05046_gb300 import scenes
from gpu_helpers import rel_linf

pytestmark = pytest.mark.gpu

TIGHT = dict(eps_r=1e-6, eps_a=0.0, max_iters=200000, ls_rel_tol=1e-5, ls_max_iters=50)


@pytest.fixture(scope="module")
def native():
    import torch
    assert torch.cuda.is_available()
    from paper_2503_05046_gb300 import native as N
    return N


def _run(native, sc, steps, graphs, cap=0, solver=TIGHT, change_h_at=None):
    sim = native.Sim(sc)
    native.mpm_set_option(sim.ctx, native.OPT_GRAPHS, 1 if graphs else 0)
    native.mpm_set_option(sim.ctx, native.OPT_SOLVE_BLOCKS, cap)
    sp = native.solver_params(**solver)
    for k in range(steps):
        h = sc["h"] * (0.5 if change_h_at is not None and k >= change_h_at else 1.0)
        sim.step(h=h, solver=sp)
    out = sim.get_particles()
    imp = sim.impulses()
    sim.close()
    return out, imp


def test_graph_replay_matches_direct_launches(native):
    sc = scenes.cube_contact(n_side=10, v0=(0.0, 0.0, -0.05))
    # 4 steps: both particle buffers' graphs are recorded and replayed; h
    # changes after step 2 (the graphs are recorded again)
    a, ia = _run(native, sc, 4, graphs=False, change_h_at=2)
    b, ib = _run(native, sc, 4, graphs=True, change_h_at=2)
    assert rel_linf(b["v"], a["v"].astype(np.float64)) < 1e-5
    assert np.max(np.abs(b["x"] - a["x"])) < 1e-7
    assert np.allclose(ib, ia, rtol=1e-4, atol=1e-4 * np.max(np.abs(ia)))


def test_solve_block_cap_matches_default(native):
    sc = scenes.cube_contact(n_side=10, v0=(0.0, 0.0, -0.05))
    a, _ = _run(native, sc, 2, graphs=True, cap=0)
    b, _ = _run(native, sc, 2, graphs=True, cap=1)
    assert rel_linf(b["v"], a["v"].astype(np.float64)) < 1e-5


def test_batched_contexts_match_one_at_a_time(native):
    """Four scenes of uneven size stepped side by side on their own streams
    equal the same scenes stepped one at a time (same launch configuration)."""
    import torch
    scs = [scenes.batch_scene(i, n_max=12000) for i in range(4)]
    # the touch-down substep of these light, stiffly sticking scenes takes
    # thousands of QN iterations: start both runs from a state one step in
    warm = native.solver_params(eps_r=5e-2, max_iters=1000)
    sp = native.solver_params(eps_r=1e-5, eps_a=0.0, max_iters=100000, ls_rel_tol=1e-5,
                              ls_max_iters=50)
    states = []
    for sc in scs:
        sim = native.Sim(sc)
        sim.step(solver=warm, check=False)
        states.append((sim.get_particles(), sim.bodies()))
        sim.close()

    def make(sc, st):
        sim = native.Sim(sc)
        native.mpm_set_option(sim.ctx, native.OPT_SOLVE_BLOCKS, 2)
        sim.set_particles(st[0]["x"], st[0]["v"], st[0]["C"], st[0]["F"])
        sim.set_bodies(st[1])
        return sim

    ref = []
    for sc, st in zip(scs, states):
        sim = make(sc, st)
        code, _ = sim.step(solver=sp, check=False)
        assert code == native.OK
        ref.append(sim.get_particles())
        sim.close()
    sims = [make(sc, st) for sc, st in zip(scs, states)]
    for sim, sc in zip(sims, scs):
        native.mpm_step(sim.ctx, sc["h"], sc["substeps"], sp, want_stats=False)
    torch.cuda.synchronize()
    for sim, r in zip(sims, ref):
        assert native.mpm_synchronize(sim.ctx) == native.OK
        out = sim.get_particles()
        assert rel_linf(out["v"], r["v"].astype(np.float64)) < 1e-4
        sim.close()


def test_batch_autotuner(native):
    """tune.tune_batch times each candidate (solve cap, P2G chunk) on the
    batch, applies the fastest and leaves every context able to step."""
    from paper_2503_05046_gb300 import tune
    scs = [scenes.batch_scene(i, n_max=8000) for i in range(3)]
    sims = [native.Sim(sc) for sc in scs]
    solver = native.solver_params(eps_r=5e-2, max_iters=1000)
    (cap, chunk), table = tune.tune_batch(sims, scs, solver, caps=(2, 4), chunks=(256, 512), steps=1)
    assert len(table) == 4 and all(t > 0 for _, _, t in table)
    assert (cap, chunk) == min(table, key=lambda r: r[2])[:2]
    for sim in sims:
        code, _ = sim.step(solver=solver, check=False)
        assert code in (native.OK, native.ERR_NOT_CONVERGED)
        sim.close()
