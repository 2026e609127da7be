"""Measured choice of launch options for many scenes.

Two ways to advance many independent scenes, each tuned by timing a few
steps of the whole set per candidate (the scenes advance while it measures:
the timed steps are ordinary steps of the simulation):

- a batch (native.Batch, mpm_batch_*): one launch per phase per substep over
  all scenes' (scene, block) work items. `tune_batch_launch` picks the
  particles per P2G warp tile (MPM_BATCH_OPT_P2G_CHUNK / 8 warps), the
  threads per G2P block, the particles per grid-phase block and the blocks
  per scene's contact solve, by coordinate descent;
- contexts side by side, each on its own stream replaying its step's CUDA
  graph (mpm_step with graphs on). `tune_batch` picks the cap on the SMs one
  context's cooperative contact solve occupies (MPM_OPT_SOLVE_BLOCKS) and the
  particles per P2G thread block (MPM_OPT_P2G_CHUNK).
"""
import time

from . import native


def _step_all(sims, scenes_, solver, steps):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        for sim, sc in zip(sims, scenes_):
            native.mpm_step(sim.ctx, sc["h"], sc["substeps"], solver, want_stats=False)
    torch.cuda.synchronize()
    return time.perf_counter() - t0


def apply(sims, solve_cap, p2g_chunk):
    for sim in sims:
        native.mpm_set_option(sim.ctx, native.OPT_SOLVE_BLOCKS, int(solve_cap))
        native.mpm_set_option(sim.ctx, native.OPT_P2G_CHUNK, int(p2g_chunk))


def tune_batch(sims, scenes_, solver, caps=(2, 4, 8, 16), chunks=(256, 512), steps=2):
    """Time `steps` steps of every scene per (solve cap, P2G chunk) after one
    untimed step (which records the graphs for the new options); apply and
    return the fastest pair and the table of (cap, chunk, seconds)."""
    table = []
    for chunk in chunks:
        for cap in caps:
            apply(sims, cap, chunk)
            _step_all(sims, scenes_, solver, 1)
            table.append((cap, chunk, _step_all(sims, scenes_, solver, steps)))
    for sim in sims:  # status of the tuning steps is not the measurement's
        native.mpm_synchronize(sim.ctx)
    cap, chunk, _ = min(table, key=lambda r: r[2])
    apply(sims, cap, chunk)
    return (cap, chunk), table


def _time_batch(batch, h, n_substeps, solver, steps):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        batch.step(h, n_substeps, solver)
    torch.cuda.synchronize()
    return time.perf_counter() - t0


def tune_batch_launch(batch, h, n_substeps, solver, steps=2, p2g_chunks=(256, 512, 1024),
                      g2p_threads=(128, 256, 512), grid_particles=(512, 2048, 8192),
                      solve_blocks=(1, 2, 4)):
    """Coordinate descent over the batch's launch options: for each knob in
    turn (P2G chunk, G2P threads, grid particles per block, blocks per
    scene's contact solve), time `steps` steps per value after one untimed
    step (which records the step's graph for the new work lists), keep the
    fastest. Applies and returns the best options (dict option -> value) and
    the table of (options, seconds)."""
    best = {native.BATCH_OPT_P2G_CHUNK: 256, native.BATCH_OPT_G2P_THREADS: 256,
            native.BATCH_OPT_GRID_PARTICLES: 2048, native.BATCH_OPT_SOLVE_BLOCKS: 1}
    table = []
    for knob, values in ((native.BATCH_OPT_P2G_CHUNK, p2g_chunks),
                         (native.BATCH_OPT_G2P_THREADS, g2p_threads),
                         (native.BATCH_OPT_GRID_PARTICLES, grid_particles),
                         (native.BATCH_OPT_SOLVE_BLOCKS, solve_blocks)):
        timed = []
        for v in values:
            cand = dict(best)
            cand[knob] = int(v)
            for opt, val in cand.items():
                batch.set_option(opt, val)
            _time_batch(batch, h, n_substeps, solver, 1)
            t = _time_batch(batch, h, n_substeps, solver, steps)
            timed.append((t, cand))
            table.append((dict(cand), t))
        best = min(timed, key=lambda r: r[0])[1]
    for opt, val in best.items():
        batch.set_option(opt, val)
    batch.synchronize(stats=False)  # status of the tuning steps is not the measurement's
    return best, table


def tune_p2g_form(sim, solver, steps=1, candidates=((0, 256), (0, 1024), (1, 256))):
    """Time the P2G launches of `steps` steps of one context for each
    (form, particles per block) candidate: the gather form (0) at 256 and
    1,024 particles per block, the scatter form (1) at 256 (phase events, so
    that the comparison does not depend on how the rest of the steps, which
    advance the simulation, differ). Apply and return the fastest
    (form, chunk) and the table of ((form, chunk), P2G milliseconds per
    launch). The gather form wins at several particles per cell, the scatter
    form near one."""
    table = []
    native.mpm_set_option(sim.ctx, native.OPT_PROFILE, 1)
    try:
        for form, chunk in candidates:
            native.mpm_set_option(sim.ctx, native.OPT_P2G_FORM, form)
            native.mpm_set_option(sim.ctx, native.OPT_P2G_CHUNK, chunk)
            native.mpm_get_phase_times(sim.ctx, reset=True)
            for _ in range(steps):
                native.mpm_step(sim.ctx, sim.scene["h"], sim.scene["substeps"], solver,
                                want_stats=False)
            ms, n = native.mpm_get_phase_times(sim.ctx, reset=True)
            table.append(((form, chunk), ms["p2g"] / max(n["p2g"], 1)))
    finally:
        native.mpm_set_option(sim.ctx, native.OPT_PROFILE, 0)
    native.mpm_synchronize(sim.ctx)
    form, chunk = min(table, key=lambda r: r[1])[0]
    native.mpm_set_option(sim.ctx, native.OPT_P2G_FORM, form)
    native.mpm_set_option(sim.ctx, native.OPT_P2G_CHUNK, chunk)
    return (form, chunk), table
