"""Measured choice of launch options for many contexts stepped side by side.

Independent scenes advance concurrently, each on its own stream replaying its
step's CUDA graph (mpm_step with graphs on). How well they share the GPU
depends on two launch options: the cap on the SMs one context's cooperative
contact solve occupies (MPM_OPT_SOLVE_BLOCKS) and the particles per P2G thread
block (MPM_OPT_P2G_CHUNK). `tune_batch` times a few steps of the whole batch
under each candidate pair and applies the fastest; the scenes advance while
it measures (the timed steps are ordinary steps of the simulation).
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
