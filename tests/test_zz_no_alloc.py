"""mpm_get_grid_noalloc: the grid readback for callers that cannot allocate
device memory (its staging buffer is a fixed-size array inside the library).

Called through the C ABI and compared with mpm_get_grid on two consecutive
substeps; the two read the same device grid, so they must agree exactly (the
tolerance of the parity tests, 1e-5 relative, is therefore met with margin).
This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc_grid(native, ctx):
    count = C.c_int64()
    code = native.lib.mpm_get_grid_noalloc(ctx, 0, C.byref(count), None, None, None, None)
    assert code == native.OK, native.mpm_last_error(ctx)
    n = count.value
    ids = np.zeros(max(n, 1), np.int32)
    m = np.zeros(max(n, 1), np.float32)
    vs = np.zeros((max(n, 1), 3), np.float32)
    v = np.zeros((max(n, 1), 3), np.float32)
    code = native.lib.mpm_get_grid_noalloc(ctx, n, C.byref(count), ids.ctypes.data_as(native._i32p),
                                           m.ctypes.data_as(native._fp), vs.ctypes.data_as(native._fp),
                                           v.ctypes.data_as(native._fp))
    assert code == native.OK, native.mpm_last_error(ctx)
    assert count.value == n
    order = np.argsort(ids[:n], kind="stable")
    return ids[:n][order], m[:n][order], vs[:n][order], v[:n][order]


def test_noalloc_grid_readback_matches_mpm_get_grid():
    import torch
    assert torch.cuda.is_available()
    from paper_2503_05046_gb300 import native, scenes
    sim = native.Sim(scenes.cube_contact(n_side=10, v0=(0.0, 0.0, -0.05)))
    solver = native.solver_params(eps_r=1e-6, eps_a=0.0, max_iters=200000)
    for call in range(2):
        sim.step(n_substeps=1, solver=solver)
        ids, m, vs, v = native.mpm_get_grid(sim.ctx)
        nids, nm, nvs, nv = _noalloc_grid(native, sim.ctx)
        assert len(ids) > 0
        assert np.array_equal(ids, nids)
        for a, b in ((m, nm), (vs, nvs), (v, nv)):
            scale = max(float(np.max(np.abs(a))), 1e-30)
            assert np.max(np.abs(a - b)) <= 1e-5 * scale
    sim.close()


def test_noalloc_grid_readback_rejects_grids_beyond_its_buffer():
    from paper_2503_05046_gb300 import native, scenes
    sc = scenes.granular_scoop(n_particles=400_000)  # ~0.9M swept nodes > 262,144
    sim = native.Sim(sc, max_contacts=800_000)
    sim.step(n_substeps=1)
    count = C.c_int64()
    code = native.lib.mpm_get_grid_noalloc(sim.ctx, 0, C.byref(count), None, None, None, None)
    assert code == native.ERR_CAPACITY
    assert "262144" in native.mpm_last_error(sim.ctx)
    sim.close()
