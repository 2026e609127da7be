"""Block-sparse grid storage (mpm_grid_spec.max_blocks): only the 4^3 blocks a
substep's particle stencils touch get nodes, from a pool, so memory follows
the active blocks rather than the domain.

- the parity cases of the dense grid (per-substep comparison with the FP64
  oracle: particles, grid, contacts, impulses) hold with a pool a little
  larger than the scenes' active blocks, including the split line search;
- a 512^3 domain with a pool of 5% of its blocks takes memory in proportion to
  the pool (a dense 512^3 grid would take ~20 GB), and an 8k-particle scene
  placed in it steps like the same scene in its own small dense domain;
- a substep touching more blocks than the pool reports MPM_ERR_CAPACITY.
The full-size workloads run sparse in tests/test_gpu_fullsize.py."""
import numpy as np
import pytest

from paper_2503_05046_gb300 import scenes
from gpu_helpers import rel_linf
from test_gpu_parity import run_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    import torch
    assert torch.cuda.is_available()
    from paper_2503_05046_gb300 import native as N
    return N


def n_blocks(grid):
    return int(np.prod([r // 4 for r in grid["res"]]))


def sparse(sc, max_blocks):
    sc = dict(sc)
    sc["grid"] = dict(sc["grid"], max_blocks=int(max_blocks))
    assert 0 < max_blocks < n_blocks(sc["grid"])
    return sc


def test_sparse_normal_contact_parity(native):
    # 12 active blocks of 4,096; a pool of 32
    sc = sparse(scenes.cube_contact(n_side=10, v0=(0.0, 0.0, -0.05)), 32)
    rep = run_parity(native, sc, n_sub=3)
    assert all(r[1] > 0 for r in rep)


def test_sparse_split_line_search_parity(native):
    # 242 active blocks of 845; more than 4,096 contacts, split line search
    sc = sparse(scenes.sand_slab(), 300)
    rep = run_parity(native, sc, n_sub=2, options=((native.OPT_CLUSTER_CONTACTS, 4096),))
    assert all(r[1] > 4096 and r[5] == 1 for r in rep), rep


def test_sparse_pool_overflow_is_reported(native):
    sc = sparse(scenes.cube_contact(n_side=10, v0=(0.0, 0.0, -0.05)), 4)
    sim = native.Sim(sc)
    code, st = sim.step(n_substeps=1, check=False)
    assert code == native.ERR_CAPACITY, native.STATUS_NAMES[code]
    sim.close()


def test_sparse_512_domain_memory_and_results(native):
    import torch
    small = scenes.cube_contact(n_side=20, v0=(0.0, 0.0, -0.05))
    g = small["grid"]
    shift = 224  # nodes: the scene sits mid-domain, far from the walls
    big_grid = dict(g, res=(512, 512, 512),
                    origin=tuple(o - shift * g["dx"] for o in g["origin"]))
    nb = n_blocks(big_grid)
    pool = int(0.05 * nb)  # 5% of the 2,097,152 blocks
    big = dict(small, grid=dict(big_grid, max_blocks=pool))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    sim_big = native.Sim(big)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    used = free0 - free1
    print("512^3 domain, pool of %d blocks: %.3f GB on the device" % (pool, used / 1e9))
    # ~150 B per storage node, 9 B per block of the domain, the particles
    dense_estimate = 150.0 * 512 ** 3
    assert used < 160.0 * (pool + 1) * 64 + 12.0 * nb + 64 * 2 ** 20, used
    assert used < 0.06 * dense_estimate, used
    sim_small = native.Sim(small)
    solver = native.solver_params(eps_r=1e-6, eps_a=0.0, max_iters=200000, ls_rel_tol=1e-5)
    for _ in range(2):
        st_b = sim_big.step(solver=solver)
        st_s = sim_small.step(solver=solver)
    assert st_b.active_blocks_max == st_s.active_blocks_max <= pool
    assert st_b.contacts_max == st_s.contacts_max > 0
    a, b = sim_big.get_particles(), sim_small.get_particles()
    # the same arithmetic up to the rounding of the shifted cell coordinates
    assert rel_linf(a["v"], b["v"].astype(np.float64)) < 1e-5
    assert np.max(np.abs(a["x"] - b["x"])) < 1e-6
    assert np.max(np.abs(a["F"] - b["F"])) < 1e-5
    ib, ob = sim_big.impulses(), sim_small.impulses()
    assert np.max(np.abs(ib - ob)) <= 1e-4 * np.max(np.abs(ob)) + 1e-12
    sim_big.close()
    sim_small.close()
