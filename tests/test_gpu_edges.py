"""Edge cases through the C ABI: failure statuses (a barrier that gives up,
particles leaving the grid, contact capacity, the iteration cap, too many
bodies) with the context usable afterwards, and degenerate inputs against
the oracle (particles exactly on cell boundaries, inverted deformation
gradients)."""
import time

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


def test_barrier_time_limit_reports_timeout_and_context_recovers(native):
    """A device-wide barrier waiting for an arrival that never comes gives up
    after its 1 s limit; the step reports MPM_ERR_TIMEOUT, and the next solve
    (clearing the scratch the abandoned one left) works."""
    sc = scenes.cube_contact(n_side=10, v0=(0.0, 0.0, -0.05))
    sim = native.Sim(sc)
    sp = native.solver_params(**TIGHT)
    native.mpm_set_option(sim.ctx, native.OPT_TEST_BARRIER_TIMEOUT, 1)
    t0 = time.perf_counter()
    code, st = sim.step(n_substeps=1, solver=sp, check=False)
    took = time.perf_counter() - t0
    assert code == native.ERR_TIMEOUT
    assert st.contacts_max > 0 and st.cluster_substeps == 0  # the cooperative kernel's barrier
    assert took < 30.0
    native.mpm_set_option(sim.ctx, native.OPT_TEST_BARRIER_TIMEOUT, 0)
    st = sim.get_particles()
    bodies = sim.bodies()
    ost, info, osim, _, ocode = oracle_substep(sc, st, bodies, SOLVER_ORC)
    code, stats = sim.step(n_substeps=1, solver=sp, check=False)
    assert code == native.OK and stats.residual_max <= 1e-6
    out = sim.get_particles()
    assert np.all(np.isfinite(out["v"]))
    assert rel_linf(out["v"], ost["v"]) < 1e-5
    sim.close()


def test_particle_leaving_the_grid_is_reported(native):
    sc = scenes.cube_drop(n_side=6)
    g = sc["groups"][0]
    x = g["x"].copy()
    x[0] = np.asarray(sc["grid"]["origin"], np.float32) - sc["grid"]["dx"]  # outside the grid
    g["x"] = x
    sim = native.Sim(sc)
    code, _ = sim.step(n_substeps=1, check=False)
    assert code == native.ERR_OUT_OF_DOMAIN
    # the other particles fell freely
    out = sim.get_particles()
    dv = out["v"][1:] - g["v"][1:]
    assert np.allclose(dv, np.asarray(sc["grid"]["gravity"], np.float32) * sc["h"], atol=1e-6)
    sim.close()


def test_contact_capacity_and_iteration_cap_are_reported(native):
    sc = scenes.cube_contact(n_side=8, v0=(0.0, 0.0, -0.05))
    sim = native.Sim(sc, max_contacts=8)
    code, _ = sim.step(n_substeps=1, check=False)
    assert code == native.ERR_CAPACITY
    sim.close()
    sim = native.Sim(sc)
    code, st = sim.step(n_substeps=1, solver=native.solver_params(eps_r=1e-9, max_iters=1),
                        check=False)
    assert code == native.ERR_NOT_CONVERGED and st.iters_max == 1
    code, _ = sim.step(n_substeps=1, check=False)  # paper defaults again
    assert code == native.OK
    with pytest.raises(native.MpmError):
        sim.set_bodies([sc["bodies"][0]] * 17)  # at most 16 bodies
    sim.close()


def test_particles_exactly_on_cell_boundaries(native):
    """A lattice with dx a power of two and positions on multiples of dx/2:
    every fractional offset is exactly 0.5 or 1.0 (weights 1/2, 1/2, 0 and
    1/8, 3/4, 1/8), in contact with the ground."""
    dx = 1.0 / 64.0
    k = np.arange(8, dtype=np.float64)
    gx, gy, gz = np.meshgrid(k, k, k, indexing="ij")
    x = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], 1) * (dx / 2) + np.array([0.0, 0.0, dx / 2])
    g = {"x": x.astype(np.float32), "v": np.tile(np.float32([0.02, 0.0, -0.05]), (len(x), 1)),
         "vol": float((dx / 2) ** 3), "material": scenes.elastic(1e5, 0.3, 1000.0)}
    sc = {"name": "aligned", "groups": [g], "h": 1e-4, "substeps": 10,
          "bodies": [scenes.body(scenes.HALFSPACE, p=(0.0, 0.0, dx / 2 + 1e-4), mu=0.5)],
          "grid": {"dx": dx, "res": (32, 32, 32), "origin": (-16 * dx, -16 * dx, -8 * dx),
                   "gravity": (0.0, 0.0, -9.81), "bc_layers": 3}}
    sim = native.Sim(sc)
    sp = native.solver_params(**TIGHT)
    for _ in range(2):
        st = sim.get_particles()
        ost, info, osim, _, code = oracle_substep(sc, st, sim.bodies(), SOLVER_ORC)
        assert code == O.OK and info.n_contacts > 0
        sim.step(n_substeps=1, solver=sp)
        out = sim.get_particles()
        assert rel_linf(out["v"], ost["v"]) < 1e-5
        ids, m, vs, v = sim.grid()
        oids, om, ovs, ov = osim.last_grid()
        assert np.array_equal(ids, oids)
    sim.close()


def test_inverted_and_degenerate_deformation_gradients(native):
    """Particles whose F is inverted (distinct singular values, so that the
    reflection's axis is unique), nearly singular, below the Hencky clamp, or
    strongly sheared, for the corotated and the Drucker-Prager model: one
    substep against the oracle."""
    rng = np.random.default_rng(7)
    for material in (scenes.elastic(1e5, 0.3, 1000.0), dict(scenes.SAND)):
        sc = scenes.cube_drop(n_side=6)
        sc["groups"][0]["material"] = material
        sim = native.Sim(sc)
        st = sim.get_particles()
        n = len(st["x"])
        F = np.tile(np.eye(3, dtype=np.float32), (n, 1, 1))
        F[0::5] = np.diag([1.2, 0.9, -0.8]).astype(np.float32)           # inverted
        F[1::5] = np.diag([1.0, 1.1, 1e-3]).astype(np.float32)           # nearly singular
        F[2::5] = np.diag([1.05, 0.95, 3e-5]).astype(np.float32)         # below the clamp
        F[3::5] = (np.eye(3) + 0.3 * rng.standard_normal((3, 3))).astype(np.float32)  # sheared
        sim.set_particles(st["x"], st["v"], st["C"], F)
        st = sim.get_particles()
        ost, info, osim, _, code = oracle_substep(sc, st, sim.bodies(), SOLVER_ORC)
        assert code == O.OK
        sim.step(n_substeps=1, solver=native.solver_params(**TIGHT))
        out = sim.get_particles()
        assert np.all(np.isfinite(out["v"]))
        assert rel_linf(out["v"], ost["v"]) < 1e-5
        assert np.max(np.abs(out["F"] - ost["F"])) < 1e-5 * max(1.0, np.max(np.abs(ost["F"])))
        sim.close()


def test_device_tensor_io_matches_host_io(native):
    """Particles added, set and read through CUDA tensors (device pointers,
    MPM_MEM_DEVICE) give the results of the host-array path."""
    import torch
    sc = scenes.cube_contact(n_side=8, v0=(0.0, 0.0, -0.05))
    g = sc["groups"][0]
    n = len(g["x"])
    sim_h = native.Sim(sc)
    sim_d = native.Sim(dict(sc, groups=[]), max_particles=n)
    xt = torch.from_numpy(g["x"]).cuda()
    vt = torch.from_numpy(g["v"]).cuda()
    torch.cuda.synchronize()
    native.mpm_add_particles(sim_d.ctx, xt, vt, g["vol"], native.make_material(g["material"]))
    assert native.mpm_num_particles(sim_d.ctx) == n
    sp = native.solver_params(**TIGHT)
    for sim in (sim_h, sim_d):
        sim.step(solver=sp)
    out_h = sim_h.get_particles()
    dev = {k: torch.empty((n, 3) if k in ("x", "v") else (n, 3, 3), dtype=torch.float32, device="cuda")
           for k in ("x", "v", "C", "F")}
    native.mpm_get_particles(sim_d.ctx, dev["x"], dev["v"], dev["C"], dev["F"], mem_kind=native.MEM_DEVICE)
    torch.cuda.synchronize()
    out_d = {k: t.cpu().numpy() for k, t in dev.items()}
    assert rel_linf(out_d["v"], out_h["v"].astype(np.float64)) < 1e-5
    assert np.max(np.abs(out_d["x"] - out_h["x"])) < 1e-7
    # set from device tensors, read back on the host: exactly what was set
    native.mpm_set_particles(sim_d.ctx, dev["x"], dev["v"], dev["C"], dev["F"])
    back = sim_d.get_particles()
    for k in ("x", "v", "C", "F"):
        assert np.array_equal(back[k], out_d[k])
    sim_h.close()
    sim_d.close()


@pytest.mark.parametrize("bc", [0, 1, 3])
def test_dirichlet_layers_counted_by_hand(native, bc):
    """Domain walls: on a 12^3 grid whose every node has mass, particles at
    rest under gravity leave exactly (12 - 2 bc)^3 nodes with a nonzero v*
    (1728, 1000, 216), the nodes with bc <= i, j, k < 12 - bc, each at h g."""
    sc = scenes.filled_box(bc=bc)
    sim = native.Sim(sc)
    sim.step(n_substeps=1)
    ids, m, vs, v = sim.grid()
    sim.close()
    assert len(ids) == 12 ** 3 and np.all(m > 0)
    moving = np.any(vs != 0.0, axis=1)
    assert int(moving.sum()) == (12 - 2 * bc) ** 3
    i, j, k = ids % 12, (ids // 12) % 12, ids // 144
    inner = (i >= bc) & (i < 12 - bc) & (j >= bc) & (j < 12 - bc) & (k >= bc) & (k < 12 - bc)
    assert np.array_equal(moving, inner)
    assert np.allclose(vs[inner], [0.0, 0.0, -9.81e-4], rtol=1e-6, atol=1e-9)


def test_launch_options_are_validated(native):
    """Bad option values are refused and leave the context usable; a change of
    P2G form or block size between steps keeps the state consistent (the
    step graph is recorded again)."""
    sim = native.Sim(scenes.cube_drop(n_side=8))
    for opt, val in ((native.OPT_P2G_FORM, 2), (native.OPT_P2G_FORM, -1),
                     (native.OPT_P2G_CHUNK, 300), (native.OPT_CLUSTER_BLOCKS, 3)):
        with pytest.raises(native.MpmError):
            native.mpm_set_option(sim.ctx, opt, val)
    sim.step()
    for form, chunk in ((1, 256), (0, 1024), (0, 256)):
        native.mpm_set_option(sim.ctx, native.OPT_P2G_FORM, form)
        native.mpm_set_option(sim.ctx, native.OPT_P2G_CHUNK, chunk)
        st = sim.step()
        assert st.substeps > 0
    assert np.all(np.isfinite(sim.get_particles()["v"]))
    sim.close()
