"""Parity at full size, in the launch configuration bench.py times (radix sort
every step, default P2G chunk): the benchmark workload (granular scooping, 1M
sand particles, 128^3 grid) and the mixed-material manipulation workload (4M
particles in 32 elastic and sand objects, 12 rigid bodies, 320 x 184 x 64
grid), each with dense and with block-sparse grid storage, from a state a few
rigid steps into the scene:

1. one substep of P2G + grid update + G2P for every particle and node, against
   the FP64 oracle from the same float32 state (rigid bodies removed, so no
   contact solve is needed and the oracle finishes in seconds);
2. the contact solve of one substep with all bodies, checked by the oracle's
   own gradient of the objective (Eq. (8)-(9)) at the CUDA path's solution:
   the stopping quantity of Alg. 1 must be small, and the depths and lagged
   normal impulses of the registered contacts must match the oracle's
   geometry.
"""
import numpy as np
import pytest

import oracle as O
from paper_2503_05046_gb300 import scenes
from gpu_helpers import align_grids, oracle_substep, particle_arrays, rel_linf

pytestmark = pytest.mark.gpu

N_FULL = 1_000_000
BENCH_SOLVER = dict(eps_r=5e-2, max_iters=1000)
TIGHT_SOLVER = dict(eps_r=1e-6, eps_a=0.0, max_iters=200000, ls_rel_tol=1e-5, ls_max_iters=50)


def _sparse(sc, max_blocks):
    sc["grid"] = dict(sc["grid"], max_blocks=max_blocks)
    return sc


# the sparse variants store only the active blocks (~17,600 of 32,768 and
# ~15,000 of 58,880) in a pool of 20,000
WORKLOADS = {
    "granular_scoop_1M": (lambda: scenes.granular_scoop(n_particles=N_FULL), 2),
    "mixed_manipulation_4M": (lambda: scenes.mixed_manipulation(), 1),
    "granular_scoop_1M_sparse":
        (lambda: _sparse(scenes.granular_scoop(n_particles=N_FULL), 20000), 2),
    "mixed_manipulation_4M_sparse": (lambda: _sparse(scenes.mixed_manipulation(), 20000), 1),
}


@pytest.fixture(scope="module", params=sorted(WORKLOADS))
def warm(request):
    import torch
    assert torch.cuda.is_available()
    from paper_2503_05046_gb300 import native
    make, warm_steps = WORKLOADS[request.param]
    sc = make()
    n = scenes.n_particles(sc)
    sim = native.Sim(sc, max_contacts=2 * n)
    solver = native.solver_params(**BENCH_SOLVER)
    for _ in range(warm_steps):
        sim.step(solver=solver, check=False)
    state, bodies = sim.get_particles(), sim.bodies()
    yield native, sc, sim, state, bodies
    sim.close()


def test_full_size_transfer_parity(warm):
    native, sc, sim, st0, bodies = warm
    sim.set_particles(st0["x"], st0["v"], st0["C"], st0["F"])
    sim.set_bodies([])
    ost, info, osim, _, code = oracle_substep(sc, st0, [], O.solver())
    assert code == O.OK and info.n_contacts == 0
    sim.step(n_substeps=1, solver=native.solver_params(**BENCH_SOLVER))
    out = sim.get_particles()
    assert rel_linf(out["v"], ost["v"]) < 1e-5
    assert np.max(np.abs(out["x"] - ost["x"])) < 1e-4 * sc["grid"]["dx"]
    vmax = np.max(np.abs(ost["v"]))
    assert np.max(np.abs(out["C"] - ost["C"])) < 1e-4 * vmax / sc["grid"]["dx"]
    assert np.max(np.abs(out["F"] - ost["F"])) < 1e-5
    mass_p = min(float(np.float32(g["vol"])) * float(np.float32(g["material"]["rho"]))
                 for g in sc["groups"])
    (m, vs, v), (om, ovs, ov) = align_grids(sim.grid(), osim.last_grid(), 1e-6 * mass_p)
    assert np.all(np.abs(m - om) <= 1e-5 * om + 1e-6 * mass_p)
    mid = om >= 1e-3 * mass_p
    assert rel_linf(vs[mid], ovs[mid]) < 1e-5
    # P2G conserves mass and momentum exactly in exact arithmetic
    mass, _, _ = particle_arrays(sc)
    assert abs(np.sum(m, dtype=np.float64) - mass.sum()) <= 1e-6 * mass.sum()


def test_full_size_contact_solve_optimality(warm):
    native, sc, sim, st0, bodies = warm
    sim.set_particles(st0["x"], st0["v"], st0["C"], st0["F"])
    sim.set_bodies(bodies)
    stats = sim.step(n_substeps=1, solver=native.solver_params(**TIGHT_SOLVER))
    assert stats.contacts_max > 100 and stats.residual_max <= 1e-6
    ids, m, vs, v = sim.grid()
    p, b, gam, phi0_gpu, n0_gpu = sim.contacts()
    g = sc["grid"]
    dx, origin, res, h = g["dx"], np.asarray(g["origin"], np.float64), g["res"], sc["h"]
    nc = len(p)
    # the contact problem of this substep, built by the oracle from the
    # start-of-substep state and the bodies
    x = st0["x"][p].astype(np.float64)
    vp = st0["v"][p].astype(np.float64)
    nodes = np.zeros((nc, 27), np.int64)
    w = np.zeros((nc, 27))
    R = np.zeros((nc, 3, 3))
    bias = np.zeros((nc, 3))
    phi0 = np.zeros(nc)
    n0 = np.zeros(nc)
    mu, k, d = np.zeros(nc), np.zeros(nc), np.zeros(nc)
    for c in range(nc):
        bd = bodies[b[c]]
        base, _, wt = O.bspline(dx, origin, x[c])
        for cz in range(3):
            for cy in range(3):
                for cx in range(3):
                    q = cx + 3 * cy + 9 * cz
                    lin = (base[0] + cx) + res[0] * ((base[1] + cy) + res[1] * (base[2] + cz))
                    nodes[c, q] = lin
                    w[c, q] = wt[0, cx] * wt[1, cy] * wt[2, cz]
        phi, nrm = O.sdf(bd, x[c])
        vr = O.body_velocity(bd, x[c])
        R[c] = O.contact_frame(nrm)
        bias[c] = R[c].T @ (-vr)
        phi0[c] = -phi
        n0[c] = O.normal_impulse(phi0[c], bd["k"], bd["d"], h, float(nrm @ (vp[c] - vr)))
        mu[c], k[c], d[c] = bd["mu"], bd["k"], bd["d"]
    assert np.all(phi0 > 0)
    assert np.allclose(phi0_gpu, phi0, rtol=1e-3, atol=1e-7 * dx)
    assert np.allclose(n0_gpu, n0, rtol=1e-3, atol=1e-6 * np.max(np.abs(n0)))
    dof = np.searchsorted(ids, nodes)
    assert np.all(ids[np.minimum(dof, len(ids) - 1)] == nodes), "contact stencil node without mass"
    prob = O.ContactProblem(m.astype(np.float64), vs.astype(np.float64), dof.astype(np.int32), w, R,
                            bias, phi0, n0, mu, k, d, h, eps_s=1e-4)
    vv = v.astype(np.float64)
    grad = prob.gradient(vv)
    mm = m.astype(np.float64)[:, None]
    jtg = mm * (vv - vs) - grad  # J^T gamma (Eq. (9))
    gn = np.sqrt(np.sum(grad ** 2 / mm))
    scale = max(np.sqrt(np.sum(mm * vv ** 2)), np.sqrt(np.sum(jtg ** 2 / mm)))
    # v is read back in FP32: its rounding (half an ulp per component) moves
    # the gradient by the Hessian times that rounding, which can dominate near
    # stiff sticking contacts; measure that floor with the oracle's gradient
    sign = np.where((np.arange(vv.size).reshape(vv.shape) % 2) == 0, 1.0, -1.0)
    dv = 0.5 * np.spacing(np.abs(v)).astype(np.float64) * sign
    floor = np.sqrt(np.sum((prob.gradient(vv + dv) - grad) ** 2 / mm))
    assert gn <= 1e-5 * scale + 2.0 * floor, \
        "optimality residual %.3e (FP32 floor %.3e)" % (gn / scale, floor / scale)
