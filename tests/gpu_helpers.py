"""Shared helpers of the GPU parity tests: run one substep on the CUDA path
(through the C ABI) and the same substep on the FP64 oracle from the same
float32 state, and compare."""
import numpy as np

import oracle as O
from paper_2503_05046_gb300 import scenes


def particle_arrays(sc):
    """Per-particle mass, rest volume and group index, in id order."""
    mass, vol, mat = [], [], []
    for gi, g in enumerate(sc["groups"]):
        n = len(g["x"])
        V = np.float32(g["vol"])
        mass.append(np.full(n, float(V) * float(np.float32(g["material"]["rho"]))))
        vol.append(np.full(n, float(V)))
        mat.append(np.full(n, gi, np.int32))
    return np.concatenate(mass), np.concatenate(vol), np.concatenate(mat)


def oracle_substep(sc, gpu_state, gpu_bodies, solver, h=None):
    """One oracle substep from the GPU's float32 state and rigid bodies."""
    mass, vol, mat = particle_arrays(sc)
    _, mats = O.from_scene(sc)
    st = O.Sim.state({"x": gpu_state["x"], "v": gpu_state["v"], "C": gpu_state["C"],
                      "F": gpu_state["F"], "mass": mass, "vol": vol, "mat": mat})
    osim = O.Sim(sc["grid"])
    cloth = O.cloth_from_scene(sc)
    if cloth is not None:
        osim.set_cloth(cloth)
    pins = O.pins_from_scene(sc)
    if pins is not None:
        osim.set_pins(*pins)
    bodies = O.bodies_from_scene({"bodies": gpu_bodies})
    imp = np.zeros(6 * max(len(bodies), 1))
    code, info = osim.substep(st, mats, [O.make_body(b) for b in bodies],
                              sc["h"] if h is None else h, solver, imp)
    return st, info, osim, imp[:6 * len(bodies)].reshape(-1, 6), code


def rel_linf(a, b):
    scale = np.max(np.abs(b))
    return float(np.max(np.abs(np.asarray(a, np.float64) - b)) / (scale if scale > 0 else 1.0))


def align_grids(gpu, orc, mass_slack):
    """Grid readbacks (ids, m, v*, v) of the CUDA path and the oracle on the
    union of their node ids. A particle within rounding of a cell boundary has
    two valid stencils that differ in a node of weight ~0, so a node may be
    present on one side only; such nodes must hold at most `mass_slack`.
    Returns both sides' (m, v*, v) on the union (zeros where absent)."""
    ids, m, vs, v = gpu
    oids, om, ovs, ov = orc
    union = np.union1d(ids, oids)
    out = []
    for i_, m_, vs_, v_ in ((ids, m, vs, v), (oids, om, ovs, ov)):
        k = np.searchsorted(union, i_)
        M = np.zeros(len(union))
        VS = np.zeros((len(union), 3))
        V = np.zeros((len(union), 3))
        M[k], VS[k], V[k] = m_, vs_, v_
        out.append((M, VS, V))
    only = np.setxor1d(ids, oids)
    if len(only):
        k = np.searchsorted(union, only)
        assert np.all(out[0][0][k] <= mass_slack) and np.all(out[1][0][k] <= mass_slack), \
            "a node present on one side only holds mass"
    return out[0], out[1]



def wall_nodes(grid, ids):
    """Dirichlet flags of linear node ids: nodes within bc_layers of a face."""
    rx, ry, rz = grid["res"]
    bc = int(grid.get("bc_layers", 3))
    i, j, k = ids % rx, (ids // rx) % ry, ids // (rx * ry)
    return ((i < bc) | (j < bc) | (k < bc) | (i >= rx - bc) | (j >= ry - bc) |
            (k >= rz - bc)).astype(np.int32)


def contact_problem(sc, st0, bodies, grid, contacts, eps_s, lagged_from_gpu=False):
    """The oracle's contact problem (Eq. (7)-(8)) of one substep: contact
    geometry from the start-of-substep particle state `st0` and the frozen
    `bodies`, grid masses and v* read back from the CUDA path, Dirichlet flags
    from the domain walls. With lagged_from_gpu the penetration depths and
    lagged normal impulses are the CUDA path's (after checking them against
    the oracle's geometry to 1e-3), so that a comparison of what is computed
    from the problem does not see their FP32 evaluation. Returns (problem,
    contact frames R [nc, 3, 3], contact positions [nc, 3])."""
    ids, m, vs, _ = grid
    p, b = contacts[0], contacts[1]
    g = sc["grid"]
    dx, origin, res, h = g["dx"], np.asarray(g["origin"], np.float64), g["res"], sc["h"]
    nc = len(p)
    x = st0["x"][p].astype(np.float64)
    vp = st0["v"][p].astype(np.float64)
    nodes = np.zeros((nc, 27), np.int64)
    w = np.zeros((nc, 27))
    R = np.zeros((nc, 3, 3))
    bias = np.zeros((nc, 3))
    phi0, n0 = np.zeros(nc), np.zeros(nc)
    mu, k, d = np.zeros(nc), np.zeros(nc), np.zeros(nc)
    for c in range(nc):
        bd = bodies[b[c]]
        base, _, wt = O.bspline(dx, origin, x[c])
        for cz in range(3):
            for cy in range(3):
                for cx in range(3):
                    q = cx + 3 * cy + 9 * cz
                    nodes[c, q] = (base[0] + cx) + res[0] * ((base[1] + cy) + res[1] * (base[2] + cz))
                    w[c, q] = wt[0, cx] * wt[1, cy] * wt[2, cz]
        phi, nrm = O.sdf(bd, x[c])
        vr = O.body_velocity(bd, x[c])
        R[c] = O.contact_frame(nrm)
        bias[c] = R[c].T @ (-vr)
        phi0[c] = -phi
        n0[c] = O.normal_impulse(phi0[c], bd["k"], bd["d"], h, float(nrm @ (vp[c] - vr)))
        mu[c], k[c], d[c] = bd["mu"], bd["k"], bd["d"]
    if lagged_from_gpu:
        phi0_gpu, n0_gpu = contacts[3].astype(np.float64), contacts[4].astype(np.float64)
        assert np.allclose(phi0_gpu, phi0, rtol=1e-3, atol=1e-7 * dx)
        assert np.allclose(n0_gpu, n0, rtol=1e-3, atol=1e-6 * np.max(np.abs(n0)))
        phi0, n0 = phi0_gpu, n0_gpu
    dof = np.searchsorted(ids, nodes)
    assert np.all(ids[np.minimum(dof, len(ids) - 1)] == nodes), "contact stencil node without mass"
    prob = O.ContactProblem(m.astype(np.float64), vs.astype(np.float64), dof.astype(np.int32), w,
                            R, bias, phi0, n0, mu, k, d, h, eps_s=eps_s,
                            fixed=wall_nodes(g, ids))
    return prob, R, x
