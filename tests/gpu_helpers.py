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

