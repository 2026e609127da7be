"""Parity of the contact-solve adjoint (mpm_contact_adjoint) with the FP64
oracle's (implicit differentiation of the optimality condition of Eq. (8)):
one substep of the touch-down cube (ground and a moving sphere, sliding and
sticking contacts) is solved tightly on the GPU, the oracle rebuilds the same
contact problem from the start-of-substep state, and both differentiate it at
the GPU's solution for the same random dL/dv."""
import numpy as np
import pytest

import oracle as O
from paper_2503_05046_gb300 import scenes
from gpu_helpers import contact_problem

pytestmark = pytest.mark.gpu

TIGHT = dict(eps_r=1e-7, eps_a=0.0, max_iters=100000, ls_rel_tol=1e-6, ls_max_iters=60)


def _scene(kind):
    sc = scenes.cube_contact()
    # the kinematic sphere pressed 1 mm into the cube's +x face, spinning, so
    # that a moving body with a moment arm has contacts too
    x_face = max(float(np.max(g["x"][:, 0])) for g in sc["groups"])
    sc["bodies"][1]["p"] = np.array([x_face + 0.05 - 1e-3, 0.0, 0.0225])
    sc["bodies"][1]["omega"] = np.array([0.0, 0.0, 2.0])
    if kind == "wall":
        # the ground 3.25 cells above the domain floor: the bottom particles'
        # stencils reach the Dirichlet layers (3 nodes), which enter J but
        # keep v = v*
        sc["grid"] = dict(sc["grid"], origin=(-0.32, -0.32, -0.03))
    return sc


@pytest.fixture(scope="module", params=["open", "wall"])
def solved(request):
    import torch
    assert torch.cuda.is_available()
    from paper_2503_05046_gb300 import native
    sc = _scene(request.param)
    sim = native.Sim(sc)
    solver = native.solver_params(**TIGHT)
    sim.step(n_substeps=1, solver=solver)  # settle the first touch-down substep
    st0, bodies = sim.get_particles(), sim.bodies()
    stats = sim.step(n_substeps=1, solver=solver)
    # both sides differentiate at the CUDA path's own solution, which needs to
    # be a near-minimiser only (stiff sphere contacts stop FP32 progress early)
    assert stats.contacts_max > 50 and stats.residual_max <= 1e-4
    grid, contacts = sim.grid(), sim.contacts()
    prob, R, xc = contact_problem(sc, st0, bodies, grid, contacts, solver.eps_s,
                                  lagged_from_gpu=True)
    assert set(np.unique(contacts[1])) == {0, 1}
    touched = np.unique(prob.nodes[prob.nodes >= 0])
    assert prob.fixed[touched].any() == (request.param == "wall")
    yield native, sc, sim, bodies, grid, contacts, prob, R, xc
    sim.close()


U32 = 2.0 ** -24  # FP32 unit roundoff


def _perturbed(prob, R, rng):
    """The oracle's problem with the rounding of an FP32 evaluation: every
    stencil weight, contact frame (a rotation by up to U32 rad about each
    axis) and world-frame bias component moved by a relative U32, random signs."""
    nc = prob.nc
    sg = lambda shape: rng.choice([-1.0, 1.0], size=shape)
    w = prob.w * (1.0 + U32 * sg(prob.w.shape))
    th = U32 * sg((nc, 3))
    K = np.zeros((nc, 3, 3))
    K[:, 0, 1], K[:, 0, 2], K[:, 1, 2] = -th[:, 2], th[:, 1], -th[:, 0]
    K -= K.transpose(0, 2, 1)
    Rp = R + R @ K
    bw = np.einsum("cij,cj->ci", R, prob.b.reshape(nc, 3))
    bw = bw * (1.0 + U32 * sg(bw.shape))
    b = np.einsum("cji,cj->ci", Rp, bw)
    return O.ContactProblem(prob.m, prob.vstar.reshape(-1, 3), prob.nodes, w, Rp, b, prob.phi0,
                            prob.n0, prob.mu, prob.k, prob.d, prob.s.h, eps_s=prob.s.eps_s,
                            fixed=prob.fixed), Rp


def _oracle_with_floor(prob, R, v, vbar, patterns=4):
    """The oracle's adjoint at v, and per output the largest change of it over
    `patterns` random FP32-rounding perturbations of the problem (_perturbed)
    and of v (half an FP32 ulp per component): the Hessian of the contact
    terms, and the friction direction u_t / s in particular near sticking
    (s ~ eps_s), is only determined to that precision by an FP32 evaluation."""
    vsb, bb, mb, st = prob.adjoint(v, vbar)
    vr = -np.einsum("cij,cj->ci", R, bb)  # dL/dv_r(x_p) = -R dL/db
    rng = np.random.default_rng(1)
    fl = [np.zeros_like(vsb), np.zeros_like(vr), np.zeros_like(mb)]
    half_ulp = 0.5 * np.spacing(np.abs(v.astype(np.float32))).astype(np.float64)
    for _ in range(patterns):
        P2, Rp = _perturbed(prob, R, rng)
        a, b, c, _ = P2.adjoint(v + half_ulp * rng.choice([-1.0, 1.0], size=v.shape), vbar)
        vr2 = -np.einsum("cij,cj->ci", Rp, b)
        for k, (x, y) in enumerate(((a, vsb), (vr2, vr), (c, mb))):
            fl[k] = np.maximum(fl[k], np.abs(x - y))
    return (vsb, vr, mb, st), fl


def test_adjoint_matches_oracle(solved):
    native, sc, sim, bodies, (ids, m, vs, v), contacts, prob, R, xc = solved
    rng = np.random.default_rng(7)
    vbar = rng.normal(size=v.shape).astype(np.float32)
    (vsb_o, vr_bar_o, mb_o, st), fl = _oracle_with_floor(prob, R, v.astype(np.float64),
                                                          vbar.astype(np.float64))
    assert st == O.OK
    vsb, cbar, bbar, ast, code = sim.contact_adjoint(ids, vbar, eps_r=1e-6, max_iters=5000)
    assert code == native.OK and ast.residual <= 1e-6 and ast.contacts == len(contacts[0])
    # dL/dv* on every node (identity away from the contacts' stencils)
    for name, got, ref, f in (("dL/dv*", vsb, vsb_o, fl[0]), ("dL/dv_r", cbar[:, :3], vr_bar_o, fl[1]),
                              ("dL/dmu", cbar[:, 3], mb_o, fl[2])):
        scale = np.max(np.abs(ref))
        assert scale > 0.0, name
        err = np.abs(got - ref)
        assert np.all(err <= 1e-4 * scale + 2.0 * f), "%s max err %.3e of %.3e (floor %.3e)" % (
            name, err.max(), scale, f[np.argmax(err)])
    # per body: sums over its contacts (moments about the body origin)
    b = contacts[1]
    for k, bd in enumerate(bodies):
        sel = b == k
        if not sel.any():
            continue
        r = xc[sel] - np.asarray(bd["p"], np.float64)
        ref = np.concatenate([vr_bar_o[sel].sum(0), np.cross(r, vr_bar_o[sel]).sum(0),
                              [mb_o[sel].sum()]])
        f = np.concatenate([fl[1][sel].sum(0), (np.abs(r).sum(1)[:, None] * fl[1][sel]).sum(0),
                            [fl[2][sel].sum()]])
        assert np.all(np.abs(bbar[k] - ref) <= 1e-4 * np.abs(ref).max() + 2.0 * f), (k, bbar[k], ref)


def test_adjoint_identity_away_from_contacts_and_state_untouched(solved):
    native, sc, sim, bodies, (ids, m, vs, v), contacts, prob, R, xc = solved
    in_stencil = np.zeros(len(ids), bool)
    in_stencil[np.unique(prob.nodes[prob.nodes >= 0])] = True
    rng = np.random.default_rng(8)
    vbar = rng.normal(size=v.shape).astype(np.float32)
    before = sim.grid()
    vsb, _, _, _, code = sim.contact_adjoint(ids, vbar, eps_r=1e-6, max_iters=5000)
    assert code == native.OK
    assert np.array_equal(vsb[~in_stencil], vbar[~in_stencil])
    after = sim.grid()
    for a, b_ in zip(before, after):
        assert np.array_equal(a, b_)
    # a subset of the nodes: unlisted nodes count as vbar = 0
    sub = np.flatnonzero(in_stencil)[::3]
    vsb_sub, _, _, _, code = sim.contact_adjoint(ids[sub], vbar[sub], eps_r=1e-6, max_iters=5000)
    vbar0 = np.zeros_like(vbar)
    vbar0[sub] = vbar[sub]
    vsb_o, _, _, st = prob.adjoint(v.astype(np.float64), vbar0.astype(np.float64))
    assert code == native.OK and st == O.OK
    scale = np.max(np.abs(vsb_o))
    assert np.max(np.abs(vsb_sub - vsb_o[sub])) <= 1e-3 * scale


def test_adjoint_device_buffers_match_host(solved):
    import torch
    native, sc, sim, bodies, (ids, m, vs, v), contacts, prob, R, xc = solved
    rng = np.random.default_rng(9)
    vbar = rng.normal(size=v.shape).astype(np.float32)
    h = sim.contact_adjoint(ids, vbar, eps_r=1e-6, max_iters=5000)
    d = sim.contact_adjoint(torch.from_numpy(ids).cuda(), torch.from_numpy(vbar).cuda(), eps_r=1e-6,
                            max_iters=5000)
    assert h[4] == native.OK and d[4] == native.OK
    for a, b_ in zip(h[:2], d[:2]):
        b_ = b_.cpu().numpy()
        assert np.allclose(a, b_, rtol=1e-4, atol=1e-5 * np.max(np.abs(a)))
    # the per-body sums cancel strongly (contacts pull both ways) and the
    # solve's atomic accumulation order varies between runs: bound their
    # difference by the rounding of the summed magnitudes
    scale = np.abs(h[1][:, :3]).sum()
    assert np.all(np.abs(h[2] - d[2].cpu().numpy()) <= 1e-4 * scale)


def test_adjoint_errors(solved):
    native, sc, sim, bodies, (ids, m, vs, v), contacts, prob, R, xc = solved
    res = sc["grid"]["res"]
    bad = np.array([res[0] * res[1] * res[2]], np.int32)
    with pytest.raises(native.MpmError) as e:
        sim.contact_adjoint(bad, np.zeros((1, 3), np.float32))
    assert e.value.code == native.ERR_INVALID_ARG
    # not converged within one iteration: reported, the context stays usable
    vbar = np.ones(v.shape, np.float32)
    _, _, _, st, code = sim.contact_adjoint(ids, vbar, eps_r=1e-12, max_iters=1, check=False)
    assert code == native.ERR_NOT_CONVERGED and st.iters == 1
    stats = sim.step(n_substeps=1, solver=native.solver_params(**TIGHT))
    assert stats.residual_max <= 1e-4
    fresh = native.Sim(scenes.cube_contact())
    with pytest.raises(native.MpmError) as e:
        fresh.contact_adjoint(ids[:1], np.zeros((1, 3), np.float32))
    assert e.value.code == native.ERR_STATE
    fresh.close()
