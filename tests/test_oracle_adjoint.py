"""Pins of the oracle's contact-solve adjoint (implicit differentiation of the
optimality condition of Eq. (8)): directional derivatives of the solve map
v(v*, b, mu) by central finite differences of tightly converged dense Newton
solves, with and without Dirichlet DoFs, against dL/dv*, dL/db and dL/dmu."""
import numpy as np
import pytest

import oracle as O

H = 1e-4
K = 1e4
D = 10.0
S_TIGHT = O.solver(eps_r=1e-14, eps_a=0.0, max_iters=200)


def _frame(rng):
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    return O.contact_frame(n, 0.0)


def _arrays(seed, n_nodes=12, n_contacts=5, fixed_frac=0.0):
    rng = np.random.default_rng(seed)
    a = dict(m=rng.uniform(0.5e-4, 2e-4, n_nodes), vstar=rng.normal(scale=0.5, size=(n_nodes, 3)))
    nodes = np.zeros((n_contacts, 27), np.int32)
    w = np.zeros((n_contacts, 27))
    for p in range(n_contacts):
        nodes[p] = rng.integers(0, n_nodes, 27)
        ww = rng.uniform(0, 1, 27)
        w[p] = ww / ww.sum()
    a.update(nodes=nodes, w=w, R=np.array([_frame(rng) for _ in range(n_contacts)]).reshape(n_contacts, 3, 3),
             b=rng.normal(scale=0.2, size=(n_contacts, 3)),
             phi0=rng.uniform(1e-7, 5e-6, n_contacts), mu=np.full(n_contacts, 0.5),
             fixed=(rng.uniform(size=n_nodes) < fixed_frac).astype(np.int32))
    a["n0"] = np.array([O.normal_impulse(a["phi0"][p], K, D, H, rng.normal(scale=0.2))
                        for p in range(n_contacts)])
    return a


def _problem(a):
    nc = len(a["phi0"])
    return O.ContactProblem(a["m"], a["vstar"], a["nodes"], a["w"], a["R"], a["b"], a["phi0"],
                            a["n0"], a["mu"], np.full(nc, K), np.full(nc, D), H, 1e-4, a["fixed"])


def _solve(a):
    v, _, info, st = _problem(a).solve_dense_newton(S_TIGHT)
    assert st == O.OK
    return v


@pytest.mark.parametrize("seed,fixed_frac", [(0, 0.0), (1, 0.0), (2, 0.25), (3, 0.25)])
def test_adjoint_matches_central_differences(seed, fixed_frac):
    a = _arrays(seed, fixed_frac=fixed_frac)
    v = _solve(a)
    rng = np.random.default_rng(100 + seed)
    vbar = rng.normal(size=v.shape)
    vsb, bb, mb, st = _problem(a).adjoint(v, vbar)
    assert st == O.OK

    def fd(key, delta, eps):
        ap, am = dict(a), dict(a)
        ap[key] = a[key] + eps * delta
        am[key] = a[key] - eps * delta
        return float(np.sum(vbar * (_solve(ap) - _solve(am))) / (2 * eps))

    dv = rng.normal(size=a["vstar"].shape)
    assert fd("vstar", dv, 1e-6) == pytest.approx(float(np.sum(vsb * dv)), rel=1e-4, abs=1e-9)
    db = rng.normal(size=a["b"].shape)
    assert fd("b", db, 1e-6) == pytest.approx(float(np.sum(bb * db)), rel=1e-4, abs=1e-9)
    dmu = rng.uniform(0.5, 1.0, size=a["mu"].shape)
    assert fd("mu", dmu, 1e-6) == pytest.approx(float(np.sum(mb * dmu)), rel=1e-4, abs=1e-9)


def test_adjoint_without_contacts_is_identity():
    a = _arrays(5, n_contacts=0)
    v = a["vstar"].copy()
    vbar = np.random.default_rng(6).normal(size=v.shape)
    vsb, bb, mb, st = _problem(a).adjoint(v, vbar)
    assert st == O.OK and np.allclose(vsb, vbar, rtol=0, atol=1e-15)
