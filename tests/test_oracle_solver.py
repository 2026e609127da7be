"""Pins of the oracle's contact solve (Eq. (7)-(10), Alg. 1) against closed
forms, a dense exact Newton solve, first-order optimality with an explicitly
assembled Jacobian, invariance to the tangent basis and the monotone decrease
the paper's convergence proof (Appendix) guarantees."""
import numpy as np
import pytest

import oracle as O

H = 1e-4
K = 1e4
D = 10.0


def _frame(rng):
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    return O.contact_frame(n, 0.0)


def random_problem(seed, n_nodes=12, n_contacts=5, fixed_frac=0.0, mu=0.5):
    rng = np.random.default_rng(seed)
    m = rng.uniform(0.5e-4, 2e-4, n_nodes)
    vstar = rng.normal(scale=0.5, size=(n_nodes, 3))
    nodes = np.zeros((n_contacts, 27), np.int32)
    w = np.zeros((n_contacts, 27))
    for p in range(n_contacts):
        nodes[p] = rng.integers(0, n_nodes, 27)
        ww = rng.uniform(0, 1, 27)
        w[p] = ww / ww.sum()
    R = np.stack([_frame(rng) for _ in range(n_contacts)])
    b = rng.normal(scale=0.2, size=(n_contacts, 3))
    phi0 = rng.uniform(1e-7, 5e-6, n_contacts)  # micrometre penetrations, as under gravity loads
    n0 = np.array([O.normal_impulse(phi0[p], K, D, H, rng.normal(scale=0.2)) for p in range(n_contacts)])
    fixed = (rng.uniform(size=n_nodes) < fixed_frac).astype(np.int32)
    return O.ContactProblem(m, vstar, nodes, w, R, b, phi0, n0, np.full(n_contacts, mu),
                            np.full(n_contacts, K), np.full(n_contacts, D), H, 1e-4, fixed)


def J_matrix(P):
    """Dense contact Jacobian, rows = contact-frame components."""
    J = np.zeros((3 * P.nc, 3 * P.n))
    for p in range(P.nc):
        R = P.R[9 * p:9 * p + 9].reshape(3, 3)
        for s in range(27):
            i = P.nodes[p, s]
            if i >= 0:
                J[3 * p:3 * p + 3, 3 * i:3 * i + 3] += P.w[p, s] * R.T
    return J


def test_no_contacts_returns_free_motion():
    rng = np.random.default_rng(0)
    m = rng.uniform(1e-4, 2e-4, 5)
    vs = rng.normal(size=(5, 3))
    P = O.ContactProblem(m, vs, np.zeros((0, 27)), np.zeros((0, 27)), np.zeros((0, 3, 3)),
                         np.zeros((0, 3)), [], [], [], [], [], H)
    v, gam, info, st = P.solve_qn(O.solver(eps_r=1e-8, eps_a=0.0))
    assert st == O.OK and info.iters == 0 and info.converged
    assert np.array_equal(v, vs)


def test_single_normal_contact_closed_form():
    """One node, one frictionless contact along +z: m (v_n - v*_n) = gamma_n(v_n)
    = h k (phi0 - h v_n)(1 - d v_n) is a quadratic in v_n."""
    m, phi0 = 1.3e-4, 3e-4
    for vsn in (-2.0, -0.5, -0.01, 0.0, 0.5):
        vstar = np.array([[0.3, -0.2, vsn]])
        P = O.ContactProblem([m], vstar, [[0] + [-1] * 26], [[1.0] + [0.0] * 26],
                             [np.eye(3)], [[0, 0, 0]], [phi0], [0.0], [0.0], [K], [D], H)
        v, gam, info, st = P.solve_qn(O.solver(eps_r=1e-14, eps_a=0.0, max_iters=200))
        assert st == O.OK
        # roots of (h k h d) x^2 - (h k (phi0 d + h) + m) x + (h k phi0 + m v*) = 0
        a = H * K * H * D
        bq = -(H * K * (phi0 * D + H) + m)
        c = H * K * phi0 + m * vsn
        x = (-bq - np.sqrt(bq * bq - 4 * a * c)) / (2 * a)
        vhat = min(phi0 / H, 1 / D)
        exact = x if x < vhat else vsn
        assert abs(v[0, 2] - exact) < 1e-11 * max(1, abs(exact))
        assert np.allclose(v[0, :2], vstar[0, :2], atol=1e-14)
        assert abs(gam[0, 2] - m * (v[0, 2] - vsn)) < 1e-12 * max(1e-6, abs(gam[0, 2]))


@pytest.mark.parametrize("vst", [1e-5, 1e-3, 0.05, 1.0])
def test_single_friction_contact_closed_form(vst):
    """One node with a fixed lagged normal impulse: the tangential balance
    m (t - t*) = -mu n0 t / sqrt(t^2 + eps^2) along v*_t, solved by bisection."""
    m, phi0, mu, eps = 1e-4, 2e-4, 0.5, 1e-4
    n0 = O.normal_impulse(phi0, K, D, H, 0.0)
    vstar = np.array([[vst, 0.0, 5.0]])  # separating: no normal impulse in the solve
    P = O.ContactProblem([m], vstar, [[0]], [[1.0]], [np.eye(3)], [[0, 0, 0]], [phi0], [n0],
                         [mu], [K], [D], H, eps)
    v, gam, info, st = P.solve_qn(O.solver(eps_r=1e-14, eps_a=0.0, max_iters=500))
    assert st == O.OK
    f = lambda t: m * (t - vst) + mu * n0 * t / np.sqrt(t * t + eps * eps)
    lo, hi = 0.0, vst
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if f(mid) < 0 else (lo, mid)
    assert abs(v[0, 0] - 0.5 * (lo + hi)) < 1e-11 * max(vst, 1e-6)
    assert abs(v[0, 1]) < 1e-15 and v[0, 2] == 5.0


@pytest.mark.parametrize("seed", range(12))
def test_qn_matches_dense_newton(seed):
    P = random_problem(seed, n_nodes=10 + seed % 5, n_contacts=3 + seed % 6,
                       fixed_frac=0.2 if seed % 3 == 0 else 0.0)
    S = O.solver(eps_r=1e-13, eps_a=0.0, max_iters=20000, ls_rel_tol=1e-12)
    vq, gq, iq, sq = P.solve_qn(S)
    vn, gn, inn, sn = P.solve_dense_newton(S)
    assert sq == O.OK and sn == O.OK
    scale = np.max(np.abs(vn))
    assert np.max(np.abs(vq - vn)) < 1e-9 * scale
    assert inn.iters <= iq.iters


@pytest.mark.parametrize("seed", range(8))
def test_optimality_with_explicit_jacobian(seed):
    """At the solution M (v - v*) = J^T gamma (Eq. (7)) on free DoFs."""
    P = random_problem(100 + seed, fixed_frac=0.25)
    v, gam, info, st = P.solve_qn(O.solver(eps_r=1e-12, eps_a=0.0, max_iters=20000))
    assert st == O.OK
    J = J_matrix(P)
    lhs = (P.m[:, None] * (v - P.vstar.reshape(-1, 3))).ravel()
    rhs = J.T @ gam.ravel()
    free = np.repeat(P.fixed == 0, 3)
    scale = max(np.max(np.abs(rhs)), np.max(np.abs(lhs)))
    assert np.max(np.abs((lhs - rhs)[free])) < 1e-9 * scale
    # fixed DoFs keep v = v*
    assert np.array_equal(v[P.fixed == 1], P.vstar.reshape(-1, 3)[P.fixed == 1])
    # gradient of l_p by central differences of the objective vanishes
    vf = v.ravel()
    eps = 1e-7
    for e in np.flatnonzero(free)[:12]:
        d = np.zeros_like(vf)
        d[e] = eps
        fd = (P.objective(vf + d) - P.objective(vf - d)) / (2 * eps)
        assert abs(fd) < 1e-8 * P.m.max() + 1e-6 * scale


@pytest.mark.parametrize("seed", range(6))
def test_objective_monotone_and_linear_rate(seed):
    P = random_problem(200 + seed, n_nodes=15, n_contacts=8)
    S = O.solver(eps_r=1e-12, eps_a=0.0, max_iters=5000)
    v, gam, info, st, hist = P.solve_qn(S, history=True)
    assert st == O.OK
    assert np.all(np.diff(hist) <= 1e-15 * np.abs(hist[:-1]).max())
    fstar = P.objective(P.solve_dense_newton(S)[0])
    gap = hist - fstar
    if len(gap) > 6:
        # at least linear: the log optimality gap falls with a negative slope
        k = np.arange(len(gap))
        ok = gap > 1e-14 * abs(fstar) + 1e-20
        slope = np.polyfit(k[ok], np.log(gap[ok]), 1)[0] if ok.sum() > 3 else -1.0
        assert slope < 0


@pytest.mark.parametrize("seed", range(6))
def test_tangent_basis_invariance(seed):
    """l_c is isotropic in the tangent plane, so rotating (t1, t2) about n (and
    expressing the bias in the new frame) leaves the solution unchanged."""
    P = random_problem(300 + seed)
    rng = np.random.default_rng(seed)
    R = P.R.reshape(-1, 3, 3)
    b = P.b.reshape(-1, 3)
    R2, b2 = [], []
    for p in range(P.nc):
        th = rng.uniform(0, 2 * np.pi)
        c, s = np.cos(th), np.sin(th)
        Rz = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])
        Rn = R[p] @ Rz
        R2.append(Rn)
        b2.append(Rn.T @ (R[p] @ b[p]))
    P2 = O.ContactProblem(P.m, P.vstar.reshape(-1, 3), P.nodes, P.w, np.stack(R2), np.stack(b2),
                          P.phi0, P.n0, P.mu, P.k, P.d, H)
    S = O.solver(eps_r=1e-13, eps_a=0.0, max_iters=20000)
    v1 = P.solve_qn(S)[0]
    v2 = P2.solve_qn(S)[0]
    assert np.max(np.abs(v1 - v2)) < 1e-10 * np.max(np.abs(v1))


def test_stopping_rule_uses_relative_tolerance():
    P = random_problem(400, n_nodes=15, n_contacts=8)
    loose = P.solve_qn(O.solver(eps_r=5e-2, eps_a=0.0))[2]
    tight = P.solve_qn(O.solver(eps_r=1e-10, eps_a=0.0, max_iters=20000))[2]
    assert loose.converged and tight.converged
    assert loose.iters <= tight.iters
    assert loose.G < 5e-2 * max(loose.P, loose.J)
    assert tight.G < 1e-10 * max(tight.P, tight.J)


def test_iteration_cap_reports_not_converged():
    P = random_problem(401, n_nodes=15, n_contacts=8)
    v, gam, info, st = P.solve_qn(O.solver(eps_r=1e-14, eps_a=0.0, max_iters=1))
    assert st == O.ERR_NOT_CONVERGED and info.iters == 1 and not info.converged


@pytest.mark.parametrize("seed,fixed_frac", [(0, 0.0), (4, 0.3)])
def test_gradient_is_the_objectives_derivative(seed, fixed_frac):
    """Eq. (9) against the objective of Eq. (8): central differences of l_p
    along each free DoF at a random velocity equal the gradient (fixed DoFs
    read zero); without contacts the gradient is M (v - v*); at the dense
    Newton minimiser it vanishes on the free DoFs."""
    P = random_problem(seed, fixed_frac=fixed_frac)
    rng = np.random.default_rng(100 + seed)
    v = rng.normal(scale=0.5, size=(P.n, 3))
    g = P.gradient(v)
    free = P.fixed == 0
    assert np.all(g[~free] == 0.0)
    eps = 1e-6
    fd = np.zeros_like(g)
    for i in np.flatnonzero(free):
        for c in range(3):
            d = np.zeros_like(v)
            d[i, c] = eps
            fd[i, c] = (P.objective(v + d) - P.objective(v - d)) / (2 * eps)
    scale = np.max(np.abs(g))
    assert np.max(np.abs(fd[free] - g[free])) <= 1e-6 * scale
    P0 = O.ContactProblem(P.m, P.vstar, np.zeros((0, 27)), np.zeros((0, 27)), np.zeros((0, 3, 3)),
                          np.zeros((0, 3)), [], [], [], [], [], H, 1e-4, P.fixed)
    g0 = P0.gradient(v)
    want = P.m[:, None] * (v - P.vstar.reshape(-1, 3))
    assert np.allclose(g0[free], want[free], rtol=1e-14, atol=0)
    vs, _, _, st = P.solve_dense_newton(O.solver(eps_r=1e-12, eps_a=0.0, max_iters=200))
    assert st == O.OK
    gs = P.gradient(vs)
    assert np.max(np.abs(gs[free])) <= 1e-9 * scale
