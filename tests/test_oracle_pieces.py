"""Pins of the oracle's building blocks against mathematics the paper fixes or
cites: B-spline moment identities, SVD against LAPACK, stresses as derivatives
of their energy densities, Drucker-Prager projection properties, SDF closed
forms and the contact potential's derivative consistency and convexity."""
import numpy as np
import pytest

import oracle as O

RNG = np.random.default_rng(1234)


# --------------------------------------------------------------- transfer kernel

@pytest.mark.parametrize("trial", range(20))
def test_bspline_moments(trial):
    """Quadratic B-spline: partition of unity, linear reproduction and second
    moment dx^2/4 I (the identity behind D_p^-1 = 4/dx^2 in MLS-MPM)."""
    dx = 0.01 * (1 + trial % 3)
    origin = RNG.uniform(-1, 1, 3)
    x = origin + RNG.uniform(2 * dx, 20 * dx, 3)
    base, fx, w = O.bspline(dx, origin, x)
    assert np.all(fx >= 0.5) and np.all(fx < 1.5)
    assert np.all(w >= 0)
    s0 = 0.0
    s1 = np.zeros(3)
    s2 = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            for c in range(3):
                wt = w[0, a] * w[1, b] * w[2, c]
                xi = origin + dx * (base + np.array([a, b, c]))
                r = xi - x
                s0 += wt
                s1 += wt * r
                s2 += wt * np.outer(r, r)
    assert abs(s0 - 1) < 1e-14
    assert np.max(np.abs(s1)) < 1e-14 * dx * 10
    assert np.allclose(s2, dx * dx / 4 * np.eye(3), rtol=0, atol=1e-14 * dx * dx * 10)


def test_bspline_values_closed_form():
    """At fx = 1 (particle on a node) the 1-D weights are (1/8, 3/4, 1/8)."""
    base, fx, w = O.bspline(0.1, np.zeros(3), np.array([0.5, 0.5, 0.5]))
    assert np.all(base == 4)
    assert np.allclose(w, [[0.125, 0.75, 0.125]] * 3, atol=1e-15)


# --------------------------------------------------------------- SVD and stresses

def _rand_F(rng, spread=0.3, allow_inverted=False):
    F = np.eye(3) + rng.uniform(-spread, spread, (3, 3))
    if allow_inverted and rng.uniform() < 0.3:
        F[:, 2] *= -1
    return F


@pytest.mark.parametrize("trial", range(40))
def test_svd3_against_lapack(trial):
    rng = np.random.default_rng(trial)
    F = _rand_F(rng, 0.8, allow_inverted=True)
    U, S, V = O.svd3(F)
    assert np.allclose(U @ np.diag(S) @ V.T, F, atol=1e-13)
    assert np.allclose(U.T @ U, np.eye(3), atol=1e-13)
    assert np.allclose(V.T @ V, np.eye(3), atol=1e-13)
    assert abs(np.linalg.det(U) - 1) < 1e-12 and abs(np.linalg.det(V) - 1) < 1e-12
    ref = np.linalg.svd(F, compute_uv=False)
    assert np.allclose(np.abs(S), ref, rtol=1e-12, atol=1e-14)
    assert (S[2] < 0) == (np.linalg.det(F) < 0)


def test_svd3_degenerate():
    for F in (np.zeros((3, 3)), np.diag([2.0, 0.0, 0.0]), np.diag([1.0, 1.0, 0.0]),
              np.eye(3), np.diag([3.0, 3.0, 3.0])):
        U, S, V = O.svd3(F)
        assert np.allclose(U @ np.diag(S) @ V.T, F, atol=1e-13)
        assert np.allclose(U.T @ U, np.eye(3), atol=1e-12)
        assert np.allclose(V.T @ V, np.eye(3), atol=1e-12)


def _corotated_energy(F, mu, lam):
    """Fixed-corotated energy density: mu sum (s_i - 1)^2 + lam/2 (J - 1)^2."""
    s = np.linalg.svd(F, compute_uv=False)
    J = np.linalg.det(F)
    if J < 0:
        s[2] = -s[2]
    return mu * np.sum((s - 1) ** 2) + 0.5 * lam * (J - 1) ** 2


def _hencky_energy(F, mu, lam):
    """Hencky energy density: mu sum ln(s_i)^2 + lam/2 (sum ln s_i)^2."""
    e = np.log(np.linalg.svd(F, compute_uv=False))
    return mu * np.sum(e ** 2) + 0.5 * lam * np.sum(e) ** 2


def _fd_grad(fun, F, h=1e-6):
    G = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            E = np.zeros((3, 3))
            E[i, j] = h
            G[i, j] = (fun(F + E) - fun(F - E)) / (2 * h)
    return G


@pytest.mark.parametrize("trial", range(15))
def test_corotated_P_is_energy_gradient(trial):
    rng = np.random.default_rng(100 + trial)
    F = _rand_F(rng, 0.3)
    mu, lam = O.lame(1e5, 0.3)
    P = O.corotated_P(F, mu, lam)
    G = _fd_grad(lambda A: _corotated_energy(A, mu, lam), F)
    assert np.allclose(P, G, rtol=1e-6, atol=1e-4)
    tau = O.corotated_tau(F, mu, lam)
    assert np.allclose(tau, P @ F.T, atol=1e-9)
    assert np.allclose(tau, tau.T, atol=1e-8)


@pytest.mark.parametrize("trial", range(15))
def test_hencky_P_is_energy_gradient(trial):
    rng = np.random.default_rng(200 + trial)
    F = _rand_F(rng, 0.3)
    if np.linalg.det(F) <= 0:
        F = np.eye(3) + 0.1 * (F - np.eye(3))
    mu, lam = O.lame(3.5e5, 0.3)
    P = O.hencky_P(F, mu, lam)
    G = _fd_grad(lambda A: _hencky_energy(A, mu, lam), F)
    assert np.allclose(P, G, rtol=1e-6, atol=1e-3)
    tau = O.hencky_tau(F, mu, lam)
    assert np.allclose(tau, tau.T, atol=1e-8)
    # principal form agrees with P F^T while nothing is clamped
    assert np.allclose(tau, P @ F.T, rtol=1e-9, atol=1e-6)


def _hencky_grad_hp(F, mu, lam):
    """Gradient of the Hencky energy density mu sum ln(s_i)^2 + lam/2
    (sum ln s_i)^2 by central differences in 40-digit arithmetic (mpmath's
    SVD): at a singular value of 1e-4, double-precision singular values limit
    a double-precision difference quotient to ~1e-4 relative."""
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 40

    def psi(A):
        e = [mpmath.log(x) for x in mp.svd_r(mpmath.matrix(A), compute_uv=False)]
        return mu * sum(x * x for x in e) + lam / 2 * sum(e) ** 2

    Fm = [[mpmath.mpf(float(F[i, j])) for j in range(3)] for i in range(3)]
    h = mpmath.mpf("1e-20")
    G = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            A = [r[:] for r in Fm]
            B = [r[:] for r in Fm]
            A[i][j] += h
            B[i][j] -= h
            G[i, j] = float((psi(A) - psi(B)) / (2 * h))
    return G


def test_hencky_tau_clamps_the_strain():
    """Singular values below 1e-4, and the negative one of an inverted F, are
    clamped to 1e-4 before the logarithm: the stress is the Kirchhoff stress
    of the clamped F_c = U diag(max(s, 1e-4)) V^T (same rotations), pinned
    here as dpsi/dF (F_c) F_c^T with the gradient of the Hencky energy density
    taken by central differences at F_c (F_c has no singular value below the
    clamp, so nothing is clamped there)."""
    mu, lam = O.lame(3.5e5, 0.3)
    rng = np.random.default_rng(11)
    for trial in range(3):
        U, V = _rotation(rng), _rotation(rng)
        s12 = rng.uniform(0.6, 1.4, 2)
        Fc = U @ np.diag([s12[0], s12[1], 1e-4]) @ V.T
        expected = _hencky_grad_hp(Fc, mu, lam) @ Fc.T
        scale = np.max(np.abs(expected))
        # (an inverted F carries its reflection on the smallest singular value)
        for s3 in (-0.5, -1e-3, 0.0, 1e-6, 9e-5):
            F = U @ np.diag([s12[0], s12[1], s3]) @ V.T
            got = O.hencky_tau(F, mu, lam)
            assert np.allclose(got, expected, rtol=0, atol=1e-9 * scale), (trial, s3)
    # a singular value just above the clamp is not clamped: the stress is P F^T
    U, V = _rotation(rng), _rotation(rng)
    F = U @ np.diag([1.1, 0.95, 2e-4]) @ V.T
    expected = _hencky_grad_hp(F, mu, lam) @ F.T
    assert np.allclose(O.hencky_tau(F, mu, lam), expected, rtol=0,
                       atol=1e-9 * np.max(np.abs(expected)))


def _rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a*a+b*b-c*c-d*d, 2*(b*c-a*d), 2*(b*d+a*c)],
                     [2*(b*c+a*d), a*a-b*b+c*c-d*d, 2*(c*d-a*b)],
                     [2*(b*d-a*c), 2*(c*d+a*b), a*a-b*b-c*c+d*d]])


def test_corotated_rest_and_frame_indifference():
    rng = np.random.default_rng(7)
    mu, lam = O.lame(1e5, 0.3)
    for _ in range(10):
        Q = _rotation(rng)
        assert np.max(np.abs(O.corotated_P(Q, mu, lam))) < 1e-9
        assert np.max(np.abs(O.hencky_P(Q, mu, lam))) < 1e-9
        F = _rand_F(rng, 0.3)
        assert np.allclose(O.corotated_P(Q @ F, mu, lam), Q @ O.corotated_P(F, mu, lam), atol=1e-8)
        assert np.allclose(O.hencky_P(Q @ F, mu, lam), Q @ O.hencky_P(F, mu, lam), atol=1e-7)


def test_small_strain_limit_is_linear_elasticity():
    """For F = I + eps (eps symmetric, small) both models give 2 mu eps + lam tr(eps) I."""
    rng = np.random.default_rng(8)
    mu, lam = O.lame(1e5, 0.3)
    A = rng.uniform(-1, 1, (3, 3))
    eps = 1e-5 * (A + A.T)
    lin = 2 * mu * eps + lam * np.trace(eps) * np.eye(3)
    for fn in (O.corotated_P, O.hencky_P):
        P = fn(np.eye(3) + eps, mu, lam)
        assert np.allclose(P, lin, rtol=1e-3, atol=1e-3 * np.max(np.abs(lin)))


def _dp_yield(F, mu, lam, phi_deg):
    s = np.linalg.svd(F, compute_uv=False)
    e = np.log(s)
    tr = e.sum()
    eh = e - tr / 3
    sphi = np.sin(np.radians(phi_deg))
    alpha = np.sqrt(2 / 3) * 2 * sphi / (3 - sphi)
    return np.linalg.norm(eh) + (3 * lam + 2 * mu) / (2 * mu) * tr * alpha, tr


@pytest.mark.parametrize("trial", range(30))
def test_drucker_prager_projection(trial):
    rng = np.random.default_rng(300 + trial)
    mu, lam = O.lame(3.5e5, 0.3)
    F = _rand_F(rng, 0.25)
    if np.linalg.det(F) <= 0:
        F = np.eye(3)
    Fp = O.dp_project(F, mu, lam, 30.0)
    # idempotent
    assert np.allclose(O.dp_project(Fp, mu, lam, 30.0), Fp, atol=1e-12)
    dg, tr = _dp_yield(Fp, mu, lam, 30.0)
    assert dg <= 1e-10
    dg0, tr0 = _dp_yield(F, mu, lam, 30.0)
    if tr0 >= 0:  # expansion: projected to the cone tip, stress free
        assert np.allclose(np.linalg.svd(Fp, compute_uv=False), 1.0, atol=1e-12)
        assert np.max(np.abs(O.hencky_P(Fp, mu, lam))) < 1e-6
    elif dg0 <= 0:  # inside the cone: unchanged
        assert np.array_equal(Fp, F)
    else:  # projected onto the cone: volume (tr eps) kept, lies on the surface
        assert abs(tr - tr0) < 1e-12
        assert abs(dg) < 1e-10
    # rotations of the SVD are kept: Fp F^-1 ... left/right singular vectors agree
    U0, _, V0 = np.linalg.svd(F)
    U1, _, V1 = np.linalg.svd(Fp)
    if tr0 < 0 and dg0 > 0:
        assert np.allclose(np.abs(np.sum(U0 * U1, 0)), 1.0, atol=1e-6)


# --------------------------------------------------------------- geometry

def _fd_normal(body, x, h=1e-7):
    g = np.zeros(3)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        g[a] = (O.sdf(body, x + e)[0] - O.sdf(body, x - e)[0]) / (2 * h)
    return g


def _bodies(rng):
    R = _rotation(rng)
    p = rng.uniform(-0.1, 0.1, 3)
    return [
        {"shape": O.HALFSPACE, "R": R, "p": p},
        {"shape": O.SPHERE, "params": [0.05, 0, 0, 0], "R": R, "p": p},
        {"shape": O.BOX, "params": [0.03, 0.05, 0.02, 0], "R": R, "p": p},
        {"shape": O.CAPSULE, "params": [0.04, 0.015, 0, 0], "R": R, "p": p},
    ]


@pytest.mark.parametrize("trial", range(10))
def test_sdf_gradient_is_normal(trial):
    rng = np.random.default_rng(400 + trial)
    for b in _bodies(rng):
        for _ in range(10):
            x = b["p"] + rng.uniform(-0.08, 0.08, 3)
            phi, n = O.sdf(b, x)
            assert abs(np.linalg.norm(n) - 1) < 1e-12
            g = _fd_normal(b, x)
            if abs(np.linalg.norm(g) - 1) < 1e-4:  # away from the medial axis
                assert np.allclose(g, n, atol=1e-5)


def test_sdf_closed_forms():
    b = {"shape": O.SPHERE, "params": [0.05, 0, 0, 0], "p": np.array([1.0, 2.0, 3.0])}
    assert abs(O.sdf(b, [1.0, 2.0, 3.0])[0] + 0.05) < 1e-15
    assert abs(O.sdf(b, [1.0, 2.0, 3.2])[0] - 0.15) < 1e-12
    box = {"shape": O.BOX, "params": [0.1, 0.2, 0.3, 0]}
    phi, n = O.sdf(box, [0.0, 0.0, 0.0])
    assert abs(phi + 0.1) < 1e-15 and np.allclose(n, [1, 0, 0])
    phi, n = O.sdf(box, [0.0, -0.15, 0.0])
    assert abs(phi + 0.05) < 1e-15 and np.allclose(n, [0, -1, 0])
    phi, n = O.sdf(box, [0.2, 0.3, 0.0])  # outside an edge
    assert abs(phi - np.hypot(0.1, 0.1)) < 1e-12
    hs = {"shape": O.HALFSPACE, "R": O_rot_y(0.3), "p": np.zeros(3)}
    phi, n = O.sdf(hs, [0.0, 0.0, -0.01])
    assert np.allclose(n, [np.sin(0.3), 0, np.cos(0.3)])
    assert abs(phi + 0.01 * np.cos(0.3)) < 1e-15
    cap = {"shape": O.CAPSULE, "params": [0.1, 0.02, 0, 0]}
    assert abs(O.sdf(cap, [0.0, 0.0, 0.12])[0] - 0.0) < 1e-15
    assert abs(O.sdf(cap, [0.05, 0.0, 0.05])[0] - 0.03) < 1e-15


def O_rot_y(t):
    c, s = np.cos(t), np.sin(t)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])


def test_body_velocity_rigid_motion():
    rng = np.random.default_rng(5)
    b = {"shape": O.SPHERE, "params": [0.1, 0, 0, 0], "p": rng.normal(size=3),
         "omega": rng.normal(size=3), "v": rng.normal(size=3)}
    x = rng.normal(size=3)
    vel = O.body_velocity(b, x)
    # finite rotation about p: x(t) = p + v t + exp(t [w]x)(x - p)
    w = b["omega"]
    W = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    dt = 1e-6
    from scipy.linalg import expm
    xp = b["p"] + b["v"] * dt + expm(dt * W) @ (x - b["p"])
    xm = b["p"] - b["v"] * dt + expm(-dt * W) @ (x - b["p"])
    assert np.allclose(vel, (xp - xm) / (2 * dt), atol=1e-7)


def test_contact_frame_orthonormal():
    rng = np.random.default_rng(6)
    for _ in range(50):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        R = O.contact_frame(n, rng.uniform(0, 6.3))
        assert np.allclose(R.T @ R, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1) < 1e-14
        assert np.allclose(R[:, 2], n)


# --------------------------------------------------------------- contact model

PRM = dict(phi0=2e-4, n0=3e-6, mu=0.5, k=1e4, d=10.0, h=1e-4, eps_s=1e-4)


def _ell(vc, **kw):
    p = dict(PRM)
    p.update(kw)
    return O.contact_potential(p["phi0"], p["n0"], p["mu"], p["k"], p["d"], p["h"],
                               p["eps_s"], vc)


def test_normal_impulse_law():
    h, k, d, phi0 = 1e-4, 1e4, 10.0, 2e-4
    assert abs(O.normal_impulse(phi0, k, d, h, 0.0) - h * k * phi0) < 1e-20
    assert O.normal_impulse(phi0, k, d, h, phi0 / h + 1e-9) == 0.0
    assert O.normal_impulse(phi0, k, d, h, 1.0 / d + 1e-9) == 0.0
    vs = np.linspace(-1, 1, 201)
    g = np.array([O.normal_impulse(phi0, k, d, h, v) for v in vs])
    assert np.all(g >= 0) and np.all(np.diff(g) <= 1e-18)  # non-increasing


@pytest.mark.parametrize("trial", range(40))
def test_contact_potential_derivatives(trial):
    rng = np.random.default_rng(500 + trial)
    vc = rng.normal(scale=[2e-4, 2e-4, 1.0], size=3)
    ell, g, H = _ell(vc)
    hstep = np.array([1e-8, 1e-8, 1e-7])
    for a in range(3):
        e = np.zeros(3)
        e[a] = hstep[a]
        fd = (_ell(vc + e)[0] - _ell(vc - e)[0]) / (2 * hstep[a])
        roundoff = 4e-16 * max(abs(ell), 1e-30) / hstep[a]
        assert abs(fd - g[a]) <= 1e-5 * abs(g[a]) + roundoff + 1e-14
        fdg = (_ell(vc + e)[1] - _ell(vc - e)[1]) / (2 * hstep[a])
        assert np.allclose(fdg, H[:, a], rtol=1e-4, atol=1e-10)
    # gamma_n = -dN/dv_n
    assert abs(-g[2] - O.normal_impulse(PRM["phi0"], PRM["k"], PRM["d"], PRM["h"], vc[2])) < 1e-15
    # convex: Hessian is PSD; the potential is zero for separating contacts at rest
    assert np.min(np.linalg.eigvalsh(H)) >= -1e-12
    assert _ell(np.array([0, 0, 1.0]))[0] == 0.0


def test_contact_potential_convex_along_lines():
    rng = np.random.default_rng(11)
    for _ in range(50):
        a = rng.normal(scale=[1e-3, 1e-3, 0.5], size=3)
        b = rng.normal(scale=[1e-3, 1e-3, 0.5], size=3)
        fa, fb = _ell(a)[0], _ell(b)[0]
        for t in np.linspace(0.1, 0.9, 5):
            assert _ell(t * a + (1 - t) * b)[0] <= t * fa + (1 - t) * fb + 1e-15


def test_friction_is_regularised_coulomb():
    mu, n0 = PRM["mu"], PRM["n0"]
    for speed in (1e-2, 1e-1, 1.0):
        _, g, _ = _ell(np.array([speed, 0, 0.5]))
        # gamma_t = -grad_t opposes sliding and saturates at mu n0
        assert g[0] > 0 and abs(g[0] - mu * n0) < mu * n0 * (PRM["eps_s"] / speed) ** 2
        assert abs(g[1]) < 1e-18
    _, g, _ = _ell(np.array([1e-6, 0, 0.5]))
    assert g[0] < mu * n0 * 0.02  # stiction region is linear in v_t


def test_drucker_prager_branches_explicit():
    """Each branch of the return map on a hand-picked deformation: expansion goes
    to the cone tip, mild compression stays, sheared compression is projected
    with its volume kept."""
    mu, lam = O.lame(3.5e5, 0.3)
    Fexp = np.diag([1.02, 1.01, 1.0])
    assert np.allclose(np.linalg.svd(O.dp_project(Fexp, mu, lam, 30.0), compute_uv=False), 1.0)
    Fin = np.diag([0.99, 0.99, 0.99])
    assert np.array_equal(O.dp_project(Fin, mu, lam, 30.0), Fin)
    Fsh = np.diag([1.05, 0.97, 0.95])
    dg0, tr0 = _dp_yield(Fsh, mu, lam, 30.0)
    assert tr0 < 0 and dg0 > 0
    Fp = O.dp_project(Fsh, mu, lam, 30.0)
    dg, tr = _dp_yield(Fp, mu, lam, 30.0)
    assert abs(dg) < 1e-12 and abs(tr - tr0) < 1e-13
