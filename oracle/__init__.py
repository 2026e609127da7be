"""ctypes front end of the FP64 CPU oracle (``mpm_oracle.c``).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It never imports the
CUDA library's binding and the CUDA library never calls it.

Inputs use the plain-data scene format of ``paper_2503_05046_gb300.scenes``
(numpy arrays and dicts); every value is widened to float64 here.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)

HALFSPACE, SPHERE, BOX, CAPSULE = 0, 1, 2, 3
COROTATED, DRUCKER_PRAGER, CLOTH = 0, 1, 2
OK, ERR_OUT_OF_DOMAIN, ERR_NOT_CONVERGED, ERR_LINE_SEARCH, ERR_ARG, ERR_NOT_SPD = range(6)


class Grid(C.Structure):
    _fields_ = [("dx", C.c_double), ("res", C.c_int * 3), ("origin", C.c_double * 3),
                ("gravity", C.c_double * 3), ("bc_layers", C.c_int)]


class Body(C.Structure):
    _fields_ = [("shape", C.c_int), ("params", C.c_double * 4), ("R", C.c_double * 9),
                ("p", C.c_double * 3), ("omega", C.c_double * 3), ("v", C.c_double * 3),
                ("mu", C.c_double), ("k", C.c_double), ("d", C.c_double),
                ("kinematic", C.c_int)]


class Dynamics(C.Structure):
    _fields_ = [("mass", C.c_double), ("inertia", C.c_double * 3), ("force", C.c_double * 3),
                ("torque", C.c_double * 3), ("dof_mask", C.c_int), ("gravity", C.c_int)]


class Material(C.Structure):
    _fields_ = [("model", C.c_int), ("E", C.c_double), ("nu", C.c_double),
                ("friction_angle_deg", C.c_double)]


class Solver(C.Structure):
    _fields_ = [("eps_r", C.c_double), ("eps_a", C.c_double), ("max_iters", C.c_int),
                ("eps_s", C.c_double), ("ls_rel_tol", C.c_double), ("ls_max_iters", C.c_int)]


class Problem(C.Structure):
    _fields_ = [("n_nodes", C.c_int), ("m", _dp), ("vstar", _dp), ("fixed", _ip),
                ("n_contacts", C.c_int), ("nodes", _ip), ("w", _dp), ("R", _dp), ("b", _dp),
                ("phi0", _dp), ("n0", _dp), ("mu", _dp), ("k", _dp), ("d", _dp),
                ("h", C.c_double), ("eps_s", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("converged", C.c_int), ("ls_evals", C.c_int),
                ("G", C.c_double), ("P", C.c_double), ("J", C.c_double), ("status", C.c_int)]


class SubstepInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("n_contacts", C.c_int), ("n_dofs", C.c_int),
                ("iters", C.c_int), ("converged", C.c_int), ("G", C.c_double),
                ("P", C.c_double), ("J", C.c_double)]


_libs = {}


def lib(openmp=False):
    """Load (building first if needed) the oracle shared library: the serial
    checker, or with openmp=True its all-core build (CPU baseline only)."""
    key = bool(openmp)
    if key not in _libs:
        path = _build.build(openmp=key)
        L = C.CDLL(path)
        L.orc_threads.restype = C.c_int
        L.orc_bspline.argtypes = [C.c_double, _dp, _dp, _ip, _dp, _dp]
        L.orc_svd3.argtypes = [_dp, _dp, _dp, _dp]
        L.orc_lame.argtypes = [C.c_double, C.c_double, _dp, _dp]
        for f in ("orc_corotated_P", "orc_corotated_tau", "orc_hencky_P", "orc_hencky_tau"):
            getattr(L, f).argtypes = [_dp, C.c_double, C.c_double, _dp]
        L.orc_dp_project.argtypes = [_dp, C.c_double, C.c_double, C.c_double, _dp]
        L.orc_sdf.argtypes = [C.POINTER(Body), _dp, _dp]
        L.orc_sdf.restype = C.c_double
        L.orc_body_velocity.argtypes = [C.POINTER(Body), _dp, _dp]
        L.orc_contact_frame.argtypes = [_dp, C.c_double, _dp]
        L.orc_normal_impulse.argtypes = [C.c_double] * 5
        L.orc_normal_impulse.restype = C.c_double
        L.orc_contact_potential.argtypes = [C.c_double] * 7 + [_dp, _dp, _dp]
        L.orc_contact_potential.restype = C.c_double
        L.orc_objective.argtypes = [C.POINTER(Problem), _dp]
        L.orc_objective.restype = C.c_double
        L.orc_gradient.argtypes = [C.POINTER(Problem), _dp, _dp]
        L.orc_solve_qn.argtypes = [C.POINTER(Problem), C.POINTER(Solver), _dp, _dp,
                                   C.POINTER(SolveInfo), _dp]
        L.orc_solve_dense_newton.argtypes = [C.POINTER(Problem), C.POINTER(Solver), _dp, _dp,
                                             C.POINTER(SolveInfo)]
        L.orc_create.argtypes = [C.POINTER(Grid)]
        L.orc_create.restype = C.c_void_p
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_substep.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _ip,
                                  C.c_int, C.POINTER(Material), C.c_int, C.POINTER(Body),
                                  C.c_double, C.POINTER(Solver), _dp, C.POINTER(SubstepInfo)]
        L.orc_last_grid.argtypes = [C.c_void_p, C.c_int, _ip, _dp, _dp, _dp]
        L.orc_last_contacts.argtypes = [C.c_void_p, C.c_int, _ip, _ip, _dp, _dp, _dp]
        L.orc_advance_kinematic.argtypes = [C.c_int, C.POINTER(Body), C.c_double]
        L.orc_contact_adjoint.argtypes = [C.POINTER(Problem), _dp, _dp, _dp, _dp, _dp]
        L.orc_rigid_dynamics_step.argtypes = [C.POINTER(Body), C.POINTER(Dynamics), _dp, _dp,
                                              C.c_double]
        L.orc_cloth_rest.argtypes = [_dp, _dp, _dp, _dp, _dp]
        L.orc_cloth_triangle.argtypes = [_dp, _dp, _dp, _dp, C.c_double, C.c_double, C.c_double,
                                         _dp]
        L.orc_cloth_triangle.restype = C.c_double
        L.orc_set_cloth.argtypes = [C.c_void_p, C.c_int, _ip, _dp, _dp, _ip]
        L.orc_set_pins.argtypes = [C.c_void_p, C.c_int, _ip, _dp]
        _libs[key] = L
    return _libs[key]


def threads(openmp=False):
    """Threads one substep of that build uses (1 for the serial checker)."""
    return int(lib(openmp).orc_threads())


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a.reshape(shape) if shape is not None else a


# --------------------------------------------------------------------------- pieces

def bspline(dx, origin, x):
    """Quadratic B-spline stencil: (base[3], fx[3], w[3,3]) with w[axis, offset]."""
    base = np.zeros(3, np.int32)
    fx = np.zeros(3)
    w = np.zeros(9)
    lib().orc_bspline(float(dx), _d(_f64(origin)), _d(_f64(x)), _i(base), _d(fx), _d(w))
    return base, fx, w.reshape(3, 3)


def svd3(F):
    U, S, V = np.zeros(9), np.zeros(3), np.zeros(9)
    lib().orc_svd3(_d(_f64(F, 9)), _d(U), _d(S), _d(V))
    return U.reshape(3, 3), S, V.reshape(3, 3)


def lame(E, nu):
    mu, lam = C.c_double(), C.c_double()
    lib().orc_lame(E, nu, C.byref(mu), C.byref(lam))
    return mu.value, lam.value


def _stress(name, F, mu, lam):
    out = np.zeros(9)
    getattr(lib(), name)(_d(_f64(F, 9)), mu, lam, _d(out))
    return out.reshape(3, 3)


def corotated_P(F, mu, lam):
    return _stress("orc_corotated_P", F, mu, lam)


def corotated_tau(F, mu, lam):
    return _stress("orc_corotated_tau", F, mu, lam)


def hencky_P(F, mu, lam):
    return _stress("orc_hencky_P", F, mu, lam)


def hencky_tau(F, mu, lam):
    return _stress("orc_hencky_tau", F, mu, lam)


def dp_project(F, mu, lam, friction_angle_deg):
    out = np.zeros(9)
    lib().orc_dp_project(_d(_f64(F, 9)), mu, lam, friction_angle_deg, _d(out))
    return out.reshape(3, 3)


def make_body(b):
    """Scene body dict -> oracle Body struct (float64)."""
    s = Body()
    s.shape = int(b["shape"])
    for i, v in enumerate(np.asarray(b.get("params", [0, 0, 0, 0]), np.float64).ravel()[:4]):
        s.params[i] = float(v)
    R = np.asarray(b.get("R", np.eye(3)), np.float64).reshape(9)
    for i in range(9):
        s.R[i] = float(R[i])
    for key in ("p", "omega", "v"):
        arr = getattr(s, key)
        val = np.asarray(b.get(key, [0, 0, 0]), np.float64).reshape(3)
        for i in range(3):
            arr[i] = float(val[i])
    s.mu = float(b.get("mu", 0.0))
    s.k = float(b.get("k", 1e4))
    s.d = float(b.get("d", 10.0))
    s.kinematic = int(b.get("kinematic", 0))
    return s


def body_dict(s):
    """Oracle Body struct -> scene body dict."""
    return {"shape": s.shape, "params": np.array(s.params[:]), "R": np.array(s.R[:]).reshape(3, 3),
            "p": np.array(s.p[:]), "omega": np.array(s.omega[:]), "v": np.array(s.v[:]),
            "mu": s.mu, "k": s.k, "d": s.d, "kinematic": s.kinematic}


def sdf(body, x):
    b = make_body(body)
    n = np.zeros(3)
    phi = lib().orc_sdf(C.byref(b), _d(_f64(x)), _d(n))
    return phi, n


def body_velocity(body, x):
    b = make_body(body)
    out = np.zeros(3)
    lib().orc_body_velocity(C.byref(b), _d(_f64(x)), _d(out))
    return out


def contact_frame(n, angle=0.0):
    R = np.zeros(9)
    lib().orc_contact_frame(_d(_f64(n)), float(angle), _d(R))
    return R.reshape(3, 3)


def normal_impulse(phi0, k, d, h, vn):
    return lib().orc_normal_impulse(phi0, k, d, h, vn)


def contact_potential(phi0, n0, mu, k, d, h, eps_s, vc):
    g = np.zeros(3)
    H = np.zeros(9)
    ell = lib().orc_contact_potential(phi0, n0, mu, k, d, h, eps_s, _d(_f64(vc)), _d(g), _d(H))
    return ell, g, H.reshape(3, 3)


def solver(eps_r=5e-2, eps_a=np.finfo(np.float64).eps, max_iters=500, eps_s=1e-4,
           ls_rel_tol=1e-10, ls_max_iters=100):
    """Alg. 1 settings. Defaults: the paper's eps_r = 5e-2 and eps_a = machine
    epsilon (Sec. VI); eps_s is the friction regularisation velocity."""
    return Solver(eps_r, eps_a, max_iters, eps_s, ls_rel_tol, ls_max_iters)


class ContactProblem:
    """The convex problem of Eq. (8) over explicit DoFs and contacts.

    m[n], vstar[n,3], fixed[n] (bool), and per contact: nodes[nc,27] (DoF index
    or -1), w[nc,27], R[nc,3,3] (columns t1 t2 n), b[nc,3] (contact frame),
    phi0, n0, mu, k, d [nc]; h, eps_s scalars.
    """

    def __init__(self, m, vstar, nodes, w, R, b, phi0, n0, mu, k, d, h, eps_s=1e-4,
                 fixed=None):
        n = len(m)
        nc = len(phi0)
        self.m = _f64(m)
        self.vstar = _f64(vstar, (n * 3,))
        self.fixed = np.ascontiguousarray(
            np.zeros(n, np.int32) if fixed is None else np.asarray(fixed, np.int32))
        nodes = np.asarray(nodes, np.int32).reshape(nc, -1) if nc else np.zeros((0, 27), np.int32)
        w = np.asarray(w, np.float64).reshape(nc, -1) if nc else np.zeros((0, 27))
        if nodes.shape[1] < 27:
            pad = 27 - nodes.shape[1]
            nodes = np.concatenate([nodes, -np.ones((nc, pad), np.int32)], 1)
            w = np.concatenate([w, np.zeros((nc, pad))], 1)
        self.nodes = np.ascontiguousarray(nodes)
        self.w = np.ascontiguousarray(w)
        self.R = _f64(R, (nc * 9,))
        self.b = _f64(b, (nc * 3,))
        self.phi0, self.n0 = _f64(phi0, (nc,)), _f64(n0, (nc,))
        self.mu, self.k, self.d = _f64(mu, (nc,)), _f64(k, (nc,)), _f64(d, (nc,))
        self.n, self.nc = n, nc
        self.s = Problem(n, _d(self.m), _d(self.vstar), _i(self.fixed), nc, _i(self.nodes),
                         _d(self.w), _d(self.R), _d(self.b), _d(self.phi0), _d(self.n0),
                         _d(self.mu), _d(self.k), _d(self.d), float(h), float(eps_s))

    def objective(self, v):
        return lib().orc_objective(C.byref(self.s), _d(_f64(v, (self.n * 3,))))

    def gradient(self, v):
        g = np.zeros(self.n * 3)
        lib().orc_gradient(C.byref(self.s), _d(_f64(v, (self.n * 3,))), _d(g))
        return g.reshape(self.n, 3)

    def solve_qn(self, S, v0=None, history=False):
        v = (self.vstar.copy() if v0 is None else _f64(v0, (self.n * 3,)).copy())
        gam = np.zeros(max(self.nc, 1) * 3)
        info = SolveInfo()
        hist = np.zeros(S.max_iters + 2) if history else None
        st = lib().orc_solve_qn(C.byref(self.s), C.byref(S), _d(v), _d(gam), C.byref(info),
                                _d(hist) if history else None)
        out = (v.reshape(self.n, 3), gam[:3 * self.nc].reshape(self.nc, 3), info, st)
        if history:
            out = out + (hist[:info.iters + 1],)
        return out

    def adjoint(self, v, vbar):
        """Adjoint of the solve at the minimiser v for dL/dv = vbar:
        (dL/dv*[n,3], dL/db[nc,3] contact frame, dL/dmu[nc], status)."""
        vsb = np.zeros(self.n * 3)
        bb = np.zeros(max(self.nc, 1) * 3)
        mb = np.zeros(max(self.nc, 1))
        st = lib().orc_contact_adjoint(C.byref(self.s), _d(_f64(v, (self.n * 3,))),
                                       _d(_f64(vbar, (self.n * 3,))), _d(vsb), _d(bb), _d(mb))
        return vsb.reshape(self.n, 3), bb[:3 * self.nc].reshape(self.nc, 3), mb[:self.nc], st

    def solve_dense_newton(self, S, v0=None):
        v = (self.vstar.copy() if v0 is None else _f64(v0, (self.n * 3,)).copy())
        gam = np.zeros(max(self.nc, 1) * 3)
        info = SolveInfo()
        st = lib().orc_solve_dense_newton(C.byref(self.s), C.byref(S), _d(v), _d(gam),
                                          C.byref(info))
        return v.reshape(self.n, 3), gam[:3 * self.nc].reshape(self.nc, 3), info, st


# --------------------------------------------------------------------------- substeps

class Sim:
    """Dense-grid FP64 simulation: orc_substep over a particle set.

    particles: dict with x[n,3], v[n,3], C[n,3,3], F[n,3,3], mass[n], vol[n],
    mat[n] (index into `materials`). materials: list of dicts {model, E, nu,
    friction_angle_deg}. grid: dict {dx, res, origin, gravity, bc_layers}.
    """

    def __init__(self, grid, openmp=False):
        self.L = lib(openmp)
        g = Grid()
        g.dx = float(grid["dx"])
        for i in range(3):
            g.res[i] = int(grid["res"][i])
            g.origin[i] = float(grid["origin"][i])
            g.gravity[i] = float(grid.get("gravity", (0.0, 0.0, -9.81))[i])
        g.bc_layers = int(grid.get("bc_layers", 3))
        self.grid = g
        self.h = self.L.orc_create(C.byref(g))

    def close(self):
        if self.h:
            self.L.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def state(particles):
        """Float64 working copy of a particle state."""
        n = len(particles["x"])
        return {
            "x": _f64(particles["x"], (n, 3)).copy(),
            "v": _f64(particles["v"], (n, 3)).copy(),
            "C": _f64(particles.get("C", np.zeros((n, 3, 3))), (n, 3, 3)).copy(),
            "F": _f64(particles.get("F", np.tile(np.eye(3), (n, 1, 1))), (n, 3, 3)).copy(),
            "mass": _f64(particles["mass"], (n,)).copy(),
            "vol": _f64(particles["vol"], (n,)).copy(),
            "mat": np.ascontiguousarray(np.asarray(particles["mat"], np.int32)),
        }

    def substep(self, st, materials, bodies, h, S, impulses=None):
        """Advance the float64 state `st` (from ``state``) by one substep in place."""
        n = len(st["x"])
        mats = (Material * max(len(materials), 1))()
        for i, mt in enumerate(materials):
            mats[i] = Material(int(mt["model"]), float(mt["E"]), float(mt["nu"]),
                               float(mt.get("friction_angle_deg", 30.0)))
        nb = len(bodies)
        bs = (Body * max(nb, 1))()
        for i, b in enumerate(bodies):
            bs[i] = b if isinstance(b, Body) else make_body(b)
        imp = impulses if impulses is not None else np.zeros(6 * max(nb, 1))
        info = SubstepInfo()
        st_code = self.L.orc_substep(self.h, n, _d(st["x"]), _d(st["v"]), _d(st["C"]), _d(st["F"]),
                                    _d(st["mass"]), _d(st["vol"]), _i(st["mat"]), len(materials),
                                    mats, nb, bs, float(h), C.byref(S), _d(imp), C.byref(info))
        return st_code, info

    def set_cloth(self, cloth):
        """The cloth meshes (dict from cloth_from_scene) for the following substeps."""
        tris = np.ascontiguousarray(cloth["tris"], np.int32).reshape(-1)
        dmi = _f64(cloth["Dm_inv"]).reshape(-1).copy()
        area = _f64(cloth["area"]).reshape(-1).copy()
        mat = np.ascontiguousarray(cloth["mat"], np.int32).reshape(-1)
        code = self.L.orc_set_cloth(self.h, len(area), _i(tris), _d(dmi), _d(area), _i(mat))
        assert code == OK
        self._cloth = (tris, dmi, area, mat)

    def set_pins(self, ids, v):
        """Pinned particles (orc_set_pins): ids [k] with prescribed velocities
        [k, 3] for the following substeps; empty ids release every pin."""
        ids = np.ascontiguousarray(ids, np.int32).reshape(-1)
        v = _f64(v).reshape(-1).copy()
        assert len(v) == 3 * len(ids)
        code = self.L.orc_set_pins(self.h, len(ids), _i(ids), _d(v))
        if code != OK:
            raise ValueError("orc_set_pins: bad pin set")
        self._pins = (ids, v)

    def last_grid(self):
        n = self.L.orc_last_grid(self.h, 0, None, None, None, None)
        ids = np.zeros(n, np.int32)
        m = np.zeros(n)
        vs = np.zeros(3 * n)
        v = np.zeros(3 * n)
        self.L.orc_last_grid(self.h, n, _i(ids), _d(m), _d(vs), _d(v))
        return ids, m, vs.reshape(n, 3), v.reshape(n, 3)

    def last_contacts(self):
        n = self.L.orc_last_contacts(self.h, 0, None, None, None, None, None)
        p = np.zeros(n, np.int32)
        b = np.zeros(n, np.int32)
        g = np.zeros(3 * n)
        phi = np.zeros(n)
        n0 = np.zeros(n)
        self.L.orc_last_contacts(self.h, n, _i(p), _i(b), _d(g), _d(phi), _d(n0))
        return p, b, g.reshape(n, 3), phi, n0


def cloth_rest(X0, X1, X2):
    """Rest shape of a cloth triangle: (Dm_inv [2, 2], area)."""
    dmi = np.zeros(4)
    area = np.zeros(1)
    lib().orc_cloth_rest(_d(_f64(X0, (3,))), _d(_f64(X1, (3,))), _d(_f64(X2, (3,))), _d(dmi),
                         _d(area))
    return dmi.reshape(2, 2), float(area[0])


def cloth_triangle(x0, x1, x2, Dm_inv, vol, mu, lam):
    """Membrane energy of a cloth triangle of rest volume vol and the forces on
    its vertices [3, 3]."""
    f = np.zeros(9)
    e = lib().orc_cloth_triangle(_d(_f64(x0, (3,))), _d(_f64(x1, (3,))), _d(_f64(x2, (3,))),
                                 _d(_f64(Dm_inv, (4,))), float(vol), float(mu), float(lam), _d(f))
    return e, f.reshape(3, 3)


def cloth_from_scene(scene):
    """The cloth meshes of a scene's groups (those with "tris"), in global
    particle ids, with rest shapes from the groups' float32 rest positions and
    rest volumes = rest area * the group's thickness."""
    tris, dmi, area, mat = [], [], [], []
    offset = 0
    for gi, g in enumerate(scene["groups"]):
        x = np.asarray(g["x"], np.float32).astype(np.float64)
        if "tris" in g:
            rest = np.asarray(g.get("rest", g["x"]), np.float32).astype(np.float64)
            for t in np.asarray(g["tris"], np.int64).reshape(-1, 3):
                d, a = cloth_rest(rest[t[0]], rest[t[1]], rest[t[2]])
                tris.append(t + offset)
                dmi.append(d.reshape(4))
                area.append(a * float(np.float32(g["thickness"])))
                mat.append(gi)
        offset += len(x)
    if not tris:
        return None
    return {"tris": np.array(tris, np.int32), "Dm_inv": np.array(dmi), "area": np.array(area),
            "mat": np.array(mat, np.int32)}


def pins_from_scene(scene):
    """The pinned particles of a scene's groups (a group's "pins": {"ids":
    local indices, "v": [k, 3] prescribed velocities}) in global particle ids,
    or None."""
    ids, vel = [], []
    offset = 0
    for g in scene["groups"]:
        if "pins" in g:
            ids.append(np.asarray(g["pins"]["ids"], np.int64).reshape(-1) + offset)
            vel.append(np.asarray(g["pins"]["v"], np.float64).reshape(-1, 3))
        offset += len(g["x"])
    if not ids:
        return None
    return np.concatenate(ids).astype(np.int32), np.concatenate(vel)


def advance_kinematic(bodies, dt):
    """Async splitting: kinematic bodies move with their frozen velocity after a
    time step (Eq. (3)-(4)). Returns new body dicts."""
    nb = len(bodies)
    bs = (Body * max(nb, 1))()
    for i, b in enumerate(bodies):
        bs[i] = make_body(b)
    lib().orc_advance_kinematic(nb, bs, float(dt))
    return [body_dict(bs[i]) for i in range(nb)]


def rollout(scene, steps, S, materials=None, bodies=None, state=None, substeps=None,
            dynamics=None, with_bodies=False):
    """Asynchronous time splitting (Sec. IV-A, Eq. (3)-(4)): `steps` rigid time
    steps of `substeps` (default scene["substeps"]; a sequence gives each
    step its own count) MPM substeps each, the
    rigid bodies frozen within a step; after it the kinematic ones advance by
    substeps*h and the dynamic ones (`dynamics`: body index -> dict as
    make_dynamics; their kinematic flag is ignored) take the rigid step of
    Eq. (3) with the step's accumulated impulses. Oracle state, materials and
    bodies default to the scene's (from_scene, bodies_from_scene); returns
    the final FP64 state, the first non-OK substep status (OK if none) and,
    with with_bodies, the final bodies."""
    st0, mats0 = from_scene(scene)
    st = Sim.state(st0 if state is None else state)
    mats = mats0 if materials is None else materials
    bds = bodies_from_scene(scene) if bodies is None else [dict(b) for b in bodies]
    n_sub = scene["substeps"] if substeps is None else substeps
    per_step = list(n_sub) if hasattr(n_sub, "__len__") else [n_sub] * steps
    dyn = dynamics or {}
    grav = scene["grid"].get("gravity", (0.0, 0.0, -9.81))
    sim = Sim(scene["grid"])
    cloth = cloth_from_scene(scene)
    if cloth is not None:
        sim.set_cloth(cloth)
    pins = pins_from_scene(scene)
    if pins is not None:
        sim.set_pins(*pins)
    code = OK
    try:
        for n_sub in per_step[:steps]:
            imp = np.zeros(6 * max(len(bds), 1))
            for _ in range(n_sub):
                c, _ = sim.substep(st, mats, bds, scene["h"], S, imp)
                if code == OK and c != OK:
                    code = c
            nxt = advance_kinematic([dict(b, kinematic=0) if i in dyn else b
                                     for i, b in enumerate(bds)], n_sub * scene["h"])
            for i, d in dyn.items():
                nxt[i] = rigid_dynamics_step(bds[i], d, grav, imp[6 * i:6 * i + 6], n_sub * scene["h"])
                nxt[i]["kinematic"] = bds[i].get("kinematic", 0)
            for i in range(len(nxt)):
                nxt[i]["shape"] = int(bds[i]["shape"])
            bds = nxt
    finally:
        sim.close()
    return (st, code, bds) if with_bodies else (st, code)


def make_dynamics(dyn):
    """dict(mass, inertia[3], force[3], torque[3], dof_mask, gravity) -> Dynamics."""
    d = Dynamics()
    d.mass = float(dyn["mass"])
    for key in ("inertia", "force", "torque"):
        arr = getattr(d, key)
        val = np.asarray(dyn.get(key, [0, 0, 0]), np.float64).reshape(3)
        for i in range(3):
            arr[i] = float(val[i])
    d.dof_mask = int(dyn.get("dof_mask", 63))
    d.gravity = int(dyn.get("gravity", 1))
    return d


def rigid_dynamics_step(body, dyn, gravity, impulse, dt):
    """Eq. (3) for one dynamic body over a time step dt with the step's impulse
    on the body and its moment about the body origin (impulse[6], world).
    Returns the new body dict."""
    b = make_body(body)
    d = make_dynamics(dyn)
    lib().orc_rigid_dynamics_step(C.byref(b), C.byref(d), _d(_f64(gravity, (3,))),
                                  _d(_f64(impulse, (6,))), float(dt))
    out = body_dict(b)
    out["shape"] = int(body["shape"])
    return out


def from_scene(scene):
    """Flatten a scene's particle groups into an oracle state and material list.

    Particle mass is rho * rest volume; C = 0 and F = I at creation.
    """
    xs, vs, mass, vol, mat, materials = [], [], [], [], [], []
    for gi, g in enumerate(scene["groups"]):
        n = len(g["x"])
        xs.append(np.asarray(g["x"], np.float64))
        vs.append(np.asarray(g["v"], np.float64))
        # the rest volume and density travel as float32 through the C-ABI
        V = float(np.float32(g["vol"]))
        rho = float(np.float32(g["material"]["rho"]))
        vol.append(np.full(n, V))
        mass.append(np.full(n, rho * V))
        mat.append(np.full(n, gi, np.int32))
        m = g["material"]
        materials.append({"model": int(m["model"]), "E": float(np.float32(m["E"])),
                          "nu": float(np.float32(m["nu"])),
                          "friction_angle_deg": float(np.float32(m.get("friction_angle_deg", 0.0)))})
    n = sum(len(a) for a in xs)
    st = {"x": np.concatenate(xs), "v": np.concatenate(vs), "C": np.zeros((n, 3, 3)),
          "F": np.tile(np.eye(3), (n, 1, 1)), "mass": np.concatenate(mass),
          "vol": np.concatenate(vol), "mat": np.concatenate(mat)}
    return Sim.state(st), materials


def bodies_from_scene(scene, f32=True):
    """Scene bodies, optionally rounded through float32 as the C-ABI carries them."""
    out = []
    for b in scene["bodies"]:
        c = dict(b)
        if f32:
            for key in ("params", "R", "p", "omega", "v"):
                c[key] = np.asarray(b[key], np.float32).astype(np.float64)
            for key in ("mu", "k", "d"):
                c[key] = float(np.float32(b[key]))
        out.append(c)
    return out
