"""Thin Python binding of the C ABI in ``include/mpmcr.h`` (``libmpmcr.so``).

Argument marshalling only: every step of the substep runs in the library's
CUDA kernels. Functions carry the C names (``mpm_create``, ``mpm_step``, ...);
``Sim`` bundles them for convenience. Device buffers may be passed as torch
CUDA tensors (``mem_kind=MEM_DEVICE``); host buffers as numpy arrays.

There is no fallback: if the library is missing or fails to load, importing
this module raises.
"""
import ctypes as C
import os

import numpy as np

from . import scenes

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpmcr.so")

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_CAPACITY, ERR_NOT_CONVERGED, ERR_OUT_OF_DOMAIN, \
    ERR_NAN, ERR_STATE, ERR_TIMEOUT, ERR_LINE_SEARCH = range(11)
STATUS_NAMES = ["MPM_OK", "MPM_ERR_INVALID_ARG", "MPM_ERR_CUDA", "MPM_ERR_OOM", "MPM_ERR_CAPACITY",
                "MPM_ERR_NOT_CONVERGED", "MPM_ERR_OUT_OF_DOMAIN", "MPM_ERR_NAN", "MPM_ERR_STATE",
                "MPM_ERR_TIMEOUT", "MPM_ERR_LINE_SEARCH"]
MEM_HOST, MEM_DEVICE = 0, 1
OPT_PROFILE, OPT_SORT_EVERY, OPT_P2G_CHUNK, OPT_GRAPHS, OPT_SOLVE_BLOCKS = 1, 2, 3, 4, 5
OPT_TAPE_SOLUTIONS = 7
OPT_CLUSTER_CONTACTS = 8
OPT_CLUSTER_BLOCKS = 9
OPT_P2G_FORM = 10
P2G_GATHER, P2G_SCATTER = 0, 1
OPT_TEST_BARRIER_TIMEOUT = 6
BATCH_OPT_GRAPHS, BATCH_OPT_P2G_CHUNK, BATCH_OPT_G2P_THREADS, BATCH_OPT_GRID_PARTICLES = 1, 2, 3, 4
BATCH_OPT_SOLVE_BLOCKS = 5
PHASES = ["sort", "p2g", "grid", "solve", "g2p"]


class GridSpec(C.Structure):
    _fields_ = [("dx", C.c_double), ("res", C.c_int32 * 3), ("origin", C.c_double * 3),
                ("gravity", C.c_double * 3), ("bc_layers", C.c_int32),
                ("max_particles", C.c_int64), ("max_contacts", C.c_int64),
                ("max_blocks", C.c_int64)]


class Material(C.Structure):
    _fields_ = [("model", C.c_int32), ("E", C.c_float), ("nu", C.c_float), ("rho", C.c_float),
                ("friction_angle_deg", C.c_float)]


class RigidBody(C.Structure):
    _fields_ = [("shape", C.c_int32), ("params", C.c_float * 4), ("R", C.c_float * 9),
                ("p", C.c_float * 3), ("omega", C.c_float * 3), ("v", C.c_float * 3),
                ("mu", C.c_float), ("k", C.c_float), ("d", C.c_float), ("kinematic", C.c_int32)]


class RigidDynamics(C.Structure):
    _fields_ = [("mass", C.c_float), ("inertia", C.c_float * 3), ("force", C.c_float * 3),
                ("torque", C.c_float * 3), ("dof_mask", C.c_int32), ("gravity", C.c_int32)]


class SolverParams(C.Structure):
    _fields_ = [("eps_r", C.c_double), ("eps_a", C.c_double), ("max_iters", C.c_int32),
                ("eps_s", C.c_float), ("ls_rel_tol", C.c_float), ("ls_max_iters", C.c_int32)]


class StepStats(C.Structure):
    _fields_ = [("substeps", C.c_int32), ("iters_total", C.c_int32), ("iters_max", C.c_int32),
                ("ls_evals_total", C.c_int32), ("contacts_max", C.c_int32),
                ("active_blocks_max", C.c_int32), ("contacts_total", C.c_int64),
                ("residual_max", C.c_double), ("status_bits", C.c_int32),
                ("p2g_global_chunks", C.c_int32), ("solve_us", C.c_float * 5),
                ("ls_split_substeps", C.c_int32), ("cluster_substeps", C.c_int32),
                ("contact_nodes_max", C.c_int32)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["solve_us"] = list(self.solve_us)
        return d


MAX_BODIES = 16  # rigid bodies per context


class AdjointParams(C.Structure):
    _fields_ = [("eps_r", C.c_double), ("max_iters", C.c_int32)]


class AdjointStats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("residual", C.c_float), ("contacts", C.c_int32),
                ("contact_nodes", C.c_int32)]


class BackwardStats(C.Structure):
    _fields_ = [("steps", C.c_int32), ("substeps", C.c_int32), ("last_iters", C.c_int32),
                ("last_residual", C.c_float)]


_vp = C.c_void_p
_fp = C.POINTER(C.c_float)
_dp = C.POINTER(C.c_double)
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)

# name -> (argtypes) ; every entry point returns mpm_status except mpm_last_error
SIGNATURES = {
    "mpm_create": [C.POINTER(GridSpec), _vp, C.POINTER(_vp)],
    "mpm_destroy": [_vp],
    "mpm_last_error": [_vp],
    "mpm_add_particles": [_vp, C.c_int64, _vp, _vp, C.c_float, C.POINTER(Material), C.c_int32,
                          _i64p],
    "mpm_num_particles": [_vp, _i64p],
    "mpm_add_cloth": [_vp, C.c_int64, _vp, _vp, C.c_int64, _i32p, C.c_float, C.POINTER(Material),
                      C.c_int32, _i64p],
    "mpm_set_pins": [_vp, C.c_int64, _i64p, _fp],
    "mpm_set_particles": [_vp, _vp, _vp, _vp, _vp, C.c_int32],
    "mpm_get_particles": [_vp, _vp, _vp, _vp, _vp, C.c_int32],
    "mpm_set_rigid_bodies": [_vp, C.c_int32, C.POINTER(RigidBody)],
    "mpm_get_rigid_bodies": [_vp, C.c_int32, C.POINTER(RigidBody)],
    "mpm_set_rigid_dynamics": [_vp, C.c_int32, C.POINTER(RigidDynamics)],
    "mpm_step": [_vp, C.c_double, C.c_int32, C.POINTER(SolverParams), C.POINTER(StepStats)],
    "mpm_get_rigid_impulses": [_vp, _dp, C.c_int32],
    "mpm_get_grid": [_vp, C.c_int64, _i64p, _i32p, _fp, _fp, _fp],
    "mpm_get_contacts": [_vp, C.c_int64, _i64p, _i32p, _i32p, _fp, _fp, _fp],
    "mpm_get_grid_noalloc": [_vp, C.c_int64, _i64p, _i32p, _fp, _fp, _fp],
    "mpm_contact_adjoint": [_vp, C.c_int32, C.c_int64, _vp, _vp, _vp, C.c_int64, _vp, _vp,
                            C.POINTER(AdjointParams), C.POINTER(AdjointStats)],
    "mpm_set_material": [_vp, C.c_int32, C.POINTER(Material)],
    "mpm_tape_begin": [_vp],
    "mpm_tape_end": [_vp],
    "mpm_backward": [_vp, C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                     C.POINTER(AdjointParams), C.POINTER(BackwardStats)],
    "mpm_synchronize": [_vp],
    "mpm_set_option": [_vp, C.c_int32, C.c_int64],
    "mpm_get_phase_times": [_vp, _dp, _i64p, C.c_int32],
    "mpm_batch_create": [C.POINTER(_vp), C.c_int32, C.POINTER(_vp)],
    "mpm_batch_step": [_vp, C.c_double, C.c_int32, C.POINTER(SolverParams)],
    "mpm_batch_sort": [_vp],
    "mpm_batch_synchronize": [_vp, _i32p, C.POINTER(StepStats)],
    "mpm_batch_set_option": [_vp, C.c_int32, C.c_int64],
    "mpm_batch_last_error": [_vp],
    "mpm_batch_destroy": [_vp],
}
_RESTYPES = {"mpm_last_error": C.c_char_p, "mpm_batch_last_error": C.c_char_p,
             "mpm_batch_destroy": None}


def load(path=LIB_PATH):
    """Load libmpmcr.so and declare the C signatures. Raises if it is missing."""
    if not os.path.exists(path):
        raise ImportError("libmpmcr.so not found at %s: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    L = C.CDLL(path)
    for name, args in SIGNATURES.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = _RESTYPES.get(name, C.c_int)
    return L


lib = load()


class MpmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[code] if 0 <= code < len(STATUS_NAMES) else code,
                                     msg))
        self.code = code


def _check(ctx, code):
    if code != OK:
        msg = lib.mpm_last_error(ctx)
        raise MpmError(code, msg.decode() if msg else "")
    return code


# ---------------------------------------------------------------- C-named calls

def mpm_create(spec, stream=None):
    out = _vp()
    _check(None, lib.mpm_create(C.byref(spec), stream, C.byref(out)))
    return out


def mpm_destroy(ctx):
    return lib.mpm_destroy(ctx)


def mpm_last_error(ctx):
    return lib.mpm_last_error(ctx).decode()


def _ptr(a):
    """(pointer, mem_kind, keepalive) for a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None, None, None
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.float32)
        return a.ctypes.data, MEM_HOST, a
    # torch tensor
    if a.dtype.is_floating_point and a.element_size() != 4:
        raise TypeError("float32 tensors required")
    if not a.is_contiguous():
        raise ValueError("contiguous tensors required")
    return a.data_ptr(), (MEM_DEVICE if a.is_cuda else MEM_HOST), a


def mpm_add_particles(ctx, x, v, volume, material):
    n = len(x)
    px, kx, kx_keep = _ptr(x)
    pv, kv, kv_keep = _ptr(v)
    if kx != kv:
        raise ValueError("x and v must live in the same memory")
    first = C.c_int64()
    _check(ctx, lib.mpm_add_particles(ctx, n, px, pv, float(volume), C.byref(material), kx,
                                      C.byref(first)))
    return first.value


def mpm_add_cloth(ctx, x, v, tris, thickness, material):
    """A triangle mesh of cloth: vertex positions / velocities [n, 3] (numpy or
    CUDA tensors), triangles [m, 3] int (host), thickness [m]; returns the first
    vertex's particle id."""
    n = len(x)
    px, kx, kx_keep = _ptr(x)
    pv, kv, kv_keep = _ptr(v)
    if kx != kv:
        raise ValueError("x and v must live in the same memory")
    t = np.ascontiguousarray(np.asarray(tris, np.int32).reshape(-1, 3))
    first = C.c_int64()
    _check(ctx, lib.mpm_add_cloth(ctx, n, px, pv, len(t), t.ctypes.data_as(_i32p), float(thickness),
                                  C.byref(material), kx, C.byref(first)))
    return first.value


def mpm_set_pins(ctx, ids, v):
    """Pinned particles: ids [k] (host) with prescribed velocities [k, 3]; an
    empty set releases every pin."""
    ids = np.ascontiguousarray(np.asarray(ids, np.int64).reshape(-1))
    v = np.ascontiguousarray(np.asarray(v, np.float32).reshape(-1, 3))
    if len(v) != len(ids):
        raise ValueError("one velocity per pinned particle")
    if len(ids) == 0:
        _check(ctx, lib.mpm_set_pins(ctx, 0, None, None))
        return
    _check(ctx, lib.mpm_set_pins(ctx, len(ids), ids.ctypes.data_as(_i64p),
                                 v.ctypes.data_as(_fp)))


def mpm_num_particles(ctx):
    n = C.c_int64()
    _check(ctx, lib.mpm_num_particles(ctx, C.byref(n)))
    return n.value


def mpm_set_particles(ctx, x=None, v=None, Cm=None, F=None):
    ptrs = [_ptr(a) for a in (x, v, Cm, F)]
    kinds = {k for _, k, _ in ptrs if k is not None}
    if len(kinds) > 1:
        raise ValueError("all buffers must live in the same memory")
    kind = kinds.pop() if kinds else MEM_HOST
    _check(ctx, lib.mpm_set_particles(ctx, *[p for p, _, _ in ptrs], kind))


def mpm_get_particles(ctx, x=None, v=None, Cm=None, F=None, mem_kind=MEM_HOST):
    ptrs = [(a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr()) if a is not None else None
            for a in (x, v, Cm, F)]
    _check(ctx, lib.mpm_get_particles(ctx, *ptrs, mem_kind))


def mpm_set_rigid_bodies(ctx, bodies):
    arr = (RigidBody * max(len(bodies), 1))()
    for i, b in enumerate(bodies):
        arr[i] = b if isinstance(b, RigidBody) else make_body(b)
    _check(ctx, lib.mpm_set_rigid_bodies(ctx, len(bodies), arr))


def make_dynamics(dyn):
    """dict(mass, inertia[3], force[3], torque[3], dof_mask, gravity) -> RigidDynamics."""
    d = RigidDynamics()
    d.mass = float(dyn["mass"])
    for key in ("inertia", "force", "torque"):
        val = np.asarray(dyn.get(key, [0.0, 0.0, 0.0]), np.float64).reshape(3)
        arr = getattr(d, key)
        for i in range(3):
            arr[i] = float(val[i])
    d.dof_mask = int(dyn.get("dof_mask", 63))
    d.gravity = int(dyn.get("gravity", 1))
    return d


def mpm_set_rigid_dynamics(ctx, index, dyn):
    _check(ctx, lib.mpm_set_rigid_dynamics(ctx, int(index),
                                           C.byref(make_dynamics(dyn)) if dyn is not None else None))


def mpm_get_rigid_bodies(ctx, n):
    arr = (RigidBody * max(n, 1))()
    _check(ctx, lib.mpm_get_rigid_bodies(ctx, n, arr))
    return [arr[i] for i in range(n)]


def mpm_step(ctx, h, n_substeps, solver=None, want_stats=True):
    st = StepStats()
    code = lib.mpm_step(ctx, float(h), int(n_substeps), C.byref(solver) if solver is not None else None,
                        C.byref(st) if want_stats else None)
    return code, (st if want_stats else None)


def mpm_get_rigid_impulses(ctx, n_bodies, reset=False):
    out = np.zeros(6 * max(n_bodies, 1))
    _check(ctx, lib.mpm_get_rigid_impulses(ctx, out.ctypes.data_as(_dp), int(reset)))
    return out[:6 * n_bodies].reshape(n_bodies, 6)


def mpm_get_grid(ctx):
    count = C.c_int64()
    _check(ctx, lib.mpm_get_grid(ctx, 0, C.byref(count), None, None, None, None))
    n = count.value
    ids = np.zeros(max(n, 1), np.int32)
    m = np.zeros(max(n, 1), np.float32)
    vs = np.zeros((max(n, 1), 3), np.float32)
    v = np.zeros((max(n, 1), 3), np.float32)
    _check(ctx, lib.mpm_get_grid(ctx, n, C.byref(count), ids.ctypes.data_as(_i32p),
                                 m.ctypes.data_as(_fp), vs.ctypes.data_as(_fp), v.ctypes.data_as(_fp)))
    n = min(n, count.value)
    order = np.argsort(ids[:n], kind="stable")
    return ids[:n][order], m[:n][order], vs[:n][order], v[:n][order]


def mpm_get_contacts(ctx):
    count = C.c_int64()
    _check(ctx, lib.mpm_get_contacts(ctx, 0, C.byref(count), None, None, None, None, None))
    n = count.value
    p = np.zeros(max(n, 1), np.int32)
    b = np.zeros(max(n, 1), np.int32)
    g = np.zeros((max(n, 1), 3), np.float32)
    phi = np.zeros(max(n, 1), np.float32)
    n0 = np.zeros(max(n, 1), np.float32)
    _check(ctx, lib.mpm_get_contacts(ctx, n, C.byref(count), p.ctypes.data_as(_i32p),
                                     b.ctypes.data_as(_i32p), g.ctypes.data_as(_fp),
                                     phi.ctypes.data_as(_fp), n0.ctypes.data_as(_fp)))
    return p[:n], b[:n], g[:n], phi[:n], n0[:n]


def mpm_contact_adjoint(ctx, node_ids, vbar, n_contacts=None, n_bodies=0, eps_r=1e-5,
                        max_iters=1000, check=True):
    """Adjoint of the last substep's contact solve (see include/mpmcr.h).

    node_ids [n] int32 and vbar [n, 3] float32, both numpy (host) or both CUDA
    tensors (device, outputs then CUDA tensors too). Returns (vstar_bar [n, 3],
    contact_bar [n_contacts, 4], body_bar [n_bodies, 7] float64, stats, status);
    n_contacts None reads the contact count first. body_bar rows are the bodies
    of the last mpm_step."""
    device = not isinstance(vbar, np.ndarray)
    if n_contacts is None:
        count = C.c_int64()
        _check(ctx, lib.mpm_get_contacts(ctx, 0, C.byref(count), None, None, None, None, None))
        n_contacts = count.value
    n = len(node_ids)
    if device:
        import torch
        if node_ids.dtype != torch.int32 or vbar.dtype != torch.float32:
            raise TypeError("int32 ids and float32 vbar required")
        ids_t, vb_t = node_ids.contiguous(), vbar.contiguous()
        vsb = torch.empty((n, 3), dtype=torch.float32, device=vbar.device)
        cbar = torch.zeros((max(n_contacts, 1), 4), dtype=torch.float32, device=vbar.device)
        bbar = torch.zeros((MAX_BODIES, 7), dtype=torch.float64, device=vbar.device)
        ptrs = (ids_t.data_ptr(), vb_t.data_ptr(), vsb.data_ptr(), cbar.data_ptr(), bbar.data_ptr())
        kind = MEM_DEVICE
    else:
        ids_t = np.ascontiguousarray(node_ids, dtype=np.int32)
        vb_t = np.ascontiguousarray(vbar, dtype=np.float32).reshape(n, 3)
        vsb = np.zeros((max(n, 1), 3), np.float32)
        cbar = np.zeros((max(n_contacts, 1), 4), np.float32)
        bbar = np.zeros((MAX_BODIES, 7), np.float64)
        ptrs = (ids_t.ctypes.data, vb_t.ctypes.data, vsb.ctypes.data, cbar.ctypes.data,
                bbar.ctypes.data)
        kind = MEM_HOST
    params = AdjointParams(float(eps_r), int(max_iters))
    st = AdjointStats()
    code = lib.mpm_contact_adjoint(ctx, kind, n, ptrs[0], ptrs[1], ptrs[2], n_contacts, ptrs[3],
                                   ptrs[4], C.byref(params), C.byref(st))
    if check:
        _check(ctx, code)
    return vsb[:n], cbar[:n_contacts], bbar[:n_bodies], st, code


def mpm_set_material(ctx, group, material):
    m = material if isinstance(material, Material) else make_material(material)
    _check(ctx, lib.mpm_set_material(ctx, int(group), C.byref(m)))


def mpm_tape_begin(ctx):
    _check(ctx, lib.mpm_tape_begin(ctx))


def mpm_tape_end(ctx):
    _check(ctx, lib.mpm_tape_end(ctx))


def mpm_backward(ctx, n, n_groups, n_bodies, x_bar=None, v_bar=None, C_bar=None, F_bar=None,
                 eps_r=1e-6, max_iters=2000, check=True, body_state_bar=None):
    """Reverse pass over the recorded steps (see include/mpmcr.h).

    body_state_bar: optional [n_bodies, 12] cotangent of the bodies' final
    state (dL/dv, dL/dp, dL/domega, dL/dtheta).

    The four cotangents are numpy arrays (host) or CUDA tensors (device, all
    alike; None for zero). Returns dict(x, v, C, F: adjoints of the first
    recorded state, E, nu: [n_groups], mu: [n_bodies], body_v, body_p, body_w,
    body_R: [n_bodies, 3] (dL/d linear velocity, initial position, angular
    velocity, initial orientation as a world-frame rotation), stats, status)."""
    given = [a for a in (x_bar, v_bar, C_bar, F_bar) if a is not None]
    device = bool(given) and not isinstance(given[0], np.ndarray)
    shapes = ((n, 3), (n, 3), (n, 3, 3), (n, 3, 3))
    if device:
        import torch
        dev = given[0].device
        ins = [None if a is None else a.to(torch.float32).contiguous() for a in (x_bar, v_bar, C_bar, F_bar)]
        outs = [torch.zeros(sh, dtype=torch.float32, device=dev) for sh in shapes]
        iptr = [None if a is None else a.data_ptr() for a in ins]
        optr = [o.data_ptr() for o in outs]
        kind = MEM_DEVICE
    else:
        ins = [None if a is None else np.ascontiguousarray(a, np.float32).reshape(sh)
               for a, sh in zip((x_bar, v_bar, C_bar, F_bar), shapes)]
        outs = [np.zeros(sh, np.float32) for sh in shapes]
        iptr = [None if a is None else a.ctypes.data for a in ins]
        optr = [o.ctypes.data for o in outs]
        kind = MEM_HOST
    mat = np.zeros(2 * max(n_groups, 1))
    bodyb = np.zeros((max(n_bodies, 1), 13))
    st = BackwardStats()
    params = AdjointParams(float(eps_r), int(max_iters))
    sbar = None
    if body_state_bar is not None:
        sbar = np.ascontiguousarray(body_state_bar, np.float64).reshape(n_bodies, 12)
    code = lib.mpm_backward(ctx, kind, *iptr, sbar.ctypes.data if sbar is not None else None, *optr,
                            mat.ctypes.data, bodyb.ctypes.data, C.byref(params), C.byref(st))
    if check:
        _check(ctx, code)
    return {"x": outs[0], "v": outs[1], "C": outs[2], "F": outs[3],
            "E": mat[0:2 * n_groups:2].copy(), "nu": mat[1:2 * n_groups:2].copy(),
            "mu": bodyb[:n_bodies, 0].copy(), "body_v": bodyb[:n_bodies, 1:4].copy(),
            "body_p": bodyb[:n_bodies, 4:7].copy(), "body_w": bodyb[:n_bodies, 7:10].copy(),
            "body_R": bodyb[:n_bodies, 10:13].copy(), "stats": st, "status": code}


def mpm_synchronize(ctx):
    return lib.mpm_synchronize(ctx)


def mpm_set_option(ctx, option, value):
    _check(ctx, lib.mpm_set_option(ctx, int(option), int(value)))


def mpm_get_phase_times(ctx, reset=False):
    ms = np.zeros(len(PHASES))
    n = np.zeros(len(PHASES), np.int64)
    _check(ctx, lib.mpm_get_phase_times(ctx, ms.ctypes.data_as(_dp), n.ctypes.data_as(_i64p),
                                        int(reset)))
    return dict(zip(PHASES, ms)), dict(zip(PHASES, n))


# ---------------------------------------------------------------- conversions

def grid_spec(grid, max_particles, max_contacts):
    s = GridSpec()
    s.dx = float(grid["dx"])
    for i in range(3):
        s.res[i] = int(grid["res"][i])
        s.origin[i] = float(grid["origin"][i])
        s.gravity[i] = float(grid.get("gravity", (0.0, 0.0, -9.81))[i])
    s.bc_layers = int(grid.get("bc_layers", 3))
    s.max_particles = int(max_particles)
    s.max_contacts = int(max_contacts)
    s.max_blocks = int(grid.get("max_blocks", 0))  # block-sparse pool (0: dense)
    return s


def make_material(m):
    return Material(int(m["model"]), float(m["E"]), float(m["nu"]), float(m["rho"]),
                    float(m.get("friction_angle_deg", 0.0)))


def make_body(b):
    r = RigidBody()
    r.shape = int(b["shape"])
    prm = np.asarray(b.get("params", [0, 0, 0, 0]), np.float32).ravel()
    for i in range(4):
        r.params[i] = float(prm[i]) if i < len(prm) else 0.0
    R = np.asarray(b.get("R", np.eye(3)), np.float32).reshape(9)
    for i in range(9):
        r.R[i] = float(R[i])
    for key in ("p", "omega", "v"):
        arr = getattr(r, key)
        val = np.asarray(b.get(key, [0, 0, 0]), np.float32).reshape(3)
        for i in range(3):
            arr[i] = float(val[i])
    r.mu = float(b.get("mu", 0.0))
    r.k = float(b.get("k", scenes.CONTACT_K))
    r.d = float(b.get("d", scenes.CONTACT_D))
    r.kinematic = int(b.get("kinematic", 0))
    return r


def body_dict(r):
    return {"shape": r.shape, "params": np.array(r.params[:], np.float64),
            "R": np.array(r.R[:], np.float64).reshape(3, 3), "p": np.array(r.p[:], np.float64),
            "omega": np.array(r.omega[:], np.float64), "v": np.array(r.v[:], np.float64),
            "mu": r.mu, "k": r.k, "d": r.d, "kinematic": r.kinematic}


def solver_params(eps_r=5e-2, eps_a=np.finfo(np.float64).eps, max_iters=1000, eps_s=scenes.EPS_S,
                  ls_rel_tol=1e-3, ls_max_iters=50):
    return SolverParams(eps_r, eps_a, max_iters, eps_s, ls_rel_tol, ls_max_iters)


class Sim:
    """One simulation context on the current CUDA device."""

    def __init__(self, scene, max_particles=None, max_contacts=None, stream=None):
        n = scenes.n_particles(scene)
        self.scene = scene
        self.max_particles = int(max_particles or max(n, 1))
        self.max_contacts = int(max_contacts or max(4 * n, 1024))
        spec = grid_spec(scene["grid"], self.max_particles, self.max_contacts)
        # the context's work runs on one stream; by default a dedicated torch
        # stream (kept alive here) so that callers can order torch work and
        # CUDA events against it
        self.torch_stream = None
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    self.torch_stream = torch.cuda.Stream()
                    stream = self.torch_stream.cuda_stream
            except ImportError:  # torch is optional for the binding
                stream = None
        self.ctx = mpm_create(spec, stream)
        try:
            import torch
            self.device = torch.device("cuda", torch.cuda.current_device())
        except (ImportError, RuntimeError, AssertionError):
            self.device = None
        for g in scene["groups"]:
            if "tris" in g:  # a cloth mesh
                mpm_add_cloth(self.ctx, np.asarray(g["x"], np.float32),
                              np.asarray(g["v"], np.float32), g["tris"], g["thickness"],
                              make_material(g["material"]))
            else:
                mpm_add_particles(self.ctx, np.asarray(g["x"], np.float32),
                                  np.asarray(g["v"], np.float32), g["vol"],
                                  make_material(g["material"]))
        pins, offset = ([], []), 0
        for g in scene["groups"]:
            if "pins" in g:  # pinned particles of the group (local ids)
                pins[0].append(np.asarray(g["pins"]["ids"], np.int64).reshape(-1) + offset)
                pins[1].append(np.asarray(g["pins"]["v"], np.float32).reshape(-1, 3))
            offset += len(g["x"])
        if pins[0]:
            mpm_set_pins(self.ctx, np.concatenate(pins[0]), np.concatenate(pins[1]))
        self.n_bodies = len(scene["bodies"])
        mpm_set_rigid_bodies(self.ctx, scene["bodies"])
        # the dynamics set on the current bodies (mpm_set_rigid_bodies clears them)
        self.dynamics = {}

    def close(self):
        if getattr(self, "ctx", None):
            mpm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n(self):
        return mpm_num_particles(self.ctx)

    def step(self, h=None, n_substeps=None, solver=None, stats=True, check=True):
        h = self.scene["h"] if h is None else h
        n_substeps = self.scene["substeps"] if n_substeps is None else n_substeps
        code, st = mpm_step(self.ctx, h, n_substeps, solver, want_stats=stats)
        if check:
            _check(self.ctx, code)
        return (code, st) if not check else st

    def get_particles(self):
        n = self.n
        x = np.zeros((n, 3), np.float32)
        v = np.zeros((n, 3), np.float32)
        Cm = np.zeros((n, 3, 3), np.float32)
        F = np.zeros((n, 3, 3), np.float32)
        mpm_get_particles(self.ctx, x, v, Cm, F)
        return {"x": x, "v": v, "C": Cm, "F": F}

    def set_particles(self, x=None, v=None, Cm=None, F=None):
        mpm_set_particles(self.ctx, x, v, Cm, F)

    def read_particles(self, x=None, v=None, Cm=None, F=None):
        """Fill the given arrays (numpy: host; CUDA tensors: device, all
        alike) with the particle state in id order."""
        given = [a for a in (x, v, Cm, F) if a is not None]
        kind = MEM_HOST if not given or isinstance(given[0], np.ndarray) else MEM_DEVICE
        mpm_get_particles(self.ctx, x, v, Cm, F, mem_kind=kind)

    def set_pins(self, ids, v):
        mpm_set_pins(self.ctx, ids, v)

    def set_bodies(self, bodies):
        """Replace the bodies; like mpm_set_rigid_bodies this clears every
        body's dynamics."""
        mpm_set_rigid_bodies(self.ctx, bodies)
        self.n_bodies = len(bodies)
        self.dynamics = {}

    def set_dynamics(self, index, dyn):
        """Make body `index` dynamic (dict as make_dynamics) or, with None, not."""
        mpm_set_rigid_dynamics(self.ctx, index, dyn)
        if dyn is None:
            self.dynamics.pop(int(index), None)
        else:
            self.dynamics[int(index)] = dict(dyn)

    def bodies(self):
        return [body_dict(b) for b in mpm_get_rigid_bodies(self.ctx, self.n_bodies)]

    def impulses(self, reset=False):
        return mpm_get_rigid_impulses(self.ctx, self.n_bodies, reset)

    def grid(self):
        return mpm_get_grid(self.ctx)

    def contacts(self):
        return mpm_get_contacts(self.ctx)

    def tape_begin(self):
        """Record a checkpoint at every following step (mpm_tape_begin)."""
        mpm_tape_begin(self.ctx)

    def tape_end(self):
        mpm_tape_end(self.ctx)

    def backward(self, x_bar=None, v_bar=None, C_bar=None, F_bar=None, eps_r=1e-6,
                 max_iters=2000, check=True, body_state_bar=None):
        """Adjoint of the recorded rollout for the cotangents of its final
        state (mpm_backward): dL/d(first recorded state), dL/dE, dL/dnu per
        group, and per body dL/dmu and the gradients of its velocities and
        pose."""
        return mpm_backward(self.ctx, self.n, len(self.scene["groups"]), self.n_bodies,
                            x_bar, v_bar, C_bar, F_bar, eps_r, max_iters, check, body_state_bar)

    def contact_adjoint(self, node_ids, vbar, eps_r=1e-5, max_iters=1000, check=True):
        """dL/dv*, per-contact (dL/dv_r, dL/dmu) and per-body gradients of the
        last substep's contact solve for vbar = dL/dv (mpm_contact_adjoint)."""
        return mpm_contact_adjoint(self.ctx, node_ids, vbar, n_bodies=self.n_bodies, eps_r=eps_r,
                                   max_iters=max_iters, check=check)


# ---------------------------------------------------------------- batches

def _bcheck(batch, code):
    if code != OK:
        msg = lib.mpm_batch_last_error(batch)
        raise MpmError(code, msg.decode() if msg else "")
    return code


def mpm_batch_create(ctxs):
    arr = (_vp * len(ctxs))(*[c.value if isinstance(c, _vp) else c for c in ctxs])
    out = _vp()
    _check(None, lib.mpm_batch_create(arr, len(ctxs), C.byref(out)))
    return out


def mpm_batch_step(batch, h, n_substeps, solver=None):
    return lib.mpm_batch_step(batch, float(h), int(n_substeps),
                              C.byref(solver) if solver is not None else None)


def mpm_batch_sort(batch):
    return lib.mpm_batch_sort(batch)


def mpm_batch_synchronize(batch, n, want_stats=True):
    """(first failure code, per-member codes [n], per-member StepStats or None)."""
    codes = np.zeros(max(n, 1), np.int32)
    stats = (StepStats * max(n, 1))() if want_stats else None
    code = lib.mpm_batch_synchronize(batch, codes.ctypes.data_as(_i32p), stats)
    return code, codes[:n], ([stats[i] for i in range(n)] if want_stats else None)


def mpm_batch_set_option(batch, option, value):
    _bcheck(batch, lib.mpm_batch_set_option(batch, int(option), int(value)))


def mpm_batch_destroy(batch):
    lib.mpm_batch_destroy(batch)


class Batch:
    """Many scenes advanced together by mpm_batch_* (one launch per phase per
    substep over all of them). The member contexts share one stream: the
    batch creates its Sims itself on a stream of its own. Scenes must share h
    and the substep count of a step."""

    def __init__(self, scenes_, max_contacts=None):
        import torch
        self.torch_stream = torch.cuda.Stream()
        stream = self.torch_stream.cuda_stream
        self.sims = [Sim(sc, max_contacts=(max_contacts(sc) if callable(max_contacts)
                                           else max_contacts), stream=stream)
                     for sc in scenes_]
        for sim in self.sims:
            sim.torch_stream = self.torch_stream
        self.batch = mpm_batch_create([sim.ctx for sim in self.sims])

    def __len__(self):
        return len(self.sims)

    def step(self, h, n_substeps, solver=None):
        _bcheck(self.batch, mpm_batch_step(self.batch, h, n_substeps, solver))

    def sort(self):
        _bcheck(self.batch, mpm_batch_sort(self.batch))

    def synchronize(self, stats=True):
        """(first failure code, per-member codes, per-member stats dicts)."""
        code, codes, st = mpm_batch_synchronize(self.batch, len(self.sims), stats)
        return code, codes, ([s.as_dict() for s in st] if st is not None else None)

    def set_option(self, option, value):
        mpm_batch_set_option(self.batch, option, value)

    def close(self):
        if getattr(self, "batch", None):
            mpm_batch_destroy(self.batch)
            self.batch = None
        for sim in getattr(self, "sims", []):
            sim.close()
        self.sims = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
