"""Seeded synthetic scenes shaped like the paper's manipulation workloads.

This module only places particles and rigid bodies with a seeded RNG; it holds
none of the method's arithmetic (no transfer weights, stresses, SDFs or contact
terms), so both the CUDA path and the CPU oracle can consume its output.

A scene is a plain dict:
  grid:    {dx, res[3], origin[3], gravity[3], bc_layers}
  groups:  list of {x: float32[n,3], v: float32[n,3], vol: float (rest volume
           per particle), material: {model, E, nu, rho, friction_angle_deg}}
  bodies:  list of {shape, params[4], R[3,3], p[3], omega[3], v[3], mu, k, d,
           kinematic}
  h:       substep size [s];  substeps: substeps per rigid time step
Shapes: 0 half-space (plane z=0 of the body frame, +z outward), 1 sphere
(params[0] = radius), 2 box (params[0:3] = half extents), 3 capsule
(params[0] = half length along body z, params[1] = radius).
Materials: model 0 fixed corotated, model 1 Drucker-Prager sand.
"""
import numpy as np

HALFSPACE, SPHERE, BOX, CAPSULE = 0, 1, 2, 3
COROTATED, DRUCKER_PRAGER = 0, 1

SEED_BASE = 20250307

# contact-model defaults (the paper names the lagged model but prints no values)
CONTACT_K = 1.0e4      # N/m per contact point
CONTACT_D = 10.0       # s/m Hunt-Crossley dissipation
EPS_S = 1.0e-4         # m/s friction regularisation

SAND = {"model": DRUCKER_PRAGER, "E": 3.5e5, "nu": 0.3, "rho": 1600.0,
        "friction_angle_deg": 30.0}


def elastic(E=1.0e5, nu=0.3, rho=1000.0):
    return {"model": COROTATED, "E": float(E), "nu": float(nu), "rho": float(rho),
            "friction_angle_deg": 0.0}


def body(shape, params=(0, 0, 0, 0), p=(0, 0, 0), R=None, v=(0, 0, 0), omega=(0, 0, 0),
         mu=0.5, k=CONTACT_K, d=CONTACT_D, kinematic=0):
    prm = np.zeros(4)
    prm[:len(params)] = params
    return {"shape": int(shape), "params": prm,
            "R": np.eye(3) if R is None else np.asarray(R, np.float64).reshape(3, 3),
            "p": np.asarray(p, np.float64), "omega": np.asarray(omega, np.float64),
            "v": np.asarray(v, np.float64), "mu": float(mu), "k": float(k), "d": float(d),
            "kinematic": int(kinematic)}


def rot_y(theta):
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def lattice_cube(n_side, spacing, center, jitter, rng):
    """n_side^3 lattice points, x fastest, with uniform jitter of +-jitter."""
    idx = np.arange(n_side, dtype=np.float64)
    gx, gy, gz = np.meshgrid(idx, idx, idx, indexing="ij")
    pts = np.stack([gx.transpose(2, 1, 0).ravel(), gy.transpose(2, 1, 0).ravel(),
                    gz.transpose(2, 1, 0).ravel()], 1)
    pts = (pts - (n_side - 1) / 2.0) * spacing + np.asarray(center, np.float64)
    if jitter > 0:
        pts = pts + rng.uniform(-jitter, jitter, pts.shape)
    return pts


def cube_group(n_side, spacing, center, v0=(0, 0, 0), material=None, jitter=0.0, rng=None):
    rng = rng if rng is not None else np.random.default_rng(SEED_BASE)
    x = lattice_cube(n_side, spacing, center, jitter, rng).astype(np.float32)
    v = np.tile(np.asarray(v0, np.float32), (len(x), 1))
    return {"x": x, "v": v, "vol": float(spacing ** 3),
            "material": material if material is not None else elastic()}


def cube_drop(seed=SEED_BASE + 0, n_side=20, drop_height=0.2, v0=(0.0, 0.0, 0.0),
              sphere_x=0.12, sphere_v=0.1, mu=0.5, h=1e-4, substeps=10):
    """Elastic cube (n_side^3 particles at 2 per dx, side n_side*dx/2) dropped onto
    a static half-space at z = 0, beside a kinematic sphere (r = 0.05 m) rolling
    towards it along -x. dx = 0.01 m on a 64^3 grid. The default is the 8,000
    particle, 0.1 m cube dropped from 0.2 m (bottom face height)."""
    rng = np.random.default_rng(seed)
    dx = 0.01
    spacing = dx / 2.0
    side = n_side * spacing
    center = (0.0, 0.0, drop_height + side / 2.0)
    g = cube_group(n_side, spacing, center, v0, elastic(1.0e5, 0.3, 1000.0),
                   jitter=1e-4 * dx, rng=rng)
    bodies = [body(HALFSPACE, mu=mu),
              body(SPHERE, (0.05,), p=(sphere_x, 0.0, 0.05), v=(-sphere_v, 0.0, 0.0), mu=mu,
                   kinematic=1)]
    grid = {"dx": dx, "res": (64, 64, 64), "origin": (-0.32, -0.32, -0.08),
            "gravity": (0.0, 0.0, -9.81), "bc_layers": 3}
    return {"name": "cube_drop_%d" % len(g["x"]), "grid": grid, "groups": [g],
            "bodies": bodies, "h": h, "substeps": substeps}


def granular_scoop(n_particles=1_000_000, seed=SEED_BASE + 1, h=5e-5, substeps=10,
                   paddle_speed=0.2, mu=0.4, res=128):
    """Drucker-Prager sand (friction angle 30 deg, rho 1600) seeded uniformly in a
    0.3 m box that sits in a static bin of five SDF boxes (floor + 4 walls), with
    two kinematic box paddles (0.02 x 0.1 x 0.15 m) moving along +x at
    `paddle_speed` through the sand; dx = 3e-3 m; block-sparse 128^3 grid."""
    rng = np.random.default_rng(seed)
    dx = 3e-3
    L = 0.15          # bin half width
    H = 0.3           # sand height
    t = 0.0075        # half wall thickness
    paddles = [((-0.09, -0.06, 0.2), (0.01, 0.05, 0.075)),
               ((-0.09, 0.06, 0.2), (0.01, 0.05, 0.075))]
    # rejection sampling against the paddles' axis-aligned boxes
    pts = np.empty((0, 3))
    need = n_particles
    while need > 0:
        cand = rng.uniform((-L, -L, 0.0), (L, L, H), (int(need * 1.15) + 64, 3))
        keep = np.ones(len(cand), bool)
        for c, hx in paddles:
            inside = np.all(np.abs(cand - np.asarray(c)) < np.asarray(hx), axis=1)
            keep &= ~inside
        cand = cand[keep][:need]
        pts = np.concatenate([pts, cand], 0)
        need = n_particles - len(pts)
    pad_vol = sum(8 * hx[0] * hx[1] * hx[2] for _, hx in paddles)
    vol = ((2 * L) ** 2 * H - pad_vol) / n_particles
    g = {"x": pts.astype(np.float32), "v": np.zeros((n_particles, 3), np.float32),
         "vol": float(vol), "material": dict(SAND)}
    bodies = [body(BOX, (L + 2 * t, L + 2 * t, t), p=(0, 0, -t), mu=mu),
              body(BOX, (t, L + 2 * t, H / 2 + 0.03), p=(-(L + t), 0, H / 2), mu=mu),
              body(BOX, (t, L + 2 * t, H / 2 + 0.03), p=((L + t), 0, H / 2), mu=mu),
              body(BOX, (L + 2 * t, t, H / 2 + 0.03), p=(0, -(L + t), H / 2), mu=mu),
              body(BOX, (L + 2 * t, t, H / 2 + 0.03), p=(0, (L + t), H / 2), mu=mu)]
    for c, hx in paddles:
        bodies.append(body(BOX, hx, p=c, v=(paddle_speed, 0, 0), mu=mu, kinematic=1))
    origin = (-res * dx / 2.0, -res * dx / 2.0, -0.03)
    grid = {"dx": dx, "res": (res, res, res), "origin": origin,
            "gravity": (0.0, 0.0, -9.81), "bc_layers": 3}
    return {"name": "granular_scoop_%d" % n_particles, "grid": grid, "groups": [g],
            "bodies": bodies, "h": h, "substeps": substeps}


def sand_column(n_side=12, seed=SEED_BASE + 11, dx=0.01, h=1e-4, with_paddle=True):
    """Small sand block resting on a half-space (bottom particle layer on the
    plane) with a kinematic box paddle moving along +x whose face touches the
    block's -x side: the granular scooping workload at a size the oracle runs
    in seconds."""
    rng = np.random.default_rng(seed)
    spacing = dx / 2.0
    half = (n_side - 1) * spacing / 2.0
    jit = 0.1 * spacing
    g = cube_group(n_side, spacing, (0.0, 0.0, half + jit), (0, 0, 0), dict(SAND), jitter=jit,
                   rng=rng)
    bodies = [body(HALFSPACE, mu=0.4)]
    if with_paddle:
        # paddle face 0.5 jitter widths inside the outermost lattice column
        bodies.append(body(BOX, (0.01, 0.02, 0.02), p=(-half - 0.01 + 0.5 * jit, 0, 0.02),
                           v=(0.2, 0, 0), mu=0.4, kinematic=1))
    grid = {"dx": dx, "res": (32, 32, 32), "origin": (-0.16, -0.16, -0.04),
            "gravity": (0.0, 0.0, -9.81), "bc_layers": 3}
    return {"name": "sand_column_%d" % len(g["x"]), "grid": grid, "groups": [g],
            "bodies": bodies, "h": h, "substeps": 10}


def sand_random(n_particles=8000, ppc=1.0, seed=SEED_BASE + 12, dx=0.01, h=1e-4,
                penetration=0.0, speed=0.1):
    """Sand sampled uniformly at random (not on a lattice) at about `ppc`
    particles per grid cell in a cube over a half-space, with seeded random
    velocities of up to `speed` per component: the sparse random sampling of
    the granular scooping workload (about one particle per cell) at a size
    the oracle runs in seconds. The cube's bottom reaches `penetration` below
    the plane, so the lowest particles start in contact."""
    rng = np.random.default_rng(seed)
    side = (n_particles / ppc) ** (1.0 / 3.0) * dx
    x = rng.uniform((-side / 2, -side / 2, -penetration),
                    (side / 2, side / 2, side - penetration), (n_particles, 3))
    v = rng.uniform(-speed, speed, (n_particles, 3))
    g = {"x": x.astype(np.float32), "v": v.astype(np.float32),
         "vol": float(side ** 3 / n_particles), "material": dict(SAND)}
    bodies = [body(HALFSPACE, mu=0.4)]
    res = 4 * int(np.ceil((side / dx + 12) / 4))  # grid sizes are multiples of 4
    grid = {"dx": dx, "res": (res, res, res), "origin": (-res * dx / 2, -res * dx / 2, -0.04),
            "gravity": (0.0, 0.0, -9.81), "bc_layers": 3}
    return {"name": "sand_random_%d" % n_particles, "grid": grid, "groups": [g],
            "bodies": bodies, "h": h, "substeps": 10}


def sand_slab(n_x=72, n_y=72, n_z=2, seed=SEED_BASE + 13, dx=0.01, h=1e-4, sink=1.2e-5,
              paddle_overlap=3e-6, v0=(0.02, 0.01, -0.02)):
    """A thin sand slab (n_x x n_y x n_z lattice at 2 particles per dx per
    axis, seeded jitter) whose bottom particle layer sits `sink` below the
    plane z = 0, moving with v0, with a kinematic box paddle along +x whose
    face overlaps the slab's -x particle column by `paddle_overlap`: a
    contact-rich case (every particle of the bottom layer, about n_x n_y
    contacts) small enough for the oracle."""
    rng = np.random.default_rng(seed)
    spacing = dx / 2.0
    jit = 1e-3 * spacing
    idx = [np.arange(k, dtype=np.float64) for k in (n_x, n_y, n_z)]
    gz, gy, gx = np.meshgrid(idx[2], idx[1], idx[0], indexing="ij")
    pts = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], 1) * spacing
    pts[:, 0] -= (n_x - 1) * spacing / 2.0
    pts[:, 1] -= (n_y - 1) * spacing / 2.0
    pts += rng.uniform(-jit, jit, pts.shape)
    pts[:, 2] += jit - sink  # the lowest particles end up inside the plane
    x = pts.astype(np.float32)
    g = {"x": x, "v": np.tile(np.asarray(v0, np.float32), (len(x), 1)), "vol": spacing ** 3,
         "material": dict(SAND)}
    edge = (n_x - 1) * spacing / 2.0 + jit
    height = n_z * spacing
    bodies = [body(HALFSPACE, mu=0.4),
              body(BOX, (0.01, n_y * spacing / 2.0 + dx, height + dx),
                   p=(-edge - 0.01 + paddle_overlap, 0.0, height), v=(0.05, 0, 0), mu=0.4,
                   kinematic=1)]
    res_xy = 4 * int(np.ceil((max(n_x, n_y) * spacing / dx + 14) / 4))
    res_z = 4 * int(np.ceil((n_z * spacing / dx + 16) / 4))
    grid = {"dx": dx, "res": (res_xy, res_xy, res_z),
            "origin": (-res_xy * dx / 2, -res_xy * dx / 2, -8 * dx),
            "gravity": (0.0, 0.0, -9.81), "bc_layers": 3}
    return {"name": "sand_slab_%d" % len(x), "grid": grid, "groups": [g], "bodies": bodies,
            "h": h, "substeps": 10}


def filled_box(res=12, bc=3, per_axis=20, dx=0.01):
    """Elastic particles at rest filling a res^3 grid (origin 0) so that every
    node has mass: per_axis^3 lattice points whose cell coordinates run from
    0.75 to res - 1.75, so that their stencils cover nodes 0 .. res - 1 and
    never leave the grid. No bodies. Used to count the Dirichlet layers."""
    t = np.linspace(0.75, res - 1.75, per_axis) * dx
    gx, gy, gz = np.meshgrid(t, t, t, indexing="ij")
    x = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], 1).astype(np.float32)
    g = {"x": x, "v": np.zeros_like(x), "vol": (dx / 2) ** 3, "material": elastic(1e5, 0.3, 1000.0)}
    grid = {"dx": dx, "res": (res, res, res), "origin": (0.0, 0.0, 0.0),
            "gravity": (0.0, 0.0, -9.81), "bc_layers": bc}
    return {"name": "filled_box_%d" % len(x), "grid": grid, "groups": [g], "bodies": [],
            "h": 1e-4, "substeps": 1}


def batch_scene(index, seed=SEED_BASE + 4, n_min=2000, n_max=64000, dx=5e-3, h=1e-4,
                penetration=1e-4):
    """Scene `index` of a batch of independent scenes of uneven size: a cube of
    n ~ U[n_min, n_max] particles at 2 per dx per axis (elastic, E log-uniform in
    [1e4, 2e5] -- the explicit substep's CFL limit at dx = 5e-3 m and h = 1e-4 s
    is E < 6e5 for rho = 1000 -- or Drucker-Prager sand, chosen by the seed)
    caught at touch-down: its bottom layer `penetration` into the ground while
    falling at 0.05 m/s, and a kinematic box gripper jaw moving along +x at
    0.05 m/s whose face overlaps the cube's -x side by `penetration`. The
    contact stiffness per contact point is scaled with the particle mass so
    that h^2 k / m_p = 0.8, the value of the 8,000-particle cube (k = 1e4 N/m,
    m_p = 1.25e-4 kg, h = 1e-4 s): these particles are 5-8x lighter, and at
    k = 1e4 the contact solve of a scene would be that much stiffer."""
    rng = np.random.default_rng(seed * 1000 + index)
    n = int(rng.integers(n_min, n_max + 1))
    n_side = max(int(round(n ** (1.0 / 3.0))), 2)
    spacing = dx / 2.0
    half = (n_side - 1) * spacing / 2.0
    if rng.random() < 0.5:
        mat = elastic(E=float(10 ** rng.uniform(4.0, np.log10(2e5))), nu=0.3, rho=1000.0)
    else:
        mat = dict(SAND)
    jit = 1e-4 * dx
    g = cube_group(n_side, spacing, (0.0, 0.0, half - penetration), (0.0, 0.0, -0.05), mat,
                   jitter=jit, rng=rng)
    mu = float(rng.uniform(0.2, 0.8))
    k = 0.8 * mat["rho"] * spacing ** 3 / h ** 2
    bodies = [body(HALFSPACE, mu=mu, k=k),
              body(BOX, (0.01, half + dx, half + dx), p=(-half - 0.01 + penetration, 0, half + dx),
                   v=(0.05, 0, 0), mu=mu, k=k, kinematic=1)]
    side = 2 * half + 0.06
    res = 4 * int(np.ceil((side / dx + 12) / 4))
    grid = {"dx": dx, "res": (res, res, res), "origin": (-res * dx / 2, -res * dx / 2, -6 * dx),
            "gravity": (0.0, 0.0, -9.81), "bc_layers": 3}
    return {"name": "batch_%d_%d" % (index, len(g["x"])), "grid": grid, "groups": [g],
            "bodies": bodies, "h": h, "substeps": 10}


def panel_squeeze(n_side=12, dx=0.01, E=1.0e5, mu=0.5, force=10.0, panel_mass=0.5,
                  overlap=1e-4, h=1e-4, substeps=1):
    """The panel squeeze of Sec. VI-A (Fig. 2): an elastic cube (n_side^3
    particles at 2 per dx, rho = 1000) between two dynamic box panels that
    may only translate along x and are pushed towards each other with
    `force` newtons each, holding the cube against gravity by friction; no
    ground. At steady state each panel carries the normal force `force` and a
    vertical friction force of half the cube's weight. Returns the scene and
    the panels' dynamics (indices 0 and 1)."""
    rng = np.random.default_rng(SEED_BASE + 41)
    spacing = dx / 2.0
    half = n_side * spacing / 2.0  # cube faces at +-half (particle cells)
    g = cube_group(n_side, spacing, (0.0, 0.0, 0.0), (0, 0, 0), elastic(E, 0.3, 1000.0),
                   jitter=1e-4 * dx, rng=rng)
    t = 0.005
    edge = (n_side - 1) * spacing / 2.0  # outermost particle column
    bodies = [body(BOX, (t, 0.05, 0.05), p=(-edge - t + overlap, 0, 0), mu=mu),
              body(BOX, (t, 0.05, 0.05), p=(edge + t - overlap, 0, 0), mu=mu)]
    inertia = [panel_mass * (0.1 ** 2 + 0.1 ** 2) / 12.0, panel_mass * (0.1 ** 2 + (2 * t) ** 2) / 12.0,
               panel_mass * (0.1 ** 2 + (2 * t) ** 2) / 12.0]
    dyn = [dict(mass=panel_mass, inertia=inertia, force=[force, 0.0, 0.0], torque=[0, 0, 0],
                dof_mask=0b000001, gravity=0),
           dict(mass=panel_mass, inertia=inertia, force=[-force, 0.0, 0.0], torque=[0, 0, 0],
                dof_mask=0b000001, gravity=0)]
    grid = {"dx": dx, "res": (32, 32, 32), "origin": (-0.16, -0.16, -0.16),
            "gravity": (0.0, 0.0, -9.81), "bc_layers": 3}
    sc = {"name": "panel_squeeze_%d" % len(g["x"]), "grid": grid, "groups": [g],
          "bodies": bodies, "h": h, "substeps": substeps}
    return sc, dyn


def ball_group(n_target, spacing, center, material, jitter, rng):
    """About n_target lattice points (x fastest) inside a sphere, with jitter."""
    r = (3.0 * n_target / (4.0 * np.pi)) ** (1.0 / 3.0) * spacing
    k = int(np.ceil(r / spacing)) + 1
    idx = np.arange(-k, k + 1, dtype=np.float64) * spacing
    gx, gy, gz = np.meshgrid(idx, idx, idx, indexing="ij")
    pts = np.stack([gx.transpose(2, 1, 0).ravel(), gy.transpose(2, 1, 0).ravel(),
                    gz.transpose(2, 1, 0).ravel()], 1)
    pts = pts[np.sum(pts * pts, 1) <= r * r] + np.asarray(center, np.float64)
    if jitter > 0:
        pts = pts + rng.uniform(-jitter, jitter, pts.shape)
    x = pts.astype(np.float32)
    return {"x": x, "v": np.zeros_like(x), "vol": float(spacing ** 3), "material": material}, r


def mixed_manipulation(n_objects=32, n_per_object=125_000, seed=SEED_BASE + 2, dx=2e-3,
                       h=2.5e-5, substeps=10):
    """Mixed-material manipulation: n_objects objects of about n_per_object
    particles each at 2 per dx per axis, half elastic (E log-uniform in
    [1e4, 1e6], rho = 1000) and half Drucker-Prager sand, alternately cubes and
    balls, on a floor in rows of 8 with 7 cm pitch; 12 rigid bodies: the floor,
    two box jaws of a parallel gripper closing on object 0 at 0.05 m/s (faces
    0.01 dx inside it), and nine static obstacles (boxes, capsules, spheres)
    between the objects; mu ~ U[0.2, 0.8] per body. h = 2.5e-5 s keeps the
    stiffest elastic objects inside the explicit substep's CFL limit."""
    rng = np.random.default_rng(seed)
    spacing = dx / 2.0
    pitch = 0.07
    cols = min(n_objects, 8)
    rows = (n_objects + cols - 1) // cols
    groups, extents = [], []
    jit = 1e-4 * dx
    for i in range(n_objects):
        r_i, c_i = divmod(i, cols)
        cx = (c_i - (cols - 1) / 2.0) * pitch
        cy = (r_i - (rows - 1) / 2.0) * pitch
        if i % 2 == 0:
            mat = elastic(E=float(10 ** rng.uniform(4.0, 6.0)), nu=0.3, rho=1000.0)
        else:
            mat = dict(SAND)
        if (i // 2) % 2 == 0:
            n_side = max(int(round(n_per_object ** (1.0 / 3.0))), 2)
            half = (n_side - 1) * spacing / 2.0
            g = cube_group(n_side, spacing, (cx, cy, half + jit), (0, 0, 0), mat, jitter=jit, rng=rng)
            extents.append((cx, cy, half))
        else:
            g0, r = ball_group(n_per_object, spacing, (cx, cy, 0.0), mat, jit, rng)
            g0["x"][:, 2] += np.float32(-g0["x"][:, 2].min() + jit)
            g = g0
            extents.append((cx, cy, r))
        groups.append(g)
    mus = rng.uniform(0.2, 0.8, 12)
    bodies = [body(HALFSPACE, mu=float(mus[0]))]
    cx0, cy0, e0 = extents[0]
    jaw = (0.01, e0 + dx, e0 + dx)
    bodies.append(body(BOX, jaw, p=(cx0 - e0 - 0.01 + 0.01 * dx, cy0, e0), v=(0.05, 0, 0),
                       mu=float(mus[1]), kinematic=1))
    bodies.append(body(BOX, jaw, p=(cx0 + e0 + 0.01 - 0.01 * dx, cy0, e0), v=(-0.05, 0, 0),
                       mu=float(mus[2]), kinematic=1))
    # static obstacles in the gaps between object rows
    for k in range(9):
        gx = ((k % cols) - (cols - 1) / 2.0 + 0.5) * pitch
        gy = ((rows - 1) / 2.0 - 0.5) * pitch if rows > 1 else pitch / 2.0
        shape = (BOX, CAPSULE, SPHERE)[k % 3]
        params = {BOX: (0.005, 0.005, 0.01), CAPSULE: (0.008, 0.004), SPHERE: (0.006,)}[shape]
        bodies.append(body(shape, params, p=(gx, gy, 0.012), mu=float(mus[3 + k])))
    span_x = cols * pitch + 0.08
    span_y = rows * pitch + 0.08
    res = (4 * int(np.ceil(span_x / dx / 4)), 4 * int(np.ceil(span_y / dx / 4)),
           4 * int(np.ceil((0.1 + 12 * dx) / dx / 4)))
    origin = (-res[0] * dx / 2.0, -res[1] * dx / 2.0, -6 * dx)
    grid = {"dx": dx, "res": res, "origin": origin, "gravity": (0.0, 0.0, -9.81), "bc_layers": 3}
    return {"name": "mixed_manipulation_%d" % sum(len(g["x"]) for g in groups), "grid": grid,
            "groups": groups, "bodies": bodies, "h": h, "substeps": substeps}


def n_particles(scene):
    return int(sum(len(g["x"]) for g in scene["groups"]))


def incline_block(theta_deg=30.0, mu=0.3, n_side=6, dx=0.01, E=1.0e6, seed=SEED_BASE + 21,
                  h=1e-4):
    """Elastic block sitting flat on a half-space tilted by theta about y
    (outward normal (sin t, 0, cos t)); downhill is +x."""
    rng = np.random.default_rng(seed)
    t = np.radians(theta_deg)
    R = rot_y(t)
    spacing = dx / 2.0
    local = lattice_cube(n_side, spacing, (0, 0, 0), 1e-4 * dx, rng)
    # bottom particle layer on the plane (contacts register for particles inside)
    center = R @ np.array([0.0, 0.0, (n_side - 1) * spacing / 2.0])
    x = (local @ R.T + center).astype(np.float32)
    g = {"x": x, "v": np.zeros_like(x), "vol": spacing ** 3,
         "material": elastic(E, 0.3, 1000.0)}
    grid = {"dx": dx, "res": (40, 16, 24), "origin": (-0.12, -0.08, -0.12),
            "gravity": (0.0, 0.0, -9.81), "bc_layers": 3}
    return {"name": "incline", "grid": grid, "groups": [g],
            "bodies": [body(HALFSPACE, R=R, mu=mu)], "h": h, "substeps": 10}


def cube_contact(n_side=10, seed=SEED_BASE + 31, v0=(0.05, 0.0, -0.05), penetration=1e-4,
                 sphere_overlap=2e-4, E=1.0e5, h=1e-4):
    """The cube-drop workload caught at touch-down: the cube's bottom particle
    layer sits `penetration` into the ground and the kinematic sphere (moving
    along -x) overlaps its side by `sphere_overlap`; a small, contact-rich case
    for per-substep parity."""
    dx = 0.01
    spacing = dx / 2.0
    side = n_side * spacing
    sc = cube_drop(seed=seed, n_side=n_side, drop_height=-spacing / 2.0 - penetration, v0=v0,
                   sphere_x=(n_side - 1) * spacing / 2.0 + 0.05 - sphere_overlap, h=h)
    sc["groups"][0]["material"] = elastic(E, 0.3, 1000.0)
    sc["name"] = "cube_contact_%d" % (n_side ** 3)
    return sc


def push_cube(n_particles=65536, side=0.1, seed=SEED_BASE + 3, dx=5e-3, h=1e-4, substeps=25,
              E=1.0e5, nu=0.3, v0=(0.0, 0.0, 0.0), push_speed=0.1, box_overlap=0.0,
              mu_ground=0.5, mu_box=0.3, sink=0.0, lattice_side=0, k_contact=1.0e3,
              material=None):
    """The differentiation workload: an elastic cube of `n_particles` seeded
    uniformly at random in a box of edge `side` (65,536 in 0.1 m at dx = 5e-3
    is ~8.2 per cell), standing on a static half-space z = 0 (its bottom
    `sink` below the plane) and pushed along +x by a kinematic box whose face
    starts `box_overlap` inside the cube's -x face. With lattice_side > 0 the
    particles sit instead on a lattice_side^3 grid at spacing side /
    lattice_side (cell centres; `sink` and `box_overlap` are then measured
    from the outer particle layers). Substeps per rigid step = the checkpoint
    interval of the rollout. Returns the scene and a seeded target point for
    the centroid loss. `material` replaces the elastic (E, nu) material (e.g.
    SAND). The contact stiffness k_contact (per contact point) is
    lower than the other scenes' 1e4 N/m: these particles are ~8x lighter, and
    a cube resting on 65k of them stays well conditioned for the solve."""
    rng = np.random.default_rng(seed)
    lo = np.array([-side / 2.0, -side / 2.0, -sink])
    if lattice_side > 0:
        sp = side / lattice_side
        i = (np.arange(lattice_side) + 0.5) * sp
        grid3 = np.stack(np.meshgrid(i, i, i, indexing="ij"), -1).reshape(-1, 3)
        x = (lo + grid3 - np.array([0.0, 0.0, sp / 2.0])).astype(np.float32)
        box_overlap = box_overlap + sp / 2.0
        n_particles = len(x)
    else:
        x = (lo + side * rng.random((n_particles, 3))).astype(np.float32)
    vol = side ** 3 / n_particles
    g = {"x": x, "v": np.tile(np.asarray(v0, np.float32), (n_particles, 1)), "vol": vol,
         "material": dict(material) if material is not None else elastic(E, nu, 1000.0)}
    half = (0.02, 0.6 * side, 0.4 * side)
    box_x = -side / 2.0 - half[0] + box_overlap
    bodies = [body(HALFSPACE, mu=mu_ground, k=k_contact),
              body(BOX, half, p=(box_x, 0.0, half[2] + 0.1 * side), v=(push_speed, 0.0, 0.0),
                   mu=mu_box, k=k_contact, kinematic=1)]
    # domain: the cube, the box's travel and a margin of Dirichlet layers
    span = 2.0 * side + 0.1
    res = int(np.ceil(span / dx / 4.0)) * 4 + 16
    grid = {"dx": dx, "res": (res, res, res), "origin": (-res * dx / 2.0, -res * dx / 2.0, -8 * dx),
            "gravity": (0.0, 0.0, -9.81), "bc_layers": 3}
    target = np.array([side, 0.0, side / 2.0]) + 0.01 * side * rng.standard_normal(3)
    sc = {"name": "push_cube_%d" % n_particles, "grid": grid, "groups": [g], "bodies": bodies,
          "h": h, "substeps": substeps}
    return sc, target


CLOTH = 2  # material model of cloth vertices (include/mpmcr.h MPM_CLOTH)


def cloth_material(E=3.2e6, nu=0.4, rho=1.5e3):
    """Cloth membrane with the E, nu and rho of the paper's cloth experiment
    (Sec. VI); the paper gives no thickness: the sheets take 0.5 mm, which at
    this density is 0.75 kg/m^2."""
    return {"model": CLOTH, "E": float(E), "nu": float(nu), "rho": float(rho),
            "friction_angle_deg": 0.0}


def cloth_sheet(n_side, spacing, center, v0=(0.0, 0.0, 0.0), material=None, thickness=5e-4):
    """A square sheet of n_side^2 vertices at `spacing` in the plane z =
    center[2], two triangles per quad (diagonals alternating), as a cloth
    particle group: its mass per vertex is rho * thickness * area / n."""
    i, j = np.meshgrid(np.arange(n_side), np.arange(n_side), indexing="ij")
    half = (n_side - 1) * spacing / 2.0
    x = np.stack([center[0] - half + i.ravel() * spacing, center[1] - half + j.ravel() * spacing,
                  np.full(n_side * n_side, center[2])], 1).astype(np.float32)
    tris = []
    for a in range(n_side - 1):
        for b in range(n_side - 1):
            v00, v10, v01, v11 = a * n_side + b, (a + 1) * n_side + b, a * n_side + b + 1, \
                (a + 1) * n_side + b + 1
            if (a + b) % 2 == 0:
                tris += [(v00, v10, v11), (v00, v11, v01)]
            else:
                tris += [(v00, v10, v01), (v10, v11, v01)]
    tris = np.array(tris, np.int32)
    xd = x.astype(np.float64)
    area = 0.5 * np.linalg.norm(np.cross(xd[tris[:, 1]] - xd[tris[:, 0]],
                                         xd[tris[:, 2]] - xd[tris[:, 0]]), axis=1).sum()
    n = len(x)
    vol = float(np.float32(np.float32(thickness) * area / n))
    return {"x": x, "v": np.tile(np.asarray(v0, np.float32), (n, 1)), "tris": tris,
            "thickness": float(thickness), "vol": vol,
            "material": dict(material) if material is not None else cloth_material()}


def cloth_drape(n_side=12, spacing=4e-3, radius=0.02, sink=2e-5, h=2e-5, substeps=10,
                mu=0.4, v0=(0.0, 0.0, -0.05)):
    """The paper's cloth-on-rigid setting in miniature: a square sheet
    (E = 3.2e6 Pa, nu = 0.4) caught on top of a static sphere (its centre
    vertices `sink` inside it) above the ground, falling at 0.05 m/s; grid
    dx = 2 spacing. The contact stiffness per contact point is scaled with the
    vertex mass as in the batch scenes (h^2 k / m = 0.8)."""
    dx = 2.0 * spacing
    g = cloth_sheet(n_side, spacing, (0.0, 0.0, 2.0 * radius - sink), v0)
    m_p = g["material"]["rho"] * g["vol"]
    k = 0.8 * m_p / h ** 2
    bodies = [body(HALFSPACE, mu=mu, k=k),
              body(SPHERE, (radius, 0, 0, 0), p=(0.0, 0.0, radius), mu=mu, k=k)]
    side = (n_side - 1) * spacing + 12 * dx
    res = 4 * int(np.ceil((side / dx + 8) / 4))
    rz = 4 * int(np.ceil((2.0 * radius / dx + 16) / 4))
    grid = {"dx": dx, "res": (res, res, rz), "origin": (-res * dx / 2, -res * dx / 2, -6 * dx),
            "gravity": (0.0, 0.0, -9.81), "bc_layers": 3}
    return {"name": "cloth_drape_%d" % len(g["x"]), "grid": grid, "groups": [g],
            "bodies": bodies, "h": h, "substeps": substeps}


def box_bagging(n_side=30, side=0.42, box_half=0.04, box_rho=1.0e3, mu=0.2, dx=1.0 / 64,
                h=2.5e-4, substeps=10, height=0.2, sink=2e-5):
    """The cloth cradle of the paper's box-bagging experiment (Sec. VI,
    simulation statistics: grid spacing 1/64 m, 10 substeps per step): a
    square sheet of n_side^2 vertices and `side` metres (E = 3.2e6 Pa,
    nu = 0.4, rho = 1500), its four corners pinned at rest `height` above the
    ground, and a dynamic box of side 2 box_half and density box_rho resting
    on its middle (its bottom `sink` into the sheet), box-cloth friction
    `mu`. The paper's 2,582 particles are a 30 x 30 mesh sampled at its
    vertices and face centroids; here the vertices alone (900) carry the
    cloth. h = 2.5e-4 s keeps the explicit membrane stable (its wave speed
    sqrt(E / rho) = 46 m/s crosses a 1.45 cm edge in 3.1e-4 s). Returns the
    scene and the box's dynamics (body 1)."""
    spacing = side / (n_side - 1)
    g = cloth_sheet(n_side, spacing, (0.0, 0.0, height), (0.0, 0.0, 0.0))
    n = n_side
    g["pins"] = {"ids": [0, n - 1, n * (n - 1), n * n - 1], "v": np.zeros((4, 3), np.float32)}
    m_p = g["material"]["rho"] * g["vol"]
    k = 0.8 * m_p / h ** 2
    bodies = [body(HALFSPACE, mu=0.4, k=k),
              body(BOX, (box_half, box_half, box_half), p=(0.0, 0.0, height + box_half - sink),
                   mu=mu, k=k)]
    m_box = box_rho * (2 * box_half) ** 3
    i_box = m_box * (2 * box_half) ** 2 / 6.0
    dyn = dict(mass=m_box, inertia=[i_box, i_box, i_box], force=[0.0, 0.0, 0.0],
               torque=[0.0, 0.0, 0.0], dof_mask=0b111111, gravity=1)
    res_xy = 4 * int(np.ceil((side / dx + 12) / 4))
    res_z = 4 * int(np.ceil(((height + 4 * box_half) / dx + 12) / 4))
    grid = {"dx": dx, "res": (res_xy, res_xy, res_z),
            "origin": (-res_xy * dx / 2, -res_xy * dx / 2, -6 * dx),
            "gravity": (0.0, 0.0, -9.81), "bc_layers": 3}
    return {"name": "box_bagging_%d" % len(g["x"]), "grid": grid, "groups": [g],
            "bodies": bodies, "h": h, "substeps": substeps}, dyn
