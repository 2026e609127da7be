/*
 * mpmcr.h -- C ABI of the GB300 (sm_103a) MPM / rigid-body convex-contact
 * substep library.
 *
 * The library advances material points (MPM) coupled to rigid bodies through
 * the convex frictional-contact formulation of Yu et al., "A Convex
 * Formulation of Material Points and Rigid Bodies with GPU-Accelerated
 * Async-Coupling for Interactive Simulation" (arXiv 2503.05046):
 *
 *   - one call to mpm_step is one rigid time step of the asynchronous time
 *     splitting (Sec. IV-A, Eq. (3)-(4)): the rigid bodies' poses and spatial
 *     velocities are frozen while N MPM substeps of size h run, and the
 *     contact impulses of all substeps are accumulated for the caller's rigid
 *     solver;
 *   - one substep (Eq. (5)) is the free motion of Eq. (6) (an explicit
 *     MLS-MPM step: particle-to-grid, grid update, later grid-to-particle with
 *     the constitutive update) followed by the contact solve of Eq. (7)-(8),
 *     the convex problem min_v 1/2 ||v - v*||_M^2 + l_c(v_c), solved by the
 *     block-diagonal quasi-Newton iteration with exact line search of Alg. 1
 *     (Sec. IV-C, V-B).
 *
 * Conventions shared by every entry point:
 *   - Units are SI; z is up in the examples but gravity is a parameter.
 *   - Particle arrays are float32, row-major per particle: x, v are [n][3];
 *     C (affine velocity) and F (deformation gradient) are [n][3][3]
 *     row-major. Particles are identified by the order in which they were
 *     added (id 0, 1, ...); the library reorders them internally (a radix sort
 *     by grid block once per time step, Sec. V-A) but every input and output
 *     is in id order.
 *   - `mem_kind` selects where a caller buffer lives: MPM_MEM_HOST (0) or
 *     MPM_MEM_DEVICE (1, a pointer on the context's device).
 *   - Caller buffers are only read or written during the call (inputs are
 *     copied); the context owns all of its device memory.
 *   - Work is ordered on the context's CUDA stream. Calls that return data to
 *     the host (mpm_get_*, mpm_step with a stats pointer, mpm_synchronize)
 *     synchronise that stream; the others are asynchronous.
 *   - No exception crosses the ABI. Every entry point returns an mpm_status.
 *     Device-side failures (a particle leaving the domain, a capacity
 *     overflow, a solve that did not converge) are recorded on the device and
 *     reported by the next synchronising call; they stay set until read.
 *     mpm_last_error gives a message for the last failure.
 */
#ifndef MPMCR_H
#define MPMCR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpm_ctx mpm_ctx;

typedef enum {
  MPM_OK = 0,
  MPM_ERR_INVALID_ARG = 1,    /* bad argument; nothing was done */
  MPM_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  MPM_ERR_OOM = 3,            /* device allocation failed */
  MPM_ERR_CAPACITY = 4,       /* more particles or contacts than the context holds */
  MPM_ERR_NOT_CONVERGED = 5,  /* a contact solve (Alg. 1) or its adjoint hit max_iters */
  MPM_ERR_OUT_OF_DOMAIN = 6,  /* a particle's stencil left the grid */
  MPM_ERR_NAN = 7,            /* a non-finite value appeared in the solve */
  MPM_ERR_STATE = 8,          /* call not valid in the context's state */
  MPM_ERR_TIMEOUT = 9,        /* a device-wide barrier gave up waiting */
  MPM_ERR_LINE_SEARCH = 10    /* the line-search bracket could not be formed */
} mpm_status;

enum { MPM_MEM_HOST = 0, MPM_MEM_DEVICE = 1 };

/* Material models: fixed corotated elasticity, Drucker-Prager sand (Hencky
   strain, the granular model the paper cites, Sec. II-A), and cloth (the
   vertices of a triangle mesh, mpm_add_cloth; Sec. VI cloth results). */
enum { MPM_COROTATED = 0, MPM_DRUCKER_PRAGER = 1, MPM_CLOTH = 2 };

/* Rigid geometry (analytic signed distance functions, body frame):
   HALFSPACE  the plane z = 0, outward normal +z (no parameters);
   SPHERE     params[0] = radius;
   BOX        params[0..2] = half extents;
   CAPSULE    params[0] = half length along z, params[1] = radius. */
enum { MPM_HALFSPACE = 0, MPM_SPHERE = 1, MPM_BOX = 2, MPM_CAPSULE = 3 };

/* Eulerian grid (Sec. V-A). Node (i,j,k) sits at origin + dx*(i,j,k). The
   grid is block-sparse in time (only 4^3 blocks touched by particles are
   swept) over an address space of res[0]*res[1]*res[2] < 2^31 nodes; each
   res[a] must be a positive multiple of 4. Nodes within bc_layers of a domain
   face are Dirichlet nodes held at zero velocity (the paper is silent on
   domain walls; this is the reading taken).
   Storage: with max_blocks = 0 (or at least the domain's 4^3 blocks) every
   block has its nodes (about 150 B per node). With 0 < max_blocks < blocks
   the storage is block-sparse: only the blocks a substep's particle stencils
   touch get nodes, from a pool of max_blocks blocks (plus 9 B per block of
   the domain for the block table), so memory follows the active blocks, not
   the domain. A substep that touches more blocks than the pool reports
   MPM_ERR_CAPACITY (its results are then not valid). Batches take dense
   contexts only. */
typedef struct {
  double dx;
  int32_t res[3];
  double origin[3];
  double gravity[3];
  int32_t bc_layers;
  int64_t max_particles;  /* capacity of the context */
  int64_t max_contacts;   /* contact points per substep (Sec. V-B) */
  int64_t max_blocks;     /* block-sparse pool (0: dense storage) */
} mpm_grid_spec;

/* Per particle group material. Lame parameters come from (E, nu);
   friction_angle_deg is used by MPM_DRUCKER_PRAGER only. */
typedef struct {
  int32_t model;
  float E;
  float nu;
  float rho;
  float friction_angle_deg;
} mpm_material;

/* A rigid body as seen by one time step (Sec. IV-A: pose and spatial
   velocity are frozen for the N substeps). R is the body-to-world rotation
   (row-major), p the body origin; omega and v are the angular velocity and
   the velocity of the body origin, world frame. mu is the friction
   coefficient; k [N/m] and d [s/m] are the stiffness and Hunt-Crossley
   dissipation of the compliant normal law of the lagged contact model
   (Sec. IV-B). If kinematic is nonzero the library advances the pose with
   the frozen velocity after each mpm_step; otherwise the pose is the
   caller's to update (static, or integrated by the caller's rigid solver
   from the impulses of mpm_get_rigid_impulses, Eq. (3)). */
typedef struct {
  int32_t shape;
  float params[4];
  float R[9];
  float p[3];
  float omega[3];
  float v[3];
  float mu;
  float k;
  float d;
  int32_t kinematic;
} mpm_rigid_body;

/* Dynamics of a rigid body that the library integrates itself (Eq. (3),
   without rigid-rigid contact): after each mpm_step its spatial velocity
   takes the step's external impulse and the contact impulses accumulated
   over the step's substeps,
     m (v+ - v) = dt (force + gravity * m) + sum_k impulse on the body,
     I (w+ - w) = dt (torque - w x I w) + sum_k moment of those impulses,
   with I = R diag(inertia) R^T and dt = n_substeps * h (semi-implicit
   Euler), then components outside dof_mask are zeroed and the pose advances
   with (v+, w+) as for a kinematic body. mass > 0; inertia: principal
   moments about the body origin in the body frame (kg m^2, > 0); force and
   torque: constant external load, world frame (N, N m); dof_mask: free
   degrees of freedom, bits 0-2 translation along world x, y, z, bits 3-5
   rotation about world x, y, z; gravity nonzero adds mass times the grid
   spec's gravity. */
typedef struct {
  float mass;
  float inertia[3];
  float force[3];
  float torque[3];
  int32_t dof_mask;
  int32_t gravity;
} mpm_rigid_dynamics;

/* Settings of the contact solve (Alg. 1). The iteration stops when
   ||M^-1/2 grad l_p|| < eps_a + eps_r max(||M^1/2 v||, ||M^-1/2 J^T gamma||);
   the paper's defaults are eps_r = 5e-2 and eps_a = machine epsilon (Sec. VI).
   eps_s [m/s] is the friction regularisation velocity of the lagged model.
   The exact line search stops when |f'(alpha)| <= ls_rel_tol |f'(0)| or
   after ls_max_iters evaluation passes (8 step lengths each); the paper
   leaves its tolerance open, and 1e-3 (the default) gave the same
   quasi-Newton iteration counts as 1e-5 on the benchmark scenes with 2-4x
   fewer passes. */
typedef struct {
  double eps_r;
  double eps_a;
  int32_t max_iters;
  float eps_s;
  float ls_rel_tol;
  int32_t ls_max_iters;
} mpm_solver_params;

/* Statistics of one mpm_step (all substeps). */
typedef struct {
  int32_t substeps;
  int32_t iters_total;       /* quasi-Newton iterations, summed over substeps */
  int32_t iters_max;
  int32_t ls_evals_total;    /* line-search evaluation passes */
  int32_t contacts_max;      /* contact points in one substep */
  int32_t active_blocks_max; /* 4^3 grid blocks swept in one substep */
  int64_t contacts_total;
  double residual_max;       /* max over substeps of the final
                                ||M^-1/2 grad|| / max(||M^1/2 v||, ||M^-1/2 J^T gamma||) */
  int32_t status_bits;       /* OR of (1 << mpm_status) seen on the device */
  int32_t p2g_global_chunks; /* P2G particle chunks too spread for one shared tile */
  /* device time of the contact solve's phases, summed over substeps [us]:
     contact-node list, gradient/Hessian scatter (G), node solve (N),
     line-search passes, impulses */
  float solve_us[5];
  /* substeps whose line-search passes were split over the solve's thread
     blocks, each pass ending in a device-wide reduction (more contacts than
     one block line-searches alone) */
  int32_t ls_split_substeps;
  /* substeps whose contact solve ran in one thread-block cluster (at most
     MPM_OPT_CLUSTER_CONTACTS contacts) */
  int32_t cluster_substeps;
  /* grid nodes in the stencil of at least one contact (the solve's DoFs), in
     one substep */
  int32_t contact_nodes_max;
} mpm_step_stats;

/* Create a context on the current CUDA device. `cuda_stream` is a
   cudaStream_t (NULL: the context creates its own stream). All device memory
   (particles, grid, contacts, sort buffers) is allocated here. */
mpm_status mpm_create(const mpm_grid_spec* spec, void* cuda_stream, mpm_ctx** out);

/* Free the context and all of its device memory. NULL is accepted. */
mpm_status mpm_destroy(mpm_ctx* ctx);

/* Message of the last failure on this context (static storage owned by the
   context; "" if none). Safe with ctx == NULL (returns a generic message). */
const char* mpm_last_error(const mpm_ctx* ctx);

/* Append n particles of one material with rest volume `particle_volume`
   (mass = rho * volume), positions x[n][3] and velocities v[n][3]; C = 0,
   F = I. Their ids are first_id .. first_id + n - 1 (first_id may be NULL).
   At most 65535 groups (calls) per context. */
mpm_status mpm_add_particles(mpm_ctx* ctx, int64_t n, const float* x, const float* v,
                             float particle_volume, const mpm_material* material,
                             int32_t mem_kind, int64_t* first_id);

/* Add a piece of cloth (the paper's cloth results, Sec. VI): a triangle mesh
   whose n_vertices vertices become particles of a new group with material
   `material` (model MPM_CLOTH; E, nu of the membrane, rho its density),
   x, v [n_vertices][3] in mem_kind memory. triangles [n_triangles][3] holds
   vertex indices 0 .. n_vertices - 1 of this call (host memory). The rest
   shape of each triangle is taken from x. Reading taken: the cloth's in-plane
   elasticity is a Lagrangian force of the mesh, the corotated membrane energy
   per triangle, rest area * thickness times mu |F - R|^2 + lam/2 (J - 1)^2 with
   F = Ds Dm^-1 (3x2), R its polar factor, J = det(sqrt(F^T F)); every substep
   the forces on the vertices are recomputed from their positions and P2G adds
   h f to their momentum. The vertices carry no stress; they collide with
   bodies, with the cloth itself and with other material through the grid and
   the contact solve. No bending. Each vertex has mass rho * thickness * (mesh
   area) / n_vertices. *first_id receives the first vertex's particle id.
   Contexts with cloth cannot record a tape or join a batch (MPM_ERR_STATE /
   MPM_ERR_INVALID_ARG there). */
mpm_status mpm_add_cloth(mpm_ctx* ctx, int64_t n_vertices, const float* x, const float* v,
                         int64_t n_triangles, const int32_t* triangles, float thickness,
                         const mpm_material* material, int32_t mem_kind, int64_t* first_id);

/* Pinned particles: Dirichlet conditions on particles (the paper's cloth
   experiment, Sec. VI, holds the cloth's corners by boundary conditions,
   moves them inward and releases two). Replaces the context's pin set:
   particle ids[j] (host memory, distinct, 0 <= id < number of particles)
   gets the prescribed velocity v[3j .. 3j+2] (m/s, host memory, finite);
   n_pins = 0 releases every pin (ids and v may then be NULL). From the next
   substep on, a pinned particle is kinematic: it enters each substep with
   v = v_pin and C = 0 (lending the grid its mass and momentum, and its
   stress if it has any), mesh forces on it are dropped, and after G2P it is
   put back on its path, x = (x at the substep's start) + h v_pin, v = v_pin,
   C = 0; F follows G2P. MPM_ERR_INVALID_ARG for a bad set, MPM_ERR_STATE
   while a tape is recording; contexts with pins cannot record a tape or
   step in a batch. Synchronises. */
mpm_status mpm_set_pins(mpm_ctx* ctx, int64_t n_pins, const int64_t* ids, const float* v);

/* Number of particles in the context. */
mpm_status mpm_num_particles(const mpm_ctx* ctx, int64_t* n);

/* Overwrite the state of all particles, in id order. Any of x, v, C, F may be
   NULL to keep that field (used for checkpoint restore and for starting a
   substep from a given state). */
mpm_status mpm_set_particles(mpm_ctx* ctx, const float* x, const float* v, const float* C,
                             const float* F, int32_t mem_kind);

/* Read the state of all particles, in id order. NULL skips a field. */
mpm_status mpm_get_particles(mpm_ctx* ctx, float* x, float* v, float* C, float* F,
                             int32_t mem_kind);

/* Change the material of particle group `group` (0-based, in the order of
   mpm_add_particles calls): model, E, nu, friction angle; the density, and
   with it the particle mass, must stay the same (MPM_ERR_INVALID_ARG
   otherwise). The stored stresses are recomputed. Not allowed while a tape
   is recorded (MPM_ERR_STATE). Synchronises. */
mpm_status mpm_set_material(mpm_ctx* ctx, int32_t group, const mpm_material* mat);

/* Replace the rigid bodies (at most 16). They apply from the next mpm_step. */
mpm_status mpm_set_rigid_bodies(mpm_ctx* ctx, int32_t n, const mpm_rigid_body* bodies);

/* Current rigid bodies (kinematic and dynamic ones after their pose
   updates; synchronises the context's stream when the device moved them). */
mpm_status mpm_get_rigid_bodies(const mpm_ctx* ctx, int32_t n, mpm_rigid_body* out);

/* Make body `index` (of the current set) dynamic with `dyn`, or, with dyn
   NULL, stop integrating it (it keeps its current pose and velocity and
   its kinematic flag applies again). A dynamic body's kinematic flag is
   ignored. The bodies' update after each step (this one, and the kinematic
   advance) runs on the device, one warp per body, inside the step's launch
   sequence, so mpm_step does not wait for it; while a tape records
   (mpm_tape_begin) the host integrates the bodies instead, synchronising at
   the end of each step. mpm_set_rigid_bodies clears all dynamics. */
mpm_status mpm_set_rigid_dynamics(mpm_ctx* ctx, int32_t index, const mpm_rigid_dynamics* dyn);

/* One rigid time step: n_substeps MPM substeps of size h with the rigid
   bodies frozen (Eq. (4)). The particle order is refreshed (radix sort) at
   the start of the step and reused by all substeps (Sec. V-A). Kinematic
   bodies then advance by n_substeps*h; dynamic bodies (see
   mpm_set_rigid_dynamics) are integrated with the step's impulses. `solver` may be NULL for the paper's
   defaults (eps_r = 5e-2, eps_a = DBL_EPSILON, eps_s = 1e-4 m/s; max_iters
   1000, ls_rel_tol 1e-3, ls_max_iters 50). With
   `stats` non-NULL the call synchronises, fills it and returns the first
   device-side failure; with NULL it returns without waiting. */
mpm_status mpm_step(mpm_ctx* ctx, double h, int32_t n_substeps,
                    const mpm_solver_params* solver, mpm_step_stats* stats);

/* Per body, the impulse on the body (3) and its moment about the body origin
   p (3), summed over the substeps since the last reset (the sum over k of
   J_r^T gamma_d^{n,k} in Eq. (3)); out has 6*n_bodies doubles, host memory.
   reset != 0 zeroes the accumulators after reading. */
mpm_status mpm_get_rigid_impulses(mpm_ctx* ctx, double* out, int32_t reset);

/* Grid of the last substep: the nodes with mass, as linear ids
   i + res[0]*(j + res[1]*k), their mass, free-motion velocity v* (Eq. (6))
   and post-contact velocity v^{k+1} (Eq. (8)). Host arrays of capacity `cap`
   (ids may not come sorted); *count receives the number of nodes even when
   it exceeds cap. Any array may be NULL. Diagnostic / testing call. */
mpm_status mpm_get_grid(mpm_ctx* ctx, int64_t cap, int64_t* count, int32_t* node_ids,
                        float* m, float* vstar, float* v);

/* Same readback as mpm_get_grid, but allocating nothing, for callers that
   cannot call cudaMalloc at this point: code that must not let an allocation
   synchronise the device or fail mid-run (real-time loops, pools that own all
   device memory), or that runs where allocation is not allowed. The paper has
   no counterpart; this is a property of the library only.
   The compacted grid is staged in one array inside the library, a file-scope
   __device__ buffer of 262,144 nodes (8,388,864 bytes, 8.4 MB) that every GPU loading the
   library holds until the process exits. The last substep may have swept at
   most 262,144 nodes (4096 blocks of 4^3), else MPM_ERR_CAPACITY (use
   mpm_get_grid). The first call on a device looks up the buffer's address
   (with that device current; the context's device must be current), so make
   that first call before any stream capture. Every call reuses the same
   buffer: calls that overlap on the GPU (from several threads or contexts of
   one device) race and must be serialised by the caller. Synchronises the
   context's stream; host output arrays as in mpm_get_grid. */
mpm_status mpm_get_grid_noalloc(mpm_ctx* ctx, int64_t cap, int64_t* count, int32_t* node_ids,
                                float* m, float* vstar, float* v);

/* Contacts of the last substep (one per particle inside a body, Sec. V-B):
   particle id, body index, impulse on the particle (world frame, 3),
   penetration depth and lagged normal impulse. Host arrays, as above. */
mpm_status mpm_get_contacts(mpm_ctx* ctx, int64_t cap, int64_t* count, int32_t* particle,
                            int32_t* body, float* gamma, float* phi0, float* n0);

/* Adjoint of the last substep's contact solve (the contact problem of
   Eq. (7)-(8) as it stood at the end of the last mpm_step), by implicit
   differentiation of its optimality condition
     M (v - v*) + J^T dl_c(J v + b) = 0   on the free grid DoFs,
   where b = -v_r(x_p) is minus the frozen body velocity at each contact point
   and l_c is the lagged contact potential of Sec. IV-B. The paper does not
   differentiate its solver; this is an extension of the library.
   Given vbar = dL/dv for a loss L of the post-contact grid velocity v, let
   lambda solve (M + J^T d2l_c J) lambda = vbar on the free DoFs (the exact
   Hessian: the 3x3 blocks of Eq. (10) and their couplings). Then
     dL/dv*      = M lambda on free nodes; on Dirichlet or massless nodes
                   (where v = v*) vbar - (J^T d2l_c J lambda);
     dL/dv_r(x_p) = d2l_c (J lambda)_c   per contact (world frame);
     dL/dmu_c    = -(n0 / s) u_t . (J lambda)_c   per contact,
   with u_t the tangential relative velocity at the solution and
   s = sqrt(|u_t|^2 + eps_s^2). The lagged depth phi0 and normal impulse n0
   are held fixed. lambda is found by conjugate gradients preconditioned by
   the 3x3 diagonal blocks of the Hessian, in one cooperative launch.

   Inputs (mem_kind MPM_MEM_HOST or MPM_MEM_DEVICE for all four node and
   contact arrays): n grid nodes as linear ids i + res[0]*(j + res[1]*k)
   (the ids of mpm_get_grid), each in [0, res[0]*res[1]*res[2]), and vbar
   [n][3]. Nodes not listed have vbar = 0; a node listed twice has its vbar
   summed and both entries receive the node's result.
   Outputs: vstar_bar [n][3] = dL/dv* at the listed nodes (vbar itself at a
   node outside the contacts' stencils, where v = v* + 0); contact_bar
   [contact_cap][4] (may be NULL with contact_cap 0): per contact, in the
   order of mpm_get_contacts, dL/dv_r(x_p) (3) and dL/dmu_c, rows beyond the
   contact count untouched; body_bar [n_bodies][7] doubles (may be NULL): per
   body of the last step, dL/dv (3) and dL/domega (3) of its spatial velocity
   (through b only: v_r(x) = v + omega x (x - p)) and dL/dmu.
   params may be NULL for eps_r = 1e-5 (stop when the residual's P^-1 norm
   falls below eps_r times vbar's) and max_iters = 1000.
   Errors: MPM_ERR_STATE before any mpm_step with n_substeps > 0;
   MPM_ERR_INVALID_ARG for bad arguments or (host ids) an id outside the
   grid, checked before any work; device ids outside the grid are reported
   after the call as MPM_ERR_INVALID_ARG and give zeros; MPM_ERR_NOT_CONVERGED
   if max_iters was reached (outputs hold the last iterate). A device-side
   failure of an earlier call is returned first, without computing.
   Synchronises the context's stream; the grid, contacts and particles are
   left as they were (mpm_get_grid / mpm_get_contacts still read them). */
typedef struct {
  double eps_r;
  int32_t max_iters;
} mpm_adjoint_params;

typedef struct {
  int32_t iters;          /* conjugate-gradient iterations */
  float residual;         /* final |r|_P^-1 / |vbar|_P^-1 on the contact nodes */
  int32_t contacts;       /* contacts of the differentiated substep */
  int32_t contact_nodes;  /* grid nodes in their stencils */
} mpm_adjoint_stats;

mpm_status mpm_contact_adjoint(mpm_ctx* ctx, int32_t mem_kind, int64_t n, const int32_t* node_ids,
                               const float* vbar, float* vstar_bar, int64_t contact_cap,
                               float* contact_bar, double* body_bar,
                               const mpm_adjoint_params* params, mpm_adjoint_stats* stats);

/* Reverse-mode differentiation of a rollout (mpm_backward). The paper does
   not differentiate its simulator; this is an extension of the library.

   mpm_tape_begin clears any previous tape and starts recording: every
   following mpm_step (with n_substeps > 0) stores a checkpoint of the
   particle state at its start (device memory, 96 bytes per particle) with the
   step's frozen bodies, h and solver parameters, and each substep's solved
   velocities on its contact nodes (16 bytes per contact node, in a pool of
   16M entries allocated at the first mpm_tape_begin; substeps beyond it are
   re-solved by the backward). mpm_tape_end stops recording and keeps the
   tape. Adding particles while recording is an error at the next mpm_step;
   setting the particles (mpm_set_particles) or the bodies
   (mpm_set_rigid_bodies) between two recorded steps breaks the chain from
   one step's end state to the next one's start, and mpm_backward then
   refuses the tape (setting them after mpm_tape_begin, before the first
   recorded step, is fine). The adjoints cover neither cloth nor pinned
   particles: mpm_tape_begin returns MPM_ERR_STATE for a context with either. */
mpm_status mpm_tape_begin(mpm_ctx* ctx);
mpm_status mpm_tape_end(mpm_ctx* ctx);

typedef struct {
  int32_t steps;          /* recorded steps differentiated */
  int32_t substeps;       /* substeps differentiated */
  int32_t last_iters;     /* CG iterations of the last contact adjoint */
  float last_residual;    /* its relative residual */
} mpm_backward_stats;

/* Gradient of a loss L of the state after the last recorded step with
   respect to the state before the first one and to the parameters, by the
   adjoint of every substep in reverse: G2P with the constitutive update,
   the contact solve by implicit differentiation of its optimality condition
   (as in mpm_contact_adjoint, Eq. (8)-(9), plus the dependence of the lagged
   contact terms phi0, n, n0 and of the contact velocity's bias and stencil
   on the particle state), the grid update and P2G (with the weights'
   gradient and the stress: fixed-corotated through its polar decomposition,
   Hencky with the Drucker-Prager return map through the singular value
   decomposition).
   Each recorded step is replayed from its checkpoint once to rebuild its
   substep states; each substep's grid and contact solve are then recomputed
   before its adjoint (the solves start from the recorded solutions), so
   memory is one checkpoint per step plus one step's substep states.

   Inputs, in id order and caller layout (x, v [n][3]; C, F [n][3][3]), any
   may be NULL for zero: dL/dx, dL/dv, dL/dC, dL/dF of the final state; and
   body_state_bar [n_bodies][12] doubles (host memory, NULL for zero): dL/dv,
   dL/dp, dL/domega, dL/dtheta of each body's state after the last step
   (theta a world-frame rotation R -> exp([theta]x) R).
   Outputs (NULL to skip): the same four for the state at the start of the
   first recorded step; material_bar [n_groups][2] doubles = dL/dE, dL/dnu
   per particle group (in the order the groups were added); body_bar
   [n_bodies][13] doubles per body index = dL/dmu, dL/dv (3), dL/dp (3),
   dL/domega (3) and dL/dtheta (3), where v and omega are the body's (frozen)
   linear and angular velocity over the recorded steps, p its position at the
   first one and theta a rotation of its orientation R there (R -> exp([theta]x) R,
   world frame): they enter every contact's bias, lagged normal impulse and
   geometry (through R^T (x - p)), and a kinematic body's pose advances by
   n_substeps h (v, omega) after each step. For a dynamic body
   (mpm_set_rigid_dynamics) v, omega, p, theta are its state at the first
   recorded step and the backward runs through each rigid step of Eq. (3):
   the step's impulse and moment depend on the contact solves (their
   cotangents enter the implicit differentiation as an extra right-hand side
   and in the contact terms), and the state's own update is differentiated
   on the host. A body must keep its kind over the tape.
   The contact solve's adjoint is solved to params->eps_r (NULL: 1e-6, 2000
   iterations); the implicit gradient is exact at an exact minimiser, so the
   recorded steps should use a tight solver tolerance.
   The return map's branch boundaries (tension, the yield cone) and the
   Hencky clamp are kinks where the one-sided derivatives differ; sand
   starting exactly at F = I with a uniform velocity sits on one.
   Requires: a tape whose steps each start where the previous one ended;
   the same particles (MPM_ERR_STATE otherwise).
   Synchronises; afterwards the particle state is the final state again, the
   impulse accumulators are as before, and the tape is kept; the grid and
   contacts hold a replayed substep, so mpm_contact_adjoint needs an
   mpm_step first (MPM_ERR_STATE otherwise). */
mpm_status mpm_backward(mpm_ctx* ctx, int32_t mem_kind, const float* x_bar, const float* v_bar,
                        const float* C_bar, const float* F_bar, const double* body_state_bar,
                        float* x0_bar, float* v0_bar, float* C0_bar, float* F0_bar,
                        double* material_bar, double* body_bar, const mpm_adjoint_params* params,
                        mpm_backward_stats* stats);

/* Wait for the context's stream and report any device-side failure. */
mpm_status mpm_synchronize(mpm_ctx* ctx);

/* Options. MPM_OPT_PROFILE: nonzero records CUDA events around each phase of
   each substep (read with mpm_get_phase_times). MPM_OPT_SORT_EVERY: sort the
   particles every k-th time step (default 1). MPM_OPT_P2G_CHUNK: particles
   per P2G thread block (256, 512 or 1024; default 256). MPM_OPT_GRAPHS:
   nonzero (default) records each step's launch sequence once as a CUDA graph
   and replays it while the particle count, substep count, h, solver
   parameters, body count and launch options stay the same (a change
   re-records; profiling launches directly); zero always launches directly.
   MPM_OPT_SOLVE_BLOCKS: at most this many thread blocks (one per SM) work on
   the contact solve (0, the default: as many as the device holds); a small
   cap lets contexts on other streams run beside a small scene's solve.
   MPM_OPT_TEST_BARRIER_TIMEOUT: for testing failure detection only; nonzero
   makes each device-wide barrier of the contact solve wait for one arrival
   more than there are blocks, so that (with two or more participating
   blocks) it gives up after its 1 s limit, the solve returns and the step
   reports MPM_ERR_TIMEOUT; the context stays usable.
   MPM_OPT_TAPE_SOLUTIONS: capacity, in contact nodes, of the pool in which a
   recorded rollout keeps each substep's contact-node solutions for
   mpm_backward (default 16,777,216 = 256 MB; 0: keep none, the backward then
   solves every replayed substep from v*); applies from the next
   mpm_tape_begin.
   MPM_OPT_CLUSTER_CONTACTS: a substep with at most this many contacts is
   solved by one thread-block cluster (up to 16 SMs exchanging their sums
   through distributed shared memory, hardware cluster barriers); more
   contacts go to the cooperative launch over as many SMs as they need, with
   device-wide barriers (default 4096; 0: always the cooperative launch).
   MPM_OPT_CLUSTER_BLOCKS: thread blocks (SMs) in that cluster, a power of two
   up to the largest the device schedules (0, the default: the largest, 16 on
   GB300).
   MPM_OPT_P2G_FORM: how a warp combines the contributions of particles that
   share a cell: MPM_P2G_GATHER (0, the default; lane j sums node j of a
   cell's stencil over the cell's particles, fastest at several particles per
   cell) or MPM_P2G_SCATTER (1; each lane computes its own particle's 27
   contributions and lanes of one cell combine them by shuffles, fastest at
   about one particle per cell). Same results up to rounding order. */
enum {
  MPM_OPT_PROFILE = 1,
  MPM_OPT_SORT_EVERY = 2,
  MPM_OPT_P2G_CHUNK = 3,
  MPM_OPT_GRAPHS = 4,
  MPM_OPT_SOLVE_BLOCKS = 5,
  MPM_OPT_TEST_BARRIER_TIMEOUT = 6,
  MPM_OPT_TAPE_SOLUTIONS = 7,
  MPM_OPT_CLUSTER_CONTACTS = 8,
  MPM_OPT_CLUSTER_BLOCKS = 9,
  MPM_OPT_P2G_FORM = 10
};
enum { MPM_P2G_GATHER = 0, MPM_P2G_SCATTER = 1 };
mpm_status mpm_set_option(mpm_ctx* ctx, int32_t option, int64_t value);

/* Phases timed when profiling is on. */
enum {
  MPM_PHASE_SORT = 0,       /* key, radix sort, permute (once per step) */
  MPM_PHASE_P2G = 1,        /* particle-to-grid + contact registration */
  MPM_PHASE_GRID = 2,       /* block compaction + grid update */
  MPM_PHASE_SOLVE = 3,      /* quasi-Newton contact solve */
  MPM_PHASE_G2P = 4,        /* grid-to-particle + constitutive update */
  MPM_NUM_PHASES = 5
};

/* Accumulated milliseconds and launch counts per phase since the last reset
   (arrays of MPM_NUM_PHASES; either may be NULL). Synchronises. */
mpm_status mpm_get_phase_times(mpm_ctx* ctx, double* ms, int64_t* launches, int32_t reset);

/* ---- Batches: many small scenes advanced by the launches of one ---------
   Launch overhead dominates small scenes (Sec. V-A: the per-substep kernel
   launches and host-device synchronisations). A batch advances n
   independent contexts together so that one substep of ALL of them costs
   five launches: P2G (with contact registration), block compaction, grid
   update, contact solve (Alg. 1) and G2P, each over a work list of
   (scene, thread block) items that covers every scene, plus one launch at
   the start and one at the end of the time step (the latter moves every
   scene's bodies on the device as mpm_step does, Eq. (3)-(4)). The time
   step replays as one CUDA graph. Each scene's contact solve runs in one
   thread block (or one thread-block cluster) of its own: its reductions need
   no device-wide barrier.

   Members are contexts created on the same device with the SAME
   cuda_stream (the batch's stream), none recording a tape; the caller keeps
   ownership and destroys them after the batch. Each member keeps its own
   particles, grid, bodies, dynamics, impulse accumulators and status, and
   every per-context entry point stays valid on a member between batch steps
   (the shared stream orders it). The batch sorts each member's particles
   once when it is created and again on mpm_batch_sort; its steps do not
   sort. After a batch step a member's contact adjoint is not available
   (mpm_contact_adjoint returns MPM_ERR_STATE until its next mpm_step).
   Particle counts may differ between members (uneven scenes). Any contact
   count is solved, each scene's in its one block: the batch suits scenes of
   up to a few thousand contacts, larger ones belong in their own context. */
typedef struct mpm_batch mpm_batch;

/* Create a batch of n >= 1 members. MPM_ERR_INVALID_ARG if a member is NULL,
   repeated, on another device or stream, recording a tape, block-sparse
   (max_blocks), or holds cloth or pinned particles (a batch step returns
   MPM_ERR_STATE for a member that gained them since). */
mpm_status mpm_batch_create(mpm_ctx* const* ctxs, int32_t n, mpm_batch** out);

/* One rigid time step of every member: n_substeps substeps of size h with
   the solver parameters (NULL: the defaults of mpm_step), then the bodies'
   update. Asynchronous; failures are reported by mpm_batch_synchronize. */
mpm_status mpm_batch_step(mpm_batch* batch, double h, int32_t n_substeps,
                          const mpm_solver_params* solver);

/* Re-sort every member's particles by grid block (per-member launches, not
   part of the step's graph). Asynchronous. */
mpm_status mpm_batch_sort(mpm_batch* batch);

/* Wait for the batch's stream. status [n] (may be NULL): each member's
   status (MPM_OK or its first device-side failure, which is then cleared);
   stats [n] (may be NULL): each member's statistics of the last batch step,
   as mpm_step reports them (status_bits: the member's status word at the
   step's end). Returns the first member failure in member order, or MPM_OK. */
mpm_status mpm_batch_synchronize(mpm_batch* batch, int32_t* status, mpm_step_stats* stats);

/* Launch options of the batch (autotuned by the Python binding):
   MPM_BATCH_OPT_GRAPHS: nonzero (default) replays the step as a CUDA graph;
   MPM_BATCH_OPT_P2G_CHUNK: particles per P2G thread block, 256, 512 or 1024
     (32, 64 or 128 per warp tile; default 256);
   MPM_BATCH_OPT_G2P_THREADS: threads (= particles) per G2P block, 64 to 512
     in multiples of 32 (default 256);
   MPM_BATCH_OPT_GRID_PARTICLES: a scene gets one grid-phase block per this
     many particles (at least one; default 2048);
   MPM_BATCH_OPT_SOLVE_BLOCKS: thread blocks per scene's contact solve, 1, 2, 4
     or 8 (default 1; more than one form a thread-block cluster per scene). The
     solves start largest scene (by particle count) first. */
enum {
  MPM_BATCH_OPT_GRAPHS = 1,
  MPM_BATCH_OPT_P2G_CHUNK = 2,
  MPM_BATCH_OPT_G2P_THREADS = 3,
  MPM_BATCH_OPT_GRID_PARTICLES = 4,
  MPM_BATCH_OPT_SOLVE_BLOCKS = 5
};
mpm_status mpm_batch_set_option(mpm_batch* batch, int32_t option, int64_t value);

/* Message of the batch's last failure (never NULL). */
const char* mpm_batch_last_error(const mpm_batch* batch);

/* Free the batch's own memory (not the members). Synchronises. */
void mpm_batch_destroy(mpm_batch* batch);

#ifdef __cplusplus
}
#endif
#endif /* MPMCR_H */
