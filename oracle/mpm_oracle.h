/*
 * mpm_oracle.h -- plain FP64 CPU oracle for one MPM substep coupled to rigid
 * bodies through the convex frictional-contact problem of Yu et al.,
 * "A Convex Formulation of Material Points and Rigid Bodies with
 * GPU-Accelerated Async-Coupling for Interactive Simulation" (arXiv 2503.05046).
 *
 * TEST INFRASTRUCTURE. This library is the slow, obviously-correct reference the
 * CUDA path is checked against. Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it. It shares no code, header,
 * table or helper with the CUDA library, and the CUDA library never calls it.
 *
 * Everything is FP64 and serial (a separate -fopenmp build of the same source,
 * used only as the all-core CPU baseline, threads the per-particle loops).
 * Conventions:
 *   - matrices are 3x3 row-major: M[3*r + c];
 *   - the grid is dense, node (ix,iy,iz) has linear id ix + rx*(iy + ry*iz) and
 *     position origin + dx*(ix,iy,iz);
 *   - z is up; a contact frame R_p has columns (t1, t2, n), so a contact
 *     velocity v_c = R_p^T u has components (v_t1, v_t2, v_n), v_n > 0 separating.
 *
 * Parity unpinned (no value in the paper fixes them): the contact stiffness k,
 * dissipation d and friction regularisation eps_s of the lagged contact model,
 * which the paper names (Sec. IV-B) but does not print; the line-search path
 * and iteration counts (only the converged minimiser is unique).
 */
#ifndef MPM_ORACLE_H
#define MPM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_OK = 0,
  ORC_ERR_OUT_OF_DOMAIN = 1,
  ORC_ERR_NOT_CONVERGED = 2,
  ORC_ERR_LINE_SEARCH = 3,
  ORC_ERR_ARG = 4,
  ORC_ERR_NOT_SPD = 5
};

enum { ORC_HALFSPACE = 0, ORC_SPHERE = 1, ORC_BOX = 2, ORC_CAPSULE = 3 };
enum { ORC_COROTATED = 0, ORC_DRUCKER_PRAGER = 1, ORC_CLOTH = 2 };

typedef struct {
  double dx;
  int res[3];
  double origin[3];
  double gravity[3];
  int bc_layers; /* nodes this close to the domain faces are held at v = 0 */
} orc_grid;

typedef struct {
  int shape;        /* ORC_HALFSPACE (plane z=0 of the body frame, +z outward),
                       ORC_SPHERE (params[0] = radius),
                       ORC_BOX (params[0..2] = half extents),
                       ORC_CAPSULE (params[0] = half length along body z,
                                    params[1] = radius) */
  double params[4];
  double R[9];      /* body -> world rotation */
  double p[3];      /* body origin, world */
  double omega[3];  /* angular velocity, world */
  double v[3];      /* velocity of the body origin, world */
  double mu, k, d;  /* friction coefficient, stiffness [N/m], dissipation [s/m] */
  int kinematic;    /* 1: pose advanced with its velocity after each time step */
} orc_body;

typedef struct {
  int model;        /* ORC_COROTATED or ORC_DRUCKER_PRAGER */
  double E, nu;
  double friction_angle_deg; /* Drucker-Prager only */
} orc_material;

typedef struct {
  double eps_r, eps_a; /* Alg. 1 stopping tolerances */
  int max_iters;       /* quasi-Newton iteration cap */
  double eps_s;        /* friction regularisation velocity [m/s] */
  double ls_rel_tol;   /* line search stops when |f'(a)| <= ls_rel_tol |f'(0)| */
  int ls_max_iters;
} orc_solver;

/* The contact problem of Eq. (7)-(8) over a set of grid DoFs. */
typedef struct {
  int n_nodes;
  const double* m;      /* [n_nodes] lumped masses (> 0) */
  const double* vstar;  /* [3 n_nodes] free-motion velocity */
  const int* fixed;     /* [n_nodes] 1: Dirichlet node, v held at vstar; may be NULL */
  int n_contacts;
  const int* nodes;     /* [27 n_contacts] DoF index or -1 */
  const double* w;      /* [27 n_contacts] transfer weights */
  const double* R;      /* [9 n_contacts] contact frames */
  const double* b;      /* [3 n_contacts] bias velocity, contact frame */
  const double* phi0;   /* [n_contacts] penetration depth (> 0) */
  const double* n0;     /* [n_contacts] lagged normal impulse */
  const double* mu;
  const double* k;
  const double* d;
  double h;             /* substep size */
  double eps_s;
} orc_problem;

typedef struct {
  int iters;          /* quasi-Newton iterations taken */
  int converged;
  int ls_evals;       /* line-search derivative evaluations in total */
  double G, P, J;     /* last ||M^-1/2 g||, ||M^1/2 v||, ||M^-1/2 J^T gamma|| */
  int status;
} orc_solve_info;

/* ---- building blocks (each pinned by the test suite) ---------------------- */

/* Quadratic B-spline stencil of a particle at x (MLS-MPM transfer kernel). */
void orc_bspline(double dx, const double origin[3], const double x[3],
                 int base[3], double fx[3], double w[9]);

/* F = U diag(S) V^T with U, V proper rotations, S sorted by magnitude,
   S[2] < 0 iff det F < 0 (one-sided Jacobi). */
void orc_svd3(const double F[9], double U[9], double S[3], double V[9]);

/* Lame parameters from (E, nu). */
void orc_lame(double E, double nu, double* mu, double* lam);

/* Fixed-corotated first Piola-Kirchhoff stress P(F) and Kirchhoff stress P F^T. */
void orc_corotated_P(const double F[9], double mu, double lam, double P[9]);
void orc_corotated_tau(const double F[9], double mu, double lam, double tau[9]);

/* Hencky (log-strain St.Venant-Kirchhoff) P and Kirchhoff stress, used with the
   Drucker-Prager model. */
void orc_hencky_P(const double F[9], double mu, double lam, double P[9]);
void orc_hencky_tau(const double F[9], double mu, double lam, double tau[9]);

/* Drucker-Prager return map in Hencky strain space; Fout may alias F. */
void orc_dp_project(const double F[9], double mu, double lam, double friction_angle_deg,
                    double Fout[9]);

/* Cloth (the paper's cloth results, Sec. VI): a triangle mesh whose vertices
   are MPM particles of an ORC_CLOTH material. Reading taken: the cloth's
   in-plane elasticity is a Lagrangian force of the mesh, the corotated
   membrane energy per triangle
     psi(F) = mu |F - R|^2 + lam/2 (J - 1)^2,   F = Ds Dm^-1 (3x2),
   R the 3x2 polar factor of F (F = R S, S = sqrt(F^T F)), J = det S, times
   the triangle's rest volume; Ds = [x1 - x0, x2 - x0], Dm the rest edges in
   the triangle's own plane. The particles carry no stress (F stays I); their
   P2G momentum gains h f_p with f_p = -dE/dx_p. Collision and self-collision
   go through the grid and the contact solve like any particle's. The energy
   of a triangle is psi times its rest volume (rest area times thickness). */

/* Rest shape of triangle (X0, X1, X2): Dm^-1 (2x2 row-major) and area. */
void orc_cloth_rest(const double X0[3], const double X1[3], const double X2[3],
                    double Dm_inv[4], double* area);
/* Energy of one triangle of rest volume vol and, if f is not NULL, the forces
   -dE/dx on its three vertices (f[9]). */
double orc_cloth_triangle(const double x0[3], const double x1[3], const double x2[3],
                          const double Dm_inv[4], double vol, double mu, double lam,
                          double f[9]);

/* Signed distance of a body at world point x and its outward unit normal. */
double orc_sdf(const orc_body* b, const double x[3], double n[3]);

/* Velocity of the body's material point at world x. */
void orc_body_velocity(const orc_body* b, const double x[3], double vel[3]);

/* Contact frame with z along n; t1 rotated by `angle` about n from the default. */
void orc_contact_frame(const double n[3], double angle, double R[9]);

/* Normal impulse gamma_n(v_n) of the compliant normal law. */
double orc_normal_impulse(double phi0, double k, double d, double h, double vn);

/* Lagged contact potential l_c at contact velocity vc = (vt1, vt2, vn):
   value, gradient and 3x3 Hessian (grad / hess may be NULL). */
double orc_contact_potential(double phi0, double n0, double mu, double k, double d,
                             double h, double eps_s, const double vc[3],
                             double grad[3], double hess[9]);

/* l_p(v) of Eq. (8) and its gradient, Eq. (9). */
double orc_objective(const orc_problem* P, const double* v);
void orc_gradient(const orc_problem* P, const double* v, double* g);

/* Alg. 1: block-diagonal quasi-Newton with exact line search.
   v: in = initial guess, out = solution. gamma: [3 nc] contact-frame impulses
   on the particles at the solution (may be NULL). hist: [max_iters+1]
   objective per iteration (may be NULL). */
int orc_solve_qn(const orc_problem* P, const orc_solver* S, double* v, double* gamma,
                 orc_solve_info* info, double* hist);

/* Same problem solved by full Newton (dense Hessian of Eq. (10), dense
   Cholesky) with the same line search. Tiny inputs only. */
int orc_solve_dense_newton(const orc_problem* P, const orc_solver* S, double* v,
                           double* gamma, orc_solve_info* info);

/* ---- one substep over particles ------------------------------------------ */

typedef struct orc_sim orc_sim;

typedef struct {
  int status;
  int n_contacts;
  int n_dofs;
  int iters;
  int converged;
  double G, P, J;
} orc_substep_info;

orc_sim* orc_create(const orc_grid* grid);
void orc_destroy(orc_sim* s);

/* The cloth meshes of the sim's particles: triangle t joins particles
   tris[3t..3t+2], with rest shape Dm_inv[4t..4t+3], rest volume vol[t] and
   the Lame parameters of material mat_of_tri[t] (copied). */
int orc_set_cloth(orc_sim* s, int n_tris, const int* tris, const double* Dm_inv,
                  const double* vol, const int* mat_of_tri);

/* Pinned particles (the held cloth corners of the paper's cloth experiment,
   Sec. VI: fixed by boundary conditions, moved inward, released). Reading
   taken: a Dirichlet condition on the particle itself. A pinned particle is
   kinematic: every substep it enters P2G with v = v_pin and C = 0 (it still
   lends the grid its mass and momentum, and its stress if it has one), mesh
   forces on it are dropped, and after G2P it is put back on its prescribed
   path, x = x_start + h v_pin, v = v_pin, C = 0 (F follows G2P). Replaces the
   pin set: particle ids[j] gets velocity v[3j..3j+2]; n_pins = 0 releases
   every pin. Ids must be distinct. */
int orc_set_pins(orc_sim* s, int n_pins, const int* ids, const double* v);

/* Threads orc_substep uses: 1 in the serial build (the checker); the
   OpenMP build (-fopenmp, a CPU baseline over all host cores only) runs P2G
   over alternating grid slabs, contact registration and G2P in parallel. */
int orc_threads(void);

/* One substep (Eq. (5)): free motion (Eq. (6)), contact registration, contact
   solve (Eq. (7)-(8), Alg. 1), G2P with the constitutive update. Particle
   arrays are updated in place. impulses [6 nb] accumulates, per body, the
   impulse on the body (3) and its moment about the body origin (3). */
int orc_substep(orc_sim* s, int n, double* x, double* v, double* C, double* F,
                const double* mass, const double* vol, const int* mat,
                int n_mat, const orc_material* mats, int nb, const orc_body* bodies,
                double h, const orc_solver* S, double* impulses, orc_substep_info* info);

/* Grid of the last substep: nodes with m > 0, ascending linear id. Returns the
   count; arrays may be NULL to query it. */
int orc_last_grid(const orc_sim* s, int cap, int* ids, double* m, double* vstar,
                  double* v);
/* Contacts of the last substep: particle, body, impulse on the particle in
   world frame, penetration, lagged normal impulse. Returns the count. */
int orc_last_contacts(const orc_sim* s, int cap, int* particle, int* body,
                      double* gamma_world, double* phi0, double* n0);

/* Adjoint of the contact solve by implicit differentiation of its optimality
   condition grad l_p(v) = 0 (Eq. (8)-(9)) at a minimiser v: with vbar = dL/dv,
   lambda solves H_hat lambda = vbar on the free DoFs, H_hat = M + J^T (d2 l_c) J
   the full Hessian (Eq. (10)); then
     dL/dv*   = M lambda on free DoFs, and vbar - J_x^T (d2 l_c) J lambda on
                Dirichlet DoFs (v = v* there, which the contacts see);
     dL/db_c  = -(d2 l_c) (J lambda)_c, contact frame (b: the bias velocity);
     dL/dmu_c = -(d/dmu dl_c/dv_c) . (J lambda)_c.
   vstar_bar [3 n_nodes], b_bar [3 n_contacts], mu_bar [n_contacts]. Dense
   Cholesky: small problems only. Returns ORC_OK or ORC_ERR_NOT_SPD. */
int orc_contact_adjoint(const orc_problem* P, const double* v, const double* vbar,
                        double* vstar_bar, double* b_bar, double* mu_bar);

/* Async time splitting (Eq. (3)-(4)): advance kinematic bodies by dt with their
   frozen velocity after the N substeps of a time step. */
void orc_advance_kinematic(int nb, orc_body* bodies, double dt);

/* A rigid body integrated with the contact impulses of a time step (Eq. (3),
   without rigid-rigid contact): mass, principal inertia about the body origin
   (body frame), constant external force and torque (world), free degrees of
   freedom (bits 0-2 translation along world x, y, z; bits 3-5 rotation about
   world x, y, z) and whether gravity acts on it. */
typedef struct {
  double mass;
  double inertia[3];
  double force[3];
  double torque[3];
  int dof_mask;
  int gravity;
} orc_dynamics;

/* One time step dt of Eq. (3): M (v+ - v) = dt k + J^T sum_k gamma with the
   step's impulse on the body (impulse[0..2], world) and its moment about the
   body origin (impulse[3..5]); k holds the external load, gravity and the
   gyroscopic term -w x (I w) at the start of the step; locked degrees of
   freedom are set to zero; the pose then advances with the new velocity. */
void orc_rigid_dynamics_step(orc_body* b, const orc_dynamics* d, const double gravity[3],
                             const double impulse[6], double dt);

#ifdef __cplusplus
}
#endif
#endif
