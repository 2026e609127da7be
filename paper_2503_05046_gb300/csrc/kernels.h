// kernels.h -- host-side launchers of the substep kernels (internal to the
// library; the public boundary is include/mpmcr.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace mpmcr {

constexpr int kRedDoubles = 4 * 256 * 16;  // contact-solve partial sums: 4 slots x 256 blocks x 16
// device-wide barrier of the cooperative solves: one 64-bit arrival counter
// (words 0 and 1) on a line of its own
constexpr int kBarWords = 32;

// Statistics written by the device, read back by mpm_step.
struct DevStats {
  int iters_total;
  int iters_max;
  int ls_evals_total;
  int contacts_max;
  int active_blocks_max;
  int substeps;
  unsigned long long contacts_total;
  float residual_max;
  int p2g_global_chunks;
  int last_contacts;     // contacts of the last substep
  int last_active;       // active blocks of the last substep
  int ls_split;          // substeps whose line search was split over the solve's blocks
  int cluster;           // substeps solved by one thread-block cluster
  int cnodes_max;        // contact nodes (the union of the contacts' stencils) in one substep
  // device time of the contact solve's phases (ns, block 0's view):
  // contact-node list, G, N, line search, impulses
  unsigned long long solve_ns[5];
};

// Scratch of the radix sort.
struct SortBuffers {
  uint32_t* keys[2];
  uint32_t* vals[2];
  uint32_t* hist;     // 256 * n_tiles
  uint32_t* partial;  // scan partials
  int hist_cap;
};

int sort_hist_len(int n);
cudaError_t sort_prepare();  // once per device: the small-scene sort's shared memory
// ---- sort.cu: block keys, LSD radix sort (8-bit digits), permutation ----
void launch_sort(const GridDev& g, const Particles& src, const Particles& dst, int n,
                 SortBuffers& sb, cudaStream_t s);
// gather particles of `src` into id order (out[pid] = state) for mem reads
void launch_to_id_order(const Particles& P, int n, float* out_x, float* out_v, float* out_C,
                        float* out_F, cudaStream_t s);
void launch_from_id_order(const Particles& P, int n, const float* in_x, const float* in_v,
                          const float* in_C, const float* in_F, cudaStream_t s);
// Kirchhoff stress planes from F (after F was set from outside)
void launch_stress_from_F(const Particles& P, int n, const DevGroup* groups, cudaStream_t s);

// ---- p2g.cu: particle-to-grid with shared-memory tiles + contact registration ----
struct P2GArgs {
  GridDev g;
  Particles P;
  int n;
  const DevGroup* groups;
  const DevBody* bodies;
  int nb;
  float h;
  GridArrays G;
  Contacts C;
  uint32_t* status;
  DevStats* stats;
  float* fext;  // cloth: per-particle mesh forces, 3 planes of fext_stride (null: none); P2G zeroes them
  long long fext_stride;
};
// form: MPM_P2G_GATHER or MPM_P2G_SCATTER
void launch_p2g(const P2GArgs& a, int chunk, int form, cudaStream_t s);
cudaError_t p2g_prepare();  // once per device: the kernel's shared-memory attributes

// ---- grid.cu: active-block compaction and grid update ----
void launch_grid(const GridDev& g, const GridArrays& G, float h, int num_sms, DevStats* stats,
                 cudaStream_t s);
// block-sparse grids, before P2G: the substep's blocks marked from the
// particles' stencils, compacted and given storage (slot_tab = g.slot)
void launch_sparse_map(const GridDev& g, const GridArrays& G, const Particles& P, int n,
                       int* slot_tab, uint32_t* status, int num_sms, cudaStream_t s);

// ---- solve.cu: quasi-Newton contact solve (Alg. 1) in one cooperative launch ----
struct SolveArgs {
  GridDev g;
  GridArrays G;
  Contacts C;
  const DevBody* bodies;
  int nb;
  float h;
  float eps_s;
  float ls_rel_tol;
  int ls_max_iters;
  double eps_r, eps_a;
  int max_iters;
  double* red;        // per-block partial sums [4][256][16]
  unsigned* bar;      // grid barrier counters [kBarWords]
  uint32_t* status;
  DevStats* stats;
  double* impulses;   // [6 nb]
  int wait_extra;     // 0; 1 makes every grid barrier wait for one block too many (test)
  int* poison;        // nonzero after a barrier gave up (set and cleared by the solve)
  int cluster_max;    // up to this many contacts one thread-block cluster solves (0: never)
};
// the cluster kernel (cluster_blocks > 0 and a.cluster_max > 0), then the
// cooperative one; each returns at once when the contact count is the other's
cudaError_t launch_solve(const SolveArgs& a, int grid_blocks, int cluster_blocks, cudaStream_t s);
int solve_cluster_blocks();  // largest cluster (16, 8 or 4 blocks) the device holds; 0: none
int solve_block_size();
const void* solve_kernel_ptr();
size_t solve_dynamic_smem();
cudaError_t solve_prepare();  // once per device, before the occupancy query

// ---- solve.cu: adjoint of the contact solve (implicit differentiation of
// Eq. (8)), conjugate gradients in one cooperative launch
struct AdjointArgs {
  GridDev g;
  GridArrays G;
  Contacts C;
  const DevBody* bodies;
  int nb;
  float h;            // substep of the differentiated solve
  float eps_s;        // its friction regularisation
  double eps_r;       // stop at |r|_P^-1 <= eps_r |vbar|_P^-1
  int max_iters;
  int n_in;           // (node id, vbar) pairs
  const int* ids;     // linear node ids i + rx (j + ry k)
  const float* vbar;  // [3 n_in]
  float* vstar_bar;   // [3 n_in]
  float* contact_bar; // [4 contact_cap]: dL/dv_r(x_p) (3), dL/dmu; may be null
  int contact_cap;
  double* body_bar;   // [kAdjBodySlots nb], zeroed by the caller
  float4* vec;        // kAdjointVectors x cnodes_cap float4
  double* red;
  unsigned* bar;
  uint32_t* status;
  int* poison;
  const DevStats* stats;  // last_contacts: the differentiated substep's contact count
  float* out;         // [4]: iterations, relative residual, contacts, contact nodes
  // mpm_backward mode (gbar non-null): vbar comes from the dense grid adjoint
  // gbar and (v*bar, mbar) go back into it on the contact nodes; the contact
  // geometry's adjoint is added to the particle adjoint planes `pbar` (slot
  // order, via slot_of[particle id]); the contact count is the live one
  float4* gbar;
  float* pbar;
  const int* slot_of;
  Particles P;
  int n_particles;
  // per body (6): the cotangent of the impulse and of its moment that the
  // substep's contacts give the body (dynamic bodies, Eq. (3)); null: none
  const double* body_gbar;
};
constexpr int kAdjointVectors = 13;
// per-body adjoint accumulators: dL/dv_r through the bias (3), its moment
// about the body origin (= dL/domega through the bias, 3), dL/dmu, and in
// mpm_backward mode dL/dp of the body position through the contact geometry
// (3), dL/dv through the lagged normal impulse (3), the adjoint of a left
// rotation of the body's orientation (3) and dL/domega through the lagged
// normal impulse (3)
constexpr int kAdjBodySlots = 19;
cudaError_t launch_adjoint(const AdjointArgs& a, int grid_blocks, cudaStream_t s);
const void* adjoint_kernel_ptr();

// ---- backward.cu: adjoints of G2P, the grid update and P2G (mpm_backward)
struct BackwardArgs {
  GridDev g;
  Particles P;        // the substep's start state (slot order)
  int n;
  const DevGroup* groups;
  GridArrays G;       // the substep's grid after P2G, grid update and solve
  float h;
  float4* gbar;       // dense grid adjoint
  const float* bin;   // adjoint of the substep's end state: 24 planes x n (slot order)
  float* bout;        // adjoint of its start state
  double* mat_bar;    // per group: dL/dmu_lame, dL/dlambda_lame
  uint32_t* status;
};
void launch_g2p_adjoint(const BackwardArgs& a, cudaStream_t s);
void launch_grid_adjoint(const BackwardArgs& a, int num_sms, cudaStream_t s);
void launch_p2g_adjoint(const BackwardArgs& a, cudaStream_t s);
void launch_reset_counters(const GridArrays& G, const Contacts& C, unsigned* bar, cudaStream_t s);
void launch_slot_map(const Particles& P, int n, int* slot_of, cudaStream_t s);
// taped solutions: append the contact-node velocities after a solve (counters:
// [0] pool fill, [1] records written); scatter record r over v*
void launch_tape_save(const GridDev& g, const GridArrays& G, int* counters, int2* recs, int rec_cap, float4* pool,
                      int pool_cap, int num_sms, cudaStream_t s);
void launch_tape_warm(const GridDev& g, const GridArrays& G, const int2* recs, int r, const float4* pool, int num_sms,
                      cudaStream_t s);
void launch_bar_in(const Particles& P, int n, const float* x, const float* v, const float* C,
                   const float* F, float* bar, cudaStream_t s);
void launch_bar_out(const Particles& P, int n, const float* bar, float* x, float* v, float* C,
                    float* F, cudaStream_t s);

// ---- cloth.cu: triangle-mesh membrane forces on cloth vertices ----
// rest shape of a triangle from its rest vertices: Dm^-1 (2x2 row-major), area
// (mpm_add_cloth replaces the area by the rest volume, area * thickness)
void cloth_rest_shape(const double X0[3], const double X1[3], const double X2[3], double out[5]);
// f (3 planes of `stride` floats, slot order, zero on entry: P2G zeroes what
// it consumes) += the mesh forces at the current positions; tris: (particle
// ids, group); rest: Dm^-1 and rest volume per triangle; pinned (by particle
// id, may be null): vertices that get no force
void launch_cloth_forces(const Particles& P, const int* slot_of, const int4* tris,
                         const double* rest, int n_tris, const DevGroup* groups,
                         const uint8_t* pinned, float* f, long long stride, cudaStream_t s);
// pinned particles: ids[j] (found through slot_of) with prescribed velocity
// (v_pin[j + c * cap]) and the substep's start position (x_pin[j + c * cap]).
// init, at a step's first substep: x_pin = the particle's x; its v = v_pin, C = 0
void launch_pin_init(const Particles& P, const int* slot_of, const int* ids, const float* v_pin,
                     float* x_pin, int n_pins, int cap, cudaStream_t s);
// after G2P: the particle's x = x_pin + h v_pin (and x_pin, the next
// substep's start), v = v_pin, C = 0
void launch_pins(const Particles& P, const int* slot_of, const int* ids, const float* v_pin,
                 float* x_pin, int n_pins, int cap, float h, cudaStream_t s);

// ---- rigid.cu: the bodies' update after a time step (Eq. (3)-(4)) ----
enum { kRigidStatic = 0, kRigidKinematic = 1, kRigidDynamic = 2 };
struct DevDyn {
  int kind;      // kRigid*
  int dof_mask;  // free DoFs of a dynamic body (bits 0-2 translation, 3-5 rotation)
  int gravity;   // nonzero: the body's weight is part of its load
  int pad;
  float mass;
  float inertia[3];  // principal moments, body frame
  float force[3];    // constant load, world frame
  float torque[3];
};
// one warp per body; imp - imp0 is the step's impulse and moment on each body
void launch_rigid_update(DevBody* bodies, const DevDyn* dyn, int nb, const double* imp,
                         const double* imp0, double dt, const double* gravity, cudaStream_t s);

// batched: one block per scene, at the start of a batch step (statistics
// cleared, imp0 = imp) and at its end (status and statistics gathered into
// status_out and stats_out, then, if `rigid`, the bodies moved as above)
struct RigidBatchArgs {
  DevBody* bodies;
  const DevDyn* dyn;
  int nb;
  int rigid;
  const double* imp;
  double* imp0;
  DevStats* stats;
  const uint32_t* status;
  double gravity[3];
};
void launch_batch_begin(const RigidBatchArgs* args, int n_scenes, cudaStream_t s);
void launch_batch_end(const RigidBatchArgs* args, int n_scenes, double dt, uint32_t* status_out,
                      DevStats* stats_out, cudaStream_t s);

// ---- g2p.cu: grid-to-particle with the constitutive update ----
struct G2PArgs {
  GridDev g;
  Particles P;
  int n;
  const DevGroup* groups;
  GridArrays G;
  Contacts C;
  float h;
  unsigned* bar;     // solve barrier, reset here
  double* red;       // solve reduction ring, reset here
  DevStats* stats;
};
void launch_g2p(const G2PArgs& a, cudaStream_t s);

// ---- batched launches: one per phase over many scenes' work items ----
// work[b] = (scene, block index within the scene); args: per scene, device
// memory. P2G blocks hold p2g_block_particles(chunk) particles, G2P blocks
// `threads` (<= 512); the grid phases give each scene n_slices blocks.
struct GridBatchArgs {
  GridDev g;
  GridArrays G;
  float h;
  int n_slices;
  DevStats* stats;
};
int p2g_block_particles(int chunk);
void launch_p2g_batch(const P2GArgs* args, const int2* work, int n_work, int chunk, cudaStream_t s);
void launch_grid_batch(const GridBatchArgs* args, const int2* work, int n_work, cudaStream_t s);
// each scene's contact solve by one block or one cluster of 2, 4 or 8 blocks,
// scenes in `order` (device, n_scenes entries)
cudaError_t launch_solve_batch(const SolveArgs* args, const int* order, int n_scenes,
                               int blocks_per_scene, cudaStream_t s);
void launch_g2p_batch(const G2PArgs* args, const int2* work, int n_work, int threads,
                      cudaStream_t s);

}  // namespace mpmcr
