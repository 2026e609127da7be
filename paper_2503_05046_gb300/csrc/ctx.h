// ctx.h -- the context behind the opaque mpm_ctx handle (internal: shared
// by the single-context entry points in api.cu and the batch in batch.cu).
#pragma once

#include <string>
#include <utility>
#include <vector>

#include "kernels.h"

using namespace mpmcr;  // (internal header of the library's own sources)

struct mpm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  mpm_grid_spec spec{};
  GridDev g{};
  int64_t cap = 0, n = 0;
  int num_sms = 0, solve_blocks = 0;
  int cluster_blocks = 0;     // blocks of the cluster solve (0: the device runs none)
  int cluster_blocks_max = 0; // the largest cluster the device schedules
  int cluster_max = 4096;     // MPM_OPT_CLUSTER_CONTACTS
  float* pbuf[2] = {nullptr, nullptr};
  uint32_t* pidbuf[2] = {nullptr, nullptr};
  uint16_t* grpbuf[2] = {nullptr, nullptr};
  Particles P[2];
  int cur = 0;
  std::vector<DevGroup> groups;
  DevGroup* groups_d = nullptr;
  int groups_cap = 0;
  std::vector<mpm_rigid_body> bodies;
  // dynamic bodies (Eq. (3)): per body, integrated by the library if set
  std::vector<int> is_dyn;
  std::vector<mpm_rigid_dynamics> dyn;
  std::vector<double> imp_seen;  // impulse accumulator at the end of the last step
  bool imp_seen_valid = false;
  DevBody* bodies_d = nullptr;
  bool bodies_dirty = true;
  // the bodies' motion on the device between steps (rigid.cu): each body's
  // kind and dynamics, and the impulse accumulator at the step's start
  DevDyn* dyn_d = nullptr;
  double* imp0_d = nullptr;
  DevBody* bodies_step_d = nullptr;  // the last step's frozen bodies (device update)
  bool last_dev_rigid = false;
  bool dyn_dirty = true;
  bool bodies_stale = false;  // the device moved the bodies since the host copy
  GridArrays G{};
  size_t n_nodes = 0;   // nodes of storage
  int n_blocks = 0;     // 4^3 blocks of the domain
  int* slot_d = nullptr;  // block-sparse grids: block -> storage block (g.slot)
  // cloth meshes (mpm_add_cloth): triangles (particle ids, group), rest shapes
  // (Dm^-1, rest volume) and the vertices' forces (3 planes of cap)
  std::vector<int4> cloth_tris;
  std::vector<double> cloth_rest;
  int4* cloth_tris_d = nullptr;
  double* cloth_rest_d = nullptr;
  float* cloth_f_d = nullptr;
  // pinned particles (mpm_set_pins): ids, prescribed velocities (3 planes of
  // pins_cap) and positions on their paths (3 planes of pins_cap)
  int n_pins = 0;
  int pins_cap = 0;
  int* pin_ids_d = nullptr;
  float* pin_v_d = nullptr;
  float* pin_x_d = nullptr;
  uint8_t* pin_mask_d = nullptr;  // by particle id: 1 if pinned (cap bytes)
  // particle id -> slot map of the buffer the substeps run on (cloth, pins)
  int* slot_of_d = nullptr;
  Contacts C{};
  double* red = nullptr;
  unsigned* bar = nullptr;
  int* poison = nullptr;
  uint32_t* status = nullptr;
  DevStats* stats = nullptr;
  double* impulses = nullptr;
  SortBuffers sb{};
  float* stage = nullptr;  // 24 floats per particle
  bool profile = false;
  // CUDA graphs of the step's launch sequence, one per particle buffer the
  // step starts from (the sort ping-pongs between the two), re-captured when
  // anything baked into the launches changes
  bool use_graphs = true;
  struct GraphKey {
    int64_t n = -1;
    int n_substeps = 0, nb = 0, chunk = 0, sort_now = 0, solve_blocks = 0, taping = 0;
    int cluster_max = 0;
    int cluster_blocks = 0;
    int p2g_form = 0;
    int rigid = 0;
    const void* tape_pool = nullptr;  // baked into the launches when taping
    float h = 0.f;
    mpm_solver_params sp{};
  } gkey[2];
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  int solve_blocks_cap = 0;  // 0: as many as the device holds
  bool wait_test = false;    // MPM_OPT_TEST_BARRIER_TIMEOUT
  int sort_every = 1;
  int p2g_chunk = 256;
  int p2g_form = 0;  // MPM_P2G_GATHER / MPM_P2G_SCATTER
  int64_t step_count = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, cudaEvent_t>> ev_marks;  // (phase starting at this event, event)
  double phase_ms[MPM_NUM_PHASES] = {0};
  int64_t phase_n[MPM_NUM_PHASES] = {0};
  // the last substep, for mpm_contact_adjoint
  bool adj_ready = false;
  float last_h = 0.f, last_eps_s = 0.f;
  int last_nb = 0;
  // the adjoint's device buffers, allocated at its first call
  float4* adj_vec = nullptr;       // kAdjointVectors x cnodes_cap
  double* adj_body = nullptr;      // kAdjBodySlots per body
  float* adj_out = nullptr;        // iterations, residual, contacts, contact nodes
  int adj_blocks = 0;
  int32_t* adj_ids = nullptr;      // staging of host inputs and outputs
  float* adj_io = nullptr;         // vbar (3n), vstar_bar (3n), contact_bar (4 cap)
  size_t adj_ids_cap = 0, adj_io_cap = 0;
  // materials as given, per particle group (for dL/dE, dL/dnu)
  std::vector<mpm_material> mats;
  // mpm_backward tape: per recorded mpm_step, the particle state at its start
  // (id order, x v C F = 24 floats per particle, one device buffer each), its
  // frozen bodies, substep size and count, and solver parameters
  struct TapeStep {
    float* state = nullptr;
    int rec_base = 0;  // record index of the step's first substep solution
    std::vector<DevBody> bodies;
    std::vector<int> kinematic;  // per body: its pose advances by n_substeps h v after the step
    std::vector<int> is_dyn;     // per body: integrated by the library after the step (Eq. (3))
    std::vector<mpm_rigid_dynamics> dyn;
    std::vector<double> imp;     // per body: the step's impulse and moment (6)
    int n_substeps = 0;
    float h = 0.f;
    mpm_solver_params sp{};
  };
  bool taping = false;
  bool tape_reset = false;  // particles or bodies set between two recorded steps
  int64_t tape_n = 0;
  std::vector<TapeStep> tape;
  // the contact-node solutions of the taped substeps (see launch_tape_save)
  float4* tape_pool = nullptr;
  int2* tape_recs = nullptr;
  int* tape_counters = nullptr;  // [0] pool fill, [1] records written
  int tape_pool_cap = 0, tape_rec_cap = 0;
  int64_t tape_pool_want = 1 << 24;  // MPM_OPT_TAPE_SOLUTIONS
  int tape_substeps = 0;         // substeps recorded so far (host count)
  // mpm_backward scratch, grown on demand
  float* bw_buf = nullptr;  // bar[2], final state, substep states: 24 floats per particle each
  size_t bw_buf_cap = 0;
  float4* bw_gbar = nullptr;
  int* bw_slot = nullptr;
  double* bw_mat = nullptr;
  size_t bw_mat_cap = 0;
  double* bw_snap = nullptr;   // per recorded step: the body accumulators after it
  size_t bw_snap_cap = 0;
  double* bw_gbody = nullptr;  // per body: the impulse and moment cotangents of a step
  std::string err;
};

namespace mpmcr {
// helpers of api.cu that the batch shares
DevBody body_to_dev(const mpm_rigid_body& b);
cudaError_t ctx_upload_dynamics(mpm_ctx* ctx);
// the context's status word read (and cleared when set) after a stream
// synchronisation, as the first error it holds
mpm_status ctx_drain_status(mpm_ctx* ctx, uint32_t* bits);
}  // namespace mpmcr
