// batch.cu -- many independent scenes advanced together (the mpm_batch_*
// entry points of include/mpmcr.h).
//
// Launch overhead is what small scenes pay for (Sec. V-A); here it is paid
// once for all scenes. A substep of the batch is five launches whatever the
// number of scenes: P2G, compaction, grid update, contact solve and G2P, each
// over a work list of (scene, block) items that the host builds from the
// scenes' particle counts and the launch options, with one argument record
// per scene in device memory (a block copies its scene's record into shared
// memory first). The contact solve gives each scene one block, or one
// cluster of 2-8 blocks, largest scenes first. A time step
// adds one launch before the substeps (statistics cleared, the impulse
// accumulators noted) and one after them (the bodies' update of
// Eq. (3)-(4), status and statistics gathered), and replays as one CUDA
// graph. The work lists and the graph depend on the launch options, the
// scenes' particle counts and the substep count only; the argument records
// (h, solver parameters, the particle buffer each scene is in) are
// re-uploaded when they change, under the same graph.
#include <algorithm>
#include <cfloat>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

struct mpm_batch {
  cudaStream_t stream = nullptr;
  int device = 0;
  std::vector<mpm_ctx*> ctx;
  // launch options
  bool use_graphs = true;
  int p2g_chunk = 256;
  int g2p_threads = 256;
  int grid_particles = 2048;
  int solve_blocks = 1;  // blocks (one cluster) per scene's contact solve
  // per-scene argument records (device) and their host images
  P2GArgs* p2g_d = nullptr;
  GridBatchArgs* grid_d = nullptr;
  SolveArgs* solve_d = nullptr;
  G2PArgs* g2p_d = nullptr;
  RigidBatchArgs* rig_d = nullptr;
  std::vector<P2GArgs> p2g_h;
  std::vector<GridBatchArgs> grid_h;
  std::vector<SolveArgs> solve_h;
  std::vector<G2PArgs> g2p_h;
  std::vector<RigidBatchArgs> rig_h;
  // what the records were built from
  struct SceneSig {
    int64_t n = -1;
    int cur = -1, nb = -1;
  };
  std::vector<SceneSig> sig;
  float rec_h = 0.f;
  mpm_solver_params rec_sp{};
  bool records_valid = false;
  // work lists: P2G items, then grid items, then G2P items; the scenes'
  // order for the contact solve (largest first)
  int* order_d = nullptr;
  int2* work_d = nullptr;
  size_t work_cap = 0;
  int n_p2g = 0, n_grid = 0, n_g2p = 0;
  int layout = 0;             // bumped whenever the work lists change
  bool work_valid = false;
  // gathered at the end of each step
  uint32_t* status_d = nullptr;
  DevStats* stats_d = nullptr;
  // the step's graph and what it was captured for
  cudaGraphExec_t gexec = nullptr;
  int g_layout = -1, g_substeps = -1;
  double g_dt = 0.0;
  std::string err;
};

using namespace mpmcr;

namespace {

mpm_status bfail(mpm_batch* b, mpm_status st, const std::string& msg) {
  if (b) b->err = msg;
  return st;
}

#define BCU(call)                                                                      \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return bfail(batch, e_ == cudaErrorMemoryAllocation ? MPM_ERR_OOM : MPM_ERR_CUDA, \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                \
  } while (0)

template <class T>
cudaError_t balloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T) + 16);
}

void release(mpm_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  cudaFree(b->p2g_d);
  cudaFree(b->grid_d);
  cudaFree(b->solve_d);
  cudaFree(b->g2p_d);
  cudaFree(b->rig_d);
  cudaFree(b->work_d);
  cudaFree(b->order_d);
  cudaFree(b->status_d);
  cudaFree(b->stats_d);
}

int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Grid-phase blocks of a scene: one per grid_particles particles, at least
// one (the update also records the scene's active-block count), at most one
// thread per node of the whole domain.
int grid_slices(const mpm_batch* b, const mpm_ctx* c) {
  const int slices = ceil_div(c->n, b->grid_particles);
  const int cap = ceil_div((int64_t)c->n_blocks * kBlockNodes, 256);
  return slices < 1 ? 1 : slices > cap ? cap : slices;
}

// The scenes' argument records for substep size h and solver parameters sp,
// each scene on its current particle buffer.
void build_records(mpm_batch* b, float h, const mpm_solver_params& sp) {
  const int ns = (int)b->ctx.size();
  for (int s = 0; s < ns; ++s) {
    mpm_ctx* c = b->ctx[s];
    const int nb = (int)c->bodies.size();
    P2GArgs& pa = b->p2g_h[s];
    pa = P2GArgs{};
    pa.g = c->g; pa.P = c->P[c->cur]; pa.n = (int)c->n; pa.groups = c->groups_d;
    pa.bodies = c->bodies_d; pa.nb = nb; pa.h = h; pa.G = c->G; pa.C = c->C;
    pa.status = c->status; pa.stats = c->stats;
    GridBatchArgs& ga = b->grid_h[s];
    ga = GridBatchArgs{};
    ga.g = c->g; ga.G = c->G; ga.h = h; ga.stats = c->stats;
    ga.n_slices = grid_slices(b, c);
    SolveArgs& sa = b->solve_h[s];
    sa = SolveArgs{};
    sa.g = c->g; sa.G = c->G; sa.C = c->C; sa.bodies = c->bodies_d; sa.nb = nb;
    sa.h = h; sa.eps_s = sp.eps_s; sa.ls_rel_tol = sp.ls_rel_tol; sa.ls_max_iters = sp.ls_max_iters;
    sa.eps_r = sp.eps_r; sa.eps_a = sp.eps_a; sa.max_iters = sp.max_iters; sa.red = c->red;
    sa.bar = c->bar; sa.status = c->status; sa.stats = c->stats; sa.impulses = c->impulses;
    sa.wait_extra = 0;
    sa.poison = c->poison;
    sa.cluster_max = 0;  // one block per scene, no cluster
    G2PArgs& qa = b->g2p_h[s];
    qa = G2PArgs{};
    qa.g = c->g; qa.P = c->P[c->cur]; qa.n = (int)c->n; qa.groups = c->groups_d; qa.G = c->G;
    qa.C = c->C; qa.h = h; qa.bar = c->bar; qa.red = c->red; qa.stats = c->stats;
    RigidBatchArgs& ra = b->rig_h[s];
    ra = RigidBatchArgs{};
    ra.bodies = c->bodies_d; ra.dyn = c->dyn_d; ra.nb = nb; ra.rigid = nb > 0 ? 1 : 0;
    ra.imp = c->impulses; ra.imp0 = c->imp0_d; ra.stats = c->stats; ra.status = c->status;
    for (int k = 0; k < 3; ++k) ra.gravity[k] = c->spec.gravity[k];
    b->sig[s].n = c->n;
    b->sig[s].cur = c->cur;
    b->sig[s].nb = nb;
  }
}

// Work lists from the scenes' particle counts and the launch options (the
// records' n_slices, built with the same options, match them).
std::vector<int2> build_work(mpm_batch* b) {
  std::vector<int2> w;
  const int ns = (int)b->ctx.size();
  const int p2g_per = p2g_block_particles(b->p2g_chunk);
  for (int s = 0; s < ns; ++s) {
    const int blocks = ceil_div(b->ctx[s]->n, p2g_per);
    for (int k = 0; k < blocks; ++k) w.push_back(make_int2(s, k));
  }
  b->n_p2g = (int)w.size();
  for (int s = 0; s < ns; ++s) {
    const int slices = grid_slices(b, b->ctx[s]);
    for (int k = 0; k < slices; ++k) w.push_back(make_int2(s, k));
  }
  b->n_grid = (int)w.size() - b->n_p2g;
  for (int s = 0; s < ns; ++s) {
    // block 0 of G2P closes the substep's counters, so even an empty scene
    // has one
    int blocks = ceil_div(b->ctx[s]->n, b->g2p_threads);
    blocks = blocks < 1 ? 1 : blocks;
    for (int k = 0; k < blocks; ++k) w.push_back(make_int2(s, k));
  }
  b->n_g2p = (int)w.size() - b->n_p2g - b->n_grid;
  return w;
}

cudaError_t enqueue(mpm_batch* b, int n_substeps, double dt) {
  const cudaStream_t s = b->stream;
  const int ns = (int)b->ctx.size();
  launch_batch_begin(b->rig_d, ns, s);
  for (int k = 0; k < n_substeps; ++k) {
    launch_p2g_batch(b->p2g_d, b->work_d, b->n_p2g, b->p2g_chunk, s);
    launch_grid_batch(b->grid_d, b->work_d + b->n_p2g, b->n_grid, s);
    const cudaError_t e = launch_solve_batch(b->solve_d, b->order_d, ns, b->solve_blocks, s);
    if (e != cudaSuccess) return e;
    launch_g2p_batch(b->g2p_d, b->work_d + b->n_p2g + b->n_grid, b->n_g2p, b->g2p_threads, s);
  }
  launch_batch_end(b->rig_d, ns, dt, b->status_d, b->stats_d, s);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

mpm_status mpm_batch_create(mpm_ctx* const* ctxs, int32_t n, mpm_batch** out) {
  if (!ctxs || n < 1 || !out) return MPM_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    const mpm_ctx* c = ctxs[i];
    if (!c || c->taping || c->g.slot || !c->cloth_tris.empty() || c->n_pins > 0 ||
        c->device != ctxs[0]->device ||
        c->stream != ctxs[0]->stream)
      return MPM_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) return MPM_ERR_INVALID_ARG;
  }
  mpm_batch* batch = new mpm_batch();
  batch->stream = ctxs[0]->stream;
  batch->device = ctxs[0]->device;
  batch->ctx.assign(ctxs, ctxs + n);
  batch->p2g_h.resize(n);
  batch->grid_h.resize(n);
  batch->solve_h.resize(n);
  batch->g2p_h.resize(n);
  batch->rig_h.resize(n);
  batch->sig.resize(n);
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess && dev != batch->device) {
    delete batch;
    return MPM_ERR_INVALID_ARG;  // the members' device must be the current one
  }
  if (e == cudaSuccess) e = balloc(&batch->p2g_d, n);
  if (e == cudaSuccess) e = balloc(&batch->grid_d, n);
  if (e == cudaSuccess) e = balloc(&batch->solve_d, n);
  if (e == cudaSuccess) e = balloc(&batch->g2p_d, n);
  if (e == cudaSuccess) e = balloc(&batch->rig_d, n);
  if (e == cudaSuccess) e = balloc(&batch->status_d, n);
  if (e == cudaSuccess) e = balloc(&batch->stats_d, n);
  if (e == cudaSuccess) e = cudaMemsetAsync(batch->status_d, 0, n * sizeof(uint32_t), batch->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(batch->stats_d, 0, n * sizeof(DevStats), batch->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    release(batch);
    delete batch;
    return e == cudaErrorMemoryAllocation ? MPM_ERR_OOM : MPM_ERR_CUDA;
  }
  *out = batch;
  return mpm_batch_sort(batch);
}

mpm_status mpm_batch_sort(mpm_batch* batch) {
  if (!batch) return MPM_ERR_INVALID_ARG;
  for (mpm_ctx* c : batch->ctx) {
    if (c->n <= 0) continue;
    launch_sort(c->g, c->P[c->cur], c->P[1 - c->cur], (int)c->n, c->sb, batch->stream);
    c->cur = 1 - c->cur;
  }
  BCU(cudaGetLastError());
  return MPM_OK;
}

mpm_status mpm_batch_step(mpm_batch* batch, double h, int32_t n_substeps,
                          const mpm_solver_params* solver) {
  if (!batch) return MPM_ERR_INVALID_ARG;
  if (!(h > 0.0) || n_substeps < 0)
    return bfail(batch, MPM_ERR_INVALID_ARG, "mpm_batch_step: h must be > 0 and n_substeps >= 0");
  mpm_solver_params sp;
  if (solver) {
    sp = *solver;
  } else {
    sp.eps_r = 5e-2;
    sp.eps_a = DBL_EPSILON;
    sp.max_iters = 1000;
    sp.eps_s = 1e-4f;
    sp.ls_rel_tol = 1e-3f;
    sp.ls_max_iters = 50;
  }
  if (!(sp.eps_r >= 0.0) || !(sp.eps_a >= 0.0) || sp.max_iters < 0 || !(sp.eps_s > 0.f) ||
      !(sp.ls_rel_tol > 0.f) || sp.ls_max_iters < 1)
    return bfail(batch, MPM_ERR_INVALID_ARG, "mpm_batch_step: bad solver parameters");
  const int ns = (int)batch->ctx.size();
  const cudaStream_t s = batch->stream;
  // members' host-side changes since the last step: bodies set by the
  // caller, dynamics, particle buffers and counts
  bool records = !batch->records_valid || batch->rec_h != (float)h ||
                 memcmp(&batch->rec_sp, &sp, sizeof(sp)) != 0;
  bool work = !batch->work_valid;
  for (int i = 0; i < ns; ++i) {
    mpm_ctx* c = batch->ctx[i];
    if (c->taping)
      return bfail(batch, MPM_ERR_STATE, "mpm_batch_step: a member is recording a tape");
    if (!c->cloth_tris.empty() || c->n_pins > 0)
      return bfail(batch, MPM_ERR_STATE, "mpm_batch_step: a member has cloth or pinned particles");
    const int nb = (int)c->bodies.size();
    if (c->bodies_dirty) {
      DevBody tmp[kMaxBodies];
      for (int k = 0; k < nb; ++k) tmp[k] = body_to_dev(c->bodies[k]);
      if (nb) BCU(cudaMemcpyAsync(c->bodies_d, tmp, nb * sizeof(DevBody), cudaMemcpyHostToDevice, s));
      c->bodies_dirty = false;
    }
    if (c->dyn_dirty) BCU(ctx_upload_dynamics(c));
    const mpm_batch::SceneSig& g = batch->sig[i];
    if (g.n != c->n) work = true;
    if (g.n != c->n || g.cur != c->cur || g.nb != nb) records = true;
  }
  if (records || work) {
    build_records(batch, (float)h, sp);
    batch->rec_h = (float)h;
    batch->rec_sp = sp;
    batch->records_valid = true;
  }
  if (work) {
    const std::vector<int2> w = build_work(batch);
    if (w.size() > batch->work_cap) {
      cudaFree(batch->work_d);
      batch->work_d = nullptr;
      batch->work_cap = 0;
      BCU(balloc(&batch->work_d, w.size()));
      batch->work_cap = w.size();
    }
    // (pageable source: the copy has read it when the call returns)
    BCU(cudaMemcpyAsync(batch->work_d, w.data(), w.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    // the contact solves largest scene first (particle count as the proxy)
    std::vector<int> order(ns);
    for (int i = 0; i < ns; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
      return batch->ctx[x]->n > batch->ctx[y]->n;
    });
    if (!batch->order_d) BCU(balloc(&batch->order_d, ns));
    BCU(cudaMemcpyAsync(batch->order_d, order.data(), ns * sizeof(int), cudaMemcpyHostToDevice, s));
    batch->work_valid = true;
    batch->layout += 1;
  }
  if (records || work) {
    BCU(cudaMemcpyAsync(batch->p2g_d, batch->p2g_h.data(), ns * sizeof(P2GArgs),
                        cudaMemcpyHostToDevice, s));
    BCU(cudaMemcpyAsync(batch->grid_d, batch->grid_h.data(), ns * sizeof(GridBatchArgs),
                        cudaMemcpyHostToDevice, s));
    BCU(cudaMemcpyAsync(batch->solve_d, batch->solve_h.data(), ns * sizeof(SolveArgs),
                        cudaMemcpyHostToDevice, s));
    BCU(cudaMemcpyAsync(batch->g2p_d, batch->g2p_h.data(), ns * sizeof(G2PArgs),
                        cudaMemcpyHostToDevice, s));
    BCU(cudaMemcpyAsync(batch->rig_d, batch->rig_h.data(), ns * sizeof(RigidBatchArgs),
                        cudaMemcpyHostToDevice, s));
  }
  const double dt = h * n_substeps;
  bool launched = false;
  if (batch->use_graphs) {
    if (!batch->gexec || batch->g_layout != batch->layout || batch->g_substeps != n_substeps ||
        batch->g_dt != dt) {
      if (batch->gexec) {
        cudaGraphExecDestroy(batch->gexec);
        batch->gexec = nullptr;
      }
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const cudaError_t le = enqueue(batch, n_substeps, dt);
        e = cudaStreamEndCapture(s, &graph);
        if (e == cudaSuccess) e = le;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&batch->gexec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e == cudaSuccess) {
        batch->g_layout = batch->layout;
        batch->g_substeps = n_substeps;
        batch->g_dt = dt;
      } else {
        // launch directly from now on (the same kernels, without the graph)
        cudaGetLastError();
        if (batch->gexec) cudaGraphExecDestroy(batch->gexec);
        batch->gexec = nullptr;
        batch->use_graphs = false;
      }
    }
    if (batch->gexec) {
      BCU(cudaGraphLaunch(batch->gexec, s));
      launched = true;
    }
  }
  if (!launched) BCU(enqueue(batch, n_substeps, dt));
  BCU(cudaGetLastError());
  // the members' host bookkeeping, as after a device-side mpm_step
  for (mpm_ctx* c : batch->ctx) {
    if (!c->bodies.empty() && n_substeps > 0) c->bodies_stale = true;
    c->imp_seen_valid = false;
    c->adj_ready = false;
    c->last_dev_rigid = true;
    c->last_h = (float)h;
    c->last_eps_s = sp.eps_s;
    c->last_nb = (int)c->bodies.size();
    c->step_count += 1;
  }
  return MPM_OK;
}

mpm_status mpm_batch_synchronize(mpm_batch* batch, int32_t* status, mpm_step_stats* stats) {
  if (!batch) return MPM_ERR_INVALID_ARG;
  const int ns = (int)batch->ctx.size();
  BCU(cudaStreamSynchronize(batch->stream));
  std::vector<uint32_t> words(ns);
  BCU(cudaMemcpy(words.data(), batch->status_d, ns * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  std::vector<DevStats> ds;
  if (stats) {
    ds.resize(ns);
    BCU(cudaMemcpy(ds.data(), batch->stats_d, ns * sizeof(DevStats), cudaMemcpyDeviceToHost));
  }
  mpm_status first = MPM_OK;
  for (int i = 0; i < ns; ++i) {
    mpm_status st = MPM_OK;
    if (words[i]) {
      // the member's own word (it may hold failures of later member calls
      // too); reading it clears it
      uint32_t bits = 0;
      st = ctx_drain_status(batch->ctx[i], &bits);
      BCU(cudaMemsetAsync(batch->status_d + i, 0, sizeof(uint32_t), batch->stream));
    }
    if (status) status[i] = (int32_t)st;
    if (st != MPM_OK && first == MPM_OK) {
      first = st;
      batch->err = "member " + std::to_string(i) + ": " + mpm_last_error(batch->ctx[i]);
    }
    if (stats) {
      mpm_step_stats& o = stats[i];
      const DevStats& d = ds[i];
      memset(&o, 0, sizeof(o));
      o.substeps = d.substeps;
      o.iters_total = d.iters_total;
      o.iters_max = d.iters_max;
      o.ls_evals_total = d.ls_evals_total;
      o.contacts_max = d.contacts_max;
      o.active_blocks_max = d.active_blocks_max;
      o.contacts_total = (int64_t)d.contacts_total;
      o.residual_max = d.residual_max;
      o.status_bits = (int32_t)words[i];
      o.p2g_global_chunks = d.p2g_global_chunks;
      o.ls_split_substeps = d.ls_split;
      o.cluster_substeps = d.cluster;
      o.contact_nodes_max = d.cnodes_max;
      for (int k = 0; k < 5; ++k) o.solve_us[k] = (float)(d.solve_ns[k] * 1e-3);
    }
  }
  BCU(cudaStreamSynchronize(batch->stream));
  return first;
}

mpm_status mpm_batch_set_option(mpm_batch* batch, int32_t option, int64_t value) {
  if (!batch) return MPM_ERR_INVALID_ARG;
  switch (option) {
    case MPM_BATCH_OPT_GRAPHS:
      batch->use_graphs = value != 0;
      return MPM_OK;
    case MPM_BATCH_OPT_P2G_CHUNK:
      if (value != 256 && value != 512 && value != 1024)
        return bfail(batch, MPM_ERR_INVALID_ARG, "P2G chunk must be 256, 512 or 1024");
      if (batch->p2g_chunk != (int)value) batch->work_valid = false;
      batch->p2g_chunk = (int)value;
      return MPM_OK;
    case MPM_BATCH_OPT_G2P_THREADS:
      if (value < 64 || value > 512 || value % 32 != 0)
        return bfail(batch, MPM_ERR_INVALID_ARG, "G2P threads must be 64..512, a multiple of 32");
      if (batch->g2p_threads != (int)value) batch->work_valid = false;
      batch->g2p_threads = (int)value;
      return MPM_OK;
    case MPM_BATCH_OPT_SOLVE_BLOCKS:
      if (value != 1 && value != 2 && value != 4 && value != 8)
        return bfail(batch, MPM_ERR_INVALID_ARG, "solve blocks per scene must be 1, 2, 4 or 8");
      if (batch->solve_blocks != (int)value) batch->work_valid = false;  // a new graph
      batch->solve_blocks = (int)value;
      return MPM_OK;
    case MPM_BATCH_OPT_GRID_PARTICLES:
      if (value < 1 || value > (int64_t)1 << 30)
        return bfail(batch, MPM_ERR_INVALID_ARG, "grid particles per block must be >= 1");
      if (batch->grid_particles != (int)value) batch->work_valid = false;
      batch->grid_particles = (int)value;
      return MPM_OK;
    default:
      return bfail(batch, MPM_ERR_INVALID_ARG, "unknown batch option");
  }
}

const char* mpm_batch_last_error(const mpm_batch* batch) {
  return batch ? batch->err.c_str() : "invalid mpm batch";
}

void mpm_batch_destroy(mpm_batch* batch) {
  if (!batch) return;
  cudaStreamSynchronize(batch->stream);
  release(batch);
  delete batch;
}

}  // extern "C"
