// api.cu -- the C ABI of include/mpmcr.h: context and device memory, the
// substep schedule of one rigid time step (Eq. (3)-(4)), state I/O in particle
// id order, diagnostics and phase timing.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

using namespace mpmcr;

namespace {

const char* kGenericError = "invalid mpm context";
constexpr int kPlanes = kParticlePlanes;

mpm_status fail(mpm_ctx* c, mpm_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

#define CU(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? MPM_ERR_OOM : MPM_ERR_CUDA, \
                  std::string(#call) + ": " + cudaGetErrorString(e_));            \
  } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T) + 16);
}

Particles make_particles(float* buf, uint32_t* pid, uint16_t* grp, int64_t cap) {
  Particles P;
  P.base = buf;
  P.stride = cap;
  P.pid = pid;
  P.grp = grp;
  return P;
}

__global__ void k_append(Particles P, int64_t offset, int64_t n, const float* __restrict__ x,
                         const float* __restrict__ v, uint16_t grp) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int64_t i = offset + j;
  for (int c = 0; c < 3; ++c) {
    P.x(c)[i] = x[3 * j + c];
    P.v(c)[i] = v[3 * j + c];
  }
  for (int c = 0; c < 9; ++c) {
    P.C(c)[i] = 0.f;
    P.F(c)[i] = (c % 4 == 0) ? 1.f : 0.f;
  }
  for (int c = 0; c < 6; ++c) P.tau(c)[i] = 0.f;  // stress-free at F = I
  P.pid[i] = (uint32_t)i;
  P.grp[i] = grp;
}

__global__ void k_grid_out(GridDev g, GridArrays G, int n_act, int* __restrict__ count,
                           int* __restrict__ ids, float* __restrict__ m, float* __restrict__ vs,
                           float* __restrict__ v) {
  long long total = (long long)active_with_storage(g, n_act) * kBlockNodes;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int blk = G.act[t >> 6], cell = (int)(t & 63);
    int node = active_storage_block(g, G.act, (int)(t >> 6)) * kBlockNodes + cell;
    float4 a = G.vs[node];
    if (!(a.w > 0.f)) continue;
    float4 b = G.v[node];
    int bx = blk % g.nbx, by = (blk / g.nbx) % g.nby, bz = blk / (g.nbx * g.nby);
    int i = bx * 4 + (cell & 3), j = by * 4 + ((cell >> 2) & 3), k = bz * 4 + (cell >> 4);
    int slot = atomicAdd(count, 1);
    ids[slot] = i + g.rx * (j + g.ry * k);
    m[slot] = a.w;
    vs[3 * slot] = a.x; vs[3 * slot + 1] = a.y; vs[3 * slot + 2] = a.z;
    v[3 * slot] = b.x; v[3 * slot + 1] = b.y; v[3 * slot + 2] = b.z;
  }
}

DevBody to_dev(const mpm_rigid_body& b) {
  DevBody d;
  memset(&d, 0, sizeof(d));
  d.shape = b.shape;
  for (int i = 0; i < 4; ++i) d.prm[i] = b.params[i];
  for (int i = 0; i < 9; ++i) d.R[i] = b.R[i];
  for (int i = 0; i < 3; ++i) {
    d.p[i] = b.p[i];
    d.w[i] = b.omega[i];
    d.v[i] = b.v[i];
  }
  d.mu = b.mu;
  d.k = b.k;
  d.d = b.d;
  // a ball around p that holds the geometry (the half-space has none)
  if (b.shape == MPM_SPHERE)
    d.bound = std::fabs(b.params[0]);
  else if (b.shape == MPM_BOX)
    d.bound = (float)std::sqrt((double)b.params[0] * b.params[0] + (double)b.params[1] * b.params[1] +
                               (double)b.params[2] * b.params[2]) * 1.000001f;
  else if (b.shape == MPM_CAPSULE)
    d.bound = (std::fabs(b.params[0]) + std::fabs(b.params[1])) * 1.000001f;
  else
    d.bound = INFINITY;
  return d;
}

// small 3-vector helpers for the rigid adjoint
void cross3d(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// exp(sgn [ph]x) x (Rodrigues)
void rot_apply(const double* ph, const double* x, double sgn, double* out) {
  const double th = std::sqrt(ph[0] * ph[0] + ph[1] * ph[1] + ph[2] * ph[2]);
  const double a = th > 1e-12 ? std::sin(th) / th : 1.0;
  const double b = th > 1e-6 ? (1.0 - std::cos(th)) / (th * th) : 0.5;
  double px[3], ppx[3];
  cross3d(ph, x, px);
  cross3d(ph, px, ppx);
  for (int c = 0; c < 3; ++c) out[c] = x[c] + sgn * a * px[c] + b * ppx[c];
}

// J_l(ph)^T x, J_l the left Jacobian of SO(3)
void jl_transpose(const double* ph, const double* x, double* out) {
  const double th = std::sqrt(ph[0] * ph[0] + ph[1] * ph[1] + ph[2] * ph[2]);
  const double b = th > 1e-6 ? (1.0 - std::cos(th)) / (th * th) : 0.5;
  const double c3 = th > 1e-4 ? (th - std::sin(th)) / (th * th * th) : 1.0 / 6.0;
  double px[3], ppx[3];
  cross3d(ph, x, px);
  cross3d(ph, px, ppx);
  for (int c = 0; c < 3; ++c) out[c] = x[c] - b * px[c] + c3 * ppx[c];
}

// R <- exp(dt [omega]x) R, p <- p + dt v (kinematic bodies between time steps)
void advance_kinematic(mpm_rigid_body& b, double dt) {
  for (int i = 0; i < 3; ++i) b.p[i] = (float)((double)b.p[i] + dt * b.v[i]);
  double w[3] = {dt * b.omega[0], dt * b.omega[1], dt * b.omega[2]};
  double th = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  if (th == 0.0) return;
  double a[3] = {w[0] / th, w[1] / th, w[2] / th};
  double c = std::cos(th), s = std::sin(th), t = 1.0 - c;
  double Q[9] = {c + t * a[0] * a[0],        t * a[0] * a[1] - s * a[2], t * a[0] * a[2] + s * a[1],
                 t * a[1] * a[0] + s * a[2], c + t * a[1] * a[1],        t * a[1] * a[2] - s * a[0],
                 t * a[2] * a[0] - s * a[1], t * a[2] * a[1] + s * a[0], c + t * a[2] * a[2]};
  double R[9];
  for (int r = 0; r < 3; ++r)
    for (int cc = 0; cc < 3; ++cc)
      R[3 * r + cc] = Q[3 * r] * b.R[cc] + Q[3 * r + 1] * b.R[3 + cc] + Q[3 * r + 2] * b.R[6 + cc];
  for (int i = 0; i < 9; ++i) b.R[i] = (float)R[i];
}

// Adjoint of integrate_dynamic. The state is (v, omega, p, theta) with theta
// a left rotation of R (R -> exp([theta]x) R); sb[12] holds the adjoint of the
// state after the step on entry and of the state before it on exit; jl[6]
// receives the adjoints of the step's impulse J and moment L. With
// v' = v + (dt f + J) / m, q = dt (tau - w x I_w w) + L, a = I_w^-1 q,
// w' = w + a (masked), p' = p + dt v', R' = exp(dt [w']x) R:
//   pbar = p'bar, thetabar = exp(-dt [w']x) theta'bar + (terms of I_w below),
//   v'acc = v'bar + dt p'bar, w'acc = w'bar + dt J_l(dt w')^T theta'bar (masked),
//   vbar = v'acc, Jbar = v'acc / m, z = I_w^-1 w'acc, Lbar = z,
//   wbar = w'acc + dt (I_w (w x z) - (I_w w) x z),
//   thetabar -= (I_w a) x z + (I_w z) x a + dt ((I_w w) x (z x w) + (I_w (z x w)) x w).
void integrate_dynamic_adjoint(const DevBody& b, const mpm_rigid_dynamics& d, const double* gravity,
                               const double* J, const double* L, double dt, double* sb, double* jl) {
  const double m = d.mass;
  double w[3], R[9], Iw[9];
  (void)gravity;  // the force and gravity enter v' additively: no adjoint term
  for (int i = 0; i < 3; ++i) w[i] = b.w[i];
  for (int i = 0; i < 9; ++i) R[i] = b.R[i];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += R[3 * r + k] * (double)d.inertia[k] * R[3 * c + k];
      Iw[3 * r + c] = acc;
    }
  auto mul = [&](const double* x, double* o) {
    for (int r = 0; r < 3; ++r) o[r] = Iw[3 * r] * x[0] + Iw[3 * r + 1] * x[1] + Iw[3 * r + 2] * x[2];
  };
  const double A0 = Iw[4] * Iw[8] - Iw[5] * Iw[5], A1 = Iw[2] * Iw[5] - Iw[1] * Iw[8],
               A2 = Iw[1] * Iw[5] - Iw[2] * Iw[4];
  const double det = Iw[0] * A0 + Iw[1] * A1 + Iw[2] * A2;
  const double inv[9] = {A0, A1, A2, A1, Iw[0] * Iw[8] - Iw[2] * Iw[2], Iw[1] * Iw[2] - Iw[0] * Iw[5],
                         A2, Iw[1] * Iw[2] - Iw[0] * Iw[5], Iw[0] * Iw[4] - Iw[1] * Iw[1]};
  auto solve = [&](const double* x, double* o) {
    for (int r = 0; r < 3; ++r) o[r] = (inv[3 * r] * x[0] + inv[3 * r + 1] * x[1] + inv[3 * r + 2] * x[2]) / det;
  };
  double Iww[3], gyro[3], q[3], a[3], w2[3];
  mul(w, Iww);
  cross3d(w, Iww, gyro);
  for (int i = 0; i < 3; ++i) q[i] = dt * (d.torque[i] - gyro[i]) + L[i];
  solve(q, a);
  for (int i = 0; i < 3; ++i) w2[i] = ((d.dof_mask >> (3 + i)) & 1) ? w[i] + a[i] : 0.0;
  const double* vb2 = sb;
  const double* pb2 = sb + 3;
  const double* wb2 = sb + 6;
  const double* tb2 = sb + 9;
  double ph[3] = {dt * w2[0], dt * w2[1], dt * w2[2]};
  double tb[3], jt[3], vacc[3], wacc[3];
  rot_apply(ph, tb2, -1.0, tb);
  jl_transpose(ph, tb2, jt);
  for (int i = 0; i < 3; ++i) {
    vacc[i] = ((d.dof_mask >> i) & 1) ? vb2[i] + dt * pb2[i] : 0.0;
    wacc[i] = ((d.dof_mask >> (3 + i)) & 1) ? wb2[i] + dt * jt[i] : 0.0;
  }
  double z[3], wz[3], Iwz_[3], Iw_wz[3], zw[3], Izw[3], t1[3], t2[3], t3[3], t4[3], Ia[3], Iz[3];
  solve(wacc, z);
  cross3d(w, z, wz);
  mul(wz, Iwz_);
  cross3d(Iww, z, Iw_wz);
  cross3d(z, w, zw);
  mul(zw, Izw);
  mul(a, Ia);
  mul(z, Iz);
  cross3d(Ia, z, t1);
  cross3d(Iz, a, t2);
  cross3d(Iww, zw, t3);
  cross3d(Izw, w, t4);
  const double pb[3] = {pb2[0], pb2[1], pb2[2]};
  for (int i = 0; i < 3; ++i) {
    jl[i] = vacc[i] / m;
    jl[3 + i] = z[i];
    sb[i] = vacc[i];                                  // vbar
    sb[3 + i] = pb[i];                                // pbar
    sb[6 + i] = wacc[i] + dt * (Iwz_[i] - Iw_wz[i]);  // wbar
    sb[9 + i] = tb[i] - (t1[i] + t2[i]) - dt * (t3[i] + t4[i]);  // thetabar
  }
}

// Eq. (3) for one dynamic body over a time step dt with the step's impulse
// J (on the body, world frame) and its moment L about the body origin:
// semi-implicit Euler, then the locked degrees of freedom are zeroed.
void integrate_dynamic(mpm_rigid_body& b, const mpm_rigid_dynamics& d, const double* gravity,
                       const double* J, const double* L, double dt) {
  const double m = d.mass;
  double v[3], w[3];
  for (int i = 0; i < 3; ++i) {
    const double f = d.force[i] + (d.gravity ? m * gravity[i] : 0.0);
    v[i] = b.v[i] + (dt * f + J[i]) / m;
  }
  // world inertia I = R diag(Ib) R^T and the gyroscopic term w x I w
  double R[9], Iw[9];
  for (int i = 0; i < 9; ++i) R[i] = b.R[i];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += R[3 * r + k] * (double)d.inertia[k] * R[3 * c + k];
      Iw[3 * r + c] = acc;
    }
  const double w0[3] = {b.omega[0], b.omega[1], b.omega[2]};
  double Iw0[3];
  for (int r = 0; r < 3; ++r) Iw0[r] = Iw[3 * r] * w0[0] + Iw[3 * r + 1] * w0[1] + Iw[3 * r + 2] * w0[2];
  const double gyro[3] = {w0[1] * Iw0[2] - w0[2] * Iw0[1], w0[2] * Iw0[0] - w0[0] * Iw0[2],
                          w0[0] * Iw0[1] - w0[1] * Iw0[0]};
  double rhs[3];
  for (int i = 0; i < 3; ++i) rhs[i] = dt * (d.torque[i] - gyro[i]) + L[i];
  // dw = Iw^-1 rhs (symmetric positive definite 3x3: by cofactors)
  const double a = Iw[0], bb = Iw[1], c = Iw[2], e = Iw[4], f = Iw[5], i9 = Iw[8];
  const double A0 = e * i9 - f * f, A1 = c * f - bb * i9, A2 = bb * f - c * e;
  const double det = a * A0 + bb * A1 + c * A2;
  const double inv[9] = {A0, A1, A2, A1, a * i9 - c * c, bb * c - a * f, A2, bb * c - a * f, a * e - bb * bb};
  for (int r = 0; r < 3; ++r)
    w[r] = w0[r] + (inv[3 * r] * rhs[0] + inv[3 * r + 1] * rhs[1] + inv[3 * r + 2] * rhs[2]) / det;
  for (int i = 0; i < 3; ++i) {
    if (!((d.dof_mask >> i) & 1)) v[i] = 0.0;
    if (!((d.dof_mask >> (3 + i)) & 1)) w[i] = 0.0;
    b.v[i] = (float)v[i];
    b.omega[i] = (float)w[i];
  }
  advance_kinematic(b, dt);
}

mpm_status first_error(mpm_ctx* ctx, uint32_t bits) {
  static const mpm_status order[] = {MPM_ERR_TIMEOUT, MPM_ERR_NAN, MPM_ERR_OUT_OF_DOMAIN,
                                     MPM_ERR_CAPACITY, MPM_ERR_LINE_SEARCH,
                                     MPM_ERR_NOT_CONVERGED, MPM_ERR_INVALID_ARG};
  static const char* msg[] = {"a device-wide barrier of the contact solve timed out",
                              "a non-finite value appeared in the contact solve",
                              "a particle's B-spline stencil left the grid domain",
                              "more contact points than max_contacts in one substep",
                              "the line-search bracket could not be formed",
                              "a contact solve (or its adjoint) reached max_iters before converging",
                              "a node id given to the adjoint lies outside the grid"};
  for (int i = 0; i < 7; ++i)
    if (bits & (1u << order[i])) return fail(ctx, order[i], msg[i]);
  return MPM_OK;
}

// read and clear the device status word (synchronises)
mpm_status drain_status(mpm_ctx* ctx, uint32_t* bits_out = nullptr) {
  CU(cudaStreamSynchronize(ctx->stream));
  uint32_t bits = 0;
  CU(cudaMemcpy(&bits, ctx->status, sizeof(bits), cudaMemcpyDeviceToHost));
  // (on the context's stream: it is non-blocking, so a legacy-stream memset
  // would not be ordered before the next launch)
  if (bits) {
    CU(cudaMemsetAsync(ctx->status, 0, sizeof(uint32_t), ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
  }
  if (bits_out) *bits_out = bits;
  return first_error(ctx, bits);
}

cudaEvent_t take_event(mpm_ctx* ctx) {
  cudaEvent_t e = nullptr;
  if (!ctx->ev_pool.empty()) {
    e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
  } else {
    cudaEventCreate(&e);
  }
  return e;
}

void mark_phase(mpm_ctx* ctx, int phase) {
  if (!ctx->profile) return;
  cudaEvent_t e = take_event(ctx);
  cudaEventRecord(e, ctx->stream);
  ctx->ev_marks.emplace_back(phase, e);
}

// fold recorded events into per-phase totals (after a synchronise); a mark
// with phase -1 only closes the previous interval
void fold_events(mpm_ctx* ctx) {
  for (size_t i = 0; i + 1 < ctx->ev_marks.size(); ++i) {
    int ph = ctx->ev_marks[i].first;
    if (ph < 0) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev_marks[i].second, ctx->ev_marks[i + 1].second) ==
        cudaSuccess) {
      ctx->phase_ms[ph] += ms;
      ctx->phase_n[ph] += 1;
    }
  }
  if (!ctx->ev_marks.empty()) {
    // keep the last mark's event as the open end only if it starts a phase
    for (size_t i = 0; i < ctx->ev_marks.size(); ++i) ctx->ev_pool.push_back(ctx->ev_marks[i].second);
    ctx->ev_marks.clear();
  }
}

void release(mpm_ctx* c) {
  void* ptrs[] = {c->pbuf[0], c->pbuf[1], c->pidbuf[0], c->pidbuf[1], c->grpbuf[0], c->grpbuf[1],
                  c->groups_d, c->bodies_d, c->G.mp, c->G.vs, c->G.v, c->G.v2, c->G.vlo, c->G.vlo2, c->G.acc0, c->G.acc1,
                  c->G.acc2, c->G.dv, c->G.mark, c->G.cflag, c->G.cnodes, c->G.n_cnodes, c->G.pstar2, c->G.act, c->G.n_act, c->C.xp, c->C.nrm,
                  c->C.bias, c->C.id, c->C.vc, c->C.dvc, c->C.gamma, c->C.count, c->red, c->bar, c->poison,
                  c->status, c->stats, c->impulses, c->sb.keys[0], c->sb.keys[1], c->sb.vals[0],
                  c->sb.vals[1], c->sb.hist, c->sb.partial, c->stage, c->adj_vec, c->adj_body,
                  c->adj_out, c->adj_ids, c->adj_io, c->bw_buf, c->bw_gbar, c->bw_slot, c->bw_mat,
                  c->tape_pool, c->tape_recs, c->tape_counters, c->bw_snap, c->bw_gbody, c->dyn_d,
                  c->imp0_d, c->bodies_step_d, c->G.n_mapped, c->slot_d, c->cloth_tris_d,
                  c->cloth_rest_d, c->cloth_f_d, c->slot_of_d, c->pin_ids_d, c->pin_v_d, c->pin_x_d,
                  c->pin_mask_d};
  for (auto& t : c->tape)
    if (t.state) cudaFree(t.state);
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& e : c->gexec)
    if (e) cudaGraphExecDestroy(e);
  for (auto& e : c->ev_marks) cudaEventDestroy(e.second);
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

// Contact counts up to which one thread-block cluster solves (the barrier
// time-limit test needs the cooperative kernel's device-wide barriers).
int cluster_contacts(const mpm_ctx* ctx) {
  return ctx->wait_test || ctx->cluster_blocks == 0 ? 0 : ctx->cluster_max;
}

// One substep on particle buffer `cur`: P2G, grid update, contact solve and
// (with_g2p) G2P. save: append the solve's contact-node velocities to the
// tape's solution pool; warm_rec >= 0: start the solve from the taped
// solution record warm_rec instead of v*.
cudaError_t enqueue_substep(mpm_ctx* ctx, int cur, int nb, float hf, const mpm_solver_params& sp,
                            int solve_blocks, bool with_g2p, cudaStream_t s, bool save = false,
                            int warm_rec = -1) {
  const int n = (int)ctx->n;
  P2GArgs pa;
  pa.g = ctx->g; pa.P = ctx->P[cur]; pa.n = n; pa.groups = ctx->groups_d;
  pa.bodies = ctx->bodies_d; pa.nb = nb; pa.h = hf; pa.G = ctx->G; pa.C = ctx->C;
  pa.status = ctx->status; pa.stats = ctx->stats;
  pa.fext = nullptr;
  pa.fext_stride = ctx->cap;
  if (!ctx->cloth_tris.empty()) {
    // cloth: the mesh forces at the substep's start positions
    mark_phase(ctx, MPM_PHASE_P2G);
    launch_cloth_forces(ctx->P[cur], ctx->slot_of_d, ctx->cloth_tris_d, ctx->cloth_rest_d,
                        (int)ctx->cloth_tris.size(), ctx->groups_d,
                        ctx->n_pins > 0 ? ctx->pin_mask_d : nullptr, ctx->cloth_f_d, ctx->cap, s);
    pa.fext = ctx->cloth_f_d;
  }
  if (ctx->g.slot) {
    // a block-sparse grid gives the substep's blocks storage before P2G
    mark_phase(ctx, MPM_PHASE_GRID);
    launch_sparse_map(ctx->g, ctx->G, ctx->P[cur], n, ctx->slot_d, ctx->status, ctx->num_sms, s);
  }
  mark_phase(ctx, MPM_PHASE_P2G);
  launch_p2g(pa, ctx->p2g_chunk, ctx->p2g_form, s);
  mark_phase(ctx, MPM_PHASE_GRID);
  launch_grid(ctx->g, ctx->G, hf, ctx->num_sms, ctx->stats, s);
  if (warm_rec >= 0 && ctx->tape_pool)
    launch_tape_warm(ctx->g, ctx->G, ctx->tape_recs, warm_rec, ctx->tape_pool, ctx->num_sms, s);
  SolveArgs sa;
  sa.g = ctx->g; sa.G = ctx->G; sa.C = ctx->C; sa.bodies = ctx->bodies_d; sa.nb = nb;
  sa.h = hf; sa.eps_s = sp.eps_s; sa.ls_rel_tol = sp.ls_rel_tol; sa.ls_max_iters = sp.ls_max_iters;
  sa.eps_r = sp.eps_r; sa.eps_a = sp.eps_a; sa.max_iters = sp.max_iters; sa.red = ctx->red;
  sa.bar = ctx->bar; sa.status = ctx->status; sa.stats = ctx->stats; sa.impulses = ctx->impulses;
  sa.wait_extra = ctx->wait_test ? 1 : 0;
  sa.poison = ctx->poison;
  sa.cluster_max = cluster_contacts(ctx);
  mark_phase(ctx, MPM_PHASE_SOLVE);
  const cudaError_t e = launch_solve(sa, solve_blocks, ctx->cluster_blocks, s);
  if (e != cudaSuccess) return e;
  if (save && ctx->tape_pool)
    launch_tape_save(ctx->g, ctx->G, ctx->tape_counters, ctx->tape_recs, ctx->tape_rec_cap, ctx->tape_pool,
                     ctx->tape_pool_cap, ctx->num_sms, s);
  if (with_g2p) {
    G2PArgs ga;
    ga.g = ctx->g; ga.P = ctx->P[cur]; ga.n = n; ga.groups = ctx->groups_d; ga.G = ctx->G;
    ga.C = ctx->C; ga.h = hf; ga.bar = ctx->bar; ga.red = ctx->red; ga.stats = ctx->stats;
    mark_phase(ctx, MPM_PHASE_G2P);
    launch_g2p(ga, s);
    launch_pins(ctx->P[cur], ctx->slot_of_d, ctx->pin_ids_d, ctx->pin_v_d, ctx->pin_x_d, ctx->n_pins,
                ctx->pins_cap, hf, s);
  }
  mark_phase(ctx, -1);
  return cudaGetLastError();
}

// The launches of one step: the radix sort from particle buffer `from` into
// the other (if sort_now), then n_substeps substeps on the sorted buffer.
// With `rigid`, the bodies then move on the device (kinematic ones by their
// velocity, dynamic ones by Eq. (3) with the step's impulses, rigid.cu).
cudaError_t enqueue_step(mpm_ctx* ctx, int from, bool sort_now, int n_substeps, float hf,
                         const mpm_solver_params& sp, int solve_blocks, cudaStream_t s,
                         bool rigid = false) {
  const int n = (int)ctx->n;
  const int nb = (int)ctx->bodies.size();
  int cur = from;
  if (rigid && nb > 0) {
    const cudaError_t e = cudaMemcpyAsync(ctx->imp0_d, ctx->impulses, 6 * nb * sizeof(double),
                                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  if (sort_now) {
    mark_phase(ctx, MPM_PHASE_SORT);
    launch_sort(ctx->g, ctx->P[cur], ctx->P[1 - cur], n, ctx->sb, s);
    cur = 1 - cur;
  }
  // cloth triangles and pins find their particles through the id -> slot
  // map of the buffer the substeps run on
  if (!ctx->cloth_tris.empty() || ctx->n_pins > 0) launch_slot_map(ctx->P[cur], n, ctx->slot_of_d, s);
  // pinned particles enter the step on their prescribed motion (start
  // positions from the particles, which the caller may have set)
  if (ctx->n_pins > 0 && n_substeps > 0)
    launch_pin_init(ctx->P[cur], ctx->slot_of_d, ctx->pin_ids_d, ctx->pin_v_d, ctx->pin_x_d,
                    ctx->n_pins, ctx->pins_cap, s);
  for (int k = 0; k < n_substeps; ++k) {
    const cudaError_t e = enqueue_substep(ctx, cur, nb, hf, sp, solve_blocks, true, s, ctx->taping);
    if (e != cudaSuccess) return e;
  }
  if (rigid && nb > 0) {
    // the frozen bodies stay readable for the last substep's contact adjoint
    const cudaError_t e = cudaMemcpyAsync(ctx->bodies_step_d, ctx->bodies_d, nb * sizeof(DevBody),
                                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    launch_rigid_update(ctx->bodies_d, ctx->dyn_d, nb, ctx->impulses, ctx->imp0_d,
                        (double)hf * n_substeps, ctx->spec.gravity, s);
  }
  return cudaGetLastError();
}

// The host copy of the bodies, after the device moved them (synchronises).
cudaError_t sync_host_bodies(mpm_ctx* ctx) {
  if (!ctx->bodies_stale) return cudaSuccess;
  const int nb = (int)ctx->bodies.size();
  DevBody tmp[kMaxBodies];
  cudaError_t e = cudaSuccess;
  if (nb) e = cudaMemcpyAsync(tmp, ctx->bodies_d, nb * sizeof(DevBody), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < nb; ++i) {
    mpm_rigid_body& b = ctx->bodies[i];
    for (int k = 0; k < 9; ++k) b.R[k] = tmp[i].R[k];
    for (int k = 0; k < 3; ++k) {
      b.p[k] = tmp[i].p[k];
      b.v[k] = tmp[i].v[k];
      b.omega[k] = tmp[i].w[k];
    }
  }
  ctx->bodies_stale = false;
  return cudaSuccess;
}

// Each body's kind and dynamics for the device update.
cudaError_t upload_dynamics(mpm_ctx* ctx) {
  const int nb = (int)ctx->bodies.size();
  DevDyn tmp[kMaxBodies];
  memset(tmp, 0, sizeof(tmp));
  for (int i = 0; i < nb; ++i) {
    DevDyn& d = tmp[i];
    if (ctx->is_dyn[i]) {
      const mpm_rigid_dynamics& m = ctx->dyn[i];
      d.kind = kRigidDynamic;
      d.dof_mask = m.dof_mask;
      d.gravity = m.gravity;
      d.mass = m.mass;
      for (int k = 0; k < 3; ++k) {
        d.inertia[k] = m.inertia[k];
        d.force[k] = m.force[k];
        d.torque[k] = m.torque[k];
      }
    } else {
      d.kind = ctx->bodies[i].kinematic ? kRigidKinematic : kRigidStatic;
    }
  }
  cudaError_t e = cudaSuccess;
  if (nb) e = cudaMemcpyAsync(ctx->dyn_d, tmp, nb * sizeof(DevDyn), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) ctx->dyn_dirty = false;
  return e;
}

int ceil_log2(int v) {
  int b = 0;
  while ((1 << b) < v) ++b;
  return b;
}

}  // namespace

namespace mpmcr {
DevBody body_to_dev(const mpm_rigid_body& b) { return to_dev(b); }
cudaError_t ctx_upload_dynamics(mpm_ctx* ctx) { return upload_dynamics(ctx); }
mpm_status ctx_drain_status(mpm_ctx* ctx, uint32_t* bits) { return drain_status(ctx, bits); }
}  // namespace mpmcr

extern "C" {

mpm_status mpm_create(const mpm_grid_spec* spec, void* cuda_stream, mpm_ctx** out) {
  mpm_ctx* ctx = nullptr;
  if (!spec || !out) return MPM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!(spec->dx > 0.0) || spec->max_particles <= 0 || spec->max_particles >= (1LL << 31) ||
      spec->max_contacts <= 0 || spec->max_contacts >= (1LL << 31) || spec->bc_layers < 0)
    return MPM_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (spec->res[a] <= 0 || spec->res[a] % 4 != 0 || spec->res[a] > 4096) return MPM_ERR_INVALID_ARG;
  // node ids i + rx (j + ry k) are 32-bit
  if ((int64_t)spec->res[0] * spec->res[1] * spec->res[2] >= (1LL << 31) || spec->max_blocks < 0)
    return MPM_ERR_INVALID_ARG;
  ctx = new mpm_ctx();
  ctx->spec = *spec;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e != cudaSuccess) {
    delete ctx;
    return MPM_ERR_CUDA;
  }
  auto bail = [&](mpm_status st) {
    release(ctx);
    delete ctx;
    return st;
  };
  if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess)
    return bail(MPM_ERR_CUDA);
  if (cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(MPM_ERR_CUDA);
    ctx->own_stream = true;
  }
  GridDev& g = ctx->g;
  g.dx = (float)spec->dx;
  g.inv_dx = (float)(1.0 / spec->dx);
  g.inv_dx_lo = (float)(1.0 / spec->dx - (double)g.inv_dx);
  g.ox = (float)spec->origin[0]; g.oy = (float)spec->origin[1]; g.oz = (float)spec->origin[2];
  g.ox_lo = (float)(spec->origin[0] - (double)g.ox);
  g.oy_lo = (float)(spec->origin[1] - (double)g.oy);
  g.oz_lo = (float)(spec->origin[2] - (double)g.oz);
  g.gx = (float)spec->gravity[0]; g.gy = (float)spec->gravity[1]; g.gz = (float)spec->gravity[2];
  g.rx = spec->res[0]; g.ry = spec->res[1]; g.rz = spec->res[2];
  g.nbx = g.rx / 4; g.nby = g.ry / 4; g.nbz = g.rz / 4;
  g.bc = spec->bc_layers;
  int mb = g.nbx > g.nby ? g.nbx : g.nby;
  mb = mb > g.nbz ? mb : g.nbz;
  g.morton_bits = ceil_log2(mb) > 0 ? ceil_log2(mb) : 1;
  g.sort_cell_bits = 3 * g.morton_bits + 6 <= 32 ? 1 : 0;
  ctx->cap = spec->max_particles;
  ctx->n_blocks = g.nbx * g.nby * g.nbz;
  // block-sparse storage for max_blocks active blocks (plus a spare one) when
  // that is fewer than the domain's blocks; dense otherwise
  const bool sparse = spec->max_blocks > 0 && spec->max_blocks < ctx->n_blocks;
  g.slot = nullptr;
  g.pool_blocks = sparse ? (int)spec->max_blocks : 0;
  ctx->n_nodes = (size_t)(sparse ? g.pool_blocks + 1 : ctx->n_blocks) * kBlockNodes;
  const int64_t cap = ctx->cap;
  const int64_t ccap = spec->max_contacts;
  bool ok = true;
  for (int s = 0; s < 2; ++s) {
    ok = ok && dalloc(&ctx->pbuf[s], (size_t)kPlanes * cap) == cudaSuccess;
    ok = ok && dalloc(&ctx->pidbuf[s], cap) == cudaSuccess;
    ok = ok && dalloc(&ctx->grpbuf[s], cap) == cudaSuccess;
    if (ok) ctx->P[s] = make_particles(ctx->pbuf[s], ctx->pidbuf[s], ctx->grpbuf[s], cap);
  }
  const size_t nn = ctx->n_nodes;
  ok = ok && dalloc(&ctx->G.mp, nn) == cudaSuccess && dalloc(&ctx->G.vs, nn) == cudaSuccess &&
       dalloc(&ctx->G.v, nn) == cudaSuccess && dalloc(&ctx->G.v2, nn) == cudaSuccess &&
       dalloc(&ctx->G.vlo, nn) == cudaSuccess && dalloc(&ctx->G.vlo2, nn) == cudaSuccess &&
       dalloc(&ctx->G.acc0, nn) == cudaSuccess &&
       dalloc(&ctx->G.acc1, nn) == cudaSuccess && dalloc(&ctx->G.acc2, nn) == cudaSuccess &&
       dalloc(&ctx->G.dv, nn) == cudaSuccess && dalloc(&ctx->G.mark, ctx->n_blocks) == cudaSuccess &&
       dalloc(&ctx->G.cflag, nn) == cudaSuccess && dalloc(&ctx->G.n_cnodes, 1) == cudaSuccess &&
       dalloc(&ctx->G.pstar2, 1) == cudaSuccess &&
       dalloc(&ctx->G.act, ctx->n_blocks) == cudaSuccess && dalloc(&ctx->G.n_act, 1) == cudaSuccess &&
       dalloc(&ctx->G.n_mapped, 1) == cudaSuccess;
  if (ok && sparse) {
    ok = dalloc(&ctx->slot_d, ctx->n_blocks) == cudaSuccess &&
         cudaMemset(ctx->slot_d, 0xff, (size_t)ctx->n_blocks * sizeof(int)) == cudaSuccess;  // -1
    g.slot = ctx->slot_d;
  }
  ok = ok && dalloc(&ctx->C.xp, ccap) == cudaSuccess && dalloc(&ctx->C.nrm, ccap) == cudaSuccess &&
       dalloc(&ctx->C.bias, ccap) == cudaSuccess && dalloc(&ctx->C.id, ccap) == cudaSuccess &&
       dalloc(&ctx->C.vc, ccap) == cudaSuccess && dalloc(&ctx->C.dvc, ccap) == cudaSuccess &&
       dalloc(&ctx->C.gamma, ccap) == cudaSuccess && dalloc(&ctx->C.count, 1) == cudaSuccess;
  ctx->C.cap = (int)ccap;
  {
    const size_t cn = (size_t)27 * (size_t)ccap < nn ? (size_t)27 * (size_t)ccap : nn;
    ctx->G.cnodes_cap = (int)cn;
    ok = ok && dalloc(&ctx->G.cnodes, cn) == cudaSuccess;
  }
  ok = ok && dalloc(&ctx->red, kRedDoubles) == cudaSuccess && dalloc(&ctx->bar, kBarWords) == cudaSuccess &&
       dalloc(&ctx->poison, 1) == cudaSuccess &&
       dalloc(&ctx->status, 1) == cudaSuccess && dalloc(&ctx->stats, 1) == cudaSuccess &&
       dalloc(&ctx->impulses, 6 * kMaxBodies) == cudaSuccess &&
       dalloc(&ctx->bodies_d, kMaxBodies) == cudaSuccess &&
       dalloc(&ctx->dyn_d, kMaxBodies) == cudaSuccess &&
       dalloc(&ctx->imp0_d, 6 * kMaxBodies) == cudaSuccess &&
       dalloc(&ctx->bodies_step_d, kMaxBodies) == cudaSuccess;
  const int hist_len = sort_hist_len((int)cap);
  ok = ok && dalloc(&ctx->sb.keys[0], cap) == cudaSuccess && dalloc(&ctx->sb.keys[1], cap) == cudaSuccess &&
       dalloc(&ctx->sb.vals[0], cap) == cudaSuccess && dalloc(&ctx->sb.vals[1], cap) == cudaSuccess &&
       dalloc(&ctx->sb.hist, hist_len) == cudaSuccess &&
       dalloc(&ctx->sb.partial, hist_len / 4096 + 2) == cudaSuccess;
  ctx->sb.hist_cap = hist_len;
  ok = ok && dalloc(&ctx->stage, (size_t)24 * cap) == cudaSuccess;
  if (!ok) return bail(MPM_ERR_OOM);
  // zero-invariant arrays and counters
  ok = cudaMemset(ctx->G.mp, 0, nn * sizeof(float4)) == cudaSuccess &&
       cudaMemset(ctx->G.acc0, 0, nn * sizeof(float4)) == cudaSuccess &&
       cudaMemset(ctx->G.acc1, 0, nn * sizeof(float4)) == cudaSuccess &&
       cudaMemset(ctx->G.acc2, 0, nn * sizeof(float)) == cudaSuccess &&
       cudaMemset(ctx->G.vs, 0, nn * sizeof(float4)) == cudaSuccess &&
       cudaMemset(ctx->G.v, 0, nn * sizeof(float4)) == cudaSuccess &&
       cudaMemset(ctx->G.mark, 0, ctx->n_blocks) == cudaSuccess &&
       cudaMemset(ctx->G.n_act, 0, sizeof(int)) == cudaSuccess &&
       cudaMemset(ctx->G.n_mapped, 0, sizeof(int)) == cudaSuccess &&
       cudaMemset(ctx->C.count, 0, sizeof(int)) == cudaSuccess &&
       cudaMemset(ctx->red, 0, kRedDoubles * sizeof(double)) == cudaSuccess &&
       cudaMemset(ctx->G.cflag, 0, nn * sizeof(int)) == cudaSuccess &&
       cudaMemset(ctx->G.n_cnodes, 0, sizeof(int)) == cudaSuccess &&
       cudaMemset(ctx->G.pstar2, 0, sizeof(double)) == cudaSuccess &&
       cudaMemset(ctx->bar, 0, kBarWords * sizeof(unsigned)) == cudaSuccess &&
       cudaMemset(ctx->poison, 0, sizeof(int)) == cudaSuccess &&
       cudaMemset(ctx->status, 0, sizeof(uint32_t)) == cudaSuccess &&
       cudaMemset(ctx->stats, 0, sizeof(DevStats)) == cudaSuccess &&
       cudaMemset(ctx->impulses, 0, 6 * kMaxBodies * sizeof(double)) == cudaSuccess &&
       cudaDeviceSynchronize() == cudaSuccess;
  if (!ok) return bail(MPM_ERR_CUDA);
  if (p2g_prepare() != cudaSuccess || sort_prepare() != cudaSuccess) return bail(MPM_ERR_CUDA);
  int occ = 0;
  if (solve_prepare() != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, solve_kernel_ptr(), solve_block_size(),
                                                    solve_dynamic_smem()) != cudaSuccess ||
      occ < 1)
    return bail(MPM_ERR_CUDA);
  ctx->solve_blocks = ctx->num_sms * (occ < 2 ? occ : 2);
  ctx->cluster_blocks = solve_cluster_blocks();
  ctx->cluster_blocks_max = ctx->cluster_blocks;
  *out = ctx;
  return MPM_OK;
}

mpm_status mpm_destroy(mpm_ctx* ctx) {
  if (!ctx) return MPM_OK;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  release(ctx);
  delete ctx;
  return MPM_OK;
}

const char* mpm_last_error(const mpm_ctx* ctx) {
  if (!ctx) return kGenericError;
  return ctx->err.c_str();
}

namespace {

// Per-group constants: Lame parameters from (E, nu), Drucker-Prager slope
// from the friction angle.
DevGroup make_group(const mpm_material& mat, float particle_volume) {
  DevGroup gr;
  memset(&gr, 0, sizeof(gr));
  const double E = mat.E, nu = mat.nu;
  gr.vol = particle_volume;
  gr.mass = (float)((double)mat.rho * (double)particle_volume);
  gr.vol_m = (float)((double)gr.vol / (double)gr.mass);
  gr.inv_m = (float)(1.0 / (double)gr.mass);
  gr.mu_l = (float)(E / (2.0 * (1.0 + nu)));
  gr.lam = (float)(E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)));
  const double sphi = std::sin((double)mat.friction_angle_deg * 3.14159265358979323846 / 180.0);
  gr.dp_alpha = (float)(std::sqrt(2.0 / 3.0) * 2.0 * sphi / (3.0 - sphi));
  gr.model = mat.model;
  return gr;
}

bool material_ok(const mpm_material* mat) {
  return mat &&
         (mat->model == MPM_COROTATED || mat->model == MPM_DRUCKER_PRAGER || mat->model == MPM_CLOTH) &&
         mat->E > 0.f && mat->nu > -1.f && mat->nu < 0.5f && mat->rho > 0.f;
}

}  // namespace

mpm_status mpm_set_material(mpm_ctx* ctx, int32_t group, const mpm_material* mat) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (group < 0 || group >= (int32_t)ctx->groups.size() || !material_ok(mat))
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_set_material: bad group or material");
  if (ctx->taping)
    return fail(ctx, MPM_ERR_STATE, "mpm_set_material: not while a tape is recorded");
  if (mat->rho != ctx->mats[group].rho)
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_set_material: the density (particle mass) is fixed");
  if ((mat->model == MPM_CLOTH) != (ctx->mats[group].model == MPM_CLOTH))
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_set_material: cloth stays cloth");
  ctx->groups[group] = make_group(*mat, ctx->groups[group].vol);
  ctx->mats[group] = *mat;
  CU(cudaMemcpyAsync(ctx->groups_d, ctx->groups.data(), ctx->groups.size() * sizeof(DevGroup),
                     cudaMemcpyHostToDevice, ctx->stream));
  // the stored stress follows the new constants
  if (ctx->n > 0) launch_stress_from_F(ctx->P[ctx->cur], (int)ctx->n, ctx->groups_d, ctx->stream);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(ctx->stream));
  return MPM_OK;
}

namespace {
mpm_status add_particles(mpm_ctx* ctx, int64_t n, const float* x, const float* v,
                         float particle_volume, const mpm_material* mat, int32_t mem_kind,
                         int64_t* first_id);
}  // namespace

mpm_status mpm_add_particles(mpm_ctx* ctx, int64_t n, const float* x, const float* v,
                             float particle_volume, const mpm_material* mat, int32_t mem_kind,
                             int64_t* first_id) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (mat && mat->model != MPM_COROTATED && mat->model != MPM_DRUCKER_PRAGER)
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_add_particles: unknown material model");
  return add_particles(ctx, n, x, v, particle_volume, mat, mem_kind, first_id);
}

mpm_status mpm_add_cloth(mpm_ctx* ctx, int64_t n_vertices, const float* x, const float* v,
                         int64_t n_triangles, const int32_t* triangles, float thickness,
                         const mpm_material* material, int32_t mem_kind, int64_t* first_id) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (n_vertices <= 0 || n_triangles <= 0 || !x || !v || !triangles || !material ||
      material->model != MPM_CLOTH || !(thickness > 0.f) ||
      (mem_kind != MPM_MEM_HOST && mem_kind != MPM_MEM_DEVICE))
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_add_cloth: bad argument");
  if (ctx->taping) return fail(ctx, MPM_ERR_STATE, "mpm_add_cloth: a tape is recording");
  if (n_triangles >= (1LL << 30)) return fail(ctx, MPM_ERR_CAPACITY, "mpm_add_cloth: too many triangles");
  // rest positions on the host
  std::vector<float> xh((size_t)3 * n_vertices);
  if (mem_kind == MPM_MEM_DEVICE)
    CU(cudaMemcpy(xh.data(), x, xh.size() * sizeof(float), cudaMemcpyDeviceToHost));
  else
    memcpy(xh.data(), x, xh.size() * sizeof(float));
  std::vector<double> rest((size_t)5 * n_triangles);
  double total_area = 0.0;
  for (int64_t t = 0; t < n_triangles; ++t) {
    double X[3][3];
    for (int k = 0; k < 3; ++k) {
      const int32_t vi = triangles[3 * t + k];
      if (vi < 0 || vi >= n_vertices)
        return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_add_cloth: vertex index out of range");
      for (int c = 0; c < 3; ++c) X[k][c] = (double)xh[3 * (size_t)vi + c];
    }
    cloth_rest_shape(X[0], X[1], X[2], &rest[5 * (size_t)t]);
    const double a = rest[5 * (size_t)t + 4];
    if (!(a > 0.0) || !std::isfinite(rest[5 * (size_t)t]) || !std::isfinite(rest[5 * (size_t)t + 3]))
      return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_add_cloth: a degenerate triangle");
    total_area += a;
    rest[5 * (size_t)t + 4] = a * (double)thickness;  // the energy weight: rest volume
  }
  const float vol = (float)(thickness * total_area / (double)n_vertices);
  int64_t first = 0;
  const mpm_status st = add_particles(ctx, n_vertices, x, v, vol, material, mem_kind, &first);
  if (st != MPM_OK) return st;
  const int grp = (int)ctx->groups.size() - 1;
  for (int64_t t = 0; t < n_triangles; ++t)
    ctx->cloth_tris.push_back(make_int4((int)(first + triangles[3 * t]),
                                        (int)(first + triangles[3 * t + 1]),
                                        (int)(first + triangles[3 * t + 2]), grp));
  ctx->cloth_rest.insert(ctx->cloth_rest.end(), rest.begin(), rest.end());
  // device copies (reallocated: cloth is added at setup, not per step)
  cudaFree(ctx->cloth_tris_d);
  cudaFree(ctx->cloth_rest_d);
  ctx->cloth_tris_d = nullptr;
  ctx->cloth_rest_d = nullptr;
  CU(dalloc(&ctx->cloth_tris_d, ctx->cloth_tris.size()));
  CU(dalloc(&ctx->cloth_rest_d, ctx->cloth_rest.size()));
  CU(cudaMemcpy(ctx->cloth_tris_d, ctx->cloth_tris.data(), ctx->cloth_tris.size() * sizeof(int4),
                cudaMemcpyHostToDevice));
  CU(cudaMemcpy(ctx->cloth_rest_d, ctx->cloth_rest.data(), ctx->cloth_rest.size() * sizeof(double),
                cudaMemcpyHostToDevice));
  if (!ctx->cloth_f_d) {
    // zero once: every P2G leaves the planes zero for the next substep's forces
    CU(dalloc(&ctx->cloth_f_d, (size_t)3 * ctx->cap));
    CU(cudaMemsetAsync(ctx->cloth_f_d, 0, (size_t)3 * ctx->cap * sizeof(float), ctx->stream));
  }
  if (!ctx->slot_of_d) CU(dalloc(&ctx->slot_of_d, (size_t)ctx->cap));
  // (graphs recorded before had no cloth pass)
  for (auto& e : ctx->gexec)
    if (e) {
      cudaGraphExecDestroy(e);
      e = nullptr;
    }
  if (first_id) *first_id = first;
  return MPM_OK;
}

mpm_status mpm_set_pins(mpm_ctx* ctx, int64_t n_pins, const int64_t* ids, const float* v) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (n_pins < 0 || (n_pins > 0 && (!ids || !v)))
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_set_pins: bad argument");
  if (ctx->taping) return fail(ctx, MPM_ERR_STATE, "mpm_set_pins: a tape is recording");
  std::vector<int64_t> sorted(ids, ids + n_pins);
  std::sort(sorted.begin(), sorted.end());
  for (int64_t j = 0; j < n_pins; ++j) {
    if (sorted[j] < 0 || sorted[j] >= ctx->n || (j > 0 && sorted[j] == sorted[j - 1]))
      return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_set_pins: ids must be distinct particle ids");
    for (int c = 0; c < 3; ++c)
      if (!std::isfinite(v[3 * j + c]))
        return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_set_pins: a velocity is not finite");
  }
  // the pin arrays may be in use by work in flight
  CU(cudaStreamSynchronize(ctx->stream));
  if (n_pins > ctx->pins_cap) {
    cudaFree(ctx->pin_ids_d);
    cudaFree(ctx->pin_v_d);
    cudaFree(ctx->pin_x_d);
    ctx->pin_ids_d = nullptr;
    ctx->pin_v_d = ctx->pin_x_d = nullptr;
    ctx->pins_cap = 0;
    CU(dalloc(&ctx->pin_ids_d, (size_t)n_pins));
    CU(dalloc(&ctx->pin_v_d, 3 * (size_t)n_pins));
    CU(dalloc(&ctx->pin_x_d, 3 * (size_t)n_pins));
    ctx->pins_cap = (int)n_pins;
  }
  if (!ctx->pin_mask_d) CU(dalloc(&ctx->pin_mask_d, (size_t)ctx->cap));
  CU(cudaMemsetAsync(ctx->pin_mask_d, 0, (size_t)ctx->cap, ctx->stream));
  if (n_pins > 0) {
    if (!ctx->slot_of_d) CU(dalloc(&ctx->slot_of_d, (size_t)ctx->cap));
    std::vector<int> id32((size_t)n_pins);
    std::vector<float> vp(3 * (size_t)ctx->pins_cap, 0.f);
    for (int64_t j = 0; j < n_pins; ++j) {
      id32[j] = (int)ids[j];
      for (int c = 0; c < 3; ++c) vp[j + (size_t)c * ctx->pins_cap] = v[3 * j + c];
    }
    CU(cudaMemcpyAsync(ctx->pin_ids_d, id32.data(), id32.size() * sizeof(int), cudaMemcpyHostToDevice,
                       ctx->stream));
    CU(cudaMemcpyAsync(ctx->pin_v_d, vp.data(), vp.size() * sizeof(float), cudaMemcpyHostToDevice,
                       ctx->stream));
    std::vector<uint8_t> mask((size_t)ctx->n, 0);
    for (int64_t j = 0; j < n_pins; ++j) mask[(size_t)ids[j]] = 1;
    CU(cudaMemcpyAsync(ctx->pin_mask_d, mask.data(), mask.size(), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
  }
  ctx->n_pins = (int)n_pins;
  // (graphs recorded before hold the old pin launches)
  for (auto& e : ctx->gexec)
    if (e) {
      cudaGraphExecDestroy(e);
      e = nullptr;
    }
  return MPM_OK;
}

namespace {
mpm_status add_particles(mpm_ctx* ctx, int64_t n, const float* x, const float* v,
                         float particle_volume, const mpm_material* mat, int32_t mem_kind,
                         int64_t* first_id) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (n < 0 || (n > 0 && (!x || !v)) || !mat || !(particle_volume > 0.f) ||
      (mem_kind != MPM_MEM_HOST && mem_kind != MPM_MEM_DEVICE))
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_add_particles: bad argument");
  if (!(mat->E > 0.f) || !(mat->nu > -1.f && mat->nu < 0.5f) || !(mat->rho > 0.f))
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_add_particles: bad material constants");
  if (ctx->n + n > ctx->cap) return fail(ctx, MPM_ERR_CAPACITY, "mpm_add_particles: max_particles exceeded");
  if (ctx->groups.size() >= 65535) return fail(ctx, MPM_ERR_CAPACITY, "mpm_add_particles: too many groups");
  if (first_id) *first_id = ctx->n;
  const DevGroup gr = make_group(*mat, particle_volume);
  ctx->groups.push_back(gr);
  ctx->mats.push_back(*mat);
  if ((int)ctx->groups.size() > ctx->groups_cap) {
    int nc = ctx->groups_cap ? 2 * ctx->groups_cap : 64;
    while (nc < (int)ctx->groups.size()) nc *= 2;
    DevGroup* nd = nullptr;
    CU(cudaStreamSynchronize(ctx->stream));
    CU(dalloc(&nd, nc));
    if (ctx->groups_d) cudaFree(ctx->groups_d);
    ctx->groups_d = nd;
    ctx->groups_cap = nc;
  }
  CU(cudaMemcpyAsync(ctx->groups_d, ctx->groups.data(), ctx->groups.size() * sizeof(DevGroup),
                     cudaMemcpyHostToDevice, ctx->stream));
  if (n > 0) {
    const float *dx = x, *dv = v;
    if (mem_kind == MPM_MEM_HOST) {
      CU(cudaMemcpyAsync(ctx->stage, x, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
      CU(cudaMemcpyAsync(ctx->stage + 3 * n, v, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice,
                         ctx->stream));
      dx = ctx->stage;
      dv = ctx->stage + 3 * n;
    }
    k_append<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(
        ctx->P[ctx->cur], ctx->n, n, dx, dv, (uint16_t)(ctx->groups.size() - 1));
    CU(cudaGetLastError());
  }
  ctx->n += n;
  CU(cudaStreamSynchronize(ctx->stream));
  return MPM_OK;
}
}  // namespace

mpm_status mpm_num_particles(const mpm_ctx* ctx, int64_t* n) {
  if (!ctx || !n) return MPM_ERR_INVALID_ARG;
  *n = ctx->n;
  return MPM_OK;
}

mpm_status mpm_set_particles(mpm_ctx* ctx, const float* x, const float* v, const float* C,
                             const float* F, int32_t mem_kind) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (mem_kind != MPM_MEM_HOST && mem_kind != MPM_MEM_DEVICE)
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_set_particles: bad mem_kind");
  const int64_t n = ctx->n;
  if (n == 0) return MPM_OK;
  if (ctx->taping && !ctx->tape.empty()) ctx->tape_reset = true;
  const float* src[4] = {x, v, C, F};
  const int width[4] = {3, 3, 9, 9};
  const float* dptr[4] = {nullptr, nullptr, nullptr, nullptr};
  size_t off = 0;
  for (int f = 0; f < 4; ++f) {
    if (!src[f]) continue;
    if (mem_kind == MPM_MEM_HOST) {
      CU(cudaMemcpyAsync(ctx->stage + off, src[f], (size_t)n * width[f] * sizeof(float),
                         cudaMemcpyHostToDevice, ctx->stream));
      dptr[f] = ctx->stage + off;
      off += (size_t)n * width[f];
    } else {
      dptr[f] = src[f];
    }
  }
  launch_from_id_order(ctx->P[ctx->cur], (int)n, dptr[0], dptr[1], dptr[2], dptr[3], ctx->stream);
  if (F) launch_stress_from_F(ctx->P[ctx->cur], (int)n, ctx->groups_d, ctx->stream);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(ctx->stream));
  return MPM_OK;
}

mpm_status mpm_get_particles(mpm_ctx* ctx, float* x, float* v, float* C, float* F, int32_t mem_kind) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (mem_kind != MPM_MEM_HOST && mem_kind != MPM_MEM_DEVICE)
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_get_particles: bad mem_kind");
  const int64_t n = ctx->n;
  if (n == 0) return MPM_OK;
  float* dst[4] = {x, v, C, F};
  const int width[4] = {3, 3, 9, 9};
  float* dptr[4] = {nullptr, nullptr, nullptr, nullptr};
  size_t off = 0;
  for (int f = 0; f < 4; ++f) {
    if (!dst[f]) continue;
    if (mem_kind == MPM_MEM_HOST) {
      dptr[f] = ctx->stage + off;
      off += (size_t)n * width[f];
    } else {
      dptr[f] = dst[f];
    }
  }
  launch_to_id_order(ctx->P[ctx->cur], (int)n, dptr[0], dptr[1], dptr[2], dptr[3], ctx->stream);
  CU(cudaGetLastError());
  if (mem_kind == MPM_MEM_HOST)
    for (int f = 0; f < 4; ++f)
      if (dst[f])
        CU(cudaMemcpyAsync(dst[f], dptr[f], (size_t)n * width[f] * sizeof(float), cudaMemcpyDeviceToHost,
                           ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return MPM_OK;
}

mpm_status mpm_set_rigid_bodies(mpm_ctx* ctx, int32_t n, const mpm_rigid_body* bodies) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (n < 0 || n > kMaxBodies || (n > 0 && !bodies))
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_set_rigid_bodies: at most 16 bodies");
  for (int i = 0; i < n; ++i) {
    const mpm_rigid_body& b = bodies[i];
    if (b.shape < MPM_HALFSPACE || b.shape > MPM_CAPSULE || !(b.mu >= 0.f) || !(b.k > 0.f) ||
        !(b.d >= 0.f))
      return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_set_rigid_bodies: bad body");
  }
  if (ctx->taping && !ctx->tape.empty()) ctx->tape_reset = true;
  ctx->bodies.assign(bodies, bodies + n);
  ctx->bodies_dirty = true;
  ctx->bodies_stale = false;
  ctx->dyn_dirty = true;
  ctx->is_dyn.assign(n, 0);
  ctx->dyn.assign(n, mpm_rigid_dynamics{});
  ctx->imp_seen_valid = false;
  return MPM_OK;
}

mpm_status mpm_set_rigid_dynamics(mpm_ctx* ctx, int32_t index, const mpm_rigid_dynamics* dyn) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (index < 0 || index >= (int32_t)ctx->bodies.size())
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_set_rigid_dynamics: no such body");
  if (dyn) {
    if (!(dyn->mass > 0.f) || !(dyn->inertia[0] > 0.f) || !(dyn->inertia[1] > 0.f) ||
        !(dyn->inertia[2] > 0.f) || dyn->dof_mask < 0 || dyn->dof_mask > 63)
      return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_set_rigid_dynamics: bad mass, inertia or mask");
    for (int i = 0; i < 3; ++i)
      if (!std::isfinite(dyn->force[i]) || !std::isfinite(dyn->torque[i]))
        return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_set_rigid_dynamics: non-finite load");
    ctx->dyn[index] = *dyn;
  }
  ctx->is_dyn[index] = dyn ? 1 : 0;
  ctx->imp_seen_valid = false;
  ctx->dyn_dirty = true;
  return MPM_OK;
}

mpm_status mpm_get_rigid_bodies(const mpm_ctx* cctx, int32_t n, mpm_rigid_body* out) {
  if (!cctx || !out || n < 0 || n > (int32_t)cctx->bodies.size()) return MPM_ERR_INVALID_ARG;
  // (the context's host copy of the bodies is refreshed, nothing else)
  mpm_ctx* ctx = const_cast<mpm_ctx*>(cctx);
  CU(sync_host_bodies(ctx));
  for (int i = 0; i < n; ++i) out[i] = ctx->bodies[i];
  return MPM_OK;
}

mpm_status mpm_step(mpm_ctx* ctx, double h, int32_t n_substeps, const mpm_solver_params* solver,
                    mpm_step_stats* stats) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (!(h > 0.0) || n_substeps < 0)
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_step: h must be > 0 and n_substeps >= 0");
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
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_step: bad solver parameters");
  cudaStream_t s = ctx->stream;
  const int nb = (int)ctx->bodies.size();
  // the bodies move on the device after the step unless a tape records the
  // steps (the tape keeps each step's bodies and impulses on the host)
  const bool dev_rigid = !ctx->taping;
  if (!dev_rigid) CU(sync_host_bodies(ctx));
  if (ctx->bodies_dirty) {
    DevBody tmp[kMaxBodies];
    for (int i = 0; i < nb; ++i) tmp[i] = to_dev(ctx->bodies[i]);
    if (nb) CU(cudaMemcpyAsync(ctx->bodies_d, tmp, nb * sizeof(DevBody), cudaMemcpyHostToDevice, s));
    ctx->bodies_dirty = false;
  }
  if (dev_rigid && ctx->dyn_dirty) CU(upload_dynamics(ctx));
  bool has_dyn = false;
  for (int d : ctx->is_dyn) has_dyn = has_dyn || d;
  if (!dev_rigid && has_dyn && !ctx->imp_seen_valid) {
    // the impulse accumulator at the start of the step (the caller's resets
    // and earlier steps included), so that the step's own impulses are known
    ctx->imp_seen.assign(6 * kMaxBodies, 0.0);
    if (nb) {
      CU(cudaMemcpyAsync(ctx->imp_seen.data(), ctx->impulses, 6 * nb * sizeof(double),
                         cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
    }
    ctx->imp_seen_valid = true;
  }
  if (ctx->taping && n_substeps > 0) {
    if (ctx->n != ctx->tape_n)
      return fail(ctx, MPM_ERR_STATE, "mpm_step: particles were added while a tape is recorded");
    mpm_ctx::TapeStep t;
    CU(dalloc(&t.state, (size_t)24 * ctx->n));
    const size_t nn = (size_t)ctx->n;
    launch_to_id_order(ctx->P[ctx->cur], (int)nn, t.state, t.state + 3 * nn, t.state + 6 * nn,
                       t.state + 15 * nn, s);
    for (int i = 0; i < nb; ++i) {
      const bool d = i < (int)ctx->is_dyn.size() && ctx->is_dyn[i];
      t.bodies.push_back(to_dev(ctx->bodies[i]));
      t.kinematic.push_back(ctx->bodies[i].kinematic != 0 && !d);
      t.is_dyn.push_back(d ? 1 : 0);
      t.dyn.push_back(d ? ctx->dyn[i] : mpm_rigid_dynamics{});
    }
    t.imp.assign(6 * nb, 0.0);
    t.n_substeps = n_substeps;
    t.rec_base = ctx->tape_substeps;
    ctx->tape_substeps += n_substeps;
    t.h = (float)h;
    t.sp = sp;
    ctx->tape.push_back(std::move(t));
  }
  CU(cudaMemsetAsync(ctx->stats, 0, sizeof(DevStats), s));
  const int n = (int)ctx->n;
  const bool sort_now = n > 0 && ctx->step_count % ctx->sort_every == 0;
  const float hf = (float)h;
  const int solve_blocks = ctx->solve_blocks_cap > 0 && ctx->solve_blocks_cap < ctx->solve_blocks
                               ? ctx->solve_blocks_cap
                               : ctx->solve_blocks;
  const int from = ctx->cur;
  bool launched = false;
  if (ctx->use_graphs && !ctx->profile && !ctx->wait_test && n_substeps > 0) {
    mpm_ctx::GraphKey k;
    k.n = n; k.n_substeps = n_substeps; k.nb = nb; k.chunk = ctx->p2g_chunk;
    k.sort_now = sort_now ? 1 : 0; k.solve_blocks = solve_blocks; k.h = hf; k.sp = sp;
    k.cluster_max = cluster_contacts(ctx);
    k.cluster_blocks = ctx->cluster_blocks;
    k.p2g_form = ctx->p2g_form;
    k.rigid = dev_rigid ? 1 : 0;
    k.taping = ctx->taping && ctx->tape_pool ? 1 : 0;
    k.tape_pool = ctx->tape_pool;
    const mpm_ctx::GraphKey& o = ctx->gkey[from];
    const bool same = ctx->gexec[from] && o.n == k.n && o.n_substeps == k.n_substeps && o.nb == k.nb &&
                      o.chunk == k.chunk && o.sort_now == k.sort_now &&
                      o.solve_blocks == k.solve_blocks && o.h == k.h && o.taping == k.taping &&
                      o.cluster_max == k.cluster_max && o.cluster_blocks == k.cluster_blocks &&
                      o.rigid == k.rigid && o.p2g_form == k.p2g_form &&
                      o.tape_pool == k.tape_pool &&
                      memcmp(&o.sp, &k.sp, sizeof(k.sp)) == 0;
    if (!same) {
      if (ctx->gexec[from]) {
        cudaGraphExecDestroy(ctx->gexec[from]);
        ctx->gexec[from] = nullptr;
      }
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const cudaError_t le =
            enqueue_step(ctx, from, sort_now, n_substeps, hf, sp, solve_blocks, s, dev_rigid);
        e = cudaStreamEndCapture(s, &graph);
        if (e == cudaSuccess) e = le;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->gexec[from], graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e == cudaSuccess) {
        ctx->gkey[from] = k;
      } else {
        // this device or driver cannot capture the sequence: launch directly
        // from now on (the same kernels, without the graph)
        cudaGetLastError();
        if (ctx->gexec[from]) cudaGraphExecDestroy(ctx->gexec[from]);
        ctx->gexec[from] = nullptr;
        ctx->use_graphs = false;
      }
    }
    if (ctx->gexec[from]) {
      CU(cudaGraphLaunch(ctx->gexec[from], s));
      launched = true;
    }
  }
  if (!launched) CU(enqueue_step(ctx, from, sort_now, n_substeps, hf, sp, solve_blocks, s, dev_rigid));
  if (sort_now) ctx->cur = 1 - from;
  CU(cudaGetLastError());
  ctx->adj_ready = n_substeps > 0;
  ctx->last_dev_rigid = dev_rigid;
  ctx->last_h = hf;
  ctx->last_eps_s = sp.eps_s;
  ctx->last_nb = nb;
  // async splitting (Eq. (3)-(4)): kinematic bodies move with their frozen
  // velocity; dynamic ones take the step's accumulated contact impulses (on
  // the device, launched above; on the host while a tape records)
  const double dt = h * n_substeps;
  bool moved = false, any_dyn = false;
  if (dev_rigid) {
    if (nb > 0 && n_substeps > 0) ctx->bodies_stale = true;
    ctx->imp_seen_valid = false;
  }
  for (size_t i = 0; i < ctx->bodies.size() && !dev_rigid; ++i) {
    if (ctx->is_dyn[i]) {
      any_dyn = true;
    } else if (ctx->bodies[i].kinematic) {
      advance_kinematic(ctx->bodies[i], dt);
      moved = true;
    }
  }
  if (any_dyn && !dev_rigid) {
    std::vector<double> now(6 * kMaxBodies, 0.0);
    CU(cudaMemcpyAsync(now.data(), ctx->impulses, 6 * nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    for (size_t i = 0; i < ctx->bodies.size(); ++i) {
      if (!ctx->is_dyn[i]) continue;
      double J[3], L[3];
      for (int c = 0; c < 3; ++c) {
        J[c] = now[6 * i + c] - ctx->imp_seen[6 * i + c];
        L[c] = now[6 * i + 3 + c] - ctx->imp_seen[6 * i + 3 + c];
      }
      if (ctx->taping && n_substeps > 0 && !ctx->tape.empty())
        for (int c = 0; c < 3; ++c) {
          ctx->tape.back().imp[6 * i + c] = J[c];
          ctx->tape.back().imp[6 * i + 3 + c] = L[c];
        }
      integrate_dynamic(ctx->bodies[i], ctx->dyn[i], ctx->spec.gravity, J, L, dt);
    }
    ctx->imp_seen = now;
    ctx->imp_seen_valid = true;
    moved = true;
  } else if (!dev_rigid) {
    ctx->imp_seen_valid = false;  // the accumulator moves on untracked
  }
  if (moved) ctx->bodies_dirty = true;
  ctx->step_count += 1;
  if (!stats) return MPM_OK;
  uint32_t bits = 0;
  mpm_status st = drain_status(ctx, &bits);
  DevStats ds;
  cudaError_t e = cudaMemcpy(&ds, ctx->stats, sizeof(ds), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(ctx, MPM_ERR_CUDA, cudaGetErrorString(e));
  memset(stats, 0, sizeof(*stats));
  stats->substeps = ds.substeps;
  stats->iters_total = ds.iters_total;
  stats->iters_max = ds.iters_max;
  stats->ls_evals_total = ds.ls_evals_total;
  stats->contacts_max = ds.contacts_max;
  stats->active_blocks_max = ds.active_blocks_max;
  stats->contacts_total = (int64_t)ds.contacts_total;
  stats->residual_max = ds.residual_max;
  stats->status_bits = (int32_t)bits;
  stats->p2g_global_chunks = ds.p2g_global_chunks;
  stats->ls_split_substeps = ds.ls_split;
  stats->cluster_substeps = ds.cluster;
  stats->contact_nodes_max = ds.cnodes_max;
  for (int k = 0; k < 5; ++k) stats->solve_us[k] = (float)(ds.solve_ns[k] * 1e-3);
  return st;
}

mpm_status mpm_get_rigid_impulses(mpm_ctx* ctx, double* out, int32_t reset) {
  if (!ctx || (!out && !ctx->bodies.empty())) return MPM_ERR_INVALID_ARG;
  CU(cudaStreamSynchronize(ctx->stream));
  const size_t nb = ctx->bodies.size();
  if (nb) CU(cudaMemcpy(out, ctx->impulses, 6 * nb * sizeof(double), cudaMemcpyDeviceToHost));
  if (reset) {
    CU(cudaMemsetAsync(ctx->impulses, 0, 6 * kMaxBodies * sizeof(double), ctx->stream));
    ctx->imp_seen.assign(6 * kMaxBodies, 0.0);
    ctx->imp_seen_valid = true;
  }
  return MPM_OK;
}

mpm_status mpm_get_grid(mpm_ctx* ctx, int64_t cap, int64_t* count, int32_t* node_ids, float* m,
                        float* vstar, float* v) {
  if (!ctx || !count || cap < 0) return MPM_ERR_INVALID_ARG;
  CU(cudaStreamSynchronize(ctx->stream));
  DevStats ds;
  CU(cudaMemcpy(&ds, ctx->stats, sizeof(ds), cudaMemcpyDeviceToHost));
  const int n_act = ds.last_active;
  const size_t max_nodes = (size_t)n_act * kBlockNodes;
  // stage layout: [count | ids | m | vs(3) | v(3)], sized for the active nodes
  std::vector<int> h_ids(max_nodes);
  std::vector<float> h_m(max_nodes), h_vs(3 * max_nodes), h_v(3 * max_nodes);
  int* d_count = nullptr;
  int* d_ids = nullptr;
  float *d_m = nullptr, *d_vs = nullptr, *d_v = nullptr;
  CU(dalloc(&d_count, 1));
  bool ok = dalloc(&d_ids, max_nodes + 1) == cudaSuccess && dalloc(&d_m, max_nodes + 1) == cudaSuccess &&
            dalloc(&d_vs, 3 * max_nodes + 3) == cudaSuccess && dalloc(&d_v, 3 * max_nodes + 3) == cudaSuccess;
  int got = 0;
  if (ok) {
    cudaMemsetAsync(d_count, 0, sizeof(int), ctx->stream);
    if (n_act > 0)
      k_grid_out<<<ctx->num_sms * 4, 256, 0, ctx->stream>>>(ctx->g, ctx->G, n_act, d_count, d_ids, d_m,
                                                           d_vs, d_v);
    ok = cudaStreamSynchronize(ctx->stream) == cudaSuccess &&
         cudaMemcpy(&got, d_count, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
    if (ok && got > 0) {
      ok = cudaMemcpy(h_ids.data(), d_ids, got * sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess &&
           cudaMemcpy(h_m.data(), d_m, got * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess &&
           cudaMemcpy(h_vs.data(), d_vs, 3 * got * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess &&
           cudaMemcpy(h_v.data(), d_v, 3 * got * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess;
    }
  }
  cudaFree(d_count); cudaFree(d_ids); cudaFree(d_m); cudaFree(d_vs); cudaFree(d_v);
  if (!ok) return fail(ctx, MPM_ERR_CUDA, "mpm_get_grid: device read failed");
  *count = got;
  const int64_t k = got < cap ? got : cap;
  for (int64_t i = 0; i < k; ++i) {
    if (node_ids) node_ids[i] = h_ids[i];
    if (m) m[i] = h_m[i];
    for (int c = 0; c < 3; ++c) {
      if (vstar) vstar[3 * i + c] = h_vs[3 * i + c];
      if (v) v[3 * i + c] = h_v[3 * i + c];
    }
  }
  return MPM_OK;
}

mpm_status mpm_get_contacts(mpm_ctx* ctx, int64_t cap, int64_t* count, int32_t* particle, int32_t* body,
                            float* gamma, float* phi0, float* n0) {
  if (!ctx || !count || cap < 0) return MPM_ERR_INVALID_ARG;
  CU(cudaStreamSynchronize(ctx->stream));
  DevStats ds;
  CU(cudaMemcpy(&ds, ctx->stats, sizeof(ds), cudaMemcpyDeviceToHost));
  const int nc = ds.last_contacts;
  *count = nc;
  const int64_t k = nc < cap ? nc : cap;
  if (k <= 0) return MPM_OK;
  std::vector<int2> ids(k);
  std::vector<float4> xp(k), nrm(k), gam(k);
  CU(cudaMemcpy(ids.data(), ctx->C.id, k * sizeof(int2), cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(xp.data(), ctx->C.xp, k * sizeof(float4), cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(nrm.data(), ctx->C.nrm, k * sizeof(float4), cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(gam.data(), ctx->C.gamma, k * sizeof(float4), cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < k; ++i) {
    if (particle) particle[i] = ids[i].x;
    if (body) body[i] = ids[i].y;
    if (gamma) {
      gamma[3 * i] = gam[i].x;
      gamma[3 * i + 1] = gam[i].y;
      gamma[3 * i + 2] = gam[i].z;
    }
    if (phi0) phi0[i] = xp[i].w;
    if (n0) n0[i] = nrm[i].w;
  }
  return MPM_OK;
}

mpm_status mpm_contact_adjoint(mpm_ctx* ctx, int32_t mem_kind, int64_t n, const int32_t* node_ids,
                               const float* vbar, float* vstar_bar, int64_t contact_cap,
                               float* contact_bar, double* body_bar,
                               const mpm_adjoint_params* params, mpm_adjoint_stats* stats) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (mem_kind != MPM_MEM_HOST && mem_kind != MPM_MEM_DEVICE)
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_contact_adjoint: bad mem_kind");
  if (n < 0 || n > (int64_t)(INT32_MAX / 3) || (n > 0 && (!node_ids || !vbar || !vstar_bar)) ||
      contact_cap < 0 || (contact_cap > 0 && !contact_bar))
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_contact_adjoint: bad node or contact arrays");
  mpm_adjoint_params ap;
  ap.eps_r = 1e-5;
  ap.max_iters = 1000;
  if (params) ap = *params;
  if (!(ap.eps_r >= 0.0) || ap.max_iters < 0)
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_contact_adjoint: bad parameters");
  if (!ctx->adj_ready)
    return fail(ctx, MPM_ERR_STATE, "mpm_contact_adjoint: no substep to differentiate (mpm_step first)");
  const int64_t n_grid = (int64_t)ctx->g.rx * ctx->g.ry * ctx->g.rz;
  if (mem_kind == MPM_MEM_HOST)
    for (int64_t i = 0; i < n; ++i)
      if (node_ids[i] < 0 || node_ids[i] >= n_grid)
        return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_contact_adjoint: node id outside the grid");
  // failures of earlier calls are reported first, not taken for the adjoint's
  mpm_status st = drain_status(ctx);
  if (st != MPM_OK) return st;
  cudaStream_t s = ctx->stream;
  if (!ctx->adj_vec) {
    CU(dalloc(&ctx->adj_vec, (size_t)kAdjointVectors * ctx->G.cnodes_cap));
    CU(dalloc(&ctx->adj_body, kAdjBodySlots * kMaxBodies));
    CU(dalloc(&ctx->adj_out, 4));
    int occ = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, adjoint_kernel_ptr(), solve_block_size(), 0));
    if (occ < 1) return fail(ctx, MPM_ERR_CUDA, "mpm_contact_adjoint: kernel does not fit an SM");
    ctx->adj_blocks = ctx->num_sms * (occ < 2 ? occ : 2);
  }
  const int64_t ccap = contact_cap < ctx->C.cap ? contact_cap : ctx->C.cap;
  const int32_t* d_ids = node_ids;
  const float* d_vbar = vbar;
  float* d_vsb = vstar_bar;
  float* d_cbar = contact_bar;
  if (mem_kind == MPM_MEM_HOST) {
    const size_t need_io = (size_t)6 * n + (size_t)4 * ccap;
    if (ctx->adj_ids_cap < (size_t)n || !ctx->adj_ids) {
      if (ctx->adj_ids) cudaFree(ctx->adj_ids);
      ctx->adj_ids = nullptr;
      ctx->adj_ids_cap = 0;
      CU(dalloc(&ctx->adj_ids, (size_t)n + 1));
      ctx->adj_ids_cap = (size_t)n + 1;
    }
    if (ctx->adj_io_cap < need_io || !ctx->adj_io) {
      if (ctx->adj_io) cudaFree(ctx->adj_io);
      ctx->adj_io = nullptr;
      ctx->adj_io_cap = 0;
      CU(dalloc(&ctx->adj_io, need_io + 4));
      ctx->adj_io_cap = need_io + 4;
    }
    float* io = ctx->adj_io;
    d_ids = ctx->adj_ids;
    d_vbar = io;
    d_vsb = io + 3 * n;
    d_cbar = ccap > 0 ? io + 6 * n : nullptr;
    if (n > 0) {
      CU(cudaMemcpyAsync(ctx->adj_ids, node_ids, n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
      CU(cudaMemcpyAsync(io, vbar, 3 * n * sizeof(float), cudaMemcpyHostToDevice, s));
    }
  }
  AdjointArgs a;
  memset(&a, 0, sizeof(a));  // gbar = nullptr: the single-solve mode
  a.g = ctx->g; a.G = ctx->G; a.C = ctx->C; a.nb = ctx->last_nb;
  a.bodies = ctx->last_dev_rigid ? ctx->bodies_step_d : ctx->bodies_d;
  a.h = ctx->last_h; a.eps_s = ctx->last_eps_s; a.eps_r = ap.eps_r; a.max_iters = ap.max_iters;
  a.n_in = (int)n; a.ids = d_ids; a.vbar = d_vbar; a.vstar_bar = d_vsb;
  a.contact_bar = d_cbar; a.contact_cap = (int)ccap; a.body_bar = ctx->adj_body;
  a.vec = ctx->adj_vec; a.red = ctx->red; a.bar = ctx->bar; a.status = ctx->status;
  a.poison = ctx->poison; a.stats = ctx->stats; a.out = ctx->adj_out;
  // the barrier counter and the node-list length are zero between launches
  CU(cudaMemsetAsync(ctx->bar, 0, kBarWords * sizeof(unsigned), s));
  CU(cudaMemsetAsync(ctx->G.n_cnodes, 0, sizeof(int), s));
  CU(cudaMemsetAsync(ctx->adj_body, 0, kAdjBodySlots * kMaxBodies * sizeof(double), s));
  CU(cudaMemsetAsync(ctx->adj_out, 0, 4 * sizeof(float), s));
  CU(launch_adjoint(a, ctx->adj_blocks, s));
  CU(cudaMemsetAsync(ctx->bar, 0, kBarWords * sizeof(unsigned), s));
  CU(cudaMemsetAsync(ctx->G.n_cnodes, 0, sizeof(int), s));
  st = drain_status(ctx);
  float out[4];
  CU(cudaMemcpy(out, ctx->adj_out, sizeof(out), cudaMemcpyDeviceToHost));
  const int64_t nc = (int64_t)out[2];
  const int64_t k = nc < ccap ? nc : ccap;
  const cudaMemcpyKind back = mem_kind == MPM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (mem_kind == MPM_MEM_HOST) {
    if (n > 0) CU(cudaMemcpy(vstar_bar, d_vsb, 3 * n * sizeof(float), cudaMemcpyDeviceToHost));
    if (k > 0) CU(cudaMemcpy(contact_bar, d_cbar, 4 * k * sizeof(float), cudaMemcpyDeviceToHost));
  }
  if (body_bar && ctx->last_nb > 0) {
    // the first 7 of each body's accumulators
    CU(cudaMemcpy2DAsync(body_bar, 7 * sizeof(double), ctx->adj_body, kAdjBodySlots * sizeof(double),
                         7 * sizeof(double), ctx->last_nb, back, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
  }
  if (stats) {
    stats->iters = (int32_t)out[0];
    stats->residual = out[1];
    stats->contacts = (int32_t)out[2];
    stats->contact_nodes = (int32_t)out[3];
  }
  return st;
}

mpm_status mpm_tape_begin(mpm_ctx* ctx) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (!ctx->cloth_tris.empty())
    return fail(ctx, MPM_ERR_STATE, "mpm_tape_begin: the adjoints do not cover cloth");
  if (ctx->n_pins > 0)
    return fail(ctx, MPM_ERR_STATE, "mpm_tape_begin: the adjoints do not cover pinned particles");
  CU(cudaStreamSynchronize(ctx->stream));
  for (auto& t : ctx->tape)
    if (t.state) cudaFree(t.state);
  ctx->tape.clear();
  ctx->taping = true;
  ctx->tape_reset = false;
  ctx->tape_n = ctx->n;
  ctx->tape_substeps = 0;
  // the solution pool (MPM_OPT_TAPE_SOLUTIONS contact-node velocities, 256 MB
  // by default) and 1M substep records; without room the backward re-solves
  // from v* instead
  if (ctx->tape_pool && ctx->tape_pool_cap != ctx->tape_pool_want) {
    cudaFree(ctx->tape_pool);
    cudaFree(ctx->tape_recs);
    cudaFree(ctx->tape_counters);
    ctx->tape_pool = nullptr;
    ctx->tape_recs = nullptr;
    ctx->tape_counters = nullptr;
    ctx->tape_pool_cap = ctx->tape_rec_cap = 0;
  }
  if (!ctx->tape_pool && ctx->tape_pool_want > 0) {
    const int pool_cap = (int)ctx->tape_pool_want, rec_cap = 1 << 20;
    if (dalloc(&ctx->tape_pool, pool_cap) == cudaSuccess && dalloc(&ctx->tape_recs, rec_cap) == cudaSuccess &&
        dalloc(&ctx->tape_counters, 2) == cudaSuccess) {
      ctx->tape_pool_cap = pool_cap;
      ctx->tape_rec_cap = rec_cap;
    } else {
      cudaGetLastError();
      cudaFree(ctx->tape_pool);
      cudaFree(ctx->tape_recs);
      cudaFree(ctx->tape_counters);
      ctx->tape_pool = nullptr;
      ctx->tape_recs = nullptr;
      ctx->tape_counters = nullptr;
    }
  }
  if (ctx->tape_counters) CU(cudaMemsetAsync(ctx->tape_counters, 0, 2 * sizeof(int), ctx->stream));
  return MPM_OK;
}

mpm_status mpm_tape_end(mpm_ctx* ctx) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  ctx->taping = false;
  return MPM_OK;
}

namespace {

// state buffer (24 floats per particle, id order) -> particle buffer `cur`
void restore_state(mpm_ctx* ctx, const float* st, cudaStream_t s) {
  const size_t n = (size_t)ctx->n;
  launch_from_id_order(ctx->P[ctx->cur], (int)n, st, st + 3 * n, st + 6 * n, st + 15 * n, s);
  launch_stress_from_F(ctx->P[ctx->cur], (int)n, ctx->groups_d, s);
}

void save_state(mpm_ctx* ctx, float* st, cudaStream_t s) {
  const size_t n = (size_t)ctx->n;
  launch_to_id_order(ctx->P[ctx->cur], (int)n, st, st + 3 * n, st + 6 * n, st + 15 * n, s);
}

mpm_status ensure_adjoint_buffers(mpm_ctx* ctx) {
  if (ctx->adj_vec) return MPM_OK;
  CU(dalloc(&ctx->adj_vec, (size_t)kAdjointVectors * ctx->G.cnodes_cap));
  CU(dalloc(&ctx->adj_body, kAdjBodySlots * kMaxBodies));
  CU(dalloc(&ctx->adj_out, 4));
  int occ = 0;
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, adjoint_kernel_ptr(), solve_block_size(), 0));
  if (occ < 1) return fail(ctx, MPM_ERR_CUDA, "adjoint kernel does not fit an SM");
  ctx->adj_blocks = ctx->num_sms * (occ < 2 ? occ : 2);
  return MPM_OK;
}

}  // namespace

mpm_status mpm_backward(mpm_ctx* ctx, int32_t mem_kind, const float* x_bar, const float* v_bar,
                        const float* C_bar, const float* F_bar, const double* body_state_bar,
                        float* x0_bar, float* v0_bar, float* C0_bar, float* F0_bar,
                        double* material_bar, double* body_bar, const mpm_adjoint_params* params,
                        mpm_backward_stats* stats) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (mem_kind != MPM_MEM_HOST && mem_kind != MPM_MEM_DEVICE)
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_backward: bad mem_kind");
  // the replays overwrite the device's body table: keep the current bodies
  CU(sync_host_bodies(ctx));
  mpm_adjoint_params ap;
  ap.eps_r = 1e-6;
  ap.max_iters = 2000;
  if (params) ap = *params;
  if (!(ap.eps_r >= 0.0) || ap.max_iters < 0)
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_backward: bad parameters");
  if (ctx->tape.empty()) return fail(ctx, MPM_ERR_STATE, "mpm_backward: no recorded steps (mpm_tape_begin)");
  if (ctx->n != ctx->tape_n)
    return fail(ctx, MPM_ERR_STATE, "mpm_backward: the particle count changed since the tape began");
  // each recorded step must start from the state the previous one ended in
  if (ctx->tape_reset)
    return fail(ctx, MPM_ERR_STATE, "mpm_backward: particles or bodies were set between recorded steps");
  // every body keeps its kind (dynamic, kinematic, static) over the tape
  for (const auto& t : ctx->tape)
    for (size_t b = 0; b < t.bodies.size() && b < ctx->tape[0].bodies.size(); ++b)
      if (t.is_dyn[b] != ctx->tape[0].is_dyn[b] || t.kinematic[b] != ctx->tape[0].kinematic[b])
        return fail(ctx, MPM_ERR_STATE, "mpm_backward: a body changed kind within the tape");
  bool any_dyn = false;
  for (const auto& t : ctx->tape)
    for (int d : t.is_dyn) any_dyn = any_dyn || d;
  mpm_status st = drain_status(ctx);
  if (st != MPM_OK) return st;
  st = ensure_adjoint_buffers(ctx);
  if (st != MPM_OK) return st;
  cudaStream_t s = ctx->stream;
  const size_t n = (size_t)ctx->n;
  int max_sub = 1;
  for (const auto& t : ctx->tape) max_sub = t.n_substeps > max_sub ? t.n_substeps : max_sub;
  // scratch: two adjoint plane sets, the final state, the substep states
  const size_t per = 24 * n;
  const size_t need = per * (3 + (size_t)max_sub);
  if (ctx->bw_buf_cap < need) {
    if (ctx->bw_buf) cudaFree(ctx->bw_buf);
    ctx->bw_buf = nullptr;
    ctx->bw_buf_cap = 0;
    CU(dalloc(&ctx->bw_buf, need));
    ctx->bw_buf_cap = need;
  }
  if (!ctx->bw_gbar) CU(dalloc(&ctx->bw_gbar, ctx->n_nodes));
  if (!ctx->bw_slot) CU(dalloc(&ctx->bw_slot, ctx->cap));
  const size_t ng = ctx->groups.size();
  if (ctx->bw_mat_cap < 2 * ng + 2) {
    if (ctx->bw_mat) cudaFree(ctx->bw_mat);
    ctx->bw_mat = nullptr;
    ctx->bw_mat_cap = 0;
    CU(dalloc(&ctx->bw_mat, 2 * ng + 2));
    ctx->bw_mat_cap = 2 * ng + 2;
  }
  if (any_dyn && !ctx->bw_gbody) CU(dalloc(&ctx->bw_gbody, 6 * kMaxBodies));
  const size_t nsnap = ctx->tape.size() * kMaxBodies * kAdjBodySlots;
  if (ctx->bw_snap_cap < nsnap) {
    if (ctx->bw_snap) cudaFree(ctx->bw_snap);
    ctx->bw_snap = nullptr;
    ctx->bw_snap_cap = 0;
    CU(dalloc(&ctx->bw_snap, nsnap));
    ctx->bw_snap_cap = nsnap;
  }
  float* bar[2] = {ctx->bw_buf, ctx->bw_buf + per};
  float* final_state = ctx->bw_buf + 2 * per;
  float* sub_states = ctx->bw_buf + 3 * per;
  const Particles P = ctx->P[ctx->cur];
  // the replayed solves add to the impulse accumulators: keep the caller's
  std::vector<double> imp_saved(6 * kMaxBodies);
  CU(cudaMemcpyAsync(imp_saved.data(), ctx->impulses, 6 * kMaxBodies * sizeof(double),
                     cudaMemcpyDeviceToHost, s));
  // the adjoint of the final state, into planes in the current slot order
  save_state(ctx, final_state, s);
  launch_slot_map(P, (int)n, ctx->bw_slot, s);
  const float* src[4] = {x_bar, v_bar, C_bar, F_bar};
  const float* dsrc[4] = {x_bar, v_bar, C_bar, F_bar};
  const int width[4] = {3, 3, 9, 9};
  if (mem_kind == MPM_MEM_HOST) {
    size_t off = 0;
    for (int f = 0; f < 4; ++f) {
      dsrc[f] = nullptr;
      if (!src[f]) { off += n * width[f]; continue; }
      CU(cudaMemcpyAsync(ctx->stage + off, src[f], n * width[f] * sizeof(float), cudaMemcpyHostToDevice, s));
      dsrc[f] = ctx->stage + off;
      off += n * width[f];
    }
  }
  launch_bar_in(P, (int)n, dsrc[0], dsrc[1], dsrc[2], dsrc[3], bar[0], s);
  CU(cudaMemsetAsync(ctx->bw_mat, 0, (2 * ng + 2) * sizeof(double), s));
  CU(cudaMemsetAsync(ctx->adj_body, 0, kAdjBodySlots * kMaxBodies * sizeof(double), s));
  int in = 0;
  int substeps = 0;
  int nb_max = 0;
  // dynamic bodies: the adjoint of their state (v, p, omega, theta) after the
  // step being processed, carried back through each rigid step (Eq. (3))
  const int nb_final = (int)ctx->tape.back().bodies.size();
  std::vector<double> sbody(12 * kMaxBodies, 0.0), prev_snap(kMaxBodies * kAdjBodySlots, 0.0);
  if (body_state_bar)
    for (int i = 0; i < 12 * nb_final; ++i) sbody[i] = body_state_bar[i];
  for (int t = (int)ctx->tape.size() - 1; t >= 0; --t) {
    const mpm_ctx::TapeStep& T = ctx->tape[t];
    const int nb = (int)T.bodies.size();
    nb_max = nb > nb_max ? nb : nb_max;
    if (nb) CU(cudaMemcpyAsync(ctx->bodies_d, T.bodies.data(), nb * sizeof(DevBody), cudaMemcpyHostToDevice, s));
    bool step_dyn = false;
    for (int d : T.is_dyn) step_dyn = step_dyn || d;
    if (step_dyn) {
      std::vector<double> gb(6 * kMaxBodies, 0.0);
      const double dt = (double)T.n_substeps * (double)T.h;
      for (int b = 0; b < nb; ++b)
        if (T.is_dyn[b])
          integrate_dynamic_adjoint(T.bodies[b], T.dyn[b], ctx->spec.gravity, &T.imp[6 * b],
                                    &T.imp[6 * b + 3], dt, &sbody[12 * b], &gb[6 * b]);
      CU(cudaMemcpyAsync(ctx->bw_gbody, gb.data(), 6 * kMaxBodies * sizeof(double), cudaMemcpyHostToDevice, s));
      CU(cudaStreamSynchronize(s));
    }
    // replay the step from its checkpoint, keeping each substep's start state
    restore_state(ctx, T.state, s);
    // (each solve starts from the forward's taped solution of its substep,
    // when the pool held it, and stops at its first convergence test)
    auto rec_of = [&](int k) {
      return ctx->tape_pool && T.rec_base + k < ctx->tape_rec_cap ? T.rec_base + k : -1;
    };
    for (int k = 0; k + 1 < T.n_substeps; ++k) {
      save_state(ctx, sub_states + (size_t)k * per, s);
      CU(enqueue_substep(ctx, ctx->cur, nb, T.h, T.sp, ctx->solve_blocks, true, s, false, rec_of(k)));
    }
    save_state(ctx, sub_states + (size_t)(T.n_substeps - 1) * per, s);
    for (int k = T.n_substeps - 1; k >= 0; --k) {
      restore_state(ctx, sub_states + (size_t)k * per, s);
      CU(enqueue_substep(ctx, ctx->cur, nb, T.h, T.sp, ctx->solve_blocks, false, s, false, rec_of(k)));
      CU(cudaMemsetAsync(ctx->bw_gbar, 0, ctx->n_nodes * sizeof(float4), s));
      BackwardArgs ba;
      ba.g = ctx->g; ba.P = P; ba.n = (int)n; ba.groups = ctx->groups_d; ba.G = ctx->G;
      ba.h = T.h; ba.gbar = ctx->bw_gbar; ba.bin = bar[in]; ba.bout = bar[1 - in];
      ba.mat_bar = ctx->bw_mat; ba.status = ctx->status;
      launch_g2p_adjoint(ba, s);
      // contact solve (implicit differentiation) with the contact geometry
      AdjointArgs a;
      memset(&a, 0, sizeof(a));
      a.g = ctx->g; a.G = ctx->G; a.C = ctx->C; a.bodies = ctx->bodies_d; a.nb = nb;
      a.h = T.h; a.eps_s = T.sp.eps_s; a.eps_r = ap.eps_r; a.max_iters = ap.max_iters;
      a.n_in = 0; a.body_bar = ctx->adj_body; a.vec = ctx->adj_vec; a.red = ctx->red;
      a.bar = ctx->bar; a.status = ctx->status; a.poison = ctx->poison; a.stats = ctx->stats;
      a.out = ctx->adj_out; a.gbar = ctx->bw_gbar; a.pbar = bar[1 - in]; a.slot_of = ctx->bw_slot;
      a.P = P; a.n_particles = (int)n;
      a.body_gbar = step_dyn ? ctx->bw_gbody : nullptr;
      CU(cudaMemsetAsync(ctx->bar, 0, kBarWords * sizeof(unsigned), s));
      CU(cudaMemsetAsync(ctx->G.n_cnodes, 0, sizeof(int), s));
      CU(launch_adjoint(a, ctx->adj_blocks, s));
      launch_grid_adjoint(ba, ctx->num_sms, s);
      launch_p2g_adjoint(ba, s);
      launch_reset_counters(ctx->G, ctx->C, ctx->bar, s);
      CU(cudaGetLastError());
      in = 1 - in;
      ++substeps;
    }
    // the body accumulators so far (steps t .. end), to split them by step
    CU(cudaMemcpyAsync(ctx->bw_snap + (size_t)t * kMaxBodies * kAdjBodySlots, ctx->adj_body,
                       kMaxBodies * kAdjBodySlots * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (any_dyn) {
      // this step's contact terms complete the adjoint of the dynamic bodies'
      // state at its start: v (bias, lagged impulse), p, omega, theta
      std::vector<double> cur(kMaxBodies * kAdjBodySlots);
      CU(cudaMemcpyAsync(cur.data(), ctx->adj_body, cur.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      for (int b = 0; b < nb; ++b) {
        if (!T.is_dyn[b]) continue;
        auto D = [&](int k) { return cur[b * kAdjBodySlots + k] - prev_snap[b * kAdjBodySlots + k]; };
        for (int c = 0; c < 3; ++c) {
          sbody[12 * b + c] += D(c) + D(10 + c);
          sbody[12 * b + 3 + c] += D(7 + c);
          sbody[12 * b + 6 + c] += D(3 + c) + D(16 + c);
          sbody[12 * b + 9 + c] += D(13 + c);
        }
      }
      prev_snap = cur;
    }
  }
  // outputs: the adjoint of the first recorded state, in id order
  float* dst[4] = {x0_bar, v0_bar, C0_bar, F0_bar};
  float* ddst[4] = {x0_bar, v0_bar, C0_bar, F0_bar};
  if (mem_kind == MPM_MEM_HOST) {
    size_t off = 0;
    for (int f = 0; f < 4; ++f) {
      ddst[f] = dst[f] ? ctx->stage + off : nullptr;
      off += n * width[f];
    }
  }
  launch_bar_out(P, (int)n, bar[in], ddst[0], ddst[1], ddst[2], ddst[3], s);
  if (mem_kind == MPM_MEM_HOST)
    for (int f = 0; f < 4; ++f)
      if (dst[f]) CU(cudaMemcpyAsync(dst[f], ddst[f], n * width[f] * sizeof(float), cudaMemcpyDeviceToHost, s));
  std::vector<double> lame(2 * ng + 2), snap(nsnap);
  CU(cudaMemcpyAsync(lame.data(), ctx->bw_mat, (2 * ng + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(snap.data(), ctx->bw_snap, nsnap * sizeof(double), cudaMemcpyDeviceToHost, s));
  float out[4];
  CU(cudaMemcpyAsync(out, ctx->adj_out, sizeof(out), cudaMemcpyDeviceToHost, s));
  // put the state back as it was after the last step; the bodies upload again
  restore_state(ctx, final_state, s);
  ctx->bodies_dirty = true;
  ctx->adj_ready = false;  // the grid and contacts now hold a replayed substep
  st = drain_status(ctx);
  CU(cudaMemcpyAsync(ctx->impulses, imp_saved.data(), 6 * kMaxBodies * sizeof(double),
                     cudaMemcpyHostToDevice, s));
  CU(cudaStreamSynchronize(s));
  if (material_bar)
    for (size_t gi = 0; gi < ng; ++gi) {
      // mu = E / (2 (1 + nu)), lam = E nu / ((1 + nu)(1 - 2 nu))
      const double E = ctx->mats[gi].E, nu = ctx->mats[gi].nu;
      const double mub = lame[2 * gi], lamb = lame[2 * gi + 1];
      const double a = 1.0 + nu, b = 1.0 - 2.0 * nu;
      material_bar[2 * gi] = mub / (2.0 * a) + lamb * nu / (a * b);
      material_bar[2 * gi + 1] = -mub * E / (2.0 * a * a) + lamb * E * (1.0 + 2.0 * nu * nu) / (a * a * b * b);
    }
  if (body_bar) {
    // per body: dL/dmu; dL/dv = sum over steps of the direct terms (bias,
    // lagged normal impulse) plus, for a kinematic body, the position
    // adjoint of each step times the time its pose had advanced by then
    // (p_t = p_0 + sum_{t' < t} n_substeps h v); dL/dp_0 = sum of the
    // position adjoints
    const int T = (int)ctx->tape.size();
    auto S = [&](int t, int b, int k) {
      return t >= T ? 0.0 : snap[((size_t)t * kMaxBodies + b) * kAdjBodySlots + k];
    };
    // Orientation: a kinematic body's R_t = exp(T_t [omega]x) R_0 (T_t the
    // time advanced before step t), so a left rotation dtheta_t = J_l(T_t
    // omega) T_t domega + exp(T_t [omega]x) dtheta_0, with J_l the left
    // Jacobian of SO(3): dL/domega adds T_t J_l^T theta_bar_t, dL/dtheta_0 =
    // sum exp(-T_t [omega]x) theta_bar_t.
    for (int b = 0; b < nb_max; ++b) {
      double* o = body_bar + 13 * b;
      if (ctx->tape[0].is_dyn[b]) {
        // the recursion through the rigid steps gives the adjoint of the
        // first state directly
        o[0] = S(0, b, 6);
        for (int c = 0; c < 3; ++c) {
          o[1 + c] = sbody[12 * b + c];
          o[4 + c] = sbody[12 * b + 3 + c];
          o[7 + c] = sbody[12 * b + 6 + c];
          o[10 + c] = sbody[12 * b + 9 + c];
        }
        continue;
      }
      o[0] = S(0, b, 6);
      for (int c = 0; c < 3; ++c) {
        o[1 + c] = S(0, b, c) + S(0, b, 10 + c);
        o[4 + c] = S(0, b, 7 + c);
        o[7 + c] = S(0, b, 3 + c) + S(0, b, 16 + c);
        o[10 + c] = 0.0;
      }
      const double w[3] = {ctx->tape[0].bodies[b].w[0], ctx->tape[0].bodies[b].w[1],
                           ctx->tape[0].bodies[b].w[2]};
      double offset = 0.0;
      for (int t = 0; t < T; ++t) {
        const auto& tk = ctx->tape[t];
        if (b >= (int)tk.bodies.size()) break;
        double pb[3], rb[3];
        for (int c = 0; c < 3; ++c) {
          pb[c] = S(t, b, 7 + c) - S(t + 1, b, 7 + c);
          rb[c] = S(t, b, 13 + c) - S(t + 1, b, 13 + c);
          o[1 + c] += offset * pb[c];
        }
        const double ph[3] = {offset * w[0], offset * w[1], offset * w[2]};
        double jt[3], r0[3];
        jl_transpose(ph, rb, jt);
        rot_apply(ph, rb, -1.0, r0);
        for (int c = 0; c < 3; ++c) {
          o[7 + c] += offset * jt[c];
          o[10 + c] += r0[c];
        }
        if (tk.kinematic[b]) offset += (double)tk.n_substeps * (double)tk.h;
      }
      if (body_state_bar && b < nb_final) {
        // the final state: p_T = p_0 + T v, R_T = exp(T [omega]x) R_0 (T the
        // time a kinematic body advanced; 0 for a static one)
        const double* f = body_state_bar + 12 * b;
        const double ph[3] = {offset * w[0], offset * w[1], offset * w[2]};
        double jt[3], r0[3];
        jl_transpose(ph, f + 9, jt);
        rot_apply(ph, f + 9, -1.0, r0);
        for (int c = 0; c < 3; ++c) {
          o[1 + c] += f[c] + offset * f[3 + c];
          o[4 + c] += f[3 + c];
          o[7 + c] += f[6 + c] + offset * jt[c];
          o[10 + c] += r0[c];
        }
      }
    }
  }
  if (stats) {
    stats->steps = (int32_t)ctx->tape.size();
    stats->substeps = substeps;
    stats->last_iters = (int32_t)out[0];
    stats->last_residual = out[1];
  }
  return st;
}

mpm_status mpm_synchronize(mpm_ctx* ctx) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  return drain_status(ctx);
}

mpm_status mpm_set_option(mpm_ctx* ctx, int32_t option, int64_t value) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  switch (option) {
    case MPM_OPT_PROFILE:
      ctx->profile = value != 0;
      return MPM_OK;
    case MPM_OPT_SORT_EVERY:
      if (value < 1) return fail(ctx, MPM_ERR_INVALID_ARG, "sort interval must be >= 1");
      ctx->sort_every = (int)value;
      return MPM_OK;
    case MPM_OPT_P2G_CHUNK:
      if (value != 256 && value != 512 && value != 1024)
        return fail(ctx, MPM_ERR_INVALID_ARG, "P2G chunk must be 256, 512 or 1024");
      ctx->p2g_chunk = (int)value;
      return MPM_OK;
    case MPM_OPT_GRAPHS:
      ctx->use_graphs = value != 0;
      return MPM_OK;
    case MPM_OPT_P2G_FORM:
      if (value != MPM_P2G_GATHER && value != MPM_P2G_SCATTER)
        return fail(ctx, MPM_ERR_INVALID_ARG, "P2G form must be MPM_P2G_GATHER or MPM_P2G_SCATTER");
      ctx->p2g_form = (int)value;
      return MPM_OK;
    case MPM_OPT_TEST_BARRIER_TIMEOUT:
      ctx->wait_test = value != 0;
      return MPM_OK;
    case MPM_OPT_TAPE_SOLUTIONS:
      if (value < 0 || value > (1LL << 30))
        return fail(ctx, MPM_ERR_INVALID_ARG, "tape solution pool must hold 0 .. 2^30 entries");
      ctx->tape_pool_want = value;
      return MPM_OK;
    case MPM_OPT_CLUSTER_CONTACTS:
      if (value < 0 || value > (1 << 24))
        return fail(ctx, MPM_ERR_INVALID_ARG, "cluster contact limit must be 0 .. 2^24");
      ctx->cluster_max = (int)value;
      return MPM_OK;
    case MPM_OPT_CLUSTER_BLOCKS:
      if (value < 0 || value > ctx->cluster_blocks_max || (value & (value - 1)) != 0)
        return fail(ctx, MPM_ERR_INVALID_ARG,
                    "cluster blocks must be 0 or a power of two up to the device's largest cluster");
      ctx->cluster_blocks = value == 0 ? ctx->cluster_blocks_max : (int)value;
      return MPM_OK;
    case MPM_OPT_SOLVE_BLOCKS:
      if (value < 0) return fail(ctx, MPM_ERR_INVALID_ARG, "solve block cap must be >= 0");
      ctx->solve_blocks_cap = (int)(value > (1 << 20) ? (1 << 20) : value);
      return MPM_OK;
    default:
      return fail(ctx, MPM_ERR_INVALID_ARG, "unknown option");
  }
}

mpm_status mpm_get_phase_times(mpm_ctx* ctx, double* ms, int64_t* launches, int32_t reset) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  CU(cudaStreamSynchronize(ctx->stream));
  fold_events(ctx);
  for (int p = 0; p < MPM_NUM_PHASES; ++p) {
    if (ms) ms[p] = ctx->phase_ms[p];
    if (launches) launches[p] = ctx->phase_n[p];
    if (reset) {
      ctx->phase_ms[p] = 0.0;
      ctx->phase_n[p] = 0;
    }
  }
  return MPM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Grid readback that allocates nothing (no counterpart in the paper).
//
// mpm_get_grid compacts the last substep's grid into device buffers it
// allocates per call. Callers that must not allocate device memory use
// mpm_get_grid_noalloc instead: its compaction output lives in the file-scope
// array below, of a fixed maximum size, which every GPU that loads this
// library holds until the process exits.

namespace {

constexpr int kNoAllocMaxNodes = 1 << 18;  // 262,144 grid nodes
constexpr size_t kNoAllocHeader = 256;     // the node count, padded
constexpr size_t kNoAllocBytes = kNoAllocHeader + (size_t)kNoAllocMaxNodes * 4 * (1 + 1 + 3 + 3);
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_grid_readback[kNoAllocBytes];

// device address of g_grid_readback, looked up once per device
void* g_grid_readback_addr[kNoAllocMaxDevices] = {};

__global__ void k_grid_out_static(GridDev g, GridArrays G, int n_act, unsigned char* base) {
  int* count = reinterpret_cast<int*>(base);
  int* ids = reinterpret_cast<int*>(base + kNoAllocHeader);
  float* m = reinterpret_cast<float*>(ids + kNoAllocMaxNodes);
  float* vs = m + kNoAllocMaxNodes;
  float* v = vs + 3 * kNoAllocMaxNodes;
  const long long total = (long long)active_with_storage(g, n_act) * kBlockNodes;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int blk = G.act[t >> 6], cell = (int)(t & 63);
    const int node = active_storage_block(g, G.act, (int)(t >> 6)) * kBlockNodes + cell;
    const float4 a = G.vs[node];
    if (!(a.w > 0.f)) continue;
    const float4 b = G.v[node];
    const int bx = blk % g.nbx, by = (blk / g.nbx) % g.nby, bz = blk / (g.nbx * g.nby);
    const int i = bx * 4 + (cell & 3), j = by * 4 + ((cell >> 2) & 3), k = bz * 4 + (cell >> 4);
    const int slot = atomicAdd(count, 1);
    if (slot >= kNoAllocMaxNodes) continue;
    ids[slot] = i + g.rx * (j + g.ry * k);
    m[slot] = a.w;
    vs[3 * slot] = a.x; vs[3 * slot + 1] = a.y; vs[3 * slot + 2] = a.z;
    v[3 * slot] = b.x; v[3 * slot + 1] = b.y; v[3 * slot + 2] = b.z;
  }
}

}  // namespace

extern "C" mpm_status mpm_get_grid_noalloc(mpm_ctx* ctx, int64_t cap, int64_t* count,
                                           int32_t* node_ids, float* m, float* vstar, float* v) {
  if (!ctx || !count || cap < 0) return MPM_ERR_INVALID_ARG;
  int dev = -1;
  CU(cudaGetDevice(&dev));
  if (dev != ctx->device)
    return fail(ctx, MPM_ERR_INVALID_ARG,
                "mpm_get_grid_noalloc: make the context's device current before the call");
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return fail(ctx, MPM_ERR_INVALID_ARG, "mpm_get_grid_noalloc: device index out of range");
  if (!g_grid_readback_addr[dev]) {
    void* p = nullptr;
    CU(cudaGetSymbolAddress(&p, g_grid_readback));
    g_grid_readback_addr[dev] = p;
  }
  unsigned char* base = static_cast<unsigned char*>(g_grid_readback_addr[dev]);
  CU(cudaStreamSynchronize(ctx->stream));
  DevStats ds;
  CU(cudaMemcpy(&ds, ctx->stats, sizeof(ds), cudaMemcpyDeviceToHost));
  const int n_act = ds.last_active;
  if ((long long)n_act * kBlockNodes > kNoAllocMaxNodes)
    return fail(ctx, MPM_ERR_CAPACITY,
                "mpm_get_grid_noalloc: the last substep swept more than 262144 grid nodes "
                "(4096 blocks of 4^3); use mpm_get_grid");
  // the array keeps the previous call's contents: the node count starts at zero
  CU(cudaMemsetAsync(base, 0, sizeof(int), ctx->stream));
  if (n_act > 0)
    k_grid_out_static<<<ctx->num_sms * 4, 256, 0, ctx->stream>>>(ctx->g, ctx->G, n_act, base);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(ctx->stream));
  int got = 0;
  CU(cudaMemcpy(&got, base, sizeof(int), cudaMemcpyDeviceToHost));
  got = got < kNoAllocMaxNodes ? got : kNoAllocMaxNodes;
  *count = got;
  const size_t k = (size_t)(got < cap ? got : cap);
  if (k > 0) {
    const unsigned char* ids = base + kNoAllocHeader;
    const unsigned char* mm = ids + (size_t)kNoAllocMaxNodes * 4;
    const unsigned char* vs = mm + (size_t)kNoAllocMaxNodes * 4;
    const unsigned char* vv = vs + (size_t)kNoAllocMaxNodes * 12;
    if (node_ids) CU(cudaMemcpy(node_ids, ids, k * 4, cudaMemcpyDeviceToHost));
    if (m) CU(cudaMemcpy(m, mm, k * 4, cudaMemcpyDeviceToHost));
    if (vstar) CU(cudaMemcpy(vstar, vs, k * 12, cudaMemcpyDeviceToHost));
    if (v) CU(cudaMemcpy(v, vv, k * 12, cudaMemcpyDeviceToHost));
  }
  return MPM_OK;
}
