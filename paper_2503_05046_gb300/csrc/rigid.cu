// rigid.cu -- the rigid bodies' update between two time steps of the
// asynchronous splitting (Sec. IV-A, Eq. (3)-(4)), on the device, so that a
// step with moving bodies needs no host round trip and replays as one graph.
//
// One warp per body (FP64). A kinematic body advances with its frozen
// velocity: p += dt v, R <- exp(dt [omega]x) R. A dynamic body takes Eq. (3)
// without rigid-rigid contact, semi-implicit Euler with the impulse J and
// moment L that the step's contact solves put on it (the accumulator now
// minus its value at the step's start):
//   m (v+ - v) = dt (f + m g) + J,
//   I (w+ - w) = dt (tau - w x I w) + L,   I = R diag(I_b) R^T,
// then the locked degrees of freedom are zeroed and the pose advances with
// (v+, w+). The 3x3 block is dense: lanes 0-8 form the world inertia's
// entries, lanes 0-2 its cofactor rows, and the solve is shared through the
// warp.
//
// A batch of scenes runs the update for all of them in one launch (one block
// per scene, one warp per body), with the step's bookkeeping around it.
#include "kernels.h"

namespace mpmcr {

namespace {

__device__ __forceinline__ double shfl_d(double x, int src) {
  return __shfl_sync(0xffffffffu, x, src);
}

// R <- exp([ph]x) R (Rodrigues), p <- p + dt v in the caller
__device__ void rotate_left(const double (&ph)[3], double (&R)[9]) {
  const double th = sqrt(ph[0] * ph[0] + ph[1] * ph[1] + ph[2] * ph[2]);
  if (th == 0.0) return;
  const double a[3] = {ph[0] / th, ph[1] / th, ph[2] / th};
  const double c = cos(th), s = sin(th), t = 1.0 - c;
  const double Q[9] = {c + t * a[0] * a[0],        t * a[0] * a[1] - s * a[2], t * a[0] * a[2] + s * a[1],
                       t * a[1] * a[0] + s * a[2], c + t * a[1] * a[1],        t * a[1] * a[2] - s * a[0],
                       t * a[2] * a[0] - s * a[1], t * a[2] * a[1] + s * a[0], c + t * a[2] * a[2]};
  double O[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int cc = 0; cc < 3; ++cc)
      O[3 * r + cc] = Q[3 * r] * R[cc] + Q[3 * r + 1] * R[3 + cc] + Q[3 * r + 2] * R[6 + cc];
#pragma unroll
  for (int i = 0; i < 9; ++i) R[i] = O[i];
}

// Body b's update by one warp.
__device__ void rigid_update_warp(DevBody* bodies, const DevDyn* dyn, int b, const double* imp,
                                  const double* imp0, double dt, double gx, double gy, double gz) {
  const int lane = threadIdx.x & 31;
  const DevDyn d = dyn[b];
  if (d.kind == kRigidStatic) return;
  DevBody& B = bodies[b];
  double R[9], v[3], w[3], p[3];
#pragma unroll
  for (int i = 0; i < 9; ++i) R[i] = B.R[i];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    v[i] = B.v[i];
    w[i] = B.w[i];
    p[i] = B.p[i];
  }
  if (d.kind == kRigidDynamic) {
    const double g[3] = {gx, gy, gz};
    double J[3], L[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      J[i] = imp[6 * b + i] - imp0[6 * b + i];
      L[i] = imp[6 * b + 3 + i] - imp0[6 * b + 3 + i];
      const double f = (double)d.force[i] + (d.gravity ? (double)d.mass * g[i] : 0.0);
      v[i] += (dt * f + J[i]) / (double)d.mass;
    }
    // world inertia, entry (r, c) on lane 3 r + c
    const int e = lane < 9 ? lane : 0, r = e / 3, c = e % 3;
    double Ie = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) Ie += R[3 * r + k] * (double)d.inertia[k] * R[3 * c + k];
    double Iw[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Iw[k] = shfl_d(Ie, k);
    // right-hand side dt (tau - w x I w) + L
    double Iww[3], rhs[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) Iww[i] = Iw[3 * i] * w[0] + Iw[3 * i + 1] * w[1] + Iw[3 * i + 2] * w[2];
    const double gyro[3] = {w[1] * Iww[2] - w[2] * Iww[1], w[2] * Iww[0] - w[0] * Iww[2],
                            w[0] * Iww[1] - w[1] * Iww[0]};
#pragma unroll
    for (int i = 0; i < 3; ++i) rhs[i] = dt * ((double)d.torque[i] - gyro[i]) + L[i];
    // cofactor row i on lane i (I is symmetric: the adjugate's row i is its
    // column), then dw = adj(I) rhs / det(I)
    const int i = lane < 3 ? lane : 0, i1 = (i + 1) % 3, i2 = (i + 2) % 3;
    double cof[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      cof[j] = Iw[3 * i1 + j1] * Iw[3 * i2 + j2] - Iw[3 * i1 + j2] * Iw[3 * i2 + j1];
    }
    const double row = cof[0] * rhs[0] + cof[1] * rhs[1] + cof[2] * rhs[2];
    const double det0 = Iw[0] * cof[0] + Iw[1] * cof[1] + Iw[2] * cof[2];  // lane 0: row 0 expansion
    const double det = shfl_d(det0, 0);
    double dw[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) dw[k] = shfl_d(row, k) / det;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      w[k] += dw[k];
      if (!((d.dof_mask >> k) & 1)) v[k] = 0.0;
      if (!((d.dof_mask >> (3 + k)) & 1)) w[k] = 0.0;
    }
  }
  // the pose advances with the velocities as stored (FP32)
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    v[k] = (double)(float)v[k];
    w[k] = (double)(float)w[k];
  }
  const double ph[3] = {dt * w[0], dt * w[1], dt * w[2]};
  rotate_left(ph, R);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 9; ++k) B.R[k] = (float)R[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      B.p[k] = (float)(p[k] + dt * v[k]);
      B.v[k] = (float)v[k];
      B.w[k] = (float)w[k];
    }
  }
}

__global__ void k_rigid_update(DevBody* bodies, const DevDyn* dyn, int nb, const double* imp,
                               const double* imp0, double dt, double gx, double gy, double gz) {
  const int b = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (b < nb) rigid_update_warp(bodies, dyn, b, imp, imp0, dt, gx, gy, gz);
}

// Batched, block s for scene s: the step's start (its statistics cleared,
// the impulse accumulator noted) ...
__global__ void k_batch_begin(const RigidBatchArgs* __restrict__ args) {
  const RigidBatchArgs& a = args[blockIdx.x];
  for (int i = threadIdx.x; i < (int)(sizeof(DevStats) / 4); i += blockDim.x)
    reinterpret_cast<int*>(a.stats)[i] = 0;
  for (int i = threadIdx.x; i < 6 * a.nb; i += blockDim.x) a.imp0[i] = a.imp[i];
}

// ... and its end: one warp per body moves the bodies, and the scene's
// status word and statistics are gathered into the batch's arrays
__global__ void k_batch_end(const RigidBatchArgs* __restrict__ args, double dt,
                            uint32_t* __restrict__ status_out, DevStats* __restrict__ stats_out) {
  const RigidBatchArgs& a = args[blockIdx.x];
  if (threadIdx.x == 0) status_out[blockIdx.x] = *a.status;
  for (int i = threadIdx.x; i < (int)(sizeof(DevStats) / 4); i += blockDim.x)
    reinterpret_cast<int*>(stats_out + blockIdx.x)[i] = reinterpret_cast<const int*>(a.stats)[i];
  const int b = (int)(threadIdx.x >> 5);
  if (a.rigid && b < a.nb)
    rigid_update_warp(a.bodies, a.dyn, b, a.imp, a.imp0, dt, a.gravity[0], a.gravity[1],
                      a.gravity[2]);
}

}  // namespace

void launch_batch_begin(const RigidBatchArgs* args, int n_scenes, cudaStream_t s) {
  if (n_scenes > 0) k_batch_begin<<<n_scenes, 128, 0, s>>>(args);
}

void launch_batch_end(const RigidBatchArgs* args, int n_scenes, double dt, uint32_t* status_out,
                      DevStats* stats_out, cudaStream_t s) {
  if (n_scenes > 0)
    k_batch_end<<<n_scenes, 32 * kMaxBodies, 0, s>>>(args, dt, status_out, stats_out);
}

void launch_rigid_update(DevBody* bodies, const DevDyn* dyn, int nb, const double* imp,
                         const double* imp0, double dt, const double* gravity, cudaStream_t s) {
  if (nb <= 0) return;
  k_rigid_update<<<1, 32 * nb, 0, s>>>(bodies, dyn, nb, imp, imp0, dt, gravity[0], gravity[1],
                                       gravity[2]);
}

}  // namespace mpmcr
