// cloth.cu -- cloth as a triangle mesh of MPM particles (the paper's cloth
// results, Sec. VI): the mesh's in-plane elasticity is a Lagrangian force on
// the vertex particles, the corotated membrane energy per triangle
//   psi(F) = mu |F - R|^2 + lam/2 (J - 1)^2,  F = Ds Dm^-1 (3x2),
// R the polar factor of F (F = R S, S = sqrt(F^T F)), J = det S, times the
// triangle's rest volume (rest area times the cloth's thickness). The forces
// f = -dE/dx are recomputed at the start of every substep and P2G adds h f
// to the vertices' momentum (and leaves the force planes zero); the vertices
// carry no stress of their own and collide (with bodies, with the cloth
// itself, with other material) through the grid and the contact solve.
//
// One thread per triangle in FP64 (a few hundred operations: near rest
// F - R is a small difference of O(1) terms, which FP32 would leave with a
// relative error of 1e-4), its three forces added to the vertices' force
// planes with FP32 atomics.
//
// Pinned particles (the held cloth corners of the same experiment): a
// Dirichlet condition on the particle. A pinned particle enters every
// substep with its prescribed velocity and C = 0 (its start position kept:
// taken from the particle at a step's first substep, carried between
// substeps), the mesh forces on it are dropped, and after G2P it is put back
// on its path, x = x_start + h v_pin (F follows G2P). One thread per pin,
// through the id -> slot map.
#include <cmath>

#include "kernels.h"

namespace mpmcr {

namespace {

__global__ void k_cloth_forces(Particles P, const int* __restrict__ slot_of,
                               const int4* __restrict__ tris, const double* __restrict__ rest,
                               int n_tris, const DevGroup* __restrict__ groups,
                               const uint8_t* __restrict__ pinned, float* __restrict__ f,
                               long long stride) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tris) return;
  const int4 tv = tris[t];
  const int sl[3] = {slot_of[tv.x], slot_of[tv.y], slot_of[tv.z]};
  double x[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) x[k][c] = (double)P.x(c)[sl[k]];
  const double* r = rest + 5 * (size_t)t;  // Dm^-1 (2x2 row-major), rest volume
  const double dmi[4] = {r[0], r[1], r[2], r[3]};
  const double vol = r[4];
  const DevGroup gr = groups[tv.w];
  const double mu = (double)gr.mu_l, lam = (double)gr.lam;
  double F[3][2];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double d1 = x[1][c] - x[0][c], d2 = x[2][c] - x[0][c];
    F[c][0] = d1 * dmi[0] + d2 * dmi[2];
    F[c][1] = d1 * dmi[1] + d2 * dmi[3];
  }
  // C = F^T F; S = sqrt(C) = (C + sqrt(det C) I) / sqrt(tr C + 2 sqrt(det C))
  const double c00 = F[0][0] * F[0][0] + F[1][0] * F[1][0] + F[2][0] * F[2][0];
  const double c01 = F[0][0] * F[0][1] + F[1][0] * F[1][1] + F[2][0] * F[2][1];
  const double c11 = F[0][1] * F[0][1] + F[1][1] * F[1][1] + F[2][1] * F[2][1];
  const double detC = c00 * c11 - c01 * c01;
  if (!(detC > 1e-30)) return;  // a collapsed triangle exerts no force
  const double J = sqrt(detC);
  const double tn = sqrt(c00 + c11 + 2.0 * J);
  const double s00 = (c00 + J) / tn, s01 = c01 / tn, s11 = (c11 + J) / tn;
  // R = F S^-1 (det S = J); P = 2 mu (F - R) + lam (J - 1) J F C^-1
  const double si00 = s11 / J, si01 = -s01 / J, si11 = s00 / J;
  const double ci00 = c11 / detC, ci01 = -c01 / detC, ci11 = c00 / detC;
  const double kl = lam * (J - 1.0) * J;
  double g[3][2];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double r0 = F[c][0] * si00 + F[c][1] * si01, r1 = F[c][0] * si01 + F[c][1] * si11;
    const double p0 = 2.0 * mu * (F[c][0] - r0) + kl * (F[c][0] * ci00 + F[c][1] * ci01);
    const double p1 = 2.0 * mu * (F[c][1] - r1) + kl * (F[c][0] * ci01 + F[c][1] * ci11);
    // dE/dDs = vol P Dm^-T
    g[c][0] = vol * (p0 * dmi[0] + p1 * dmi[1]);
    g[c][1] = vol * (p0 * dmi[2] + p1 * dmi[3]);
  }
  // a pinned vertex is held: the mesh does not push it
  const bool hold[3] = {pinned && pinned[tv.x], pinned && pinned[tv.y], pinned && pinned[tv.z]};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float* fc = f + (size_t)c * stride;
    if (!hold[0]) atomicAdd(fc + sl[0], (float)(g[c][0] + g[c][1]));
    if (!hold[1]) atomicAdd(fc + sl[1], (float)(-g[c][0]));
    if (!hold[2]) atomicAdd(fc + sl[2], (float)(-g[c][1]));
  }
}

__global__ void k_pin_init(Particles P, const int* __restrict__ slot_of, const int* __restrict__ ids,
                           const float* __restrict__ v_pin, float* __restrict__ x_pin, int n_pins,
                           int cap) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_pins) return;
  const int sl = slot_of[ids[j]];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    x_pin[j + c * cap] = P.x(c)[sl];
    P.v(c)[sl] = v_pin[j + c * cap];
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) P.C(c)[sl] = 0.f;
}

__global__ void k_pins(Particles P, const int* __restrict__ slot_of, const int* __restrict__ ids,
                       const float* __restrict__ v_pin, float* __restrict__ x_pin, int n_pins,
                       int cap, float h) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_pins) return;
  const int sl = slot_of[ids[j]];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float vp = v_pin[j + c * cap];
    const float xp = fmaf(h, vp, x_pin[j + c * cap]);
    P.x(c)[sl] = xp;
    x_pin[j + c * cap] = xp;  // the next substep's start
    P.v(c)[sl] = vp;
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) P.C(c)[sl] = 0.f;
}

}  // namespace

void cloth_rest_shape(const double X0[3], const double X1[3], const double X2[3], double out[5]) {
  // the rest edges in the triangle's own frame (t1 along the first edge, t2
  // in its plane): Dm = [[|e1|, e2.t1], [0, e2.t2]], inverted; then the area
  double e1[3], e2[3];
  for (int a = 0; a < 3; ++a) {
    e1[a] = X1[a] - X0[a];
    e2[a] = X2[a] - X0[a];
  }
  const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                       e1[0] * e2[1] - e1[1] * e2[0]};
  const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  const double l1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  const double t1[3] = {e1[0] / l1, e1[1] / l1, e1[2] / l1};
  const double u[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
  const double t2[3] = {u[1] * t1[2] - u[2] * t1[1], u[2] * t1[0] - u[0] * t1[2],
                        u[0] * t1[1] - u[1] * t1[0]};
  const double a00 = l1, a01 = e2[0] * t1[0] + e2[1] * t1[1] + e2[2] * t1[2];
  const double a11 = e2[0] * t2[0] + e2[1] * t2[1] + e2[2] * t2[2];
  out[0] = 1.0 / a00;
  out[1] = -a01 / (a00 * a11);
  out[2] = 0.0;
  out[3] = 1.0 / a11;
  out[4] = 0.5 * nn;
}

void launch_cloth_forces(const Particles& P, const int* slot_of, const int4* tris,
                         const double* rest, int n_tris, const DevGroup* groups,
                         const uint8_t* pinned, float* f, long long stride, cudaStream_t s) {
  // one warp per block: a mesh of a few thousand triangles then spreads over
  // as many SMs as it has warps, since each SM's FP64 pipe is narrow
  if (n_tris > 0)
    k_cloth_forces<<<(n_tris + 31) / 32, 32, 0, s>>>(P, slot_of, tris, rest, n_tris, groups,
                                                      pinned, f, stride);
}

void launch_pin_init(const Particles& P, const int* slot_of, const int* ids, const float* v_pin,
                     float* x_pin, int n_pins, int cap, cudaStream_t s) {
  if (n_pins > 0)
    k_pin_init<<<(n_pins + 127) / 128, 128, 0, s>>>(P, slot_of, ids, v_pin, x_pin, n_pins, cap);
}

void launch_pins(const Particles& P, const int* slot_of, const int* ids, const float* v_pin,
                 float* x_pin, int n_pins, int cap, float h, cudaStream_t s) {
  if (n_pins > 0)
    k_pins<<<(n_pins + 127) / 128, 128, 0, s>>>(P, slot_of, ids, v_pin, x_pin, n_pins, cap, h);
}

}  // namespace mpmcr
