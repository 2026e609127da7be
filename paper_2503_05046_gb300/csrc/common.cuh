// common.cuh -- device-side data layout and per-particle / per-contact math of
// the sm_103a MPM-rigid convex-contact substep (Yu et al., arXiv 2503.05046).
//
// Everything here is FP32 and written for one thread per particle or per
// contact. Grid nodes live in a dense block-major address space: node
// (i, j, k) is in 4^3 block (i>>2, j>>2, k>>2) and has index
// block * 64 + (k & 3) * 16 + (j & 3) * 4 + (i & 3), so a block is 64
// consecutive nodes and only blocks touched by particles are ever swept.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mpmcr.h"

namespace mpmcr {

constexpr int kMaxBodies = 16;
constexpr int kBlockNodes = 64;

// Device status bits (1 << mpm_status).
constexpr uint32_t kStOutOfDomain = 1u << MPM_ERR_OUT_OF_DOMAIN;
constexpr uint32_t kStCapacity = 1u << MPM_ERR_CAPACITY;
constexpr uint32_t kStNotConverged = 1u << MPM_ERR_NOT_CONVERGED;
constexpr uint32_t kStNan = 1u << MPM_ERR_NAN;
constexpr uint32_t kStTimeout = 1u << MPM_ERR_TIMEOUT;
constexpr uint32_t kStLineSearch = 1u << MPM_ERR_LINE_SEARCH;

struct GridDev {
  float dx, inv_dx;
  float ox, oy, oz;       // origin
  float gx, gy, gz;       // gravity
  int rx, ry, rz;         // nodes per axis
  int nbx, nby, nbz;      // 4^3 blocks per axis
  int bc;                 // Dirichlet layers
  int morton_bits;        // bits per axis of the block sort key
};

// Rigid body frozen for a time step (Eq. (3)-(4)); 32 words.
struct DevBody {
  int shape;
  float prm[4];
  float R[9];
  float p[3];
  float w[3];
  float v[3];
  float mu, k, d;
  float bound;  // radius of a sphere around p holding the geometry (inf: unbounded)
  int pad[5];
};
static_assert(sizeof(DevBody) == 32 * 4, "DevBody layout");

// Per particle-group constants.
struct DevGroup {
  float vol, mass;        // rest volume, mass
  float mu_l, lam;        // Lame parameters
  float dp_alpha;         // Drucker-Prager cone slope
  int model;
  float pad[2];
};

// Particle state, structure of arrays (one float plane per component).
struct Particles {
  float* x[3];
  float* v[3];
  float* C[9];
  float* F[9];
  uint32_t* pid;    // particle id (order of addition)
  uint16_t* grp;    // particle group
};

// Grid node arrays (dense, block-major).
struct GridArrays {
  float4* mp;      // (m, p): P2G accumulator, all zero outside a substep
  float4* vs;      // (v*, m)
  float4* v;       // current grid velocity, .w unused
  float4* acc0;    // contact terms of the solve: (g_x, g_y, g_z, H_xx), zero outside use
  float4* acc1;    // (H_yy, H_zz, H_xy, H_xz)
  float* acc2;     // H_yz
  float4* dv;      // search direction
  uint8_t* mark;   // per block: touched by P2G this substep (zero outside)
  int* act;        // active block list
  int* n_act;      // its length (device)
};

// Contact points (Sec. V-B), structure of arrays.
struct Contacts {
  float4* xp;      // particle position, phi0
  float4* nrm;     // contact normal (world), lagged normal impulse n0
  float4* bias;    // -v_rigid(x_p) (world), unused
  int2* id;        // (particle id, body)
  float4* vc;      // relative contact velocity (world) during the solve
  float4* dvc;     // its search direction
  float4* gamma;   // impulse on the particle at the solution (world)
  int* count;
  int cap;
};

// --------------------------------------------------------------------------
// small helpers

__device__ __forceinline__ void red_add_v4(float4* addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b),
               "f"(c), "f"(d)
               : "memory");
}

__device__ __forceinline__ void red_add_f32(float* addr, float a) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(addr), "f"(a) : "memory");
}

__device__ __forceinline__ int node_index(const GridDev& g, int i, int j, int k) {
  int b = ((k >> 2) * g.nby + (j >> 2)) * g.nbx + (i >> 2);
  return b * kBlockNodes + ((k & 3) << 4) + ((j & 3) << 2) + (i & 3);
}

__device__ __forceinline__ uint32_t spread_bits3(uint32_t v) {
  // insert two zero bits between the low 10 bits of v
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Quadratic B-spline stencil of the MLS-MPM transfers (free motion, Eq. (6)).
struct Stencil {
  int base[3];
  float fx[3];
  float w[3][3];
};

__device__ __forceinline__ void stencil(const GridDev& g, float x, float y, float z,
                                        Stencil& s) {
  float xi[3] = {(x - g.ox) * g.inv_dx, (y - g.oy) * g.inv_dx, (z - g.oz) * g.inv_dx};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float b = floorf(xi[a] - 0.5f);
    s.base[a] = (int)b;
    float f = xi[a] - b;
    s.fx[a] = f;
    float t0 = 1.5f - f, t1 = f - 1.0f, t2 = f - 0.5f;
    s.w[a][0] = 0.5f * t0 * t0;
    s.w[a][1] = 0.75f - t1 * t1;
    s.w[a][2] = 0.5f * t2 * t2;
  }
}

__device__ __forceinline__ bool stencil_inside(const GridDev& g, const Stencil& s) {
  return s.base[0] >= 0 && s.base[1] >= 0 && s.base[2] >= 0 && s.base[0] + 2 < g.rx &&
         s.base[1] + 2 < g.ry && s.base[2] + 2 < g.rz;
}

// --------------------------------------------------------------------------
// 3x3 SVD, F = U diag(S) V^T with U, V proper rotations and S[2] < 0 iff
// det F < 0. Cyclic Jacobi on the symmetric F^T F gives V; the columns of
// F V are ordered by length and an orthogonal-triangular factorisation by
// Givens rotations gives U and the singular values (McAdams et al. 2011,
// "Computing the singular value decomposition of 3x3 matrices with minimal
// branching", with exact rather than approximate rotations).

__device__ __forceinline__ void jacobi_pair(float& app, float& aqq, float& apq, float& arp,
                                            float& arq, float (&V)[9], int p, int q) {
  if (apq == 0.0f) return;
  float theta = (aqq - app) / (2.0f * apq);
  float t = copysignf(1.0f, theta) / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.0f)));
  float c = rsqrtf(fmaf(t, t, 1.0f));
  float s = t * c;
  app = app - t * apq;
  aqq = aqq + t * apq;
  apq = 0.0f;
  float rp = arp, rq = arq;
  arp = c * rp - s * rq;
  arq = s * rp + c * rq;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    float vp = V[3 * r + p], vq = V[3 * r + q];
    V[3 * r + p] = c * vp - s * vq;
    V[3 * r + q] = s * vp + c * vq;
  }
}

__device__ __forceinline__ void givens_rows(float (&B)[9], float (&U)[9], int i, int k, int j) {
  float a = B[3 * i + j], b = B[3 * k + j];
  float r2 = a * a + b * b;
  if (r2 == 0.0f) return;
  float inv = rsqrtf(r2);
  float c = a * inv, s = b * inv;
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    float bi = B[3 * i + m], bk = B[3 * k + m];
    B[3 * i + m] = c * bi + s * bk;
    B[3 * k + m] = -s * bi + c * bk;
    float ui = U[3 * m + i], uk = U[3 * m + k];
    U[3 * m + i] = c * ui + s * uk;
    U[3 * m + k] = -s * ui + c * uk;
  }
}

__device__ __forceinline__ void svd3(const float (&F)[9], float (&U)[9], float (&S)[3],
                                     float (&V)[9]) {
  // A = F^T F
  float a00 = F[0] * F[0] + F[3] * F[3] + F[6] * F[6];
  float a11 = F[1] * F[1] + F[4] * F[4] + F[7] * F[7];
  float a22 = F[2] * F[2] + F[5] * F[5] + F[8] * F[8];
  float a01 = F[0] * F[1] + F[3] * F[4] + F[6] * F[7];
  float a02 = F[0] * F[2] + F[3] * F[5] + F[6] * F[8];
  float a12 = F[1] * F[2] + F[4] * F[5] + F[7] * F[8];
#pragma unroll
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0f : 0.0f;
#pragma unroll 1
  for (int sweep = 0; sweep < 6; ++sweep) {
    jacobi_pair(a00, a11, a01, a02, a12, V, 0, 1);  // r = 2
    jacobi_pair(a00, a22, a02, a01, a12, V, 0, 2);  // r = 1
    jacobi_pair(a11, a22, a12, a01, a02, V, 1, 2);  // r = 0
  }
  // B = F V
  float B[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      B[3 * r + c] = F[3 * r] * V[c] + F[3 * r + 1] * V[3 + c] + F[3 * r + 2] * V[6 + c];
  // order columns by decreasing length; each swap negates one column so V
  // stays a rotation
  auto col2 = [&](int c) { return B[c] * B[c] + B[3 + c] * B[3 + c] + B[6 + c] * B[6 + c]; };
  auto swapneg = [&](int c0, int c1) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      float t = B[3 * r + c0];
      B[3 * r + c0] = -B[3 * r + c1];
      B[3 * r + c1] = t;
      t = V[3 * r + c0];
      V[3 * r + c0] = -V[3 * r + c1];
      V[3 * r + c1] = t;
    }
  };
  float l0 = col2(0), l1 = col2(1), l2 = col2(2);
  if (l0 < l1) { swapneg(0, 1); float t = l0; l0 = l1; l1 = t; }
  if (l0 < l2) { swapneg(0, 2); float t = l0; l0 = l2; l2 = t; }
  if (l1 < l2) { swapneg(1, 2); }
#pragma unroll
  for (int i = 0; i < 9; ++i) U[i] = (i % 4 == 0) ? 1.0f : 0.0f;
  givens_rows(B, U, 0, 1, 0);
  givens_rows(B, U, 0, 2, 0);
  givens_rows(B, U, 1, 2, 1);
  S[0] = B[0];
  S[1] = B[4];
  S[2] = B[8];
}

__device__ __forceinline__ float det3(const float (&A)[9]) {
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}

constexpr float kHenckySigmaMin = 1e-4f;

// Kirchhoff stress tau = P(F) F^T (symmetric, 6 entries xx yy zz xy xz yz).
__device__ __forceinline__ void kirchhoff(const DevGroup& gr, const float (&F)[9], float (&t)[6]) {
  float U[9], S[3], V[9];
  svd3(F, U, S, V);
  if (gr.model == MPM_DRUCKER_PRAGER) {
    // Hencky: tau = U diag(2 mu e + lam tr e) U^T, e = log S
    float e[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) e[a] = logf(fmaxf(S[a], kHenckySigmaMin));
    float tr = e[0] + e[1] + e[2];
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = 2.0f * gr.mu_l * e[a] + gr.lam * tr;
    auto ent = [&](int r, int c) {
      return U[3 * r] * d[0] * U[3 * c] + U[3 * r + 1] * d[1] * U[3 * c + 1] +
             U[3 * r + 2] * d[2] * U[3 * c + 2];
    };
    t[0] = ent(0, 0); t[1] = ent(1, 1); t[2] = ent(2, 2);
    t[3] = ent(0, 1); t[4] = ent(0, 2); t[5] = ent(1, 2);
  } else {
    // fixed corotated: tau = 2 mu (F - R) F^T + lam J (J - 1) I, R = U V^T
    float R[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        R[3 * r + c] = U[3 * r] * V[3 * c] + U[3 * r + 1] * V[3 * c + 1] + U[3 * r + 2] * V[3 * c + 2];
    float J = det3(F);
    float D[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) D[i] = F[i] - R[i];
    auto ent = [&](int r, int c) {
      return D[3 * r] * F[3 * c] + D[3 * r + 1] * F[3 * c + 1] + D[3 * r + 2] * F[3 * c + 2];
    };
    float vol = gr.lam * J * (J - 1.0f);
    float m2 = 2.0f * gr.mu_l;
    t[0] = m2 * ent(0, 0) + vol; t[1] = m2 * ent(1, 1) + vol; t[2] = m2 * ent(2, 2) + vol;
    t[3] = m2 * 0.5f * (ent(0, 1) + ent(1, 0));
    t[4] = m2 * 0.5f * (ent(0, 2) + ent(2, 0));
    t[5] = m2 * 0.5f * (ent(1, 2) + ent(2, 1));
  }
}

// Drucker-Prager return map in Hencky strain space (sand); F updated in place.
__device__ __forceinline__ void dp_project(const DevGroup& gr, float (&F)[9]) {
  float U[9], S[3], V[9];
  svd3(F, U, S, V);
  bool clamped = false;
  float e[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float s = S[a];
    if (s < kHenckySigmaMin) { s = kHenckySigmaMin; clamped = true; }
    e[a] = logf(s);
  }
  float tr = e[0] + e[1] + e[2];
  float eh[3] = {e[0] - tr / 3.0f, e[1] - tr / 3.0f, e[2] - tr / 3.0f};
  float nh = sqrtf(eh[0] * eh[0] + eh[1] * eh[1] + eh[2] * eh[2]);
  float en[3] = {e[0], e[1], e[2]};
  bool project = false;
  if (tr >= 0.0f) {
    en[0] = en[1] = en[2] = 0.0f;
    project = true;
  } else {
    float dg = nh + (3.0f * gr.lam + 2.0f * gr.mu_l) / (2.0f * gr.mu_l) * tr * gr.dp_alpha;
    if (dg > 0.0f) {
#pragma unroll
      for (int a = 0; a < 3; ++a) en[a] = e[a] - dg * eh[a] / nh;
      project = true;
    }
  }
  if (!project && !clamped) return;
  float s[3] = {expf(en[0]), expf(en[1]), expf(en[2])};
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      F[3 * r + c] = U[3 * r] * s[0] * V[3 * c] + U[3 * r + 1] * s[1] * V[3 * c + 1] +
                     U[3 * r + 2] * s[2] * V[3 * c + 2];
}

// --------------------------------------------------------------------------
// Rigid geometry: signed distance and outward normal (world frame).

__device__ __forceinline__ float body_sdf(const DevBody& b, float x, float y, float z,
                                          float (&n)[3]) {
  float r0 = x - b.p[0], r1 = y - b.p[1], r2 = z - b.p[2];
  float yb[3] = {b.R[0] * r0 + b.R[3] * r1 + b.R[6] * r2, b.R[1] * r0 + b.R[4] * r1 + b.R[7] * r2,
                 b.R[2] * r0 + b.R[5] * r1 + b.R[8] * r2};
  float nb[3] = {0.0f, 0.0f, 1.0f};
  float phi;
  if (b.shape == MPM_HALFSPACE) {
    phi = yb[2];
  } else if (b.shape == MPM_SPHERE) {
    float dist = sqrtf(yb[0] * yb[0] + yb[1] * yb[1] + yb[2] * yb[2]);
    phi = dist - b.prm[0];
    if (dist > 0.0f) { nb[0] = yb[0] / dist; nb[1] = yb[1] / dist; nb[2] = yb[2] / dist; }
  } else if (b.shape == MPM_BOX) {
    float q[3];
    int am = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) q[a] = fabsf(yb[a]) - b.prm[a];
    if (q[1] > q[am]) am = 1;
    if (q[2] > q[am]) am = 2;
    if (q[am] <= 0.0f) {
      phi = q[am];
      nb[0] = nb[1] = nb[2] = 0.0f;
      nb[am] = yb[am] >= 0.0f ? 1.0f : -1.0f;
    } else {
      float o[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) o[a] = fmaxf(q[a], 0.0f) * (yb[a] >= 0.0f ? 1.0f : -1.0f);
      phi = sqrtf(o[0] * o[0] + o[1] * o[1] + o[2] * o[2]);
      nb[0] = o[0] / phi; nb[1] = o[1] / phi; nb[2] = o[2] / phi;
    }
  } else {  // capsule
    float L = b.prm[0];
    float cz = fminf(fmaxf(yb[2], -L), L);
    float o[3] = {yb[0], yb[1], yb[2] - cz};
    float dist = sqrtf(o[0] * o[0] + o[1] * o[1] + o[2] * o[2]);
    phi = dist - b.prm[1];
    if (dist > 0.0f) { nb[0] = o[0] / dist; nb[1] = o[1] / dist; nb[2] = o[2] / dist; }
    else { nb[0] = 1.0f; nb[1] = 0.0f; nb[2] = 0.0f; }
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) n[r] = b.R[3 * r] * nb[0] + b.R[3 * r + 1] * nb[1] + b.R[3 * r + 2] * nb[2];
  return phi;
}

__device__ __forceinline__ void body_velocity(const DevBody& b, float x, float y, float z,
                                              float (&vel)[3]) {
  float r0 = x - b.p[0], r1 = y - b.p[1], r2 = z - b.p[2];
  vel[0] = b.v[0] + b.w[1] * r2 - b.w[2] * r1;
  vel[1] = b.v[1] + b.w[2] * r0 - b.w[0] * r2;
  vel[2] = b.v[2] + b.w[0] * r1 - b.w[1] * r0;
}

// Normal impulse of the compliant normal law, gamma_n(v_n) = h k (phi0 - h v_n)+ (1 - d v_n)+.
__device__ __forceinline__ float normal_impulse(float phi0, float k, float d, float h, float vn) {
  float a = phi0 - h * vn, c = 1.0f - d * vn;
  return (a > 0.0f && c > 0.0f) ? h * k * a * c : 0.0f;
}

// Lagged contact potential l_c (Sec. IV-B) at relative velocity u (world):
// the derivatives N'(v_n), N''(v_n) of the convex normal potential and the
// friction weight c / s of the regularised Coulomb term.
struct ContactLaw {
  float dN, d2N;    // N', N''
  float cs;         // mu n0 / s
  float inv_s2;     // 1 / s^2
  float vn;
  float ut[3];      // tangential relative velocity
};

__device__ __forceinline__ void contact_law(float phi0, float n0, float mu, float k, float d,
                                            float h, float eps_s, const float (&n)[3],
                                            const float (&u)[3], ContactLaw& L) {
  float vn = n[0] * u[0] + n[1] * u[1] + n[2] * u[2];
  L.vn = vn;
  float vhat = phi0 / h;
  if (d > 0.0f) vhat = fminf(vhat, 1.0f / d);
  if (vn < vhat) {
    float a = phi0 - h * vn, c = 1.0f - d * vn;
    L.dN = -h * k * a * c;
    L.d2N = h * k * (h * c + d * a);
  } else {
    L.dN = 0.0f;
    L.d2N = 0.0f;
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) L.ut[r] = u[r] - vn * n[r];
  float s2 = L.ut[0] * L.ut[0] + L.ut[1] * L.ut[1] + L.ut[2] * L.ut[2] + eps_s * eps_s;
  float inv_s = rsqrtf(s2);
  L.cs = mu * n0 * inv_s;
  L.inv_s2 = inv_s * inv_s;
}

// gradient of l_c in world frame: N' n + (mu n0 / s) u_t
__device__ __forceinline__ void contact_grad(const ContactLaw& L, const float (&n)[3],
                                             float (&g)[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) g[r] = L.dN * n[r] + L.cs * L.ut[r];
}

// Hessian of l_c in world frame (symmetric: xx yy zz xy xz yz):
// N'' n n^T + (mu n0 / s) (I - n n^T - u_t u_t^T / s^2)
__device__ __forceinline__ void contact_hess(const ContactLaw& L, const float (&n)[3],
                                             float (&H)[6]) {
  auto e = [&](int r, int c) {
    float id = (r == c) ? 1.0f : 0.0f;
    return L.d2N * n[r] * n[c] + L.cs * (id - n[r] * n[c] - L.ut[r] * L.ut[c] * L.inv_s2);
  };
  H[0] = e(0, 0); H[1] = e(1, 1); H[2] = e(2, 2);
  H[3] = e(0, 1); H[4] = e(0, 2); H[5] = e(1, 2);
}

// directional first and second derivatives along e (line search, Sec. V-B)
__device__ __forceinline__ void contact_dir(const ContactLaw& L, const float (&n)[3],
                                            const float (&e)[3], float& d1, float& d2) {
  float en = n[0] * e[0] + n[1] * e[1] + n[2] * e[2];
  float et2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2] - en * en;
  float ute = L.ut[0] * e[0] + L.ut[1] * e[1] + L.ut[2] * e[2];
  d1 = L.dN * en + L.cs * ute;
  d2 = L.d2N * en * en + L.cs * (et2 - ute * ute * L.inv_s2);
}

}  // namespace mpmcr
