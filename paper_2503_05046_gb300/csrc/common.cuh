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
  float inv_dx_lo;        // 1/dx = inv_dx + inv_dx_lo (double-float)
  float ox, oy, oz;       // origin
  float ox_lo, oy_lo, oz_lo;  // origin = o + o_lo (double-float)
  float gx, gy, gz;       // gravity
  int rx, ry, rz;         // nodes per axis
  int nbx, nby, nbz;      // 4^3 blocks per axis
  int bc;                 // Dirichlet layers
  int morton_bits;        // bits per axis of the block sort key
  int sort_cell_bits;     // 1: the sort key also orders cells within a block
  // Block-sparse storage (null: dense, every 4^3 block has its nodes at
  // block * 64): slot[b] is the storage block of grid block b during a
  // substep (-1: none), out of pool_blocks storage blocks plus one spare
  // that takes the blocks beyond the pool (reported as a capacity error).
  const int* slot;
  int pool_blocks;
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
  float vol_m, inv_m;     // vol / mass and 1 / mass (P2G's per-unit-mass record)
};

// Particle state, structure of arrays: one float plane per component, planes
// `stride` floats apart: x 0-2, v 3-5, C 6-14, F 15-23 (row-major 3x3), and the
// Kirchhoff stress P(F) F^T of the current F, 24-29 (xx yy zz xy xz yz).
struct Particles {
  float* base;
  long long stride;
  uint32_t* pid;    // particle id (order of addition)
  uint16_t* grp;    // particle group
  __host__ __device__ float* plane(int k) const { return base + (long long)k * stride; }
  __host__ __device__ float* x(int c) const { return plane(c); }
  __host__ __device__ float* v(int c) const { return plane(3 + c); }
  __host__ __device__ float* C(int c) const { return plane(6 + c); }
  __host__ __device__ float* F(int c) const { return plane(15 + c); }
  __host__ __device__ float* tau(int c) const { return plane(24 + c); }
};
constexpr int kParticlePlanes = 30;

// Grid node arrays (block-major storage; see GridDev for the sparse pool).
struct GridArrays {
  float4* mp;      // (m, p): P2G accumulator, all zero outside a substep
  float4* vs;      // (v*, m)
  float4* v;       // grid velocity (.w flags a Dirichlet node); holds v^{k+1} after the solve
  float4* v2;      // second buffer of the solve's iterate
  float4* vlo;     // low parts of the iterate (double-float: v = v + vlo)
  float4* vlo2;    // low parts of the second buffer
  float4* acc0;    // contact terms of the solve: (g_x, g_y, g_z, H_xx), zero outside use
  float4* acc1;    // (H_yy, H_zz, H_xy, H_xz)
  float* acc2;     // H_yz
  float4* dv;      // search direction
  uint8_t* mark;   // per block: touched by P2G this substep (zero outside)
  int* cflag;      // per node: in the stencil of a contact this substep (zero outside)
  int* cnodes;     // contact-node list of the substep's solve
  int* n_cnodes;   // its length (device)
  int cnodes_cap;
  double* pstar2;  // sum over free nodes of m |v*|^2 (grid update), zero outside
  int* act;        // active block list
  int* n_act;      // its length (device)
  int* n_mapped;   // sparse: the length of the list the slot table holds
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

// Error-free transformations for double-float (hi + lo) arithmetic in FP32.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) += x, renormalised so that |lo| <= ulp(hi) / 2
__device__ __forceinline__ void dd_add(float& hi, float& lo, float x) {
  float s, e;
  two_sum(hi, x, s, e);
  e += lo;
  hi = s + e;
  lo = e - (hi - s);
}

// compensated accumulator: S + E tracks a sum of FP32 products and terms
struct CompSum {
  float S = 0.f, E = 0.f;
  __device__ __forceinline__ void add(float x) {
    float s, e;
    two_sum(S, x, s, e);
    S = s;
    E += e;
  }
  __device__ __forceinline__ void add_prod(float w, float x) {
    const float p = w * x;
    const float pe = fmaf(w, x, -p);
    add(p);
    E += pe;
  }
  __device__ __forceinline__ float value() const { return S + E; }
};

// Storage index of node (i, j, k): its block's storage block (the block
// itself when dense) times 64 plus the cell in the block. kDense: the caller
// knows the grid is dense (no table lookup).
template <bool kDense = false>
__device__ __forceinline__ int node_index(const GridDev& g, int i, int j, int k) {
  int b = ((k >> 2) * g.nby + (j >> 2)) * g.nbx + (i >> 2);
  if (!kDense && g.slot) b = g.slot[b];
  return b * kBlockNodes + ((k & 3) << 4) + ((j & 3) << 2) + (i & 3);
}

// Storage block of entry t of the active-block list: the list's order when
// sparse (slot[act[t]] = t), the block itself when dense.
__device__ __forceinline__ int active_storage_block(const GridDev& g, const int* act, int t) {
  return g.slot ? t : act[t];
}

// Nodes of storage (all blocks when dense; the pool and its spare block when
// sparse).
__device__ __forceinline__ long long storage_nodes(const GridDev& g) {
  return (long long)(g.slot ? g.pool_blocks + 1 : g.nbx * g.nby * g.nbz) * kBlockNodes;
}

// Active blocks that have storage (the pool caps a sparse grid's list).
__device__ __forceinline__ int active_with_storage(const GridDev& g, int n_act) {
  return g.slot && n_act > g.pool_blocks ? g.pool_blocks : n_act;
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

// Base node and fractional offset of coordinate x along one axis: the cell
// coordinate (x - origin) / dx is formed in double-float (the origin and 1/dx
// are stored as FP32 pairs), so that f is accurate to FP32 rounding of f
// itself (~6e-8 of a cell) instead of FP32 rounding of the cell coordinate
// (~1e-7 of the node index, 1e-5 of a cell on a 128-node axis): the B-spline
// weights then depend only on the stored position.
__device__ __forceinline__ void cell_coord(float x, float o, float o_lo, float inv, float inv_lo,
                                           int& base, float& f) {
  float dh, dl;
  two_sum(x, -o, dh, dl);
  dl -= o_lo;
  const float p = dh * inv;
  const float lo = fmaf(dh, inv, -p) + fmaf(dh, inv_lo, dl * inv);
  const float b = floorf(p - 0.5f);
  f = (p - b) + lo;  // p - b is exact
  base = (int)b;
  if (f < 0.5f) {
    f += 1.0f;
    base -= 1;
  } else if (f >= 1.5f) {
    f -= 1.0f;
    base += 1;
  }
}

__device__ __forceinline__ void stencil(const GridDev& g, float x, float y, float z,
                                        Stencil& s) {
  cell_coord(x, g.ox, g.ox_lo, g.inv_dx, g.inv_dx_lo, s.base[0], s.fx[0]);
  cell_coord(y, g.oy, g.oy_lo, g.inv_dx, g.inv_dx_lo, s.base[1], s.fx[1]);
  cell_coord(z, g.oz, g.oz_lo, g.inv_dx, g.inv_dx_lo, s.base[2], s.fx[2]);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float f = s.fx[a];
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
// 3x3 singular value decomposition for the constitutive models,
// F = U diag(s) V^T with U, V proper rotations and s[2] < 0 iff det F < 0,
// computed so that s - 1 stays accurate when F is close to a rotation (the
// usual state of an elastic body): with D = F - I (exact in FP32 for entries
// near 1), M = F^T F - I = D + D^T + D^T D is formed without cancellation and
// diagonalised by cyclic Jacobi rotations (V, eigenvalues l); then
// s = sqrt(1 + l) and s - 1 = l / (1 + sqrt(1 + l)). U follows from F V by
// Gram-Schmidt with u2 = u0 x u1. A plain SVD of F in FP32 loses s - 1 (and
// with it the stress) to roundoff of order 1e-7 near F = I.

struct Polar {
  float U[9], V[9];
  float s[3];    // signed singular values, ordered by decreasing magnitude
  float sm1[3];  // s - 1
};

__device__ __forceinline__ void jacobi_pair(float& app, float& aqq, float& apq, float& arp,
                                            float& arq, float (&V)[9], int p, int q) {
  if (apq == 0.0f) return;
  // any rotation angle close to the exact one converges; approximate division
  const float theta = __fdividef(aqq - app, 2.0f * apq);
  const float t = __fdividef(copysignf(1.0f, theta), fabsf(theta) + sqrtf(fmaf(theta, theta, 1.0f)));
  const float c = rsqrtf(fmaf(t, t, 1.0f));
  const float s = t * c;
  app = app - t * apq;
  aqq = aqq + t * apq;
  apq = 0.0f;
  const float rp = arp, rq = arq;
  arp = c * rp - s * rq;
  arq = s * rp + c * rq;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float vp = V[3 * r + p], vq = V[3 * r + q];
    V[3 * r + p] = c * vp - s * vq;
    V[3 * r + q] = s * vp + c * vq;
  }
}

__device__ __forceinline__ float det3(const float (&A)[9]) {
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}

constexpr int kSvdSweeps = 5;      // most cyclic Jacobi sweeps from the identity
// From the V of the SVD that the stored (rounded) F was rebuilt from,
// V^T (F^T F - I) V is diagonal up to that rounding: its diagonal gives the
// eigenvalues to second order, and keeping V misplaces the singular vectors
// only within nearly equal singular values, where the stress does not depend
// on them to first order. No sweep is needed.
constexpr int kSvdWarmSweeps = 0;

// V0 (optional): a rotation that nearly diagonalises F^T F (the V of a nearby
// F), from which `sweeps` Jacobi sweeps suffice.
__device__ __forceinline__ void polar_svd(const float (&F)[9], Polar& P, const float* V0 = nullptr,
                                          int sweeps = kSvdSweeps) {
  float D[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) D[i] = F[i];
  D[0] -= 1.0f; D[4] -= 1.0f; D[8] -= 1.0f;
  auto dtd = [&](int a, int b) {
    return D[a] * D[b] + D[3 + a] * D[3 + b] + D[6 + a] * D[6 + b];
  };
  float a00 = 2.0f * D[0] + dtd(0, 0);
  float a11 = 2.0f * D[4] + dtd(1, 1);
  float a22 = 2.0f * D[8] + dtd(2, 2);
  float a01 = D[1] + D[3] + dtd(0, 1);
  float a02 = D[2] + D[6] + dtd(0, 2);
  float a12 = D[5] + D[7] + dtd(1, 2);
  float* V = P.V;
  if (V0) {
    // A <- V0^T A V0 (orthogonal congruence: the absolute accuracy of A near
    // F = I is kept) and V <- V0
    const float M[9] = {a00, a01, a02, a01, a11, a12, a02, a12, a22};
    float W[9];  // M V0
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        W[3 * r + c] = M[3 * r] * V0[c] + M[3 * r + 1] * V0[3 + c] + M[3 * r + 2] * V0[6 + c];
    auto vtw = [&](int r, int c) {
      return V0[r] * W[c] + V0[3 + r] * W[3 + c] + V0[6 + r] * W[6 + c];
    };
    a00 = vtw(0, 0); a11 = vtw(1, 1); a22 = vtw(2, 2);
    a01 = vtw(0, 1); a02 = vtw(0, 2); a12 = vtw(1, 2);
#pragma unroll
    for (int i = 0; i < 9; ++i) V[i] = V0[i];
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0f : 0.0f;
  }
  float (&Vr)[9] = P.V;
#pragma unroll 1
  for (int sweep = 0; sweep < sweeps; ++sweep) {
    // converged once the off-diagonal part is below FP32 resolution of the
    // diagonal (squared norms; a zero matrix needs no rotation)
    const float off = a01 * a01 + a02 * a02 + a12 * a12;
    const float dia = a00 * a00 + a11 * a11 + a22 * a22;
    if (off <= 1e-15f * dia) break;
    jacobi_pair(a00, a11, a01, a02, a12, Vr, 0, 1);
    jacobi_pair(a00, a22, a02, a01, a12, Vr, 0, 2);
    jacobi_pair(a11, a22, a12, a01, a02, Vr, 1, 2);
  }
  float l[3] = {a00, a11, a22};
  // order by decreasing eigenvalue; each swap negates one column so V stays a rotation
  auto swapneg = [&](int c0, int c1) {
    float t = l[c0]; l[c0] = l[c1]; l[c1] = t;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      float v = V[3 * r + c0];
      V[3 * r + c0] = -V[3 * r + c1];
      V[3 * r + c1] = v;
    }
  };
  if (l[0] < l[1]) swapneg(0, 1);
  if (l[0] < l[2]) swapneg(0, 2);
  if (l[1] < l[2]) swapneg(1, 2);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float la = fmaxf(l[a], -1.0f);
    const float sa = sqrtf(1.0f + la);
    P.s[a] = sa;
    P.sm1[a] = la / (1.0f + sa);
  }
  // U from F V: u0 = Fv0/|Fv0|, u1 = Gram-Schmidt of Fv1, u2 = u0 x u1
  float b[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int r = 0; r < 3; ++r)
      b[c][r] = F[3 * r] * V[c] + F[3 * r + 1] * V[3 + c] + F[3 * r + 2] * V[6 + c];
  // a singular value far below 1 is taken as |F v| (relative accuracy
  // ~eps / s) instead of sqrt(1 + lambda), where 1 + lambda cancels
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (l[a] < -0.5f) {
      const float sa = sqrtf(b[a][0] * b[a][0] + b[a][1] * b[a][1] + b[a][2] * b[a][2]);
      P.s[a] = sa;
      P.sm1[a] = sa - 1.0f;
    }
  }
  float u0[3], u1[3];
  float n0 = b[0][0] * b[0][0] + b[0][1] * b[0][1] + b[0][2] * b[0][2];
  if (n0 > 1e-30f) {
    const float inv = rsqrtf(n0);
    u0[0] = b[0][0] * inv; u0[1] = b[0][1] * inv; u0[2] = b[0][2] * inv;
  } else {
    u0[0] = 1.0f; u0[1] = 0.0f; u0[2] = 0.0f;
  }
  const float pr = u0[0] * b[1][0] + u0[1] * b[1][1] + u0[2] * b[1][2];
  u1[0] = b[1][0] - pr * u0[0]; u1[1] = b[1][1] - pr * u0[1]; u1[2] = b[1][2] - pr * u0[2];
  float n1 = u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2];
  if (!(n1 > 1e-30f)) {  // any unit vector orthogonal to u0
    const int a = (fabsf(u0[0]) <= fabsf(u0[1]) && fabsf(u0[0]) <= fabsf(u0[2])) ? 0
                  : (fabsf(u0[1]) <= fabsf(u0[2])) ? 1 : 2;
    float e[3] = {0.0f, 0.0f, 0.0f};
    e[a] = 1.0f;
    u1[0] = u0[1] * e[2] - u0[2] * e[1];
    u1[1] = u0[2] * e[0] - u0[0] * e[2];
    u1[2] = u0[0] * e[1] - u0[1] * e[0];
    n1 = u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2];
  }
  const float inv1 = rsqrtf(n1);
  u1[0] *= inv1; u1[1] *= inv1; u1[2] *= inv1;
  const float u2[3] = {u0[1] * u1[2] - u0[2] * u1[1], u0[2] * u1[0] - u0[0] * u1[2],
                       u0[0] * u1[1] - u0[1] * u1[0]};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    P.U[3 * r] = u0[r];
    P.U[3 * r + 1] = u1[r];
    P.U[3 * r + 2] = u2[r];
  }
  if (det3(F) < 0.0f) {  // reflection carried by the smallest singular value
    P.s[2] = -P.s[2];
    P.sm1[2] = P.s[2] - 1.0f;
  }
}

constexpr float kHenckySigmaMin = 1e-4f;

// Kirchhoff stress tau = U diag(d) U^T + iso I as 6 entries (xx yy zz xy xz yz).
__device__ __forceinline__ void tau_from(const float* U, const float (&d)[3], float iso,
                                         float (&t)[6]) {
  auto ent = [&](int r, int c) {
    return U[3 * r] * d[0] * U[3 * c] + U[3 * r + 1] * d[1] * U[3 * c + 1] +
           U[3 * r + 2] * d[2] * U[3 * c + 2];
  };
  t[0] = ent(0, 0) + iso; t[1] = ent(1, 1) + iso; t[2] = ent(2, 2) + iso;
  t[3] = ent(0, 1); t[4] = ent(0, 2); t[5] = ent(1, 2);
}

// Hencky log strains of the singular values, clamped below at kHenckySigmaMin
__device__ __forceinline__ bool hencky_strain(const Polar& P, float (&e)[3]) {
  bool clamped = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (P.s[a] > kHenckySigmaMin) {
      e[a] = log1pf(P.sm1[a]);
    } else {
      e[a] = logf(kHenckySigmaMin);
      clamped = true;
    }
  }
  return clamped;
}

// Hencky: tau = U diag(2 mu e + lam tr e) U^T
__device__ __forceinline__ void tau_hencky(const DevGroup& gr, const float* U, const float (&e)[3],
                                           float (&t)[6]) {
  const float tr = e[0] + e[1] + e[2];
  const float d[3] = {2.0f * gr.mu_l * e[0] + gr.lam * tr, 2.0f * gr.mu_l * e[1] + gr.lam * tr,
                      2.0f * gr.mu_l * e[2] + gr.lam * tr};
  tau_from(U, d, 0.0f, t);
}

// fixed corotated: tau = 2 mu (F - R) F^T + lam J (J - 1) I
//                      = U diag(2 mu s (s - 1)) U^T + lam J (J - 1) I
__device__ __forceinline__ void tau_corotated(const DevGroup& gr, const Polar& P, float (&t)[6]) {
  const float a = P.sm1[0], b = P.sm1[1], c = P.sm1[2];
  const float jm1 = a + b + c + a * b + a * c + b * c + a * b * c;  // J - 1
  const float d[3] = {2.0f * gr.mu_l * P.s[0] * a, 2.0f * gr.mu_l * P.s[1] * b,
                      2.0f * gr.mu_l * P.s[2] * c};
  tau_from(P.U, d, gr.lam * (1.0f + jm1) * jm1, t);
}

// Kirchhoff stress of a given F (no plastic projection); V0 as in polar_svd.
__device__ __forceinline__ void kirchhoff(const DevGroup& gr, const float (&F)[9], float (&t)[6],
                                          const float* V0 = nullptr, int sweeps = kSvdSweeps) {
  if (gr.model == MPM_CLOTH) {  // stress-free particles (the mesh carries the elasticity)
#pragma unroll
    for (int c = 0; c < 6; ++c) t[c] = 0.f;
    return;
  }
  Polar P;
  polar_svd(F, P, V0, sweeps);
  if (gr.model == MPM_DRUCKER_PRAGER) {
    float e[3];
    hencky_strain(P, e);
    tau_hencky(gr, P.U, e, t);
  } else {
    tau_corotated(gr, P, t);
  }
}

// Constitutive update at the end of G2P: the Drucker-Prager return map in
// Hencky strain space for sand (F projected in place), then the Kirchhoff
// stress of the final F for the next P2G. For an unprojected F one SVD serves
// both; a projected F = U diag(exp e') V^T is rounded to FP32 when stored, so
// its stress is taken from the stored value (a second decomposition, in the
// first one's V, which diagonalises it up to the rounding) to keep tau equal
// to the stress of the state F.
__device__ __forceinline__ void constitutive_update(const DevGroup& gr, float (&F)[9],
                                                    float (&t)[6]) {
  Polar P;
  polar_svd(F, P);
  if (gr.model != MPM_DRUCKER_PRAGER) {
    tau_corotated(gr, P, t);
    return;
  }
  float e[3];
  const bool clamped = hencky_strain(P, e);
  const float tr = e[0] + e[1] + e[2];
  const float eh[3] = {e[0] - tr / 3.0f, e[1] - tr / 3.0f, e[2] - tr / 3.0f};
  const float nh = sqrtf(eh[0] * eh[0] + eh[1] * eh[1] + eh[2] * eh[2]);
  float en[3] = {e[0], e[1], e[2]};
  bool project = false;
  if (tr >= 0.0f) {
    en[0] = en[1] = en[2] = 0.0f;
    project = true;
  } else {
    const float dg = nh + (3.0f * gr.lam + 2.0f * gr.mu_l) / (2.0f * gr.mu_l) * tr * gr.dp_alpha;
    if (dg > 0.0f) {
#pragma unroll
      for (int a = 0; a < 3; ++a) en[a] = e[a] - dg * eh[a] / nh;
      project = true;
    }
  }
  if (!project && !clamped) {
    tau_hencky(gr, P.U, en, t);
    return;
  }
  const float sv[3] = {expf(en[0]), expf(en[1]), expf(en[2])};
  const float* U = P.U;
  const float* V = P.V;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      F[3 * r + c] = U[3 * r] * sv[0] * V[3 * c] + U[3 * r + 1] * sv[1] * V[3 * c + 1] +
                     U[3 * r + 2] * sv[2] * V[3 * c + 2];
  kirchhoff(gr, F, t, V, kSvdWarmSweeps);
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

// The same signed distance evaluated in FP64 from the FP32 inputs. A
// penetration of 1e-4 m at 0.05 m from a body origin is only known to ~4e-5
// relative in FP32, so contact registration and the penetration depth phi0
// use this value for the (few) particles the FP32 test puts near a surface.
__device__ __forceinline__ double body_sdf_f64(const DevBody& b, float x, float y, float z) {
  const double r0 = (double)x - (double)b.p[0], r1 = (double)y - (double)b.p[1],
               r2 = (double)z - (double)b.p[2];
  double yb[3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    yb[c] = (double)b.R[c] * r0 + (double)b.R[3 + c] * r1 + (double)b.R[6 + c] * r2;
  if (b.shape == MPM_HALFSPACE) return yb[2];
  if (b.shape == MPM_SPHERE) return sqrt(yb[0] * yb[0] + yb[1] * yb[1] + yb[2] * yb[2]) - (double)b.prm[0];
  if (b.shape == MPM_BOX) {
    double q[3], o2 = 0.0, qm = -1e300;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      q[a] = fabs(yb[a]) - (double)b.prm[a];
      qm = fmax(qm, q[a]);
      const double qp = fmax(q[a], 0.0);
      o2 += qp * qp;
    }
    return qm <= 0.0 ? qm : sqrt(o2);
  }
  const double L = (double)b.prm[0];
  const double cz = fmin(fmax(yb[2], -L), L);
  const double o0 = yb[0], o1 = yb[1], o2 = yb[2] - cz;
  return sqrt(o0 * o0 + o1 * o1 + o2 * o2) - (double)b.prm[1];
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

// The contact potential on the line u(alpha) = v_c + alpha e of the line
// search (Sec. V-B): the per-contact invariants are formed once, after which
// f' and f'' contributions at any alpha cost a few FMAs and one rsqrt
// (u_t(alpha) = (v_c - v_n n) + alpha (e - e_n n)).
struct ContactLine {
  float vn0, en, vhat, phi0, hk, h, d, mun0, eps2, et2;
  float vt[3], et[3];
};

__device__ __forceinline__ void contact_line(float phi0, float n0, float mu, float k, float d,
                                             float h, float eps_s, const float (&n)[3],
                                             const float (&u)[3], const float (&e)[3],
                                             ContactLine& L) {
  L.vn0 = n[0] * u[0] + n[1] * u[1] + n[2] * u[2];
  L.en = n[0] * e[0] + n[1] * e[1] + n[2] * e[2];
  float vhat = phi0 / h;
  if (d > 0.0f) vhat = fminf(vhat, 1.0f / d);
  L.vhat = vhat;
  L.phi0 = phi0;
  L.hk = h * k;
  L.h = h;
  L.d = d;
  L.mun0 = mu * n0;
  L.eps2 = eps_s * eps_s;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    L.vt[r] = u[r] - L.vn0 * n[r];
    L.et[r] = e[r] - L.en * n[r];
  }
  L.et2 = L.et[0] * L.et[0] + L.et[1] * L.et[1] + L.et[2] * L.et[2];
}

// d/dalpha and d2/dalpha2 of l_c(v_c + alpha e)
__device__ __forceinline__ void contact_line_eval(const ContactLine& L, float al, float& d1,
                                                  float& d2) {
  const float vn = fmaf(al, L.en, L.vn0);
  float dN = 0.0f, d2N = 0.0f;
  if (vn < L.vhat) {
    const float a = L.phi0 - L.h * vn, c = 1.0f - L.d * vn;
    dN = -L.hk * a * c;
    d2N = L.hk * (L.h * c + L.d * a);
  }
  const float u0 = fmaf(al, L.et[0], L.vt[0]), u1 = fmaf(al, L.et[1], L.vt[1]),
              u2 = fmaf(al, L.et[2], L.vt[2]);
  const float s2 = u0 * u0 + u1 * u1 + u2 * u2 + L.eps2;
  const float inv_s = rsqrtf(s2);
  const float cs = L.mun0 * inv_s;
  const float ute = u0 * L.et[0] + u1 * L.et[1] + u2 * L.et[2];
  d1 = dN * L.en + cs * ute;
  d2 = d2N * L.en * L.en + cs * (L.et2 - ute * ute * inv_s * inv_s);
}

// A batched launch's per-scene argument record, copied from global into
// shared memory by all threads of the block (the caller then syncs).
template <class T>
__device__ __forceinline__ void load_args(const T* __restrict__ src, T& dst) {
  static_assert(sizeof(T) % 4 == 0, "argument records are whole words");
  for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += blockDim.x)
    reinterpret_cast<int*>(&dst)[i] = reinterpret_cast<const int*>(src)[i];
}

}  // namespace mpmcr
