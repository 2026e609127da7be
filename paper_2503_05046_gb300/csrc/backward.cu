// backward.cu -- reverse-mode adjoint of one MPM substep (the free motion of
// Eq. (6) and G2P with the constitutive update: fixed-corotated stress, or the
// Hencky stress with the Drucker-Prager return map), for mpm_backward. The contact
// solve's part (implicit differentiation of Eq. (8)-(9), with the contact
// geometry's dependence on the particle state) is k_adjoint in solve.cu.
//
// Forward substep from the particle state s = (x, v, C, F), with
// k = 4 / dx^2, w_ip the quadratic B-spline weights and d_ip = x_i - x_p:
//   P2G    m_i = sum_p w_ip m_p,  p_i = sum_p w_ip (m_p v_p + A_p d_ip),
//          A_p = m_p C_p - h k V_p tau(F_p)
//   grid   v*_i = p_i / m_i + h g   (0 on Dirichlet wall nodes)
//   solve  v = argmin of Eq. (8)
//   G2P    v'_p = sum_i w_ip v_i,  C'_p = k sum_i w_ip v_i d_ip^T,
//          x'_p = x_p + h v'_p,  F'_p = (I + h C'_p) F_p
// The kernels below take the adjoint of s' (per particle, planes in slot
// order) and produce the adjoint of s, in the reverse order: G2P, [solve],
// grid, P2G. Grid adjoints live in one dense float4 per node: after G2P it
// holds vbar (xyz), the solve's adjoint turns it into (v*bar, mbar) on the
// contact nodes, and the grid adjoint into (pbar, mbar).
#include "kernels.h"

namespace mpmcr {

namespace {

constexpr int kThreads = 256;

// weights, their gradients (physical units) and node offsets of a stencil
struct StencilGrad {
  Stencil s;
  float dw[3][3];  // d w_a[c] / d x_a
};

__device__ __forceinline__ void stencil_grad(const GridDev& g, float x, float y, float z,
                                             StencilGrad& S) {
  stencil(g, x, y, z, S.s);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float f = S.s.fx[a];
    S.dw[a][0] = -(1.5f - f) * g.inv_dx;
    S.dw[a][1] = -2.0f * (f - 1.0f) * g.inv_dx;
    S.dw[a][2] = (f - 0.5f) * g.inv_dx;
  }
}

__device__ __forceinline__ float4 ld_bar3(const float* bar, int plane, size_t n, int i) {
  return make_float4(bar[plane * n + i], bar[(plane + 1) * n + i], bar[(plane + 2) * n + i], 0.f);
}

// ---- adjoints of spectral matrix functions ----------------------------------
// G(F) = U diag(h(s)) V^T for F = U diag(s) V^T. With M = U^T dF V (ds_i =
// M_ii; the rotations follow from the off-diagonal M), U^T dG V has diagonal
// sum_j dh_i/ds_j M_jj and, for i != j, (a + b)/2 M_ij + (a - b)/2 M_ji with
// a = (h_i - h_j) / (s_i - s_j), b = (h_i + h_j) / (s_i + s_j). The 2x2 map on
// (M_ij, M_ji) is symmetric, so the adjoint has the same form on A = U^T Gbar V;
// Fbar = U Mbar V^T. The divided differences a come from the caller: near
// rest the s_i differ by ~1e-5 and h_i - h_j formed in FP32 would keep only
// two or three digits, so each caller writes them out in closed form.
__device__ void spectral_adjoint(const Polar& P, const float (&h)[3], const float (&dh)[3][3],
                                 const float (&a)[3][3], const float (&Gb)[9], float (&Fb)[9]) {
  const float* U = P.U;
  const float* V = P.V;
  float T[9], A[9], Mb[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) T[3 * r + q] = Gb[3 * r] * V[q] + Gb[3 * r + 1] * V[3 + q] + Gb[3 * r + 2] * V[6 + q];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) A[3 * r + q] = U[r] * T[q] + U[3 + r] * T[3 + q] + U[6 + r] * T[6 + q];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float d = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j) d += dh[j][i] * A[4 * j];
    Mb[4 * i] = d;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (i == j) continue;
      float ss = P.s[i] + P.s[j];
      if (fabsf(ss) < 1e-6f) ss = ss < 0.f ? -1e-6f : 1e-6f;
      const float b = (h[i] + h[j]) / ss;
      Mb[3 * i + j] = 0.5f * (a[i][j] + b) * A[3 * i + j] + 0.5f * (a[i][j] - b) * A[3 * j + i];
    }
  float MV[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) MV[3 * r + q] = Mb[3 * r] * V[3 * q] + Mb[3 * r + 1] * V[3 * q + 1] + Mb[3 * r + 2] * V[3 * q + 2];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) Fb[3 * r + q] = U[3 * r] * MV[q] + U[3 * r + 1] * MV[3 + q] + U[3 * r + 2] * MV[6 + q];
}

// s_i - s_j from the accurate s - 1, and (log s_i - log s_j) / (s_i - s_j)
__device__ __forceinline__ float ds_of(const Polar& P, int i, int j) { return P.sm1[i] - P.sm1[j]; }
__device__ __forceinline__ float dlog_ratio(const Polar& P, int i, int j) {
  const float ds = ds_of(P, i, j);
  const float r = ds / P.s[j];
  return fabsf(r) > 1e-4f ? log1pf(r) / ds : (1.0f - 0.5f * r + r * r / 3.0f) / P.s[j];
}

// divided differences of an h with h_i = H(s_i, common terms), generic form
__device__ __forceinline__ float divided(const Polar& P, const float (&h)[3], const float (&dh)[3][3],
                                         int i, int j) {
  const float ds = ds_of(P, i, j);
  return fabsf(ds) > 1e-4f * (fabsf(P.s[i]) + fabsf(P.s[j])) ? (h[i] - h[j]) / ds
                                                                : dh[i][i] - dh[i][j];
}

// Hencky log strain of a singular value and its derivative (0 where clamped)
__device__ __forceinline__ void hencky_eps(const Polar& P, float (&e)[3], float (&de)[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (P.s[a] > kHenckySigmaMin) {
      e[a] = log1pf(P.sm1[a]);
      de[a] = 1.0f / P.s[a];
    } else {
      e[a] = logf(kHenckySigmaMin);
      de[a] = 0.0f;
    }
  }
}

// Hencky Kirchhoff stress tau = U diag(g) U^T, g = 2 mu e + lam tr(e) 1, as
// tau = Pt F^T with Pt = U diag(g / s) V^T: Fbar = (spectral adjoint of Pt
// at Ptbar = taubar F) + taubar^T Pt; mubar = 2 sum e_a u_a^T taubar u_a,
// lambar = tr(taubar) tr(e). Divided differences of h = g / s:
// (h_i - h_j) / (s_i - s_j) = (2 mu (s_j q_ij - e_j) - lam tr e) / (s_i s_j),
// q_ij = (e_i - e_j) / (s_i - s_j).
__device__ void hencky_adjoint(const float (&F)[9], const float (&tb)[9], float mu, float lam,
                               float (&Fb)[9], float& mub, float& lamb) {
  Polar P;
  polar_svd(F, P);
  float e[3], de[3];
  hencky_eps(P, e, de);
  const bool clamped = de[0] == 0.f || de[1] == 0.f || de[2] == 0.f;
  const float tr = e[0] + e[1] + e[2];
  float g[3], h[3], dh[3][3], a[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    g[i] = 2.0f * mu * e[i] + lam * tr;
    float s = P.s[i];
    if (fabsf(s) < 1e-12f) s = s < 0.f ? -1e-12f : 1e-12f;
    h[i] = g[i] / s;
#pragma unroll
    for (int j = 0; j < 3; ++j) dh[i][j] = ((i == j ? 2.0f * mu : 0.0f) + lam) * de[j] / s;
    dh[i][i] -= g[i] / (s * s);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      a[i][j] = (i == j) ? 0.f
                : clamped ? divided(P, h, dh, i, j)
                          : (2.0f * mu * (P.s[j] * dlog_ratio(P, i, j) - e[j]) - lam * tr) / (P.s[i] * P.s[j]);
  float Pb[9], Pt[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      Pb[3 * r + q] = tb[3 * r] * F[q] + tb[3 * r + 1] * F[3 + q] + tb[3 * r + 2] * F[6 + q];
      Pt[3 * r + q] = P.U[3 * r] * h[0] * P.V[3 * q] + P.U[3 * r + 1] * h[1] * P.V[3 * q + 1] +
                      P.U[3 * r + 2] * h[2] * P.V[3 * q + 2];
    }
  spectral_adjoint(P, h, dh, a, Pb, Fb);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q)
      Fb[3 * r + q] += tb[r] * Pt[q] + tb[3 + r] * Pt[3 + q] + tb[6 + r] * Pt[6 + q];  // taubar^T Pt
  float m = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float utu = 0.f;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int q = 0; q < 3; ++q) utu += P.U[3 * r + k] * tb[3 * r + q] * P.U[3 * q + k];
    m += e[k] * utu;
  }
  mub = 2.0f * m;
  lamb = (tb[0] + tb[4] + tb[8]) * tr;
}

// Drucker-Prager return map in Hencky strain (the forward's
// constitutive_update): F_new = U exp(e') V^T with e = log s (clamped) and
//   tr e >= 0:            e' = 0
//   dgamma = |e^| + c tr e > 0 (c = (3 lam + 2 mu) / (2 mu) alpha):
//                         e' = (tr e / 3) 1 - c tr e n,  n = e^ / |e^|
//   otherwise:            e' = e (F_new = F_trial).
// Given Fbar of F_new: Fbar of F_trial (spectral adjoint with h = exp(e'),
// dh_i/ds_j = exp(e'_i) (de'_i/de_j) de_j/ds_j, and on the plastic branch
// (h_i - h_j) / (s_i - s_j) = exp(e'_j) expm1(e'_i - e'_j) / (s_i - s_j) with
// e'_i - e'_j = -c tr (e_i - e_j) / |e^|) and the adjoints of mu and lam
// through c (de'/dc = -tr e n).
__device__ void dp_return_adjoint(const DevGroup& gr, const float (&Ft)[9], const float (&Gb)[9],
                                  float (&Fb)[9], float& mub, float& lamb) {
  mub = lamb = 0.f;
  Polar P;
  polar_svd(Ft, P);
  float e[3], de[3];
  hencky_eps(P, e, de);
  const bool clamped = de[0] == 0.f || de[1] == 0.f || de[2] == 0.f;
  const float tr = e[0] + e[1] + e[2];
  const float eh[3] = {e[0] - tr / 3.0f, e[1] - tr / 3.0f, e[2] - tr / 3.0f};
  const float nh = sqrtf(eh[0] * eh[0] + eh[1] * eh[1] + eh[2] * eh[2]);
  const float c = (3.0f * gr.lam + 2.0f * gr.mu_l) / (2.0f * gr.mu_l) * gr.dp_alpha;
  float ep[3] = {e[0], e[1], e[2]};
  float J[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
  int branch = 0;  // 0 elastic, 1 tensile (e' = 0), 2 plastic
  float n[3] = {0.f, 0.f, 0.f};
  if (tr >= 0.0f) {
    branch = 1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      ep[i] = 0.f;
#pragma unroll
      for (int j = 0; j < 3; ++j) J[i][j] = 0.f;
    }
  } else if (nh + c * tr > 0.0f) {
    branch = 2;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      n[i] = eh[i] / nh;
      ep[i] = tr / 3.0f - c * tr * n[i];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        J[i][j] = 1.0f / 3.0f - c * n[i] -
                  c * tr * ((i == j ? 1.0f : 0.0f) - 1.0f / 3.0f - n[i] * n[j]) / nh;
  } else if (!clamped) {
    // elastic, no clamp: F_new = F_trial
#pragma unroll
    for (int k = 0; k < 9; ++k) Fb[k] = Gb[k];
    return;
  }
  float h[3], dh[3][3], a[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    h[i] = expf(ep[i]);
#pragma unroll
    for (int j = 0; j < 3; ++j) dh[i][j] = h[i] * J[i][j] * de[j];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (i == j) { a[i][j] = 0.f; continue; }
      if (branch == 1) {
        a[i][j] = 0.f;  // h = 1
      } else if (branch == 2 && !clamped) {
        const float ds = ds_of(P, i, j);
        const float dq = dlog_ratio(P, i, j);              // (e_i - e_j) / ds
        const float dep = -c * tr * dq / nh;               // (e'_i - e'_j) / ds
        const float x = dep * ds;                          // e'_i - e'_j
        a[i][j] = h[j] * (fabsf(x) > 1e-4f ? expm1f(x) / ds : dep * (1.0f + 0.5f * x));
      } else {
        a[i][j] = divided(P, h, dh, i, j);
      }
    }
  spectral_adjoint(P, h, dh, a, Gb, Fb);
  if (branch == 2) {
    // cbar = sum_i hbar_i h_i de'_i/dc, hbar_i = (U^T Gbar V)_ii
    float cb = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float A = 0.f;
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int q = 0; q < 3; ++q) A += P.U[3 * r + i] * Gb[3 * r + q] * P.V[3 * q + i];
      cb += A * h[i] * (-tr * n[i]);
    }
    // c = (3 lam / (2 mu) + 1) alpha
    lamb = cb * 3.0f * gr.dp_alpha / (2.0f * gr.mu_l);
    mub = -cb * 3.0f * gr.lam * gr.dp_alpha / (2.0f * gr.mu_l * gr.mu_l);
  }
}

// ---- G2P adjoint -----------------------------------------------------------
// vbar'_tot = vbar' + h xbar'  (x' = x + h v')
// Cbar'_tot = Cbar' + h Fbar' F^T,  Fbar = (I + h C')^T Fbar'
// vbar_i  += w (vbar'_tot + k Cbar'_tot d_i)
// xbar    += xbar' + sum_i grad w_i (vbar'_tot . v_i + k v_i^T Cbar'_tot d_i)
//            - k sum_i w_i Cbar'_tot^T v_i
__global__ void __launch_bounds__(kThreads) k_g2p_adjoint(BackwardArgs a) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  if (i >= a.n) return;
  const GridDev& g = a.g;
  const size_t n = (size_t)a.n;
  const float xp[3] = {a.P.x(0)[i], a.P.x(1)[i], a.P.x(2)[i]};
  StencilGrad S;
  stencil_grad(g, xp[0], xp[1], xp[2], S);
  if (!stencil_inside(g, S.s)) return;
  const float kk = 4.0f * g.inv_dx * g.inv_dx;
  const float h = a.h;
  // recompute C' = k sum w v_i d_i^T
  float Bm[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) Bm[c] = 0.f;
  for (int cz = 0; cz < 3; ++cz)
    for (int cy = 0; cy < 3; ++cy)
#pragma unroll
      for (int cx = 0; cx < 3; ++cx) {
        const float w = S.s.w[0][cx] * S.s.w[1][cy] * S.s.w[2][cz];
        const float d[3] = {(cx - S.s.fx[0]) * g.dx, (cy - S.s.fx[1]) * g.dx, (cz - S.s.fx[2]) * g.dx};
        const float4 v = __ldg(a.G.v + node_index(g, S.s.base[0] + cx, S.s.base[1] + cy, S.s.base[2] + cz));
        const float vv[3] = {v.x, v.y, v.z};
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c) Bm[3 * r + c] += w * vv[r] * d[c];
      }
  float Cn[9], F[9], Fb[9], Cb[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    Cn[c] = kk * Bm[c];
    F[c] = a.P.F(c)[i];
    Fb[c] = a.bin[(15 + c) * n + i];
    Cb[c] = a.bin[(6 + c) * n + i];
  }
  const float4 xb = ld_bar3(a.bin, 0, n, i), vb = ld_bar3(a.bin, 3, n, i);
  const float ub[3] = {vb.x + h * xb.x, vb.y + h * xb.y, vb.z + h * xb.z};
  // sand: the stored F is the return map of F_trial = (I + h C') F; carry
  // Fbar back through it (the corotated F is F_trial itself)
  const int grp = a.P.grp[i];
  const DevGroup gr = a.groups[grp];
  if (gr.model == MPM_DRUCKER_PRAGER) {
    float Ft[9], Gt[9], mub, lamb;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        Ft[3 * r + c] = F[3 * r + c] + h * (Cn[3 * r] * F[c] + Cn[3 * r + 1] * F[3 + c] + Cn[3 * r + 2] * F[6 + c]);
    dp_return_adjoint(gr, Ft, Fb, Gt, mub, lamb);
#pragma unroll
    for (int c = 0; c < 9; ++c) Fb[c] = Gt[c];
    if (mub != 0.f) atomicAdd(a.mat_bar + 2 * grp, (double)mub);
    if (lamb != 0.f) atomicAdd(a.mat_bar + 2 * grp + 1, (double)lamb);
  }
  float Ch[9], Fo[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // Cbar'_tot = Cbar' + h Fbar' F^T ; Fbar = Fbar' + h C'^T Fbar'
      Ch[3 * r + c] = Cb[3 * r + c] + h * (Fb[3 * r] * F[3 * c] + Fb[3 * r + 1] * F[3 * c + 1] +
                                           Fb[3 * r + 2] * F[3 * c + 2]);
      Fo[3 * r + c] = Fb[3 * r + c] + h * (Cn[r] * Fb[c] + Cn[3 + r] * Fb[3 + c] + Cn[6 + r] * Fb[6 + c]);
    }
  float xo[3] = {xb.x, xb.y, xb.z};
  for (int cz = 0; cz < 3; ++cz)
    for (int cy = 0; cy < 3; ++cy)
#pragma unroll
      for (int cx = 0; cx < 3; ++cx) {
        const float w = S.s.w[0][cx] * S.s.w[1][cy] * S.s.w[2][cz];
        const float gw[3] = {S.dw[0][cx] * S.s.w[1][cy] * S.s.w[2][cz],
                             S.s.w[0][cx] * S.dw[1][cy] * S.s.w[2][cz],
                             S.s.w[0][cx] * S.s.w[1][cy] * S.dw[2][cz]};
        const float d[3] = {(cx - S.s.fx[0]) * g.dx, (cy - S.s.fx[1]) * g.dx, (cz - S.s.fx[2]) * g.dx};
        const int node = node_index(g, S.s.base[0] + cx, S.s.base[1] + cy, S.s.base[2] + cz);
        const float4 v = __ldg(a.G.v + node);
        const float vv[3] = {v.x, v.y, v.z};
        float Cd[3], CTv[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          Cd[r] = Ch[3 * r] * d[0] + Ch[3 * r + 1] * d[1] + Ch[3 * r + 2] * d[2];
          CTv[r] = Ch[r] * vv[0] + Ch[3 + r] * vv[1] + Ch[6 + r] * vv[2];
        }
        const float t = ub[0] * vv[0] + ub[1] * vv[1] + ub[2] * vv[2] +
                        kk * (vv[0] * Cd[0] + vv[1] * Cd[1] + vv[2] * Cd[2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) xo[c] += t * gw[c] - kk * w * CTv[c];
        red_add_v4(a.gbar + node, w * (ub[0] + kk * Cd[0]), w * (ub[1] + kk * Cd[1]),
                   w * (ub[2] + kk * Cd[2]), 0.f);
      }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    a.bout[c * n + i] = xo[c];
    a.bout[(3 + c) * n + i] = 0.f;
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    a.bout[(6 + c) * n + i] = 0.f;
    a.bout[(15 + c) * n + i] = Fo[c];
  }
}

// ---- grid update adjoint ---------------------------------------------------
// on free nodes with mass: pbar = v*bar / m, mbar += -v*bar . (v* - h g) / m;
// walls hold v* = 0 (no dependence on p or m)
__global__ void __launch_bounds__(kThreads) k_grid_adjoint(BackwardArgs a) {
  const GridDev& g = a.g;
  const int n_act = *a.G.n_act;
  const long long total = (long long)active_with_storage(g, n_act) * kBlockNodes;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int blk = a.G.act[t >> 6];
    const int cell = (int)(t & 63);
    const int node = active_storage_block(g, a.G.act, (int)(t >> 6)) * kBlockNodes + cell;
    const float4 vs = a.G.vs[node];
    const float4 gb = a.gbar[node];
    const int bx = blk % g.nbx, by = (blk / g.nbx) % g.nby, bz = blk / (g.nbx * g.nby);
    const int ii = bx * 4 + (cell & 3), jj = by * 4 + ((cell >> 2) & 3), kk = bz * 4 + (cell >> 4);
    const bool wall = ii < g.bc || jj < g.bc || kk < g.bc || ii >= g.rx - g.bc ||
                      jj >= g.ry - g.bc || kk >= g.rz - g.bc;
    float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
    if (vs.w > 0.f) {
      if (wall) {
        o.w = gb.w;
      } else {
        const float inv_m = 1.0f / vs.w;
        const float px = vs.x - a.h * g.gx, py = vs.y - a.h * g.gy, pz = vs.z - a.h * g.gz;  // p / m
        o = make_float4(gb.x * inv_m, gb.y * inv_m, gb.z * inv_m,
                        gb.w - (gb.x * px + gb.y * py + gb.z * pz) * inv_m);
      }
    }
    a.gbar[node] = o;
  }
}

// ---- corotated stress adjoint ----------------------------------------------
// tau = 2 mu (F F^T - R F^T) + lam J (J - 1) I, R = U V^T from F = U S V^T.
// For taubar (full 3x3):
//   Fbar = 2 mu (taubar + taubar^T) F - 2 mu (taubar^T R + U X V^T)
//          + lam (2 J - 1) tr(taubar) cof(F),
// where Rbar = taubar F, Y = U^T Rbar V and X_ij = (Y_ij - Y_ji) / (s_i + s_j)
// (the adjoint of the polar rotation, dR = U Omega V^T with
// Omega_ij = (M_ij - M_ji) / (s_i + s_j), M = U^T dF V);
//   mubar = 2 sum_a s_a (s_a - 1) u_a^T taubar u_a,  lambar = tr(taubar) J (J - 1).
__device__ void corotated_adjoint(const float (&F)[9], const float (&tb)[9], float mu, float lam,
                                  float (&Fb)[9], float& mub, float& lamb) {
  Polar P;
  polar_svd(F, P);
  const float* U = P.U;
  const float* V = P.V;
  float R[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      R[3 * r + c] = U[3 * r] * V[3 * c] + U[3 * r + 1] * V[3 * c + 1] + U[3 * r + 2] * V[3 * c + 2];
  const float a = P.sm1[0], b = P.sm1[1], c = P.sm1[2];
  const float jm1 = a + b + c + a * b + a * c + b * c + a * b * c;  // J - 1
  const float J = 1.0f + jm1;
  // Rbar = taubar F ; Y = U^T Rbar V
  float Rb[9], T1[9], Y[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q)
      Rb[3 * r + q] = tb[3 * r] * F[q] + tb[3 * r + 1] * F[3 + q] + tb[3 * r + 2] * F[6 + q];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q)
      T1[3 * r + q] = Rb[3 * r] * V[q] + Rb[3 * r + 1] * V[3 + q] + Rb[3 * r + 2] * V[6 + q];  // Rbar V
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) Y[3 * r + q] = U[r] * T1[q] + U[3 + r] * T1[3 + q] + U[6 + r] * T1[6 + q];
  float X[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q)
      if (r != q) {
        float den = P.s[r] + P.s[q];
        if (fabsf(den) < 1e-6f) den = den < 0.f ? -1e-6f : 1e-6f;
        X[3 * r + q] = (Y[3 * r + q] - Y[3 * q + r]) / den;
      }
  // U X V^T
  float XV[9], UXV[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) XV[3 * r + q] = X[3 * r] * V[3 * q] + X[3 * r + 1] * V[3 * q + 1] + X[3 * r + 2] * V[3 * q + 2];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) UXV[3 * r + q] = U[3 * r] * XV[q] + U[3 * r + 1] * XV[3 + q] + U[3 * r + 2] * XV[6 + q];
  const float cof[9] = {F[4] * F[8] - F[5] * F[7], F[5] * F[6] - F[3] * F[8], F[3] * F[7] - F[4] * F[6],
                        F[2] * F[7] - F[1] * F[8], F[0] * F[8] - F[2] * F[6], F[1] * F[6] - F[0] * F[7],
                        F[1] * F[5] - F[2] * F[4], F[2] * F[3] - F[0] * F[5], F[0] * F[4] - F[1] * F[3]};
  const float tr = tb[0] + tb[4] + tb[8];
  const float cj = lam * (2.0f * J - 1.0f) * tr;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float sF = 0.f, tR = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        sF += (tb[3 * r + k] + tb[3 * k + r]) * F[3 * k + q];
        tR += tb[3 * k + r] * R[3 * k + q];
      }
      Fb[3 * r + q] = 2.0f * mu * (sF - tR - UXV[3 * r + q]) + cj * cof[3 * r + q];
    }
  float m = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float utu = 0.f;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int q = 0; q < 3; ++q) utu += U[3 * r + k] * tb[3 * r + q] * U[3 * q + k];
    m += P.s[k] * P.sm1[k] * utu;
  }
  mub = 2.0f * m;
  lamb = tr * J * jm1;
}

// ---- P2G adjoint -----------------------------------------------------------
// With (pbar_i, mbar_i) from the grid adjoint and q_i = m_p v_p + A_p d_i:
//   vbar += m_p sum w pbar_i ;  Abar = sum w pbar_i d_i^T
//   xbar += sum grad w_i (pbar_i . q_i + mbar_i m_p) - A_p^T sum w pbar_i
//   Cbar += m_p Abar ;  taubar = -h k V_p Abar -> Fbar (corotated_adjoint)
__global__ void __launch_bounds__(kThreads) k_p2g_adjoint(BackwardArgs a) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const GridDev& g = a.g;
  const size_t n = (size_t)a.n;
  float mub = 0.f, lamb = 0.f;
  int grp = -1;
  if (i < a.n) {
    const float xp[3] = {a.P.x(0)[i], a.P.x(1)[i], a.P.x(2)[i]};
    StencilGrad S;
    stencil_grad(g, xp[0], xp[1], xp[2], S);
    if (stencil_inside(g, S.s)) {
      grp = a.P.grp[i];
      const DevGroup gr = a.groups[grp];
      const float kk = 4.0f * g.inv_dx * g.inv_dx;
      const float sc = a.h * kk * gr.vol;
      float tau[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) tau[c] = a.P.tau(c)[i];
      const float tf[9] = {tau[0], tau[3], tau[4], tau[3], tau[1], tau[5], tau[4], tau[5], tau[2]};
      float A[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) A[c] = gr.mass * a.P.C(c)[i] - sc * tf[c];
      const float mv[3] = {gr.mass * a.P.v(0)[i], gr.mass * a.P.v(1)[i], gr.mass * a.P.v(2)[i]};
      float s1[3] = {0.f, 0.f, 0.f}, Ab[9], xg[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int c = 0; c < 9; ++c) Ab[c] = 0.f;
      for (int cz = 0; cz < 3; ++cz)
        for (int cy = 0; cy < 3; ++cy)
#pragma unroll
          for (int cx = 0; cx < 3; ++cx) {
            const float w = S.s.w[0][cx] * S.s.w[1][cy] * S.s.w[2][cz];
            const float gw[3] = {S.dw[0][cx] * S.s.w[1][cy] * S.s.w[2][cz],
                                 S.s.w[0][cx] * S.dw[1][cy] * S.s.w[2][cz],
                                 S.s.w[0][cx] * S.s.w[1][cy] * S.dw[2][cz]};
            const float d[3] = {(cx - S.s.fx[0]) * g.dx, (cy - S.s.fx[1]) * g.dx, (cz - S.s.fx[2]) * g.dx};
            const float4 pb = __ldg(a.gbar + node_index(g, S.s.base[0] + cx, S.s.base[1] + cy, S.s.base[2] + cz));
            const float pv[3] = {pb.x, pb.y, pb.z};
            float pq = 0.f;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
              s1[r] += w * pv[r];
              pq += pv[r] * (mv[r] + A[3 * r] * d[0] + A[3 * r + 1] * d[1] + A[3 * r + 2] * d[2]);
#pragma unroll
              for (int c = 0; c < 3; ++c) Ab[3 * r + c] += w * pv[r] * d[c];
            }
            const float t = pq + pb.w * gr.mass;
#pragma unroll
            for (int c = 0; c < 3; ++c) xg[c] += t * gw[c];
          }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float ATs = A[c] * s1[0] + A[3 + c] * s1[1] + A[6 + c] * s1[2];
        a.bout[c * n + i] += xg[c] - ATs;
        a.bout[(3 + c) * n + i] += gr.mass * s1[c];
      }
#pragma unroll
      for (int c = 0; c < 9; ++c) a.bout[(6 + c) * n + i] += gr.mass * Ab[c];
      float F[9], tb[9], Fb[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        F[c] = a.P.F(c)[i];
        tb[c] = -sc * Ab[c];
      }
      if (gr.model == MPM_COROTATED)
        corotated_adjoint(F, tb, gr.mu_l, gr.lam, Fb, mub, lamb);
      else
        hencky_adjoint(F, tb, gr.mu_l, gr.lam, Fb, mub, lamb);
#pragma unroll
      for (int c = 0; c < 9; ++c) a.bout[(15 + c) * n + i] += Fb[c];
    }
  }
  // per-group parameter adjoints: warp sums when the warp shares a group
  // (particles of a group are contiguous in most orders), else per lane
  const bool same = __all_sync(0xffffffffu, grp == __shfl_sync(0xffffffffu, grp, 0));
  if (same) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mub += __shfl_xor_sync(0xffffffffu, mub, o);
      lamb += __shfl_xor_sync(0xffffffffu, lamb, o);
    }
    if (lane == 0 && grp >= 0) {
      atomicAdd(a.mat_bar + 2 * grp, (double)mub);
      atomicAdd(a.mat_bar + 2 * grp + 1, (double)lamb);
    }
  } else if (grp >= 0) {
    atomicAdd(a.mat_bar + 2 * grp, (double)mub);
    atomicAdd(a.mat_bar + 2 * grp + 1, (double)lamb);
  }
}

// The per-substep counters that G2P resets in the forward pass (the
// backward replays P2G, grid and solve without G2P).
__global__ void k_reset_counters(GridArrays G, Contacts C, unsigned* bar) {
  *C.count = 0;
  *G.n_act = 0;
  *G.n_cnodes = 0;
  *G.pstar2 = 0.0;
  bar[0] = 0u;  // the solve's 64-bit barrier counter
  bar[1] = 0u;
}

// ---- solutions of the taped substeps ---------------------------------------
// After each recorded solve, the velocities of its contact nodes (the only
// nodes the solve changes) are appended to a pool as (v.x, v.y, v.z, node),
// one record (offset, count) per substep, in order; count = -1 marks a
// substep that did not fit. mpm_backward scatters a record back over v* to
// start that substep's replayed solves at their solution.
__global__ void k_tape_alloc(GridArrays G, int* __restrict__ counters, int2* __restrict__ recs,
                             int rec_cap, int pool_cap) {
  const int n = min(*G.n_cnodes, G.cnodes_cap);
  const int r = counters[1];
  const int off = counters[0];
  const bool fits = off + n <= pool_cap;
  if (r < rec_cap) recs[r] = make_int2(off, fits ? n : -1);
  if (fits) counters[0] = off + n;
  counters[1] = r + 1;
}

// Records name nodes by grid block * 64 + cell, which a replayed substep of
// a sparse grid maps to its own storage (the same blocks are active there).
__global__ void k_tape_copy(GridDev g, GridArrays G, const int* __restrict__ counters,
                            const int2* __restrict__ recs, int rec_cap, float4* __restrict__ pool) {
  const int r = counters[1] - 1;
  if (r >= rec_cap) return;
  const int2 rec = recs[r];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < rec.y; t += gridDim.x * blockDim.x) {
    const int node = G.cnodes[t];
    const float4 v = G.v[node];
    const int id = g.slot ? G.act[node >> 6] * kBlockNodes + (node & 63) : node;
    pool[rec.x + t] = make_float4(v.x, v.y, v.z, __int_as_float(id));
  }
}

__global__ void k_tape_warm(GridDev g, GridArrays G, const int2* __restrict__ recs, int r,
                            const float4* __restrict__ pool) {
  const int2 rec = recs[r];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < rec.y; t += gridDim.x * blockDim.x) {
    const float4 q = pool[rec.x + t];
    const int id = __float_as_int(q.w);
    const int sb = g.slot ? g.slot[id >> 6] : id >> 6;
    if (sb < 0) continue;  // (a block no longer active: not warm-started)
    float4* v = G.v + sb * kBlockNodes + (id & 63);
    const float w = v->w;  // the Dirichlet flag of this substep's grid update
    *v = make_float4(q.x, q.y, q.z, w);
  }
}

// slot_of[pid[i]] = i
__global__ void k_slot_map(const uint32_t* __restrict__ pid, int n, int* __restrict__ slot_of) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) slot_of[pid[i]] = i;
}

// caller layout (id order; x, v [n][3], C, F [n][3][3]) <-> planes in slot order
__global__ void k_bar_in(const uint32_t* __restrict__ pid, int n, const float* __restrict__ x,
                         const float* __restrict__ v, const float* __restrict__ C,
                         const float* __restrict__ F, float* __restrict__ bar) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t id = pid[i], nn = (size_t)n;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    bar[c * nn + i] = x ? x[3 * id + c] : 0.f;
    bar[(3 + c) * nn + i] = v ? v[3 * id + c] : 0.f;
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    bar[(6 + c) * nn + i] = C ? C[9 * id + c] : 0.f;
    bar[(15 + c) * nn + i] = F ? F[9 * id + c] : 0.f;
  }
}

__global__ void k_bar_out(const uint32_t* __restrict__ pid, int n, const float* __restrict__ bar,
                          float* __restrict__ x, float* __restrict__ v, float* __restrict__ C,
                          float* __restrict__ F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t id = pid[i], nn = (size_t)n;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (x) x[3 * id + c] = bar[c * nn + i];
    if (v) v[3 * id + c] = bar[(3 + c) * nn + i];
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    if (C) C[9 * id + c] = bar[(6 + c) * nn + i];
    if (F) F[9 * id + c] = bar[(15 + c) * nn + i];
  }
}

}  // namespace

void launch_g2p_adjoint(const BackwardArgs& a, cudaStream_t s) {
  if (a.n > 0) k_g2p_adjoint<<<(a.n + kThreads - 1) / kThreads, kThreads, 0, s>>>(a);
}

void launch_grid_adjoint(const BackwardArgs& a, int num_sms, cudaStream_t s) {
  k_grid_adjoint<<<num_sms * 8, kThreads, 0, s>>>(a);
}

void launch_p2g_adjoint(const BackwardArgs& a, cudaStream_t s) {
  if (a.n > 0) k_p2g_adjoint<<<(a.n + kThreads - 1) / kThreads, kThreads, 0, s>>>(a);
}

void launch_reset_counters(const GridArrays& G, const Contacts& C, unsigned* bar, cudaStream_t s) {
  k_reset_counters<<<1, 1, 0, s>>>(G, C, bar);
}

void launch_tape_save(const GridDev& g, const GridArrays& G, int* counters, int2* recs, int rec_cap, float4* pool,
                      int pool_cap, int num_sms, cudaStream_t s) {
  k_tape_alloc<<<1, 1, 0, s>>>(G, counters, recs, rec_cap, pool_cap);
  k_tape_copy<<<num_sms, 256, 0, s>>>(g, G, counters, recs, rec_cap, pool);
}

void launch_tape_warm(const GridDev& g, const GridArrays& G, const int2* recs, int r, const float4* pool, int num_sms,
                      cudaStream_t s) {
  k_tape_warm<<<num_sms, 256, 0, s>>>(g, G, recs, r, pool);
}

void launch_slot_map(const Particles& P, int n, int* slot_of, cudaStream_t s) {
  if (n > 0) k_slot_map<<<(n + 255) / 256, 256, 0, s>>>(P.pid, n, slot_of);
}

void launch_bar_in(const Particles& P, int n, const float* x, const float* v, const float* C,
                   const float* F, float* bar, cudaStream_t s) {
  if (n > 0) k_bar_in<<<(n + 255) / 256, 256, 0, s>>>(P.pid, n, x, v, C, F, bar);
}

void launch_bar_out(const Particles& P, int n, const float* bar, float* x, float* v, float* C,
                    float* F, cudaStream_t s) {
  if (n > 0) k_bar_out<<<(n + 255) / 256, 256, 0, s>>>(P.pid, n, bar, x, v, C, F);
}

}  // namespace mpmcr
