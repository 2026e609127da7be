// g2p.cu -- grid-to-particle transfer with the constitutive update (Sec. V-A
// op (3), MLS-MPM): v_p = sum_i w v_i, C_p = (4/dx^2) sum_i w v_i (x_i - x_p)^T,
// x_p += h v_p, F_p <- (I + h C_p) F_p, then the Drucker-Prager return map for
// sand, fused with the stress update: the Kirchhoff stress of the new F is
// stored for the next P2G, so one SVD per particle and substep serves both
// the plasticity and the stress. One thread per particle; particle planes are read and written with
// coalesced loads and stores, grid velocities are gathered from L2.
//
// Block 0 also closes the substep: it records the contact / active-block
// counts for diagnostics and resets the per-substep counters, the solve's
// barrier word, so the next substep needs no memset.
#include "kernels.h"

namespace mpmcr {

namespace {

constexpr int kThreads = 256;

// Block `block` of G2P over one scene's particles, blockDim.x particles (a
// thread block of the single-scene launch, or a work item of the batched one).
template <bool kDense>
__device__ __forceinline__ void g2p_block(const G2PArgs& a, int block) {
  const GridDev& g = a.g;
  if (block == 0) {
    if (threadIdx.x == 0) {
      const int count = *a.C.count;
      const int nc = count < a.C.cap ? count : a.C.cap;
      a.stats->last_contacts = nc;
      atomicMax(&a.stats->contacts_max, nc);
      atomicAdd(&a.stats->contacts_total, (unsigned long long)nc);
      atomicAdd(&a.stats->substeps, 1);
      *a.C.count = 0;
      *a.G.n_act = 0;
      *a.G.n_cnodes = 0;
      *a.G.pstar2 = 0.0;
    }
    if (threadIdx.x < 2) a.bar[threadIdx.x] = 0u;  // the solve's 64-bit barrier counter
  }
  const int i = block * (int)blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const float xp[3] = {a.P.x(0)[i], a.P.x(1)[i], a.P.x(2)[i]};
  Stencil s;
  stencil(g, xp[0], xp[1], xp[2], s);
  if (!stencil_inside(g, s)) return;  // reported by P2G
  // dense node address = ax[cx] + ay[cy] + az[cz] (block-major: each axis
  // contributes its block and its cell within the block)
  int ax[3], ay[3], az[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int ix = s.base[0] + c, iy = s.base[1] + c, iz = s.base[2] + c;
    ax[c] = (ix >> 2) * kBlockNodes + (ix & 3);
    ay[c] = (iy >> 2) * (g.nbx * kBlockNodes) + ((iy & 3) << 2);
    az[c] = (iz >> 2) * (g.nbx * g.nby * kBlockNodes) + ((iz & 3) << 4);
  }
  // x and y components go in pairs (paired FP32 ops): v_xy, and the x, y
  // rows of B = sum w v (x_i - x_p)^T as (B_xx, B_yx), (B_xy, B_yy), (B_xz, B_yz)
  float2 vxy = make_float2(0.f, 0.f), B0 = vxy, B1 = vxy, B2 = vxy;
  float vz = 0.f, Bz0 = 0.f, Bz1 = 0.f, Bz2 = 0.f;
  const float dx0[3] = {(0.f - s.fx[0]) * g.dx, (1.f - s.fx[0]) * g.dx, (2.f - s.fx[0]) * g.dx};
#pragma unroll
  for (int cz = 0; cz < 3; ++cz) {
    const float dz = (cz - s.fx[2]) * g.dx;
#pragma unroll
    for (int cy = 0; cy < 3; ++cy) {
      const float dy = (cy - s.fx[1]) * g.dx;
      const float wyz = s.w[1][cy] * s.w[2][cz];
      // the row's sums of w v and of w v (x_i - x_p), then its dy, dz terms
      float2 Sxy = make_float2(0.f, 0.f), Txy = Sxy;
      float Sz = 0.f, Tz = 0.f;
#pragma unroll
      for (int cx = 0; cx < 3; ++cx) {
        const float w = s.w[0][cx] * wyz;
        const int node = kDense ? az[cz] + ay[cy] + ax[cx]
                                : node_index(g, s.base[0] + cx, s.base[1] + cy, s.base[2] + cz);
        const float4 v = __ldg(a.G.v + node);
        const float2 wv = __fmul2_rn(make_float2(w, w), make_float2(v.x, v.y));
        const float wvz = w * v.z;
        Sxy = __fadd2_rn(Sxy, wv);
        Txy = __ffma2_rn(wv, make_float2(dx0[cx], dx0[cx]), Txy);
        Sz += wvz;
        Tz = fmaf(wvz, dx0[cx], Tz);
      }
      vxy = __fadd2_rn(vxy, Sxy);
      B0 = __fadd2_rn(B0, Txy);
      B1 = __ffma2_rn(Sxy, make_float2(dy, dy), B1);
      B2 = __ffma2_rn(Sxy, make_float2(dz, dz), B2);
      vz += Sz;
      Bz0 += Tz;
      Bz1 = fmaf(Sz, dy, Bz1);
      Bz2 = fmaf(Sz, dz, Bz2);
    }
  }
  const float vp[3] = {vxy.x, vxy.y, vz};
  const float Bm[9] = {B0.x, B1.x, B2.x, B0.y, B1.y, B2.y, Bz0, Bz1, Bz2};
  const float dinv = 4.0f * g.inv_dx * g.inv_dx;
  const float h = a.h;
  float C[9], F[9], Fn[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    C[c] = dinv * Bm[c];
    F[c] = a.P.F(c)[i];
  }
  const DevGroup gr = a.groups[a.P.grp[i]];
  float tau[6];
  if (gr.model == MPM_CLOTH) {
    // the mesh carries the cloth's elasticity: F stays, no stress
#pragma unroll
    for (int c = 0; c < 9; ++c) Fn[c] = F[c];
#pragma unroll
    for (int c = 0; c < 6; ++c) tau[c] = 0.f;
  } else {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        Fn[3 * r + c] =
            F[3 * r + c] + h * (C[3 * r] * F[c] + C[3 * r + 1] * F[3 + c] + C[3 * r + 2] * F[6 + c]);
    constitutive_update(gr, Fn, tau);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    a.P.v(c)[i] = vp[c];
    a.P.x(c)[i] = xp[c] + h * vp[c];
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    a.P.C(c)[i] = C[c];
    a.P.F(c)[i] = Fn[c];
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) a.P.tau(c)[i] = tau[c];
}

// kDense: a dense grid's node addresses (no block-table lookup)
template <bool kDense>
__global__ void __launch_bounds__(kThreads, 4) k_g2p(G2PArgs a) {
  g2p_block<kDense>(a, blockIdx.x);
}

// Batched: thread block b is block work[b].y of scene work[b].x
__global__ void __launch_bounds__(512, 2) k_g2p_batch(const G2PArgs* __restrict__ args,
                                                      const int2* __restrict__ work) {
  __shared__ G2PArgs s_a;
  const int2 wk = work[blockIdx.x];
  load_args(args + wk.x, s_a);
  __syncthreads();
  g2p_block<true>(s_a, wk.y);  // (batches take dense grids)
}

}  // namespace

void launch_g2p(const G2PArgs& a, cudaStream_t s) {
  const int blocks = a.n > 0 ? (a.n + kThreads - 1) / kThreads : 1;
  if (a.g.slot)
    k_g2p<false><<<blocks, kThreads, 0, s>>>(a);
  else
    k_g2p<true><<<blocks, kThreads, 0, s>>>(a);
}

void launch_g2p_batch(const G2PArgs* args, const int2* work, int n_work, int threads,
                      cudaStream_t s) {
  if (n_work > 0) k_g2p_batch<<<n_work, threads, 0, s>>>(args, work);
}

}  // namespace mpmcr
