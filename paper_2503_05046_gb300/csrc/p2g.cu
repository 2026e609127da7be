// p2g.cu -- particle-to-grid transfer of the free-motion solve (Eq. (6),
// MLS-MPM with quadratic B-splines) fused with contact registration
// (Sec. V-B: one contact point per particle inside a rigid geometry, at the
// start of the substep).
//
// GB300 layout: each thread block takes a contiguous chunk of block-sorted
// particles, finds the bounding box of their stencils and accumulates mass and
// momentum into a shared-memory tile of that box. Lanes of a warp whose
// particles share a base cell first combine their contributions with a
// segmented shuffle reduction (the warp-level pre-reduction of Sec. V-A), so
// one shared-memory atomic per node and run is issued. The tile is
// then flushed with one 16-byte vector reduction (red.global.add.v4.f32) per
// touched node. When the chunk's box exceeds the tile (the Morton order jumps
// at a coarse cell boundary, or the chunk straddles the edge of the material)
// each warp uses its own sub-tile of its own box; only a warp whose box is
// still too large reduces straight into the grid. The Kirchhoff stress comes
// precomputed from the previous G2P, so no SVD runs here. Particle planes are
// read with coalesced 4-byte loads.
#include "kernels.h"

namespace mpmcr {

namespace {

constexpr int kTileCap = 2048;  // nodes in the shared tile (32 KB)
constexpr int kThreads = 256;
constexpr int kWarpTileCap = kTileCap / (kThreads / 32);  // 256 nodes per warp

template <int ITEMS>
__global__ void __launch_bounds__(kThreads, 3) k_p2g(P2GArgs a) {
  __shared__ float t_m[kTileCap], t_px[kTileCap], t_py[kTileCap], t_pz[kTileCap];
  __shared__ DevBody s_body[kMaxBodies];
  __shared__ int s_min[3], s_max[3];
  __shared__ unsigned s_cand;
  const GridDev& g = a.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int first = blockIdx.x * kThreads * ITEMS;

  if (tid < 3) { s_min[tid] = 0x7fffffff; s_max[tid] = -0x7fffffff; }
  for (int i = tid; i < a.nb * (int)(sizeof(DevBody) / 4); i += kThreads)
    reinterpret_cast<float*>(s_body)[i] = reinterpret_cast<const float*>(a.bodies)[i];
  __syncthreads();

  // stencils of this thread's particles; bounding boxes of the warp and chunk
  // (the stencils are recomputed below rather than held in registers)
  bool valid[ITEMS];
  int lo[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, hi[3] = {-0x7fffffff, -0x7fffffff, -0x7fffffff};
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const int i = first + it * kThreads + tid;
    valid[it] = i < a.n;
    if (valid[it]) {
      Stencil st;
      stencil(g, a.P.x(0)[i], a.P.x(1)[i], a.P.x(2)[i], st);
      if (!stencil_inside(g, st)) {
        valid[it] = false;
        atomicOr(a.status, kStOutOfDomain);
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          lo[c] = min(lo[c], st.base[c]);
          hi[c] = max(hi[c], st.base[c]);
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[c] = min(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
      hi[c] = max(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) { atomicMin(&s_min[c], lo[c]); atomicMax(&s_max[c], hi[c]); }
  }
  __syncthreads();
  const bool any = s_max[0] >= s_min[0];
  const int cx0 = s_min[0], cy0 = s_min[1], cz0 = s_min[2];
  const int cex = any ? s_max[0] - cx0 + 3 : 0, cey = any ? s_max[1] - cy0 + 3 : 0,
            cez = any ? s_max[2] - cz0 + 3 : 0;
  const bool block_tile = any && cex * cey * cez <= kTileCap;
  // the tile this thread accumulates into: the chunk's, or its warp's
  const bool wany = hi[0] >= lo[0];
  const int wex = wany ? hi[0] - lo[0] + 3 : 0, wey = wany ? hi[1] - lo[1] + 3 : 0,
            wez = wany ? hi[2] - lo[2] + 3 : 0;
  const bool warp_tile = !block_tile && wany && wex * wey * wez <= kWarpTileCap;
  const bool use_tile = block_tile || warp_tile;
  const int b0 = block_tile ? cx0 : lo[0], b1 = block_tile ? cy0 : lo[1], b2 = block_tile ? cz0 : lo[2];
  const int ex = block_tile ? cex : wex, ey = block_tile ? cey : wey, ez = block_tile ? cez : wez;
  const int toff = block_tile ? 0 : warp * kWarpTileCap;
  const int tile_n = use_tile ? ex * ey * ez : 0;
  if (block_tile) {
    for (int t = tid; t < tile_n; t += kThreads) { t_m[t] = 0.f; t_px[t] = 0.f; t_py[t] = 0.f; t_pz[t] = 0.f; }
  } else if (warp_tile) {
    for (int t = lane; t < tile_n; t += 32) {
      t_m[toff + t] = 0.f; t_px[toff + t] = 0.f; t_py[toff + t] = 0.f; t_pz[toff + t] = 0.f;
    }
  }
  if (any && !block_tile && tid == 0) atomicAdd(&a.stats->p2g_global_chunks, 1);
  // bodies that may hold a particle of this chunk: the signed distance is
  // 1-Lipschitz, so a body whose distance at the box centre exceeds the half
  // diagonal cannot contain any point of the box
  if (tid < 32) {
    bool cand = false;
    if (any && tid < a.nb) {
      const float c0 = g.ox + g.dx * (0.5f * (cx0 + s_max[0]) + 1.0f);
      const float c1 = g.oy + g.dx * (0.5f * (cy0 + s_max[1]) + 1.0f);
      const float c2 = g.oz + g.dx * (0.5f * (cz0 + s_max[2]) + 1.0f);
      const float h0 = 0.5f * g.dx * (s_max[0] - cx0 + 1), h1 = 0.5f * g.dx * (s_max[1] - cy0 + 1),
                  h2 = 0.5f * g.dx * (s_max[2] - cz0 + 1);
      float nrm[3];
      const float phi = body_sdf(s_body[tid], c0, c1, c2, nrm);
      cand = phi <= sqrtf(h0 * h0 + h1 * h1 + h2 * h2) * 1.001f + 1e-6f;
    }
    const unsigned m = __ballot_sync(0xffffffffu, cand);
    if (tid == 0) s_cand = m;
  }
  __syncthreads();
  const unsigned cand = s_cand;
  const float h = a.h;
  const float dinv = 4.0f * g.inv_dx * g.inv_dx;

  // not unrolled: one copy of the large per-particle body keeps the
  // instruction footprint small
#pragma unroll 1
  for (int it = 0; it < ITEMS; ++it) {
    const int i = first + it * kThreads + tid;
    Stencil st = Stencil{};
    if (valid[it]) stencil(g, a.P.x(0)[i], a.P.x(1)[i], a.P.x(2)[i], st);
    if (use_tile) {
      // warp-level pre-reduction (Sec. V-A): lanes whose stencils share a
      // base cell (adjacent after the cell-ordered sort) add their 27 node
      // contributions with a segmented shuffle reduction, and only the first
      // lane of each run issues the shared-memory atomics
      const Stencil& s = st;
      float mass = 0.f, mvx = 0.f, mvy = 0.f, mvz = 0.f;
      float A[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) A[c] = 0.f;
      int l0 = 0, l1 = 0, l2 = 0, key = -1 - lane;
      if (valid[it]) {
        const DevGroup gr = a.groups[a.P.grp[i]];
        float tau[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) tau[c] = a.P.tau(c)[i];
        // affine momentum m C - h (4/dx^2) V tau
        const float sc = h * dinv * gr.vol;
        const float tf[9] = {tau[0], tau[3], tau[4], tau[3], tau[1], tau[5], tau[4], tau[5], tau[2]};
#pragma unroll
        for (int c = 0; c < 9; ++c) A[c] = gr.mass * a.P.C(c)[i] - sc * tf[c];
        mass = gr.mass;
        mvx = gr.mass * a.P.v(0)[i];
        mvy = gr.mass * a.P.v(1)[i];
        mvz = gr.mass * a.P.v(2)[i];
        l0 = s.base[0] - b0;
        l1 = s.base[1] - b1;
        l2 = s.base[2] - b2;
        key = (l2 * ey + l1) * ex + l0;
      }
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      const int head = __ffs(peers) - 1, seg_end = 31 - __clz(peers);
      const unsigned run = (0xffffffffu >> (31 - seg_end)) & (0xffffffffu << head);
      const bool contiguous = __all_sync(0xffffffffu, peers == run);
      const int len = contiguous ? seg_end - head + 1 : 1;
      const int maxlen = __reduce_max_sync(0xffffffffu, (unsigned)len);
      const int steps = maxlen > 1 ? 32 - __clz(maxlen - 1) : 0;
      const bool issue = valid[it] && (!contiguous || lane == head);
#pragma unroll
      for (int cz = 0; cz < 3; ++cz) {
        const float dz = (cz - s.fx[2]) * g.dx;
#pragma unroll
        for (int cy = 0; cy < 3; ++cy) {
          const float dy = (cy - s.fx[1]) * g.dx;
          const float wyz = s.w[1][cy] * s.w[2][cz];
          const int row = toff + ((l2 + cz) * ey + (l1 + cy)) * ex + l0;
#pragma unroll
          for (int cx = 0; cx < 3; ++cx) {
            const float dxp = (cx - s.fx[0]) * g.dx;
            const float w = valid[it] ? s.w[0][cx] * wyz : 0.f;
            float q0 = w * mass;
            float q1 = w * (mvx + A[0] * dxp + A[1] * dy + A[2] * dz);
            float q2 = w * (mvy + A[3] * dxp + A[4] * dy + A[5] * dz);
            float q3 = w * (mvz + A[6] * dxp + A[7] * dy + A[8] * dz);
#pragma unroll
            for (int k = 0; k < 5; ++k) {
              if (k < steps) {
                const int off = 1 << k;
                const float r0 = __shfl_down_sync(0xffffffffu, q0, off);
                const float r1 = __shfl_down_sync(0xffffffffu, q1, off);
                const float r2 = __shfl_down_sync(0xffffffffu, q2, off);
                const float r3 = __shfl_down_sync(0xffffffffu, q3, off);
                if (lane + off <= seg_end) { q0 += r0; q1 += r1; q2 += r2; q3 += r3; }
              }
            }
            if (issue) {
              const int t = row + cx;
              atomicAdd(&t_m[t], q0);
              atomicAdd(&t_px[t], q1);
              atomicAdd(&t_py[t], q2);
              atomicAdd(&t_pz[t], q3);
            }
          }
        }
      }
    } else if (valid[it]) {
      const Stencil& s = st;
      const DevGroup gr = a.groups[a.P.grp[i]];
      const float vp[3] = {a.P.v(0)[i], a.P.v(1)[i], a.P.v(2)[i]};
      float tau[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) tau[c] = a.P.tau(c)[i];
      // affine momentum m C - h (4/dx^2) V tau
      const float sc = h * dinv * gr.vol;
      const float tf[9] = {tau[0], tau[3], tau[4], tau[3], tau[1], tau[5], tau[4], tau[5], tau[2]};
      float A[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) A[c] = gr.mass * a.P.C(c)[i] - sc * tf[c];
      const float mvx = gr.mass * vp[0], mvy = gr.mass * vp[1], mvz = gr.mass * vp[2];
#pragma unroll
      for (int cz = 0; cz < 3; ++cz) {
        const float dz = (cz - s.fx[2]) * g.dx;
#pragma unroll
        for (int cy = 0; cy < 3; ++cy) {
          const float dy = (cy - s.fx[1]) * g.dx;
          const float wyz = s.w[1][cy] * s.w[2][cz];
#pragma unroll
          for (int cx = 0; cx < 3; ++cx) {
            const float dxp = (cx - s.fx[0]) * g.dx;
            const float w = s.w[0][cx] * wyz;
            const int node = node_index(g, s.base[0] + cx, s.base[1] + cy, s.base[2] + cz);
            red_add_v4(a.G.mp + node, w * gr.mass, w * (mvx + A[0] * dxp + A[1] * dy + A[2] * dz),
                       w * (mvy + A[3] * dxp + A[4] * dy + A[5] * dz),
                       w * (mvz + A[6] * dxp + A[7] * dy + A[8] * dz));
          }
        }
      }
      // mark the (up to 8) blocks of this stencil
#pragma unroll
      for (int cz = 0; cz < 2; ++cz)
#pragma unroll
        for (int cy = 0; cy < 2; ++cy)
#pragma unroll
          for (int cx = 0; cx < 2; ++cx) {
            const int bi = (s.base[0] + 2 * cx) >> 2, bj = (s.base[1] + 2 * cy) >> 2,
                      bk = (s.base[2] + 2 * cz) >> 2;
            a.G.mark[(bk * g.nby + bj) * g.nbx + bi] = 1;
          }
    }
    // contact registration: warp-aggregated append, one contact per
    // (particle, body) pair with the particle strictly inside
    if (cand) {
      float xp[3] = {0.f, 0.f, 0.f}, vp[3] = {0.f, 0.f, 0.f};
      if (valid[it]) {
#pragma unroll
        for (int c = 0; c < 3; ++c) { xp[c] = a.P.x(c)[i]; vp[c] = a.P.v(c)[i]; }
      }
      for (int b = 0; b < a.nb; ++b) {
        if (!((cand >> b) & 1u)) continue;
        float nrm[3] = {0.f, 0.f, 1.f};
        float phi = 1.0f;
        if (valid[it]) {
          phi = body_sdf(s_body[b], xp[0], xp[1], xp[2], nrm);
          // near the surface the sign and the depth come from FP64
          if (phi < 1e-6f + 1e-6f * (fabsf(xp[0]) + fabsf(xp[1]) + fabsf(xp[2])))
            phi = (float)body_sdf_f64(s_body[b], xp[0], xp[1], xp[2]);
        }
        const bool hit = valid[it] && phi < 0.0f;
        const unsigned mask = __ballot_sync(0xffffffffu, hit);
        if (mask == 0u) continue;
        const int leader = __ffs(mask) - 1;
        int slot0 = 0;
        if (lane == leader) slot0 = atomicAdd(a.C.count, __popc(mask));
        slot0 = __shfl_sync(0xffffffffu, slot0, leader);
        if (hit) {
          const int slot = slot0 + __popc(mask & ((1u << lane) - 1u));
          if (slot < a.C.cap) {
            const DevBody& bd = s_body[b];
            float vr[3];
            body_velocity(bd, xp[0], xp[1], xp[2], vr);
            const float vn0 = nrm[0] * (vp[0] - vr[0]) + nrm[1] * (vp[1] - vr[1]) + nrm[2] * (vp[2] - vr[2]);
            const float phi0 = -phi;
            const float n0 = normal_impulse(phi0, bd.k, bd.d, h, vn0);
            a.C.xp[slot] = make_float4(xp[0], xp[1], xp[2], phi0);
            a.C.nrm[slot] = make_float4(nrm[0], nrm[1], nrm[2], n0);
            a.C.bias[slot] = make_float4(-vr[0], -vr[1], -vr[2], 0.f);
            a.C.id[slot] = make_int2((int)a.P.pid[i], b);
          } else {
            atomicOr(a.status, kStCapacity);
          }
        }
      }
    }
  }
  __syncthreads();
  if (!use_tile) return;
  // flush: one vector reduction per touched node of the (chunk or warp) tile
  const int fstart = block_tile ? tid : lane, fstride = block_tile ? kThreads : 32;
  for (int t = fstart; t < tile_n; t += fstride) {
    const int q = toff + t;
    const float m = t_m[q];
    if (m != 0.0f || t_px[q] != 0.0f || t_py[q] != 0.0f || t_pz[q] != 0.0f) {
      const int lx = t % ex, r = t / ex, ly = r % ey, lz = r / ey;
      const int node = node_index(g, b0 + lx, b1 + ly, b2 + lz);
      red_add_v4(a.G.mp + node, m, t_px[q], t_py[q], t_pz[q]);
    }
  }
  // mark the 4^3 blocks the tile overlaps
  const int bx0 = b0 >> 2, by0 = b1 >> 2, bz0 = b2 >> 2;
  const int bnx = ((b0 + ex - 1) >> 2) - bx0 + 1, bny = ((b1 + ey - 1) >> 2) - by0 + 1,
            bnz = ((b2 + ez - 1) >> 2) - bz0 + 1;
  for (int t = fstart; t < bnx * bny * bnz; t += fstride) {
    const int qx = t % bnx, r = t / bnx, qy = r % bny, qz = r / bny;
    a.G.mark[((bz0 + qz) * g.nby + (by0 + qy)) * g.nbx + (bx0 + qx)] = 1;
  }
}

}  // namespace

void launch_p2g(const P2GArgs& a, int chunk, cudaStream_t s) {
  if (a.n <= 0) return;
  const int items = chunk / kThreads;
  if (items <= 1) {
    k_p2g<1><<<(a.n + kThreads - 1) / kThreads, kThreads, 0, s>>>(a);
  } else if (items == 2) {
    k_p2g<2><<<(a.n + 2 * kThreads - 1) / (2 * kThreads), kThreads, 0, s>>>(a);
  } else {
    k_p2g<4><<<(a.n + 4 * kThreads - 1) / (4 * kThreads), kThreads, 0, s>>>(a);
  }
}

}  // namespace mpmcr
