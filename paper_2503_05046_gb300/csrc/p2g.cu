// p2g.cu -- particle-to-grid transfer of the free-motion solve (Eq. (6),
// MLS-MPM with quadratic B-splines) fused with contact registration
// (Sec. V-B: one contact point per particle inside a rigid geometry, at the
// start of the substep).
//
// Two forms of the warp's work (MPM_OPT_P2G_FORM), same results up to
// rounding order:
//
// Gather (the default, k_p2g_g): the warp stages its particles' transfer
// data in shared memory and lane j sums node j of a cell's 27-node stencil
// over the particles of that cell, into a window of the 6^3 nodes one 4^3
// block's stencils reach, flushed with one red.global.add.v4.f32 per touched
// node when the walk leaves the block (details at p2g_gather_block).
//
// Scatter (k_p2g): each warp takes a contiguous run of 32 x ITEMS
// cell-sorted particles and accumulates their mass and momentum into a
// private shared-memory tile of the bounding box of their stencils. Lanes
// whose particles share a base cell first combine their 27 node
// contributions with a segmented shuffle reduction (the warp-level
// pre-reduction of Sec. V-A); the remaining lanes have distinct base cells,
// so within one node offset they touch distinct nodes and update the tile
// with plain read-modify-write. A warp whose box exceeds its tile reduces
// straight into the grid.
//
// The Kirchhoff stress comes precomputed from the previous G2P, so no SVD
// runs here.
#include "kernels.h"

namespace mpmcr {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kWarpTileCap = 384;  // nodes per warp tile (6 KB)

// dynamic shared memory: kWarps tiles of kWarpTileCap float4
constexpr size_t kDynSmem = sizeof(float4) * kWarps * kWarpTileCap;

// Whether body b may hold a point of the box with centre c and half extents
// h. The signed distance is 1-Lipschitz, so a body whose distance at c exceeds
// the half diagonal holds none. A body inside the ball of radius b.bound
// around its origin is at least |c - p| - bound away from c, so the ball is
// tried first (with slack, so it only rejects bodies the distance would
// reject too) and the signed distance, whose branch differs between the
// lanes' primitives, is evaluated only for the bodies that it leaves.
__device__ __forceinline__ bool box_may_touch(const DevBody& b, float c0, float c1, float c2,
                                              float h0, float h1, float h2) {
  const float thr = sqrtf(h0 * h0 + h1 * h1 + h2 * h2) * 1.001f + 1e-6f;
  const float r0 = c0 - b.p[0], r1 = c1 - b.p[1], r2 = c2 - b.p[2];
  const float lim = (b.bound + thr) * 1.0001f + 1e-5f;  // inf for an unbounded body
  if (r0 * r0 + r1 * r1 + r2 * r2 > lim * lim) return false;
  float nrm[3];
  return body_sdf(b, c0, c1, c2, nrm) <= thr;
}

// Block `block` of P2G over one scene's particles (a thread block of the
// single-scene launch, or a work item of the batched one).
template <int ITEMS>
__device__ __forceinline__ void p2g_block(const P2GArgs& a, int block) {
  extern __shared__ float4 s_tiles[];
  __shared__ DevBody s_body[kMaxBodies];
  const GridDev& g = a.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // this warp's particles: [first, first + 32 * ITEMS), lane-contiguous per item
  const int first = (block * kWarps + warp) * 32 * ITEMS;
  float4* tile = s_tiles + warp * kWarpTileCap;

  for (int i = tid; i < a.nb * (int)(sizeof(DevBody) / 4); i += kThreads)
    reinterpret_cast<float*>(s_body)[i] = reinterpret_cast<const float*>(a.bodies)[i];
  __syncthreads();
  if (first >= a.n) return;

  // bounding box of the warp's stencils (base nodes)
  bool valid[ITEMS];
  int lo[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, hi[3] = {-0x7fffffff, -0x7fffffff, -0x7fffffff};
#pragma unroll
  for (int it = 0; it < ITEMS; ++it) {
    const int i = first + it * 32 + lane;
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
    lo[c] = __reduce_min_sync(0xffffffffu, lo[c]);
    hi[c] = __reduce_max_sync(0xffffffffu, hi[c]);
  }
  const bool any = hi[0] >= lo[0];
  const int ex = any ? hi[0] - lo[0] + 3 : 0, ey = any ? hi[1] - lo[1] + 3 : 0,
            ez = any ? hi[2] - lo[2] + 3 : 0;
  const bool use_tile = any && ex * ey * ez <= kWarpTileCap;
  const int tile_n = use_tile ? ex * ey * ez : 0;
  for (int t = lane; t < tile_n; t += 32) tile[t] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (any && !use_tile && lane == 0) atomicAdd(&a.stats->p2g_global_chunks, 1);
  // bodies that may hold a particle of this warp: the signed distance is
  // 1-Lipschitz, so a body whose distance at the box centre exceeds the half
  // diagonal cannot contain any point of the box
  bool cand_b = false;
  if (any && lane < a.nb) {
    const float c0 = g.ox + g.dx * (0.5f * (lo[0] + hi[0]) + 1.0f);
    const float c1 = g.oy + g.dx * (0.5f * (lo[1] + hi[1]) + 1.0f);
    const float c2 = g.oz + g.dx * (0.5f * (lo[2] + hi[2]) + 1.0f);
    const float h0 = 0.5f * g.dx * (hi[0] - lo[0] + 1), h1 = 0.5f * g.dx * (hi[1] - lo[1] + 1),
                h2 = 0.5f * g.dx * (hi[2] - lo[2] + 1);
    cand_b = box_may_touch(s_body[lane], c0, c1, c2, h0, h1, h2);
  }
  const unsigned cand = __ballot_sync(0xffffffffu, cand_b);
  __syncwarp();
  const float h = a.h;
  const float dinv = 4.0f * g.inv_dx * g.inv_dx;

  // not unrolled: one copy of the large per-particle body keeps the
  // instruction footprint small
#pragma unroll 1
  for (int it = 0; it < ITEMS; ++it) {
    const int i = first + it * 32 + lane;
    Stencil st = Stencil{};
    if (valid[it]) stencil(g, a.P.x(0)[i], a.P.x(1)[i], a.P.x(2)[i], st);
    // runs of lanes sharing a base cell (contiguous in cell order); without
    // that order this item of the warp reduces straight into the grid
    int key = -1 - lane;
    if (use_tile && valid[it])
      key = ((st.base[2] - lo[2]) * ey + (st.base[1] - lo[1])) * ex + (st.base[0] - lo[0]);
    unsigned peers = 1u << lane;
    bool tile_item = false;
    if (use_tile) {
      peers = __match_any_sync(0xffffffffu, key);
      const int h0 = __ffs(peers) - 1, h1 = 31 - __clz(peers);
      tile_item = __all_sync(0xffffffffu, peers == ((0xffffffffu >> (31 - h1)) & (0xffffffffu << h0)));
    }
    if (tile_item) {
      const Stencil& s = st;
      float mass = 0.f, mvx = 0.f, mvy = 0.f, mvz = 0.f;
      float A[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) A[c] = 0.f;
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
        if (a.fext) {  // cloth: + h f, the force planes left zero for the next substep
          mvx = fmaf(h, a.fext[i], mvx);
          mvy = fmaf(h, a.fext[a.fext_stride + i], mvy);
          mvz = fmaf(h, a.fext[2 * a.fext_stride + i], mvz);
          a.fext[i] = a.fext[a.fext_stride + i] = a.fext[2 * a.fext_stride + i] = 0.f;
        }
      }
      const int head = __ffs(peers) - 1, seg_end = 31 - __clz(peers);
      const int maxlen = __reduce_max_sync(0xffffffffu, (unsigned)(seg_end - head + 1));
      const int steps = maxlen > 1 ? 32 - __clz(maxlen - 1) : 0;
      // the run's first lane updates the tile
      const bool issue = valid[it] && lane == head;
      const int kz = key / (ex * ey);  // tile-local base cell (valid lanes)
      const int base_row = key - kz * ex * ey;
      // (invalid lanes carry zero mass, momentum and weights)
      const float dx0[3] = {(0.f - s.fx[0]) * g.dx, (1.f - s.fx[0]) * g.dx, (2.f - s.fx[0]) * g.dx};
#pragma unroll
      for (int cz = 0; cz < 3; ++cz) {
        const float dz = (cz - s.fx[2]) * g.dx;
#pragma unroll
        for (int cy = 0; cy < 3; ++cy) {
          const float dy = (cy - s.fx[1]) * g.dx;
          const float wyz = s.w[1][cy] * s.w[2][cz];
          const int row = (kz + cz) * ex * ey + base_row + cy * ex;
          // momentum of the row's nodes up to the x term: m v + A (., dy, dz)
          const float rx = fmaf(A[2], dz, fmaf(A[1], dy, mvx));
          const float ry = fmaf(A[5], dz, fmaf(A[4], dy, mvy));
          const float rz = fmaf(A[8], dz, fmaf(A[7], dy, mvz));
#pragma unroll
          for (int cx = 0; cx < 3; ++cx) {
            const float w = s.w[0][cx] * wyz;
            float q0 = w * mass;
            float q1 = w * fmaf(A[0], dx0[cx], rx);
            float q2 = w * fmaf(A[3], dx0[cx], ry);
            float q3 = w * fmaf(A[6], dx0[cx], rz);
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
              float4* t = tile + row + cx;
              const float4 o = *t;
              *t = make_float4(o.x + q0, o.y + q1, o.z + q2, o.w + q3);
            }
            // the issuing lanes of one node offset hit distinct nodes; order
            // this offset's updates before the next offset's reads
            __syncwarp();
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
      float mvx = gr.mass * vp[0], mvy = gr.mass * vp[1], mvz = gr.mass * vp[2];
      if (a.fext) {  // cloth: + h f, the force planes left zero for the next substep
        mvx = fmaf(h, a.fext[i], mvx);
        mvy = fmaf(h, a.fext[a.fext_stride + i], mvy);
        mvz = fmaf(h, a.fext[2 * a.fext_stride + i], mvz);
        a.fext[i] = a.fext[a.fext_stride + i] = a.fext[2 * a.fext_stride + i] = 0.f;
      }
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
      // mark the (up to 8) blocks of this stencil (a sparse grid marked them
      // before P2G)
      if (!g.slot) {
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
  if (!use_tile) return;
  __syncwarp();
  // flush: one vector reduction per touched node of the warp tile
  // t / ex and r / ey by float reciprocals: exact, since t < 2^22 and the
  // fractional parts stay at least 0.5 / ex away from an integer
  const float inv_ex = 1.0f / ex, inv_ey = 1.0f / ey;
  for (int t = lane; t < tile_n; t += 32) {
    const float4 q = tile[t];
    if (q.x != 0.0f || q.y != 0.0f || q.z != 0.0f || q.w != 0.0f) {
      const int r = __float2int_rz(((float)t + 0.5f) * inv_ex), lx = t - r * ex;
      const int lz = __float2int_rz(((float)r + 0.5f) * inv_ey), ly = r - lz * ey;
      const int node = node_index(g, lo[0] + lx, lo[1] + ly, lo[2] + lz);
      red_add_v4(a.G.mp + node, q.x, q.y, q.z, q.w);
    }
  }
  // mark the 4^3 blocks the tile overlaps (a sparse grid marked its blocks
  // before P2G)
  if (g.slot) return;
  const int bx0 = lo[0] >> 2, by0 = lo[1] >> 2, bz0 = lo[2] >> 2;
  const int bnx = ((lo[0] + ex - 1) >> 2) - bx0 + 1, bny = ((lo[1] + ey - 1) >> 2) - by0 + 1,
            bnz = ((lo[2] + ez - 1) >> 2) - bz0 + 1;
  for (int t = lane; t < bnx * bny * bnz; t += 32) {
    const int qx = t % bnx, r = t / bnx, qy = r % bny, qz = r / bny;
    a.G.mark[((bz0 + qz) * g.nby + (by0 + qy)) * g.nbx + (bx0 + qx)] = 1;
  }
}

// ---- node-parallel gather form ----
// The warp stages its 32 particles' transfer data in shared memory and walks
// them in cell order. Lane j < 27 owns node j of the current cell's 27-node
// stencil and adds w_jp m_p (1, b_p - A_p c_j) for every particle of the
// cell's run, with the per-unit-mass b = v (+ h f_ext / m) + A f and
// A = -dx (C - h 4/dx^2 (V/m) tau), f the particle's position in its base cell
// and c_j the node's offset from the base (so that m (b - A c) is the APIC
// momentum m v + (m C - h 4/dx^2 V tau)(x_j - x_p)). The particle's data come
// by broadcast loads; its weights are stored as the nine products m wx wy and
// the three wz, so that a lane reads two and multiplies once. No shuffle
// reduction, and the lanes of one update hold distinct nodes.
// A run's sums go into the warp's window: the 6^3 nodes that the stencils of
// one 4^3 block's cells reach; the window is flushed to the grid (one vector
// reduction per touched node) when the walk enters another block.
constexpr int kWin = 216;     // 6^3 nodes of a block's stencils
constexpr int kRecRows = 6;   // float4 rows of a particle record
constexpr size_t kGatherSmem = sizeof(float4) * kWarps * (kWin + kRecRows * 32);

// the window of block (bx, by, bz) to the grid; the window is zero afterwards.
// lo*, hi*: the least and greatest cell (0..3) of the block whose run reached
// the window along each axis, so that only slots lo .. hi + 2 can be nonzero.
__device__ __forceinline__ void flush_window(const P2GArgs& a, const GridDev& g, float4* win,
                                             int lane, int bx, int by, int bz, int lo0, int lo1,
                                             int lo2, int hi0, int hi1, int hi2) {
  const int e0 = hi0 - lo0 + 3, e1 = hi1 - lo1 + 3, e2 = hi2 - lo2 + 3;
  // t / e0 and r / e1 by float reciprocals: exact, since t < 216 and the
  // fractional parts stay at least 0.5 / e away from an integer
  const float inv0 = 1.0f / e0, inv1 = 1.0f / e1;
  for (int t = lane; t < e0 * e1 * e2; t += 32) {
    const int r = __float2int_rz(((float)t + 0.5f) * inv0), x = t - r * e0;
    const int z = __float2int_rz(((float)r + 0.5f) * inv1), y = r - z * e1;
    const int lx = lo0 + x, ly = lo1 + y, lz = lo2 + z;
    float4* slot = win + (lz * 6 + ly) * 6 + lx;
    const float4 q = *slot;
    if (q.x != 0.0f || q.y != 0.0f || q.z != 0.0f || q.w != 0.0f) {
      red_add_v4(a.G.mp + node_index(g, 4 * bx + lx, 4 * by + ly, 4 * bz + lz), q.x, q.y, q.z, q.w);
      *slot = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  // the (up to 8) blocks the window's stencils reach (a sparse grid marked
  // them before P2G)
  if (!g.slot && lane < 8) {
    const int ox = lane & 1, oy = (lane >> 1) & 1, oz = lane >> 2;
    if ((!ox || hi0 >= 2) && (!oy || hi1 >= 2) && (!oz || hi2 >= 2))
      a.G.mark[((bz + oz) * g.nby + (by + oy)) * g.nbx + (bx + ox)] = 1;
  }
  __syncwarp();
}

template <int ITEMS>
__device__ __forceinline__ void p2g_gather_block(const P2GArgs& a, int block) {
  extern __shared__ float4 s_dyn[];
  __shared__ DevBody s_body[kMaxBodies];
  const GridDev& g = a.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int first = (block * kWarps + warp) * 32 * ITEMS;
  float4* win = s_dyn + warp * kWin;
  float4* rec = s_dyn + kWarps * kWin + warp * (kRecRows * 32);  // [kRecRows][32]
  const float* recf = reinterpret_cast<const float*>(rec);

  for (int i = tid; i < a.nb * (int)(sizeof(DevBody) / 4); i += kThreads)
    reinterpret_cast<float*>(s_body)[i] = reinterpret_cast<const float*>(a.bodies)[i];
  for (int t = lane; t < kWin; t += 32) win[t] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  if (first >= a.n) return;
  const float h = a.h;
  const float dinv = 4.0f * g.inv_dx * g.inv_dx;

  // this lane's node of a stencil: offsets c, the window offset of a block's
  // cell (0,0,0), and the float offsets of its three weights in a record
  const bool node_lane = lane < 27;
  const int oc0 = lane % 3, oc1 = (lane / 3) % 3, oc2 = min(lane / 9, 2);
  const float nc0 = -(float)oc0, nc1 = -(float)oc1, nc2 = -(float)oc2;
  const float2 nc00 = make_float2(nc0, nc0), nc11 = make_float2(nc1, nc1), nc22 = make_float2(nc2, nc2);
  const int woff_node = (oc2 * 6 + oc1) * 6 + oc0;
  // m wx wy of product e = oc0 + 3 oc1 at row 3 + e / 4, component e % 4;
  // wz of oc2 at row 5, component 1 + oc2
  const int exy = oc0 + 3 * oc1;
  const int wfxy = ((3 + exy / 4) * 32) * 4 + (exy & 3);
  const int wfz = (5 * 32) * 4 + 1 + oc2;

  int wb = -1, wbx = 0, wby = 0, wbz = 0;  // the window's block
  int wl0 = 3, wl1 = 3, wl2 = 3, wh0 = 0, wh1 = 0, wh2 = 0;  // its runs' cells
#pragma unroll 1
  for (int it = 0; it < ITEMS; ++it) {
    const int i = first + it * 32 + lane;
    int key = -1, bkey = -1, base[3] = {0, 0, 0};
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0, r3 = r0, r4 = r0, r5 = r0;
    float xp[3] = {0.f, 0.f, 0.f};
    bool valid = false;
    if (i < a.n) {
      Stencil st;
#pragma unroll
      for (int c = 0; c < 3; ++c) xp[c] = a.P.x(c)[i];
      stencil(g, xp[0], xp[1], xp[2], st);
      if (!stencil_inside(g, st)) {
        atomicOr(a.status, kStOutOfDomain);
      } else {
        valid = true;
#pragma unroll
        for (int c = 0; c < 3; ++c) base[c] = st.base[c];
        key = (base[2] * g.nby * 4 + base[1]) * (g.nbx * 4) + base[0];
        bkey = ((base[2] >> 2) * g.nby + (base[1] >> 2)) * g.nbx + (base[0] >> 2);
        const DevGroup gr = a.groups[a.P.grp[i]];
        float tau[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) tau[c] = a.P.tau(c)[i];
        // per unit mass: A = A' / m = -dx (C - h (4/dx^2) (V/m) tau) and
        // b = b' / m = v (+ h f_ext / m) + A f, with A' and b' of the sum
        // w (b' - A' c) = w m (b - A c)
        const float sc = h * dinv * gr.vol_m;
        const float tf[9] = {tau[0], tau[3], tau[4], tau[3], tau[1], tau[5], tau[4], tau[5], tau[2]};
        float A[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) A[c] = -g.dx * (a.P.C(c)[i] - sc * tf[c]);
        float vv[3] = {a.P.v(0)[i], a.P.v(1)[i], a.P.v(2)[i]};
        if (a.fext) {  // cloth: + h f / m, the force planes left zero for the next substep
          const float hm = h * gr.inv_m;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            vv[c] = fmaf(hm, a.fext[c * a.fext_stride + i], vv[c]);
            a.fext[c * a.fext_stride + i] = 0.f;
          }
        }
        float b[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
          b[c] = fmaf(A[3 * c], st.fx[0], fmaf(A[3 * c + 1], st.fx[1], fmaf(A[3 * c + 2], st.fx[2], vv[c])));
        r0 = make_float4(b[0], b[1], b[2], A[8]);
        // rows x and y of A interleaved, so that both rows step in one
        // paired FMA: (Axx, Ayx, Axy, Ayy), (Axz, Ayz, Azx, Azy)
        r1 = make_float4(A[0], A[3], A[1], A[4]);
        r2 = make_float4(A[2], A[5], A[6], A[7]);
        // weights: the nine products m wx wy (x fastest) and the three wz, so
        // that a lane forms w m of its node with one multiply
        {
          float wxm[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) wxm[c] = gr.mass * st.w[0][c];
          r3 = make_float4(wxm[0] * st.w[1][0], wxm[1] * st.w[1][0], wxm[2] * st.w[1][0], wxm[0] * st.w[1][1]);
          r4 = make_float4(wxm[1] * st.w[1][1], wxm[2] * st.w[1][1], wxm[0] * st.w[1][2], wxm[1] * st.w[1][2]);
          r5 = make_float4(wxm[2] * st.w[1][2], st.w[2][0], st.w[2][1], st.w[2][2]);
        }
      }
    }
    rec[lane] = r0;
    rec[32 + lane] = r1;
    rec[64 + lane] = r2;
    rec[96 + lane] = r3;
    rec[128 + lane] = r4;
    rec[160 + lane] = r5;
    __syncwarp();
    // runs of equal base cell (contiguous in cell order; any order is
    // correct, with more runs); invalid lanes carry key -1
    for (int p = 0; p < 32;) {
      const int kp = __shfl_sync(0xffffffffu, key, p);
      const unsigned eq = __ballot_sync(0xffffffffu, key == kp) >> p;
      const int len = ~eq == 0u ? 32 - p : __ffs(~eq) - 1;
      if (kp >= 0) {
        const int b0 = __shfl_sync(0xffffffffu, base[0], p), b1 = __shfl_sync(0xffffffffu, base[1], p),
                  b2 = __shfl_sync(0xffffffffu, base[2], p);
        const int kb = __shfl_sync(0xffffffffu, bkey, p);
        if (kb != wb) {
          if (wb >= 0) flush_window(a, g, win, lane, wbx, wby, wbz, wl0, wl1, wl2, wh0, wh1, wh2);
          wb = kb;
          wbx = b0 >> 2;
          wby = b1 >> 2;
          wbz = b2 >> 2;
          wl0 = wl1 = wl2 = 3;
          wh0 = wh1 = wh2 = 0;
        }
        const int l0 = b0 & 3, l1 = b1 & 3, l2 = b2 & 3;
        wl0 = min(wl0, l0); wl1 = min(wl1, l1); wl2 = min(wl2, l2);
        wh0 = max(wh0, l0); wh1 = max(wh1, l1); wh2 = max(wh2, l2);
        float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
        const int pe = p + len;
        // (acc1, acc2) and the momentum's x, y rows go in pairs (FFMA2)
        float2 acc12 = make_float2(0.f, 0.f);
#pragma unroll 2
        for (int q = p; q < pe; ++q) {
          const float4 q0 = rec[q], q1 = rec[32 + q], q2 = rec[64 + q];
          const float wm = recf[wfxy + 4 * q] * recf[wfz + 4 * q];  // w m
          // b - A c (velocity units); the node receives w m and w m (b - A c)
          const float2 m01 =
              __ffma2_rn(make_float2(q1.x, q1.y), nc00,
                         __ffma2_rn(make_float2(q1.z, q1.w), nc11,
                                    __ffma2_rn(make_float2(q2.x, q2.y), nc22, make_float2(q0.x, q0.y))));
          const float m2 = fmaf(q2.z, nc0, fmaf(q2.w, nc1, fmaf(q0.w, nc2, q0.z)));
          acc0 += wm;
          acc12 = __ffma2_rn(make_float2(wm, wm), m01, acc12);
          acc3 = fmaf(wm, m2, acc3);
        }
        acc1 = acc12.x;
        acc2 = acc12.y;
        if (node_lane) {
          float4* t = win + (l2 * 6 + l1) * 6 + l0 + woff_node;
          const float4 o = *t;
          *t = make_float4(o.x + acc0, o.y + acc1, o.z + acc2, o.w + acc3);
        }
        __syncwarp();
      }
      p += len;
    }
    // contact registration: bodies that may hold a particle of this item
    // (the signed distance is 1-Lipschitz: a body whose distance at the
    // centre of the item's box exceeds its half diagonal holds none), then a
    // warp-aggregated append, one contact per (particle, body) pair with the
    // particle strictly inside
    int lo[3], hi[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      lo[c] = __reduce_min_sync(0xffffffffu, valid ? base[c] : 0x7fffffff);
      hi[c] = __reduce_max_sync(0xffffffffu, valid ? base[c] : -0x7fffffff);
    }
    bool cand_b = false;
    if (hi[0] >= lo[0] && lane < a.nb) {
      const float c0 = g.ox + g.dx * (0.5f * (lo[0] + hi[0]) + 1.0f);
      const float c1 = g.oy + g.dx * (0.5f * (lo[1] + hi[1]) + 1.0f);
      const float c2 = g.oz + g.dx * (0.5f * (lo[2] + hi[2]) + 1.0f);
      const float h0 = 0.5f * g.dx * (hi[0] - lo[0] + 1), h1 = 0.5f * g.dx * (hi[1] - lo[1] + 1),
                  h2 = 0.5f * g.dx * (hi[2] - lo[2] + 1);
      cand_b = box_may_touch(s_body[lane], c0, c1, c2, h0, h1, h2);
    }
    const unsigned cand = __ballot_sync(0xffffffffu, cand_b);
    if (cand) {
      float vp[3] = {0.f, 0.f, 0.f};
      if (valid) {
#pragma unroll
        for (int c = 0; c < 3; ++c) vp[c] = a.P.v(c)[i];
      }
      for (int b = 0; b < a.nb; ++b) {
        if (!((cand >> b) & 1u)) continue;
        float nrm[3] = {0.f, 0.f, 1.f};
        float phi = 1.0f;
        if (valid) {
          phi = body_sdf(s_body[b], xp[0], xp[1], xp[2], nrm);
          // near the surface the sign and the depth come from FP64
          if (phi < 1e-6f + 1e-6f * (fabsf(xp[0]) + fabsf(xp[1]) + fabsf(xp[2])))
            phi = (float)body_sdf_f64(s_body[b], xp[0], xp[1], xp[2]);
        }
        const bool hit = valid && phi < 0.0f;
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
  if (wb >= 0) flush_window(a, g, win, lane, wbx, wby, wbz, wl0, wl1, wl2, wh0, wh1, wh2);
}

template <int ITEMS>
__global__ void __launch_bounds__(kThreads, 4) k_p2g_g(P2GArgs a) {
  p2g_gather_block<ITEMS>(a, blockIdx.x);
}

template <int ITEMS>
__global__ void __launch_bounds__(kThreads, 4) k_p2g_g_batch(const P2GArgs* __restrict__ args,
                                                             const int2* __restrict__ work) {
  __shared__ P2GArgs s_a;
  const int2 wk = work[blockIdx.x];
  load_args(args + wk.x, s_a);
  __syncthreads();
  p2g_gather_block<ITEMS>(s_a, wk.y);
}

template <int ITEMS>
__global__ void __launch_bounds__(kThreads, 4) k_p2g(P2GArgs a) {
  p2g_block<ITEMS>(a, blockIdx.x);
}

template <int ITEMS>
void launch_items(const P2GArgs& a, int form, cudaStream_t s) {
  const int per_block = kThreads * ITEMS;
  const int nblk = (a.n + per_block - 1) / per_block;
  if (form == MPM_P2G_SCATTER)
    k_p2g<ITEMS><<<nblk, kThreads, kDynSmem, s>>>(a);
  else
    k_p2g_g<ITEMS><<<nblk, kThreads, kGatherSmem, s>>>(a);
}

template <int ITEMS>
cudaError_t prepare_items() {
  // dynamic shared memory beyond 48 KB, and room for four blocks per SM
  cudaError_t e = cudaFuncSetAttribute(k_p2g<ITEMS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kDynSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_p2g_g<ITEMS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kGatherSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_p2g_g_batch<ITEMS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kGatherSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_p2g<ITEMS>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_p2g_g<ITEMS>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_p2g_g_batch<ITEMS>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

}  // namespace

cudaError_t p2g_prepare() {
  cudaError_t e = prepare_items<1>();
  if (e == cudaSuccess) e = prepare_items<2>();
  if (e == cudaSuccess) e = prepare_items<4>();
  return e;
}

namespace {
int items_of(int chunk) {
  const int items = chunk / kThreads;
  return items <= 1 ? 1 : items == 2 ? 2 : 4;
}
}  // namespace

int p2g_block_particles(int chunk) { return items_of(chunk) * kThreads; }

void launch_p2g_batch(const P2GArgs* args, const int2* work, int n_work, int chunk, cudaStream_t s) {
  if (n_work <= 0) return;
  switch (items_of(chunk)) {
    case 1: k_p2g_g_batch<1><<<n_work, kThreads, kGatherSmem, s>>>(args, work); break;
    case 2: k_p2g_g_batch<2><<<n_work, kThreads, kGatherSmem, s>>>(args, work); break;
    default: k_p2g_g_batch<4><<<n_work, kThreads, kGatherSmem, s>>>(args, work); break;
  }
}

void launch_p2g(const P2GArgs& a, int chunk, int form, cudaStream_t s) {
  if (a.n <= 0) return;
  const int items = chunk / kThreads;
  if (items <= 1)
    launch_items<1>(a, form, s);
  else if (items == 2)
    launch_items<2>(a, form, s);
  else
    launch_items<4>(a, form, s);
}

}  // namespace mpmcr
