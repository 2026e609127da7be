// grid.cu -- active-block compaction and the grid update of the free-motion
// solve (Sec. V-A op (2): v* = p / m + h g on every node with mass), with the
// domain walls held at zero velocity.
//
// Only 4^3 blocks marked by P2G are swept. The update also clears the P2G
// accumulator it consumed, so the accumulator is all zero between substeps
// and no separate clearing pass is needed.
//
// A block-sparse grid (GridDev::slot) stores only the substep's active
// blocks: before P2G the blocks of the particles' stencils are marked and
// compacted, and entry t of the active list gets storage block t (the slot
// table maps the grid block to it; the previous substep's entries are unmapped
// first, so unmapped blocks read -1). Blocks beyond the pool share its spare
// block and the substep reports a capacity error.
#include "kernels.h"

namespace mpmcr {

namespace {

// Compaction of one scene's block marks into its active-block list, the
// threads striding by `stride` from `start` (taken warp-aligned).
__device__ __forceinline__ void compact_range(uint8_t* __restrict__ mark, int start, int stride,
                                              int n_blocks, int* __restrict__ act,
                                              int* __restrict__ n_act,
                                              int* __restrict__ slot_tab = nullptr, int pool = 0,
                                              uint32_t* __restrict__ status = nullptr) {
  const int lane = threadIdx.x & 31;
  for (int base = start & ~31; base < n_blocks; base += stride) {
    const int b = base + lane;
    const bool on = b < n_blocks && mark[b] != 0;
    const unsigned m = __ballot_sync(0xffffffffu, on);
    if (m == 0u) continue;
    int slot0 = 0;
    if (lane == 0) slot0 = atomicAdd(n_act, __popc(m));
    slot0 = __shfl_sync(0xffffffffu, slot0, 0);
    if (on) {
      const int t = slot0 + __popc(m & ((1u << lane) - 1u));
      act[t] = b;
      mark[b] = 0;
      if (slot_tab) {
        slot_tab[b] = t < pool ? t : pool;  // beyond the pool: the spare block
        if (t >= pool) atomicOr(status, kStCapacity);
      }
    }
  }
}

// Sparse grids, before P2G: unmap the previous substep's blocks, then mark
// the blocks of every particle's stencil (the nodes P2G, the solve and G2P
// of this substep touch).
__global__ void k_mark_sparse(GridDev g, Particles P, int n, uint8_t* __restrict__ mark,
                              const int* __restrict__ act, const int* __restrict__ n_mapped,
                              int* __restrict__ slot_tab) {
  const int stride = gridDim.x * blockDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nm = *n_mapped;
  for (int t = tid; t < nm; t += stride) slot_tab[act[t]] = -1;
  for (int i = tid; i < n; i += stride) {
    Stencil st;
    stencil(g, P.x(0)[i], P.x(1)[i], P.x(2)[i], st);
    if (!stencil_inside(g, st)) continue;  // reported by P2G
    const int bx0 = st.base[0] >> 2, by0 = st.base[1] >> 2, bz0 = st.base[2] >> 2;
    const int bx1 = (st.base[0] + 2) >> 2, by1 = (st.base[1] + 2) >> 2, bz1 = (st.base[2] + 2) >> 2;
    for (int bz = bz0; bz <= bz1; ++bz)
      for (int by = by0; by <= by1; ++by)
        for (int bx = bx0; bx <= bx1; ++bx) mark[(bz * g.nby + by) * g.nbx + bx] = 1;
  }
}

__global__ void k_compact_sparse(uint8_t* __restrict__ mark, int n_blocks, int* __restrict__ act,
                                 int* __restrict__ n_act, int* __restrict__ slot_tab, int pool,
                                 uint32_t* __restrict__ status) {
  compact_range(mark, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, n_blocks,
                act, n_act, slot_tab, pool, status);
}

__global__ void k_compact(uint8_t* __restrict__ mark, int n_blocks, int* __restrict__ act,
                          int* __restrict__ n_act) {
  compact_range(mark, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, n_blocks,
                act, n_act);
}

// The grid update of nodes t = start, start + stride, ... of the active
// blocks' nodes; `first`: the thread that records the active-block count.
__device__ __forceinline__ void grid_update_range(const GridDev& g, const GridArrays& G, float h,
                                                  DevStats* stats, long long start,
                                                  long long stride, bool first) {
  const int n_act = *G.n_act;
  if (first) {
    atomicMax(&stats->active_blocks_max, n_act);
    stats->last_active = n_act;
    if (g.slot) *G.n_mapped = n_act;  // the list the slot table now holds
  }
  const long long total = (long long)active_with_storage(g, n_act) * kBlockNodes;
  float p2 = 0.f;  // sum of m |v*|^2 over free nodes (the momentum norm of Alg. 1)
  for (long long t = start; t < total; t += stride) {
    const int blk = G.act[t >> 6];
    const int cell = (int)(t & 63);
    const int node = active_storage_block(g, G.act, (int)(t >> 6)) * kBlockNodes + cell;
    const float4 mp = G.mp[node];
    float4 vs = make_float4(0.f, 0.f, 0.f, 0.f);
    const int bx = blk % g.nbx, by = (blk / g.nbx) % g.nby, bz = blk / (g.nbx * g.nby);
    const int i = bx * 4 + (cell & 3), j = by * 4 + ((cell >> 2) & 3), k = bz * 4 + (cell >> 4);
    const bool wall = i < g.bc || j < g.bc || k < g.bc || i >= g.rx - g.bc ||
                      j >= g.ry - g.bc || k >= g.rz - g.bc;
    if (mp.x > 0.0f) {
      const float inv_m = 1.0f / mp.x;
      vs.x = wall ? 0.0f : mp.y * inv_m + h * g.gx;
      vs.y = wall ? 0.0f : mp.z * inv_m + h * g.gy;
      vs.z = wall ? 0.0f : mp.w * inv_m + h * g.gz;
      vs.w = mp.x;
      if (!wall) p2 += mp.x * (vs.x * vs.x + vs.y * vs.y + vs.z * vs.z);
    }
    G.mp[node] = make_float4(0.f, 0.f, 0.f, 0.f);
    G.vs[node] = vs;
    // .w flags a Dirichlet node for the contact solve
    G.v[node] = make_float4(vs.x, vs.y, vs.z, wall ? 1.f : 0.f);
    G.vlo[node] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __shared__ double s_p2[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) p2 += __shfl_xor_sync(0xffffffffu, p2, o);
  if ((threadIdx.x & 31) == 0) s_p2[threadIdx.x >> 5] = (double)p2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += s_p2[w];
    if (sum != 0.0) atomicAdd(G.pstar2, sum);
  }
}

__global__ void __launch_bounds__(256) k_grid_update(GridDev g, GridArrays G, float h,
                                                     DevStats* stats) {
  grid_update_range(g, G, h, stats, (long long)blockIdx.x * blockDim.x + threadIdx.x,
                    (long long)gridDim.x * blockDim.x, blockIdx.x == 0 && threadIdx.x == 0);
}

// Batched: thread block b is slice work[b].y of work[b].x's scene; a scene's
// n_slices blocks stride together over its marks (compaction) or its active
// nodes (update)
__global__ void __launch_bounds__(256) k_compact_batch(const GridBatchArgs* __restrict__ args,
                                                       const int2* __restrict__ work) {
  const int2 wk = work[blockIdx.x];
  const GridBatchArgs& a = args[wk.x];
  compact_range(a.G.mark, wk.y * blockDim.x + threadIdx.x, a.n_slices * blockDim.x,
                a.g.nbx * a.g.nby * a.g.nbz, a.G.act, a.G.n_act);
}

__global__ void __launch_bounds__(256) k_grid_update_batch(const GridBatchArgs* __restrict__ args,
                                                           const int2* __restrict__ work) {
  __shared__ GridBatchArgs s_a;
  const int2 wk = work[blockIdx.x];
  load_args(args + wk.x, s_a);
  __syncthreads();
  grid_update_range(s_a.g, s_a.G, s_a.h, s_a.stats, (long long)wk.y * blockDim.x + threadIdx.x,
                    (long long)s_a.n_slices * blockDim.x, wk.y == 0 && threadIdx.x == 0);
}

}  // namespace

void launch_grid(const GridDev& g, const GridArrays& G, float h, int num_sms, DevStats* stats,
                 cudaStream_t s) {
  int n_blocks = g.nbx * g.nby * g.nbz;
  int cb = (n_blocks + 255) / 256;
  cb = cb > num_sms * 8 ? num_sms * 8 : cb;
  // (a sparse grid compacted its marks before P2G)
  if (!g.slot) k_compact<<<cb, 256, 0, s>>>(G.mark, n_blocks, G.act, G.n_act);
  k_grid_update<<<num_sms * 8, 256, 0, s>>>(g, G, h, stats);
}

void launch_sparse_map(const GridDev& g, const GridArrays& G, const Particles& P, int n,
                       int* slot_tab, uint32_t* status, int num_sms, cudaStream_t s) {
  const int n_blocks = g.nbx * g.nby * g.nbz;
  const int pb = (n + 255) / 256;
  k_mark_sparse<<<pb < num_sms * 8 ? (pb > 0 ? pb : 1) : num_sms * 8, 256, 0, s>>>(
      g, P, n, G.mark, G.act, G.n_mapped, slot_tab);
  int cb = (n_blocks + 255) / 256;
  cb = cb > num_sms * 8 ? num_sms * 8 : cb;
  k_compact_sparse<<<cb, 256, 0, s>>>(G.mark, n_blocks, G.act, G.n_act, slot_tab, g.pool_blocks,
                                      status);
}

void launch_grid_batch(const GridBatchArgs* args, const int2* work, int n_work, cudaStream_t s) {
  if (n_work <= 0) return;
  k_compact_batch<<<n_work, 256, 0, s>>>(args, work);
  k_grid_update_batch<<<n_work, 256, 0, s>>>(args, work);
}

}  // namespace mpmcr
