// sort.cu -- particle ordering by grid block (Sec. V-A: particles sorted by
// cell so that particles writing the same grid nodes are processed together;
// the order is computed once per time step and reused by its N substeps).
//
// Key: Morton code of the 4^3 block holding the particle's B-spline base
// node, so that a run of consecutive particles covers a compact box of
// blocks, followed by the base cell within the block (x fastest), so that
// the lanes of a warp touch consecutive nodes of P2G's shared tile and lanes
// sharing a cell are adjacent (for the warp-level pre-reduction). Sort:
// stable LSD radix sort with 8-bit digits, one pass per digit of the key (a
// 128^3 grid has 15 + 6 key bits: three passes). Each pass is a
// per-warp-tile histogram, an exclusive scan over (digit, tile), and a
// stable per-warp scatter whose in-warp ranks come from __match_any_sync.
// The permutation is then applied to every particle plane at once. Up to
// 8,192 particles the keys are sorted by one thread block instead (a bitonic
// network over (key, index) pairs in shared memory: the same order, two
// launches in place of a dozen, which is what a small scene's step notices).
#include "kernels.h"

namespace mpmcr {

namespace {

constexpr int kRadix = 256;
constexpr int kWarpTile = 1024;       // keys per warp tile (32 rounds of 32)
constexpr int kSortWarps = 4;         // warps per thread block
constexpr int kScanChunk = 4096;      // elements per scan thread block
constexpr int kScanThreads = 256;

constexpr int kSmallSortMax = 8192;      // particles sorted by one thread block
constexpr int kSmallSortThreads = 1024;

// the sort key of a particle at (x, y, z)
__device__ __forceinline__ uint32_t sort_key(const GridDev& g, float x, float y, float z) {
  // the base node of the particle's stencil, as P2G computes it
  Stencil st;
  stencil(g, x, y, z, st);
  int lim[3] = {g.nbx - 1, g.nby - 1, g.nbz - 1};
  uint32_t b[3], c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int base = st.base[a];
    int blk = base >> 2;  // arithmetic shift: floor division for negatives
    c[a] = (uint32_t)(base & 3);
    if (blk < 0) { blk = 0; c[a] = 0; }
    if (blk > lim[a]) { blk = lim[a]; c[a] = 3; }
    b[a] = (uint32_t)blk;
  }
  uint32_t key = spread_bits3(b[0]) | (spread_bits3(b[1]) << 1) | (spread_bits3(b[2]) << 2);
  // cell within the block, x fastest (the order of the P2G tile), when it fits
  if (g.sort_cell_bits) key = (key << 6) | (c[2] << 4) | (c[1] << 2) | c[0];
  return key;
}

__global__ void k_keys(GridDev g, const float* __restrict__ x0, const float* __restrict__ x1,
                       const float* __restrict__ x2, int n, uint32_t* __restrict__ keys,
                       uint32_t* __restrict__ vals) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = sort_key(g, x0[i], x1[i], x2[i]);
  vals[i] = (uint32_t)i;
}

// Up to kSmallSortMax particles in one thread block: the (key, index) pairs,
// each distinct thanks to the index, sorted by a bitonic network in shared
// memory, so that the order is the stable radix sort's; the permutation goes
// to vals. A small scene's sort is then one launch instead of a dozen.
__global__ void __launch_bounds__(kSmallSortThreads) k_sort_small(
    GridDev g, const float* __restrict__ x0, const float* __restrict__ x1,
    const float* __restrict__ x2, int n, uint32_t* __restrict__ vals) {
  extern __shared__ unsigned long long s_kv[];
  int m = 1;
  while (m < n) m <<= 1;
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    s_kv[i] = i < n ? ((unsigned long long)sort_key(g, x0[i], x1[i], x2[i]) << 32) | (unsigned)i
                    : ~0ull;
  __syncthreads();
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < (m >> 1); t += blockDim.x) {
        const int i = 2 * t - (t & (j - 1));  // t-th index with bit j clear; its partner i + j
        const unsigned long long a = s_kv[i], b = s_kv[i + j];
        if ((a > b) == ((i & k) == 0)) {
          s_kv[i] = b;
          s_kv[i + j] = a;
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) vals[i] = (uint32_t)s_kv[i];
}

__global__ void k_hist(const uint32_t* __restrict__ keys, int n, int shift, int n_tiles,
                       uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[kSortWarps][kRadix];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int d = lane; d < kRadix; d += 32) h[w][d] = 0;
  __syncwarp();
  int tile = blockIdx.x * kSortWarps + w;
  if (tile >= n_tiles) return;
  int start = tile * kWarpTile;
  for (int r = 0; r < kWarpTile / 32; ++r) {
    int i = start + r * 32 + lane;
    if (i < n) atomicAdd(&h[w][(keys[i] >> shift) & (kRadix - 1)], 1u);
  }
  __syncwarp();
  for (int d = lane; d < kRadix; d += 32) hist[(size_t)d * n_tiles + tile] = h[w][d];
}

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* smem_warp,
                                                          uint32_t& total) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t s = lane < nw ? smem_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) smem_warp[lane] = s;
  }
  __syncthreads();
  uint32_t warp_off = w > 0 ? smem_warp[w - 1] : 0;
  total = smem_warp[nw - 1];
  __syncthreads();
  return warp_off + x - v;
}

// per-chunk totals
__global__ void k_scan_reduce(const uint32_t* __restrict__ data, int len,
                              uint32_t* __restrict__ partial) {
  __shared__ uint32_t sw[32];
  int base = blockIdx.x * kScanChunk;
  uint32_t s = 0;
  for (int i = threadIdx.x; i < kScanChunk; i += blockDim.x)
    if (base + i < len) s += data[base + i];
  uint32_t total;
  block_exclusive_scan(s, sw, total);
  if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// exclusive scan of the chunk totals by one thread block, in order
__global__ void k_scan_partials(uint32_t* partial, int n_part) {
  __shared__ uint32_t sw[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n_part; base += blockDim.x) {
    int i = base + threadIdx.x;
    uint32_t v = i < n_part ? partial[i] : 0;
    uint32_t total;
    uint32_t ex = block_exclusive_scan(v, sw, total);
    if (i < n_part) partial[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
}

// in-place exclusive scan of one chunk given its carry-in
__global__ void k_scan_apply(uint32_t* __restrict__ data, int len,
                             const uint32_t* __restrict__ partial) {
  __shared__ uint32_t sw[32];
  constexpr int kPer = kScanChunk / kScanThreads;
  int base = blockIdx.x * kScanChunk + threadIdx.x * kPer;
  uint32_t v[kPer];
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    v[j] = base + j < len ? data[base + j] : 0;
    s += v[j];
  }
  uint32_t total;
  uint32_t ex = block_exclusive_scan(s, sw, total) + partial[blockIdx.x];
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    if (base + j < len) data[base + j] = ex;
    ex += v[j];
  }
}

__global__ void k_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                          uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int n,
                          int shift, int n_tiles, const uint32_t* __restrict__ offs) {
  __shared__ uint32_t base[kSortWarps][kRadix];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int tile = blockIdx.x * kSortWarps + w;
  if (tile >= n_tiles) return;
  for (int d = lane; d < kRadix; d += 32) base[w][d] = offs[(size_t)d * n_tiles + tile];
  __syncwarp();
  unsigned lt = (1u << lane) - 1u;
  int start = tile * kWarpTile;
  for (int r = 0; r < kWarpTile / 32; ++r) {
    int i = start + r * 32 + lane;
    bool valid = i < n;
    uint32_t key = valid ? kin[i] : 0u;
    uint32_t d = (key >> shift) & (kRadix - 1);
    unsigned peers = __match_any_sync(0xffffffffu, valid ? d : (kRadix + 0u));
    unsigned rank = __popc(peers & lt);
    uint32_t pos = 0;
    if (valid) {
      pos = base[w][d] + rank;
      kout[pos] = key;
      vout[pos] = vin[i];
    }
    __syncwarp();
    if (valid && rank == 0) base[w][d] += __popc(peers);
    __syncwarp();
  }
}

__global__ void k_permute(Particles src, Particles dst, const uint32_t* __restrict__ perm, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t j = perm[i];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    dst.x(c)[i] = src.x(c)[j];
    dst.v(c)[i] = src.v(c)[j];
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    dst.C(c)[i] = src.C(c)[j];
    dst.F(c)[i] = src.F(c)[j];
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) dst.tau(c)[i] = src.tau(c)[j];
  dst.pid[i] = src.pid[j];
  dst.grp[i] = src.grp[j];
}

__global__ void k_to_id(Particles P, int n, float* __restrict__ ox, float* __restrict__ ov,
                        float* __restrict__ oC, float* __restrict__ oF) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  size_t id = P.pid[i];
  if (ox)
    for (int c = 0; c < 3; ++c) ox[3 * id + c] = P.x(c)[i];
  if (ov)
    for (int c = 0; c < 3; ++c) ov[3 * id + c] = P.v(c)[i];
  if (oC)
    for (int c = 0; c < 9; ++c) oC[9 * id + c] = P.C(c)[i];
  if (oF)
    for (int c = 0; c < 9; ++c) oF[9 * id + c] = P.F(c)[i];
}

__global__ void k_from_id(Particles P, int n, const float* __restrict__ ix,
                          const float* __restrict__ iv, const float* __restrict__ iC,
                          const float* __restrict__ iF) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  size_t id = P.pid[i];
  if (ix)
    for (int c = 0; c < 3; ++c) P.x(c)[i] = ix[3 * id + c];
  if (iv)
    for (int c = 0; c < 3; ++c) P.v(c)[i] = iv[3 * id + c];
  if (iC)
    for (int c = 0; c < 9; ++c) P.C(c)[i] = iC[9 * id + c];
  if (iF)
    for (int c = 0; c < 9; ++c) P.F(c)[i] = iF[9 * id + c];
}

__global__ void k_stress(Particles P, int n, const DevGroup* __restrict__ groups) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float F[9], t[6];
#pragma unroll
  for (int c = 0; c < 9; ++c) F[c] = P.F(c)[i];
  kirchhoff(groups[P.grp[i]], F, t);
#pragma unroll
  for (int c = 0; c < 6; ++c) P.tau(c)[i] = t[c];
}

void exclusive_scan(uint32_t* data, int len, uint32_t* partial, cudaStream_t s) {
  int n_part = (len + kScanChunk - 1) / kScanChunk;
  k_scan_reduce<<<n_part, kScanThreads, 0, s>>>(data, len, partial);
  k_scan_partials<<<1, 1024, 0, s>>>(partial, n_part);
  k_scan_apply<<<n_part, kScanThreads, 0, s>>>(data, len, partial);
}

}  // namespace

cudaError_t sort_prepare() {
  return cudaFuncSetAttribute(k_sort_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(kSmallSortMax * sizeof(unsigned long long)));
}

int sort_hist_len(int n) {
  int n_tiles = (n + kWarpTile - 1) / kWarpTile;
  return kRadix * (n_tiles > 0 ? n_tiles : 1);
}

void launch_sort(const GridDev& g, const Particles& src, const Particles& dst, int n,
                 SortBuffers& sb, cudaStream_t s) {
  if (n <= 0) return;
  int tpb = 256;
  if (n <= kSmallSortMax) {
    int m = 1;
    while (m < n) m <<= 1;
    k_sort_small<<<1, kSmallSortThreads, m * sizeof(unsigned long long), s>>>(
        g, src.x(0), src.x(1), src.x(2), n, sb.vals[0]);
    k_permute<<<(n + tpb - 1) / tpb, tpb, 0, s>>>(src, dst, sb.vals[0], n);
    return;
  }
  k_keys<<<(n + tpb - 1) / tpb, tpb, 0, s>>>(g, src.x(0), src.x(1), src.x(2), n, sb.keys[0],
                                            sb.vals[0]);
  int key_bits = 3 * g.morton_bits + (g.sort_cell_bits ? 6 : 0);
  int passes = (key_bits + 7) / 8;
  int n_tiles = (n + kWarpTile - 1) / kWarpTile;
  int blocks = (n_tiles + kSortWarps - 1) / kSortWarps;
  int cur = 0;
  for (int p = 0; p < passes; ++p) {
    int shift = 8 * p;
    k_hist<<<blocks, 32 * kSortWarps, 0, s>>>(sb.keys[cur], n, shift, n_tiles, sb.hist);
    exclusive_scan(sb.hist, kRadix * n_tiles, sb.partial, s);
    k_scatter<<<blocks, 32 * kSortWarps, 0, s>>>(sb.keys[cur], sb.vals[cur], sb.keys[1 - cur],
                                                 sb.vals[1 - cur], n, shift, n_tiles, sb.hist);
    cur = 1 - cur;
  }
  k_permute<<<(n + tpb - 1) / tpb, tpb, 0, s>>>(src, dst, sb.vals[cur], n);
}

void launch_to_id_order(const Particles& P, int n, float* ox, float* ov, float* oC, float* oF,
                        cudaStream_t s) {
  if (n <= 0) return;
  k_to_id<<<(n + 255) / 256, 256, 0, s>>>(P, n, ox, ov, oC, oF);
}

void launch_from_id_order(const Particles& P, int n, const float* ix, const float* iv,
                          const float* iC, const float* iF, cudaStream_t s) {
  if (n <= 0) return;
  k_from_id<<<(n + 255) / 256, 256, 0, s>>>(P, n, ix, iv, iC, iF);
}

}  // namespace mpmcr

namespace mpmcr {
void launch_stress_from_F(const Particles& P, int n, const DevGroup* groups, cudaStream_t s) {
  if (n <= 0) return;
  k_stress<<<(n + 255) / 256, 256, 0, s>>>(P, n, groups);
}
}  // namespace mpmcr
